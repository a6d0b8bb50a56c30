// The hopping stencil H_{p,1-p} (Eq. 4) and the kernels built on it (the
// kernel templates; one translation unit per precision instantiates them):
//   M_HOP   out = H in                       (qcd_dslash_eo)
//   M_MULT  out = F^-1 H in                  (MULT = H~, Sec. II-B)
//   M_DHAT  out = a*y + cc*F^-1 H in + d*z   (second half of D^ = 1 - k^2 H~_eo H~_oe,
//                                             with the dot products of Alg. 2 fused)
//   M_SRC   out = F^-1 (a*y + cc*H in)       (b^_e, Eq. 6, and x_o, Eq. 7)
//   M_FULL  out = a*F y + cc*H in + d*z      (D = F - kappa H on one parity, residuals)
//   M_RECON out = F^-1 u, u = a*y + cc*H in, with |u - F out|^2 reduced (x_o of
//                                             Eq. 7 and the odd part of b - D x in one pass)
//
// One thread computes one output site (and one right-hand side: the
// right-hand sides of a site sit in the same block so that its links and
// clover entries are fetched from HBM once and hit L1 for the others).
// For each of the 8 directions the neighbour spinor is projected with
// (1 -/+ gamma_mu) to two spin components before the colour multiply
// (the rank-2 structure of Eq. 4), the link is rebuilt from 12 reals for
// FP32/FP16 (Sec. III-A), multiplied, and expanded back.
#pragma once

#include "stencil.cuh"

namespace qcd {

// <o|v> and |o|^2 of one site into red[0..2] (the omega of Alg. 2)
template <class T, class RA>
__device__ __forceinline__ void omega_sums(const Spinor<T> &o_, const Spinor<T> &v_, RA red[4])
{
    T dr = 0, di = 0, nn = 0;
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const cx<T> o = o_.s[s][i], v = v_.s[s][i];
            dr += o.r * v.r + o.i * v.i;
            di += o.r * v.i - o.i * v.r;
            nn += o.r * o.r + o.i * o.i;
        }
    red[0] += acc_cast<RA>(dr);
    red[1] += acc_cast<RA>(di);
    red[2] += acc_cast<RA>(nn);
}

// One output site cb (right-hand side r): the hops, the mode's epilogue, the
// site's contributions to the fused reductions.  The result is left in acc
// for the caller to store (true), so that a kernel with a grid reduction
// can publish its block's partial before its output stores are issued.
// hop(acc) computes acc = H in at the site, clov(x) applies the site's clover
// term (F^-1, or F for M_FULL) to x in place: from global memory, or from
// the staged shared-memory copies.
template <int P, int MODE, int RED, bool DAG, class RA, class HopF, class CloF>
__device__ __forceinline__ bool stencil_site(const StencilArgs &A, int cb, int r, RA red[4],
                                             Spinor<typename Prec<P>::T> &acc, const HopF &hop, const CloF &clov)
{
    using T = typename Prec<P>::T;
    const SpinorPtr out = rhs_ptr(A.out, r, A.rhs_stride, A.norm_stride);
    hop(acc);
    if (MODE == M_MULT) {
        clov(acc);
    } else if (MODE == M_DHAT) {
        clov(acc);
        Spinor<T> y;
        Prec<P>::load(rhs_ptr(A.y, r, A.rhs_stride, A.norm_stride), cb, y);
        axpby_sp(acc, sarg<T>(A.cc, A.ccf), acc, sarg<T>(A.a, A.af), y);
        if (A.has_z) {
            Spinor<T> z;
            Prec<P>::load(rhs_ptr(A.z, r, A.rhs_stride, A.norm_stride), cb, z);
            axpby_sp(acc, T(1), acc, sarg<T>(A.d, A.df32), z);
        }
        if (RED == R_OMEGA) {  // <out|aux>, |out|^2 (aux is usually y)
            if (A.aux.p != A.y.p) Prec<P>::load(rhs_ptr(A.aux, r, A.rhs_stride, A.norm_stride), cb, y);
            omega_sums<T, RA>(acc, y, red);
        }
    } else if (MODE == M_SRC) {
        Spinor<T> y;
        Prec<P>::load(rhs_ptr(A.y, r, A.rhs_stride, A.norm_stride), cb, y);
        axpby_sp(acc, sarg<T>(A.cc, A.ccf), acc, sarg<T>(A.a, A.af), y);
        clov(acc);
    } else if (MODE == M_RECON) {
        // x_o = F^-1 u with u = b_o + kappa H_oe x_e, and the odd rows of the
        // residual, b_o - (F_oo x_o - kappa H_oe x_e) = u - F x_o, from the
        // same hopping term
        Spinor<T> y;
        Prec<P>::load(rhs_ptr(A.y, r, A.rhs_stride, A.norm_stride), cb, y);
        axpby_sp(acc, sarg<T>(A.cc, A.ccf), acc, sarg<T>(A.a, A.af), y);  // u
        Spinor<T> xo = acc;
        clover_any<P>(A.C, A.out_par, cb, xo);
        Prec<P>::store(out, cb, xo);
        clover_any<P>(A.Cf, A.out_par, cb, xo);  // F x_o
        if (RED == R_NORM) {
            T nn = 0;
#pragma unroll
            for (int s = 0; s < 4; ++s)
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const cx<T> d = acc.s[s][i] - xo.s[s][i];
                    nn += d.r * d.r + d.i * d.i;
                }
            red[0] += acc_cast<RA>(nn);
        }
        return false;
    } else if (MODE == M_FULL) {
        // also the second half of the gamma5-hermitian S_ee = F_ee - k^2 H_eo F_oo^-1 H_oe
        // (a = 1, cc = -k^2, y = the operator's input), with its dot products
        Spinor<T> y;
        Prec<P>::load(rhs_ptr(A.y, r, A.rhs_stride, A.norm_stride), cb, y);
        Spinor<T> fy = y;
        clov(fy);
        axpby_sp(acc, sarg<T>(A.cc, A.ccf), acc, sarg<T>(A.a, A.af), fy);
        if (A.has_z) {
            Spinor<T> z;
            Prec<P>::load(rhs_ptr(A.z, r, A.rhs_stride, A.norm_stride), cb, z);
            axpby_sp(acc, T(1), acc, sarg<T>(A.d, A.df32), z);
        }
        if (RED == R_OMEGA) {  // <out|aux>, |out|^2 (aux is usually y)
            if (A.aux.p != A.y.p) Prec<P>::load(rhs_ptr(A.aux, r, A.rhs_stride, A.norm_stride), cb, y);
            omega_sums<T, RA>(acc, y, red);
        }
    }
    if (RED == R_DOT_AUX) {  // <aux|out>
        Spinor<T> w;
        Prec<P>::load(rhs_ptr(A.aux, r, A.rhs_stride, A.norm_stride), cb, w);
        T dr = 0, di = 0;
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const cx<T> a = w.s[s][i], o = acc.s[s][i];
                dr += a.r * o.r + a.i * o.i;
                di += a.r * o.i - a.i * o.r;
            }
        red[0] += acc_cast<RA>(dr);
        red[1] += acc_cast<RA>(di);
    } else if (RED == R_NORM) {
        T nn = 0;
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int i = 0; i < 3; ++i) nn += acc.s[s][i].r * acc.s[s][i].r + acc.s[s][i].i * acc.s[s][i].i;
        red[0] += acc_cast<RA>(nn);
    }
    return true;
}

template <int P, int MODE, int RED, bool DAG>
__device__ __forceinline__ void stencil_body(const StencilArgs &A)
{
    pdl_enter();
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0;
    if (A.done && *A.done) {
        if (A.skip && lead) *A.skip = 1;
        return;
    }
    if (A.skip && lead) *A.skip = 0;
    const int r = threadIdx.y;
    // reduction type: float at the FP32 / FP16 levels (see grid_reduce)
    using RA = typename std::conditional<P == QCD_F32 || P == QCD_F16, float, double>::type;
    RA red[4] = {RA(0), RA(0), RA(0), RA(0)};
    const int cb = blockIdx.x * blockDim.x + threadIdx.x;
    using T = typename Prec<P>::T;
    Spinor<T> acc;
    bool pending = false;
    if (cb < A.g.Vh) {
        const SpinorPtr in = rhs_ptr(A.in, r, A.rhs_stride, A.norm_stride);
        pending = stencil_site<P, MODE, RED, DAG>(
            A, cb, r, red, acc, [&](Spinor<T> &a) { hopping_any<P, DAG>(A.g, A.U, in, A.out_par, cb, a); },
            [&](Spinor<T> &x) { clover_any<P>(A.C, A.out_par, cb, x); });
    }
    if constexpr (RED != R_NONE) grid_reduce<RED == R_OMEGA ? 3 : RED == R_DOT_AUX ? 2 : 1>(red, A.red);
    // the output after the partial: the release that publishes the block's
    // partial does not wait for these stores (the next kernel, not the
    // finishing block, reads them)
    if (pending) Prec<P>::store(rhs_ptr(A.out, r, A.rhs_stride, A.norm_stride), cb, acc);
}

// Two register budgets of the same kernel; the autotuner picks one per
// launch configuration.  The default lets the compiler use what it needs
// (384 threads per block at most); the capped one trades a few spills for
// more resident warps, i.e. more loads in flight.
template <int P, int MODE, int RED, bool DAG>
__global__ void __launch_bounds__(384) stencil_kernel(StencilArgs A)
{
    stencil_body<P, MODE, RED, DAG>(A);
}

template <int P, int MODE, int RED, bool DAG>
__global__ void __maxnreg__(80) stencil_kernel_r80(StencilArgs A)
{
    stencil_body<P, MODE, RED, DAG>(A);
}

// The pipelined variant (FP32 / FP16, one right-hand side): the hops of
// hopping_pipe, the clover term from global memory; the compiler's register
// budget (the prefetched raw data of one hop lives beside the current one)
template <int P, int MODE, int RED, bool DAG>
__device__ __forceinline__ void stencil_body_pipe(const StencilArgs &A)
{
    pdl_enter();
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    if (A.done && *A.done) {
        if (A.skip && lead) *A.skip = 1;
        return;
    }
    if (A.skip && lead) *A.skip = 0;
    float red[4] = {0.f, 0.f, 0.f, 0.f};
    const int cb = blockIdx.x * blockDim.x + threadIdx.x;
    Spinor<float> acc;
    bool pending = false;
    if (cb < A.g.Vh)
        pending = stencil_site<P, MODE, RED, DAG>(
            A, cb, 0, red, acc, [&](Spinor<float> &a) { hopping_pipe<P, DAG>(A.g, A.U, A.in, A.out_par, cb, a); },
            [&](Spinor<float> &x) { clover_any<P>(A.C, A.out_par, cb, x); });
    if constexpr (RED != R_NONE) grid_reduce<RED == R_OMEGA ? 3 : RED == R_DOT_AUX ? 2 : 1>(red, A.red);
    if (pending) Prec<P>::store(A.out, cb, acc);
}

template <int P, int MODE, int RED, bool DAG>
__global__ void __launch_bounds__(256) stencil_kernel_pipe(StencilArgs A)
{
    if constexpr (P == QCD_F32 || P == QCD_F16) stencil_body_pipe<P, MODE, RED, DAG>(A);
}

// Second halves with fused dot products for a lockstep multi-RHS solve: the
// right-hand sides run as the fastest grid dimension (blockIdx.x = r,
// blockIdx.y = site block), so the blocks of one site block's right-hand
// sides are dispatched together and read its links and clover from HBM once
// (from L2 for the others); each right-hand side keeps its own reduction
// (partials, counter, solver state) and its own done flag, and equals the
// single-RHS kernel's result at the same sites per block to the bit.
template <int P, int MODE, int RED>
__device__ __forceinline__ void stencil_body_rg(const StencilArgs &A)
{
    pdl_enter();
    const int r = blockIdx.x;
    if (A.done && A.done[(size_t)r * A.done_stride]) return;  // uniform over the blocks of r
    using RA = typename std::conditional<P == QCD_F32 || P == QCD_F16, float, double>::type;
    RA red[4] = {RA(0), RA(0), RA(0), RA(0)};
    const int cb = blockIdx.y * blockDim.x + threadIdx.x;
    using T = typename Prec<P>::T;
    Spinor<T> acc;
    bool pending = false;
    if (cb < A.g.Vh) {
        const SpinorPtr in = rhs_ptr(A.in, r, A.rhs_stride, A.norm_stride);
        pending = stencil_site<P, MODE, RED, false>(
            A, cb, r, red, acc, [&](Spinor<T> &a) { hopping_any<P, false>(A.g, A.U, in, A.out_par, cb, a); },
            [&](Spinor<T> &x) { clover_any<P>(A.C, A.out_par, cb, x); });
    }
    RedArgs ra = A.red;
    ra.partials += (size_t)r * A.red_pstride;
    ra.counter += r;
    ra.st += r;
    grid_reduce_ex<RED == R_OMEGA ? 3 : RED == R_DOT_AUX ? 2 : 1>(red, ra, (int)blockIdx.y, (int)gridDim.y);
    if (pending) Prec<P>::store(rhs_ptr(A.out, r, A.rhs_stride, A.norm_stride), cb, acc);
}

template <int P, int MODE, int RED>
__global__ void __launch_bounds__(384) stencil_kernel_rg(StencilArgs A)
{
    stencil_body_rg<P, MODE, RED>(A);
}

template <int P, int MODE, int RED>
__global__ void __maxnreg__(80) stencil_kernel_rg_r80(StencilArgs A)
{
    stencil_body_rg<P, MODE, RED>(A);
}

// the launcher of the lockstep second halves (FP32 D^_ee with <r~|q> or
// omega): grid (nrhs, site blocks), the single-RHS entry's register budget
template <int P>
int dispatch_rg(const StencilCall &sc, const StencilArgs &A, int bx, cudaStream_t s, int variant)
{
    if constexpr (P == QCD_F32) {
        const dim3 grid(A.nrhs, nblocks(A.g.Vh, bx)), block(bx);
        if (sc.mode == M_DHAT && (sc.red == R_DOT_AUX || sc.red == R_OMEGA)) {
            if (sc.red == R_DOT_AUX) {
                if (variant == 1) launch_pdl(stencil_kernel_rg_r80<P, M_DHAT, R_DOT_AUX>, grid, block, 0, s, A);
                else launch_pdl(stencil_kernel_rg<P, M_DHAT, R_DOT_AUX>, grid, block, 0, s, A);
            } else {
                if (variant == 1) launch_pdl(stencil_kernel_rg_r80<P, M_DHAT, R_OMEGA>, grid, block, 0, s, A);
                else launch_pdl(stencil_kernel_rg<P, M_DHAT, R_OMEGA>, grid, block, 0, s, A);
            }
            return QCD_OK;
        }
    }
    set_error_message("the right-hand sides on the grid: FP32 D^ second halves with <r~|q> or omega only");
    return QCD_EINVAL;
}

// DF64 (arithmetic-bound, ~165 registers by default): a 128-register cap
// gives four 128-thread blocks per SM instead of three
template <int P, int MODE, int RED, bool DAG>
__global__ void __maxnreg__(128) stencil_kernel_r128(StencilArgs A)
{
    stencil_body<P, MODE, RED, DAG>(A);
}

// ---- host launcher -------------------------------------------------------
template <int P, int MODE, int RED, bool DAG>
static void launch_t(const StencilArgs &A, dim3 grid, dim3 block, cudaStream_t s, int variant)
{
    if constexpr (P == QCD_F32 || P == QCD_F16) {
        if (variant == 1) {
            launch_pdl(stencil_kernel_r80<P, MODE, RED, DAG>, grid, block, 0, s, A);
            return;
        }
        if constexpr (MODE == M_MULT || MODE == M_DHAT || MODE == M_FULL) {
            if (variant == 2 && block.y == 1 && block.x <= 256) {
                launch_pdl(stencil_kernel_pipe<P, MODE, RED, DAG>, grid, block, 0, s, A);
                return;
            }
        }
    }
    if constexpr (P == QCD_DF64) {
        if (variant == 1) {
            launch_pdl(stencil_kernel_r128<P, MODE, RED, DAG>, grid, block, 0, s, A);
            return;
        }
    }
    launch_pdl(stencil_kernel<P, MODE, RED, DAG>, grid, block, 0, s, A);
}

template <int P>
int dispatch(const StencilCall &sc, const StencilArgs &A, dim3 grid, dim3 block, cudaStream_t s, int v)
{
#define QCD_CASE(MODE, RED)                                                   \
    if (sc.mode == MODE && sc.red == RED) {                                   \
        if (sc.dagger) launch_t<P, MODE, RED, true>(A, grid, block, s, v);    \
        else launch_t<P, MODE, RED, false>(A, grid, block, s, v);             \
        return QCD_OK;                                                        \
    }
    QCD_CASE(M_HOP, R_NONE)
    QCD_CASE(M_MULT, R_NONE)
#undef QCD_CASE
    if (sc.dagger) {
        set_error_message("dagger is only available for the hopping and MULT kernels");
        return QCD_EINVAL;
    }
#define QCD_CASE(MODE, RED)                                                   \
    if (sc.mode == MODE && sc.red == RED) {                                   \
        launch_t<P, MODE, RED, false>(A, grid, block, s, v);                  \
        return QCD_OK;                                                        \
    }
    QCD_CASE(M_DHAT, R_NONE)
    QCD_CASE(M_DHAT, R_DOT_AUX)
    QCD_CASE(M_DHAT, R_OMEGA)
    QCD_CASE(M_DHAT, R_NORM)
    QCD_CASE(M_SRC, R_NONE)
    QCD_CASE(M_SRC, R_NORM)
    QCD_CASE(M_FULL, R_NONE)
    QCD_CASE(M_FULL, R_NORM)
    QCD_CASE(M_FULL, R_DOT_AUX)
    QCD_CASE(M_FULL, R_OMEGA)
    if constexpr (P == QCD_F64) {  // the FP64 reconstruction with its residual
        QCD_CASE(M_RECON, R_NORM)
    }
#undef QCD_CASE
    set_error_message("unsupported stencil mode %d / reduction %d", sc.mode, sc.red);
    return QCD_EINVAL;
}

}  // namespace qcd
