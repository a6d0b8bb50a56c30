// The hopping stencil H_{p,1-p} (Eq. 4) and the kernels built on it:
//   M_HOP   out = H in                       (qcd_dslash_eo)
//   M_MULT  out = F^-1 H in                  (MULT = H~, Sec. II-B)
//   M_DHAT  out = a*y + cc*F^-1 H in + d*z   (second half of D^ = 1 - k^2 H~_eo H~_oe,
//                                             with the dot products of Alg. 2 fused)
//   M_SRC   out = F^-1 (a*y + cc*H in)       (b^_e, Eq. 6, and x_o, Eq. 7)
//   M_FULL  out = a*F y + cc*H in + d*z      (D = F - kappa H on one parity, residuals)
//
// One thread computes one output site (and one right-hand side: the
// right-hand sides of a site sit in the same block so that its links and
// clover entries are fetched from HBM once and hit L1 for the others).
// For each of the 8 directions the neighbour spinor is projected with
// (1 -/+ gamma_mu) to two spin components before the colour multiply
// (the rank-2 structure of Eq. 4), the link is rebuilt from 12 reals for
// FP32/FP16 (Sec. III-A), multiplied, and expanded back.
#include "stencil.cuh"

namespace qcd {

template <int P, int MODE, int RED, bool DAG>
__device__ __forceinline__ void stencil_body(const StencilArgs &A)
{
    using T = typename Prec<P>::T;
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
    // A.spt sites per thread, in block-sized steps so that each step's loads
    // stay coalesced
    for (int k = 0; k < A.spt; ++k) {
        const int cb = (blockIdx.x * A.spt + k) * blockDim.x + threadIdx.x;
        if (cb >= A.g.Vh) break;
        const SpinorPtr in = rhs_ptr(A.in, r, A.rhs_stride, A.norm_stride);
        const SpinorPtr out = rhs_ptr(A.out, r, A.rhs_stride, A.norm_stride);
        Spinor<T> acc;
        hopping_any<P, DAG>(A.g, A.U, in, A.out_par, cb, acc);
        if (MODE == M_MULT) {
            clover_any<P>(A.C,A.out_par, cb, acc);
        } else if (MODE == M_DHAT) {
            clover_any<P>(A.C,A.out_par, cb, acc);
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
                T dr = 0, di = 0, nn = 0;
#pragma unroll
                for (int s = 0; s < 4; ++s)
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        const cx<T> o = acc.s[s][i], v = y.s[s][i];
                        dr += o.r * v.r + o.i * v.i;
                        di += o.r * v.i - o.i * v.r;
                        nn += o.r * o.r + o.i * o.i;
                    }
                red[0] += acc_cast<RA>(dr);
                red[1] += acc_cast<RA>(di);
                red[2] += acc_cast<RA>(nn);
            }
        } else if (MODE == M_SRC) {
            Spinor<T> y;
            Prec<P>::load(rhs_ptr(A.y, r, A.rhs_stride, A.norm_stride), cb, y);
            axpby_sp(acc, sarg<T>(A.cc, A.ccf), acc, sarg<T>(A.a, A.af), y);
            clover_any<P>(A.C,A.out_par, cb, acc);
        } else if (MODE == M_FULL) {
            Spinor<T> y;
            Prec<P>::load(rhs_ptr(A.y, r, A.rhs_stride, A.norm_stride), cb, y);
            clover_any<P>(A.C,A.out_par, cb, y);
            axpby_sp(acc, sarg<T>(A.cc, A.ccf), acc, sarg<T>(A.a, A.af), y);
            if (A.has_z) {
                Spinor<T> z;
                Prec<P>::load(rhs_ptr(A.z, r, A.rhs_stride, A.norm_stride), cb, z);
                axpby_sp(acc, T(1), acc, sarg<T>(A.d, A.df32), z);
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
        Prec<P>::store(out, cb, acc);
    }
    if constexpr (RED != R_NONE) grid_reduce<RED == R_OMEGA ? 3 : RED == R_DOT_AUX ? 2 : 1>(red, A.red);
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

// DF64 (arithmetic-bound, ~165 registers by default): a 128-register cap
// gives four 128-thread blocks per SM instead of three
template <int P, int MODE, int RED, bool DAG>
__global__ void __maxnreg__(128) stencil_kernel_r128(StencilArgs A)
{
    stencil_body<P, MODE, RED, DAG>(A);
}

// ---- multi-RHS FP32 MULT / hopping with shared-memory staging -------------
// One block = one 32-site layout block x nrhs right-hand sides.  The block
// first stages, for its 32 sites, the 8 neighbour indices, the 8 links
// rebuilt to 18 reals (forward links contiguous, backward links gathered),
// the time-boundary flags and the clover blocks in shared memory -- read from
// HBM and rebuilt once for all right-hand sides, since with 12 right-hand
// sides the kernel is close to issue-bound -- then thread (site, rhs)
// applies the stencil.
constexpr int MR_CLV4 = 18 * SB;        // float4 [comp][site]
constexpr int MR_LINK = 8 * 9 * SB;     // float2 [dir][comp][site], dir = 2 mu + (0 fwd, 1 bwd)
constexpr int MR_NB = 8 * SB;           // int    [dir][site]
constexpr size_t MR_BYTES = MR_CLV4 * sizeof(float4) + MR_LINK * sizeof(float2) + (MR_NB + SB) * sizeof(int);

template <int MU, int SF>
__device__ __forceinline__ void hop_dir_mrhs(const SpinorPtr &in, const float2 *s_lnk, const int *s_nb, int lane,
                                             int tflag, int t_bc, Spinor<float> &acc)
{
#pragma unroll
    for (int bwd = 0; bwd < 2; ++bwd) {
        const int d = 2 * MU + bwd;
        Spinor<float> psi;
        Prec<QCD_F32>::load(in, s_nb[d * SB + lane], psi);
        cx<float> h[2][3], q[2][3];
        if (bwd) project<MU, -SF>(psi, h);
        else project<MU, SF>(psi, h);
        Link<float> L;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const float2 f = s_lnk[(d * 9 + k) * SB + lane];
            L.u[k / 3][k % 3] = mk(f.x, f.y);
        }
        if (bwd) colour_mul<true>(L, h, q);
        else colour_mul<false>(L, h, q);
        if (MU == 3 && t_bc < 0 && (tflag & (1 << bwd)))
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int i = 0; i < 3; ++i) q[a][i] = -q[a][i];
        if (bwd) expand<MU, -SF>(acc, q);
        else expand<MU, SF>(acc, q);
    }
}

template <int MODE, bool DAG>
__device__ __forceinline__ void mrhs_body(const StencilArgs &A)
{
    extern __shared__ float4 sm[];
    float4 *s_clv = sm;
    float2 *s_lnk = (float2 *)(sm + MR_CLV4);
    int *s_nb = (int *)(s_lnk + MR_LINK);
    int *s_tf = s_nb + MR_NB;
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int nthr = blockDim.x * blockDim.y;
    const int cb0 = blockIdx.x * SB;
    for (int k = tid; k < 8 * SB; k += nthr) {
        const int l = k & (SB - 1), d = k >> 5;
        const int mu = d >> 1;
        const bool fwd = (d & 1) == 0;
        const int cb = cb0 + l;
        Link<float> U;
        int nb = 0;
        if (cb < A.g.Vh) {
            int c[4];
            site_coords(A.g, A.out_par, cb, c);
            nb = lex_hop(A.g, lex_of(A.g, c), c, mu, fwd ? +1 : -1) >> 1;
            Prec<QCD_F32>::load_link(A.U, fwd ? A.out_par : 1 - A.out_par, fwd ? cb : nb, mu, U);
            if (d == 0) s_tf[l] = (c[3] == A.g.L[3] - 1 ? 1 : 0) | (c[3] == 0 ? 2 : 0);
        } else {
#pragma unroll
            for (int k2 = 0; k2 < 9; ++k2) U.u[k2 / 3][k2 % 3] = mk(0.f, 0.f);
            if (d == 0) s_tf[l] = 0;
        }
        s_nb[d * SB + l] = nb;
#pragma unroll
        for (int k2 = 0; k2 < 9; ++k2) s_lnk[(d * 9 + k2) * SB + l] = make_float2(U.u[k2 / 3][k2 % 3].r, U.u[k2 / 3][k2 % 3].i);
    }
    if (MODE == M_MULT) {
        const float4 *Cl = (const float4 *)A.C.p[A.out_par];
        for (int k = tid; k < 18 * SB; k += nthr) {
            const int l = k & (SB - 1), comp = k >> 5;
            s_clv[k] = (cb0 + l < A.g.Vh) ? ld_stream(Cl + soa(cb0 + l, 18, comp)) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    __syncthreads();
    const int lane = threadIdx.x, cb = cb0 + lane, r = blockIdx.y * blockDim.y + threadIdx.y;
    if (cb >= A.g.Vh || r >= A.nrhs) return;
    const SpinorPtr in = rhs_ptr(A.in, r, A.rhs_stride, A.norm_stride);
    const SpinorPtr out = rhs_ptr(A.out, r, A.rhs_stride, A.norm_stride);
    const int tflag = s_tf[lane];
    Spinor<float> acc;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i) acc.s[a][i] = mk(0.f, 0.f);
    constexpr int SF = DAG ? -1 : 1;
    hop_dir_mrhs<0, SF>(in, s_lnk, s_nb, lane, tflag, A.g.t_bc, acc);
    hop_dir_mrhs<1, SF>(in, s_lnk, s_nb, lane, tflag, A.g.t_bc, acc);
    hop_dir_mrhs<2, SF>(in, s_lnk, s_nb, lane, tflag, A.g.t_bc, acc);
    hop_dir_mrhs<3, SF>(in, s_lnk, s_nb, lane, tflag, A.g.t_bc, acc);
    if (MODE == M_MULT) {
        // the clover inverse from shared memory (the F32 layout of load_clover)
        cx<float> xp[6], xm[6], yp[6], ym[6];
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                xp[3 * a + i] = acc.s[a][i] - acc.s[a + 2][i];
                xm[3 * a + i] = acc.s[a][i] + acc.s[a + 2][i];
            }
#pragma unroll
        for (int blk = 0; blk < 2; ++blk) {
            float rr[36];
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const float4 f = s_clv[(blk * 9 + k) * SB + lane];
                rr[4 * k] = f.x;
                rr[4 * k + 1] = f.y;
                rr[4 * k + 2] = f.z;
                rr[4 * k + 3] = f.w;
            }
            float d[6];
            cx<float> o[15];
#pragma unroll
            for (int k = 0; k < 6; ++k) d[k] = rr[k];
#pragma unroll
            for (int k = 0; k < 15; ++k) o[k] = mk(rr[6 + 2 * k], rr[7 + 2 * k]);
            herm6(d, o, blk == 0 ? xp : xm, blk == 0 ? yp : ym);
        }
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                acc.s[a][i] = 0.5f * (yp[3 * a + i] + ym[3 * a + i]);
                acc.s[a + 2][i] = 0.5f * (ym[3 * a + i] - yp[3 * a + i]);
            }
    }
    Prec<QCD_F32>::store(out, cb, acc);
}

template <int MODE, bool DAG>
__global__ void __launch_bounds__(512) mrhs_kernel(StencilArgs A)
{
    mrhs_body<MODE, DAG>(A);
}

template <int MODE, bool DAG>
__global__ void __maxnreg__(80) mrhs_kernel_r80(StencilArgs A)
{
    mrhs_body<MODE, DAG>(A);
}

// tile: right-hand sides per block (the links and clover of a 32-site block
// are staged once per tile; the autotuner picks the tile)
static int launch_mrhs(const StencilCall &sc, const StencilArgs &A, int nrhs, cudaStream_t s, int variant, int tile)
{
    if (tile < 1 || tile > nrhs) tile = nrhs;
    dim3 block(SB, tile), grid(nblocks(A.g.Vh, SB), (nrhs + tile - 1) / tile);
    const size_t smem = MR_BYTES;
#define QCD_MR(MODE, DAG)                                                                              \
    do {                                                                                               \
        if (variant == 1) mrhs_kernel_r80<MODE, DAG><<<grid, block, smem, s>>>(A);                     \
        else mrhs_kernel<MODE, DAG><<<grid, block, smem, s>>>(A);                                      \
    } while (0)
    if (sc.mode == M_MULT) {
        if (sc.dagger) QCD_MR(M_MULT, true);
        else QCD_MR(M_MULT, false);
    } else {
        if (sc.dagger) QCD_MR(M_HOP, true);
        else QCD_MR(M_HOP, false);
    }
#undef QCD_MR
    return QCD_OK;
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
static int dispatch(const StencilCall &sc, const StencilArgs &A, dim3 grid, dim3 block, cudaStream_t s, int v)
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
#undef QCD_CASE
    set_error_message("unsupported stencil mode %d / reduction %d", sc.mode, sc.red);
    return QCD_EINVAL;
}

// Algorithmic bytes per output site of one stencil launch (each input read
// once, the output written once), by precision: spinor, link, clover.
static void site_bytes(int prec, double &spinor, double &link, double &clover)
{
    if (prec == QCD_F64 || prec == QCD_DF64) { spinor = 192; link = 144; clover = 576; }
    else if (prec == QCD_F32) { spinor = 96; link = 48; clover = 288; }
    else { spinor = 52; link = 24; clover = 144; }
}

unsigned tune_key(const StencilCall &sc)
{
    const unsigned nr = sc.nrhs < 1 ? 1 : (sc.nrhs > 31 ? 31 : sc.nrhs);
    return (unsigned)sc.prec | ((unsigned)sc.mode << 2) | ((unsigned)sc.red << 5) | ((unsigned)(sc.dagger != 0) << 7) |
           (nr << 8);
}

double stencil_bytes(const qcd_ctx *c, const StencilCall &sc)
{
    double sp, lk, cl;
    site_bytes(sc.prec, sp, lk, cl);
    const int nrhs = sc.nrhs < 1 ? 1 : sc.nrhs;
    double per_site = nrhs * 2 * sp + 8 * lk;  // in, out, links
    if (sc.mode != M_HOP) per_site += cl;
    if (sc.mode == M_DHAT || sc.mode == M_SRC || sc.mode == M_FULL) per_site += nrhs * sp;  // y
    if (sc.d != 0.0 && (sc.mode == M_DHAT || sc.mode == M_FULL)) per_site += nrhs * sp;   // z
    if (sc.red == R_DOT_AUX || (sc.red == R_OMEGA && sc.aux.p != sc.y.p)) per_site += nrhs * sp;
    return per_site * c->g.Vh;
}

bool is_mrhs(const StencilCall &sc)
{
    return sc.prec == QCD_F32 && sc.nrhs > 1 && sc.red == R_NONE && (sc.mode == M_MULT || sc.mode == M_HOP);
}

int launch_stencil(qcd_ctx *c, const StencilCall &sc)
{
    StencilArgs A;
    A.g = c->g;
    const int p = sc.prec;
    for (int par = 0; par < 2; ++par) {
        A.U.a[par] = p == QCD_F64 ? c->U64[par] : p == QCD_F32 ? c->U32[par] : p == QCD_DF64 ? c->UDF[par] : c->U16a[par];
        A.U.b[par] = c->U16b[par];
        A.C.p[par] = (sc.mode == M_FULL) ? c->C[p][par] : c->Ci[p][par];
    }
    A.out = sc.out.sp();
    A.in = sc.in.sp();
    A.y = sc.y.sp();
    A.aux = sc.aux.sp();
    A.z = sc.z.sp();
    A.out_par = sc.out_par;
    A.a = sc.a;
    A.cc = sc.cc;
    A.d = sc.d;
    A.af = (float)sc.a;
    A.ccf = (float)sc.cc;
    A.df32 = (float)sc.d;
    A.has_z = sc.d != 0.0;
    A.rhs_stride = sc.rhs_stride;
    A.norm_stride = sc.norm_stride;
    A.nrhs = sc.nrhs < 1 ? 1 : sc.nrhs;
    A.red = sc.red_args;
    A.done = sc.done;
    const int nrhs = sc.nrhs < 1 ? 1 : sc.nrhs;
    if (nrhs > 16) {
        set_error_message("nrhs > 16 per launch");
        return QCD_EINVAL;
    }
    int bx = 128, variant = 0;  // bx: sites per block, or for the multi-RHS kernel the RHS tile
    if (nrhs > 1) bx = is_mrhs(sc) ? nrhs : nrhs <= 4 ? 64 : 32;
    if (sc.force_variant >= 0) {
        variant = sc.force_variant;
        bx = sc.force_bx;
    } else {
        auto it = c->tune.find(tune_key(sc));
        if (it != c->tune.end()) {
            variant = it->second.variant;
            bx = it->second.bx;
        }
    }
    // variant bit 0: register budget; bit 1: two sites per thread
    A.spt = is_mrhs(sc) ? 1 : 1 + ((variant >> 1) & 1);
    dim3 block(bx, nrhs);
    dim3 grid(nblocks(c->g.Vh, bx * A.spt));
    if (!is_mrhs(sc) && sc.red != R_NONE && (int)grid.x > c->partial_blocks) {
        set_error_message("reduction grid too large");
        return QCD_EINVAL;
    }
    const int cls = p == QCD_F32    ? (sc.mode == M_DHAT ? QCD_K_DHAT_F32 : QCD_K_MULT_F32)
                    : p == QCD_F16  ? QCD_K_MULT_F16
                    : p == QCD_DF64 ? QCD_K_MULT_DF64
                                    : QCD_K_MULT_F64;
    ProfScope prof(c, cls, stencil_bytes(c, sc));
    A.skip = prof.flag;
    int rc;
    const int rv = variant & 1;
    if (is_mrhs(sc)) rc = launch_mrhs(sc, A, nrhs, c->stream, rv, bx);
    else if (p == QCD_F64) rc = dispatch<QCD_F64>(sc, A, grid, block, c->stream, rv);
    else if (p == QCD_F32) rc = dispatch<QCD_F32>(sc, A, grid, block, c->stream, rv);
    else if (p == QCD_DF64) rc = dispatch<QCD_DF64>(sc, A, grid, block, c->stream, rv);
    else rc = dispatch<QCD_F16>(sc, A, grid, block, c->stream, rv);
    if (rc != QCD_OK) return rc;
    QCD_CUDA_CHECK(cudaGetLastError());
    return QCD_OK;
}

}  // namespace qcd
