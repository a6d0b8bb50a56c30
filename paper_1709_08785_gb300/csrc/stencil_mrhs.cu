// Multi-right-hand-side FP32 MULT and hopping term (Eq. 4): the links and
// clover blocks of each 32-site block staged once for all right-hand sides of
// a tile (in shared memory, or copied on into tensor memory), and packed FP32
// pair arithmetic.
#include <atomic>

#include "stencil.cuh"
#include "tmem.cuh"

namespace qcd {

// ---- multi-RHS FP32 MULT / hopping ---------------------------------------
// One block = one 32-site layout block x a tile of right-hand sides.  The
// block first stages, for its 32 sites, the 8 neighbour indices, the 8 links
// rebuilt to 18 reals (forward links contiguous, backward links gathered),
// the time-boundary flags and the clover blocks -- read from HBM and rebuilt
// once for all right-hand sides -- then thread (site, rhs) applies the
// stencil.
//
// Per site and right-hand side the stencil reads 864 bytes of neighbour
// spinors and output through the L1 data pipe, and 984 bytes of staged links
// and clover.  From shared memory those share the L1 pipe's 128 bytes per
// clock, which then bounds the kernel above the HBM time; with TMEM = true the
// staged words are copied once per block into tensor memory (256 columns, the
// site's words in the lane of its thread, replicated in the four lane
// quarters) and read from there with tcgen05.ld, a path of its own.
//
// The arithmetic runs on packed FP32 pairs (one instruction, two lanes, each
// rounded as the scalar fmaf / add / mul):
// * the hops pair the two spin rows of a half spinor: the link products of
//   rows 0 and 1 share every link element; the accumulator holds the upper
//   spins as {s0, s1} and the lower ones as {s3, s2}, the order in which the
//   x, y and t expansions need no exchange of lanes;
// * the clover pairs its two chiral blocks, lane 0 acting on chi_+ and lane 1
//   on chi_- with the same element of the other block.
// Each lane performs the scalar kernel's operations in the scalar kernel's
// order (a negated operand is moved to the other factor, which is exact, and
// the clover's final 1/2 is folded into the staged blocks, a power of two),
// so every right-hand side equals the single-RHS kernel's result to the bit.
//
// Staged words of a site (one 32-bit column each, 64 groups of 4):
//   links     col 16 d + 2 k + {re, im}, elements k = 0..7 of direction d
//             col 128 + 2 d + {re, im}, element 8 (d = 2 mu + bwd)
//   clover    col 144 + 2 i + {+, -}, diagonal i = 0..5 of the two blocks
//             col 160 + 4 k + {re+, re-, im+, im-}, off-diagonal k = 0..14
//             col 224 + 2 k + {-im+, -im-}
// each times 1/2 for the clover.
constexpr int MR_COLS = 256;
constexpr int MR_GRP = MR_COLS / 4;
constexpr int MR_NB = 8 * SB;  // int [dir][site]
constexpr size_t MR_BYTES = (size_t)MR_GRP * SB * sizeof(float4) + (MR_NB + SB) * sizeof(int) + 16;

__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }

// the staged words of this thread's site: from shared memory (s_col[group][site])
// or from the warp's lane quarter of tensor memory
template <bool TMEM>
struct Cols {
    const float4 *s_col;
    int lane;
    uint32_t t;  // TMEM: column 0 of the warp's lane quarter
    template <int N>
    __device__ __forceinline__ void get(int col, float *v) const
    {
        if constexpr (TMEM) {
            if constexpr (N == 16) tm::ld16(t + col, v);
            else if constexpr (N == 8) tm::ld8(t + col, v);
            else tm::ld2(t + col, v);
        } else {
            if constexpr (N == 2) {
                const float2 f = ((const float2 *)s_col)[((col >> 2) * SB + lane) * 2 + ((col >> 1) & 1)];
                v[0] = f.x;
                v[1] = f.y;
            } else {
#pragma unroll
                for (int g = 0; g < N / 4; ++g) {
                    const float4 f = s_col[((col >> 2) + g) * SB + lane];
                    v[4 * g] = f.x;
                    v[4 * g + 1] = f.y;
                    v[4 * g + 2] = f.z;
                    v[4 * g + 3] = f.w;
                }
            }
        }
    }
    __device__ __forceinline__ void sync() const
    {
        if constexpr (TMEM) tm::wait_ld();
    }
};

// G = U H (BWD = 0) or U^dag H (BWD = 1) for the spin-row pair H, element
// k = 3 i + j of the link at L[2 k], L[2 k + 1]; the lane sequence of
// colour_mul's fma_ / fmac_
template <int BWD>
__device__ __forceinline__ void colour_mul_pair(const float L[18], const float2 Hr[3], const float2 Hi[3], float2 Gr[3],
                                                float2 Gi[3])
{
    const float2 m1 = make_float2(-1.f, -1.f);
    float2 N[3];  // (-u_im) x = u_im (-x): -H_im for U, -H_re for U^dag
#pragma unroll
    for (int j = 0; j < 3; ++j) N[j] = pmul(BWD ? Hr[j] : Hi[j], m1);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        float2 sr = make_float2(0.f, 0.f), si = make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int k = BWD ? 3 * j + i : 3 * i + j;
            const float2 ur = make_float2(L[2 * k], L[2 * k]), ui = make_float2(L[2 * k + 1], L[2 * k + 1]);
            sr = pfma(ur, Hr[j], sr);
            sr = pfma(ui, BWD ? Hi[j] : N[j], sr);
            si = pfma(ur, Hi[j], si);
            si = pfma(ui, BWD ? N[j] : Hr[j], si);
        }
        Gr[i] = sr;
        Gi[i] = si;
    }
}

// the spinor accumulator as lane pairs: U = {s0, s1}, L = {s3, s2}
struct PairAcc {
    float2 Ur[3], Ui[3], Lr[3], Li[3];
};

template <int MU, int S>
__device__ __forceinline__ void project_pair(const Spinor<float> &psi, float2 Hr[3], float2 Hi[3])
{
    cx<float> h[2][3];
    project<MU, S>(psi, h);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        // mu = t, S = +1 feeds the lower pair {s3, s2}: rows in the order {h1, h0}
        const int a0 = (MU == 3 && S > 0) ? 1 : 0;
        Hr[c] = make_float2(h[a0][c].r, h[1 - a0][c].r);
        Hi[c] = make_float2(h[a0][c].i, h[1 - a0][c].i);
    }
}

// expand's accumulation on the pairs (f = +-2 for mu = t: the projector's
// factor 2 and the boundary sign)
template <int MU, int S>
__device__ __forceinline__ void expand_pair(PairAcc &A, const float2 Gr[3], const float2 Gi[3], float f)
{
    const float2 m1 = make_float2(-1.f, -1.f);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        if (MU == 3) {
            const float2 w = make_float2(f, f);
            if (S > 0) {
                A.Lr[c] = pfma(Gr[c], w, A.Lr[c]);
                A.Li[c] = pfma(Gi[c], w, A.Li[c]);
            } else {
                A.Ur[c] = pfma(Gr[c], w, A.Ur[c]);
                A.Ui[c] = pfma(Gi[c], w, A.Ui[c]);
            }
        } else {
            A.Ur[c] = padd(A.Ur[c], Gr[c]);
            A.Ui[c] = padd(A.Ui[c], Gi[c]);
            if (MU == 0) {  // {s3, s2} += -S i {g0, g1}
                if (S > 0) {
                    A.Lr[c] = padd(A.Lr[c], Gi[c]);
                    A.Li[c] = pfma(Gr[c], m1, A.Li[c]);
                } else {
                    A.Lr[c] = pfma(Gi[c], m1, A.Lr[c]);
                    A.Li[c] = padd(A.Li[c], Gr[c]);
                }
            } else if (MU == 1) {  // {s3, s2} += S {g0, -g1}
                const float2 sg = S > 0 ? make_float2(1.f, -1.f) : make_float2(-1.f, 1.f);
                A.Lr[c] = pfma(Gr[c], sg, A.Lr[c]);
                A.Li[c] = pfma(Gi[c], sg, A.Li[c]);
            } else {  // {s3, s2} += -S i {-g1, g0}: lanes exchanged, scalar
                if (S > 0) {
                    A.Lr[c].x = A.Lr[c].x - Gi[c].y;
                    A.Lr[c].y = A.Lr[c].y + Gi[c].x;
                    A.Li[c].x = A.Li[c].x + Gr[c].y;
                    A.Li[c].y = A.Li[c].y - Gr[c].x;
                } else {
                    A.Lr[c].x = A.Lr[c].x + Gi[c].y;
                    A.Lr[c].y = A.Lr[c].y - Gi[c].x;
                    A.Li[c].x = A.Li[c].x - Gr[c].y;
                    A.Li[c].y = A.Li[c].y + Gr[c].x;
                }
            }
        }
    }
}

template <int MU, int SF, bool TMEM>
__device__ __forceinline__ void hop_dir_mrhs(const SpinorPtr &in, const Cols<TMEM> &cols, const int *s_nb, int lane,
                                             int tflag, int t_bc, PairAcc &A)
{
#pragma unroll
    for (int bwd = 0; bwd < 2; ++bwd) {
        const int d = 2 * MU + bwd;
        Spinor<float> psi;
        Prec<QCD_F32>::load(in, s_nb[d * SB + lane], psi);
        float L[18];
        cols.template get<16>(16 * d, L);
        cols.template get<2>(128 + 2 * d, L + 16);
        float2 Hr[3], Hi[3], Gr[3], Gi[3];
        if (bwd) project_pair<MU, -SF>(psi, Hr, Hi);
        else project_pair<MU, SF>(psi, Hr, Hi);
        cols.sync();
        if (bwd) colour_mul_pair<1>(L, Hr, Hi, Gr, Gi);
        else colour_mul_pair<0>(L, Hr, Hi, Gr, Gi);
        const float f = (MU == 3 && t_bc < 0 && (tflag & (1 << bwd))) ? -2.f : 2.f;
        if (bwd) expand_pair<MU, -SF>(A, Gr, Gi, f);
        else expand_pair<MU, SF>(A, Gr, Gi, f);
    }
}

// y = (A+ xp, A- xm) for the clover blocks in lane pairs, in herm6's order
template <bool TMEM>
__device__ __forceinline__ void herm6_pair(const Cols<TMEM> &cols, const float2 Xr[6], const float2 Xi[6], float2 Yr[6],
                                           float2 Yi[6])
{
    {
        float dd[16];
        cols.template get<16>(144, dd);
        cols.sync();
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            const float2 d = make_float2(dd[2 * i], dd[2 * i + 1]);
            Yr[i] = pmul(d, Xr[i]);
            Yi[i] = pmul(d, Xi[i]);
        }
    }
    // off-diagonal k = (i, j), i = 1..5, j < i, row by row; four at a time
    float o[16], n[8];
    int k = 0;
#pragma unroll
    for (int i = 1; i < 6; ++i)
#pragma unroll
        for (int j = 0; j < i; ++j) {
            if ((k & 3) == 0) {
                cols.template get<16>(160 + 4 * k, o);
                cols.template get<8>(224 + 2 * k, n);
                cols.sync();
            }
            const int kk = k & 3;
            const float2 orr = make_float2(o[4 * kk], o[4 * kk + 1]), oi = make_float2(o[4 * kk + 2], o[4 * kk + 3]);
            const float2 noi = make_float2(n[2 * kk], n[2 * kk + 1]);
            // y_i += A_ij x_j
            Yr[i] = pfma(orr, Xr[j], Yr[i]);
            Yr[i] = pfma(noi, Xi[j], Yr[i]);
            Yi[i] = pfma(orr, Xi[j], Yi[i]);
            Yi[i] = pfma(oi, Xr[j], Yi[i]);
            // y_j += conj(A_ij) x_i
            Yr[j] = pfma(orr, Xr[i], Yr[j]);
            Yr[j] = pfma(oi, Xi[i], Yr[j]);
            Yi[j] = pfma(orr, Xi[i], Yi[j]);
            Yi[j] = pfma(noi, Xr[i], Yi[j]);
            ++k;
        }
}

template <int MODE, bool DAG, bool TMEM>
__device__ __forceinline__ void mrhs_body(const StencilArgs &A)
{
    extern __shared__ float4 sm[];
    float4 *s_col = sm;
    int *s_nb = (int *)(s_col + MR_GRP * SB);
    int *s_tf = s_nb + MR_NB;
    uint32_t *s_taddr = (uint32_t *)(s_tf + SB);
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int nthr = blockDim.x * blockDim.y;
    const int warp = threadIdx.y;  // blockDim.x == 32
    const int cb0 = blockIdx.x * SB;
    constexpr int ncols = MODE == M_MULT ? MR_COLS : 144;  // the hopping term reads no clover
    if (TMEM && warp == 0) tm::alloc(s_taddr, MR_COLS);
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
        for (int g = 0; g < 4; ++g) {
            const cx<float> a = U.u[(2 * g) / 3][(2 * g) % 3], b = U.u[(2 * g + 1) / 3][(2 * g + 1) % 3];
            s_col[(4 * d + g) * SB + l] = make_float4(a.r, a.i, b.r, b.i);
        }
        ((float2 *)s_col)[((32 + (d >> 1)) * SB + l) * 2 + (d & 1)] = make_float2(U.u[2][2].r, U.u[2][2].i);
    }
    if (MODE == M_MULT) {
        // float4 k of block 0 and float4 k of block 1 (reals 4k..4k+3 of
        // each: d[0..5], then o[q] as (re, im) from real 6), times 1/2
        const float4 *Cl = (const float4 *)A.C.p[A.out_par];
        float *cf = (float *)s_col;
        auto at = [&](int col, int l) -> float & { return cf[((col >> 2) * SB + l) * 4 + (col & 3)]; };
        for (int k = tid; k < 9 * SB; k += nthr) {
            const int l = k & (SB - 1), q4 = k >> 5;
            const bool in = cb0 + l < A.g.Vh;
            const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 f0 = in ? ld_stream(Cl + soa(cb0 + l, 18, q4)) : z;
            const float4 f1 = in ? ld_stream(Cl + soa(cb0 + l, 18, q4 + 9)) : z;
            const float a[4] = {f0.x, f0.y, f0.z, f0.w}, b[4] = {f1.x, f1.y, f1.z, f1.w};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int r = 4 * q4 + t;
                const float p = 0.5f * a[t], m = 0.5f * b[t];
                if (r < 6) {
                    at(144 + 2 * r, l) = p;
                    at(145 + 2 * r, l) = m;
                } else {
                    const int o = (r - 6) >> 1, im = (r - 6) & 1;
                    at(160 + 4 * o + 2 * im, l) = p;
                    at(161 + 4 * o + 2 * im, l) = m;
                    if (im) {
                        at(224 + 2 * o, l) = -p;
                        at(225 + 2 * o, l) = -m;
                    }
                }
            }
        }
    }
    if (TMEM) tm::fence_before();
    __syncthreads();
    uint32_t tq = 0;
    if (TMEM) {
        tm::fence_after();
        // the warps of each lane quarter copy the staged words, 16 columns a
        // store, into their quarter
        tq = tm::addr(*s_taddr, warp, 0);
        const int nw = blockDim.y, q = warp & 3, nq = (nw - q + 3) / 4;
        for (int ch = warp >> 2; ch < ncols / 16; ch += nq) {
            float v[16];
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                const float4 f = s_col[(4 * ch + g) * SB + threadIdx.x];
                v[4 * g] = f.x;
                v[4 * g + 1] = f.y;
                v[4 * g + 2] = f.z;
                v[4 * g + 3] = f.w;
            }
            tm::st16(tq + 16 * ch, v);
        }
        tm::wait_st();
        tm::fence_before();
        __syncthreads();
        tm::fence_after();
    }
    const int lane = threadIdx.x, cb = cb0 + lane, r = blockIdx.y * blockDim.y + threadIdx.y;
    // with TMEM every thread of a warp takes part in the warp-wide loads: a
    // thread past the lattice or the last right-hand side computes on a valid
    // site and right-hand side and stores nothing
    const bool valid = cb < A.g.Vh && r < A.nrhs;
    if (!TMEM && !valid) return;
    const int rr = r < A.nrhs ? r : 0;
    const SpinorPtr in = rhs_ptr(A.in, rr, A.rhs_stride, A.norm_stride);
    const SpinorPtr out = rhs_ptr(A.out, rr, A.rhs_stride, A.norm_stride);
    const Cols<TMEM> cols{s_col, lane, tq};
    const int tflag = s_tf[lane];
    PairAcc P;
#pragma unroll
    for (int c = 0; c < 3; ++c) P.Ur[c] = P.Ui[c] = P.Lr[c] = P.Li[c] = make_float2(0.f, 0.f);
    constexpr int SF = DAG ? -1 : 1;
    hop_dir_mrhs<0, SF, TMEM>(in, cols, s_nb, lane, tflag, A.g.t_bc, P);
    hop_dir_mrhs<1, SF, TMEM>(in, cols, s_nb, lane, tflag, A.g.t_bc, P);
    hop_dir_mrhs<2, SF, TMEM>(in, cols, s_nb, lane, tflag, A.g.t_bc, P);
    hop_dir_mrhs<3, SF, TMEM>(in, cols, s_nb, lane, tflag, A.g.t_bc, P);
    Spinor<float> acc;
    if (MODE == M_MULT) {
        // X = {xp, xm} with xp = s_a - s_a+2, xm = s_a + s_a+2 (a = 0: s0 = U.x,
        // s2 = L.y; a = 1: s1 = U.y, s3 = L.x)
        float2 Xr[6], Xi[6], Yr[6], Yi[6];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            Xr[c] = make_float2(P.Ur[c].x - P.Lr[c].y, P.Ur[c].x + P.Lr[c].y);
            Xi[c] = make_float2(P.Ui[c].x - P.Li[c].y, P.Ui[c].x + P.Li[c].y);
            Xr[3 + c] = make_float2(P.Ur[c].y - P.Lr[c].x, P.Ur[c].y + P.Lr[c].x);
            Xi[3 + c] = make_float2(P.Ui[c].y - P.Li[c].x, P.Ui[c].y + P.Li[c].x);
        }
        herm6_pair<TMEM>(cols, Xr, Xi, Yr, Yi);
        // (yp + ym) / 2 and (ym - yp) / 2, the halves already in the blocks
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float2 yr = Yr[3 * a + c], yi = Yi[3 * a + c];
                acc.s[a][c] = mk(yr.x + yr.y, yi.x + yi.y);
                acc.s[a + 2][c] = mk(yr.y - yr.x, yi.y - yi.x);
            }
    } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            acc.s[0][c] = mk(P.Ur[c].x, P.Ui[c].x);
            acc.s[1][c] = mk(P.Ur[c].y, P.Ui[c].y);
            acc.s[2][c] = mk(P.Lr[c].y, P.Li[c].y);
            acc.s[3][c] = mk(P.Lr[c].x, P.Li[c].x);
        }
    }
    if (valid) Prec<QCD_F32>::store(out, cb, acc);
    if (TMEM) {
        tm::fence_before();
        __syncthreads();
        tm::fence_after();
        if (warp == 0) tm::dealloc(*s_taddr, MR_COLS);
    }
}

template <int MODE, bool DAG, bool TMEM>
__global__ void __launch_bounds__(512) mrhs_kernel(StencilArgs A)
{
    mrhs_body<MODE, DAG, TMEM>(A);
}

template <int MODE, bool DAG, bool TMEM>
__global__ void __maxnreg__(80) mrhs_kernel_r80(StencilArgs A)
{
    mrhs_body<MODE, DAG, TMEM>(A);
}

// the staging area is above the 48 KB default: opt in once per device and kernel
template <auto K>
static void smem_opt_in(size_t bytes)
{
    static std::atomic<unsigned long long> done{0};
    int dev = 0;
    cudaGetDevice(&dev);
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(done.load(std::memory_order_relaxed) & bit)) {
        cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        done.fetch_or(bit);
    }
}

// tile: right-hand sides per block (the links and clover of a 32-site block
// are staged once per tile; the autotuner picks the tile); variants 0 / 1:
// staged words read from shared memory, 2 / 3: from tensor memory; 1 / 3
// with the 80-register cap
int launch_mrhs(const StencilCall &sc, const StencilArgs &A, int nrhs, cudaStream_t s, int variant, int tile)
{
    if (tile < 1 || tile > nrhs) tile = nrhs;
    dim3 block(SB, tile), grid(nblocks(A.g.Vh, SB), (nrhs + tile - 1) / tile);
    const size_t smem = MR_BYTES;
#define QCD_MR_K(KERN, MODE, DAG, TM)                                                                  \
    do {                                                                                               \
        smem_opt_in<KERN<MODE, DAG, TM>>(smem);                                                        \
        KERN<MODE, DAG, TM><<<grid, block, smem, s>>>(A);                                              \
    } while (0)
#define QCD_MR(MODE, DAG)                                                                              \
    do {                                                                                               \
        if (variant == 1) QCD_MR_K(mrhs_kernel_r80, MODE, DAG, false);                                 \
        else if (variant == 2) QCD_MR_K(mrhs_kernel, MODE, DAG, true);                                 \
        else if (variant == 3) QCD_MR_K(mrhs_kernel_r80, MODE, DAG, true);                             \
        else QCD_MR_K(mrhs_kernel, MODE, DAG, false);                                                  \
    } while (0)
    if (sc.mode == M_MULT) {
        if (sc.dagger) QCD_MR(M_MULT, true);
        else QCD_MR(M_MULT, false);
    } else {
        if (sc.dagger) QCD_MR(M_HOP, true);
        else QCD_MR(M_HOP, false);
    }
#undef QCD_MR
#undef QCD_MR_K
    return QCD_OK;
}

}  // namespace qcd
