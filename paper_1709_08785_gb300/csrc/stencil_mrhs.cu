// Multi-right-hand-side FP32 MULT and hopping term (Eq. 4): the links and
// clover blocks of each 32-site block staged once for all right-hand sides of
// a tile, by resident blocks that copy the next site block in while they
// compute the current one, and packed FP32 pair arithmetic.
#include <atomic>

#include "stencil.cuh"

namespace qcd {

// ---- multi-RHS FP32 MULT / hopping ---------------------------------------
// A block = a 32-site layout block x a tile of right-hand sides at a time.
// For its 32 sites it stages the 8 neighbour indices, the 8 links rebuilt to
// 18 reals (forward links contiguous, backward links gathered), the
// time-boundary flags and the clover blocks in shared memory -- read from HBM
// and rebuilt once for all right-hand sides -- then thread (site, rhs) applies
// the stencil.
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
// Staged words of a site (one 32-bit word each, 64 groups of 4, [group][site]):
//   links     word 16 d + 2 k + {re, im}, elements k = 0..7 of direction d
//             word 128 + 2 d + {re, im}, element 8 (d = 2 mu + bwd)
//   clover    word 144 + 2 i + {+, -}, diagonal i = 0..5 of the two blocks
//             word 160 + 4 k + {re+, re-, im+, im-}, off-diagonal k = 0..14
// each times 1/2 for the clover (the negated imaginary parts the FP32-pair
// FMAs need are formed in registers: shared-memory reads, not arithmetic,
// bound this kernel).
constexpr int MR_COLS = 220;  // staged words per site
constexpr int MR_GRP = MR_COLS / 4;
constexpr int MR_NB = 8 * SB;  // int [dir][site]
constexpr size_t MR_BYTES = (size_t)(MR_GRP * SB + 8 * 3 * SB + 18 * SB) * sizeof(float4) + 2 * (MR_NB + SB) * sizeof(int);

// the staged words of this thread's site (s_col[group][site])
struct Cols {
    const float4 *s_col;
    int lane;
    template <int N>
    __device__ __forceinline__ void get(int col, float *v) const
    {
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
};

// the spinor accumulator as lane pairs: U = {s0, s1}, L = {s3, s2}
struct PairAcc {
    float2 Ur[3], Ui[3], Lr[3], Li[3];
};

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

template <int MU, int SF>
__device__ __forceinline__ void hop_dir_mrhs(const SpinorPtr &in, const Cols &cols, const int *s_nb, int lane,
                                             int tflag, int t_bc, PairAcc &A)
{
#pragma unroll
    for (int bwd = 0; bwd < 2; ++bwd) {
        const int d = 2 * MU + bwd;
        Spinor<float> psi;
        Prec<QCD_F32>::load(in, s_nb[d * SB + lane], psi);
        float L[18];
        cols.get<16>(16 * d, L);
        cols.get<2>(128 + 2 * d, L + 16);
        float2 Hr[3], Hi[3], Gr[3], Gi[3];
        if (bwd) project_pair<MU, -SF>(psi, Hr, Hi);
        else project_pair<MU, SF>(psi, Hr, Hi);
        const auto u = [&](int k) { return make_float2(L[2 * k], L[2 * k + 1]); };
        if (bwd) colour_mul_pair<1>(u, Hr, Hi, Gr, Gi);
        else colour_mul_pair<0>(u, Hr, Hi, Gr, Gi);
        const float f = (MU == 3 && t_bc < 0 && (tflag & (1 << bwd))) ? -2.f : 2.f;
        if (bwd) expand_pair<MU, -SF>(A, Gr, Gi, f);
        else expand_pair<MU, SF>(A, Gr, Gi, f);
    }
}

// y = (A+ xp, A- xm) for the clover blocks in lane pairs, in herm6's order
__device__ __forceinline__ void herm6_pair(const Cols &cols, const float2 Xr[6], const float2 Xi[6], float2 Yr[6],
                                           float2 Yi[6])
{
    {
        float dd[16];
        cols.get<16>(144, dd);
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            const float2 d = make_float2(dd[2 * i], dd[2 * i + 1]);
            Yr[i] = pmul(d, Xr[i]);
            Yi[i] = pmul(d, Xi[i]);
        }
    }
    // off-diagonal k = (i, j), i = 1..5, j < i, row by row; four at a time
    const float2 m1 = make_float2(-1.f, -1.f);
    float o[16];
    int k = 0;
#pragma unroll
    for (int i = 1; i < 6; ++i)
#pragma unroll
        for (int j = 0; j < i; ++j) {
            if ((k & 3) == 0) cols.get<16>(160 + 4 * k, o);
            const int kk = k & 3;
            const float2 orr = make_float2(o[4 * kk], o[4 * kk + 1]), oi = make_float2(o[4 * kk + 2], o[4 * kk + 3]);
            const float2 noi = pmul(oi, m1);  // -im, exact
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

// ---- staging of a site block ----------------------------------------------
// The raw words of a site block as global memory holds them: 12 stored link
// reals per direction (3 float4: forward links at the site, backward ones at
// the neighbour) and the 18 clover float4 of the site, copied by cp.async,
// which holds no register while the copy is in flight.
constexpr int MR_RL = 8 * 3 * SB;  // float4 [d][k][site]
constexpr int MR_RC = 18 * SB;     // float4 [q][site]

__device__ __forceinline__ void cp16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// issue the copies of the block starting at site cb0, and write its
// neighbour indices and time-boundary flags
template <bool CLOVER>
__device__ __forceinline__ void mrhs_prefetch(const StencilArgs &A, int cb0, float4 *raw_l, float4 *raw_c, int *s_nb,
                                              int *s_tf, int tid, int nthr)
{
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int k = tid; k < 8 * SB; k += nthr) {
        const int l = k & (SB - 1), d = k >> 5, mu = d >> 1, cb = cb0 + l;
        const bool fwd = (d & 1) == 0;
        int nb = 0, tf = 0;
        if (cb < A.g.Vh) {
            int c[4];
            site_coords(A.g, A.out_par, cb, c);
            nb = lex_hop(A.g, lex_of(A.g, c), c, mu, fwd ? +1 : -1) >> 1;
            tf = (c[3] == A.g.L[3] - 1 ? 1 : 0) | (c[3] == 0 ? 2 : 0);
            const float4 *p = (const float4 *)A.U.a[fwd ? A.out_par : 1 - A.out_par];
            const int ls = fwd ? cb : nb;
#pragma unroll
            for (int kk = 0; kk < 3; ++kk) cp16(raw_l + (d * 3 + kk) * SB + l, p + soa(ls, 12, mu * 3 + kk));
        } else {
#pragma unroll
            for (int kk = 0; kk < 3; ++kk) raw_l[(d * 3 + kk) * SB + l] = z;
        }
        s_nb[d * SB + l] = nb;
        if (d == 0) s_tf[l] = tf;
    }
    if (CLOVER) {
        const float4 *Cl = (const float4 *)A.C.p[A.out_par];
        for (int k = tid; k < 18 * SB; k += nthr) {
            const int l = k & (SB - 1), q = k >> 5;
            if (cb0 + l < A.g.Vh) cp16(raw_c + q * SB + l, Cl + soa(cb0 + l, 18, q));
            else raw_c[q * SB + l] = z;
        }
    }
    cp_commit();
}

// the raw words to the staged layout: links rebuilt to 18 reals, the two
// clover blocks in lane pairs, times 1/2
template <bool CLOVER>
__device__ __forceinline__ void mrhs_unpack(const float4 *raw_l, const float4 *raw_c, float4 *s_col, int tid, int nthr)
{
    for (int k = tid; k < 8 * SB; k += nthr) {
        const int l = k & (SB - 1), d = k >> 5;
        Link<float> U;
        Prec<QCD_F32>::unpack_link(raw_l[(d * 3) * SB + l], raw_l[(d * 3 + 1) * SB + l], raw_l[(d * 3 + 2) * SB + l], U);
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            const cx<float> a = U.u[(2 * g) / 3][(2 * g) % 3], b = U.u[(2 * g + 1) / 3][(2 * g + 1) % 3];
            s_col[(4 * d + g) * SB + l] = make_float4(a.r, a.i, b.r, b.i);
        }
        ((float2 *)s_col)[((32 + (d >> 1)) * SB + l) * 2 + (d & 1)] = make_float2(U.u[2][2].r, U.u[2][2].i);
    }
    if (CLOVER) {
        float *cf = (float *)s_col;
        auto at = [&](int col, int l) -> float & { return cf[((col >> 2) * SB + l) * 4 + (col & 3)]; };
        for (int k = tid; k < 9 * SB; k += nthr) {
            // float4 q4 of block 0 and of block 1: reals 4 q4 .. 4 q4 + 3 of
            // each (d[0..5], then o[q] as (re, im) from real 6)
            const int l = k & (SB - 1), q4 = k >> 5;
            const float4 f0 = raw_c[q4 * SB + l], f1 = raw_c[(q4 + 9) * SB + l];
            const float a4[4] = {f0.x, f0.y, f0.z, f0.w}, b4[4] = {f1.x, f1.y, f1.z, f1.w};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int r = 4 * q4 + t;
                const float pp = 0.5f * a4[t], mm = 0.5f * b4[t];
                if (r < 6) {
                    at(144 + 2 * r, l) = pp;
                    at(145 + 2 * r, l) = mm;
                } else {
                    const int o = (r - 6) >> 1, im = (r - 6) & 1;
                    at(160 + 4 * o + 2 * im, l) = pp;
                    at(161 + 4 * o + 2 * im, l) = mm;
                }
            }
        }
    }
}

// the stencil of (site cb0 + lane, right-hand side r) from the staged words
template <int MODE, bool DAG>
__device__ __forceinline__ void mrhs_compute(const StencilArgs &A, const Cols &cols, const int *s_nb,
                                             const int *s_tf, int cb0, int lane, int r)
{
    const int cb = cb0 + lane;
    // every thread takes part in the block's barriers: a thread past the
    // lattice or the last right-hand side computes on a valid site and
    // right-hand side and stores nothing
    const bool valid = cb < A.g.Vh && r < A.nrhs;
    const int rr = r < A.nrhs ? r : 0;
    const SpinorPtr in = rhs_ptr(A.in, rr, A.rhs_stride, A.norm_stride);
    const SpinorPtr out = rhs_ptr(A.out, rr, A.rhs_stride, A.norm_stride);
    const int tflag = s_tf[lane];
    PairAcc P;
#pragma unroll
    for (int c = 0; c < 3; ++c) P.Ur[c] = P.Ui[c] = P.Lr[c] = P.Li[c] = make_float2(0.f, 0.f);
    constexpr int SF = DAG ? -1 : 1;
    hop_dir_mrhs<0, SF>(in, cols, s_nb, lane, tflag, A.g.t_bc, P);
    hop_dir_mrhs<1, SF>(in, cols, s_nb, lane, tflag, A.g.t_bc, P);
    hop_dir_mrhs<2, SF>(in, cols, s_nb, lane, tflag, A.g.t_bc, P);
    hop_dir_mrhs<3, SF>(in, cols, s_nb, lane, tflag, A.g.t_bc, P);
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
        herm6_pair(cols, Xr, Xi, Yr, Yi);
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
}

// A block stays resident and takes the site blocks blockIdx.x, + gridDim.x,
// ... (the blocks running at one time cover consecutive site blocks, whose
// neighbours they share in L2); it copies the next site block's raw words
// while it computes the current one, so only the on-chip unpack lies between
// two site blocks.
template <int MODE, bool DAG>
__device__ __forceinline__ void mrhs_body(const StencilArgs &A)
{
    constexpr bool CL = MODE == M_MULT;
    extern __shared__ float4 sm[];
    float4 *s_col = sm;
    float4 *raw_l = s_col + MR_GRP * SB;
    float4 *raw_c = raw_l + MR_RL;
    int *s_nb = (int *)(raw_c + MR_RC);  // [2][8 SB]
    int *s_tf = s_nb + 2 * MR_NB;        // [2][SB]
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int nthr = blockDim.x * blockDim.y;
    const int nsb = (A.g.Vh + SB - 1) / SB;
    const int r = blockIdx.y * blockDim.y + threadIdx.y;
    if (A.done) {  // a lockstep solve: nothing to do once every right-hand side of the tile has converged
        bool all = true;
        for (int k = 0; k < (int)blockDim.y; ++k) {
            const int rr = blockIdx.y * blockDim.y + k;
            if (rr < A.nrhs && !A.done[(size_t)rr * A.done_stride]) all = false;
        }
        if (all) return;  // the same decision in every thread: no barrier is left waiting
    }
    int sb = blockIdx.x, buf = 0;
    if (sb < nsb) mrhs_prefetch<CL>(A, sb * SB, raw_l, raw_c, s_nb, s_tf, tid, nthr);
    cp_wait_all();
    __syncthreads();
    const Cols cols{s_col, (int)threadIdx.x};
    while (sb < nsb) {
        mrhs_unpack<CL>(raw_l, raw_c, s_col, tid, nthr);
        __syncthreads();
        const int nx = sb + gridDim.x;
        if (nx < nsb) mrhs_prefetch<CL>(A, nx * SB, raw_l, raw_c, s_nb + (buf ^ 1) * MR_NB, s_tf + (buf ^ 1) * SB, tid, nthr);
        mrhs_compute<MODE, DAG>(A, cols, s_nb + buf * MR_NB, s_tf + buf * SB, sb * SB, threadIdx.x, r);
        cp_wait_all();
        __syncthreads();
        sb = nx;
        buf ^= 1;
    }
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

// resident blocks per SM of a kernel at a block size (cached per tile)
template <auto K>
static int resident(int threads, size_t smem)
{
    static std::atomic<int> occ[17];
    const int t = threads / SB;
    int n = t <= 16 ? occ[t].load(std::memory_order_relaxed) : 0;
    if (n <= 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, K, threads, smem) != cudaSuccess || n < 1) n = 1;
        if (t <= 16) occ[t].store(n, std::memory_order_relaxed);
    }
    return n;
}

// tile: right-hand sides per block (the links and clover of a 32-site block
// are staged once per tile; the autotuner picks the tile); variant 1 with
// the 80-register cap.  One wave of resident blocks walks the site blocks.
int launch_mrhs(const StencilCall &sc, const StencilArgs &A, int nrhs, cudaStream_t s, int variant, int tile,
                int num_sms)
{
    if (tile < 1 || tile > nrhs) tile = nrhs;
    const int nsb = (int)nblocks(A.g.Vh, SB), gy = (nrhs + tile - 1) / tile;
    const size_t smem = MR_BYTES;
#define QCD_MR_K(KERN, MODE, DAG)                                                                      \
    do {                                                                                               \
        smem_opt_in<KERN<MODE, DAG>>(smem);                                                            \
        int gx = resident<KERN<MODE, DAG>>(SB * tile, smem) * num_sms / gy;                            \
        gx = gx < 1 ? 1 : gx > nsb ? nsb : gx;                                                         \
        KERN<MODE, DAG><<<dim3(gx, gy), dim3(SB, tile), smem, s>>>(A);                                 \
    } while (0)
#define QCD_MR(MODE, DAG)                                                                              \
    do {                                                                                               \
        if (variant == 1) QCD_MR_K(mrhs_kernel_r80, MODE, DAG);                                        \
        else QCD_MR_K(mrhs_kernel, MODE, DAG);                                                         \
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
