// Multi-right-hand-side FP32 MULT and hopping term (Eq. 4) with shared-memory
// staging of the links, neighbour indices and clover blocks of each 32-site
// block, for all right-hand sides of a tile.
#include "stencil.cuh"

namespace qcd {

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
int launch_mrhs(const StencilCall &sc, const StencilArgs &A, int nrhs, cudaStream_t s, int variant, int tile)
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

}  // namespace qcd
