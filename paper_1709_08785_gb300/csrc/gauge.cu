// Gauge-field ingest (the conversion [U, F] -> [U^SP, F^SP] of Alg. 1) and
// the clover term: F(n) = 1 - (csw kappa/2) sum_{mu!=nu} sigma_munu F_munu(n)
// with F_munu = (Q_munu - Q_munu^dag)/(8i) from the four plaquette leaves,
// built and inverted site by site in FP64 (Sec. II-B: "inverted easily"),
// stored as two 6x6 Hermitian blocks (Sec. III-A).
//
// Chiral blocks.  In the Dirac basis used here sigma_jk = -eps_jkl
// diag(s_l, s_l) and sigma_k4 = [[0, -s_k], [-s_k, 0]].  Both commute with
// gamma5; on chi_+ = (psi_up - psi_dn)/sqrt2 and chi_- = (psi_up + psi_dn)/sqrt2
// they act as sigma_jk -> -eps_jkl s_l and sigma_k4 -> +-s_k.  Hence
//   A_+- = 1 + csw kappa sum_l s_l (x) (B_l -+ E_l),
//   B_1 = F_yz, B_2 = F_zx, B_3 = F_xy, E_k = F_kt,
// each a 6x6 Hermitian matrix indexed 3*spin + colour.
#include "ctx.cuh"

namespace qcd {

// ---------------------------------------------------------------- links
__device__ __forceinline__ float4 df_pair(double2 z)
{
    const df r(z.x), i(z.y);
    return make_float4(r.hi, r.lo, i.hi, i.lo);
}

__global__ void k_gauge_convert(Geom g, const double2 *__restrict__ U, double2 *U64e, double2 *U64o, float4 *U32e,
                                float4 *U32o, uint4 *U16ae, uint4 *U16ao, uint2 *U16be, uint2 *U16bo, float4 *UDFe,
                                float4 *UDFo)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    int c[4], t = s;
    for (int mu = 0; mu < 4; ++mu) {
        c[mu] = t % g.L[mu];
        t /= g.L[mu];
    }
    const int par = (c[0] + c[1] + c[2] + c[3]) & 1;
    const int cb = s >> 1;
    double2 *u64 = par ? U64o : U64e;
    float4 *u32 = par ? U32o : U32e;
    uint4 *u16a = par ? U16ao : U16ae;
    uint2 *u16b = par ? U16bo : U16be;
    for (int mu = 0; mu < 4; ++mu) {
        double2 m[9];
        for (int k = 0; k < 9; ++k) m[k] = U[((size_t)s * 4 + mu) * 9 + k];
        for (int k = 0; k < 9; ++k) u64[soa(cb, 36, mu * 9 + k)] = m[k];
        float4 *udf = par ? UDFo : UDFe;
        for (int k = 0; k < 9; ++k) udf[soa(cb, 36, mu * 9 + k)] = df_pair(m[k]);
        // first two columns: a = (m00, m10, m20), b = (m01, m11, m21)
        const double2 a0 = m[0], a1 = m[3], a2 = m[6], b0 = m[1], b1 = m[4], b2 = m[7];
        u32[soa(cb, 12, mu * 3 + 0)] = make_float4(a0.x, a0.y, a1.x, a1.y);
        u32[soa(cb, 12, mu * 3 + 1)] = make_float4(a2.x, a2.y, b0.x, b0.y);
        u32[soa(cb, 12, mu * 3 + 2)] = make_float4(b1.x, b1.y, b2.x, b2.y);
        auto hh = [](double2 z) { return h2u(__floats2half2_rn((float)z.x, (float)z.y)); };
        u16a[soa(cb, 4, mu)] = make_uint4(hh(a0), hh(a1), hh(a2), hh(b0));
        u16b[soa(cb, 4, mu)] = make_uint2(hh(b1), hh(b2));
    }
}

int gauge_convert(qcd_ctx *c, const void *U_dev)
{
    k_gauge_convert<<<nblocks(c->g.V, 256), 256, 0, c->stream>>>(
        c->g, (const double2 *)U_dev, (double2 *)c->U64[0], (double2 *)c->U64[1], (float4 *)c->U32[0],
        (float4 *)c->U32[1], (uint4 *)c->U16a[0], (uint4 *)c->U16a[1], (uint2 *)c->U16b[0], (uint2 *)c->U16b[1],
        (float4 *)c->UDF[0], (float4 *)c->UDF[1]);
    QCD_CUDA_CHECK(cudaGetLastError());
    return QCD_OK;
}

// ---------------------------------------------------------------- clover
struct M3 {
    cx<double> m[3][3];
};

__device__ __forceinline__ M3 mul(const M3 &a, const M3 &b)
{
    M3 c;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            cx<double> s = mk(0.0, 0.0);
#pragma unroll
            for (int k = 0; k < 3; ++k) fma_(s, a.m[i][k], b.m[k][j]);
            c.m[i][j] = s;
        }
    return c;
}

__device__ __forceinline__ M3 dag(const M3 &a)
{
    M3 c;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) c.m[i][j] = conj(a.m[j][i]);
    return c;
}

// link U_mu at lexicographic site s
__device__ __forceinline__ M3 link_at(const Geom &g, const GaugePtr &U, int s, int mu)
{
    int c[4], t = s;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        c[k] = t % g.L[k];
        t /= g.L[k];
    }
    const int par = (c[0] + c[1] + c[2] + c[3]) & 1;
    Link<double> L;
    Prec<QCD_F64>::load_link(U, par, s >> 1, mu, L);
    M3 m;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) m.m[i][j] = L.u[i][j];
    return m;
}

// lexicographic site s + dm*mu + dn*nu
__device__ __forceinline__ int shift2(const Geom &g, const int c[4], int mu, int dm, int nu, int dn)
{
    int d[4] = {c[0], c[1], c[2], c[3]};
    d[mu] = (d[mu] + dm + g.L[mu]) % g.L[mu];
    d[nu] = (d[nu] + dn + g.L[nu]) % g.L[nu];
    return lex_of(g, d);
}

// F_munu(n) = (Q - Q^dag)/(8i), Q = sum of the four counter-clockwise leaves
// at n in the (mu, nu) plane.
__device__ M3 field_strength(const Geom &g, const GaugePtr &U, const int c[4], int mu, int nu)
{
    const int n = lex_of(g, c);
    const int n_pm = shift2(g, c, mu, 1, nu, 0), n_pn = shift2(g, c, mu, 0, nu, 1);
    const int n_mm = shift2(g, c, mu, -1, nu, 0), n_mn = shift2(g, c, mu, 0, nu, -1);
    const int n_mm_pn = shift2(g, c, mu, -1, nu, 1), n_pm_mn = shift2(g, c, mu, 1, nu, -1);
    const int n_mm_mn = shift2(g, c, mu, -1, nu, -1);
    M3 Q;
    // U_mu(n) U_nu(n+mu) U_mu(n+nu)^dag U_nu(n)^dag
    M3 t = mul(mul(link_at(g, U, n, mu), link_at(g, U, n_pm, nu)), mul(dag(link_at(g, U, n_pn, mu)), dag(link_at(g, U, n, nu))));
    Q = t;
    // U_nu(n) U_mu(n-mu+nu)^dag U_nu(n-mu)^dag U_mu(n-mu)
    t = mul(mul(link_at(g, U, n, nu), dag(link_at(g, U, n_mm_pn, mu))), mul(dag(link_at(g, U, n_mm, nu)), link_at(g, U, n_mm, mu)));
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Q.m[i][j] = Q.m[i][j] + t.m[i][j];
    // U_mu(n-mu)^dag U_nu(n-mu-nu)^dag U_mu(n-mu-nu) U_nu(n-nu)
    t = mul(mul(dag(link_at(g, U, n_mm, mu)), dag(link_at(g, U, n_mm_mn, nu))), mul(link_at(g, U, n_mm_mn, mu), link_at(g, U, n_mn, nu)));
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Q.m[i][j] = Q.m[i][j] + t.m[i][j];
    // U_nu(n-nu)^dag U_mu(n-nu) U_nu(n+mu-nu) U_mu(n)^dag
    t = mul(mul(dag(link_at(g, U, n_mn, nu)), link_at(g, U, n_mn, mu)), mul(link_at(g, U, n_pm_mn, nu), dag(link_at(g, U, n, mu))));
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) Q.m[i][j] = Q.m[i][j] + t.m[i][j];
    M3 F;
    // (Q - Q^dag)/(8i) = -i (Q - Q^dag)/8
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) F.m[i][j] = 0.125 * tmi(Q.m[i][j] - conj(Q.m[j][i]));
    return F;
}

// A += coef * (s_l (x) G), 6x6 indexed 3*spin + colour
__device__ __forceinline__ void add_kron(cx<double> A[6][6], double coef, int l, const M3 &G)
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            const cx<double> gv = coef * G.m[i][j];
            if (l == 1) {  // s_1 = [[0,1],[1,0]]
                A[i][3 + j] = A[i][3 + j] + gv;
                A[3 + i][j] = A[3 + i][j] + gv;
            } else if (l == 2) {  // s_2 = [[0,-i],[i,0]]
                A[i][3 + j] = A[i][3 + j] + tmi(gv);
                A[3 + i][j] = A[3 + i][j] + ti(gv);
            } else {  // s_3 = diag(1,-1)
                A[i][j] = A[i][j] + gv;
                A[3 + i][3 + j] = A[3 + i][3 + j] - gv;
            }
        }
}

// Hermitian 6x6 inverse by A = L D L^dag (no pivoting; the clover blocks
// are close to the identity).  Returns false on a (near-)zero pivot.
__device__ bool herm_inverse6(const cx<double> A[6][6], cx<double> Ai[6][6])
{
    cx<double> L[6][6];
    double D[6];
    double amax = 0.0;
    for (int i = 0; i < 6; ++i) amax = fmax(amax, fabs(A[i][i].r));
    for (int j = 0; j < 6; ++j) {
        double dj = A[j][j].r;
        for (int k = 0; k < j; ++k) dj -= (L[j][k].r * L[j][k].r + L[j][k].i * L[j][k].i) * D[k];
        if (!(fabs(dj) > 1e-12 * amax) || !isfinite(dj)) return false;
        D[j] = dj;
        L[j][j] = mk(1.0, 0.0);
        for (int i = j + 1; i < 6; ++i) {
            cx<double> s = A[i][j];
            for (int k = 0; k < j; ++k) {
                const cx<double> t = D[k] * L[i][k];
                s = s - t * conj(L[j][k]);
            }
            L[i][j] = (1.0 / dj) * s;
        }
        for (int i = 0; i < j; ++i) L[i][j] = mk(0.0, 0.0);
    }
    // M = L^-1 (unit lower triangular)
    cx<double> M[6][6];
    for (int j = 0; j < 6; ++j) {
        for (int i = 0; i < 6; ++i) M[i][j] = mk(i == j ? 1.0 : 0.0, 0.0);
        for (int i = j + 1; i < 6; ++i) {
            cx<double> s = mk(0.0, 0.0);
            for (int k = j; k < i; ++k) fma_(s, L[i][k], M[k][j]);
            M[i][j] = -s;
        }
    }
    // A^-1 = M^dag D^-1 M
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j <= i; ++j) {
            cx<double> s = mk(0.0, 0.0);
            for (int k = i; k < 6; ++k) {
                const cx<double> t = (1.0 / D[k]) * M[k][j];
                fmac_(s, M[k][i], t);
            }
            Ai[i][j] = s;
            Ai[j][i] = conj(s);
        }
    return true;
}

// store one block (diag reals then the lower triangle) in all precisions
__device__ void store_block(const cx<double> A[6][6], int blk, int cb, double2 *p64, float4 *p32, uint4 *p16,
                            float4 *pdf)
{
    double r[36];
    for (int i = 0; i < 6; ++i) r[i] = A[i][i].r;
    int k = 0;
    for (int i = 1; i < 6; ++i)
        for (int j = 0; j < i; ++j) {
            r[6 + 2 * k] = A[i][j].r;
            r[7 + 2 * k] = A[i][j].i;
            ++k;
        }
    for (int q = 0; q < 18; ++q) p64[soa(cb, 36, blk * 18 + q)] = make_double2(r[2 * q], r[2 * q + 1]);
    for (int q = 0; q < 18; ++q) pdf[soa(cb, 36, blk * 18 + q)] = df_pair(make_double2(r[2 * q], r[2 * q + 1]));
    for (int q = 0; q < 9; ++q)
        p32[soa(cb, 18, blk * 9 + q)] = make_float4((float)r[4 * q], (float)r[4 * q + 1], (float)r[4 * q + 2], (float)r[4 * q + 3]);
    // halves: element e of the site = blk*36 + j; uint4 q holds elements 8q..8q+7
    __half *h = reinterpret_cast<__half *>(p16);
    for (int j = 0; j < 36; ++j) {
        const int e = blk * 36 + j;
        const int q = e >> 3, w = e & 7;
        h[soa(cb, 9, q) * 8 + w] = __double2half(r[j]);
    }
}

__global__ void k_clover_build(Geom g, GaugePtr U, int par, double ck, double2 *F64, float4 *F32, uint4 *F16,
                               float4 *FDF, double2 *Fi64, float4 *Fi32, uint4 *Fi16, float4 *FiDF, int *bad)
{
    const int cb = blockIdx.x * blockDim.x + threadIdx.x;
    if (cb >= g.Vh) return;
    int c[4];
    site_coords(g, par, cb, c);
    for (int blk = 0; blk < 2; ++blk) {
        // blk 0: A_+ (gamma5 = +1), blk 1: A_-
        const double se = blk == 0 ? -1.0 : 1.0;  // sign of E_l in B_l -+ E_l
        cx<double> A[6][6];
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 6; ++j) A[i][j] = mk(i == j ? 1.0 : 0.0, 0.0);
        add_kron(A, ck, 3, field_strength(g, U, c, 0, 1));   // B_3 = F_xy
        add_kron(A, -ck, 2, field_strength(g, U, c, 0, 2));  // B_2 = F_zx = -F_xz
        add_kron(A, ck, 1, field_strength(g, U, c, 1, 2));   // B_1 = F_yz
        add_kron(A, se * ck, 1, field_strength(g, U, c, 0, 3));  // E_1 = F_xt
        add_kron(A, se * ck, 2, field_strength(g, U, c, 1, 3));  // E_2 = F_yt
        add_kron(A, se * ck, 3, field_strength(g, U, c, 2, 3));  // E_3 = F_zt
        // exact Hermiticity
        for (int i = 0; i < 6; ++i) {
            A[i][i].i = 0.0;
            for (int j = 0; j < i; ++j) {
                const cx<double> m = 0.5 * (A[i][j] + conj(A[j][i]));
                A[i][j] = m;
                A[j][i] = conj(m);
            }
        }
        store_block(A, blk, cb, F64, F32, F16, FDF);
        cx<double> Ai[6][6];
        if (!herm_inverse6(A, Ai)) {
            atomicExch(bad, 1);
            for (int i = 0; i < 6; ++i)
                for (int j = 0; j < 6; ++j) Ai[i][j] = mk(0.0, 0.0);
        }
        store_block(Ai, blk, cb, Fi64, Fi32, Fi16, FiDF);
    }
}

int clover_build(qcd_ctx *c, double kappa, double csw)
{
    GaugePtr U;
    for (int p = 0; p < 2; ++p) {
        U.a[p] = c->U64[p];
        U.b[p] = nullptr;
    }
    QCD_CUDA_CHECK(cudaMemsetAsync(c->flag_dev, 0, sizeof(int), c->stream));
    for (int par = 0; par < 2; ++par) {
        k_clover_build<<<nblocks(c->g.Vh, 64), 64, 0, c->stream>>>(
            c->g, U, par, csw * kappa, (double2 *)c->C[QCD_F64][par], (float4 *)c->C[QCD_F32][par],
            (uint4 *)c->C[QCD_F16][par], (float4 *)c->C[QCD_DF64][par], (double2 *)c->Ci[QCD_F64][par],
            (float4 *)c->Ci[QCD_F32][par], (uint4 *)c->Ci[QCD_F16][par], (float4 *)c->Ci[QCD_DF64][par],
            c->flag_dev);
        QCD_CUDA_CHECK(cudaGetLastError());
    }
    int bad = 0;
    QCD_CUDA_CHECK(cudaMemcpyAsync(&bad, c->flag_dev, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    QCD_CUDA_CHECK(cudaStreamSynchronize(c->stream));
    if (bad) {
        set_error_message("clover block with a zero pivot (kappa=%g, csw=%g)", kappa, csw);
        return QCD_ECLOVER_SINGULAR;
    }
    return QCD_OK;
}

}  // namespace qcd
