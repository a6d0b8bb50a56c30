// Adjoint pieces: lambda = D^-dag g through gamma5-hermiticity
// (D^dag = gamma5 D gamma5, so D^-dag = gamma5 D^-1 gamma5), and the link
// gradient ("force") of f(U) = -Re<lambda, D[U] x> for fixed x, lambda, in the
// convention G = df/dRe U + i df/dIm U.  With x = D^-1 b and lambda = D^-dag g,
// -Re<lambda, dD x> is the change of Re<g, x>, so G is the gradient of a loss
// whose gradient with respect to x is g.
//
// Hopping part (Eq. 4): U_mu(m) enters (1 - g_mu) U_mu(m) x(m+mu) at m and
// (1 + g_mu) U_mu(m)^dag x(m) at m+mu; with bc the boundary phase,
//   G_mu(m) += kappa bc [ sum_s ((1-g_mu) lambda(m))_s (x) conj(x_s(m+mu))
//                       + sum_s x_s(m) (x) conj(((1+g_mu) lambda(m+mu))_s) ].
// Clover part: f_clov = csw kappa Re sum_n sum_{mu<nu} Tr(S^T F_munu), with
// S_ij = sum_ab conj(lambda_ai) sigma_munu,ab x_bj; since F = (Q - Q^dag)/(8i),
// this is Re sum Tr(Y Q) with Y = csw kappa (S^T + conj(S))/(8i).  Every
// plaquette of Q enters at its four corners, so the derivative with respect
// to one link collects the two plaquettes of each plane through it with Y
// inserted at each corner (a staple with insertions).
#include "blas.cuh"

namespace qcd {

namespace {

using C = cx<double>;

struct M3 {
    C m[3][3];
};

__device__ __forceinline__ M3 zero3()
{
    M3 r;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) r.m[i][j] = mk(0.0, 0.0);
    return r;
}

__device__ __forceinline__ M3 mul(const M3 &a, const M3 &b)
{
    M3 c;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            C s = mk(0.0, 0.0);
            for (int k = 0; k < 3; ++k) fma_(s, a.m[i][k], b.m[k][j]);
            c.m[i][j] = s;
        }
    return c;
}

__device__ __forceinline__ M3 dagm(const M3 &a)
{
    M3 c;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) c.m[i][j] = conj(a.m[j][i]);
    return c;
}

__device__ __forceinline__ void addm(M3 &a, const M3 &b)
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) a.m[i][j] = a.m[i][j] + b.m[i][j];
}

// canonical links [V][4][3][3] complex128
__device__ __forceinline__ M3 link(const double2 *U, int s, int mu)
{
    M3 r;
    const double2 *p = U + ((size_t)s * 4 + mu) * 9;
    for (int k = 0; k < 9; ++k) r.m[k / 3][k % 3] = mk(p[k].x, p[k].y);
    return r;
}

__device__ __forceinline__ int site_shift(const Geom &g, int s, int mu, int d)
{
    int c[4], t = s;
    for (int k = 0; k < 4; ++k) {
        c[k] = t % g.L[k];
        t /= g.L[k];
    }
    c[mu] = (c[mu] + d + g.L[mu]) % g.L[mu];
    return lex_of(g, c);
}

__device__ __forceinline__ void load_spinor(const double2 *v, int s, C out[4][3])
{
    const double2 *p = v + (size_t)s * 12;
    for (int k = 0; k < 12; ++k) out[k / 3][k % 3] = mk(p[k].x, p[k].y);
}

// (1 - sg * gamma_mu) v in the Dirac basis
__device__ void one_minus_gamma(const C v[4][3], int mu, int sg, C o[4][3])
{
    for (int i = 0; i < 3; ++i) {
        C g0, g1, g2, g3;  // gamma_mu v
        if (mu == 0) {
            g0 = tmi(v[3][i]); g1 = tmi(v[2][i]); g2 = ti(v[1][i]); g3 = ti(v[0][i]);
        } else if (mu == 1) {
            g0 = -v[3][i]; g1 = v[2][i]; g2 = v[1][i]; g3 = -v[0][i];
        } else if (mu == 2) {
            g0 = tmi(v[2][i]); g1 = ti(v[3][i]); g2 = ti(v[0][i]); g3 = tmi(v[1][i]);
        } else {
            g0 = v[0][i]; g1 = v[1][i]; g2 = -v[2][i]; g3 = -v[3][i];
        }
        const double s = (double)sg;
        o[0][i] = v[0][i] - s * g0;
        o[1][i] = v[1][i] - s * g1;
        o[2][i] = v[2][i] - s * g2;
        o[3][i] = v[3][i] - s * g3;
    }
}

// sigma_munu for the six planes (mu < nu) in the order (x,y) (x,z) (x,t)
// (y,z) (y,t) (z,t): each row has one non-zero entry, a phase:
// (sigma v)_a = phase[a] * v[perm[a]].  Worked out from
// sigma_jk = -eps_jkl diag(s_l, s_l) and sigma_k4 = [[0, -s_k], [-s_k, 0]].
__constant__ int c_sig_perm[6][4] = {
    {0, 1, 2, 3}, {1, 0, 3, 2}, {3, 2, 1, 0}, {1, 0, 3, 2}, {3, 2, 1, 0}, {2, 3, 0, 1}};
// phases as (re, im)
__constant__ double c_sig_ph[6][4][2] = {
    {{-1, 0}, {1, 0}, {-1, 0}, {1, 0}},     // sigma_xy = -diag(s3, s3)
    {{0, -1}, {0, 1}, {0, -1}, {0, 1}},     // sigma_xz = +diag(s2, s2)
    {{-1, 0}, {-1, 0}, {-1, 0}, {-1, 0}},   // sigma_xt = [[0,-s1],[-s1,0]]
    {{-1, 0}, {-1, 0}, {-1, 0}, {-1, 0}},   // sigma_yz = -diag(s1, s1)
    {{0, 1}, {0, -1}, {0, 1}, {0, -1}},     // sigma_yt = [[0,-s2],[-s2,0]]
    {{-1, 0}, {1, 0}, {-1, 0}, {1, 0}}};    // sigma_zt = [[0,-s3],[-s3,0]]

__device__ __forceinline__ int plane_index(int mu, int nu)
{
    // mu < nu
    return mu == 0 ? nu - 1 : (mu == 1 ? nu + 1 : 5);
}

// Y_p(n) = csw kappa (S^T + conj(S)) / (8i) for the six planes
__global__ void k_force_Y(Geom g, const double2 *__restrict__ x, const double2 *__restrict__ lam, double ck, double2 *Y)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    C X[4][3], L[4][3];
    load_spinor(x, s, X);
    load_spinor(lam, s, L);
    for (int p = 0; p < 6; ++p) {
        C S[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                C acc = mk(0.0, 0.0);
                for (int a = 0; a < 4; ++a) {
                    const C ph = mk(c_sig_ph[p][a][0], c_sig_ph[p][a][1]);
                    const C sx = ph * X[c_sig_perm[p][a]][j];
                    fmac_(acc, L[a][i], sx);  // conj(lambda_ai) (sigma x)_aj
                }
                S[i][j] = acc;
            }
        double2 *out = Y + ((size_t)s * 6 + p) * 9;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                const C t = S[j][i] + conj(S[i][j]);
                const C y = (ck * 0.125) * tmi(t);  // t / (8i)
                out[i * 3 + j] = make_double2(y.r, y.i);
            }
    }
}

// Y of the ordered plane (mu, nu), mu != nu, at site s: for mu > nu the loop
// runs the other way round, which is the same as inserting Y_{nu mu}^dag.
__device__ __forceinline__ M3 Yeff(const double2 *Y, int s, int mu, int nu)
{
    M3 r;
    const bool fwd = mu < nu;
    const int p = fwd ? plane_index(mu, nu) : plane_index(nu, mu);
    const double2 *q = Y + ((size_t)s * 6 + p) * 9;
    for (int k = 0; k < 9; ++k) r.m[k / 3][k % 3] = mk(q[k].x, q[k].y);
    return fwd ? r : dagm(r);
}

__global__ void k_force_link(Geom g, const double2 *__restrict__ U, const double2 *__restrict__ x,
                             const double2 *__restrict__ lam, const double2 *__restrict__ Y, double kappa,
                             int with_clover, double2 *G)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= 4 * g.V) return;
    const int m = tid >> 2, mu = tid & 3;
    const int mp = site_shift(g, m, mu, +1);
    M3 Gm = zero3();
    // ---- hopping part
    {
        int c[4], t = m;
        for (int k = 0; k < 4; ++k) {
            c[k] = t % g.L[k];
            t /= g.L[k];
        }
        const double bc = (mu == 3 && c[3] == g.L[3] - 1) ? (double)g.t_bc : 1.0;
        C Lm[4][3], Xp[4][3], Xm[4][3], Lp[4][3], PL[4][3], QL[4][3];
        load_spinor(lam, m, Lm);
        load_spinor(x, mp, Xp);
        load_spinor(x, m, Xm);
        load_spinor(lam, mp, Lp);
        one_minus_gamma(Lm, mu, +1, PL);  // (1 - g_mu) lambda(m)
        one_minus_gamma(Lp, mu, -1, QL);  // (1 + g_mu) lambda(m+mu)
        const double f = kappa * bc;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                C acc = mk(0.0, 0.0);
                for (int s = 0; s < 4; ++s) {
                    fmac_(acc, Xp[s][j], PL[s][i]);  // PL_si conj(Xp_sj)
                    fmac_(acc, QL[s][j], Xm[s][i]);  // Xm_si conj(QL_sj)
                }
                Gm.m[i][j] = f * acc;
            }
    }
    // ---- clover part: the two plaquettes of each plane (mu, nu) through U_mu(m)
    if (with_clover) {
        for (int nu = 0; nu < 4; ++nu) {
            if (nu == mu) continue;
            {  // above: corners m, m+mu, m+mu+nu, m+nu
                const int mn = site_shift(g, m, nu, +1);
                const int mpn = site_shift(g, mp, nu, +1);
                const M3 Unu_mp = link(U, mp, nu), Umu_mn_d = dagm(link(U, mn, mu)), Unu_m_d = dagm(link(U, m, nu));
                const M3 W = mul(Unu_mp, Umu_mn_d);  // U_nu(m+mu) U_mu(m+nu)^dag
                const M3 A = mul(W, Unu_m_d);
                M3 R = mul(A, Yeff(Y, m, mu, nu));
                addm(R, mul(Yeff(Y, mp, mu, nu), A));
                addm(R, mul(mul(Unu_mp, Yeff(Y, mpn, mu, nu)), mul(Umu_mn_d, Unu_m_d)));
                addm(R, mul(mul(W, Yeff(Y, mn, mu, nu)), Unu_m_d));
                addm(Gm, dagm(R));  // U_mu(m) enters undaggered: G += R^dag
            }
            {  // below: corners m-nu, m-nu+mu, m+mu, m
                const int q = site_shift(g, m, nu, -1);
                const int qp = site_shift(g, q, mu, +1);
                const M3 Unu_q_d = dagm(link(U, q, nu)), Umu_q = link(U, q, mu), Unu_qp = link(U, qp, nu);
                const M3 V = mul(Unu_q_d, Umu_q);  // U_nu(q)^dag U_mu(q)
                const M3 B = mul(V, Unu_qp);
                M3 R = mul(mul(Unu_q_d, Yeff(Y, q, mu, nu)), mul(Umu_q, Unu_qp));
                addm(R, mul(mul(V, Yeff(Y, qp, mu, nu)), Unu_qp));
                addm(R, mul(B, Yeff(Y, mp, mu, nu)));
                addm(R, mul(Yeff(Y, m, mu, nu), B));
                addm(Gm, R);  // U_mu(m) enters daggered: G += R
            }
        }
    }
    double2 *out = G + (size_t)tid * 9;
    for (int k = 0; k < 9; ++k) out[k] = make_double2(Gm.m[k / 3][k % 3].r, Gm.m[k / 3][k % 3].i);
}

// v -> gamma5 v on canonical full-lattice vectors, gamma5 = -[[0,1],[1,0]];
// in and out may be the same buffer (no __restrict__: each thread reads its
// site completely before writing it)
__global__ void k_gamma5(int V, const double2 *in, double2 *out)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
    const double2 *p = in + (size_t)s * 12;
    double2 v[12];
    for (int k = 0; k < 12; ++k) v[k] = p[k];
    double2 *o = out + (size_t)s * 12;
    for (int k = 0; k < 6; ++k) {
        o[k] = make_double2(-v[k + 6].x, -v[k + 6].y);
        o[k + 6] = make_double2(-v[k].x, -v[k].y);
    }
}

}  // namespace

int force(qcd_ctx *c, const void *x, const void *lam, void *G, const void *U_canon)
{
    const size_t ybytes = (size_t)c->g.V * 6 * 9 * 16;
    if (c->force_bytes < ybytes) {
        if (c->force_buf) {
            cudaStreamSynchronize(c->stream);
            cudaFree(c->force_buf);
            for (auto &p : c->pool)
                if (p == c->force_buf) p = nullptr;
            c->force_buf = nullptr;
            c->force_bytes = 0;
        }
        int rc = dev_alloc(c, &c->force_buf, ybytes);
        if (rc) return rc;
        c->force_bytes = ybytes;
    }
    {
        ProfScope prof(c, QCD_K_OTHER, 0.0);
        k_force_Y<<<nblocks(c->g.V, 128), 128, 0, c->stream>>>(c->g, (const double2 *)x, (const double2 *)lam,
                                                              c->csw * c->kappa, (double2 *)c->force_buf);
        QCD_CUDA_CHECK(cudaGetLastError());
    }
    {
        ProfScope prof(c, QCD_K_OTHER, 0.0);
        k_force_link<<<nblocks(4L * c->g.V, 64), 64, 0, c->stream>>>(
            c->g, (const double2 *)U_canon, (const double2 *)x, (const double2 *)lam, (const double2 *)c->force_buf,
            c->kappa, c->csw != 0.0, (double2 *)G);
        QCD_CUDA_CHECK(cudaGetLastError());
    }
    return QCD_OK;
}

int gamma5_full(qcd_ctx *c, const void *in, void *out)
{
    ProfScope prof(c, QCD_K_OTHER, 0.0);
    k_gamma5<<<nblocks(c->g.V, 128), 128, 0, c->stream>>>(c->g.V, (const double2 *)in, (double2 *)out);
    QCD_CUDA_CHECK(cudaGetLastError());
    return QCD_OK;
}

}  // namespace qcd
