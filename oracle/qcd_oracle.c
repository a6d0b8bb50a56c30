/*
 * qcd_oracle.c -- plain, slow FP64 CPU reference of the O(a)-improved (clover)
 * Wilson operator and of the BiCGStab iterations that solve D x = b.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA path is
 * checked against.  Only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark may load it; the product library never links it and shares
 * no code, header, table or helper with it.
 *
 * Everything is written from the definitions, with no blocking, fusion or
 * spin-projection tricks:
 *   - D = F - kappa*H                                   (Sec. II-A, Eq. 3)
 *   - H = sum_mu (1-g_mu) U_mu(n) d_{n+mu,m}
 *               + (1+g_mu) U_mu(m)^dag d_{n-mu,m}        (Sec. II-A, Eq. 4)
 *   - F = 1 - (csw*kappa/2) sum_{mu!=nu} sigma_munu (x) F_munu,
 *     F_munu = (Q_munu - Q_munu^dag)/(8i), Q = sum of the four plaquette
 *     leaves around n (the Sheikholeslami-Wohlert clover term the paper
 *     cites in Sec. II-A; the paper does not print it, this is the standard
 *     hopping-parameter normalisation).
 *   - even-odd Schur complement D^_ee = 1 - kappa^2 F_ee^-1 H_eo F_oo^-1 H_oe,
 *     b^_e and x_o                                      (Sec. II-B, Eqs. 5-9;
 *     the printed "H~_eo H~_eo" is read as H~_eo H~_oe, the only product the
 *     Schur complement of D allows)
 *   - the gamma5-hermitian even-odd operator S_ee = F_ee - kappa^2 H_eo
 *     F_oo^-1 H_oe (the Schur complement of D on the even sites, i.e.
 *     F_ee D^_ee) with its source b_e + kappa H_eo F_oo^-1 b_o
 *   - BiCGStab: Alg. 2, and the flexible nested form of Alg. 1, with
 *     alpha = rho0/<r~|q> and beta = (rho1/rho0)(alpha/omega) (the printed
 *     alpha = <r~|q> and beta = (rho1/rho0)/(alpha/omega) are read as the
 *     standard van der Vorst recurrences).
 *
 * Conventions (shared with the public C-ABI only through documentation):
 *   site  s = x + Lx*(y + Ly*(z + Lz*t)), mu = 0..3 for x, y, z, t
 *   link  U[s][mu][i][j]      complex, U_mu(n) is the link from n to n+mu
 *   spinor psi[s][alpha][i]   alpha = 0..3 spin, i = 0..2 colour
 *   half-lattice vectors are indexed by cb = s/2 within one parity,
 *   parity = (x+y+z+t) mod 2, 0 = even.
 *   Gamma matrices: Dirac basis, g_k = [[0,-i s_k],[i s_k,0]], g_t =
 *   diag(1,1,-1,-1) (g_t diagonal as Sec. II-A states), g5 = g1 g2 g3 g4.
 *   t_bc = +1 periodic, -1 antiperiodic in time: the hopping terms that
 *   cross the time boundary are multiplied by t_bc; the clover uses the
 *   unmodified links.
 *
 * parity pins: every function here is checked in the CPU test-suite against
 * closed forms, invariants and brute force (free-field plane waves, unit-link
 * and constant abelian clover fields, gamma5-hermiticity, gauge covariance,
 * a dense 2^4 matrix, dense LU solves, finite differences).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* The loops over sites of the operator applications are marked SITE_LOOP.
 * Built with -fopenmp (the multi-core timing build), they are split across
 * threads; every site's arithmetic and every reduction (the serial vector
 * dot products and norms) is unchanged, so both builds give the same bits.
 * Built without it, the pragma does nothing. */
#ifdef _OPENMP
#define SITE_LOOP _Pragma("omp parallel for schedule(static)")
#else
#define SITE_LOOP
#endif

/* threads the site loops use (1 without OpenMP) */
int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------ */
/* lattice geometry                                                    */
/* ------------------------------------------------------------------ */

static long vol(const int L[4]) { return (long)L[0] * L[1] * L[2] * L[3]; }

static long lex_of(const int L[4], const int c[4])
{
    return c[0] + (long)L[0] * (c[1] + (long)L[1] * (c[2] + (long)L[2] * c[3]));
}

static void coords_of(const int L[4], long s, int c[4])
{
    for (int mu = 0; mu < 4; ++mu) {
        c[mu] = (int)(s % L[mu]);
        s /= L[mu];
    }
}

/* site reached from s by the displacement d (periodic wrap) */
static long shifted(const int L[4], long s, const int d[4])
{
    int c[4];
    coords_of(L, s, c);
    for (int mu = 0; mu < 4; ++mu) {
        c[mu] = ((c[mu] + d[mu]) % L[mu] + L[mu]) % L[mu];
    }
    return lex_of(L, c);
}

static long step(const int L[4], long s, int mu, int sign)
{
    int d[4] = {0, 0, 0, 0};
    d[mu] = sign;
    return shifted(L, s, d);
}

static int parity_of(const int L[4], long s)
{
    int c[4];
    coords_of(L, s, c);
    return (c[0] + c[1] + c[2] + c[3]) & 1;
}

/* ------------------------------------------------------------------ */
/* Dirac algebra                                                       */
/* ------------------------------------------------------------------ */

/* g[mu] for mu = 0..3 (x,y,z,t) and g[4] = gamma5, Dirac basis. */
static void build_gammas(cplx g[5][4][4])
{
    const cplx im = _Complex_I;
    cplx pauli[3][2][2] = {
        {{0, 1}, {1, 0}},
        {{0, -im}, {im, 0}},
        {{1, 0}, {0, -1}},
    };
    memset(g, 0, sizeof(cplx) * 5 * 16);
    for (int k = 0; k < 3; ++k)
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                g[k][a][2 + b] = -im * pauli[k][a][b];
                g[k][2 + a][b] = im * pauli[k][a][b];
            }
    g[3][0][0] = g[3][1][1] = 1;
    g[3][2][2] = g[3][3][3] = -1;
    /* gamma5 = g1 g2 g3 g4 */
    cplx t1[4][4], t2[4][4];
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
            cplx acc = 0;
            for (int c = 0; c < 4; ++c) acc += g[0][a][c] * g[1][c][b];
            t1[a][b] = acc;
        }
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
            cplx acc = 0;
            for (int c = 0; c < 4; ++c) acc += t1[a][c] * g[2][c][b];
            t2[a][b] = acc;
        }
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
            cplx acc = 0;
            for (int c = 0; c < 4; ++c) acc += t2[a][c] * g[3][c][b];
            g[4][a][b] = acc;
        }
}

void oracle_gamma(int which, double *out /* complex [4][4] */)
{
    cplx g[5][4][4];
    build_gammas(g);
    memcpy(out, g[which], sizeof(cplx) * 16);
}

/* sigma_munu = (i/2)[g_mu, g_nu] */
static void build_sigma(cplx g[5][4][4], int mu, int nu, cplx s[4][4])
{
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
            cplx acc = 0;
            for (int c = 0; c < 4; ++c) acc += g[mu][a][c] * g[nu][c][b] - g[nu][a][c] * g[mu][c][b];
            s[a][b] = 0.5 * _Complex_I * acc;
        }
}

/* ------------------------------------------------------------------ */
/* 3x3 colour matrices                                                 */
/* ------------------------------------------------------------------ */

static void mat_load(const cplx *U, long s, int mu, int dag, cplx m[3][3])
{
    const cplx *u = U + (s * 4 + mu) * 9;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) m[i][j] = dag ? conj(u[j * 3 + i]) : u[i * 3 + j];
}

static void mat_mul(cplx a[3][3], cplx b[3][3], cplx c[3][3])
{
    cplx t[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            cplx acc = 0;
            for (int k = 0; k < 3; ++k) acc += a[i][k] * b[k][j];
            t[i][j] = acc;
        }
    memcpy(c, t, sizeof(t));
}

/* ------------------------------------------------------------------ */
/* the clover leaves                                                   */
/* ------------------------------------------------------------------ */

/* One factor of a leaf: the link U_dir(n + off), daggered or not. */
typedef struct { int off_mu, off_nu; int along_nu; int dag; } leaf_factor;

/* The four counter-clockwise plaquettes in the (mu,nu) plane that touch n,
 * each written as the ordered product of four links starting and ending at n.
 * Offsets are in units of (mu-hat, nu-hat).  along_nu selects U_nu instead
 * of U_mu.                                                               */
static const leaf_factor LEAVES[4][4] = {
    /* U_mu(n) U_nu(n+mu) U_mu(n+nu)^dag U_nu(n)^dag */
    {{0, 0, 0, 0}, {1, 0, 1, 0}, {0, 1, 0, 1}, {0, 0, 1, 1}},
    /* U_nu(n) U_mu(n-mu+nu)^dag U_nu(n-mu)^dag U_mu(n-mu) */
    {{0, 0, 1, 0}, {-1, 1, 0, 1}, {-1, 0, 1, 1}, {-1, 0, 0, 0}},
    /* U_mu(n-mu)^dag U_nu(n-mu-nu)^dag U_mu(n-mu-nu) U_nu(n-nu) */
    {{-1, 0, 0, 1}, {-1, -1, 1, 1}, {-1, -1, 0, 0}, {0, -1, 1, 0}},
    /* U_nu(n-nu)^dag U_mu(n-nu) U_nu(n+mu-nu) U_mu(n)^dag */
    {{0, -1, 1, 1}, {0, -1, 0, 0}, {1, -1, 1, 0}, {0, 0, 0, 1}},
};

static long leaf_site(const int L[4], long n, int mu, int nu, const leaf_factor *f)
{
    int d[4] = {0, 0, 0, 0};
    d[mu] += f->off_mu;
    d[nu] += f->off_nu;
    return shifted(L, n, d);
}

/* Q_munu(n) = sum of the four leaves */
static void clover_Q(const int L[4], const cplx *U, long n, int mu, int nu, cplx Q[3][3])
{
    memset(Q, 0, sizeof(cplx) * 9);
    for (int l = 0; l < 4; ++l) {
        cplx P[3][3], M[3][3];
        for (int k = 0; k < 4; ++k) {
            const leaf_factor *f = &LEAVES[l][k];
            long s = leaf_site(L, n, mu, nu, f);
            mat_load(U, s, f->along_nu ? nu : mu, f->dag, M);
            if (k == 0) memcpy(P, M, sizeof(M));
            else mat_mul(P, M, P);
        }
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) Q[i][j] += P[i][j];
    }
}

/* F_munu(n) = (Q - Q^dag)/(8i) */
static void field_strength(const int L[4], const cplx *U, long n, int mu, int nu, cplx Fmn[3][3])
{
    cplx Q[3][3];
    clover_Q(L, U, n, mu, nu, Q);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Fmn[i][j] = (Q[i][j] - conj(Q[j][i])) / (8.0 * _Complex_I);
}

/* F(n) as a 12x12 matrix, index a = alpha*3 + i */
static void clover_site(const int L[4], const cplx *U, long n, double kappa, double csw,
                        cplx g[5][4][4], cplx *F /* [12][12] */)
{
    memset(F, 0, sizeof(cplx) * 144);
    for (int a = 0; a < 12; ++a) F[a * 12 + a] = 1.0;
    for (int mu = 0; mu < 4; ++mu)
        for (int nu = 0; nu < 4; ++nu) {
            if (mu == nu) continue;
            cplx s[4][4], Fmn[3][3];
            build_sigma(g, mu, nu, s);
            field_strength(L, U, n, mu, nu, Fmn);
            for (int al = 0; al < 4; ++al)
                for (int be = 0; be < 4; ++be) {
                    if (s[al][be] == 0) continue;
                    for (int i = 0; i < 3; ++i)
                        for (int j = 0; j < 3; ++j)
                            F[(al * 3 + i) * 12 + be * 3 + j] -= 0.5 * csw * kappa * s[al][be] * Fmn[i][j];
                }
        }
}

void oracle_clover_field(const int L[4], const double *U_, double kappa, double csw, double *F_)
{
    const cplx *U = (const cplx *)U_;
    cplx *F = (cplx *)F_;
    cplx g[5][4][4];
    build_gammas(g);
    long V = vol(L);
    SITE_LOOP
    for (long n = 0; n < V; ++n) clover_site(L, U, n, kappa, csw, g, F + n * 144);
}

void oracle_field_strength(const int L[4], const double *U_, long n, int mu, int nu, double *out)
{
    field_strength(L, (const cplx *)U_, n, mu, nu, (cplx (*)[3])out);
}

/* ------------------------------------------------------------------ */
/* dense 12x12 inverse: Gauss-Jordan with partial pivoting             */
/* ------------------------------------------------------------------ */

static int invert12(const cplx *A_, cplx *Ainv)
{
    cplx A[12][24];
    for (int i = 0; i < 12; ++i)
        for (int j = 0; j < 12; ++j) {
            A[i][j] = A_[i * 12 + j];
            A[i][12 + j] = (i == j) ? 1.0 : 0.0;
        }
    for (int c = 0; c < 12; ++c) {
        int piv = c;
        for (int r = c + 1; r < 12; ++r)
            if (cabs(A[r][c]) > cabs(A[piv][c])) piv = r;
        if (cabs(A[piv][c]) == 0.0) return -1;
        if (piv != c)
            for (int j = 0; j < 24; ++j) {
                cplx t = A[c][j];
                A[c][j] = A[piv][j];
                A[piv][j] = t;
            }
        cplx inv = 1.0 / A[c][c];
        for (int j = 0; j < 24; ++j) A[c][j] *= inv;
        for (int r = 0; r < 12; ++r) {
            if (r == c) continue;
            cplx f = A[r][c];
            if (f == 0) continue;
            for (int j = 0; j < 24; ++j) A[r][j] -= f * A[c][j];
        }
    }
    for (int i = 0; i < 12; ++i)
        for (int j = 0; j < 12; ++j) Ainv[i * 12 + j] = A[i][12 + j];
    return 0;
}

int oracle_invert_sites(long nsites, const double *F_, double *Finv_)
{
    const cplx *F = (const cplx *)F_;
    cplx *Fi = (cplx *)Finv_;
    for (long n = 0; n < nsites; ++n)
        if (invert12(F + n * 144, Fi + n * 144)) return -1;
    return 0;
}

/* out(n) = M(n) in(n) for a field of 12x12 site matrices */
void oracle_site_apply(long nsites, const double *M_, const double *in_, double *out_)
{
    const cplx *M = (const cplx *)M_;
    const cplx *in = (const cplx *)in_;
    cplx *out = (cplx *)out_;
    SITE_LOOP
    for (long n = 0; n < nsites; ++n) {
        cplx t[12];
        for (int a = 0; a < 12; ++a) {
            cplx acc = 0;
            for (int b = 0; b < 12; ++b) acc += M[n * 144 + a * 12 + b] * in[n * 12 + b];
            t[a] = acc;
        }
        memcpy(out + n * 12, t, sizeof(t));
    }
}

/* ------------------------------------------------------------------ */
/* the hopping matrix, Eq. (4), full 4x4 spin matrices                 */
/* ------------------------------------------------------------------ */

static double bc_factor(const int L[4], long s, int mu, int sign, int t_bc)
{
    /* the hop from s along sign*mu crosses the time boundary */
    if (mu != 3) return 1.0;
    int c[4];
    coords_of(L, s, c);
    if (sign > 0 && c[3] == L[3] - 1) return (double)t_bc;
    if (sign < 0 && c[3] == 0) return (double)t_bc;
    return 1.0;
}

static void hop_site(const int L[4], int t_bc, const cplx *U, const cplx *in, long n, cplx g[5][4][4],
                     int dagger, cplx out[12])
{
    for (int a = 0; a < 12; ++a) out[a] = 0;
    /* dagger = gamma5 H gamma5 = H with the projector signs exchanged */
    double sg = dagger ? -1.0 : 1.0;
    for (int mu = 0; mu < 4; ++mu) {
        for (int sign = 1; sign >= -1; sign -= 2) {
            long m = step(L, n, mu, sign);
            cplx Um[3][3];
            double bc = bc_factor(L, n, mu, sign, t_bc);
            if (sign > 0) mat_load(U, n, mu, 0, Um);  /* U_mu(n) */
            else mat_load(U, m, mu, 1, Um);           /* U_mu(n-mu)^dag */
            /* P = 1 - sign*g_mu (times sg for the dagger) */
            cplx P[4][4];
            for (int a = 0; a < 4; ++a)
                for (int b = 0; b < 4; ++b) P[a][b] = (a == b ? 1.0 : 0.0) - sg * sign * g[mu][a][b];
            for (int al = 0; al < 4; ++al)
                for (int i = 0; i < 3; ++i) {
                    cplx acc = 0;
                    for (int be = 0; be < 4; ++be) {
                        if (P[al][be] == 0) continue;
                        for (int j = 0; j < 3; ++j) acc += P[al][be] * Um[i][j] * in[m * 12 + be * 3 + j];
                    }
                    out[al * 3 + i] += bc * acc;
                }
        }
    }
}

void oracle_hopping(const int L[4], int t_bc, const double *U_, const double *in_, double *out_, int dagger)
{
    cplx g[5][4][4];
    build_gammas(g);
    long V = vol(L);
    const cplx *U = (const cplx *)U_;
    const cplx *in = (const cplx *)in_;
    cplx *out = (cplx *)out_;
    SITE_LOOP
    for (long n = 0; n < V; ++n) hop_site(L, t_bc, U, in, n, g, dagger, out + n * 12);
}

/* D x = F x - kappa H x, F given as a site-matrix field */
void oracle_dirac(const int L[4], int t_bc, const double *U_, const double *F_, double kappa,
                  const double *in_, double *out_)
{
    cplx g[5][4][4];
    build_gammas(g);
    long V = vol(L);
    const cplx *U = (const cplx *)U_;
    const cplx *F = (const cplx *)F_;
    const cplx *in = (const cplx *)in_;
    cplx *out = (cplx *)out_;
    SITE_LOOP
    for (long n = 0; n < V; ++n) {
        cplx h[12];
        hop_site(L, t_bc, U, in, n, g, 0, h);
        for (int a = 0; a < 12; ++a) {
            cplx acc = 0;
            for (int b = 0; b < 12; ++b) acc += F[n * 144 + a * 12 + b] * in[n * 12 + b];
            out[n * 12 + a] = acc - kappa * h[a];
        }
    }
}

/* (D x)(n) at a list of sites only, with the clover built on the fly: used
 * to check large solutions at sampled sites without storing F. */
void oracle_dirac_sites(const int L[4], int t_bc, const double *U_, double kappa, double csw,
                        const double *in_, long nsamp, const long *sites, double *out_)
{
    cplx g[5][4][4];
    build_gammas(g);
    const cplx *U = (const cplx *)U_;
    const cplx *in = (const cplx *)in_;
    cplx *out = (cplx *)out_;
    cplx F[144];
    for (long k = 0; k < nsamp; ++k) {
        long n = sites[k];
        cplx h[12];
        hop_site(L, t_bc, U, in, n, g, 0, h);
        clover_site(L, U, n, kappa, csw, g, F);
        for (int a = 0; a < 12; ++a) {
            cplx acc = 0;
            for (int b = 0; b < 12; ++b) acc += F[a * 12 + b] * in[n * 12 + b];
            out[k * 12 + a] = acc - kappa * h[a];
        }
    }
}

/* (H psi)(n) at a list of sites only (psi a full-lattice vector) */
void oracle_hop_sites(const int L[4], int t_bc, const double *U_, const double *in_, long nsamp, const long *sites,
                      double *out_, int dagger)
{
    cplx g[5][4][4];
    build_gammas(g);
    const cplx *U = (const cplx *)U_;
    const cplx *in = (const cplx *)in_;
    cplx *out = (cplx *)out_;
    for (long k = 0; k < nsamp; ++k) hop_site(L, t_bc, U, in, sites[k], g, dagger, out + k * 12);
}

/* F(n) as 12x12 matrices at a list of sites only */
void oracle_clover_sites(const int L[4], const double *U_, double kappa, double csw, long nsamp, const long *sites,
                         double *F_)
{
    cplx g[5][4][4];
    build_gammas(g);
    const cplx *U = (const cplx *)U_;
    cplx *F = (cplx *)F_;
    for (long k = 0; k < nsamp; ++k) clover_site(L, U, sites[k], kappa, csw, g, F + k * 144);
}

/* ------------------------------------------------------------------ */
/* even-odd pieces, Eqs. (5)-(9)                                       */
/* ------------------------------------------------------------------ */

/* lex site of the cb-th site of the given parity */
static long site_of_cb(const int L[4], int parity, long cb)
{
    long s = 2 * cb;
    if (parity_of(L, s) != parity) s += 1;
    return s;
}

void oracle_half_to_full(const int L[4], int parity, const double *half_, double *full_)
{
    const cplx *half = (const cplx *)half_;
    cplx *full = (cplx *)full_;
    long V = vol(L);
    memset(full, 0, sizeof(cplx) * 12 * V);
    for (long cb = 0; cb < V / 2; ++cb) {
        long s = site_of_cb(L, parity, cb);
        memcpy(full + s * 12, half + cb * 12, sizeof(cplx) * 12);
    }
}

void oracle_full_to_half(const int L[4], int parity, const double *full_, double *half_)
{
    const cplx *full = (const cplx *)full_;
    cplx *half = (cplx *)half_;
    long V = vol(L);
    for (long cb = 0; cb < V / 2; ++cb) {
        long s = site_of_cb(L, parity, cb);
        memcpy(half + cb * 12, full + s * 12, sizeof(cplx) * 12);
    }
}

/* H_{p,1-p} on half vectors: embed, apply the full hopping matrix, restrict */
void oracle_hop_eo(const int L[4], int t_bc, const double *U, int out_parity, const double *in_half,
                   double *out_half, int dagger)
{
    long V = vol(L);
    double *a = malloc(sizeof(cplx) * 12 * V);
    double *b = malloc(sizeof(cplx) * 12 * V);
    oracle_half_to_full(L, 1 - out_parity, in_half, a);
    oracle_hopping(L, t_bc, U, a, b, dagger);
    oracle_full_to_half(L, out_parity, b, out_half);
    free(a);
    free(b);
}

/* restriction of a full site-matrix field to one parity (half field) */
void oracle_field_to_half(const int L[4], int parity, const double *Ffull_, double *Fhalf_)
{
    const cplx *Ff = (const cplx *)Ffull_;
    cplx *Fh = (cplx *)Fhalf_;
    long V = vol(L);
    for (long cb = 0; cb < V / 2; ++cb) {
        long s = site_of_cb(L, parity, cb);
        memcpy(Fh + cb * 144, Ff + s * 144, sizeof(cplx) * 144);
    }
}

typedef struct {
    int L[4];
    int t_bc;
    const double *U;
    const double *Finv; /* full field of inverses, [V][12][12] */
    const double *F;    /* full clover field */
    double kappa;
} eo_op;

/* M(n) in(n) at the sites of parity p, M a full field of 12x12 site
 * matrices (the clover term F or its inverse), in/out half vectors */
static void site_matrix_half(const int L[4], const double *M_, int parity, const double *in_, double *out_)
{
    const cplx *Fi = (const cplx *)M_;
    const cplx *in = (const cplx *)in_;
    cplx *out = (cplx *)out_;
    long V = vol(L);
    SITE_LOOP
    for (long cb = 0; cb < V / 2; ++cb) {
        long s = site_of_cb(L, parity, cb);
        cplx t[12];
        for (int a = 0; a < 12; ++a) {
            cplx acc = 0;
            for (int b = 0; b < 12; ++b) acc += Fi[s * 144 + a * 12 + b] * in[cb * 12 + b];
            t[a] = acc;
        }
        memcpy(out + cb * 12, t, sizeof(t));
    }
}

/* F_pp^-1 applied to a half vector of parity p */
static void clover_inv_half(const eo_op *op, int parity, const double *in_, double *out_)
{
    const cplx *Fi = (const cplx *)op->Finv;
    const cplx *in = (const cplx *)in_;
    cplx *out = (cplx *)out_;
    long V = vol(op->L);
    SITE_LOOP
    for (long cb = 0; cb < V / 2; ++cb) {
        long s = site_of_cb(op->L, parity, cb);
        cplx t[12];
        for (int a = 0; a < 12; ++a) {
            cplx acc = 0;
            for (int b = 0; b < 12; ++b) acc += Fi[s * 144 + a * 12 + b] * in[cb * 12 + b];
            t[a] = acc;
        }
        memcpy(out + cb * 12, t, sizeof(t));
    }
}

/* MULT: H~_{p,1-p} v = F_pp^-1 H_{p,1-p} v  (Sec. II-B) */
void oracle_mult(const int L[4], int t_bc, const double *U, const double *Finv, int out_parity,
                 const double *in_half, double *out_half)
{
    eo_op op = {{L[0], L[1], L[2], L[3]}, t_bc, U, Finv, NULL, 0.0};
    long Vh = vol(L) / 2;
    double *t = malloc(sizeof(cplx) * 12 * Vh);
    oracle_hop_eo(L, t_bc, U, out_parity, in_half, t, 0);
    clover_inv_half(&op, out_parity, t, out_half);
    free(t);
}

/* D^_ee p = p - kappa^2 H~_eo H~_oe p */
static void dhat(const eo_op *op, const double *p_, double *q_)
{
    long Vh = vol(op->L) / 2;
    double *to = malloc(sizeof(cplx) * 12 * Vh);
    double *te = malloc(sizeof(cplx) * 12 * Vh);
    oracle_mult(op->L, op->t_bc, op->U, op->Finv, 1, p_, to);
    oracle_mult(op->L, op->t_bc, op->U, op->Finv, 0, to, te);
    const cplx *p = (const cplx *)p_;
    cplx *q = (cplx *)q_;
    const cplx *w = (const cplx *)te;
    double k2 = op->kappa * op->kappa;
    for (long i = 0; i < 12 * Vh; ++i) q[i] = p[i] - k2 * w[i];
    free(to);
    free(te);
}

void oracle_dhat(const int L[4], int t_bc, const double *U, const double *Finv, double kappa,
                 const double *p, double *q)
{
    eo_op op = {{L[0], L[1], L[2], L[3]}, t_bc, U, Finv, NULL, kappa};
    dhat(&op, p, q);
}

/* The gamma5-hermitian even-odd operator: the Schur complement of D on the
 * even sites itself,
 *     S_ee = F_ee - kappa^2 H_eo F_oo^-1 H_oe       (Sec. II-B, Eqs. 5-8),
 * i.e. D^_ee of Eq. 8 before its left factor F_ee^-1 (D^_ee = F_ee^-1 S_ee).
 * F is the full clover field and Finv its inverse, both [V][12][12]. */
static void schur_ee(const eo_op *op, const double *p_, double *q_)
{
    long Vh = vol(op->L) / 2;
    double *ho = malloc(sizeof(cplx) * 12 * Vh);   /* H_oe p */
    double *fo = malloc(sizeof(cplx) * 12 * Vh);   /* F_oo^-1 H_oe p */
    double *he = malloc(sizeof(cplx) * 12 * Vh);   /* H_eo F_oo^-1 H_oe p */
    double *fe = malloc(sizeof(cplx) * 12 * Vh);   /* F_ee p */
    oracle_hop_eo(op->L, op->t_bc, op->U, 1, p_, ho, 0);
    site_matrix_half(op->L, op->Finv, 1, ho, fo);
    oracle_hop_eo(op->L, op->t_bc, op->U, 0, fo, he, 0);
    site_matrix_half(op->L, op->F, 0, p_, fe);
    cplx *q = (cplx *)q_;
    const cplx *a = (const cplx *)fe, *h = (const cplx *)he;
    double k2 = op->kappa * op->kappa;
    for (long i = 0; i < 12 * Vh; ++i) q[i] = a[i] - k2 * h[i];
    free(ho); free(fo); free(he); free(fe);
}

void oracle_schur_ee(const int L[4], int t_bc, const double *U, const double *F, const double *Finv, double kappa,
                     const double *p, double *q)
{
    eo_op op = {{L[0], L[1], L[2], L[3]}, t_bc, U, Finv, F, kappa};
    schur_ee(&op, p, q);
}

/* Its right-hand side: with b = D x, S_ee x_e = b_e + kappa H_eo F_oo^-1 b_o
 * (the even rows of D x = b with x_o eliminated through the odd rows) */
void oracle_schur_source(const int L[4], int t_bc, const double *U, const double *Finv, double kappa,
                         const double *b_full, double *src_e_)
{
    long Vh = vol(L) / 2;
    double *be = malloc(sizeof(cplx) * 12 * Vh), *bo = malloc(sizeof(cplx) * 12 * Vh);
    double *fo = malloc(sizeof(cplx) * 12 * Vh), *he = malloc(sizeof(cplx) * 12 * Vh);
    oracle_full_to_half(L, 0, b_full, be);
    oracle_full_to_half(L, 1, b_full, bo);
    site_matrix_half(L, Finv, 1, bo, fo);        /* F_oo^-1 b_o */
    oracle_hop_eo(L, t_bc, U, 0, fo, he, 0);     /* H_eo F_oo^-1 b_o */
    cplx *o = (cplx *)src_e_;
    const cplx *a = (const cplx *)be, *h = (const cplx *)he;
    for (long i = 0; i < 12 * Vh; ++i) o[i] = a[i] + kappa * h[i];
    free(be); free(bo); free(fo); free(he);
}

/* b^_e = F_ee^-1 b_e + kappa H~_eo F_oo^-1 b_o  (Eq. 6) */
void oracle_eo_source(const int L[4], int t_bc, const double *U, const double *Finv, double kappa,
                      const double *b_full, double *bhat_e_)
{
    eo_op op = {{L[0], L[1], L[2], L[3]}, t_bc, U, Finv, NULL, kappa};
    long Vh = vol(L) / 2;
    double *be = malloc(sizeof(cplx) * 12 * Vh), *bo = malloc(sizeof(cplx) * 12 * Vh);
    double *t1 = malloc(sizeof(cplx) * 12 * Vh), *t2 = malloc(sizeof(cplx) * 12 * Vh);
    oracle_full_to_half(L, 0, b_full, be);
    oracle_full_to_half(L, 1, b_full, bo);
    clover_inv_half(&op, 1, bo, t1);                 /* F_oo^-1 b_o */
    oracle_mult(L, t_bc, U, Finv, 0, t1, t2);        /* H~_eo F_oo^-1 b_o */
    clover_inv_half(&op, 0, be, t1);                 /* F_ee^-1 b_e */
    cplx *bh = (cplx *)bhat_e_;
    const cplx *a = (const cplx *)t1, *c = (const cplx *)t2;
    for (long i = 0; i < 12 * Vh; ++i) bh[i] = a[i] + kappa * c[i];
    free(be); free(bo); free(t1); free(t2);
}

/* x_o = F_oo^-1 b_o + kappa H~_oe x_e (Eq. 7); writes the full solution */
void oracle_eo_reconstruct(const int L[4], int t_bc, const double *U, const double *Finv, double kappa,
                           const double *b_full, const double *x_e, double *x_full_)
{
    eo_op op = {{L[0], L[1], L[2], L[3]}, t_bc, U, Finv, NULL, kappa};
    long Vh = vol(L) / 2, V = vol(L);
    double *bo = malloc(sizeof(cplx) * 12 * Vh), *t1 = malloc(sizeof(cplx) * 12 * Vh);
    double *t2 = malloc(sizeof(cplx) * 12 * Vh), *xo = malloc(sizeof(cplx) * 12 * Vh);
    double *tmp = malloc(sizeof(cplx) * 12 * V);
    oracle_full_to_half(L, 1, b_full, bo);
    clover_inv_half(&op, 1, bo, t1);
    oracle_mult(L, t_bc, U, Finv, 1, x_e, t2);
    cplx *o = (cplx *)xo;
    const cplx *a = (const cplx *)t1, *c = (const cplx *)t2;
    for (long i = 0; i < 12 * Vh; ++i) o[i] = a[i] + kappa * c[i];
    cplx *xf = (cplx *)x_full_;
    oracle_half_to_full(L, 0, x_e, x_full_);
    oracle_half_to_full(L, 1, xo, tmp);
    const cplx *tt = (const cplx *)tmp;
    for (long s = 0; s < V; ++s)
        if (parity_of(L, s) == 1) memcpy(xf + s * 12, tt + s * 12, sizeof(cplx) * 12);
    free(bo); free(t1); free(t2); free(xo); free(tmp);
}

/* ------------------------------------------------------------------ */
/* vector helpers                                                      */
/* ------------------------------------------------------------------ */

static cplx vdot(long n, const cplx *a, const cplx *b)
{
    cplx acc = 0;
    for (long i = 0; i < n; ++i) acc += conj(a[i]) * b[i];
    return acc;
}

static double vnorm2(long n, const cplx *a)
{
    double acc = 0;
    for (long i = 0; i < n; ++i) acc += creal(a[i]) * creal(a[i]) + cimag(a[i]) * cimag(a[i]);
    return acc;
}

/* ||b - D x|| / ||b|| on the full lattice */
double oracle_true_residual(const int L[4], int t_bc, const double *U, const double *F, double kappa,
                            const double *b_, const double *x_)
{
    long V = vol(L);
    double *Dx = malloc(sizeof(cplx) * 12 * V);
    oracle_dirac(L, t_bc, U, F, kappa, x_, Dx);
    const cplx *b = (const cplx *)b_;
    cplx *r = (cplx *)Dx;
    for (long i = 0; i < 12 * V; ++i) r[i] = b[i] - r[i];
    double res = sqrt(vnorm2(12 * V, r) / vnorm2(12 * V, b));
    free(Dx);
    return res;
}

/* ------------------------------------------------------------------ */
/* BiCGStab, Alg. 2, for a generic linear operator                     */
/* ------------------------------------------------------------------ */

typedef void (*apply_fn)(const void *ctx, const double *in, double *out);

typedef struct {
    int iters;      /* completed iterations (each holds two applications) */
    int applies;    /* operator applications */
    int status;     /* 0 converged, 1 iteration cap, 2 breakdown */
} solve_stats;

/* Solve A x = b from x = x0 (x holds x0 on entry).  Exit when
 * ||r|| < tol_abs.  Both half-steps test the residual (Alg. 2). */
static void bicgstab(apply_fn A, const void *ctx, long n, const cplx *b, cplx *x, double tol_abs,
                     int maxit, solve_stats *st)
{
    cplx *r = malloc(sizeof(cplx) * n), *rt = malloc(sizeof(cplx) * n), *p = malloc(sizeof(cplx) * n);
    cplx *q = malloc(sizeof(cplx) * n), *t = malloc(sizeof(cplx) * n);
    st->iters = 0;
    st->applies = 0;
    st->status = 1;
    A(ctx, (const double *)x, (double *)q);
    st->applies++;
    for (long i = 0; i < n; ++i) r[i] = b[i] - q[i];
    memcpy(rt, r, sizeof(cplx) * n);
    memcpy(p, r, sizeof(cplx) * n);
    cplx rho0 = vdot(n, rt, r);
    if (sqrt(vnorm2(n, r)) < tol_abs) { st->status = 0; goto done; }
    for (int it = 0; it < maxit; ++it) {
        A(ctx, (const double *)p, (double *)q);
        st->applies++;
        cplx rq = vdot(n, rt, q);
        if (rq == 0 || !isfinite(creal(rq)) || !isfinite(cimag(rq))) { st->status = 2; break; }
        cplx alpha = rho0 / rq;
        for (long i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
        st->iters = it + 1;
        if (sqrt(vnorm2(n, r)) < tol_abs) { st->status = 0; break; }
        A(ctx, (const double *)r, (double *)t);
        st->applies++;
        double tt = vnorm2(n, t);
        if (tt == 0) { st->status = 2; break; }
        cplx omega = vdot(n, t, r) / tt;
        if (omega == 0) { st->status = 2; break; }
        for (long i = 0; i < n; ++i) { x[i] += omega * r[i]; r[i] -= omega * t[i]; }
        if (sqrt(vnorm2(n, r)) < tol_abs) { st->status = 0; break; }
        cplx rho1 = vdot(n, rt, r);
        if (rho1 == 0) { st->status = 2; break; }
        cplx beta = (rho1 / rho0) * (alpha / omega);
        rho0 = rho1;
        for (long i = 0; i < n; ++i) p[i] = r[i] + beta * (p[i] - omega * q[i]);
    }
done:
    free(r); free(rt); free(p); free(q); free(t);
}

typedef struct { int L[4]; int t_bc; const double *U, *F; double kappa; } full_op;

static void apply_full(const void *ctx, const double *in, double *out)
{
    const full_op *op = ctx;
    oracle_dirac(op->L, op->t_bc, op->U, op->F, op->kappa, in, out);
}

static void apply_dhat(const void *ctx, const double *in, double *out) { dhat((const eo_op *)ctx, in, out); }

/* Unpreconditioned BiCGStab on D (x = 0 start), exit on ||r||/||b|| < tol. */
int oracle_bicgstab_full(const int L[4], int t_bc, const double *U, const double *F, double kappa,
                         const double *b_, double *x_, double tol, int maxit, int *iters_out)
{
    full_op op = {{L[0], L[1], L[2], L[3]}, t_bc, U, F, kappa};
    long n = 12 * vol(L);
    const cplx *b = (const cplx *)b_;
    memset(x_, 0, sizeof(cplx) * n);
    solve_stats st;
    bicgstab(apply_full, &op, n, b, (cplx *)x_, tol * sqrt(vnorm2(n, b)), maxit, &st);
    if (iters_out) *iters_out = st.iters;
    return st.status;
}

/* Even-odd preconditioned FP64 BiCGStab on D^_ee: b^_e, solve, x_o. */
int oracle_bicgstab_eo(const int L[4], int t_bc, const double *U, const double *Finv, double kappa,
                       const double *b_full, double *x_full, double tol_eo, int maxit, int *iters_out)
{
    eo_op op = {{L[0], L[1], L[2], L[3]}, t_bc, U, Finv, NULL, kappa};
    long Vh = vol(L) / 2, n = 12 * Vh;
    cplx *bh = malloc(sizeof(cplx) * n), *xe = calloc(n, sizeof(cplx));
    oracle_eo_source(L, t_bc, U, Finv, kappa, b_full, (double *)bh);
    solve_stats st;
    bicgstab(apply_dhat, &op, n, bh, xe, tol_eo * sqrt(vnorm2(n, bh)), maxit, &st);
    oracle_eo_reconstruct(L, t_bc, U, Finv, kappa, b_full, (const double *)xe, x_full);
    if (iters_out) *iters_out = st.iters;
    free(bh); free(xe);
    return st.status;
}

static void apply_schur(const void *ctx, const double *in, double *out) { schur_ee((const eo_op *)ctx, in, out); }

/* FP64 BiCGStab on the gamma5-hermitian operator S_ee: its source, the
 * solve (exit on ||r|| < tol_eo ||src||), and x_o as for D^_ee (Eq. 7). */
int oracle_bicgstab_schur(const int L[4], int t_bc, const double *U, const double *F, const double *Finv,
                          double kappa, const double *b_full, double *x_full, double tol_eo, int maxit,
                          int *iters_out)
{
    eo_op op = {{L[0], L[1], L[2], L[3]}, t_bc, U, Finv, F, kappa};
    long Vh = vol(L) / 2, n = 12 * Vh;
    cplx *src = malloc(sizeof(cplx) * n), *xe = calloc(n, sizeof(cplx));
    oracle_schur_source(L, t_bc, U, Finv, kappa, b_full, (double *)src);
    solve_stats st;
    bicgstab(apply_schur, &op, n, src, xe, tol_eo * sqrt(vnorm2(n, src)), maxit, &st);
    oracle_eo_reconstruct(L, t_bc, U, Finv, kappa, b_full, (const double *)xe, x_full);
    if (iters_out) *iters_out = st.iters;
    free(src); free(xe);
    return st.status;
}

/* Alg. 2: v = M p.  The right-hand side is normalised to one, the start is
 * x = 0, the exit test is |r| < tol on the normalised system, and the
 * result is scaled back by |p|.  Run in FP64 here: the oracle checks the
 * logic of the nesting, not the rounding of a lower precision. */
static void inner_solve(const eo_op *op, long n, const cplx *p, cplx *v, double tol, int maxit,
                        solve_stats *st)
{
    if (n <= 0) return;
    double nrm = sqrt(vnorm2(n, p));
    cplx *bn = calloc(n, sizeof(cplx));
    for (long i = 0; i < n; ++i) bn[i] = p[i] / nrm;
    memset(v, 0, sizeof(cplx) * n);
    bicgstab(apply_dhat, op, n, bn, v, tol, maxit, st);
    for (long i = 0; i < n; ++i) v[i] *= nrm;
    free(bn);
}

/* Alg. 1: flexible BiCGStab on D^_ee, right-preconditioned by the inner
 * solve of Alg. 2, exit on |r|/src < tol (recursive residual). */
int oracle_nested_bicgstab(const int L[4], int t_bc, const double *U, const double *Finv, double kappa,
                           const double *b_full, double *x_full, double tol_eo, double inner_tol,
                           int inner_maxit, int maxit, int *outer_out, int *inner_applies_out)
{
    eo_op op = {{L[0], L[1], L[2], L[3]}, t_bc, U, Finv, NULL, kappa};
    long Vh = vol(L) / 2, n = 12 * Vh;
    cplx *bh = malloc(sizeof(cplx) * n), *x = calloc(n, sizeof(cplx)), *r = malloc(sizeof(cplx) * n);
    cplx *rt = malloc(sizeof(cplx) * n), *p = malloc(sizeof(cplx) * n), *v = malloc(sizeof(cplx) * n);
    cplx *q = malloc(sizeof(cplx) * n), *t = malloc(sizeof(cplx) * n);
    oracle_eo_source(L, t_bc, U, Finv, kappa, b_full, (double *)bh);
    memcpy(r, bh, sizeof(cplx) * n);
    memcpy(rt, bh, sizeof(cplx) * n);
    memcpy(p, bh, sizeof(cplx) * n);
    double src = sqrt(vnorm2(n, bh));
    cplx rho0 = src * src;
    int status = 1, outer = 0, inner_applies = 0;
    solve_stats st;
    for (int it = 0; it <= maxit; ++it) {
        outer = it + 1;
        inner_solve(&op, n, p, v, inner_tol, inner_maxit, &st);
        inner_applies += st.applies;
        dhat(&op, (const double *)v, (double *)q);
        cplx alpha = rho0 / vdot(n, rt, q);
        for (long i = 0; i < n; ++i) { x[i] += alpha * v[i]; r[i] -= alpha * q[i]; }
        if (sqrt(vnorm2(n, r)) / src < tol_eo) { status = 0; break; }
        inner_solve(&op, n, r, v, inner_tol, inner_maxit, &st);
        inner_applies += st.applies;
        dhat(&op, (const double *)v, (double *)t);
        cplx omega = vdot(n, t, r) / vnorm2(n, t);
        for (long i = 0; i < n; ++i) { x[i] += omega * v[i]; r[i] -= omega * t[i]; }
        if (sqrt(vnorm2(n, r)) / src < tol_eo) { status = 0; break; }
        cplx rho1 = vdot(n, rt, r);
        cplx beta = (rho1 / rho0) * (alpha / omega);
        rho0 = rho1;
        for (long i = 0; i < n; ++i) p[i] = r[i] + beta * (p[i] - omega * q[i]);
    }
    oracle_eo_reconstruct(L, t_bc, U, Finv, kappa, b_full, (const double *)x, x_full);
    if (outer_out) *outer_out = outer;
    if (inner_applies_out) *inner_applies_out = inner_applies;
    free(bh); free(x); free(r); free(rt); free(p); free(v); free(q); free(t);
    return status;
}

/* ------------------------------------------------------------------ */
/* link gradient by the product rule                                   */
/* ------------------------------------------------------------------ */

/* G = dF/dU for f(U) = -Re <lam, D[U] x>, with x and lam held fixed, in the
 * convention G = df/dRe U + i df/dIm U (the gradient torch returns for a
 * real function of a complex tensor).  Every occurrence of a link entry in D
 * is visited: for f = Re(c * u) the entry gets conj(c), for
 * f = Re(c * conj(u)) it gets c.                                          */
void oracle_link_grad(const int L[4], int t_bc, const double *U_, double kappa, double csw,
                      const double *x_, const double *lam_, double *G_)
{
    const cplx *U = (const cplx *)U_;
    const cplx *x = (const cplx *)x_;
    const cplx *lam = (const cplx *)lam_;
    cplx *G = (cplx *)G_;
    cplx g[5][4][4];
    build_gammas(g);
    long V = vol(L);
    memset(G, 0, sizeof(cplx) * 36 * V);

    /* hopping part: f_hop = +kappa Re <lam, H x> */
    for (long n = 0; n < V; ++n)
        for (int mu = 0; mu < 4; ++mu) {
            long m = step(L, n, mu, +1);
            double bcf = bc_factor(L, n, mu, +1, t_bc);
            /* forward term at n: conj(lam(n)) (1-g_mu) U_mu(n) x(n+mu) */
            /* backward term at m=n+mu: conj(lam(m)) (1+g_mu) U_mu(n)^dag x(n) */
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    cplx cf = 0, cb = 0;
                    for (int al = 0; al < 4; ++al)
                        for (int be = 0; be < 4; ++be) {
                            cplx pm = (al == be ? 1.0 : 0.0) - g[mu][al][be];
                            cplx pp = (al == be ? 1.0 : 0.0) + g[mu][al][be];
                            cf += conj(lam[n * 12 + al * 3 + i]) * pm * x[m * 12 + be * 3 + j];
                            /* coefficient of conj(U_ij): (U^dag)_ji = conj(U_ij) */
                            cb += conj(lam[m * 12 + al * 3 + j]) * pp * x[n * 12 + be * 3 + i];
                        }
                    cf *= kappa * bcf;
                    cb *= kappa * bcf;
                    G[(n * 4 + mu) * 9 + i * 3 + j] += conj(cf) + cb;
                }
        }

    /* clover part: f_clov = -Re <lam, F x>
     *   = (csw kappa / 2) Re sum_n sum_{mu!=nu} sum_ij S_ij F_munu,ij
     * with S_ij = sum_ab conj(lam_ai) sigma_munu,ab x_bj.  With
     * F = (Q - Q^dag)/(8i):  sum_ij S_ij F_ij = sum_ij Z_ij Q_ij (real part)
     * where Z = S/(8i) + conj(-S^T/(8i)).  For a leaf P = L1 L2 L3 L4,
     * Re sum_ij Z_ij P_ij = Re Tr(Z^T L1 L2 L3 L4); the derivative in L_k
     * is Re Tr(dL_k R_k), R_k = L_{k+1}..L_4 Z^T L_1..L_{k-1}.          */
    for (long n = 0; n < V; ++n)
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = 0; nu < 4; ++nu) {
                if (mu == nu) continue;
                cplx s[4][4];
                build_sigma(g, mu, nu, s);
                cplx S[3][3], ZT[3][3];
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) {
                        cplx acc = 0;
                        for (int al = 0; al < 4; ++al)
                            for (int be = 0; be < 4; ++be)
                                acc += conj(lam[n * 12 + al * 3 + i]) * s[al][be] * x[n * 12 + be * 3 + j];
                        S[i][j] = 0.5 * csw * kappa * acc;
                    }
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) {
                        cplx z = S[i][j] / (8.0 * _Complex_I) + conj(-S[j][i] / (8.0 * _Complex_I));
                        ZT[j][i] = z;
                    }
                for (int l = 0; l < 4; ++l) {
                    cplx Lk[4][3][3];
                    long sk[4];
                    int dk[4], dirk[4];
                    for (int k = 0; k < 4; ++k) {
                        const leaf_factor *f = &LEAVES[l][k];
                        sk[k] = leaf_site(L, n, mu, nu, f);
                        dirk[k] = f->along_nu ? nu : mu;
                        dk[k] = f->dag;
                        mat_load(U, sk[k], dirk[k], dk[k], Lk[k]);
                    }
                    /* the trace Tr(Z^T L0 L1 L2 L3) as a cycle of five factors */
                    cplx (*cyc[5])[3] = {ZT, Lk[0], Lk[1], Lk[2], Lk[3]};
                    for (int k = 0; k < 4; ++k) {
                        /* R_k: the four factors that follow L_k around the cycle */
                        int pos = k + 1;
                        cplx R[3][3];
                        memcpy(R, cyc[(pos + 1) % 5], sizeof(R));
                        for (int a = 2; a <= 4; ++a) mat_mul(R, cyc[(pos + a) % 5], R);
                        cplx *Gl = G + (sk[k] * 4 + dirk[k]) * 9;
                        for (int a = 0; a < 3; ++a)
                            for (int b = 0; b < 3; ++b) {
                                if (!dk[k]) Gl[a * 3 + b] += conj(R[b][a]);  /* L = U: coeff of U_ab is R_ba */
                                else Gl[b * 3 + a] += R[b][a];              /* L = U^dag: L_ab = conj(U_ba) */
                            }
                    }
                }
            }
}
