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
#include "reduce.cuh"

namespace qcd {

// ---- spin projection in the Dirac basis --------------------------------
// S = +1: projector (1 - gamma_mu);  S = -1: (1 + gamma_mu).
// For mu = x, y, z: (1 - S g_k) psi = (h, -S i s_k h) with
// h = psi_up + S i s_k psi_dn.  For mu = t: (1 - S g_t) keeps the lower
// (S = +1) or upper (S = -1) pair, times 2.
template <int MU, int S, class T>
__device__ __forceinline__ void project(const Spinor<T> &p, cx<T> h[2][3])
{
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (MU == 0) {  // i s_1 psi_dn = (i psi3, i psi2)
            h[0][i] = S > 0 ? p.s[0][i] + ti(p.s[3][i]) : p.s[0][i] - ti(p.s[3][i]);
            h[1][i] = S > 0 ? p.s[1][i] + ti(p.s[2][i]) : p.s[1][i] - ti(p.s[2][i]);
        } else if (MU == 1) {  // i s_2 psi_dn = (psi3, -psi2)
            h[0][i] = S > 0 ? p.s[0][i] + p.s[3][i] : p.s[0][i] - p.s[3][i];
            h[1][i] = S > 0 ? p.s[1][i] - p.s[2][i] : p.s[1][i] + p.s[2][i];
        } else if (MU == 2) {  // i s_3 psi_dn = (i psi2, -i psi3)
            h[0][i] = S > 0 ? p.s[0][i] + ti(p.s[2][i]) : p.s[0][i] - ti(p.s[2][i]);
            h[1][i] = S > 0 ? p.s[1][i] - ti(p.s[3][i]) : p.s[1][i] + ti(p.s[3][i]);
        } else {
            const T two = T(2);
            h[0][i] = S > 0 ? two * p.s[2][i] : two * p.s[0][i];
            h[1][i] = S > 0 ? two * p.s[3][i] : two * p.s[1][i];
        }
    }
}

// acc += expansion of the projected, colour-multiplied pair g
template <int MU, int S, class T>
__device__ __forceinline__ void expand(Spinor<T> &acc, const cx<T> g[2][3])
{
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (MU == 3) {
            if (S > 0) {
                acc.s[2][i] = acc.s[2][i] + g[0][i];
                acc.s[3][i] = acc.s[3][i] + g[1][i];
            } else {
                acc.s[0][i] = acc.s[0][i] + g[0][i];
                acc.s[1][i] = acc.s[1][i] + g[1][i];
            }
        } else {
            acc.s[0][i] = acc.s[0][i] + g[0][i];
            acc.s[1][i] = acc.s[1][i] + g[1][i];
            if (MU == 0) {  // lower = -S i (g1, g0)
                acc.s[2][i] = S > 0 ? acc.s[2][i] - ti(g[1][i]) : acc.s[2][i] + ti(g[1][i]);
                acc.s[3][i] = S > 0 ? acc.s[3][i] - ti(g[0][i]) : acc.s[3][i] + ti(g[0][i]);
            } else if (MU == 1) {  // lower = -S (g1, -g0)
                acc.s[2][i] = S > 0 ? acc.s[2][i] - g[1][i] : acc.s[2][i] + g[1][i];
                acc.s[3][i] = S > 0 ? acc.s[3][i] + g[0][i] : acc.s[3][i] - g[0][i];
            } else {  // lower = -S i (g0, -g1)
                acc.s[2][i] = S > 0 ? acc.s[2][i] - ti(g[0][i]) : acc.s[2][i] + ti(g[0][i]);
                acc.s[3][i] = S > 0 ? acc.s[3][i] + ti(g[1][i]) : acc.s[3][i] - ti(g[1][i]);
            }
        }
    }
}

// g = U h  or  g = U^dag h, for both spin rows
template <bool DAG, class T>
__device__ __forceinline__ void colour_mul(const Link<T> &U, const cx<T> h[2][3], cx<T> g[2][3])
{
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            cx<T> s = mk(T(0), T(0));
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                if (DAG) fmac_(s, U.u[j][i], h[a][j]);
                else fma_(s, U.u[i][j], h[a][j]);
            }
            g[a][i] = s;
        }
}

template <int P, int MU, int SF>
__device__ __forceinline__ void hop_dir(const Geom &g, const GaugePtr &U, const SpinorPtr &in, int out_par, int cb,
                                        int lex, const int c[4], Spinor<typename Prec<P>::T> &acc)
{
    using T = typename Prec<P>::T;
    const int in_par = 1 - out_par;
    {  // forward hop: (1 - SF g_mu) U_mu(n) psi(n + mu)
        const int nb = lex_hop(g, lex, c, MU, +1) >> 1;
        Spinor<T> psi;
        Prec<P>::load(in, nb, psi);
        cx<T> h[2][3], q[2][3];
        project<MU, SF>(psi, h);
        Link<T> L;
        Prec<P>::load_link(U, out_par, cb, MU, L);
        colour_mul<false>(L, h, q);
        if (MU == 3 && g.t_bc < 0 && c[3] == g.L[3] - 1) {
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int i = 0; i < 3; ++i) q[a][i] = -q[a][i];
        }
        expand<MU, SF>(acc, q);
    }
    {  // backward hop: (1 + SF g_mu) U_mu(n - mu)^dag psi(n - mu)
        const int nb = lex_hop(g, lex, c, MU, -1) >> 1;
        Spinor<T> psi;
        Prec<P>::load(in, nb, psi);
        cx<T> h[2][3], q[2][3];
        project<MU, -SF>(psi, h);
        Link<T> L;
        Prec<P>::load_link(U, in_par, nb, MU, L);
        colour_mul<true>(L, h, q);
        if (MU == 3 && g.t_bc < 0 && c[3] == 0) {
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int i = 0; i < 3; ++i) q[a][i] = -q[a][i];
        }
        expand<MU, -SF>(acc, q);
    }
}

// acc = H in at site cb of parity out_par (DAG: gamma5 H gamma5, i.e. the
// projector signs exchanged)
template <int P, bool DAG>
__device__ __forceinline__ void hopping(const Geom &g, const GaugePtr &U, const SpinorPtr &in, int out_par, int cb,
                                        Spinor<typename Prec<P>::T> &acc)
{
    using T = typename Prec<P>::T;
    int c[4];
    site_coords(g, out_par, cb, c);
    const int lex = lex_of(g, c);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i) acc.s[a][i] = mk(T(0), T(0));
    constexpr int SF = DAG ? -1 : 1;
    hop_dir<P, 0, SF>(g, U, in, out_par, cb, lex, c, acc);
    hop_dir<P, 1, SF>(g, U, in, out_par, cb, lex, c, acc);
    hop_dir<P, 2, SF>(g, U, in, out_par, cb, lex, c, acc);
    hop_dir<P, 3, SF>(g, U, in, out_par, cb, lex, c, acc);
}

struct StencilArgs {
    Geom g;
    GaugePtr U;
    CloverPtr C;
    SpinorPtr out, in, y, aux, z;
    int out_par;
    double a, cc, d;
    size_t rhs_stride;   // in 16-byte elements
    size_t norm_stride;  // in floats
    RedArgs red;
    const int *done;
    int *skip;  // profiling: set to 1 when the launch returns early
};

__device__ __forceinline__ SpinorPtr rhs_ptr(const SpinorPtr &v, int r, size_t stride, size_t nstride)
{
    SpinorPtr o;
    o.p = v.p ? (void *)((uint4 *)v.p + r * stride) : nullptr;
    o.norm = v.norm ? v.norm + r * nstride : nullptr;
    return o;
}

template <class T>
__device__ __forceinline__ void axpby_sp(Spinor<T> &o, T a, const Spinor<T> &x, T b, const Spinor<T> &y)
{
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int i = 0; i < 3; ++i) o.s[s][i] = mk(a * x.s[s][i].r + b * y.s[s][i].r, a * x.s[s][i].i + b * y.s[s][i].i);
}

template <int P, int MODE, int RED, bool DAG>
__global__ void __launch_bounds__(384) stencil_kernel(StencilArgs A)
{
    using T = typename Prec<P>::T;
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0;
    if (A.done && *A.done) {
        if (A.skip && lead) *A.skip = 1;
        return;
    }
    if (A.skip && lead) *A.skip = 0;
    const int cb = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = threadIdx.y;
    double red[4] = {0.0, 0.0, 0.0, 0.0};
    if (cb < A.g.Vh) {
        const SpinorPtr in = rhs_ptr(A.in, r, A.rhs_stride, A.norm_stride);
        const SpinorPtr out = rhs_ptr(A.out, r, A.rhs_stride, A.norm_stride);
        Spinor<T> acc;
        hopping<P, DAG>(A.g, A.U, in, A.out_par, cb, acc);
        if (MODE == M_MULT) {
            apply_clover<P>(A.C, A.out_par, cb, acc);
        } else if (MODE == M_DHAT) {
            apply_clover<P>(A.C, A.out_par, cb, acc);
            Spinor<T> y;
            Prec<P>::load(rhs_ptr(A.y, r, A.rhs_stride, A.norm_stride), cb, y);
            axpby_sp(acc, T(A.cc), acc, T(A.a), y);
            if (A.d != 0.0) {
                Spinor<T> z;
                Prec<P>::load(rhs_ptr(A.z, r, A.rhs_stride, A.norm_stride), cb, z);
                axpby_sp(acc, T(1), acc, T(A.d), z);
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
                red[0] = dr;
                red[1] = di;
                red[2] = nn;
            }
        } else if (MODE == M_SRC) {
            Spinor<T> y;
            Prec<P>::load(rhs_ptr(A.y, r, A.rhs_stride, A.norm_stride), cb, y);
            axpby_sp(acc, T(A.cc), acc, T(A.a), y);
            apply_clover<P>(A.C, A.out_par, cb, acc);
        } else if (MODE == M_FULL) {
            Spinor<T> y;
            Prec<P>::load(rhs_ptr(A.y, r, A.rhs_stride, A.norm_stride), cb, y);
            apply_clover<P>(A.C, A.out_par, cb, y);
            axpby_sp(acc, T(A.cc), acc, T(A.a), y);
            if (A.d != 0.0) {
                Spinor<T> z;
                Prec<P>::load(rhs_ptr(A.z, r, A.rhs_stride, A.norm_stride), cb, z);
                axpby_sp(acc, T(1), acc, T(A.d), z);
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
            red[0] = dr;
            red[1] = di;
        } else if (RED == R_NORM) {
            T nn = 0;
#pragma unroll
            for (int s = 0; s < 4; ++s)
#pragma unroll
                for (int i = 0; i < 3; ++i) nn += acc.s[s][i].r * acc.s[s][i].r + acc.s[s][i].i * acc.s[s][i].i;
            red[0] = nn;
        }
        Prec<P>::store(out, cb, acc);
    }
    if constexpr (RED != R_NONE) grid_reduce<3>(red, A.red);
}

// ---- host launcher -------------------------------------------------------
template <int P, int MODE, int RED, bool DAG>
static void launch_t(const StencilArgs &A, dim3 grid, dim3 block, cudaStream_t s)
{
    stencil_kernel<P, MODE, RED, DAG><<<grid, block, 0, s>>>(A);
}

template <int P>
static int dispatch(const StencilCall &sc, const StencilArgs &A, dim3 grid, dim3 block, cudaStream_t s)
{
#define QCD_CASE(MODE, RED)                                                   \
    if (sc.mode == MODE && sc.red == RED) {                                   \
        if (sc.dagger) launch_t<P, MODE, RED, true>(A, grid, block, s);       \
        else launch_t<P, MODE, RED, false>(A, grid, block, s);                \
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
        launch_t<P, MODE, RED, false>(A, grid, block, s);                     \
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
    if (prec == QCD_F64) { spinor = 192; link = 144; clover = 576; }
    else if (prec == QCD_F32) { spinor = 96; link = 48; clover = 288; }
    else { spinor = 52; link = 24; clover = 144; }
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

int launch_stencil(qcd_ctx *c, const StencilCall &sc)
{
    StencilArgs A;
    A.g = c->g;
    const int p = sc.prec;
    for (int par = 0; par < 2; ++par) {
        A.U.a[par] = p == QCD_F64 ? c->U64[par] : p == QCD_F32 ? c->U32[par] : c->U16a[par];
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
    A.rhs_stride = sc.rhs_stride;
    A.norm_stride = sc.norm_stride;
    A.red = sc.red_args;
    A.done = sc.done;
    const int nrhs = sc.nrhs < 1 ? 1 : sc.nrhs;
    if (nrhs > 16) {
        set_error_message("nrhs > 16 per launch");
        return QCD_EINVAL;
    }
    int bx = 128;
    if (nrhs > 1) bx = nrhs <= 4 ? 64 : 32;
    dim3 block(bx, nrhs);
    dim3 grid(nblocks(c->g.Vh, bx));
    if (sc.red != R_NONE && (int)grid.x > c->partial_blocks) {
        set_error_message("reduction grid too large");
        return QCD_EINVAL;
    }
    ProfScope prof(c, p == QCD_F64 ? QCD_K_MULT_F64 : p == QCD_F32 ? QCD_K_MULT_F32 : QCD_K_MULT_F16,
                   stencil_bytes(c, sc));
    A.skip = prof.flag;
    int rc;
    if (p == QCD_F64) rc = dispatch<QCD_F64>(sc, A, grid, block, c->stream);
    else if (p == QCD_F32) rc = dispatch<QCD_F32>(sc, A, grid, block, c->stream);
    else rc = dispatch<QCD_F16>(sc, A, grid, block, c->stream);
    if (rc != QCD_OK) return rc;
    QCD_CUDA_CHECK(cudaGetLastError());
    return QCD_OK;
}

}  // namespace qcd
