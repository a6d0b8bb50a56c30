// Device pieces of the hopping stencil (Eq. 4) shared by the stencil
// kernels and the batched persistent solver: spin projection before the
// colour multiply, 12-real link reconstruction through Prec<P>, and the
// 8-direction accumulation.
#pragma once

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

// acc += w * expansion of g (w real): the FP16 kernels fold the neighbour's
// per-site norm (and the time-boundary sign) into the accumulation, one FMA
// per real where the unscaled form has one add
template <int MU, int S, class T>
__device__ __forceinline__ void expand_w(Spinor<T> &acc, const cx<T> g[2][3], T w)
{
    const T nw = -w;
    static_assert(std::is_same<T, float>::value, "FP32 arithmetic of the FP16-storage kernels");
    auto add = [](cx<T> &a, const cx<T> &b, T f) { a = mk(::fmaf(f, b.r, a.r), ::fmaf(f, b.i, a.i)); };
    // a += f * (i b) = (a.r - f b.i, a.i + f b.r)
    auto addi = [](cx<T> &a, const cx<T> &b, T f) { a = mk(::fmaf(-f, b.i, a.r), ::fmaf(f, b.r, a.i)); };
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (MU == 3) {
            if (S > 0) {
                add(acc.s[2][i], g[0][i], w);
                add(acc.s[3][i], g[1][i], w);
            } else {
                add(acc.s[0][i], g[0][i], w);
                add(acc.s[1][i], g[1][i], w);
            }
        } else {
            add(acc.s[0][i], g[0][i], w);
            add(acc.s[1][i], g[1][i], w);
            if (MU == 0) {  // lower = -S i (g1, g0)
                addi(acc.s[2][i], g[1][i], S > 0 ? nw : w);
                addi(acc.s[3][i], g[0][i], S > 0 ? nw : w);
            } else if (MU == 1) {  // lower = -S (g1, -g0)
                add(acc.s[2][i], g[1][i], S > 0 ? nw : w);
                add(acc.s[3][i], g[0][i], S > 0 ? w : nw);
            } else {  // lower = -S i (g0, -g1)
                addi(acc.s[2][i], g[0][i], S > 0 ? nw : w);
                addi(acc.s[3][i], g[1][i], S > 0 ? w : nw);
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
        const bool flip = MU == 3 && g.t_bc < 0 && c[3] == g.L[3] - 1;
        Spinor<T> psi;
        cx<T> h[2][3], q[2][3];
        Link<T> L;
        if constexpr (P == QCD_F16) {  // the neighbour's norm and the boundary sign go into the accumulation
            const T w = Prec<P>::load_raw(in, nb, psi);
            project<MU, SF>(psi, h);
            Prec<P>::load_link(U, out_par, cb, MU, L);
            colour_mul<false>(L, h, q);
            expand_w<MU, SF>(acc, q, flip ? -w : w);
        } else {
            Prec<P>::load(in, nb, psi);
            project<MU, SF>(psi, h);
            Prec<P>::load_link(U, out_par, cb, MU, L);
            colour_mul<false>(L, h, q);
            if (flip) {
#pragma unroll
                for (int a = 0; a < 2; ++a)
#pragma unroll
                    for (int i = 0; i < 3; ++i) q[a][i] = -q[a][i];
            }
            expand<MU, SF>(acc, q);
        }
    }
    {  // backward hop: (1 + SF g_mu) U_mu(n - mu)^dag psi(n - mu)
        const int nb = lex_hop(g, lex, c, MU, -1) >> 1;
        const bool flip = MU == 3 && g.t_bc < 0 && c[3] == 0;
        Spinor<T> psi;
        cx<T> h[2][3], q[2][3];
        Link<T> L;
        if constexpr (P == QCD_F16) {
            const T w = Prec<P>::load_raw(in, nb, psi);
            project<MU, -SF>(psi, h);
            Prec<P>::load_link(U, in_par, nb, MU, L);
            colour_mul<true>(L, h, q);
            expand_w<MU, -SF>(acc, q, flip ? -w : w);
        } else {
            Prec<P>::load(in, nb, psi);
            project<MU, -SF>(psi, h);
            Prec<P>::load_link(U, in_par, nb, MU, L);
            colour_mul<true>(L, h, q);
            if (flip) {
#pragma unroll
                for (int a = 0; a < 2; ++a)
#pragma unroll
                    for (int i = 0; i < 3; ++i) q[a][i] = -q[a][i];
            }
            expand<MU, -SF>(acc, q);
        }
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

// ---- rolled forms ----------------------------------------------------------
// For the double-float arithmetic each complex multiply-add is ~60 FP32
// instructions; the fully unrolled stencil would not fit the instruction
// cache and the SM would wait on instruction fetch.  These forms loop over
// the 8 directions and the clover rows at run time instead.
template <class T>
__device__ __forceinline__ void project_rt(int mu, int s, const Spinor<T> &p, cx<T> h[2][3])
{
    switch (2 * mu + (s > 0 ? 0 : 1)) {
    case 0: project<0, 1>(p, h); break;
    case 1: project<0, -1>(p, h); break;
    case 2: project<1, 1>(p, h); break;
    case 3: project<1, -1>(p, h); break;
    case 4: project<2, 1>(p, h); break;
    case 5: project<2, -1>(p, h); break;
    case 6: project<3, 1>(p, h); break;
    default: project<3, -1>(p, h); break;
    }
}

template <class T>
__device__ __forceinline__ void expand_rt(int mu, int s, Spinor<T> &acc, const cx<T> g[2][3])
{
    switch (2 * mu + (s > 0 ? 0 : 1)) {
    case 0: expand<0, 1>(acc, g); break;
    case 1: expand<0, -1>(acc, g); break;
    case 2: expand<1, 1>(acc, g); break;
    case 3: expand<1, -1>(acc, g); break;
    case 4: expand<2, 1>(acc, g); break;
    case 5: expand<2, -1>(acc, g); break;
    case 6: expand<3, 1>(acc, g); break;
    default: expand<3, -1>(acc, g); break;
    }
}

template <int P, bool DAG>
__device__ void hopping_rolled(const Geom &g, const GaugePtr &U, const SpinorPtr &in, int out_par, int cb,
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
#pragma unroll 1
    for (int d = 0; d < 8; ++d) {
        const int mu = d >> 1;
        const bool fwd = (d & 1) == 0;
        // forward: (1 - SF g_mu) U_mu(n) psi(n+mu); backward: (1 + SF g_mu) U_mu(n-mu)^dag psi(n-mu)
        const int nb = lex_hop(g, lex, c, mu, fwd ? +1 : -1) >> 1;
        const int s = fwd ? SF : -SF;
        Spinor<T> psi;
        Prec<P>::load(in, nb, psi);
        cx<T> h[2][3], q[2][3];
        project_rt(mu, s, psi, h);
        Link<T> L;
        Prec<P>::load_link(U, fwd ? out_par : 1 - out_par, fwd ? cb : nb, mu, L);
        if (!fwd) {
            Link<T> D;
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) D.u[i][j] = conj(L.u[j][i]);
            L = D;
        }
        colour_mul<false>(L, h, q);
        if (mu == 3 && g.t_bc < 0 && (fwd ? c[3] == g.L[3] - 1 : c[3] == 0)) {
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int i = 0; i < 3; ++i) q[a][i] = -q[a][i];
        }
        expand_rt(mu, s, acc, q);
    }
}

// y = A x for one Hermitian 6x6 block with rolled loops (see herm6)
template <class T>
__device__ void herm6_rolled(const T d[6], const cx<T> o[15], const cx<T> x[6], cx<T> y[6])
{
#pragma unroll 1
    for (int i = 0; i < 6; ++i) {
        cx<T> a = mk(d[i] * x[i].r, d[i] * x[i].i);
#pragma unroll 1
        for (int j = 0; j < 6; ++j) {
            if (j < i) fma_(a, o[i * (i - 1) / 2 + j], x[j]);
            else if (j > i) fmac_(a, o[j * (j - 1) / 2 + i], x[j]);
        }
        y[i] = a;
    }
}

template <int P>
__device__ void apply_clover_rolled(const CloverPtr &cl, int par, int cb, Spinor<typename Prec<P>::T> &s)
{
    using T = typename Prec<P>::T;
    cx<T> x[2][6], y[2][6];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            x[0][3 * a + i] = s.s[a][i] - s.s[a + 2][i];
            x[1][3 * a + i] = s.s[a][i] + s.s[a + 2][i];
        }
#pragma unroll 1
    for (int blk = 0; blk < 2; ++blk) {
        T d[6];
        cx<T> o[15];
        Prec<P>::load_clover(cl, par, cb, blk, d, o);
        herm6_rolled(d, o, x[blk], y[blk]);
    }
    const T h = T(0.5);
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            s.s[a][i] = h * (y[0][3 * a + i] + y[1][3 * a + i]);
            s.s[a + 2][i] = h * (y[1][3 * a + i] - y[0][3 * a + i]);
        }
}

// the forms each precision uses
template <int P, bool DAG>
__device__ __forceinline__ void hopping_any(const Geom &g, const GaugePtr &U, const SpinorPtr &in, int out_par, int cb,
                                            Spinor<typename Prec<P>::T> &acc)
{
    if constexpr (P == QCD_DF64) hopping_rolled<P, DAG>(g, U, in, out_par, cb, acc);
    else hopping<P, DAG>(g, U, in, out_par, cb, acc);
}

template <int P>
__device__ __forceinline__ void clover_any(const CloverPtr &cl, int par, int cb, Spinor<typename Prec<P>::T> &s)
{
    if constexpr (P == QCD_DF64) apply_clover_rolled<P>(cl, par, cb, s);
    else apply_clover<P>(cl, par, cb, s);
}

struct StencilArgs {
    Geom g;
    GaugePtr U;
    CloverPtr C;
    SpinorPtr out, in, y, aux, z;
    int out_par;
    double a, cc, d;
    float af, ccf, df32;  // the same rounded on the host, for the FP32 / FP16 kernels
    int has_z;            // d != 0
    size_t rhs_stride;   // in 16-byte elements
    size_t norm_stride;  // in floats
    RedArgs red;
    const int *done;
    int *skip;  // profiling: set to 1 when the launch returns early
    int nrhs;   // right-hand sides of the launch (multi-RHS: blockIdx.y selects a tile of them)
};

// a host-supplied scalar in the kernel's arithmetic type (float: the
// host-rounded copy, so no FP64 conversion runs per thread)
template <class T>
__device__ __forceinline__ T sarg(double d, float f)
{
    if constexpr (std::is_same<T, float>::value) return f;
    else return T(d);
}

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

}  // namespace qcd
