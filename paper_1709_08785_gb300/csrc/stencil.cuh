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
// (S = +1) or upper (S = -1) pair, times 2; the factor 2 is applied in the
// expansion (exact, so the result is the same to the bit).
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
            h[0][i] = S > 0 ? p.s[2][i] : p.s[0][i];
            h[1][i] = S > 0 ? p.s[3][i] : p.s[1][i];
        }
    }
}

// ---- projection of a stored FP16 spinor -------------------------------------
// The 12 half2 words (re, im) of a neighbour spinor as loaded, component
// 3 a + i in word 3 a + i, unscaled (the site's norm goes into the expansion).
struct HalfSpinor {
    unsigned w[12];
};
__device__ __forceinline__ unsigned short hre(unsigned w) { return (unsigned short)(w & 0xffffu); }
__device__ __forceinline__ unsigned short him(unsigned w) { return (unsigned short)(w >> 16); }
__device__ __forceinline__ float hf(unsigned short h) { return __half2float(__ushort_as_half(h)); }
// a + b and a - b with the half a widened inside the add (exact), one rounding
// as in float(a) +- b
__device__ __forceinline__ float hadd(unsigned short a, float b)
{
    float d;
    asm("add.rn.f32.f16 %0, %1, %2;" : "=f"(d) : "h"(a), "f"(b));
    return d;
}
__device__ __forceinline__ float hsub(unsigned short a, float b)
{
    float d;
    asm("sub.rn.f32.f16 %0, %1, %2;" : "=f"(d) : "h"(a), "f"(b));
    return d;
}

// project<MU, S> on the stored halves: each projected real is the first
// spin's half plus or minus the second spin's half widened, the same single
// rounding as the FP32 form, one conversion fewer
template <int MU, int S>
__device__ __forceinline__ void project_h(const HalfSpinor &p, cx<float> h[2][3])
{
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const unsigned p0 = p.w[i], p1 = p.w[3 + i], p2 = p.w[6 + i], p3 = p.w[9 + i];
        if (MU == 0) {  // h0 = p0 +- i p3, h1 = p1 +- i p2
            h[0][i] = S > 0 ? mk(hsub(hre(p0), hf(him(p3))), hadd(him(p0), hf(hre(p3))))
                            : mk(hadd(hre(p0), hf(him(p3))), hsub(him(p0), hf(hre(p3))));
            h[1][i] = S > 0 ? mk(hsub(hre(p1), hf(him(p2))), hadd(him(p1), hf(hre(p2))))
                            : mk(hadd(hre(p1), hf(him(p2))), hsub(him(p1), hf(hre(p2))));
        } else if (MU == 1) {  // h0 = p0 +- p3, h1 = p1 -+ p2
            h[0][i] = S > 0 ? mk(hadd(hre(p0), hf(hre(p3))), hadd(him(p0), hf(him(p3))))
                            : mk(hsub(hre(p0), hf(hre(p3))), hsub(him(p0), hf(him(p3))));
            h[1][i] = S > 0 ? mk(hsub(hre(p1), hf(hre(p2))), hsub(him(p1), hf(him(p2))))
                            : mk(hadd(hre(p1), hf(hre(p2))), hadd(him(p1), hf(him(p2))));
        } else if (MU == 2) {  // h0 = p0 +- i p2, h1 = p1 -+ i p3
            h[0][i] = S > 0 ? mk(hsub(hre(p0), hf(him(p2))), hadd(him(p0), hf(hre(p2))))
                            : mk(hadd(hre(p0), hf(him(p2))), hsub(him(p0), hf(hre(p2))));
            h[1][i] = S > 0 ? mk(hadd(hre(p1), hf(him(p3))), hsub(him(p1), hf(hre(p3))))
                            : mk(hsub(hre(p1), hf(him(p3))), hadd(him(p1), hf(hre(p3))));
        } else {
            const unsigned a = S > 0 ? p2 : p0, b = S > 0 ? p3 : p1;
            h[0][i] = mk(hf(hre(a)), hf(him(a)));
            h[1][i] = mk(hf(hre(b)), hf(him(b)));
        }
    }
}

// 2 a, exactly
template <class T>
__device__ __forceinline__ cx<T> twice(cx<T> a)
{
    if constexpr (std::is_same<T, df>::value) return mk(df(2.f * a.r.hi, 2.f * a.r.lo), df(2.f * a.i.hi, 2.f * a.i.lo));
    else return mk(T(2) * a.r, T(2) * a.i);
}

// acc += expansion of the projected, colour-multiplied pair g
template <int MU, int S, class T>
__device__ __forceinline__ void expand(Spinor<T> &acc, const cx<T> g[2][3])
{
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (MU == 3) {  // the projector's factor 2 (see project)
            if (S > 0) {
                acc.s[2][i] = acc.s[2][i] + twice(g[0][i]);
                acc.s[3][i] = acc.s[3][i] + twice(g[1][i]);
            } else {
                acc.s[0][i] = acc.s[0][i] + twice(g[0][i]);
                acc.s[1][i] = acc.s[1][i] + twice(g[1][i]);
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
    const T w2 = T(2) * w;  // mu = t: the projector's factor 2 (see project)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (MU == 3) {
            if (S > 0) {
                add(acc.s[2][i], g[0][i], w2);
                add(acc.s[3][i], g[1][i], w2);
            } else {
                add(acc.s[0][i], g[0][i], w2);
                add(acc.s[1][i], g[1][i], w2);
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

// ---- packed FP32 pairs -------------------------------------------------------
// Blackwell issues an FP32 operation on a register pair as one instruction
// (two lanes, each rounded as the scalar fmaf / add / mul).  The multi-RHS
// hops use it on the two spin rows of a half spinor: the link products of
// rows 0 and 1 share every link element, and the accumulator's upper spins
// pair as {s0, s1}, its lower ones as {s3, s2} -- the order in which the x, y
// and t expansions keep their lanes.  Each lane repeats the scalar forms'
// operations in their order (a negated operand moved to the other factor,
// which is exact), so the results equal theirs to the bit.  (In the
// single-RHS FP16 hops the pairs cost more registers than they save issue
// slots: no faster, measured.)
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }

// project's rows as the pair {h0, h1}; mu = t, S = +1 feeds the lower pair
// {s3, s2} and is ordered {h1, h0}
template <int MU, int S>
__device__ __forceinline__ void project_pair(const Spinor<float> &psi, float2 Hr[3], float2 Hi[3])
{
    cx<float> h[2][3];
    project<MU, S>(psi, h);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int a0 = (MU == 3 && S > 0) ? 1 : 0;
        Hr[c] = make_float2(h[a0][c].r, h[1 - a0][c].r);
        Hi[c] = make_float2(h[a0][c].i, h[1 - a0][c].i);
    }
}

// G = U H (BWD = 0) or U^dag H (BWD = 1) on the row pair H, u(k) the link
// element k = 3 i + j as {re, im}; colour_mul's fma_ / fmac_ lane by lane
template <int BWD, class LinkAt>
__device__ __forceinline__ void colour_mul_pair(const LinkAt &u, const float2 Hr[3], const float2 Hi[3], float2 Gr[3],
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
            const float2 e = u(BWD ? 3 * j + i : 3 * i + j);
            const float2 ur = make_float2(e.x, e.x), ui = make_float2(e.y, e.y);
            sr = pfma(ur, Hr[j], sr);
            sr = pfma(ui, BWD ? Hi[j] : N[j], sr);
            si = pfma(ur, Hi[j], si);
            si = pfma(ui, BWD ? N[j] : Hr[j], si);
        }
        Gr[i] = sr;
        Gi[i] = si;
    }
}

// complex double-float products gathered in compensated accumulators
// (dacc): a += x*y, a += conj(x)*y
__device__ __forceinline__ void cdacc_fma(dacc &ar, dacc &ai, const cx<df> &x, const cx<df> &y)
{
    dacc_fma(ar, x.r, y.r);
    dacc_fma(ar, -x.i, y.i);
    dacc_fma(ai, x.r, y.i);
    dacc_fma(ai, x.i, y.r);
}
__device__ __forceinline__ void cdacc_fmac(dacc &ar, dacc &ai, const cx<df> &x, const cx<df> &y)
{
    dacc_fma(ar, x.r, y.r);
    dacc_fma(ar, x.i, y.i);
    dacc_fma(ai, x.r, y.i);
    dacc_fma(ai, -x.i, y.r);
}

// g = U h  or  g = U^dag h, for both spin rows
template <bool DAG, class T>
__device__ __forceinline__ void colour_mul(const Link<T> &U, const cx<T> h[2][3], cx<T> g[2][3])
{
    if constexpr (std::is_same<T, df>::value) {  // each row a compensated dot product
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                dacc sr, si;
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    if (DAG) cdacc_fmac(sr, si, U.u[j][i], h[a][j]);
                    else cdacc_fma(sr, si, U.u[i][j], h[a][j]);
                }
                g[a][i] = mk(dacc_get(sr), dacc_get(si));
            }
        return;
    }
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

// The links of a site's eight hops, read from global memory: the forward
// link U_mu(n) at the site itself, the backward one U_mu(n - mu) at the
// neighbour (the other parity)
template <int P>
struct GlobalLinks {
    const GaugePtr &U;  // the kernel's parameter, not a copy in registers
    int out_par, cb;
    template <int MU, int BWD>
    __device__ __forceinline__ void load(int nb, Link<typename Prec<P>::T> &L) const
    {
        Prec<P>::load_link(U, BWD ? 1 - out_par : out_par, BWD ? nb : cb, MU, L);
    }
};

template <int P, int MU, int SF, class LinkF>
__device__ __forceinline__ void hop_dir(const Geom &g, const LinkF &links, const SpinorPtr &in, int out_par, int cb,
                                        int lex, const int c[4], Spinor<typename Prec<P>::T> &acc)
{
    using T = typename Prec<P>::T;
    {  // forward hop: (1 - SF g_mu) U_mu(n) psi(n + mu)
        const int nb = lex_hop(g, lex, c, MU, +1) >> 1;
        const bool flip = MU == 3 && g.t_bc < 0 && c[3] == g.L[3] - 1;
        Spinor<T> psi;
        cx<T> h[2][3], q[2][3];
        Link<T> L;
        if constexpr (P == QCD_F16) {  // the neighbour's norm and the boundary sign go into the accumulation
            HalfSpinor hs;
            const T w = Prec<P>::load_half(in, nb, hs.w);
            project_h<MU, SF>(hs, h);
            links.template load<MU, 0>(nb, L);
            colour_mul<false>(L, h, q);
            expand_w<MU, SF>(acc, q, flip ? -w : w);
        } else {
            Prec<P>::load(in, nb, psi);
            project<MU, SF>(psi, h);
            links.template load<MU, 0>(nb, L);
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
            HalfSpinor hs;
            const T w = Prec<P>::load_half(in, nb, hs.w);
            project_h<MU, -SF>(hs, h);
            links.template load<MU, 1>(nb, L);
            colour_mul<true>(L, h, q);
            expand_w<MU, -SF>(acc, q, flip ? -w : w);
        } else {
            Prec<P>::load(in, nb, psi);
            project<MU, -SF>(psi, h);
            links.template load<MU, 1>(nb, L);
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
template <int P, bool DAG, class LinkF>
__device__ __forceinline__ void hopping_l(const Geom &g, const LinkF &links, const SpinorPtr &in, int out_par, int cb,
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
    hop_dir<P, 0, SF>(g, links, in, out_par, cb, lex, c, acc);
    hop_dir<P, 1, SF>(g, links, in, out_par, cb, lex, c, acc);
    hop_dir<P, 2, SF>(g, links, in, out_par, cb, lex, c, acc);
    hop_dir<P, 3, SF>(g, links, in, out_par, cb, lex, c, acc);
}

template <int P, bool DAG>
__device__ __forceinline__ void hopping(const Geom &g, const GaugePtr &U, const SpinorPtr &in, int out_par, int cb,
                                        Spinor<typename Prec<P>::T> &acc)
{
    hopping_l<P, DAG>(g, GlobalLinks<P>{U, out_par, cb}, in, out_par, cb, acc);
}

// ---- software-pipelined hops (FP32 / FP16) -----------------------------------
// The eight hops of a site in a fixed order d = 2 mu + bwd, with the raw
// loads (neighbour spinor, link) of hop d + 1 issued before hop d computes:
// two hops' loads in flight per thread instead of one, which halves the
// chain of memory latencies a site waits through (the autotuner's
// "pipelined" variant, at the cost of the registers holding the raw data).
template <int P>
struct RawHop;
template <>
struct RawHop<QCD_F32> {
    float4 s[6], l[3];
};
template <>
struct RawHop<QCD_F16> {
    uint4 s[3];
    float n;
    uint4 la;
    uint2 lb;
};

template <int P, int D>
__device__ __forceinline__ void raw_hop_load(const Geom &g, const GaugePtr &U, const SpinorPtr &in, int out_par,
                                             int cb, int lex, const int c[4], RawHop<P> &R)
{
    constexpr int MU = D >> 1, BWD = D & 1;
    const int nb = lex_hop(g, lex, c, MU, BWD ? -1 : +1) >> 1;
    const int lpar = BWD ? 1 - out_par : out_par, lsite = BWD ? nb : cb;
    if constexpr (P == QCD_F32) {
#pragma unroll
        for (int k = 0; k < 6; ++k) R.s[k] = __ldg((const float4 *)in.p + soa(nb, 6, k));
#pragma unroll
        for (int k = 0; k < 3; ++k) R.l[k] = ld_stream((const float4 *)U.a[lpar] + soa(lsite, 12, MU * 3 + k));
    } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) R.s[k] = __ldg((const uint4 *)in.p + soa(nb, 3, k));
        R.n = __ldg(in.norm + nb);
        R.la = ld_stream((const uint4 *)U.a[lpar] + soa(lsite, 4, MU));
        R.lb = ld_stream((const uint2 *)U.b[lpar] + soa(lsite, 4, MU));
    }
}

template <int P, int D, int SF>
__device__ __forceinline__ void raw_hop_apply(const Geom &g, const int c[4], const RawHop<P> &R, Spinor<float> &acc)
{
    constexpr int MU = D >> 1, BWD = D & 1;
    constexpr int S = BWD ? -SF : SF;  // forward (1 - SF g_mu), backward (1 + SF g_mu)
    const bool flip = MU == 3 && g.t_bc < 0 && (BWD ? c[3] == 0 : c[3] == g.L[3] - 1);
    Spinor<float> psi;
    Link<float> L;
    cx<float> h[2][3], q[2][3];
    if constexpr (P == QCD_F32) {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            psi.s[(2 * k) / 3][(2 * k) % 3] = mk(R.s[k].x, R.s[k].y);
            psi.s[(2 * k + 1) / 3][(2 * k + 1) % 3] = mk(R.s[k].z, R.s[k].w);
        }
        Prec<P>::unpack_link(R.l[0], R.l[1], R.l[2], L);
        project<MU, S>(psi, h);
        colour_mul<BWD == 1>(L, h, q);
        if (flip) {
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int i = 0; i < 3; ++i) q[a][i] = -q[a][i];
        }
        expand<MU, S>(acc, q);
    } else {
        const HalfSpinor hs{{R.s[0].x, R.s[0].y, R.s[0].z, R.s[0].w, R.s[1].x, R.s[1].y, R.s[1].z, R.s[1].w, R.s[2].x,
                             R.s[2].y, R.s[2].z, R.s[2].w}};
        Prec<P>::unpack_link(R.la, R.lb, L);
        project_h<MU, S>(hs, h);
        colour_mul<BWD == 1>(L, h, q);
        expand_w<MU, S>(acc, q, flip ? -R.n : R.n);  // the neighbour's norm and the boundary sign
    }
}

template <int P, bool DAG>
__device__ __forceinline__ void hopping_pipe(const Geom &g, const GaugePtr &U, const SpinorPtr &in, int out_par,
                                             int cb, Spinor<float> &acc)
{
    int c[4];
    site_coords(g, out_par, cb, c);
    const int lex = lex_of(g, c);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i) acc.s[a][i] = mk(0.f, 0.f);
    constexpr int SF = DAG ? -1 : 1;
    RawHop<P> R0, R1;
    raw_hop_load<P, 0>(g, U, in, out_par, cb, lex, c, R0);
    raw_hop_load<P, 1>(g, U, in, out_par, cb, lex, c, R1);
    raw_hop_apply<P, 0, SF>(g, c, R0, acc);
    raw_hop_load<P, 2>(g, U, in, out_par, cb, lex, c, R0);
    raw_hop_apply<P, 1, SF>(g, c, R1, acc);
    raw_hop_load<P, 3>(g, U, in, out_par, cb, lex, c, R1);
    raw_hop_apply<P, 2, SF>(g, c, R0, acc);
    raw_hop_load<P, 4>(g, U, in, out_par, cb, lex, c, R0);
    raw_hop_apply<P, 3, SF>(g, c, R1, acc);
    raw_hop_load<P, 5>(g, U, in, out_par, cb, lex, c, R1);
    raw_hop_apply<P, 4, SF>(g, c, R0, acc);
    raw_hop_load<P, 6>(g, U, in, out_par, cb, lex, c, R0);
    raw_hop_apply<P, 5, SF>(g, c, R1, acc);
    raw_hop_load<P, 7>(g, U, in, out_par, cb, lex, c, R1);
    raw_hop_apply<P, 6, SF>(g, c, R0, acc);
    raw_hop_apply<P, 7, SF>(g, c, R1, acc);
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
    if constexpr (std::is_same<T, df>::value) {  // each row a compensated dot product
#pragma unroll 1
        for (int i = 0; i < 6; ++i) {
            dacc sr, si;
            dacc_fma(sr, d[i], x[i].r);
            dacc_fma(si, d[i], x[i].i);
#pragma unroll 1
            for (int j = 0; j < 6; ++j) {
                if (j < i) cdacc_fma(sr, si, o[i * (i - 1) / 2 + j], x[j]);
                else if (j > i) cdacc_fmac(sr, si, o[j * (j - 1) / 2 + i], x[j]);
            }
            y[i] = mk(dacc_get(sr), dacc_get(si));
        }
        return;
    }
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
    CloverPtr Cf;  // the clover term F itself, for M_RECON (C holds F^-1 there)
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
    int done_stride;      // lockstep solves: right-hand side r's done flag is done[r done_stride]
    size_t red_pstride;   // and its reduction's partials start red.partials + r red_pstride
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
