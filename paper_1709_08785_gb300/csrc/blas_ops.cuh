// Per-site BLAS-1 building blocks of BiCGStab (Table I: axpy/xpay, dot,
// norm) as functors over one site, shared by the grid-stride kernels of
// blas.cu and the batched persistent solver.
#pragma once

#include <type_traits>

#include "reduce.cuh"

namespace qcd {

// ---------------------------------------------------------------- helpers
template <class T>
__device__ __forceinline__ double norm2_sp(const Spinor<T> &a)
{
    T s = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int i = 0; i < 3; ++i) s += a.s[k][i].r * a.s[k][i].r + a.s[k][i].i * a.s[k][i].i;
    return (double)s;
}

// <a|b> = sum conj(a) b
template <class T>
__device__ __forceinline__ void dot_sp(const Spinor<T> &a, const Spinor<T> &b, double &re, double &im)
{
    T r = 0, i = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            r += a.s[k][c].r * b.s[k][c].r + a.s[k][c].i * b.s[k][c].i;
            i += a.s[k][c].r * b.s[k][c].i - a.s[k][c].i * b.s[k][c].r;
        }
    re += (double)r;
    im += (double)i;
}

// Accumulation into the reduction type A of a kernel (float at the FP32 and
// FP16 levels, double otherwise): the site's sum is formed in the spinor's
// arithmetic type T and converted once (acc_cast).
template <class A, class T>
__device__ __forceinline__ void acc_norm2(A &acc, const Spinor<T> &a)
{
    T s = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int i = 0; i < 3; ++i) s += a.s[k][i].r * a.s[k][i].r + a.s[k][i].i * a.s[k][i].i;
    acc += acc_cast<A>(s);
}

// re + i im += <a|b> = sum conj(a) b
template <class A, class T>
__device__ __forceinline__ void acc_dot(const Spinor<T> &a, const Spinor<T> &b, A &re, A &im)
{
    T r = 0, i = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            r += a.s[k][c].r * b.s[k][c].r + a.s[k][c].i * b.s[k][c].i;
            i += a.s[k][c].r * b.s[k][c].i - a.s[k][c].i * b.s[k][c].r;
        }
    re += acc_cast<A>(r);
    im += acc_cast<A>(i);
}

// The reduction type of a BLAS functor: float for single-precision-level
// functors (OpX<QCD_F32> and the like), double for every other one.
template <class Op>
struct AccOf {
    using type = double;
};
template <template <int> class O, int P>
struct AccOf<O<P>> {
    using type = typename std::conditional<P == QCD_F32 || P == QCD_F16, float, double>::type;
};

// y += a x (complex a)
template <class T>
__device__ __forceinline__ void caxpy(Spinor<T> &y, cx<T> a, const Spinor<T> &x)
{
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) fma_(y.s[k][c], a, x.s[k][c]);
}

template <class T>
__device__ __forceinline__ cx<T> scal(const double *v, double sgn = 1.0)
{
    return mk(T(sgn * v[0]), T(sgn * v[1]));
}

// alpha (0), omega (1) or beta (2) of a solver state, times sgn = +-1, in the
// arithmetic type T: the finaliser's FP32 copies for float, so that no FP64
// arithmetic (1/64 of the FP32 rate on GB300) runs per site
enum { C_ALPHA = 0, C_OMEGA = 1, C_BETA = 2 };
template <class T>
__device__ __forceinline__ cx<T> coef(const SolverState *st, int which, int sgn)
{
    if constexpr (std::is_same<T, float>::value) {
        const float s = (float)sgn;
        return mk(s * st->coef[2 * which], s * st->coef[2 * which + 1]);
    } else {
        const double *v = which == C_ALPHA ? st->alpha : which == C_OMEGA ? st->omega : st->beta;
        return scal<T>(v, (double)sgn);
    }
}

template <class T>
__device__ __forceinline__ void zero_sp(Spinor<T> &a)
{
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) a.s[k][c] = mk(T(0), T(0));
}

template <class T>
__device__ __forceinline__ void scale_sp(Spinor<T> &a, T s)
{
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) a.s[k][c] = mk(a.s[k][c].r * s, a.s[k][c].i * s);
}

template <class TO, class TI>
__device__ __forceinline__ void cvt_sp(Spinor<TO> &o, const Spinor<TI> &a)
{
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) o.s[k][c] = mk((TO)a.s[k][c].r, (TO)a.s[k][c].i);
}

// ---------------------------------------------------------------- BiCGStab updates
// s = r - alpha q (r overwritten), |s|^2
template <int P>
struct OpS {
    SpinorPtr r, q;
    const SolverState *st;
    template <class Acc>
    __device__ void operator()(int cb, Acc *acc) const
    {
        using T = typename Prec<P>::T;
        Spinor<T> R, Q;
        Prec<P>::load(r, cb, R);
        Prec<P>::load(q, cb, Q);
        caxpy(R, coef<T>(st, C_ALPHA, -1), Q);
        Prec<P>::store(r, cb, R);
        acc_norm2(acc[0], R);
    }
};

// x += alpha p + omega s; r = s - omega t; |r|^2, <r~|r>
template <int P>
struct OpX {
    SpinorPtr x, p, r, t, rt;
    const SolverState *st;
    template <class Acc>
    __device__ void operator()(int cb, Acc *acc) const
    {
        using T = typename Prec<P>::T;
        Spinor<T> X, Pp, R, Tt, Rt;
        Prec<P>::load(x, cb, X);
        Prec<P>::load(p, cb, Pp);
        Prec<P>::load(r, cb, R);
        caxpy(X, coef<T>(st, C_ALPHA, 1), Pp);
        caxpy(X, coef<T>(st, C_OMEGA, 1), R);
        Prec<P>::store(x, cb, X);
        Prec<P>::load(t, cb, Tt);
        caxpy(R, coef<T>(st, C_OMEGA, -1), Tt);
        Prec<P>::store(r, cb, R);
        Prec<P>::load(rt, cb, Rt);
        acc_norm2(acc[0], R);
        acc_dot(Rt, R, acc[1], acc[2]);
    }
};

// p = r + beta (p - omega q), |p|^2
template <int P>
struct OpP {
    SpinorPtr p, r, q;
    const SolverState *st;
    template <class Acc>
    __device__ void operator()(int cb, Acc *acc) const
    {
        using T = typename Prec<P>::T;
        Spinor<T> Pp, R, Q;
        Prec<P>::load(p, cb, Pp);
        Prec<P>::load(q, cb, Q);
        caxpy(Pp, coef<T>(st, C_OMEGA, -1), Q);
        Prec<P>::load(r, cb, R);
        const cx<T> b = coef<T>(st, C_BETA, 1);
        Spinor<T> O = R;
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int c = 0; c < 3; ++c) fma_(O.s[k][c], b, Pp.s[k][c]);
        Prec<P>::store(p, cb, O);
        acc_norm2(acc[0], O);
    }
};

// x += alpha p when the iteration stopped after its first half-step
template <int P>
struct OpHalf {
    SpinorPtr x, p;
    const SolverState *st;
    template <class Acc>
    __device__ void operator()(int cb, Acc *) const
    {
        using T = typename Prec<P>::T;
        if (!st->exit_half) return;
        Spinor<T> X, Pp;
        Prec<P>::load(x, cb, X);
        Prec<P>::load(p, cb, Pp);
        caxpy(X, coef<T>(st, C_ALPHA, 1), Pp);
        Prec<P>::store(x, cb, X);
    }
};

// flexible (Alg. 1) updates: x += alpha v; r -= alpha q; |r|^2
template <int P>
struct OpFlex1 {
    SpinorPtr x, v, r, q;
    const SolverState *st;
    template <class Acc>
    __device__ void operator()(int cb, Acc *acc) const
    {
        using T = typename Prec<P>::T;
        Spinor<T> X, V, R, Q;
        Prec<P>::load(x, cb, X);
        Prec<P>::load(v, cb, V);
        caxpy(X, coef<T>(st, C_ALPHA, 1), V);
        Prec<P>::store(x, cb, X);
        Prec<P>::load(r, cb, R);
        Prec<P>::load(q, cb, Q);
        caxpy(R, coef<T>(st, C_ALPHA, -1), Q);
        Prec<P>::store(r, cb, R);
        acc_norm2(acc[0], R);
    }
};

// x += omega v; r -= omega t; |r|^2, <r~|r>
template <int P>
struct OpFlex2 {
    SpinorPtr x, v, r, t, rt;
    const SolverState *st;
    template <class Acc>
    __device__ void operator()(int cb, Acc *acc) const
    {
        using T = typename Prec<P>::T;
        Spinor<T> X, V, R, Tt, Rt;
        Prec<P>::load(x, cb, X);
        Prec<P>::load(v, cb, V);
        caxpy(X, coef<T>(st, C_OMEGA, 1), V);
        Prec<P>::store(x, cb, X);
        Prec<P>::load(r, cb, R);
        Prec<P>::load(t, cb, Tt);
        caxpy(R, coef<T>(st, C_OMEGA, -1), Tt);
        Prec<P>::store(r, cb, R);
        Prec<P>::load(rt, cb, Rt);
        acc_norm2(acc[0], R);
        acc_dot(Rt, R, acc[1], acc[2]);
    }
};

// The flexible updates with the solution in a wider storage than the
// iteration's own vectors: x (precision PX, FP64) += coef * v, where v and
// the residual vectors are in P (DF64).  v is widened to PX and the update
// runs in PX arithmetic, so the accumulated solution carries PX's precision
// whatever the operator's arithmetic was.
template <int P, int PX>
__device__ __forceinline__ void acc_x(SpinorPtr x, int cb, const SolverState *st, int which,
                                      const Spinor<typename Prec<P>::T> &V)
{
    using TX = typename Prec<PX>::T;
    Spinor<TX> X, Vx;
    Prec<PX>::load(x, cb, X);
    cvt_sp(Vx, V);
    caxpy(X, coef<TX>(st, which, 1), Vx);
    Prec<PX>::store(x, cb, X);
}

// OpFlex1 with x in PX: x += alpha v; r -= alpha q; |r|^2
template <int P, int PX>
struct OpFlex1X {
    SpinorPtr x, v, r, q;
    const SolverState *st;
    template <class Acc>
    __device__ void operator()(int cb, Acc *acc) const
    {
        using T = typename Prec<P>::T;
        Spinor<T> V, R, Q;
        Prec<P>::load(v, cb, V);
        acc_x<P, PX>(x, cb, st, C_ALPHA, V);
        Prec<P>::load(r, cb, R);
        Prec<P>::load(q, cb, Q);
        caxpy(R, coef<T>(st, C_ALPHA, -1), Q);
        Prec<P>::store(r, cb, R);
        acc_norm2(acc[0], R);
    }
};

// OpFlex2 with x in PX: x += omega v; r -= omega t; |r|^2, <r~|r>
template <int P, int PX>
struct OpFlex2X {
    SpinorPtr x, v, r, t, rt;
    const SolverState *st;
    template <class Acc>
    __device__ void operator()(int cb, Acc *acc) const
    {
        using T = typename Prec<P>::T;
        Spinor<T> V, R, Tt, Rt;
        Prec<P>::load(v, cb, V);
        acc_x<P, PX>(x, cb, st, C_OMEGA, V);
        Prec<P>::load(r, cb, R);
        Prec<P>::load(t, cb, Tt);
        caxpy(R, coef<T>(st, C_OMEGA, -1), Tt);
        Prec<P>::store(r, cb, R);
        Prec<P>::load(rt, cb, Rt);
        acc_norm2(acc[0], R);
        acc_dot(Rt, R, acc[1], acc[2]);
    }
};

// r = r~ = p = src (optionally x = 0), |r|^2
template <int P>
struct OpInit {
    SpinorPtr src, r, rt, p, x;
    int zero_x;
    template <class Acc>
    __device__ void operator()(int cb, Acc *acc) const
    {
        using T = typename Prec<P>::T;
        Spinor<T> S;
        Prec<P>::load(src, cb, S);
        if (r.p != src.p) Prec<P>::store(r, cb, S);
        Prec<P>::store(rt, cb, S);
        Prec<P>::store(p, cb, S);
        if (zero_x) {
            Spinor<T> Z;
            zero_sp(Z);
            Prec<P>::store(x, cb, Z);
        }
        acc_norm2(acc[0], S);
    }
};

// lower-precision start of an inner solve (Alg. 2): b = src/|src|,
// r = r~ = p = b, x = 0
template <int PS, int PD>
struct OpInner {
    SpinorPtr src, r, rt, p, x;
    const double *src_norm2;
    template <class Acc>
    __device__ void operator()(int cb, Acc *) const
    {
        using TS = typename Prec<PS>::T;
        using TD = typename Prec<PD>::T;
        Spinor<TS> S;
        Prec<PS>::load(src, cb, S);
        const double n2 = *src_norm2;
        const TS inv = n2 > 0.0 ? TS(1.0 / sqrt(n2)) : TS(0);
        scale_sp(S, inv);
        Spinor<TD> D;
        cvt_sp(D, S);
        Prec<PD>::store(r, cb, D);
        Prec<PD>::store(rt, cb, D);
        Prec<PD>::store(p, cb, D);
        Spinor<TD> Z;
        zero_sp(Z);
        Prec<PD>::store(x, cb, Z);
    }
};

// v (higher precision) = |src| * x (lower precision), Alg. 2's last step
template <int PS, int PD>
struct OpLift {
    SpinorPtr x, v;
    const double *src_norm2;
    template <class Acc>
    __device__ void operator()(int cb, Acc *) const
    {
        using TS = typename Prec<PS>::T;
        using TD = typename Prec<PD>::T;
        Spinor<TS> X;
        Prec<PS>::load(x, cb, X);
        Spinor<TD> V;
        cvt_sp(V, X);
        scale_sp(V, TD(sqrt(*src_norm2)));
        Prec<PD>::store(v, cb, V);
    }
};

template <int P>
struct OpNorm {
    SpinorPtr a;
    template <class Acc>
    __device__ void operator()(int cb, Acc *acc) const
    {
        using T = typename Prec<P>::T;
        Spinor<T> A;
        Prec<P>::load(a, cb, A);
        acc_norm2(acc[0], A);
    }
};

// <a|b>
template <int P>
struct OpDot {
    SpinorPtr a, b;
    template <class Acc>
    __device__ void operator()(int cb, Acc *acc) const
    {
        using T = typename Prec<P>::T;
        Spinor<T> A, B;
        Prec<P>::load(a, cb, A);
        Prec<P>::load(b, cb, B);
        acc_dot(A, B, acc[0], acc[1]);
    }
};

// <t|r>, |t|^2
template <int P>
struct OpOmega {
    SpinorPtr t, r;
    template <class Acc>
    __device__ void operator()(int cb, Acc *acc) const
    {
        using T = typename Prec<P>::T;
        Spinor<T> A, B;
        Prec<P>::load(t, cb, A);
        Prec<P>::load(r, cb, B);
        acc_dot(A, B, acc[0], acc[1]);
        acc_norm2(acc[2], A);
    }
};

}  // namespace qcd
