// Fused BLAS-1 updates of BiCGStab (Table I: axpy/xpay, dot, norm) with the
// dot products and norms they feed reduced in the same pass, layout
// conversions between the canonical and the site-blocked internal layouts,
// and the clover apply of the public API.
//
// Every update kernel reads its scalars (alpha, omega, beta, scales) from
// the solver state in device memory and returns at once when that state is
// marked done, so a host can queue iterations ahead without reading
// anything back.
#include <atomic>

#include "blas.cuh"
#include "blas_ops.cuh"

namespace qcd {

// Grid-stride driver: each thread applies op to its sites, reduces NRED
// doubles over the grid and runs the finaliser.
template <int NRED, class Op>
__global__ void __launch_bounds__(256) blas_kernel(int n, Op op, RedArgs red, const int *done, int *skip)
{
    pdl_enter();
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    if (done && *done) {
        if (skip && lead) *skip = 1;
        return;
    }
    if (skip && lead) *skip = 0;
    using A = typename AccOf<Op>::type;
    A acc[4] = {A(0), A(0), A(0), A(0)};
    for (int cb = blockIdx.x * blockDim.x + threadIdx.x; cb < n; cb += gridDim.x * blockDim.x) op(cb, acc);
    if constexpr (NRED > 0) grid_reduce<NRED>(acc, red);
}

// Blocks of blas_kernel<NRED, Op> resident on one SM (256 threads each),
// from the kernel's register and shared-memory needs
template <int NRED, class Op>
static int blocks_per_sm()
{
    static std::atomic<int> occ{0};
    int n = occ.load(std::memory_order_relaxed);
    if (n <= 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, blas_kernel<NRED, Op>, 256, 0) != cudaSuccess || n < 1) {
            cudaGetLastError();
            n = 2;
        }
        occ.store(n, std::memory_order_relaxed);
    }
    return n;
}

template <int NRED, class Op>
static int run(qcd_ctx *c, int nsites, const Op &op, int fin, SolverState *st, const int *done, int cls, double bytes)
{
    const int threads = 256;
    int blocks = (int)nblocks(nsites, threads);
    // one wave of resident blocks walking the sites: a grid larger than the
    // SMs hold runs its last partial wave at a fraction of the occupancy
    // (the x, r update at 66 registers holds three blocks per SM, not four)
    const int cap = blocks_per_sm<NRED, Op>() * c->num_sms;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    RedArgs ra;
    ra.partials = c->partials;
    ra.counter = c->counters;
    ra.st = st;
    ra.op = fin;
    ProfScope prof(c, cls, bytes);
    launch_pdl(blas_kernel<NRED, Op>, dim3(blocks), dim3(threads), 0, c->stream, nsites, op, ra, done, prof.flag);
    QCD_CUDA_CHECK(cudaGetLastError());
    return QCD_OK;
}

static double sp_bytes(int prec) { return prec == QCD_F32 ? 96.0 : prec == QCD_F16 ? 52.0 : 192.0; }

// timing class of a BLAS launch: the FP32 level's kernels apart from the rest
static int bcls(int prec) { return prec == QCD_F32 ? QCD_K_BLAS_F32 : QCD_K_BLAS; }

// ---------------------------------------------------------------- state
__global__ void k_state_init(SolverState *st, double tol2, double tol2_rel, int maxit, double bd_eps, int unit)
{
    SolverState s = {};
    s.tol2 = tol2;
    s.tol2_rel = tol2_rel;
    s.maxit = maxit;
    s.bd_eps = bd_eps;
    s.status = QCD_OK;
    if (unit) {  // unit-norm right-hand side of Alg. 2: rho0 = 1
        s.rho0[0] = 1.0;
        s.rr = 1.0;
        s.rt2 = 1.0;
        s.norm2[1] = 1.0;
    }
    *st = s;
}

// a right-hand side that takes no part in a lockstep inner solve: its
// kernels return at once
__global__ void k_state_mark_done(SolverState *st) { st->done = 1; }

// dst->tol2 = factor * src->norm2[slot]
__global__ void k_set_tol2(SolverState *dst, const SolverState *src, int slot, double factor)
{
    dst->tol2 = factor * src->norm2[slot];
}

// ---------------------------------------------------------------- launchers
#define PREC_SWITCH(p, ...)                                  \
    switch (p) {                                             \
    case QCD_F64: { constexpr int P = QCD_F64; __VA_ARGS__; } \
    case QCD_F32: { constexpr int P = QCD_F32; __VA_ARGS__; } \
    case QCD_DF64: { constexpr int P = QCD_DF64; __VA_ARGS__; } \
    default: { constexpr int P = QCD_F16; __VA_ARGS__; }      \
    }

int state_init(qcd_ctx *c, SolverState *st, double tol2, double tol2_rel, int maxit, double bd_eps, int unit)
{
    c->launches += 1;
    k_state_init<<<1, 1, 0, c->stream>>>(st, tol2, tol2_rel, maxit, bd_eps, unit);
    QCD_CUDA_CHECK(cudaGetLastError());
    return QCD_OK;
}

int state_mark_done(qcd_ctx *c, SolverState *st)
{
    c->launches += 1;
    k_state_mark_done<<<1, 1, 0, c->stream>>>(st);
    QCD_CUDA_CHECK(cudaGetLastError());
    return QCD_OK;
}

int set_tol2(qcd_ctx *c, SolverState *dst, const SolverState *src, int slot, double factor)
{
    c->launches += 1;
    k_set_tol2<<<1, 1, 0, c->stream>>>(dst, src, slot, factor);
    QCD_CUDA_CHECK(cudaGetLastError());
    return QCD_OK;
}

int blas_update_s(qcd_ctx *c, int prec, int n, HVec r, HVec q, SolverState *st)
{
    const double by = 3 * sp_bytes(prec) * n;
    PREC_SWITCH(prec, return run<1>(c, n, OpS<P>{r.sp(), q.sp(), st}, FIN_S, st, &st->done, bcls(prec), by));
}

int blas_update_x(qcd_ctx *c, int prec, int n, HVec x, HVec p, HVec r, HVec t, HVec rt, SolverState *st)
{
    const double by = 7 * sp_bytes(prec) * n;
    PREC_SWITCH(prec, return run<3>(c, n, OpX<P>{x.sp(), p.sp(), r.sp(), t.sp(), rt.sp(), st}, FIN_X, st, &st->done,
                                    bcls(prec), by));
}

int blas_update_p(qcd_ctx *c, int prec, int n, HVec p, HVec r, HVec q, SolverState *st, int fin)
{
    const double by = 4 * sp_bytes(prec) * n;
    if (fin == FIN_NONE)
        PREC_SWITCH(prec, return run<0>(c, n, OpP<P>{p.sp(), r.sp(), q.sp(), st}, fin, st, &st->done, bcls(prec), by));
    PREC_SWITCH(prec, return run<1>(c, n, OpP<P>{p.sp(), r.sp(), q.sp(), st}, fin, st, &st->done, bcls(prec), by));
}

int blas_finish_half(qcd_ctx *c, int prec, int n, HVec x, HVec p, SolverState *st)
{
    const double by = 3 * sp_bytes(prec) * n;
    PREC_SWITCH(prec, return run<0>(c, n, OpHalf<P>{x.sp(), p.sp(), st}, FIN_NONE, st, nullptr, bcls(prec), by));
}

// x may be wider than the other vectors (FP64 solution, DF64 iteration)
static int mixed_x(int prec, const HVec &x)
{
    if (x.prec == prec) return 0;
    if (x.prec == QCD_F64 && prec == QCD_DF64) return 1;
    set_error_message("unsupported solution precision %d for an iteration in %d", x.prec, prec);
    return -1;
}

int blas_flex1(qcd_ctx *c, int prec, int n, HVec x, HVec v, HVec r, HVec q, SolverState *st)
{
    const double by = 6 * sp_bytes(prec) * n;
    const int mx = mixed_x(prec, x);
    if (mx < 0) return QCD_EINVAL;
    if (mx)
        return run<1>(c, n, OpFlex1X<QCD_DF64, QCD_F64>{x.sp(), v.sp(), r.sp(), q.sp(), st}, FIN_S, st, &st->done,
                      bcls(prec), by);
    PREC_SWITCH(prec, return run<1>(c, n, OpFlex1<P>{x.sp(), v.sp(), r.sp(), q.sp(), st}, FIN_S, st, &st->done,
                                    bcls(prec), by));
}

int blas_flex2(qcd_ctx *c, int prec, int n, HVec x, HVec v, HVec r, HVec t, HVec rt, SolverState *st)
{
    const double by = 7 * sp_bytes(prec) * n;
    const int mx = mixed_x(prec, x);
    if (mx < 0) return QCD_EINVAL;
    if (mx)
        return run<3>(c, n, OpFlex2X<QCD_DF64, QCD_F64>{x.sp(), v.sp(), r.sp(), t.sp(), rt.sp(), st}, FIN_X, st,
                      &st->done, bcls(prec), by);
    PREC_SWITCH(prec, return run<3>(c, n, OpFlex2<P>{x.sp(), v.sp(), r.sp(), t.sp(), rt.sp(), st}, FIN_X, st,
                                    &st->done, bcls(prec), by));
}

int blas_init(qcd_ctx *c, int prec, int n, HVec src, HVec r, HVec rt, HVec p, HVec x, int zero_x, SolverState *st,
              int fin)
{
    const double by = (4 + zero_x) * sp_bytes(prec) * n;
    PREC_SWITCH(prec, return run<1>(c, n, OpInit<P>{src.sp(), r.sp(), rt.sp(), p.sp(), x.sp(), zero_x}, fin, st, nullptr,
                                    bcls(prec), by));
}

int blas_norm2(qcd_ctx *c, int prec, int n, HVec a, SolverState *st, int fin)
{
    const double by = sp_bytes(prec) * n;
    PREC_SWITCH(prec, return run<1>(c, n, OpNorm<P>{a.sp()}, fin, st, nullptr, bcls(prec), by));
}

int blas_dot(qcd_ctx *c, int prec, int n, HVec a, HVec b, SolverState *st, int fin, const int *done)
{
    const double by = 2 * sp_bytes(prec) * n;
    PREC_SWITCH(prec, return run<2>(c, n, OpDot<P>{a.sp(), b.sp()}, fin, st, done, bcls(prec), by));
}

int blas_omega(qcd_ctx *c, int prec, int n, HVec t, HVec r, SolverState *st, const int *done)
{
    const double by = 2 * sp_bytes(prec) * n;
    PREC_SWITCH(prec, return run<3>(c, n, OpOmega<P>{t.sp(), r.sp()}, FIN_OMEGA, st, done, bcls(prec), by));
}

int blas_inner_init(qcd_ctx *c, int ps, int pd, int n, HVec src, const double *src_norm2, HVec r, HVec rt, HVec p,
                    HVec x, const int *done)
{
    const double by = (sp_bytes(ps) + 4 * sp_bytes(pd)) * n;
    if (ps == QCD_F64 && pd == QCD_F32)
        return run<0>(c, n, OpInner<QCD_F64, QCD_F32>{src.sp(), r.sp(), rt.sp(), p.sp(), x.sp(), src_norm2}, FIN_NONE,
                      nullptr, done, bcls(pd), by);
    if (ps == QCD_F32 && pd == QCD_F16)
        return run<0>(c, n, OpInner<QCD_F32, QCD_F16>{src.sp(), r.sp(), rt.sp(), p.sp(), x.sp(), src_norm2}, FIN_NONE,
                      nullptr, done, bcls(pd), by);
    if (ps == QCD_F64 && pd == QCD_F16)
        return run<0>(c, n, OpInner<QCD_F64, QCD_F16>{src.sp(), r.sp(), rt.sp(), p.sp(), x.sp(), src_norm2}, FIN_NONE,
                      nullptr, done, bcls(pd), by);
    if (ps == QCD_DF64 && pd == QCD_F32)
        return run<0>(c, n, OpInner<QCD_DF64, QCD_F32>{src.sp(), r.sp(), rt.sp(), p.sp(), x.sp(), src_norm2}, FIN_NONE,
                      nullptr, done, bcls(pd), by);
    set_error_message("unsupported precision pair %d -> %d", ps, pd);
    return QCD_EINVAL;
}

int blas_lift(qcd_ctx *c, int ps, int pd, int n, HVec x, HVec v, const double *src_norm2, const int *done)
{
    const double by = (sp_bytes(ps) + sp_bytes(pd)) * n;
    if (ps == QCD_F32 && pd == QCD_F64)
        return run<0>(c, n, OpLift<QCD_F32, QCD_F64>{x.sp(), v.sp(), src_norm2}, FIN_NONE, nullptr, done, bcls(ps), by);
    if (ps == QCD_F16 && pd == QCD_F32)
        return run<0>(c, n, OpLift<QCD_F16, QCD_F32>{x.sp(), v.sp(), src_norm2}, FIN_NONE, nullptr, done, bcls(ps), by);
    if (ps == QCD_F16 && pd == QCD_F64)
        return run<0>(c, n, OpLift<QCD_F16, QCD_F64>{x.sp(), v.sp(), src_norm2}, FIN_NONE, nullptr, done, bcls(ps), by);
    if (ps == QCD_F32 && pd == QCD_DF64)
        return run<0>(c, n, OpLift<QCD_F32, QCD_DF64>{x.sp(), v.sp(), src_norm2}, FIN_NONE, nullptr, done, bcls(ps),
                      by);
    set_error_message("unsupported precision pair %d -> %d", ps, pd);
    return QCD_EINVAL;
}

// ---------------------------------------------------------------- layouts
// canonical (complex128 or complex64, [sites][4][3]) <-> internal half vector.
// full >= 0: the canonical buffer is a full-lattice vector and parity `full`
// is taken; full < 0: it is a half vector indexed by cb.
template <int P, class TC>
__global__ void k_canon_to_half(Geom g, const TC *__restrict__ src, SpinorPtr dst, int full, size_t in_stride,
                                size_t rhs_stride, size_t norm_stride)
{
    const int cb = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (cb >= g.Vh_pad) return;
    using T = typename Prec<P>::T;
    SpinorPtr d;
    d.p = (void *)((uint4 *)dst.p + r * rhs_stride);
    d.norm = dst.norm ? dst.norm + r * norm_stride : nullptr;
    Spinor<T> S;
    if (cb >= g.Vh) {
        zero_sp(S);
    } else {
        int site = cb;
        if (full >= 0) {
            int c[4];
            site_coords(g, full, cb, c);
            site = lex_of(g, c);
        }
        const TC *q = src + r * in_stride + (size_t)site * 24;
#pragma unroll
        for (int k = 0; k < 12; ++k) S.s[k / 3][k % 3] = mk((T)q[2 * k], (T)q[2 * k + 1]);
    }
    Prec<P>::store(d, cb, S);
}

template <int P, class TC>
__global__ void k_half_to_canon(Geom g, SpinorPtr src, TC *__restrict__ dst, int full, size_t out_stride,
                                size_t rhs_stride, size_t norm_stride)
{
    const int cb = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (cb >= g.Vh) return;
    using T = typename Prec<P>::T;
    SpinorPtr s;
    s.p = (void *)((uint4 *)src.p + r * rhs_stride);
    s.norm = src.norm ? src.norm + r * norm_stride : nullptr;
    Spinor<T> S;
    Prec<P>::load(s, cb, S);
    int site = cb;
    if (full >= 0) {
        int c[4];
        site_coords(g, full, cb, c);
        site = lex_of(g, c);
    }
    TC *q = dst + r * out_stride + (size_t)site * 24;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        q[2 * k] = (TC)S.s[k / 3][k % 3].r;
        q[2 * k + 1] = (TC)S.s[k / 3][k % 3].i;
    }
}

size_t hvec_elems(const Geom &g, int prec)  // 16-byte elements of one half vector
{
    const int nc = prec == QCD_F32 ? 6 : prec == QCD_F16 ? 3 : 12;
    return (size_t)g.Vh_pad * nc;
}

int canon_to_half(qcd_ctx *c, int prec, int src_is_f32, const void *src, int full, HVec dst, int nrhs,
                  size_t rhs_stride)
{
    dim3 grid(nblocks(c->g.Vh_pad, 128), nrhs);
    const size_t in_stride = (size_t)(full >= 0 ? c->g.V : c->g.Vh) * 24;
    const size_t ns = (size_t)c->g.Vh_pad;
    ProfScope prof(c, QCD_K_OTHER, 0.0);
    if (src_is_f32) {
        PREC_SWITCH(prec, k_canon_to_half<P, float><<<grid, 128, 0, c->stream>>>(c->g, (const float *)src, dst.sp(), full,
                                                                               in_stride, rhs_stride, ns);
                    break);
    } else {
        PREC_SWITCH(prec, k_canon_to_half<P, double><<<grid, 128, 0, c->stream>>>(c->g, (const double *)src, dst.sp(),
                                                                                full, in_stride, rhs_stride, ns);
                    break);
    }
    QCD_CUDA_CHECK(cudaGetLastError());
    return QCD_OK;
}

int half_to_canon(qcd_ctx *c, int prec, int dst_is_f32, HVec src, void *dst, int full, int nrhs, size_t rhs_stride)
{
    dim3 grid(nblocks(c->g.Vh, 128), nrhs);
    const size_t out_stride = (size_t)(full >= 0 ? c->g.V : c->g.Vh) * 24;
    const size_t ns = (size_t)c->g.Vh_pad;
    ProfScope prof(c, QCD_K_OTHER, 0.0);
    if (dst_is_f32) {
        PREC_SWITCH(prec, k_half_to_canon<P, float><<<grid, 128, 0, c->stream>>>(c->g, src.sp(), (float *)dst, full,
                                                                               out_stride, rhs_stride, ns);
                    break);
    } else {
        PREC_SWITCH(prec, k_half_to_canon<P, double><<<grid, 128, 0, c->stream>>>(c->g, src.sp(), (double *)dst, full,
                                                                                out_stride, rhs_stride, ns);
                    break);
    }
    QCD_CUDA_CHECK(cudaGetLastError());
    return QCD_OK;
}

// deterministic smooth data for benchmarks: component k of site cb of
// right-hand side r is (sin(a), cos(a)) with a = 0.37 cb + 1.1 k + 2.3 r + seed
template <int P>
__global__ void k_fill(Geom g, SpinorPtr v, size_t rhs_stride, size_t norm_stride, int seed)
{
    const int cb = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (cb >= g.Vh_pad) return;
    using T = typename Prec<P>::T;
    SpinorPtr d;
    d.p = (void *)((uint4 *)v.p + r * rhs_stride);
    d.norm = v.norm ? v.norm + r * norm_stride : nullptr;
    Spinor<T> S;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const float a = 0.37f * (cb % 1021) + 1.1f * k + 2.3f * r + seed;
        S.s[k / 3][k % 3] = mk((T)(cb < g.Vh ? __sinf(a) : 0.f), (T)(cb < g.Vh ? __cosf(a) : 0.f));
    }
    Prec<P>::store(d, cb, S);
}

int fill_pattern(qcd_ctx *c, int prec, HVec v, int nrhs, size_t rhs_stride, int seed)
{
    dim3 grid(nblocks(c->g.Vh_pad, 128), nrhs);
    ProfScope prof(c, QCD_K_OTHER, 0.0);
    PREC_SWITCH(prec, k_fill<P><<<grid, 128, 0, c->stream>>>(c->g, v.sp(), rhs_stride, (size_t)c->g.Vh_pad, seed);
                break);
    QCD_CUDA_CHECK(cudaGetLastError());
    return QCD_OK;
}

// one half vector from one precision to another
template <int PS, int PD>
struct OpConvert {
    SpinorPtr src, dst;
    __device__ void operator()(int cb, double *) const
    {
        Spinor<typename Prec<PS>::T> S;
        Prec<PS>::load(src, cb, S);
        Spinor<typename Prec<PD>::T> D;
        cvt_sp(D, S);
        Prec<PD>::store(dst, cb, D);
    }
};

int convert_half(qcd_ctx *c, HVec src, HVec dst)
{
    const int n = c->g.Vh_pad;
    const double by = (sp_bytes(src.prec) + sp_bytes(dst.prec)) * n;
    if (src.prec == QCD_F64 && dst.prec == QCD_DF64)
        return run<0>(c, n, OpConvert<QCD_F64, QCD_DF64>{src.sp(), dst.sp()}, FIN_NONE, nullptr, nullptr, QCD_K_BLAS, by);
    if (src.prec == QCD_DF64 && dst.prec == QCD_F64)
        return run<0>(c, n, OpConvert<QCD_DF64, QCD_F64>{src.sp(), dst.sp()}, FIN_NONE, nullptr, nullptr, QCD_K_BLAS, by);
    set_error_message("unsupported conversion %d -> %d", src.prec, dst.prec);
    return QCD_EINVAL;
}

// ---------------------------------------------------------------- clover apply
template <int P>
__global__ void k_clover_apply(Geom g, CloverPtr C, int par, SpinorPtr in, SpinorPtr out, size_t rhs_stride,
                               size_t norm_stride)
{
    const int cb = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (cb >= g.Vh) return;
    using T = typename Prec<P>::T;
    SpinorPtr i, o;
    i.p = (void *)((uint4 *)in.p + r * rhs_stride);
    i.norm = in.norm ? in.norm + r * norm_stride : nullptr;
    o.p = (void *)((uint4 *)out.p + r * rhs_stride);
    o.norm = out.norm ? out.norm + r * norm_stride : nullptr;
    Spinor<T> S;
    Prec<P>::load(i, cb, S);
    apply_clover<P>(C, par, cb, S);
    Prec<P>::store(o, cb, S);
}

int clover_apply_half(qcd_ctx *c, int prec, int parity, int inverse, HVec in, HVec out, int nrhs, size_t rhs_stride)
{
    CloverPtr C;
    for (int p = 0; p < 2; ++p) C.p[p] = inverse ? c->Ci[prec][p] : c->C[prec][p];
    dim3 grid(nblocks(c->g.Vh, 128), nrhs);
    const double cl = prec == QCD_F32 ? 288 : prec == QCD_F16 ? 144 : 576;
    ProfScope prof(c, QCD_K_OTHER, (cl + 2 * nrhs * sp_bytes(prec)) * c->g.Vh);
    PREC_SWITCH(prec, k_clover_apply<P><<<grid, 128, 0, c->stream>>>(c->g, C, parity, in.sp(), out.sp(), rhs_stride,
                                                                    (size_t)c->g.Vh_pad);
                break);
    QCD_CUDA_CHECK(cudaGetLastError());
    return QCD_OK;
}

}  // namespace qcd
