// The C ABI (include/qcd.h): context lifetime, field ingest, the operator
// entry points, the solver entry point, error reporting and kernel timing.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "blas.cuh"

namespace qcd {

static thread_local char g_err[512] = "";

void set_error_message(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

void set_cuda_error(cudaError_t e, const char *what, const char *file, int line)
{
    set_error_message("%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
}

int dev_alloc(qcd_ctx *c, void **p, size_t bytes)
{
    *p = nullptr;
    if (bytes == 0) return QCD_OK;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error_message("cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
        *p = nullptr;
        return QCD_ENOMEM;
    }
    c->pool.push_back(*p);
    e = cudaMemsetAsync(*p, 0, bytes, c->stream);
    if (e != cudaSuccess) {
        set_cuda_error(e, "cudaMemsetAsync", __FILE__, __LINE__);
        return QCD_ECUDA;
    }
    return QCD_OK;
}

size_t hvec_bytes(const Geom &g, int prec) { return hvec_elems(g, prec) * 16; }

constexpr int NWORK = 16;

// All slots of one precision come from one allocation, so slots 2k and
// 2k+1 are contiguous and form a full-lattice vector (even then odd).
int get_work(qcd_ctx *c, int prec, int slot, HVec *out)
{
    if (slot < 0 || slot >= NWORK) {
        set_error_message("workspace slot %d out of range", slot);
        return QCD_EINVAL;
    }
    if (!c->work[prec][0].p) {
        const size_t hb = hvec_bytes(c->g, prec);
        const size_t nb = prec == QCD_F16 ? (size_t)c->g.Vh_pad * sizeof(float) : 0;
        void *base = nullptr, *nbase = nullptr;
        int rc = dev_alloc(c, &base, hb * NWORK);
        if (rc) return rc;
        if (nb) {
            rc = dev_alloc(c, &nbase, nb * NWORK);
            if (rc) return rc;
        }
        for (int k = 0; k < NWORK; ++k) {
            c->work[prec][k].p = (char *)base + k * hb;
            c->work[prec][k].norm = nb ? (float *)((char *)nbase + k * nb) : nullptr;
            c->work[prec][k].prec = prec;
        }
    }
    *out = c->work[prec][slot];
    return QCD_OK;
}

int ensure_staging(qcd_ctx *c, size_t bytes)
{
    if (c->staging_bytes >= bytes) return QCD_OK;
    if (c->staging) {
        cudaStreamSynchronize(c->stream);
        cudaFree(c->staging);
        for (auto &p : c->pool)
            if (p == c->staging) p = nullptr;
        c->staging = nullptr;
        c->staging_bytes = 0;
    }
    int rc = dev_alloc(c, &c->staging, bytes);
    if (rc) return rc;
    c->staging_bytes = bytes;
    return QCD_OK;
}

// ---------------------------------------------------------------- profiling
ProfScope::ProfScope(qcd_ctx *c_, int cls_, double bytes_) : c(c_), cls(cls_), bytes(bytes_)
{
    c->launches += 1;
    if (c->chunk_timing) c->chunk_bytes += bytes;
    if (!c->profiling) return;
    if ((int)c->pending.size() >= PROF_CAP) collect_profile(c);
    const size_t need = 2;
    while (c->event_pool.size() < need) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        c->event_pool.push_back(e);
    }
    a = c->event_pool.back();
    c->event_pool.pop_back();
    b = c->event_pool.back();
    c->event_pool.pop_back();
    flag = c->prof_flags + c->pending.size();
    cudaEventRecord(a, c->stream);
}

ProfScope::~ProfScope()
{
    if (!a) return;
    cudaEventRecord(b, c->stream);
    c->pending.push_back(qcd_ctx::Pending{a, b, cls, bytes});
}

int collect_profile(qcd_ctx *c)
{
    if (c->pending.empty()) return QCD_OK;
    const size_t n = c->pending.size();
    QCD_CUDA_CHECK(cudaMemcpyAsync(c->prof_flags_host, c->prof_flags, n * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    QCD_CUDA_CHECK(cudaStreamSynchronize(c->stream));
    for (size_t i = 0; i < n; ++i) {
        auto &p = c->pending[i];
        float ms = 0.f;
        cudaEventElapsedTime(&ms, p.a, p.b);
        if (c->prof_flags_host[i] != 1) {
            c->stats[p.cls].launches += 1;
            c->stats[p.cls].ms += ms;
            c->stats[p.cls].bytes += p.bytes;
        }
        c->event_pool.push_back(p.a);
        c->event_pool.push_back(p.b);
    }
    c->pending.clear();
    // launches without a done flag never write theirs: reset for the next round
    QCD_CUDA_CHECK(cudaMemsetAsync(c->prof_flags, 0, n * sizeof(int), c->stream));
    return QCD_OK;
}

}  // namespace qcd

using namespace qcd;

// ---------------------------------------------------------------- lifetime
extern "C" int qcd_create(qcd_ctx **out, const int dims[4], int t_bc, void *stream)
{
    if (!out || !dims) {
        set_error_message("null argument");
        return QCD_EINVAL;
    }
    *out = nullptr;
    long V = 1;
    for (int k = 0; k < 4; ++k) {
        if (dims[k] < 2 || (dims[k] & 1)) {
            set_error_message("lattice extent %d = %d: every extent must be even and >= 2", k, dims[k]);
            return QCD_EINVAL;
        }
        V *= dims[k];
    }
    if (V >= (1L << 31) / 4) {
        set_error_message("lattice of %ld sites is too large", V);
        return QCD_EINVAL;
    }
    if (t_bc != 1 && t_bc != -1) {
        set_error_message("t_bc must be +1 or -1");
        return QCD_EINVAL;
    }
    qcd_ctx *c = new (std::nothrow) qcd_ctx();
    if (!c) return QCD_ENOMEM;
    Geom &g = c->g;
    for (int k = 0; k < 4; ++k) g.L[k] = dims[k];
    g.Lxh = dims[0] / 2;
    g.st[0] = 1;
    g.st[1] = dims[0];
    g.st[2] = dims[0] * dims[1];
    g.st[3] = dims[0] * dims[1] * dims[2];
    g.V = (int)V;
    g.Vh = (int)(V / 2);
    g.Vh_pad = (int)pad_sites(V / 2);
    g.t_bc = t_bc;
    c->stream = (cudaStream_t)stream;
    int rc = QCD_OK;
    auto fail = [&](int r) {
        qcd_destroy(c);
        return r;
    };
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        set_error_message("no CUDA device");
        return fail(QCD_ECUDA);
    }
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (c->num_sms <= 0) c->num_sms = 1;
    const size_t vp = (size_t)g.Vh_pad;
    for (int p = 0; p < 2; ++p) {
        if ((rc = dev_alloc(c, &c->U64[p], vp * 36 * 16))) return fail(rc);
        if ((rc = dev_alloc(c, &c->U32[p], vp * 12 * 16))) return fail(rc);
        if ((rc = dev_alloc(c, &c->U16a[p], vp * 4 * 16))) return fail(rc);
        if ((rc = dev_alloc(c, &c->U16b[p], vp * 4 * 8))) return fail(rc);
        if ((rc = dev_alloc(c, &c->UDF[p], vp * 36 * 16))) return fail(rc);
        const size_t cl[4] = {vp * 36 * 16, vp * 18 * 16, vp * 9 * 16, vp * 36 * 16};
        for (int q = 0; q < 4; ++q) {
            if ((rc = dev_alloc(c, &c->C[q][p], cl[q]))) return fail(rc);
            if ((rc = dev_alloc(c, &c->Ci[q][p], cl[q]))) return fail(rc);
        }
    }
    c->partial_blocks = (int)nblocks(2 * vp, 32) + 64;
    if ((rc = dev_alloc(c, (void **)&c->partials, (size_t)c->partial_blocks * 4 * sizeof(double)))) return fail(rc);
    if ((rc = dev_alloc(c, (void **)&c->counters, 64 * sizeof(unsigned)))) return fail(rc);
    if ((rc = dev_alloc(c, (void **)&c->states, NSTATES * sizeof(SolverState)))) return fail(rc);
    if ((rc = dev_alloc(c, (void **)&c->flag_dev, 64 * sizeof(int)))) return fail(rc);
    if ((rc = dev_alloc(c, (void **)&c->prof_flags, PROF_CAP * sizeof(int)))) return fail(rc);
    if (cudaMallocHost(&c->states_host, NSTATES * sizeof(SolverState)) != cudaSuccess ||
        cudaMallocHost(&c->prof_flags_host, PROF_CAP * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        set_error_message("pinned host allocation failed");
        return fail(QCD_ENOMEM);
    }
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
        set_error_message("stream synchronisation failed after allocation");
        return fail(QCD_ECUDA);
    }
    *out = c;
    return QCD_OK;
}

extern "C" int qcd_destroy(qcd_ctx *c)
{
    if (!c) return QCD_OK;
    cudaStreamSynchronize(c->stream);
    for (void *p : c->pool)
        if (p) cudaFree(p);
    if (c->states_host) cudaFreeHost(c->states_host);
    if (c->prof_flags_host) cudaFreeHost(c->prof_flags_host);
    for (auto &p : c->pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto e : c->event_pool) cudaEventDestroy(e);
    if (c->out_stream) {
        cudaStreamSynchronize(c->out_stream);
        cudaStreamDestroy(c->out_stream);
    }
    if (c->out_ready) cudaEventDestroy(c->out_ready);
    for (auto e : c->chunk_ev)
        if (e) cudaEventDestroy(e);
    if (c->out_copied) cudaEventDestroy(c->out_copied);
    delete c;
    return QCD_OK;
}

extern "C" int qcd_set_stream(qcd_ctx *c, void *stream)
{
    if (!c) return QCD_EINVAL;
    c->stream = (cudaStream_t)stream;
    return QCD_OK;
}

extern "C" long qcd_volume(const qcd_ctx *c) { return c ? (long)c->g.V : 0; }

// ---------------------------------------------------------------- fields
static bool is_device_ptr(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

extern "C" int qcd_gauge_load(qcd_ctx *c, const void *U, int on_device)
{
    if (!c || !U) {
        set_error_message("null argument");
        return QCD_EINVAL;
    }
    const size_t bytes = (size_t)c->g.V * 36 * 16;
    const void *src = U;
    if (!on_device) {
        int rc = ensure_staging(c, bytes);
        if (rc) return rc;
        QCD_CUDA_CHECK(cudaMemcpyAsync(c->staging, U, bytes, cudaMemcpyHostToDevice, c->stream));
        src = c->staging;
    }
    int rc = gauge_convert(c, src);
    if (rc) return rc;
    QCD_CUDA_CHECK(cudaStreamSynchronize(c->stream));
    c->have_gauge = true;
    c->have_clover = false;
    return QCD_OK;
}

extern "C" int qcd_clover_build(qcd_ctx *c, double kappa, double csw)
{
    if (!c) return QCD_EINVAL;
    if (!c->have_gauge) {
        set_error_message("qcd_clover_build before qcd_gauge_load");
        return QCD_ESTATE;
    }
    c->have_clover = false;
    int rc = clover_build(c, kappa, csw);
    if (rc) return rc;
    c->kappa = kappa;
    c->csw = csw;
    c->have_clover = true;
    return QCD_OK;
}

// ---------------------------------------------------------------- operators
namespace {

// per-call device buffers for the canonical <-> internal conversion of the
// operator entry points: nrhs half vectors of one precision, in and out
struct ApiBufs {
    HVec in, out, tmp;
    size_t stride;  // 16-byte elements between right-hand sides
};

int api_bufs(qcd_ctx *c, int prec, int nrhs, ApiBufs *b)
{
    const size_t hb = hvec_bytes(c->g, prec);
    const size_t nb = prec == QCD_F16 ? (size_t)c->g.Vh_pad * sizeof(float) : 0;
    // three regions of nrhs vectors each, plus norms
    const size_t need = 3 * nrhs * (hb + nb);
    int rc = ensure_staging(c, need > (size_t)c->g.V * 12 * 16 * 2 ? need : (size_t)c->g.V * 12 * 16 * 2);
    if (rc) return rc;
    char *base = (char *)c->staging;
    HVec *v[3] = {&b->in, &b->out, &b->tmp};
    for (int k = 0; k < 3; ++k) {
        v[k]->p = base + (size_t)k * nrhs * hb;
        v[k]->norm = nb ? (float *)(base + 3 * nrhs * hb + (size_t)k * nrhs * nb) : nullptr;
        v[k]->prec = prec;
    }
    b->stride = hvec_elems(c->g, prec);
    return QCD_OK;
}

int check_op_args(qcd_ctx *c, void *out, const void *in, int prec, int nrhs, bool need_clover)
{
    if (!c || !out || !in) {
        set_error_message("null argument");
        return QCD_EINVAL;
    }
    if (prec < QCD_F64 || prec > QCD_DF64 || nrhs < 1) {
        set_error_message("bad precision %d or nrhs %d", prec, nrhs);
        return QCD_EINVAL;
    }
    if (!c->have_gauge) {
        set_error_message("no gauge field loaded");
        return QCD_ESTATE;
    }
    if (need_clover && !c->have_clover) {
        set_error_message("no clover term built");
        return QCD_ESTATE;
    }
    return QCD_OK;
}

constexpr int RHS_TILE = 16;

// shared body of dslash / mult / dhat / clover on canonical half vectors
int op_half(qcd_ctx *c, void *out, const void *in, int prec, int nrhs, int kind, int out_par, int dagger, int inverse)
{
    const bool f32io = prec == QCD_F32 || prec == QCD_F16;
    const size_t cbytes = (size_t)c->g.Vh * 12 * (f32io ? 8 : 16);
    for (int r0 = 0; r0 < nrhs; r0 += RHS_TILE) {
        const int nr = nrhs - r0 < RHS_TILE ? nrhs - r0 : RHS_TILE;
        ApiBufs B;
        int rc = api_bufs(c, prec, nr, &B);
        if (rc) return rc;
        const char *src = (const char *)in + r0 * cbytes;
        char *dst = (char *)out + r0 * cbytes;
        rc = canon_to_half(c, prec, f32io, src, -1, B.in, nr, B.stride);
        if (rc) return rc;
        if (kind == 3) {
            rc = clover_apply_half(c, prec, out_par, inverse, B.in, B.out, nr, B.stride);
        } else {
            StencilCall s;
            s.prec = prec;
            s.nrhs = nr;
            s.rhs_stride = B.stride;
            s.norm_stride = (size_t)c->g.Vh_pad;
            s.dagger = dagger;
            if (kind == 2 || kind == 4) {  // D^ = 1 - kappa^2 H~_eo H~_oe, or S_ee = F_ee D^
                s.mode = M_MULT;
                s.out_par = 1;
                s.out = B.tmp;
                s.in = B.in;
                rc = launch_stencil(c, s);
                if (rc) return rc;
                s.mode = kind == 4 ? M_FULL : M_DHAT;
                s.out_par = 0;
                s.out = B.out;
                s.in = B.tmp;
                s.y = B.in;
                s.a = 1.0;
                s.cc = -c->kappa * c->kappa;
            } else {
                s.mode = kind == 0 ? M_HOP : M_MULT;
                s.out_par = out_par;
                s.out = B.out;
                s.in = B.in;
            }
            rc = launch_stencil(c, s);
        }
        if (rc) return rc;
        rc = half_to_canon(c, prec, f32io, B.out, dst, -1, nr, B.stride);
        if (rc) return rc;
    }
    return QCD_OK;
}

}  // namespace

extern "C" int qcd_dslash_eo(qcd_ctx *c, void *out, const void *in, int out_parity, int dagger, int prec, int nrhs)
{
    int rc = check_op_args(c, out, in, prec, nrhs, false);
    if (rc) return rc;
    if (out_parity != 0 && out_parity != 1) return QCD_EINVAL;
    return op_half(c, out, in, prec, nrhs, 0, out_parity, dagger ? 1 : 0, 0);
}

extern "C" int qcd_mult_eo(qcd_ctx *c, void *out, const void *in, int out_parity, int dagger, int prec, int nrhs)
{
    int rc = check_op_args(c, out, in, prec, nrhs, true);
    if (rc) return rc;
    if (out_parity != 0 && out_parity != 1) return QCD_EINVAL;
    return op_half(c, out, in, prec, nrhs, 1, out_parity, dagger ? 1 : 0, 0);
}

extern "C" int qcd_dhat(qcd_ctx *c, void *out, const void *in, int prec, int nrhs)
{
    int rc = check_op_args(c, out, in, prec, nrhs, true);
    if (rc) return rc;
    return op_half(c, out, in, prec, nrhs, 2, 0, 0, 0);
}

extern "C" int qcd_schur_ee(qcd_ctx *c, void *out, const void *in, int prec, int nrhs)
{
    int rc = check_op_args(c, out, in, prec, nrhs, true);
    if (rc) return rc;
    return op_half(c, out, in, prec, nrhs, 4, 0, 0, 0);
}

extern "C" int qcd_clover_apply(qcd_ctx *c, void *out, const void *in, int parity, int inverse, int prec, int nrhs)
{
    int rc = check_op_args(c, out, in, prec, nrhs, true);
    if (rc) return rc;
    if (parity != 0 && parity != 1) return QCD_EINVAL;
    return op_half(c, out, in, prec, nrhs, 3, parity, 0, inverse ? 1 : 0);
}

extern "C" int qcd_dirac(qcd_ctx *c, void *out, const void *in)
{
    int rc = check_op_args(c, out, in, QCD_F64, 1, true);
    if (rc) return rc;
    HVec ie, io, oe, oo;
    // the last four FP64 work slots
    if ((rc = get_work(c, QCD_F64, 12, &ie)) || (rc = get_work(c, QCD_F64, 13, &io)) ||
        (rc = get_work(c, QCD_F64, 14, &oe)) || (rc = get_work(c, QCD_F64, 15, &oo)))
        return rc;
    if ((rc = canon_to_half(c, QCD_F64, 0, in, 0, ie, 1, 0)) || (rc = canon_to_half(c, QCD_F64, 0, in, 1, io, 1, 0)))
        return rc;
    for (int par = 0; par < 2; ++par) {
        StencilCall s;
        s.prec = QCD_F64;
        s.mode = M_FULL;
        s.out_par = par;
        s.out = par ? oo : oe;
        s.in = par ? ie : io;
        s.y = par ? io : ie;
        s.a = 1.0;
        s.cc = -c->kappa;
        if ((rc = launch_stencil(c, s))) return rc;
    }
    if ((rc = half_to_canon(c, QCD_F64, 0, oe, out, 0, 1, 0)) || (rc = half_to_canon(c, QCD_F64, 0, oo, out, 1, 1, 0)))
        return rc;
    return QCD_OK;
}

// ---------------------------------------------------------------- solver
extern "C" void qcd_solve_opts_default(qcd_solve_opts *o)
{
    if (!o) return;
    o->precision_levels = 2;
    o->even_odd = 1;
    o->inner_tol[0] = 1e-5;
    o->inner_tol[1] = 1e-2;
    o->max_outer = 200;
    o->max_inner[0] = 250;
    o->max_inner[1] = 250;
    o->max_restarts = 5;
    o->use_x0 = 0;
    o->outer_df64 = 1;
    o->eo_hermitian = 0;
}

extern "C" int qcd_solve(qcd_ctx *c, const void *b, void *x, double tol, const qcd_solve_opts *opts,
                         qcd_solve_info *info)
{
    if (!c || !b || !x) {
        set_error_message("null argument");
        return QCD_EINVAL;
    }
    qcd_solve_opts o;
    qcd_solve_opts_default(&o);
    if (opts) o = *opts;
    if (o.precision_levels < 1 || o.precision_levels > 3 || (!o.even_odd && o.precision_levels != 1) ||
        !(tol > 0.0) || o.max_outer < 1 || o.max_inner[0] < 1 || o.max_inner[1] < 1 || o.max_restarts < 0 ||
        !(o.inner_tol[0] > 0.0) || !(o.inner_tol[1] > 0.0) || o.outer_df64 < 0 || o.outer_df64 > 2 ||
        o.eo_hermitian < 0 || o.eo_hermitian > 1) {
        set_error_message("invalid solver options");
        return QCD_EINVAL;
    }
    if (!c->have_clover) {
        set_error_message("qcd_solve needs qcd_gauge_load and qcd_clover_build first");
        return QCD_ESTATE;
    }
    const size_t vbytes = (size_t)c->g.V * 12 * 16;
    const bool b_dev = is_device_ptr(b), x_dev = is_device_ptr(x);
    const void *bd = b;
    void *xd = x;
    if (!b_dev || !x_dev) {
        int rc = ensure_staging(c, 2 * vbytes);
        if (rc) return rc;
        if (!b_dev) {
            bd = c->staging;
            QCD_CUDA_CHECK(cudaMemcpyAsync(c->staging, b, vbytes, cudaMemcpyHostToDevice, c->stream));
        }
        if (!x_dev) {
            xd = (char *)c->staging + vbytes;
            if (o.use_x0) QCD_CUDA_CHECK(cudaMemcpyAsync(xd, x, vbytes, cudaMemcpyHostToDevice, c->stream));
        }
    }
    if (!x_dev) {
        // the solver copies x out as soon as it is emitted (before its true
        // residual is checked) on a second stream
        if (!c->out_stream) {
            QCD_CUDA_CHECK(cudaStreamCreateWithFlags(&c->out_stream, cudaStreamNonBlocking));
            QCD_CUDA_CHECK(cudaEventCreateWithFlags(&c->out_ready, cudaEventDisableTiming));
            QCD_CUDA_CHECK(cudaEventCreateWithFlags(&c->out_copied, cudaEventDisableTiming));
        }
        c->x_host = x;
        c->x_host_bytes = vbytes;
        c->x_host_issued = false;
    }
    // the reduction counters start from zero: a bounded wait that gave up
    // (QCD_ETIMEOUT) in an earlier call may have left a count behind
    QCD_CUDA_CHECK(cudaMemsetAsync(c->counters, 0, 64 * sizeof(unsigned), c->stream));
    int rc = solve(c, bd, xd, tol, o, info);
    if (!x_dev) {
        const bool issued = c->x_host_issued;
        c->x_host = nullptr;
        c->x_host_issued = false;
        // a path that emitted no x (the unpreconditioned solver, an early
        // error) is copied out here, after the solve
        if (!issued) QCD_CUDA_CHECK(cudaMemcpyAsync(x, xd, vbytes, cudaMemcpyDeviceToHost, c->stream));
        QCD_CUDA_CHECK(cudaStreamSynchronize(c->stream));
        QCD_CUDA_CHECK(cudaStreamSynchronize(c->out_stream));
    }
    return rc;
}

// ---------------------------------------------------------------- lockstep multi-RHS
extern "C" int qcd_solve_multi(qcd_ctx *c, const void *b, void *x, int nrhs, double tol, const qcd_solve_opts *opts,
                               qcd_solve_info *infos)
{
    if (!c || !b || !x) {
        set_error_message("null argument");
        return QCD_EINVAL;
    }
    if (nrhs < 1 || nrhs > 16) {
        set_error_message("qcd_solve_multi: nrhs = %d outside 1..16", nrhs);
        return QCD_EINVAL;
    }
    qcd_solve_opts o;
    qcd_solve_opts_default(&o);
    if (opts) o = *opts;
    if (o.precision_levels != 2 || !o.even_odd || o.use_x0 || !(tol > 0.0) || o.max_outer < 1 ||
        o.max_inner[0] < 1 || !(o.inner_tol[0] > 0.0) || o.max_restarts < 0 || o.outer_df64 < 0 ||
        o.outer_df64 > 1 || o.eo_hermitian != 0) {
        set_error_message("qcd_solve_multi: two levels, even-odd D^_ee, x = 0 start, outer_df64 0 or 1");
        return QCD_EINVAL;
    }
    if (!c->have_clover) {
        set_error_message("qcd_solve_multi needs qcd_gauge_load and qcd_clover_build first");
        return QCD_ESTATE;
    }
    if (!is_device_ptr(b) || !is_device_ptr(x)) {
        set_error_message("qcd_solve_multi: b and x must be device memory");
        return QCD_EINVAL;
    }
    c->x_host = nullptr;
    QCD_CUDA_CHECK(cudaMemsetAsync(c->counters, 0, 64 * sizeof(unsigned), c->stream));
    return solve_multi(c, b, x, nrhs, tol, o, infos);
}

// ---------------------------------------------------------------- batched
static long long g_wait_limit = 10000000LL;  // ~1 s of bounded spinning per device wait
static int g_use_graphs = 1;

extern "C" int qcd_set_wait_limit(long long spins)
{
    if (spins < 1) return QCD_EINVAL;
    g_wait_limit = spins;
    return QCD_OK;
}

extern "C" int qcd_set_graphs(int on)
{
    g_use_graphs = on ? 1 : 0;
    return QCD_OK;
}

extern "C" int qcd_solve_batched(qcd_ctx *const *ctxs, int n, const void *const *b, void *const *x,
                                 const double *tol, const qcd_solve_opts *opts, qcd_solve_info *infos)
{
    if (!ctxs || n < 1 || !b || !x || !tol) {
        set_error_message("null argument or empty batch");
        return QCD_EINVAL;
    }
    qcd_solve_opts o;
    qcd_solve_opts_default(&o);
    if (opts) o = *opts;
    if (o.precision_levels != 2 || !o.even_odd || o.use_x0 || o.max_outer < 1 || o.max_inner[0] < 1 ||
        !(o.inner_tol[0] > 0.0) || o.outer_df64 < 0 || o.outer_df64 > 2 || o.eo_hermitian != 0) {
        set_error_message("batched solves run the even-odd FP64/FP32 scheme from x = 0");
        return QCD_EINVAL;
    }
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i] || !b[i] || !x[i] || !(tol[i] > 0.0)) {
            set_error_message("problem %d: null argument or bad tolerance", i);
            return QCD_EINVAL;
        }
        if (!is_device_ptr(b[i]) || !is_device_ptr(x[i])) {
            set_error_message("problem %d: qcd_solve_batched takes device buffers", i);
            return QCD_EINVAL;
        }
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) {
                set_error_message("problems %d and %d share a context", j, i);
                return QCD_EINVAL;
            }
    }
    // every context's reduction counters from zero (see qcd_solve)
    for (int i = 0; i < n; ++i)
        QCD_CUDA_CHECK(cudaMemsetAsync(ctxs[i]->counters, 0, 64 * sizeof(unsigned), ctxs[0]->stream));
    cudaEvent_t e0, e1;
    QCD_CUDA_CHECK(cudaEventCreate(&e0));
    QCD_CUDA_CHECK(cudaEventCreate(&e1));
    QCD_CUDA_CHECK(cudaEventRecord(e0, ctxs[0]->stream));
    const int rc = batched_solve((qcd_ctx **)ctxs, n, b, x, tol, o, infos, g_wait_limit, g_use_graphs);
    cudaEventRecord(e1, ctxs[0]->stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (infos)
        for (int i = 0; i < n; ++i) infos[i].seconds = ms * 1e-3;
    return rc;
}

// ---------------------------------------------------------------- adjoint
extern "C" int qcd_solve_adjoint(qcd_ctx *c, const void *g, void *lam, double tol, const qcd_solve_opts *opts,
                                 qcd_solve_info *info)
{
    if (!c || !g || !lam) {
        set_error_message("null argument");
        return QCD_EINVAL;
    }
    if (!is_device_ptr(g) || !is_device_ptr(lam)) {
        set_error_message("qcd_solve_adjoint takes device buffers");
        return QCD_EINVAL;
    }
    if (!c->have_clover) {
        set_error_message("qcd_solve_adjoint needs qcd_gauge_load and qcd_clover_build first");
        return QCD_ESTATE;
    }
    int rc;
    if (!c->adj_buf && (rc = dev_alloc(c, &c->adj_buf, (size_t)c->g.V * 12 * 16))) return rc;
    // D^-dag = gamma5 D^-1 gamma5
    if ((rc = gamma5_full(c, g, c->adj_buf))) return rc;
    const int src = qcd_solve(c, c->adj_buf, lam, tol, opts, info);
    if (src != QCD_OK && src != QCD_ENOTCONV && src != QCD_EBREAKDOWN) return src;
    if ((rc = gamma5_full(c, lam, lam))) return rc;
    QCD_CUDA_CHECK(cudaStreamSynchronize(c->stream));
    return src;
}

extern "C" int qcd_force(qcd_ctx *c, const void *U, const void *x, const void *lam, void *G)
{
    if (!c || !U || !x || !lam || !G) {
        set_error_message("null argument");
        return QCD_EINVAL;
    }
    if (!is_device_ptr(U) || !is_device_ptr(x) || !is_device_ptr(lam) || !is_device_ptr(G)) {
        set_error_message("qcd_force takes device buffers");
        return QCD_EINVAL;
    }
    if (!c->have_clover) {
        set_error_message("qcd_force needs kappa and csw from qcd_clover_build");
        return QCD_ESTATE;
    }
    return force(c, x, lam, G, U);
}

// ---------------------------------------------------------------- profiling
extern "C" int qcd_set_profiling(qcd_ctx *c, int on)
{
    if (!c || on < 0 || on > 2) return QCD_EINVAL;
    if (on != 1) {
        int rc = collect_profile(c);
        if (rc) return rc;
    }
    c->profiling = on == 1;
    c->chunk_timing = on == 2;
    if (on == 2)
        for (auto &e : c->chunk_ev)
            if (!e) QCD_CUDA_CHECK(cudaEventCreate(&e));
    return QCD_OK;
}

extern "C" int qcd_kernel_stats(qcd_ctx *c, int cls, qcd_kernel_stat *out)
{
    if (!c || !out || cls < 0 || cls >= QCD_K_COUNT) return QCD_EINVAL;
    int rc = collect_profile(c);
    if (rc) return rc;
    *out = c->stats[cls];
    return QCD_OK;
}

extern "C" int qcd_reset_kernel_stats(qcd_ctx *c)
{
    if (!c) return QCD_EINVAL;
    int rc = collect_profile(c);
    if (rc) return rc;
    std::memset(c->stats, 0, sizeof(c->stats));
    return QCD_OK;
}

extern "C" long qcd_launch_count(const qcd_ctx *c) { return c ? c->launches : 0; }

extern "C" int qcd_autotune(qcd_ctx *c, const char *cache_path)
{
    if (!c) return QCD_EINVAL;
    return autotune(c, cache_path);
}

extern "C" int qcd_tune_info(qcd_ctx *c, int max, unsigned *keys, int *variant, int *threads, double *us)
{
    if (!c || max < 0) return QCD_EINVAL;
    return tune_entries(c, max, keys, variant, threads, us);
}

namespace {

// The benchmark buffers: nrhs input and output vectors in precision prec,
// the input filled with a fixed pattern.
int bench_buffers(qcd_ctx *c, int prec, int nrhs, StencilCall &s)
{
    const size_t hb = hvec_bytes(c->g, prec);
    const size_t nb = (size_t)c->g.Vh_pad * sizeof(float);
    const size_t need = 2 * nrhs * (hb + nb);
    int rc;
    if (c->bench_bytes < need) {
        if (c->bench_buf) {
            cudaStreamSynchronize(c->stream);
            cudaFree(c->bench_buf);
            for (auto &p : c->pool)
                if (p == c->bench_buf) p = nullptr;
            c->bench_buf = nullptr;
            c->bench_bytes = 0;
        }
        if ((rc = dev_alloc(c, &c->bench_buf, need))) return rc;
        c->bench_bytes = need;
    }
    char *base = (char *)c->bench_buf;
    HVec in, out;
    in.prec = out.prec = prec;
    in.p = base;
    out.p = base + nrhs * hb;
    in.norm = (float *)(base + 2 * nrhs * hb);
    out.norm = (float *)(base + 2 * nrhs * hb + nrhs * nb);
    const size_t stride = hvec_elems(c->g, prec);
    if ((rc = fill_pattern(c, prec, in, nrhs, stride, 7))) return rc;
    s.prec = prec;
    s.mode = M_MULT;
    s.out_par = 0;
    s.out = out;
    s.in = in;
    s.nrhs = nrhs;
    s.rhs_stride = stride;
    s.norm_stride = (size_t)c->g.Vh_pad;
    return QCD_OK;
}

int bench_check(qcd_ctx *c, int prec, int nrhs, int iters, const void *a, const void *b)
{
    if (!c || !a || !b || prec < QCD_F64 || prec > QCD_DF64 || nrhs < 1 || nrhs > 16 || iters < 1) {
        set_error_message("invalid benchmark arguments");
        return QCD_EINVAL;
    }
    if (!c->have_clover) {
        set_error_message("the MULT benchmarks need the clover term");
        return QCD_ESTATE;
    }
    return QCD_OK;
}

}  // namespace

extern "C" int qcd_mult_benchmark(qcd_ctx *c, int prec, int nrhs, int iters, double *ms_per_launch,
                                  double *bytes_per_launch)
{
    int rc;
    if ((rc = bench_check(c, prec, nrhs, iters, ms_per_launch, bytes_per_launch))) return rc;
    StencilCall s;
    if ((rc = bench_buffers(c, prec, nrhs, s))) return rc;
    cudaEvent_t e0, e1;
    QCD_CUDA_CHECK(cudaEventCreate(&e0));
    QCD_CUDA_CHECK(cudaEventCreate(&e1));
    double total = 0.0;
    for (int it = -2; it < iters; ++it) {  // two untimed warm-up launches
        if ((rc = l2_evict(c))) break;
        QCD_CUDA_CHECK(cudaEventRecord(e0, c->stream));
        if ((rc = launch_stencil(c, s))) break;
        QCD_CUDA_CHECK(cudaEventRecord(e1, c->stream));
        QCD_CUDA_CHECK(cudaEventSynchronize(e1));
        float ms = 0.f;
        QCD_CUDA_CHECK(cudaEventElapsedTime(&ms, e0, e1));
        if (it >= 0) total += ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    *ms_per_launch = total / iters;
    *bytes_per_launch = stencil_bytes(c, s);
    return QCD_OK;
}

extern "C" int qcd_mult_throughput(qcd_ctx *c, int prec, int nrhs, int iters, double *ms_per_launch,
                                   double *bytes_per_launch)
{
    int rc;
    if ((rc = bench_check(c, prec, nrhs, iters, ms_per_launch, bytes_per_launch))) return rc;
    StencilCall s;
    if ((rc = bench_buffers(c, prec, nrhs, s))) return rc;
    cudaEvent_t e0, e1;
    QCD_CUDA_CHECK(cudaEventCreate(&e0));
    QCD_CUDA_CHECK(cudaEventCreate(&e1));
    for (int it = 0; it < 2 && !rc; ++it) rc = launch_stencil(c, s);  // warm-up
    if (!rc) QCD_CUDA_CHECK(cudaEventRecord(e0, c->stream));
    for (int it = 0; it < iters && !rc; ++it) rc = launch_stencil(c, s);
    float ms = 0.f;
    if (!rc) {
        QCD_CUDA_CHECK(cudaEventRecord(e1, c->stream));
        QCD_CUDA_CHECK(cudaEventSynchronize(e1));
        QCD_CUDA_CHECK(cudaEventElapsedTime(&ms, e0, e1));
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    *ms_per_launch = ms / iters;
    *bytes_per_launch = stencil_bytes(c, s);
    return QCD_OK;
}

extern "C" int qcd_pion_correlator(qcd_ctx *c, const void *S, int ncol, int on_device, double *C)
{
    if (!c || !S || !C || ncol < 1) {
        set_error_message("qcd_pion_correlator: NULL pointer or ncol < 1");
        return QCD_EINVAL;
    }
    return pion_correlator(c, S, ncol, on_device, C);
}

extern "C" const char *qcd_strerror(int s)
{
    switch (s) {
    case QCD_OK: return "ok";
    case QCD_EINVAL: return "invalid argument";
    case QCD_ECUDA: return "CUDA error";
    case QCD_ENOMEM: return "out of memory";
    case QCD_ENOTCONV: return "not converged";
    case QCD_EBREAKDOWN: return "BiCGStab breakdown";
    case QCD_ENONFINITE: return "non-finite value";
    case QCD_ECLOVER_SINGULAR: return "singular clover block";
    case QCD_ETIMEOUT: return "device wait timed out";
    case QCD_ESTATE: return "call out of order";
    default: return "unknown status";
    }
}

extern "C" const char *qcd_last_error(void) { return g_err; }
