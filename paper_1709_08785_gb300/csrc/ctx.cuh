// The library context and the internal interfaces between translation
// units: field storage, solver state kept in device memory, the
// single-pass grid reduction, and the kernel launchers.
#pragma once

#include <unordered_map>
#include <utility>
#include <vector>

#include "qcd_internal.cuh"

namespace qcd {

// Launch with programmatic stream serialization: the kernel (which starts
// with pdl_enter) may become resident before its predecessor in the stream
// has finished, and waits on the device for it.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args &&...args)
{
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// An internal half-lattice vector in the site-blocked layout.
struct HVec {
    void *p = nullptr;
    float *norm = nullptr;  // F16 only
    int prec = QCD_F64;
    SpinorPtr sp() const { return SpinorPtr{p, norm}; }
};

// Scalars of one BiCGStab level, kept in device memory so that no
// iteration needs the host.  Complex numbers are (re, im) pairs.
struct SolverState {
    double sum[4];     // result of the last grid reduction
    double rho0[2];
    double alpha[2];
    double omega[2];
    double beta[2];
    double rr;         // |r|^2 after the last update
    double tol2;       // exit when |r|^2 < tol2
    double tol2_rel;   // if > 0, FIN_INIT sets tol2 = tol2_rel * |r|^2
    double norm2[4];   // saved squared norms (e.g. |p|^2, |b|^2)
    double rt2;        // |r~|^2, for the breakdown test
    double bd_eps;     // breakdown threshold on |rho1| / (|r~| |r|)
    int iter;
    int maxit;
    int done;          // set once converged / capped / broken down
    int status;        // qcd_status
    int exit_half;     // 1: stopped after the first half-step of Alg. 2
    int pad[3];
    float coef[6];     // alpha, omega, beta rounded to FP32 by the finaliser, for the
                       // FP32 / FP16 levels (no per-site FP64 conversion)
};

// Finaliser run by the last block of a reduction kernel.
enum FinOp {
    FIN_NONE = 0,
    FIN_ALPHA,     // sum = <r~|q>            -> alpha = rho0 / <r~|q>
    FIN_S,         // sum = |s|^2             -> half-step exit test
    FIN_OMEGA,     // sum = <t|r>, |t|^2      -> omega
    FIN_X,         // sum = |r|^2, <r~|r>     -> exit test, beta, rho0
    FIN_INIT,      // sum = |r|^2             -> start: rho0 = rt2 = rr = norm2[1] = |r|^2 (and tol2)
    FIN_RESTART,   // sum = |r|^2             -> restart from a recomputed residual
    FIN_SETN = 16, // FIN_SETN + k: norm2[k] = sum[0]
    FIN_ADDN = 20, // FIN_ADDN + k: norm2[k] += sum[0]
};

struct RedArgs {
    double *partials = nullptr;  // [gridDim.x][4]
    unsigned *counter = nullptr;
    SolverState *st = nullptr;
    int op = FIN_NONE;
};

enum StencilMode { M_HOP = 0, M_MULT = 1, M_DHAT = 2, M_SRC = 3, M_FULL = 4, M_RECON = 5 };
enum StencilRed { R_NONE = 0, R_DOT_AUX = 1, R_OMEGA = 2, R_NORM = 3 };

}  // namespace qcd

struct qcd_ctx {
    qcd::Geom g;
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 0;

    // gauge links per parity of the base site
    void *U64[2] = {nullptr, nullptr};
    void *U32[2] = {nullptr, nullptr};
    void *U16a[2] = {nullptr, nullptr};
    void *U16b[2] = {nullptr, nullptr};
    void *UDF[2] = {nullptr, nullptr};  // DF64: 18 reals as float pairs
    bool have_gauge = false;

    // clover term F and inverse, [precision][parity]
    void *C[4][2] = {};
    void *Ci[4][2] = {};
    bool have_clover = false;
    double kappa = 0.0, csw = 0.0;

    // reductions and solver scalars
    double *partials = nullptr;
    unsigned *counters = nullptr;          // one per reduction chain
    qcd::SolverState *states = nullptr;    // device, NSTATES
    qcd::SolverState *states_host = nullptr;  // pinned mirror
    int *flag_dev = nullptr;
    int partial_blocks = 0;

    // workspace vectors, allocated on first use
    std::vector<void *> pool;
    qcd::HVec work[4][16];  // [precision][slot]
    void *staging = nullptr;        // canonical full-lattice complex128 staging
    size_t staging_bytes = 0;

    // host output of qcd_solve: when x_host is set, the even-odd solver
    // copies each FP64 solution it emits to x_host on out_stream, so that
    // the copy overlaps the true-residual check
    void *x_host = nullptr;
    size_t x_host_bytes = 0;
    bool x_host_issued = false;  // a copy of the current x is in flight or done
    cudaStream_t out_stream = nullptr;
    cudaEvent_t out_ready = nullptr, out_copied = nullptr;

    // profiling
    bool profiling = false;
    // chunk timing (qcd_set_profiling(ctx, 2)): one event pair around each
    // queued chunk of FP32-level iterations, none around single launches;
    // chunk_bytes sums the algorithmic bytes of the launches issued
    bool chunk_timing = false;
    double chunk_bytes = 0.0;
    cudaEvent_t chunk_ev[2] = {nullptr, nullptr};
    struct Pending {
        cudaEvent_t a, b;
        int cls;
        double bytes;
    };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> event_pool;
    int *prof_flags = nullptr;       // device: 1 if the launch returned early
    int *prof_flags_host = nullptr;  // pinned mirror
    qcd_kernel_stat stats[QCD_K_COUNT] = {};
    long launches = 0;  // every kernel launch of this context

    // qcd_mult_benchmark buffers
    void *bench_buf = nullptr;
    size_t bench_bytes = 0;
    void *flush_buf = nullptr;

    // force: the per-site insertion matrices; adjoint solve: gamma5 g
    void *force_buf = nullptr;
    size_t force_bytes = 0;
    void *adj_buf = nullptr;

    // autotuned launch configurations of the stencil kernels, by tune_key
    struct TuneEntry {
        int variant;  // 0: compiler's register budget; 1: capped at 80 (DF64: 128); 2: pipelined hops
        int bx;       // threads per block along the sites
        double us;    // measured time of one launch
    };
    std::unordered_map<unsigned, TuneEntry> tune;
    void *tune_buf = nullptr;
    size_t tune_bytes = 0;

    // batched solves led by this context: problem descriptors, barrier words
    void *batch_buf = nullptr;
    size_t batch_bytes = 0;

    // lockstep multi-RHS solves: per-RHS vectors, states and partials
    void *multi_buf = nullptr;
    size_t multi_bytes = 0;
};

namespace qcd {

constexpr int NSTATES = 8;
constexpr int PROF_CAP = 1 << 16;  // profiled launches between two collections
enum StateSlot { ST_OUTER = 0, ST_MID = 1, ST_INNER = 2, ST_AUX = 3, ST_TUNE = 4 };

// allocation helpers (api.cu)
int dev_alloc(qcd_ctx *c, void **p, size_t bytes);
size_t hvec_bytes(const Geom &g, int prec);
int get_work(qcd_ctx *c, int prec, int slot, HVec *out);
int ensure_staging(qcd_ctx *c, size_t bytes);

// profiling (api.cu)
struct ProfScope {
    qcd_ctx *c;
    int cls;
    double bytes;
    cudaEvent_t a = nullptr, b = nullptr;
    int *flag = nullptr;  // device slot the kernel marks when it skips its work
    ProfScope(qcd_ctx *c_, int cls_, double bytes_);
    ~ProfScope();
};
int collect_profile(qcd_ctx *c);

// gauge.cu
int gauge_convert(qcd_ctx *c, const void *U_dev);
int clover_build(qcd_ctx *c, double kappa, double csw);

// stencil.cu
struct StencilCall {
    int prec = QCD_F64;
    int mode = M_MULT;
    int red = R_NONE;
    int dagger = 0;
    int out_par = 0;
    HVec out, in, y, aux, z;
    double a = 1.0, cc = 1.0, d = 0.0;
    int nrhs = 1;
    size_t rhs_stride = 0;  // sites*components stride between right-hand sides (elements of 16 bytes)
    size_t norm_stride = 0;
    RedArgs red_args;
    const int *done = nullptr;
    int force_variant = -1;  // >= 0: bypass the tuned configuration (autotuner)
    int force_bx = 128;
    // Lockstep multi-RHS solves: each right-hand side has its own solver
    // state (done flag every done_stride ints, reduction state red_args.st + r)
    // and, for a second half with fused dots, its own reduction: partials
    // red_args.partials + r red_pstride, counter red_args.counter + r.  With
    // rhs_grid the right-hand sides run as the fastest grid dimension.
    int done_stride = 0;
    size_t red_pstride = 0;
    bool rhs_grid = false;
};
int launch_stencil(qcd_ctx *c, const StencilCall &s);
unsigned tune_key(const StencilCall &s);
// F32 hopping / MULT on several right-hand sides: the shared-memory staged kernel
bool is_mrhs(const StencilCall &s);
double stencil_bytes(const qcd_ctx *c, const StencilCall &s);  // algorithmic bytes of one launch
int fill_pattern(qcd_ctx *c, int prec, HVec v, int nrhs, size_t rhs_stride, int seed);

// blas.cu -- conversions between canonical and internal layouts
int canon_to_half(qcd_ctx *c, int prec, int src_is_f32, const void *src, int parity_full, HVec dst, int nrhs, size_t rhs_stride);
int convert_half(qcd_ctx *c, HVec src, HVec dst);  // between precisions, one half vector
int half_to_canon(qcd_ctx *c, int prec, int dst_is_f32, HVec src, void *dst, int parity_full, int nrhs, size_t rhs_stride);
int clover_apply_half(qcd_ctx *c, int prec, int parity, int inverse, HVec in, HVec out, int nrhs, size_t rhs_stride);

// solver.cu
int solve(qcd_ctx *c, const void *b_dev, void *x_dev, double tol, const qcd_solve_opts &o, qcd_solve_info *info);
int solve_multi(qcd_ctx *c, const void *b_dev, void *x_dev, int nrhs, double tol, const qcd_solve_opts &o,
                qcd_solve_info *info);

// batched.cu
int batched_solve(qcd_ctx **ctxs, int n, const void *const *b, void *const *x, const double *tol,
                  const qcd_solve_opts &o, qcd_solve_info *infos, long long spin_limit, int use_graph);

// tune.cu
int autotune(qcd_ctx *c, const char *cache_path);
int l2_evict(qcd_ctx *c);  // read a 256 MB buffer: L2 holds nothing of earlier kernels
int tune_entries(qcd_ctx *c, int max, unsigned *keys, int *variant, int *bx, double *us);

// force.cu
int force(qcd_ctx *c, const void *x, const void *lam, void *G, const void *U_canon);
// correlator.cu
int pion_correlator(qcd_ctx *c, const void *S, int ncol, int on_device, double *C_host);
int gamma5_full(qcd_ctx *c, const void *in, void *out);

}  // namespace qcd
