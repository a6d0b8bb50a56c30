/*
 * qcd.h -- C ABI of the GB300 (sm_103a) library for the even-odd
 * preconditioned O(a)-improved (clover) Wilson operator and the nested
 * mixed-precision BiCGStab that solves with it.
 *
 * The paper this follows: Boku, Ishikawa, Kuramashi, Meadows, "Mixed
 * Precision Solver Scalable to 16000 MPI Processes for Lattice QCD
 * Simulations on the Oakforest-PACS System" (arXiv:1709.08785).
 *
 * Conventions used by every call
 * ------------------------------
 * Lattice: extents dims = {Lx, Ly, Lz, Lt}, every extent even and >= 2;
 *   site n = (x, y, z, t), lexicographic index s = x + Lx*(y + Ly*(z + Lz*t));
 *   parity (x+y+z+t) mod 2, 0 = even ("e"), 1 = odd ("o") (Sec. II-B).
 *   A half-lattice vector of parity p holds the sites of that parity in the
 *   order of cb = s/2.
 * Fields handed across the boundary (all canonical, row-major, interleaved
 *   complex, i.e. C99 double _Complex / float _Complex):
 *   gauge    U[s][mu][i][j], mu = x, y, z, t, U_mu(n) the link n -> n+mu,
 *            complex128, SU(3) (det U = 1 is assumed by the 12-real storage)
 *   spinor   psi[s][alpha][i], spin alpha = 0..3, colour i = 0..2
 *   half     psi[cb][alpha][i] on one parity
 * Gamma matrices: Dirac basis, gamma_k = [[0, -i s_k], [i s_k, 0]] (k = x,
 *   y, z), gamma_t = diag(1, 1, -1, -1) (gamma_t diagonal, Sec. II-A),
 *   gamma5 = gamma_x gamma_y gamma_z gamma_t = -[[0, 1], [1, 0]].
 * Operator (Sec. II-A, Eqs. 3-4):
 *   D = F - kappa H,
 *   H(n,m) = sum_mu (1 - gamma_mu) U_mu(n) delta_{n+mu,m}
 *                 + (1 + gamma_mu) U_mu(m)^dag delta_{n-mu,m},
 *   F(n) = 1 - (csw kappa / 2) sum_{mu != nu} sigma_munu F_munu(n),
 *   sigma_munu = (i/2)[gamma_mu, gamma_nu], F_munu = (Q_munu - Q_munu^dag)/(8i),
 *   Q_munu the sum of the four plaquette leaves around n (the clover term
 *   the paper cites; stored as two 6x6 Hermitian blocks, Sec. III-A).
 *   t_bc = -1 multiplies the hops that cross the time boundary by -1
 *   (antiperiodic quark fields); the clover term uses the unmodified links.
 *
 * Precisions: QCD_F64 operates on complex128 buffers; QCD_F32 on complex64
 *   buffers; QCD_F16 on complex64 buffers that are stored internally in IEEE
 *   half with one float scale per site (links and clover in half too) and
 *   operated on in FP32.
 *
 * Memory and streams: pointers marked "device" must be device memory of the
 *   context's device; all work is ordered on the context's stream; calls
 *   return when the work is enqueued unless stated otherwise.  The caller
 *   owns every buffer it passes; the context owns the gauge and clover
 *   fields and its workspaces.  A context is not thread-safe.
 * Errors: every call returns a qcd_status; on failure the output buffers
 *   are unspecified, the context stays usable, and qcd_last_error() gives a
 *   message for the calling thread.
 */
#ifndef QCD_GB300_H
#define QCD_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qcd_ctx qcd_ctx;

typedef enum {
    QCD_OK = 0,
    QCD_EINVAL = -1,            /* bad argument (null pointer, size, flag) */
    QCD_ECUDA = -2,             /* a CUDA runtime call failed */
    QCD_ENOMEM = -3,            /* device or host allocation failed */
    QCD_ENOTCONV = -4,          /* iteration cap reached before the tolerance */
    QCD_EBREAKDOWN = -5,        /* BiCGStab breakdown (rho or omega zero or non-finite) */
    QCD_ENONFINITE = -6,        /* non-finite input or intermediate */
    QCD_ECLOVER_SINGULAR = -7,  /* a clover block has a zero pivot */
    QCD_ETIMEOUT = -8,          /* a bounded device wait gave up */
    QCD_ESTATE = -9             /* call out of order (e.g. no gauge field loaded) */
} qcd_status;

/* QCD_DF64: FP64-sized storage, arithmetic in pairs of floats (double-float,
 * about 48 significant bits): the outer level of the mixed solvers, since
 * GB300 issues FP32 at about 64x its FP64 rate.  Operator calls with
 * QCD_DF64 take complex128 buffers. */
typedef enum { QCD_F64 = 0, QCD_F32 = 1, QCD_F16 = 2, QCD_DF64 = 3 } qcd_prec;

/* Create a context for one lattice on the current CUDA device.
 * dims: host array of 4 even extents >= 2 (Lx*Ly*Lz*Lt < 2^31).
 * t_bc: +1 periodic or -1 antiperiodic in time (Sec. II-A states periodic
 *       boundaries; antiperiodic time is the usual choice for quarks).
 * stream: a cudaStream_t (NULL = legacy default stream).
 * Errors: QCD_EINVAL for bad dims or t_bc. */
int qcd_create(qcd_ctx **ctx, const int dims[4], int t_bc, void *stream);
int qcd_destroy(qcd_ctx *ctx);
/* change the stream later calls are ordered on */
int qcd_set_stream(qcd_ctx *ctx, void *stream);

/* Load the gauge field U (canonical complex128 [V][4][3][3]), from device
 * memory (on_device = 1) or host memory (0), and build the internal copies:
 * FP64 with 18 reals per link, FP32 and FP16 with the first two columns
 * only (12 reals, SU(3) reconstruction, Sec. III-A) -- the conversion
 * [U, F] -> [U^SP, F^SP] of Alg. 1.  Invalidates the clover term.
 * Synchronous with respect to the host buffer (it may be reused on return). */
int qcd_gauge_load(qcd_ctx *ctx, const void *U, int on_device);

/* Build the clover term F and its site-local inverse F^-1 (Sec. II-B: F_ee,
 * F_oo are block diagonal and "inverted easily") in FP64 from the FP64
 * links, as two 6x6 Hermitian blocks per site in the chiral basis
 * (Sec. III-A), then round them to FP32 and FP16.
 * Errors: QCD_ESTATE without a gauge field; QCD_ECLOVER_SINGULAR if a block
 * has a (near-)zero pivot. */
int qcd_clover_build(qcd_ctx *ctx, double kappa, double csw);

/* out = H_{p,1-p} in (Eq. 4 restricted to one parity, Sec. II-B), or with
 * dagger = 1, gamma5 H gamma5 = H^dag.  out has parity out_parity, in the
 * opposite parity.  in/out: device half vectors, complex128 for QCD_F64 and
 * complex64 otherwise, nrhs of them back to back ([nrhs][Vh][4][3]).
 * The right-hand sides share every link load. */
int qcd_dslash_eo(qcd_ctx *ctx, void *out, const void *in, int out_parity, int dagger, int prec, int nrhs);

/* qcd_dslash_eo for callers that must not allocate device memory during the
 * call (the paper has no counterpart; this is an interface convenience).
 * qcd_dslash_eo stages its input and output through a buffer the context
 * allocates on first use; a real-time or serving loop whose allocator must
 * stay untouched after start-up, or a caller with a fixed memory budget or
 * a thread that must not synchronise the device (cudaMalloc/cudaFree can),
 * cannot take that allocation.  This variant stages through a fixed 24 MiB
 * device array that is part of the library itself (every GPU that loads the
 * library holds it until the process exits) and calls no cudaMalloc,
 * cudaFree or other allocating routine.  The context (qcd_create,
 * qcd_gauge_load) is still set up beforehand by the caller.
 * Limits: nrhs = 1; the input and output of one half vector must fit in
 * 24 MiB: Vh <= 65536 sites in QCD_F64 or QCD_DF64 (a 16^3 x 32 lattice),
 * more in the lower precisions; larger lattices return QCD_EINVAL.  The
 * context's device must be the current device (QCD_EINVAL otherwise): the
 * array has one address per device.
 * The first call on each device looks up the array's device address (with
 * that device current), and the first call with each precision and dagger
 * value lets the driver load the kernels it uses (with lazy module loading
 * the driver may take device memory for their code then); make these calls
 * during set-up, before any stream capture.  All
 * calls share the one array: calls that overlap on the GPU (other streams,
 * other contexts, other host threads) race; order them on one stream.
 * Same buffer conventions and result as qcd_dslash_eo. */
int qcd_dslash_eo_noalloc(qcd_ctx *ctx, void *out, const void *in, int out_parity, int dagger, int prec);

/* out = F_pp in (inverse = 0) or F_pp^-1 in (inverse = 1) on parity p.
 * Same buffer conventions as qcd_dslash_eo.  Needs qcd_clover_build. */
int qcd_clover_apply(qcd_ctx *ctx, void *out, const void *in, int parity, int inverse, int prec, int nrhs);

/* MULT (Sec. II-B): out = F_pp^-1 H_{p,1-p} in, the fused hopping + clover
 * inverse kernel the paper optimises (H~_eo, H~_oe); with dagger = 1 the
 * hopping term is gamma5 H gamma5.  Same buffer conventions. */
int qcd_mult_eo(qcd_ctx *ctx, void *out, const void *in, int out_parity, int dagger, int prec, int nrhs);

/* out = D^_ee in = in - kappa^2 H~_eo H~_oe in (Eq. 8; the printed
 * "H~_eo H~_eo" read as the Schur complement's H~_eo H~_oe), on even half
 * vectors.  Same buffer conventions (nrhs right-hand sides). */
int qcd_dhat(qcd_ctx *ctx, void *out, const void *in, int prec, int nrhs);

/* out = S_ee in = F_ee in - kappa^2 H_eo F_oo^-1 H_oe in, the Schur
 * complement of D on the even sites (Sec. II-B, Eqs. 5-8: D^_ee of Eq. 8 is
 * F_ee^-1 S_ee), which unlike D^_ee is gamma5-hermitian: S_ee^dag =
 * gamma5 S_ee gamma5.  Even half vectors, same buffer conventions as
 * qcd_dhat (nrhs right-hand sides).  Needs qcd_clover_build. */
int qcd_schur_ee(qcd_ctx *ctx, void *out, const void *in, int prec, int nrhs);

/* out = D in = F in - kappa H in on the full lattice (Eq. 3), FP64,
 * canonical complex128 [V][4][3] device buffers. */
int qcd_dirac(qcd_ctx *ctx, void *out, const void *in);

typedef struct {
    int precision_levels; /* 1: FP64 BiCGStab; 2: FP64 outer (Alg. 1) with
                             FP32 inner (Alg. 2); 3: FP64 outer, FP32
                             flexible middle, FP16-storage inner */
    int even_odd;         /* 1: solve D^_ee x_e = b^_e (Eqs. 5-7); 0: plain
                             BiCGStab on the full D (precision_levels 1 only) */
    double inner_tol[2];  /* |r| exit threshold of the inner levels on their
                             unit-norm right-hand side (Alg. 2); level 2, 3 */
    int max_outer;        /* iteration cap of the FP64 level */
    int max_inner[2];     /* iteration caps of the lower levels */
    int max_restarts;     /* restarts from the true residual (FP64) */
    int use_x0;           /* 1: x holds an initial guess; 0: x = 0 (Alg. 1) */
    int outer_df64;       /* arithmetic of the outer level (Alg. 1) when
                             precision_levels >= 2:
                             0: FP64 throughout;
                             1 (default): the solution x_e, the source b^_e
                                (Eq. 6) and the reconstruction x_o (Eq. 7)
                                are FP64 and accumulated in FP64 arithmetic;
                                the outer D^ applications and the iteration's
                                own vectors (r, r~, p, q, t, v) are QCD_DF64;
                             2: QCD_DF64 for all of the outer level.
                             Outer dot products and norms are summed in FP64
                             and the final true residual is FP64 in every
                             mode; QCD_EINVAL outside 0..2 */
    int eo_hermitian;     /* even_odd = 1: 0 (default) iterates on
                             D^_ee = 1 - kappa^2 F_ee^-1 H_eo F_oo^-1 H_oe
                             (Eq. 8); 1 on the gamma5-hermitian Schur
                             complement S_ee = F_ee D^_ee = F_ee - kappa^2
                             H_eo F_oo^-1 H_oe with right-hand side
                             b_e + kappa H_eo F_oo^-1 b_o (its residual is the
                             even part of b - D x itself); x_o as Eq. 7.
                             Every level uses the chosen operator.  Not
                             available to qcd_solve_batched (QCD_EINVAL) */
} qcd_solve_opts;

typedef struct {
    int status;            /* qcd_status of the solve */
    int outer_iters;       /* FP64-level iterations */
    int inner_iters[2];    /* iterations summed over the lower levels */
    int restarts;          /* true-residual restarts */
    long dhat_applies[3];  /* D^ (or D) applications by precision F64/F32/F16 */
    double true_resid;     /* ||b - D x|| / ||b|| in FP64 at exit */
    double seconds;        /* wall time of the call (device events) */
} qcd_solve_info;

/* Defaults: precision_levels 2, even_odd 1, inner_tol {1e-5, 1e-2},
 * max_outer 200, max_inner {250, 250}, max_restarts 5, use_x0 0,
 * outer_df64 1, eo_hermitian 0. */
void qcd_solve_opts_default(qcd_solve_opts *opts);

/* Solve D x = b to ||b - D x|| / ||b|| <= tol (recomputed in FP64 at exit;
 * a restart from the true residual follows if the recursive residual
 * drifted).  b, x: full-lattice complex128 [V][4][3], device or host memory
 * (host buffers are staged through the device inside the call; a host x
 * is copied out on a second stream of the context while the true residual
 * is checked, and is complete when the call returns).  The
 * nested scheme is Alg. 1 (flexible BiCGStab, FP64) around Alg. 2
 * (BiCGStab on a unit-norm right-hand side from x = 0, lower precision).
 * Blocks until the solve ends.  info may be NULL.
 * Errors: QCD_ESTATE without clover term; QCD_ENOTCONV, QCD_EBREAKDOWN,
 * QCD_ENONFINITE as the iteration ends; x then holds the last iterate. */
int qcd_solve(qcd_ctx *ctx, const void *b, void *x, double tol, const qcd_solve_opts *opts,
              qcd_solve_info *info);

/* Lockstep multi-RHS solves: nrhs systems D x_r = b_r on the context's gauge
 * field (e.g. the 12 spin-colour point sources of a propagator), each to
 * ||b_r - D x_r|| / ||b_r|| <= tol.  The nested scheme of qcd_solve (Alg. 1
 * around Alg. 2, Eqs. 5-7) runs for all right-hand sides together: every
 * FP32 iteration applies D^_ee (Eq. 8) to all of them at once -- the
 * multi-RHS MULT (Sec. II-B; the links and clover blocks of a site block
 * read once for all right-hand sides) and a second half whose blocks of one
 * site block's right-hand sides run together -- with each right-hand side's
 * own scalars, dot products and exit test; a converged right-hand side is
 * skipped.  (With fewer than 4 right-hand sides the MULT runs per
 * right-hand side: the staged kernel's tiles would leave the GPU short of
 * warps.)  Each x_r equals what qcd_solve returns for b_r, bit for bit.
 * b, x: device memory, nrhs canonical full-lattice complex128 vectors back
 * to back ([nrhs][V][4][3]); caller-owned.  infos: NULL or nrhs entries.
 * opts: precision_levels 2, even_odd 1, use_x0 0, outer_df64 0 or 1,
 * eo_hermitian 0 (anything else: QCD_EINVAL); 1 <= nrhs <= 16.  The
 * context keeps a workspace of about 16 FP64 and 7 FP32 half vectors per
 * right-hand side until it is destroyed.  Kernel timing (qcd_set_profiling)
 * does not bracket the lockstep second halves of D^.  Returns QCD_OK when
 * every right-hand side converged, else the first failing status (each
 * entry of infos has its own). */
int qcd_solve_multi(qcd_ctx *ctx, const void *b, void *x, int nrhs, double tol, const qcd_solve_opts *opts,
                    qcd_solve_info *infos);

/* Batched solves: n independent problems, problem i solving D_i x_i = b_i on
 * the lattice, gauge field and clover term of context ctxs[i] (distinct
 * contexts on one device; their lattices may differ), each to
 * ||b_i - D_i x_i|| / ||b_i|| <= tol[i].  The nested FP64/FP32 scheme of
 * Algs. 1-2 runs for all problems at once: every outer half-step is one
 * persistent cooperative kernel whose phases (the whole inner FP32
 * iteration, then the FP64 D^ and update) walk work tiles across all
 * lattices, with per-problem scalars and exit flags in device memory; the
 * two half-steps of an outer iteration are captured in a CUDA graph and
 * replayed until every problem has converged.  A problem whose true
 * residual misses its tolerance is restarted alone from its iterate.
 * b[i], x[i]: device, full-lattice complex128 [V_i][4][3].  opts: NULL or
 * precision_levels = 2, even_odd = 1, use_x0 = 0 (inner_tol[0], max_outer,
 * max_inner[0] are used).  infos: NULL or n entries (seconds = the whole
 * batch).  Work is ordered on ctxs[0]'s stream; synchronous.
 * Errors: QCD_ETIMEOUT if a grid barrier gave up (see qcd_set_wait_limit);
 * the first failing problem's status otherwise. */
int qcd_solve_batched(qcd_ctx *const *ctxs, int n, const void *const *b, void *const *x, const double *tol,
                      const qcd_solve_opts *opts, qcd_solve_info *infos);

/* Every device-side wait of the library (the grid barriers of the batched
 * kernel) spins at most this many times (about 100 ns each) before it
 * records QCD_ETIMEOUT and the kernel returns; default 1e7 (about a second).
 * Process-wide. */
int qcd_set_wait_limit(long long spins);

/* Use CUDA graphs for the batched solver's replayed launches (1, default) or
 * launch directly (0).  Process-wide. */
int qcd_set_graphs(int on);

/* lambda = D^-dag g, through gamma5-hermiticity D^dag = gamma5 D gamma5
 * (F commutes with gamma5 and H^dag = gamma5 H gamma5, Eq. 4): lambda =
 * gamma5 D^-1 gamma5 g, solved by qcd_solve with the same options.  g, lam:
 * device, full-lattice complex128 [V][4][3].  Used by the backward pass of a
 * solve: for x = D^-1 b and a real loss with gradient g with respect to x,
 * the gradient with respect to b is lambda.  Returns qcd_solve's status. */
int qcd_solve_adjoint(qcd_ctx *ctx, const void *g, void *lam, double tol, const qcd_solve_opts *opts,
                      qcd_solve_info *info);

/* Link gradient ("force"): G = df/dRe U + i df/dIm U of
 * f(U) = -Re <lam, D[U] x> with x and lam held fixed -- for x = D^-1 b and
 * lam = D^-dag g this is the gradient of a real loss with respect to the
 * links (the convention torch uses for complex tensors).  Both the hopping
 * term (Eq. 4; outer products of lam and the spin-projected x across each
 * link) and the clover term (the plaquette leaves with the spin-traced
 * insertion Tr_spin[sigma_munu x lam^dag] at each corner) contribute.
 * U: the device gauge field in canonical layout (the one loaded); x, lam:
 * device complex128 [V][4][3]; G: device complex128 [V][4][3][3]. FP64. */
int qcd_force(qcd_ctx *ctx, const void *U, const void *x, const void *lam, void *G);

/* Kernel timing.  qcd_set_profiling(ctx, 1): each launch of the operator
 * and BLAS kernels is bracketed by CUDA events on the context stream and
 * qcd_kernel_stats sums them by class (a bracketed launch cannot overlap
 * its predecessor, so its time includes its own launch latency).
 * qcd_set_profiling(ctx, 2): chunk timing -- one event pair around each
 * chunk of FP32-level BiCGStab iterations the solver queues, the launches
 * inside left back to back as in any solve; the class QCD_K_INNER_ITER then
 * sums whole iterations (launches = iterations, their algorithmic bytes).
 * 0 turns timing off.  QCD_EINVAL for other values. */
typedef enum {
    QCD_K_MULT_F64 = 0,  /* stencil kernels (MULT, D^, b^, x_o, D), by precision; */
    QCD_K_MULT_F32 = 1,  /* FP32: all but the second half of D^, which is QCD_K_DHAT_F32 */
    QCD_K_MULT_F16 = 2,
    QCD_K_BLAS = 3,      /* fused BLAS-1 + reduction kernels (all but the FP32 level's) */
    QCD_K_OTHER = 4,
    QCD_K_DHAT_F32 = 5,  /* FP32 second half of D^ with its fused update and dot products */
    QCD_K_MULT_DF64 = 6, /* DF64 stencil kernels */
    QCD_K_BLAS_F32 = 7,  /* fused BLAS-1 + reduction kernels of the FP32 level */
    QCD_K_INNER_ITER = 8, /* whole FP32-level BiCGStab iterations (chunk timing, see
                             qcd_set_profiling): launches = iterations */
    QCD_K_COUNT = 9
} qcd_kernel_class;

typedef struct {
    long launches;
    double ms;     /* summed device time */
    double bytes;  /* summed algorithmic bytes */
} qcd_kernel_stat;

int qcd_set_profiling(qcd_ctx *ctx, int on);
int qcd_kernel_stats(qcd_ctx *ctx, int kernel_class, qcd_kernel_stat *out);
int qcd_reset_kernel_stats(qcd_ctx *ctx);

/* Number of kernels this context has launched since it was created. */
long qcd_launch_count(const qcd_ctx *ctx);

/* Autotune the launch configurations of the operator kernels the solvers
 * use (register budget and threads per block -- or, for the multi-RHS
 * kernel, right-hand sides per block -- for each precision,
 * fused reduction and right-hand-side count): every candidate is timed on scratch
 * buffers, with L2 evicted, and the fastest kept for this context.  If
 * cache_path is not NULL the choices are read from and added to that JSON
 * file, keyed by device name, lattice extents and configuration, so a later
 * context tunes nothing it finds there.  Needs qcd_clover_build.
 * Synchronous. */
int qcd_autotune(qcd_ctx *ctx, const char *cache_path);

/* The tuned configurations: up to max entries (key; variant: 0 the
 * compiler's register budget, 1 capped at 80 registers (128 for QCD_DF64),
 * 2 the FP32 / FP16 kernel whose hops are software-pipelined (the next
 * hop's neighbour spinor and link loaded before the current hop computes);
 * threads per block along the sites, or
 * right-hand sides per block for the multi-RHS kernel; microseconds per
 * launch); returns the number of entries held. Any output pointer may be
 * NULL. */
int qcd_tune_info(qcd_ctx *ctx, int max, unsigned *keys, int *variant, int *threads, double *us);

/* Time the fused MULT kernel (Sec. II-B, out = F^-1 H_{p,1-p} in) alone on
 * internal, already-resident buffers: `iters` launches on nrhs right-hand
 * sides (nrhs <= 16) in precision prec, each launch bracketed by CUDA
 * events and preceded by a read of a 256 MB buffer that evicts L2 (clean
 * lines replace the cache contents, so no write-back of earlier kernels'
 * data falls inside the timed launch).  Returns the mean device time of one
 * launch and its algorithmic bytes (each input read once, the output
 * written once).  Synchronous.  Needs the clover term (QCD_ESTATE);
 * QCD_EINVAL for a NULL output pointer, prec outside 0..3, nrhs outside
 * 1..16 or iters < 1.  Allocates two nrhs-vector buffers and the flush
 * buffer on first use. */
int qcd_mult_benchmark(qcd_ctx *ctx, int prec, int nrhs, int iters, double *ms_per_launch,
                       double *bytes_per_launch);

/* As qcd_mult_benchmark, but `iters` launches back to back with one pair of
 * CUDA events around all of them and no eviction in between: the rate of a
 * stream of MULTs, as inside a solver (the input vector stays in L2 from one
 * launch to the next; the links and clover, larger than L2 at production
 * sizes, stream from HBM).  Returns the mean time of one launch, launch
 * gaps included, and its algorithmic bytes.  Same arguments and errors. */
int qcd_mult_throughput(qcd_ctx *ctx, int prec, int nrhs, int iters, double *ms_per_launch,
                        double *bytes_per_launch);

/* Pion two-point function from propagator columns (Sec. II-A: the solutions
 * of Eq. 1 feed expectation values of observables made of quarks).  S holds
 * ncol full-lattice solutions one after another, each complex128 in the
 * canonical layout of qcd_solve's x ([V][spin 4][colour 3], V in the order
 * [t][z][y][x]), on the device (on_device != 0) or in host memory.  With S the
 * 12 spin-colour columns of the propagator from a point source,
 * gamma5-hermiticity makes the pion correlator
 *     C(t) = sum_columns sum_{x in timeslice t} sum_{spin,colour} |S(x)|^2,
 * which is written to the host array C[Lt] (caller-owned).  Sums run in
 * FP64 in a fixed order (bitwise repeatable).  Synchronous.  QCD_EINVAL for a
 * NULL pointer or ncol < 1; host columns are staged one at a time through a
 * device buffer of one column. */
int qcd_pion_correlator(qcd_ctx *ctx, const void *S, int ncol, int on_device, double *C);

const char *qcd_strerror(int status);
const char *qcd_last_error(void);

/* number of sites and of sites per parity of the context's lattice */
long qcd_volume(const qcd_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* QCD_GB300_H */
