// Solver drivers: the nested BiCGStab of Algs. 1-2 (FP64 flexible outer
// iteration around a lower-precision BiCGStab on a unit-norm right-hand
// side), its three-level form (FP64 / FP32 / FP16 storage), the plain FP64
// BiCGStab on D^_ee, and the unpreconditioned FP64 BiCGStab on D.
//
// Every scalar lives in device memory (SolverState); the host only queues
// kernels.  A lower level's iterations are queued in chunks whose size is
// predicted from the convergence rate so far; kernels queued past
// convergence see the state marked done and return at once.  The host reads
// the state back once per chunk and once per half-iteration of the FP64
// level.
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "blas.cuh"

namespace qcd {

namespace {

// bd_eps of the breakdown test |rho1| <= bd_eps |r~| |r| (the paper has
// none; FP64 levels use 1e-30, lower precisions 1e-12)
constexpr double BD_EPS_F64 = 1e-30;
constexpr double BD_EPS_LOW = 1e-12;

struct Level {
    int prec = QCD_F64;
    int form = 0;                    // 0: D^_ee (Eq. 8); 1: S_ee = F_ee D^_ee (gamma5-hermitian)
    HVec x, r, rt, p, q, t, v, tmp;  // tmp: odd-parity workspace of D^
    SolverState *st = nullptr;       // device
    int slot = 0;                    // index into the state arrays
};

int read_state(qcd_ctx *c, int slot, SolverState *out)
{
    QCD_CUDA_CHECK(cudaMemcpyAsync(c->states_host + slot, c->states + slot, sizeof(SolverState), cudaMemcpyDeviceToHost,
                                   c->stream));
    QCD_CUDA_CHECK(cudaStreamSynchronize(c->stream));
    *out = c->states_host[slot];
    return QCD_OK;
}

#define TRY(x)                     \
    do {                           \
        int rc__ = (x);            \
        if (rc__ != QCD_OK) return rc__; \
    } while (0)

// out = D^ in = in - kappa^2 F_ee^-1 H_eo F_oo^-1 H_oe in (Eq. 8), or for
// form 1 the gamma5-hermitian S_ee in = F_ee in - kappa^2 H_eo F_oo^-1 H_oe in,
// with a reduction fused into the second half.
int dhat(qcd_ctx *c, int prec, HVec in, HVec out, HVec tmp, int red, HVec aux, SolverState *st, int fin,
         const int *done, int form)
{
    StencilCall s1;
    s1.prec = prec;
    s1.mode = M_MULT;
    s1.out_par = 1;
    s1.out = tmp;
    s1.in = in;
    s1.done = done;
    TRY(launch_stencil(c, s1));
    StencilCall s2;
    s2.prec = prec;
    s2.mode = form ? M_FULL : M_DHAT;  // F_ee in (M_FULL) or in (M_DHAT), minus kappa^2 [F_ee^-1] H_eo tmp
    s2.out_par = 0;
    s2.out = out;
    s2.in = tmp;
    s2.y = in;
    s2.a = 1.0;
    s2.cc = -c->kappa * c->kappa;
    s2.red = red;
    s2.aux = aux;
    s2.red_args.partials = c->partials;
    s2.red_args.counter = c->counters;
    s2.red_args.st = st;
    s2.red_args.op = fin;
    s2.done = done;
    return launch_stencil(c, s2);
}

// One iteration of Alg. 2 on level L (all in L.prec).
int bicg_iteration(qcd_ctx *c, Level &L)
{
    const int n = c->g.Vh_pad;
    const int *done = &L.st->done;
    TRY(dhat(c, L.prec, L.p, L.q, L.tmp, R_DOT_AUX, L.rt, L.st, FIN_ALPHA, done, L.form));  // q = D^ p, alpha
    TRY(blas_update_s(c, L.prec, n, L.r, L.q, L.st));                              // s = r - alpha q
    TRY(dhat(c, L.prec, L.r, L.t, L.tmp, R_OMEGA, L.r, L.st, FIN_OMEGA, done, L.form));     // t = D^ s, omega
    TRY(blas_update_x(c, L.prec, n, L.x, L.p, L.r, L.t, L.rt, L.st));              // x, r, beta
    TRY(blas_update_p(c, L.prec, n, L.p, L.r, L.q, L.st, FIN_NONE));               // p
    return QCD_OK;
}

// Run Alg. 2 iterations on L until its state is done; returns the
// iterations executed.
int run_bicg(qcd_ctx *c, Level &L, SolverState *final_state)
{
    SolverState h;
    int queued = 0;
    int chunk = 3;
    double rr0 = -1.0;
    // chunk timing of the FP32 level: the launches of a chunk run back to
    // back as in any solve, one event pair around them
    const bool timed = c->chunk_timing && L.prec == QCD_F32;
    int it_before = 0;
    for (;;) {
        const double by0 = c->chunk_bytes;
        if (timed) QCD_CUDA_CHECK(cudaEventRecord(c->chunk_ev[0], c->stream));
        for (int k = 0; k < chunk; ++k) TRY(bicg_iteration(c, L));
        if (timed) QCD_CUDA_CHECK(cudaEventRecord(c->chunk_ev[1], c->stream));
        queued += chunk;
        TRY(read_state(c, L.slot, &h));
        if (timed) {
            float ms = 0.f;
            QCD_CUDA_CHECK(cudaEventElapsedTime(&ms, c->chunk_ev[0], c->chunk_ev[1]));
            // iterations the chunk ran (the queue may overrun convergence:
            // those launches return at once and move no data)
            const int ran = h.iter - it_before;
            it_before = h.iter;
            qcd_kernel_stat &k = c->stats[QCD_K_INNER_ITER];
            k.launches += ran;
            k.ms += ms;
            k.bytes += (c->chunk_bytes - by0) * ran / chunk;
        }
        if (rr0 < 0.0) rr0 = h.rr > 0 ? h.rr : 1.0;
        if (h.done) break;
        if (queued > h.maxit + 8) {  // cannot happen: FIN_X caps at maxit
            set_error_message("iteration queue overran the cap");
            return QCD_ETIMEOUT;
        }
        // predict the remaining iterations from the mean contraction so far
        int pred = 8;
        if (h.iter > 0 && h.rr > 0.0 && h.rr < rr0 && h.tol2 > 0.0) {
            const double rate = std::log(h.rr / rr0) / h.iter;  // < 0
            pred = (int)std::ceil(std::log(h.tol2 / h.rr) / rate);
        }
        if (pred < 2) pred = 2;
        if (pred > 64) pred = 64;
        if (pred > h.maxit - h.iter + 1) pred = h.maxit - h.iter + 1;
        chunk = pred < 1 ? 1 : pred;
    }
    TRY(blas_finish_half(c, L.prec, c->g.Vh_pad, L.x, L.p, L.st));
    *final_state = h;
    return QCD_OK;
}

// ||b - D x|| / ||b|| from norm2[2] = |b - D x|^2 and norm2[0] = |b|^2;
// non-finite if either is; 0 for b = 0 (x = 0 is then exact)
double resid_ratio(const SolverState &a)
{
    const double b2 = a.norm2[0], r2 = a.norm2[2];
    if (!std::isfinite(b2) || !std::isfinite(r2)) return NAN;
    if (b2 == 0.0) return r2 == 0.0 ? 0.0 : INFINITY;
    return std::sqrt(r2 / b2);
}

struct Solver {
    qcd_ctx *c;
    qcd_solve_opts o;
    qcd_solve_info info;
    Level lv[3];  // 0: FP64, 1: FP32, 2: FP16
    HVec be, bo, bhat, xo, re, ro;
    HVec bhat0;  // b^_e in the outer operator's precision (residual restarts)
    SolverState *aux;
};

int get_level(qcd_ctx *c, Level &L, int prec, int first_slot, int state_slot, int form)
{
    L.prec = prec;
    L.form = form;
    HVec *v[8] = {&L.x, &L.r, &L.rt, &L.p, &L.q, &L.t, &L.v, &L.tmp};
    for (int k = 0; k < 8; ++k) TRY(get_work(c, prec, first_slot + k, v[k]));
    L.slot = state_slot;
    L.st = c->states + state_slot;
    return QCD_OK;
}

// v = M src: the lower levels approximately solve D^ v = src (Alg. 2, and
// for three levels the flexible FP32 middle level around it).
int precondition(Solver &S, int level, HVec src, int src_prec, const double *src_norm2, HVec v, const int *done);

// Alg. 1 on level `lev` (flexible BiCGStab, preconditioned by the level
// below), from the state already initialised by blas_init.
int flexible(Solver &S, int lev)
{
    qcd_ctx *c = S.c;
    Level &L = S.lv[lev];
    const int n = c->g.Vh_pad;
    const int *done = &L.st->done;
    SolverState h;
    TRY(read_state(c, L.slot, &h));
    if (h.done) return QCD_OK;
    for (;;) {
        TRY(precondition(S, lev + 1, L.p, L.prec, &L.st->norm2[1], L.v, done));      // v = M p
        TRY(dhat(c, L.prec, L.v, L.q, L.tmp, R_DOT_AUX, L.rt, L.st, FIN_ALPHA, done, L.form));  // q = D^ v, alpha
        TRY(blas_flex1(c, L.prec, n, L.x, L.v, L.r, L.q, L.st));                       // x, r, |r|
        S.info.dhat_applies[L.prec == QCD_DF64 ? QCD_F64 : L.prec] += 1;  // DF64 counts as the FP64 level
        TRY(read_state(c, L.slot, &h));
        if (h.done) break;
        TRY(precondition(S, lev + 1, L.r, L.prec, &L.st->rr, L.v, done));                // v = M r
        TRY(dhat(c, L.prec, L.v, L.t, L.tmp, R_OMEGA, L.r, L.st, FIN_OMEGA, done, L.form));      // t = D^ v, omega
        TRY(blas_flex2(c, L.prec, n, L.x, L.v, L.r, L.t, L.rt, L.st));                  // x, r, beta
        TRY(blas_update_p(c, L.prec, n, L.p, L.r, L.q, L.st, FIN_SETN + 1));             // p, |p|
        S.info.dhat_applies[L.prec == QCD_DF64 ? QCD_F64 : L.prec] += 1;
        TRY(read_state(c, L.slot, &h));
        if (h.done) break;
    }
    return QCD_OK;
}

int precondition(Solver &S, int level, HVec src, int src_prec, const double *src_norm2, HVec v, const int *done)
{
    qcd_ctx *c = S.c;
    Level &L = S.lv[level];
    const int n = c->g.Vh_pad;
    const bool last = level == S.o.precision_levels - 1;
    const double tol = S.o.inner_tol[level - 1];
    TRY(state_init(c, L.st, tol * tol, 0.0, S.o.max_inner[level - 1], BD_EPS_LOW, 1));
    TRY(blas_inner_init(c, src_prec, L.prec, n, src, src_norm2, L.r, L.rt, L.p, L.x, done));
    SolverState h;
    if (last) {
        TRY(run_bicg(c, L, &h));
        S.info.inner_iters[level - 1] += h.iter;
        S.info.dhat_applies[L.prec] += 2L * h.iter - h.exit_half;
    } else {
        // the middle level is itself flexible (Alg. 1 in FP32) and needs
        // norm2[1] = |p|^2 = 1 of its unit-norm start
        TRY(flexible(S, level));
        TRY(read_state(c, L.slot, &h));
        S.info.inner_iters[level - 1] += h.iter;
    }
    return blas_lift(c, L.prec, src_prec, n, L.x, v, src_norm2, done);
}

int residual_eo(Solver &S, HVec xe, HVec out, SolverState *st, int fin)
{
    // out = b^ - D^ x_e = b^ - x_e + kappa^2 H~_eo H~_oe x_e (or for the
    // gamma5-hermitian form src - F_ee x_e + kappa^2 H_eo F_oo^-1 H_oe x_e),
    // in the outer level's arithmetic
    qcd_ctx *c = S.c;
    Level &L = S.lv[0];
    StencilCall s1;
    s1.prec = L.prec;
    s1.mode = M_MULT;
    s1.out_par = 1;
    s1.out = L.tmp;
    s1.in = xe;
    TRY(launch_stencil(c, s1));
    StencilCall s2;
    s2.prec = L.prec;
    s2.mode = L.form ? M_FULL : M_DHAT;
    s2.out_par = 0;
    s2.out = out;
    s2.in = L.tmp;
    s2.y = xe;
    s2.a = -1.0;
    s2.cc = c->kappa * c->kappa;
    s2.z = S.bhat0;
    s2.d = 1.0;
    s2.red = R_NORM;
    s2.red_args = RedArgs{c->partials, c->counters, st, fin};
    return launch_stencil(c, s2);
}

// ||b - D x||^2 of the full solution (x_e, x_o) into aux->norm2[2], in
// precision P (every vector, S.re and S.ro included, of that precision)
int true_residual(Solver &S, int P, HVec xe, HVec xo, HVec be, HVec bo)
{
    qcd_ctx *c = S.c;
    for (int par = 0; par < 2; ++par) {
        StencilCall s;
        s.prec = P;
        s.mode = M_FULL;
        s.out_par = par;
        s.out = par ? S.ro : S.re;
        s.in = par ? xe : xo;
        s.y = par ? xo : xe;
        s.a = -1.0;
        s.cc = c->kappa;
        s.z = par ? bo : be;
        s.d = 1.0;
        s.red = R_NORM;
        s.red_args = RedArgs{c->partials, c->counters, S.aux, par ? FIN_ADDN + 2 : FIN_SETN + 2};
        TRY(launch_stencil(c, s));
    }
    return QCD_OK;
}

// |b_e - (D x)_e|^2 = |b_e - F_ee x_e + kappa H_eo x_o|^2 in FP64, added to
// aux->norm2[2], which the reconstruction pass (M_RECON) set to the odd rows'
int residual_even(Solver &S, HVec xe, HVec xo)
{
    qcd_ctx *c = S.c;
    StencilCall s;
    s.prec = QCD_F64;
    s.mode = M_FULL;
    s.out_par = 0;
    s.out = S.re;
    s.in = xo;
    s.y = xe;
    s.a = -1.0;
    s.cc = c->kappa;
    s.z = S.be;
    s.d = 1.0;
    s.red = R_NORM;
    s.red_args = RedArgs{c->partials, c->counters, S.aux, FIN_ADDN + 2};
    return launch_stencil(c, s);
}

// x (canonical FP64, device) from the half vectors; when the caller's x is
// in host memory, its copy is issued on the output stream at once, so that
// it overlaps the true-residual check that follows.  A later emission (after
// a restart) first waits for that copy to finish.
int emit_x(qcd_ctx *c, HVec xe, HVec xo, void *x)
{
    if (c->x_host && c->x_host_issued) QCD_CUDA_CHECK(cudaStreamWaitEvent(c->stream, c->out_copied, 0));
    TRY(half_to_canon(c, QCD_F64, 0, xe, x, 0, 1, 0));
    TRY(half_to_canon(c, QCD_F64, 0, xo, x, 1, 1, 0));
    if (c->x_host) {
        QCD_CUDA_CHECK(cudaEventRecord(c->out_ready, c->stream));
        QCD_CUDA_CHECK(cudaStreamWaitEvent(c->out_stream, c->out_ready, 0));
        QCD_CUDA_CHECK(cudaMemcpyAsync(c->x_host, x, c->x_host_bytes, cudaMemcpyDeviceToHost, c->out_stream));
        QCD_CUDA_CHECK(cudaEventRecord(c->out_copied, c->out_stream));
        c->x_host_issued = true;
    }
    return QCD_OK;
}

int solve_eo(Solver &S, const void *b, void *x, double tol)
{
    qcd_ctx *c = S.c;
    const int n = c->g.Vh_pad;
    Level &O = S.lv[0];
    // Precisions of the outer level (Alg. 1).  P0: the outer D^ and the
    // iteration's own vectors r, r~, p, q, t, v.  PX: the solution x_e, the
    // source b^_e (Eq. 6) and the reconstruction x_o (Eq. 7).
    //   outer_df64 = 0: P0 = PX = FP64 (Alg. 1 as printed);
    //   outer_df64 = 1: P0 = DF64, PX = FP64 -- the solution is accumulated
    //                   in FP64 arithmetic, the operator applications and the
    //                   recursions run in float pairs (GB300's FP64 rate is
    //                   ~1/64 of its FP32 rate);
    //   outer_df64 = 2: P0 = PX = DF64.
    // Dot products and norms of the outer level are summed in FP64 in every
    // mode, and the true-residual check ||b - D x|| that decides convergence
    // is FP64 from the FP64 links and clover term.
    const int mode = S.o.precision_levels >= 2 ? S.o.outer_df64 : 0;
    // the even-odd operator: D^_ee of Eq. 8 (form 0) or the gamma5-hermitian
    // S_ee = F_ee D^_ee (form 1), whose right-hand side is F_ee b^_e =
    // b_e + kappa H_eo F_oo^-1 b_o and whose residual is the even part of the
    // full residual itself
    const int form = S.o.eo_hermitian ? 1 : 0;
    const int P0 = mode ? QCD_DF64 : QCD_F64;
    const int PX = mode == 2 ? QCD_DF64 : QCD_F64;
    TRY(get_work(c, QCD_F64, 0, &S.be));
    TRY(get_work(c, QCD_F64, 1, &S.bo));
    TRY(get_work(c, QCD_F64, 3, &S.xo));
    TRY(get_work(c, QCD_F64, 4, &S.re));
    TRY(get_work(c, QCD_F64, 5, &S.ro));
    TRY(get_work(c, PX, 2, &S.bhat));
    TRY(get_level(c, O, P0, 6, ST_OUTER, form));
    HVec beX = S.be, boX = S.bo, xoX = S.xo, xe64 = O.x, xe0 = O.x, tmpX = O.tmp;
    S.bhat0 = S.bhat;
    if (PX != QCD_F64) {  // all-DF64 outer level: DF64 copies of b_e, b_o, x_o
        TRY(get_work(c, PX, 0, &beX));
        TRY(get_work(c, PX, 1, &boX));
        TRY(get_work(c, PX, 3, &xoX));
        TRY(get_work(c, QCD_F64, 6, &xe64));
    }
    if (PX != P0) {  // FP64 solution around a DF64 iteration
        TRY(get_work(c, QCD_F64, 6, &O.x));  // x_e in FP64
        xe64 = O.x;
        TRY(get_work(c, P0, 2, &S.bhat0));   // b^_e rounded to DF64
        tmpX = S.re;                          // FP64 scratch before the true residual needs it
    }
    if (S.o.precision_levels >= 2) TRY(get_level(c, S.lv[1], QCD_F32, 0, ST_MID, form));
    if (S.o.precision_levels >= 3) TRY(get_level(c, S.lv[2], QCD_F16, 0, ST_INNER, form));
    S.aux = c->states + ST_AUX;

    // b -> (b_e, b_o); |b|^2
    TRY(canon_to_half(c, QCD_F64, 0, b, 0, S.be, 1, 0));
    TRY(canon_to_half(c, QCD_F64, 0, b, 1, S.bo, 1, 0));
    TRY(state_init(c, S.aux, 0.0, 0.0, 0, 0.0, 0));
    TRY(blas_norm2(c, QCD_F64, n, S.be, S.aux, FIN_SETN + 0));
    TRY(blas_norm2(c, QCD_F64, n, S.bo, S.aux, FIN_ADDN + 0));
    if (PX != QCD_F64) {
        TRY(convert_half(c, S.be, beX));
        TRY(convert_half(c, S.bo, boX));
    }
    // b^_e = F_ee^-1 (b_e + kappa H_eo F_oo^-1 b_o)   (Eq. 6, Alg. 1 line 3),
    // for form 1 without the left F_ee^-1
    TRY(clover_apply_half(c, PX, 1, 1, boX, tmpX, 1, 0));
    {
        StencilCall s;
        s.prec = PX;
        s.out_par = 0;
        s.out = S.bhat;
        s.in = tmpX;
        s.y = beX;
        s.cc = c->kappa;
        if (form) {  // 0 F_ee b_e + kappa H_eo tmp + b_e
            s.mode = M_FULL;
            s.a = 0.0;
            s.z = beX;
            s.d = 1.0;
        } else {
            s.mode = M_SRC;
            s.a = 1.0;
        }
        TRY(launch_stencil(c, s));
    }
    if (PX != P0) TRY(convert_half(c, S.bhat, S.bhat0));
    // x_e in the operator's precision, for a recomputed residual b^ - D^ x_e
    auto x_for_operator = [&]() -> int {
        if (PX == P0) return QCD_OK;
        TRY(get_work(c, P0, 6, &xe0));
        return convert_half(c, O.x, xe0);
    };
    // the recursive residual |r^_e| is driven below tol |b| / 2: the full
    // residual is F_ee r^_e with |F_ee| close to one; the true residual
    // is checked at the end and the iteration restarted from it if needed
    const int maxit = S.o.max_outer;
    TRY(state_init(c, O.st, 0.0, 0.0, maxit, BD_EPS_F64, 0));
    TRY(set_tol2(c, O.st, S.aux, 0, 0.25 * tol * tol));
    if (S.o.use_x0) {
        TRY(canon_to_half(c, PX, 0, x, 0, O.x, 1, 0));
        TRY(x_for_operator());
        TRY(residual_eo(S, xe0, O.r, O.st, FIN_NONE));
        TRY(blas_init(c, P0, n, O.r, O.r, O.rt, O.p, O.x, 0, O.st, FIN_INIT));
    } else {
        // x_e = 0: a zero complex is all zero bits in the FP64 and DF64
        // layouts alike, so the DF64 init clears an FP64 x_e as well
        TRY(blas_init(c, P0, n, S.bhat0, O.r, O.rt, O.p, O.x, 1, O.st, FIN_INIT));
    }
    SolverState h, ha;
    int status = QCD_OK;
    for (int restart = 0;; ++restart) {
        if (S.o.precision_levels == 1) {
            TRY(run_bicg(c, O, &h));
            S.info.dhat_applies[QCD_F64] += 2L * h.iter - h.exit_half;
        } else {
            TRY(flexible(S, 0));
            TRY(read_state(c, O.slot, &h));
        }
        S.info.outer_iters = h.iter;
        status = h.status;
        // x_o = F_oo^-1 (b_o + kappa H_oe x_e)   (Eq. 7, Alg. 1 line 19); with
        // an FP64 solution the same pass yields the odd rows of the FP64
        // true residual b - D x, so that only the even rows need a pass of
        // their own
        StencilCall s;
        s.prec = PX;
        s.mode = PX == QCD_F64 ? M_RECON : M_SRC;
        s.out_par = 1;
        s.out = xoX;
        s.in = O.x;
        s.y = boX;
        s.a = 1.0;
        s.cc = c->kappa;
        if (PX == QCD_F64) {
            s.red = R_NORM;
            s.red_args = RedArgs{c->partials, c->counters, S.aux, FIN_SETN + 2};  // |r_o|^2
        }
        TRY(launch_stencil(c, s));
        if (PX != QCD_F64) {
            TRY(convert_half(c, O.x, xe64));
            TRY(convert_half(c, xoX, S.xo));
        }
        TRY(emit_x(c, xe64, S.xo, x));
        if (PX == QCD_F64) TRY(residual_even(S, xe64, S.xo));
        else TRY(true_residual(S, QCD_F64, xe64, S.xo, S.be, S.bo));
        TRY(read_state(c, ST_AUX, &ha));
        S.info.true_resid = resid_ratio(ha);
        if (!std::isfinite(S.info.true_resid)) {
            status = QCD_ENONFINITE;
            break;
        }
        if (S.info.true_resid <= tol) {
            status = QCD_OK;
            break;
        }
        if (status == QCD_ENONFINITE) break;
        if (restart >= S.o.max_restarts || h.iter >= maxit) {
            if (status == QCD_OK) status = QCD_ENOTCONV;
            break;
        }
        // restart from the recomputed residual r = b^ - D^ x_e
        S.info.restarts += 1;
        TRY(state_init(c, O.st, 0.0, 0.0, maxit, BD_EPS_F64, 0));
        TRY(set_tol2(c, O.st, S.aux, 0, 0.25 * tol * tol));
        TRY(x_for_operator());
        TRY(residual_eo(S, xe0, O.r, O.st, FIN_NONE));
        TRY(blas_init(c, P0, n, O.r, O.r, O.rt, O.p, O.x, 0, O.st, FIN_RESTART));
    }
    return status;
}

// Unpreconditioned FP64 BiCGStab on the full D (both parities as one vector
// of 2*Vh_pad sites).
int solve_full(Solver &S, const void *b, void *x, double tol)
{
    qcd_ctx *c = S.c;
    const int n = 2 * c->g.Vh_pad;
    const size_t hb = hvec_bytes(c->g, QCD_F64);
    HVec F[8];  // b, x, r, rt, p, q, t, spare : each two halves
    for (int k = 0; k < 8; ++k) {
        TRY(get_work(c, QCD_F64, 2 * k, &F[k]));
        HVec odd;
        TRY(get_work(c, QCD_F64, 2 * k + 1, &odd));
        if ((char *)odd.p != (char *)F[k].p + hb) {
            set_error_message("workspace halves not contiguous");
            return QCD_ESTATE;
        }
    }
    auto half = [&](HVec v, int par) {
        HVec h = v;
        if (par) h.p = (char *)v.p + hb;
        return h;
    };
    HVec &B = F[0], &X = F[1], &R = F[2], &RT = F[3], &P = F[4], &Q = F[5], &T = F[6];
    SolverState *st = c->states + ST_OUTER;
    const int *done = &st->done;
    auto applyD = [&](HVec in, HVec out) -> int {
        for (int par = 0; par < 2; ++par) {
            StencilCall s;
            s.prec = QCD_F64;
            s.mode = M_FULL;
            s.out_par = par;
            s.out = half(out, par);
            s.in = half(in, 1 - par);
            s.y = half(in, par);
            s.a = 1.0;
            s.cc = -c->kappa;
            s.done = done;
            TRY(launch_stencil(c, s));
        }
        return QCD_OK;
    };
    TRY(canon_to_half(c, QCD_F64, 0, b, 0, half(B, 0), 1, 0));
    TRY(canon_to_half(c, QCD_F64, 0, b, 1, half(B, 1), 1, 0));
    S.aux = c->states + ST_AUX;
    if (S.o.use_x0) {
        TRY(canon_to_half(c, QCD_F64, 0, x, 0, half(X, 0), 1, 0));
        TRY(canon_to_half(c, QCD_F64, 0, x, 1, half(X, 1), 1, 0));
        // r = b - D x
        for (int par = 0; par < 2; ++par) {
            StencilCall s;
            s.prec = QCD_F64;
            s.mode = M_FULL;
            s.out_par = par;
            s.out = half(R, par);
            s.in = half(X, 1 - par);
            s.y = half(X, par);
            s.a = -1.0;
            s.cc = c->kappa;
            s.z = half(B, par);
            s.d = 1.0;
            TRY(launch_stencil(c, s));
        }
        TRY(state_init(c, S.aux, 0.0, 0.0, 0, 0.0, 0));
        TRY(blas_norm2(c, QCD_F64, n, B, S.aux, FIN_SETN + 0));
        TRY(state_init(c, st, 0.0, 0.0, S.o.max_outer, BD_EPS_F64, 0));
        TRY(set_tol2(c, st, S.aux, 0, tol * tol));
        TRY(blas_init(c, QCD_F64, n, R, R, RT, P, X, 0, st, FIN_INIT));
    } else {
        TRY(state_init(c, st, 0.0, tol * tol, S.o.max_outer, BD_EPS_F64, 0));
        TRY(blas_init(c, QCD_F64, n, B, R, RT, P, X, 1, st, FIN_INIT));
    }
    SolverState h;
    int queued = 0;
    for (;;) {
        for (int k = 0; k < 8; ++k) {
            TRY(applyD(P, Q));
            TRY(blas_dot(c, QCD_F64, n, RT, Q, st, FIN_ALPHA, done));
            TRY(blas_update_s(c, QCD_F64, n, R, Q, st));
            TRY(applyD(R, T));
            TRY(blas_omega(c, QCD_F64, n, T, R, st, done));
            TRY(blas_update_x(c, QCD_F64, n, X, P, R, T, RT, st));
            TRY(blas_update_p(c, QCD_F64, n, P, R, Q, st, FIN_NONE));
        }
        queued += 8;
        TRY(read_state(c, ST_OUTER, &h));
        if (h.done || queued > h.maxit + 16) break;
    }
    TRY(blas_finish_half(c, QCD_F64, n, X, P, st));
    S.info.outer_iters = h.iter;
    S.info.dhat_applies[QCD_F64] = 2L * h.iter - h.exit_half;
    // true residual
    S.aux = c->states + ST_AUX;
    TRY(state_init(c, S.aux, 0.0, 0.0, 0, 0.0, 0));
    TRY(blas_norm2(c, QCD_F64, n, B, S.aux, FIN_SETN + 0));
    S.be = half(B, 0);
    S.bo = half(B, 1);
    S.re = half(Q, 0);
    S.ro = half(Q, 1);
    TRY(true_residual(S, QCD_F64, half(X, 0), half(X, 1), S.be, S.bo));
    SolverState ha;
    TRY(read_state(c, ST_AUX, &ha));
    S.info.true_resid = resid_ratio(ha);
    TRY(half_to_canon(c, QCD_F64, 0, half(X, 0), x, 0, 1, 0));
    TRY(half_to_canon(c, QCD_F64, 0, half(X, 1), x, 1, 1, 0));
    int status = h.status;
    if (!std::isfinite(S.info.true_resid)) status = QCD_ENONFINITE;
    else if (S.info.true_resid <= tol) status = QCD_OK;
    else if (status == QCD_OK) status = QCD_ENOTCONV;
    return status;
}

// ---------------------------------------------------------------- lockstep multi-RHS solves
// n systems D x_r = b_r on one gauge field, solved together: every FP32
// iteration (Alg. 2) applies D^ to all right-hand sides at once -- the
// multi-RHS MULT, which stages each site block's links and clover once for
// all of them, and a second half whose blocks of one site block's
// right-hand sides are dispatched together -- with each right-hand side's
// own scalars, dot products and exit test; Alg. 1, the FP64 source,
// reconstruction and true-residual check run right-hand side by right-hand
// side.  A right-hand side that has converged is skipped.  Each right-hand
// side repeats qcd_solve's operations in qcd_solve's order (the multi-RHS
// MULT equals the single-RHS one to the bit, the second half and the BLAS
// passes are the single-RHS launch shapes), so its solution equals
// qcd_solve's to the bit.
struct Multi {
    qcd_ctx *c = nullptr;
    qcd_solve_opts o;
    int n = 0;
    int P0 = QCD_F64, PX = QCD_F64;
    std::vector<Solver> S;        // per right-hand side: outer level, b_e, b_o, b^_e, x_o, residual vectors
    std::vector<HVec> xe0;        // x_e in the outer operator's precision (restarts)
    HVec X, R, RT, P, Q, T, TMP;  // FP32 level: n vectors each, rhs_stride apart
    size_t stride32 = 0;          // in 16-byte elements
    SolverState *st = nullptr;    // [3][n]: inner (contiguous: the lockstep kernels index it), outer, aux
    double *partials = nullptr;   // [n][pstride]
    size_t pstride = 0;           // doubles
    unsigned *counters = nullptr; // [n]
    std::vector<SolverState> h;   // host copies of the 3 n states
    SolverState *in(int r) { return st + r; }
    SolverState *out(int r) { return st + n + r; }
    SolverState *aux(int r) { return st + 2 * n + r; }
};

HVec rhs_at(const HVec &v, int r, size_t stride)
{
    HVec o = v;
    o.p = (char *)v.p + (size_t)r * stride * 16;
    return o;
}

int read_multi(Multi &M)
{
    const size_t bytes = 3 * (size_t)M.n * sizeof(SolverState);
    QCD_CUDA_CHECK(cudaMemcpyAsync(M.h.data(), M.st, bytes, cudaMemcpyDeviceToHost, M.c->stream));
    QCD_CUDA_CHECK(cudaStreamSynchronize(M.c->stream));
    return QCD_OK;
}

// one device allocation for every per-RHS vector, state and partial
int multi_workspace(Multi &M)
{
    qcd_ctx *c = M.c;
    const int n = M.n;
    const size_t h64 = hvec_bytes(c->g, QCD_F64), h32 = hvec_bytes(c->g, QCD_F32);  // DF64 is FP64-sized
    const size_t G = nblocks(c->g.Vh, 32);  // partials of the smallest block the tuner uses
    M.pstride = G * 4;
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t b64 = up(16 * (size_t)n * h64), b32 = up(7 * (size_t)n * h32);
    const size_t bst = up(3 * (size_t)n * sizeof(SolverState)), bpart = up((size_t)n * M.pstride * sizeof(double));
    const size_t need = b64 + b32 + bst + bpart + up(n * sizeof(unsigned));
    if (c->multi_bytes < need) {
        if (c->multi_buf) {
            QCD_CUDA_CHECK(cudaStreamSynchronize(c->stream));
            cudaFree(c->multi_buf);
            for (void *&q : c->pool)
                if (q == c->multi_buf) q = nullptr;
            c->multi_buf = nullptr;
            c->multi_bytes = 0;
        }
        TRY(dev_alloc(c, &c->multi_buf, need));
        c->multi_bytes = need;
    }
    char *base = (char *)c->multi_buf;
    auto v64 = [&](int k, int r, int prec) {
        HVec v;
        v.p = base + ((size_t)k * n + r) * h64;
        v.prec = prec;
        return v;
    };
    M.S.assign(n, Solver{});
    M.xe0.assign(n, HVec{});
    for (int r = 0; r < n; ++r) {
        Solver &S = M.S[r];
        S.c = c;
        S.o = M.o;
        std::memset(&S.info, 0, sizeof(S.info));
        S.be = v64(0, r, QCD_F64);
        S.bo = v64(1, r, QCD_F64);
        S.bhat = v64(2, r, QCD_F64);
        S.xo = v64(3, r, QCD_F64);
        S.re = v64(4, r, QCD_F64);
        S.ro = v64(5, r, QCD_F64);
        Level &O = S.lv[0];
        O.prec = M.P0;
        O.form = 0;
        O.x = v64(6, r, QCD_F64);  // the solution x_e is FP64 in both outer modes
        HVec *lv[7] = {&O.r, &O.rt, &O.p, &O.q, &O.t, &O.v, &O.tmp};
        for (int k = 0; k < 7; ++k) *lv[k] = v64(7 + k, r, M.P0);
        S.bhat0 = M.PX != M.P0 ? v64(14, r, M.P0) : S.bhat;
        M.xe0[r] = M.PX != M.P0 ? v64(15, r, M.P0) : O.x;
    }
    char *p32 = base + b64;
    M.stride32 = hvec_elems(c->g, QCD_F32);
    HVec *a32[7] = {&M.X, &M.R, &M.RT, &M.P, &M.Q, &M.T, &M.TMP};
    for (int k = 0; k < 7; ++k) {
        a32[k]->p = p32 + (size_t)k * n * h32;
        a32[k]->norm = nullptr;
        a32[k]->prec = QCD_F32;
    }
    M.st = (SolverState *)(base + b64 + b32);
    M.partials = (double *)(base + b64 + b32 + bst);
    M.counters = (unsigned *)(base + b64 + b32 + bst + bpart);
    for (int r = 0; r < n; ++r) {
        M.S[r].lv[0].st = M.out(r);
        M.S[r].aux = M.aux(r);
    }
    M.h.assign(3 * (size_t)n, SolverState{});
    QCD_CUDA_CHECK(cudaMemsetAsync(M.counters, 0, n * sizeof(unsigned), c->stream));
    return QCD_OK;
}

// right-hand sides from which the FP32 MULT runs as one staged multi-RHS
// launch: with fewer, the staged kernel's tiles leave the SMs short of warps
// (24^3x48, two right-hand sides: the lockstep solve 7% slower than two
// single solves; from four on it is faster)
constexpr int MULTI_MIN_MRHS = 4;

// one Alg. 2 iteration of every right-hand side of the FP32 level
int bicg_iteration_multi(Multi &M)
{
    qcd_ctx *c = M.c;
    const int ns = c->g.Vh_pad, n = M.n;
    const int dstride = (int)(sizeof(SolverState) / sizeof(int));
    auto half = [&](HVec in, HVec out, int red, HVec aux, int fin) -> int {
        StencilCall s1;
        s1.prec = QCD_F32;
        s1.mode = M_MULT;
        s1.out_par = 1;
        if (n >= MULTI_MIN_MRHS) {  // the staged multi-RHS MULT
            s1.out = M.TMP;
            s1.in = in;
            s1.nrhs = n;
            s1.rhs_stride = M.stride32;
            s1.done = &M.in(0)->done;
            s1.done_stride = dstride;
            TRY(launch_stencil(c, s1));
        } else {  // too few right-hand sides to fill the SMs with staged tiles: one MULT each
            for (int r = 0; r < n; ++r) {
                s1.out = rhs_at(M.TMP, r, M.stride32);
                s1.in = rhs_at(in, r, M.stride32);
                s1.done = &M.in(r)->done;
                TRY(launch_stencil(c, s1));
            }
        }
        StencilCall s2;
        s2.prec = QCD_F32;
        s2.mode = M_DHAT;
        s2.out_par = 0;
        s2.out = out;
        s2.in = M.TMP;
        s2.y = in;
        s2.a = 1.0;
        s2.cc = -c->kappa * c->kappa;
        s2.red = red;
        s2.aux = aux;
        s2.red_args = RedArgs{M.partials, M.counters, M.in(0), fin};
        s2.nrhs = n;
        s2.rhs_stride = M.stride32;
        s2.done = &M.in(0)->done;
        s2.done_stride = dstride;
        s2.red_pstride = M.pstride;
        s2.rhs_grid = true;
        return launch_stencil(c, s2);
    };
    auto at = [&](const HVec &v, int r) { return rhs_at(v, r, M.stride32); };
    TRY(half(M.P, M.Q, R_DOT_AUX, M.RT, FIN_ALPHA));  // q = D^ p, alpha
    for (int r = 0; r < n; ++r) TRY(blas_update_s(c, QCD_F32, ns, at(M.R, r), at(M.Q, r), M.in(r)));  // s = r - alpha q
    TRY(half(M.R, M.T, R_OMEGA, M.R, FIN_OMEGA));  // t = D^ s, omega
    for (int r = 0; r < n; ++r)
        TRY(blas_update_x(c, QCD_F32, ns, at(M.X, r), at(M.P, r), at(M.R, r), at(M.T, r), at(M.RT, r), M.in(r)));
    for (int r = 0; r < n; ++r) TRY(blas_update_p(c, QCD_F32, ns, at(M.P, r), at(M.R, r), at(M.Q, r), M.in(r), FIN_NONE));
    return QCD_OK;
}

// v_r = M src_r for the right-hand sides in `act`: Alg. 2 in FP32 on the
// unit-norm src_r / |src_r|, all of them in lockstep, lifted back
int precondition_multi(Multi &M, const std::vector<char> &act, const std::vector<HVec> &src,
                       const std::vector<const double *> &src_norm2, const std::vector<HVec> &v)
{
    qcd_ctx *c = M.c;
    const int ns = c->g.Vh_pad, n = M.n;
    const double tol = M.o.inner_tol[0];
    auto at = [&](const HVec &x, int r) { return rhs_at(x, r, M.stride32); };
    for (int r = 0; r < n; ++r) {
        TRY(state_init(c, M.in(r), tol * tol, 0.0, M.o.max_inner[0], BD_EPS_LOW, 1));
        if (act[r])
            TRY(blas_inner_init(c, M.P0, QCD_F32, ns, src[r], src_norm2[r], at(M.R, r), at(M.RT, r), at(M.P, r),
                                at(M.X, r), &M.out(r)->done));
        else TRY(state_mark_done(c, M.in(r)));
    }
    int queued = 0, chunk = 3, maxit = M.o.max_inner[0];
    std::vector<double> rr0(n, -1.0);
    for (;;) {
        for (int k = 0; k < chunk; ++k) TRY(bicg_iteration_multi(M));
        queued += chunk;
        TRY(read_multi(M));
        int pred = 1;
        bool all = true;
        for (int r = 0; r < n; ++r) {
            const SolverState &h = M.h[r];
            if (rr0[r] < 0.0) rr0[r] = h.rr > 0 ? h.rr : 1.0;
            if (h.done) continue;
            all = false;
            // the remaining iterations predicted from this right-hand side's contraction so far
            int pr = 8;
            if (h.iter > 0 && h.rr > 0.0 && h.rr < rr0[r] && h.tol2 > 0.0) {
                const double rate = std::log(h.rr / rr0[r]) / h.iter;
                pr = (int)std::ceil(std::log(h.tol2 / h.rr) / rate);
            }
            if (pr < 2) pr = 2;
            if (pr > maxit - h.iter + 1) pr = maxit - h.iter + 1;
            if (pr > pred) pred = pr;
        }
        if (all) break;
        if (queued > maxit + 8) {  // cannot happen: FIN_X caps every right-hand side at maxit
            set_error_message("iteration queue overran the cap");
            return QCD_ETIMEOUT;
        }
        chunk = pred > 64 ? 64 : pred < 1 ? 1 : pred;
    }
    for (int r = 0; r < n; ++r) {
        if (!act[r]) continue;
        const SolverState &h = M.h[r];
        M.S[r].info.inner_iters[0] += h.iter;
        M.S[r].info.dhat_applies[QCD_F32] += 2L * h.iter - h.exit_half;
        TRY(blas_finish_half(c, QCD_F32, ns, at(M.X, r), at(M.P, r), M.in(r)));
        TRY(blas_lift(c, QCD_F32, M.P0, ns, at(M.X, r), v[r], src_norm2[r], &M.out(r)->done));
    }
    return QCD_OK;
}

// Alg. 1 for the right-hand sides in `act` until each has converged
int flexible_multi(Multi &M, std::vector<char> act)
{
    qcd_ctx *c = M.c;
    const int ns = c->g.Vh_pad, n = M.n;
    std::vector<HVec> src(n), v(n);
    std::vector<const double *> nrm(n);
    auto refresh = [&]() -> int {  // drop the right-hand sides whose outer level is done
        TRY(read_multi(M));
        int left = 0;
        for (int r = 0; r < n; ++r) {
            if (act[r] && M.h[n + r].done) act[r] = 0;
            left += act[r];
        }
        return left;
    };
    int left = refresh();
    if (left < 0) return left;
    while (left > 0) {
        for (int r = 0; r < n; ++r) {
            Level &O = M.S[r].lv[0];
            src[r] = O.p;
            nrm[r] = &O.st->norm2[1];
            v[r] = O.v;
        }
        TRY(precondition_multi(M, act, src, nrm, v));  // v = M p
        for (int r = 0; r < n; ++r) {
            if (!act[r]) continue;
            Level &O = M.S[r].lv[0];
            TRY(dhat(c, O.prec, O.v, O.q, O.tmp, R_DOT_AUX, O.rt, O.st, FIN_ALPHA, &O.st->done, 0));  // q = D^ v, alpha
            TRY(blas_flex1(c, O.prec, ns, O.x, O.v, O.r, O.q, O.st));                                    // x, r, |r|
            M.S[r].info.dhat_applies[QCD_F64] += 1;
        }
        if ((left = refresh()) <= 0) break;
        for (int r = 0; r < n; ++r) {
            Level &O = M.S[r].lv[0];
            src[r] = O.r;
            nrm[r] = &O.st->rr;
        }
        TRY(precondition_multi(M, act, src, nrm, v));  // v = M r
        for (int r = 0; r < n; ++r) {
            if (!act[r]) continue;
            Level &O = M.S[r].lv[0];
            TRY(dhat(c, O.prec, O.v, O.t, O.tmp, R_OMEGA, O.r, O.st, FIN_OMEGA, &O.st->done, 0));  // t = D^ v, omega
            TRY(blas_flex2(c, O.prec, ns, O.x, O.v, O.r, O.t, O.rt, O.st));                         // x, r, beta
            TRY(blas_update_p(c, O.prec, ns, O.p, O.r, O.q, O.st, FIN_SETN + 1));                   // p, |p|
            M.S[r].info.dhat_applies[QCD_F64] += 1;
        }
        left = refresh();
    }
    return left < 0 ? left : QCD_OK;
}

// the n solves: b, x hold n full-lattice complex128 vectors back to back
int solve_multi_eo(Multi &M, const void *b, void *x, double tol, std::vector<int> &status)
{
    qcd_ctx *c = M.c;
    const int ns = c->g.Vh_pad, n = M.n;
    const size_t vbytes = (size_t)c->g.V * 12 * 16;
    const int maxit = M.o.max_outer;
    for (int r = 0; r < n; ++r) {
        Solver &S = M.S[r];
        Level &O = S.lv[0];
        const void *br = (const char *)b + r * vbytes;
        TRY(canon_to_half(c, QCD_F64, 0, br, 0, S.be, 1, 0));
        TRY(canon_to_half(c, QCD_F64, 0, br, 1, S.bo, 1, 0));
        TRY(state_init(c, S.aux, 0.0, 0.0, 0, 0.0, 0));
        TRY(blas_norm2(c, QCD_F64, ns, S.be, S.aux, FIN_SETN + 0));
        TRY(blas_norm2(c, QCD_F64, ns, S.bo, S.aux, FIN_ADDN + 0));
        // b^_e = F_ee^-1 (b_e + kappa H_eo F_oo^-1 b_o)   (Eq. 6), in FP64
        TRY(clover_apply_half(c, QCD_F64, 1, 1, S.bo, S.re, 1, 0));
        StencilCall s;
        s.prec = QCD_F64;
        s.mode = M_SRC;
        s.out_par = 0;
        s.out = S.bhat;
        s.in = S.re;
        s.y = S.be;
        s.a = 1.0;
        s.cc = c->kappa;
        TRY(launch_stencil(c, s));
        if (M.PX != M.P0) TRY(convert_half(c, S.bhat, S.bhat0));
        TRY(state_init(c, O.st, 0.0, 0.0, maxit, BD_EPS_F64, 0));
        TRY(set_tol2(c, O.st, S.aux, 0, 0.25 * tol * tol));
        TRY(blas_init(c, M.P0, ns, S.bhat0, O.r, O.rt, O.p, O.x, 1, O.st, FIN_INIT));
    }
    std::vector<char> act(n, 1);
    status.assign(n, QCD_OK);
    for (int restart = 0;; ++restart) {
        TRY(flexible_multi(M, act));
        // x_o = F_oo^-1 (b_o + kappa H_oe x_e) with the odd rows of b - D x
        // (Eq. 7), the even rows, x out: FP64, per right-hand side
        for (int r = 0; r < n; ++r) {
            if (!act[r]) continue;
            Solver &S = M.S[r];
            StencilCall s;
            s.prec = QCD_F64;
            s.mode = M_RECON;
            s.out_par = 1;
            s.out = S.xo;
            s.in = S.lv[0].x;
            s.y = S.bo;
            s.a = 1.0;
            s.cc = c->kappa;
            s.red = R_NORM;
            s.red_args = RedArgs{c->partials, c->counters, S.aux, FIN_SETN + 2};
            TRY(launch_stencil(c, s));
            TRY(emit_x(c, S.lv[0].x, S.xo, (char *)x + r * vbytes));
            TRY(residual_even(S, S.lv[0].x, S.xo));
        }
        TRY(read_multi(M));
        std::vector<char> again(n, 0);
        int nagain = 0;
        for (int r = 0; r < n; ++r) {
            if (!act[r]) continue;
            Solver &S = M.S[r];
            const SolverState &ho = M.h[n + r], &ha = M.h[2 * n + r];
            S.info.outer_iters = ho.iter;
            S.info.true_resid = resid_ratio(ha);
            int st = ho.status;
            if (!std::isfinite(S.info.true_resid)) st = QCD_ENONFINITE;
            else if (S.info.true_resid <= tol) st = QCD_OK;
            else if (st != QCD_ENONFINITE && restart < M.o.max_restarts && ho.iter < maxit) {
                again[r] = 1;
                ++nagain;
            } else if (st == QCD_OK) st = QCD_ENOTCONV;
            status[r] = st;
        }
        if (!nagain) break;
        // restart from the recomputed residual r = b^ - D^ x_e
        for (int r = 0; r < n; ++r) {
            if (!again[r]) continue;
            Solver &S = M.S[r];
            Level &O = S.lv[0];
            S.info.restarts += 1;
            TRY(state_init(c, O.st, 0.0, 0.0, maxit, BD_EPS_F64, 0));
            TRY(set_tol2(c, O.st, S.aux, 0, 0.25 * tol * tol));
            if (M.PX != M.P0) TRY(convert_half(c, O.x, M.xe0[r]));
            TRY(residual_eo(S, M.xe0[r], O.r, O.st, FIN_NONE));
            TRY(blas_init(c, M.P0, ns, O.r, O.r, O.rt, O.p, O.x, 0, O.st, FIN_RESTART));
        }
        act = again;
    }
    return QCD_OK;
}

}  // namespace

int solve(qcd_ctx *c, const void *b_dev, void *x_dev, double tol, const qcd_solve_opts &o, qcd_solve_info *info)
{
    Solver S;
    S.c = c;
    S.o = o;
    std::memset(&S.info, 0, sizeof(S.info));
    cudaEvent_t e0, e1;
    QCD_CUDA_CHECK(cudaEventCreate(&e0));
    QCD_CUDA_CHECK(cudaEventCreate(&e1));
    QCD_CUDA_CHECK(cudaEventRecord(e0, c->stream));
    int rc = o.even_odd ? solve_eo(S, b_dev, x_dev, tol) : solve_full(S, b_dev, x_dev, tol);
    cudaEventRecord(e1, c->stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    S.info.seconds = ms * 1e-3;
    S.info.status = rc;
    if (info) *info = S.info;
    return rc;
}

int solve_multi(qcd_ctx *c, const void *b_dev, void *x_dev, int nrhs, double tol, const qcd_solve_opts &o,
                qcd_solve_info *info)
{
    Multi M;
    M.c = c;
    M.o = o;
    M.n = nrhs;
    M.P0 = o.outer_df64 ? QCD_DF64 : QCD_F64;
    M.PX = QCD_F64;
    cudaEvent_t e0, e1;
    QCD_CUDA_CHECK(cudaEventCreate(&e0));
    QCD_CUDA_CHECK(cudaEventCreate(&e1));
    QCD_CUDA_CHECK(cudaEventRecord(e0, c->stream));
    std::vector<int> status;
    int rc = multi_workspace(M);
    if (rc == QCD_OK) rc = solve_multi_eo(M, b_dev, x_dev, tol, status);
    cudaEventRecord(e1, c->stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int worst = rc;
    for (int r = 0; r < nrhs && r < (int)M.S.size(); ++r) {
        qcd_solve_info &in = M.S[r].info;
        in.seconds = ms * 1e-3;
        in.status = rc != QCD_OK ? rc : r < (int)status.size() ? status[r] : QCD_ESTATE;
        if (worst == QCD_OK && in.status != QCD_OK) worst = in.status;
        if (info) info[r] = in;
    }
    return worst;
}

}  // namespace qcd
