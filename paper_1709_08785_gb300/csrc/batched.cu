// Batched solves: many independent nested solves (Algs. 1-2), each on its
// own lattice, gauge field and kappa, advanced together by two persistent
// cooperative kernels per outer half-step:
//
//   batched_inner (FP32, Alg. 2, every problem to its own exit):
//     init | { MULT | D^ 2nd half + <r~|q> | alpha | s = r - a q, |s| | exit? |
//              MULT | D^ 2nd half + <t|s>,|t|^2 | omega | x, r, <r~|r> | beta, exit? | p }
//     | lift v = |src| x into the outer precision
//   batched_outer (the outer D^ and recursions in DF64 by default, FP64 on
//     request; the solution x_e accumulated in FP64 unless the all-DF64
//     outer level is asked for): outer D^ with its dot | alpha or omega |
//     outer update and exit test | (second half-step) p update
//
// Each phase walks work tiles (256 sites of one parity of one problem)
// across all lattices; tiles of problems that have finished are skipped.
// Dot products reduce per tile into per-problem partials; a finaliser phase
// adds them in tile order (deterministic) and runs the BiCGStab scalar
// recurrences of that problem.  Phases are separated by a grid barrier whose
// waits are bounded: a barrier that does not complete within the spin limit
// records QCD_ETIMEOUT and every block returns.  The two kernels exist
// because their register needs differ (~80 for the FP32 phases, ~170 for
// the float-pair arithmetic): one kernel held the FP32 phases to one block
// per SM.  The four launches of an outer iteration are captured once in a
// CUDA graph and replayed until every problem has converged.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "blas.cuh"
#include "blas_ops.cuh"
#include "stencil.cuh"

namespace qcd {

namespace {

constexpr int TILE = 256;  // sites per work tile = threads per block
// spinors written and read inside one launch: coherent loads (see Prec)
constexpr int C32 = QCD_F32 + COHERENT, C64 = QCD_F64 + COHERENT, CDF = QCD_DF64 + COHERENT;
constexpr int STATE_WORDS = sizeof(SolverState) / sizeof(double);
static_assert(sizeof(SolverState) % sizeof(double) == 0, "SolverState is copied as doubles");

// work-slot assignment shared with the single-solve driver (solver.cu)
constexpr int S64_BE = 0, S64_BO = 1, S64_BHAT = 2, S64_XO = 3, S64_RE = 4, S64_RO = 5, S64_LEVEL = 6;
constexpr int S32_LEVEL = 0;

struct BProb {
    Geom g;
    double k2;  // kappa^2
    float k2f;  // kappa^2 rounded to FP32 on the host, for the FP32 phases
    GaugePtr U32, UO;
    CloverPtr Ci32, CiO;                       // UO, CiO: in the outer level's precision
    SpinorPtr x, r, rt, p, q, t, tmp;          // FP32 inner (tmp: odd parity)
    SpinorPtr X, R, RT, P, Q, T, Vv, TMP;      // outer level: DF64 (default) or FP64; X in PX
    SolverState *in, *out;                     // inner, outer scalars
    double *partials;                          // [ntiles][4]
    int tile0, ntiles;
};

struct BatchArgs {
    BProb *probs;
    int nprob;
    int total_tiles;
    int half;  // 0: precondition p, alpha update; 1: precondition r, omega/beta updates, p
    int inner_maxit;
    double inner_tol2;
    unsigned *bar_count;
    unsigned *bar_gen;
    int *err;
    long long spin_limit;
};

__device__ __forceinline__ bool grid_barrier(const BatchArgs &A)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *genp = A.bar_gen;
        const unsigned gen = *genp;
        __threadfence();
        const unsigned arrived = atomicAdd(A.bar_count, 1u) + 1u;
        if (arrived == gridDim.x) {
            *A.bar_count = 0u;
            __threadfence();
            atomicAdd((unsigned *)A.bar_gen, 1u);
        } else {
            long long n = 0;
            while (*genp == gen) {
                if (++n > A.spin_limit) {
                    atomicExch(A.err, QCD_ETIMEOUT);
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *(volatile int *)A.err == 0;
}

__device__ __forceinline__ int find_prob(const BatchArgs &A, int tile)
{
    int lo = 0, hi = A.nprob - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (A.probs[mid].tile0 <= tile) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// block-level sum of N values into thread 0's out: the warp stage in the
// accumulator type A (float in the FP32 phases, see grid_reduce), the warp
// sums in FP64
template <int N, class A>
__device__ __forceinline__ void block_sum(A v[N], double out[N])
{
    __shared__ double sh[TILE / 32][4];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < N; ++k)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < N; ++k) sh[wid][k] = (double)v[k];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 0; k < N; ++k) {
            double t = 0.0;
            for (int w = 0; w < TILE / 32; ++w) t += sh[w][k];
            out[k] = t;
        }
    __syncthreads();
}

enum Phase {
    PH_INIT, PH_MULT_P, PH_DHAT_Q, PH_S, PH_MULT_S, PH_DHAT_T, PH_X, PH_P,
    PH_LIFT, PH_OMULT, PH_ODHAT, PH_OUPD, PH_OP
};

// the outer level's hopping term: the rolled loops for DF64 (instruction cache)
template <int PO>
__device__ __forceinline__ void hop_outer(const BProb &pr, const SpinorPtr &in, int out_par, int cb,
                                          Spinor<typename Prec<PO>::T> &a)
{
    if constexpr (PO == CDF) {
        hopping_rolled<PO, false>(pr.g, pr.UO, in, out_par, cb, a);
        apply_clover_rolled<PO>(pr.CiO, out_par, cb, a);
    } else {
        hopping<PO, false>(pr.g, pr.UO, in, out_par, cb, a);
        apply_clover<PO>(pr.CiO, out_par, cb, a);
    }
}

// one phase over all tiles of all live problems; PO: the outer level's
// (coherent) precision, DF64 or FP64; PX: the precision of the outer
// solution x_e (FP64, or PO)
template <int PO, int PX, bool OUTER>
__device__ void run_phase(const BatchArgs &A, int ph)
{
    using TO = typename Prec<PO>::T;
    for (int tile = blockIdx.x; tile < A.total_tiles; tile += gridDim.x) {
        const int pi = find_prob(A, tile);
        const BProb &pr = A.probs[pi];
        // the scalars other blocks finalised: read through L2 into shared memory
        __shared__ SolverState s_in, s_out;
        __syncthreads();
        if (threadIdx.x < STATE_WORDS) {
            ((double *)&s_in)[threadIdx.x] = __ldcg((const double *)pr.in + threadIdx.x);
            ((double *)&s_out)[threadIdx.x] = __ldcg((const double *)pr.out + threadIdx.x);
        }
        __syncthreads();
        const bool outer_live = !s_out.done;
        bool live;
        if (ph == PH_INIT || ph == PH_LIFT || ph >= PH_OMULT) live = outer_live;
        else live = outer_live && !s_in.done;
        if (!live) continue;  // uniform over the block
        const int lt = tile - pr.tile0;
        const int cb = lt * TILE + threadIdx.x;
        const bool in_range = cb < pr.g.Vh_pad;
        const bool site = cb < pr.g.Vh;
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        float accf[4] = {0.f, 0.f, 0.f, 0.f};  // the FP32 phases' sums
        int nred = 0;
        bool f32red = false;
        switch (ph) {
        case PH_INIT: {  // b = src/|src|, r = r~ = p = b, x = 0 (src: p or r of the outer level)
            if constexpr (OUTER) break;
            const SpinorPtr src = A.half == 0 ? pr.P : pr.R;
            const double *n2 = A.half == 0 ? &s_out.norm2[1] : &s_out.rr;
            if (in_range) OpInner<PO, C32>{src, pr.r, pr.rt, pr.p, pr.x, n2}(cb, acc);
            break;
        }
        case PH_MULT_P:
        case PH_MULT_S:
            if constexpr (OUTER) break;
            if (site) {
                Spinor<float> a;
                hopping<C32, false>(pr.g, pr.U32, ph == PH_MULT_P ? pr.p : pr.r, 1, cb, a);
                apply_clover<C32>(pr.Ci32, 1, cb, a);
                Prec<C32>::store(pr.tmp, cb, a);
            }
            break;
        case PH_DHAT_Q:
        case PH_DHAT_T:
            if constexpr (OUTER) break;
            if (site) {
                Spinor<float> a, y;
                hopping<C32, false>(pr.g, pr.U32, pr.tmp, 0, cb, a);
                apply_clover<C32>(pr.Ci32, 0, cb, a);
                const SpinorPtr yv = ph == PH_DHAT_Q ? pr.p : pr.r;
                Prec<C32>::load(yv, cb, y);
                axpby_sp(a, -pr.k2f, a, 1.0f, y);
                Prec<C32>::store(ph == PH_DHAT_Q ? pr.q : pr.t, cb, a);
                if (ph == PH_DHAT_Q) {
                    Spinor<float> w;
                    Prec<C32>::load(pr.rt, cb, w);
                    acc_dot(w, a, accf[0], accf[1]);
                } else {
                    acc_dot(a, y, accf[0], accf[1]);
                    acc_norm2(accf[2], a);
                }
            }
            nred = 3;
            f32red = true;
            break;
        case PH_S:
            if constexpr (OUTER) break;
            if (in_range) OpS<C32>{pr.r, pr.q, &s_in}(cb, accf);
            nred = 1;
            f32red = true;
            break;
        case PH_X:
            if constexpr (OUTER) break;
            if (in_range) OpX<C32>{pr.x, pr.p, pr.r, pr.t, pr.rt, &s_in}(cb, accf);
            nred = 3;
            f32red = true;
            break;
        case PH_P:
            if constexpr (OUTER) break;
            if (in_range) OpP<C32>{pr.p, pr.r, pr.q, &s_in}(cb, accf);
            break;
        case PH_LIFT:  // finish the inner solve: x += alpha p after a first-half exit; v = |src| x
            if constexpr (OUTER) break;
            if (in_range) {
                OpHalf<C32>{pr.x, pr.p, &s_in}(cb, acc);
                const double *n2 = A.half == 0 ? &s_out.norm2[1] : &s_out.rr;
                OpLift<C32, PO>{pr.x, pr.Vv, n2}(cb, acc);
            }
            break;
        case PH_OMULT:
            if constexpr (!OUTER) break;
            if (site) {
                Spinor<TO> a;
                hop_outer<PO>(pr, pr.Vv, 1, cb, a);
                Prec<PO>::store(pr.TMP, cb, a);
            }
            break;
        case PH_ODHAT:
            if constexpr (!OUTER) break;
            if (site) {
                Spinor<TO> a, v;
                hop_outer<PO>(pr, pr.TMP, 0, cb, a);
                Prec<PO>::load(pr.Vv, cb, v);
                axpby_sp(a, TO(-pr.k2), a, TO(1.0), v);
                Prec<PO>::store(A.half == 0 ? pr.Q : pr.T, cb, a);
                if (A.half == 0) {
                    Spinor<TO> w;
                    Prec<PO>::load(pr.RT, cb, w);
                    acc_dot(w, a, acc[0], acc[1]);
                } else {
                    Spinor<TO> rr;
                    Prec<PO>::load(pr.R, cb, rr);
                    acc_dot(a, rr, acc[0], acc[1]);
                    acc_norm2(acc[2], a);
                }
            }
            nred = 3;
            break;
        case PH_OUPD:
            if constexpr (!OUTER) break;
            if (in_range) {
                if constexpr (PX == PO) {
                    if (A.half == 0) OpFlex1<PO>{pr.X, pr.Vv, pr.R, pr.Q, &s_out}(cb, acc);
                    else OpFlex2<PO>{pr.X, pr.Vv, pr.R, pr.T, pr.RT, &s_out}(cb, acc);
                } else {
                    if (A.half == 0) OpFlex1X<PO, PX>{pr.X, pr.Vv, pr.R, pr.Q, &s_out}(cb, acc);
                    else OpFlex2X<PO, PX>{pr.X, pr.Vv, pr.R, pr.T, pr.RT, &s_out}(cb, acc);
                }
            }
            nred = 3;
            break;
        case PH_OP:
            if constexpr (!OUTER) break;
            if (in_range) OpP<PO>{pr.P, pr.R, pr.Q, &s_out}(cb, acc);
            nred = 1;
            break;
        }
        if (nred) {
            if (f32red) block_sum<3>(accf, acc);
            else block_sum<3>(acc, acc);
            if (threadIdx.x == 0)
                for (int k = 0; k < 4; ++k) pr.partials[(size_t)lt * 4 + k] = k < 3 ? acc[k] : 0.0;
        }
    }
}

// sum the partials of each problem in tile order and run the finaliser
__device__ void run_finalise(const BatchArgs &A, int ph)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int warps = blockDim.x >> 5;
    for (int pi = blockIdx.x * warps + wid; pi < A.nprob; pi += gridDim.x * warps) {
        const BProb &pr = A.probs[pi];
        const bool outer_level = ph >= PH_OMULT;
        if (__ldcg(&pr.out->done) || (!outer_level && __ldcg(&pr.in->done))) continue;
        int op;
        switch (ph) {
        case PH_DHAT_Q: op = FIN_ALPHA; break;
        case PH_S: op = FIN_S; break;
        case PH_DHAT_T: op = FIN_OMEGA; break;
        case PH_X: op = FIN_X; break;
        case PH_ODHAT: op = A.half == 0 ? FIN_ALPHA : FIN_OMEGA; break;
        case PH_OUPD: op = A.half == 0 ? FIN_S : FIN_X; break;
        default: op = FIN_SETN + 1; break;  // PH_OP: |p|^2
        }
        double s[3] = {0.0, 0.0, 0.0};
        for (int t = lane; t < pr.ntiles; t += 32)
            for (int k = 0; k < 3; ++k) s[k] += __ldcg(pr.partials + (size_t)t * 4 + k);
        for (int k = 0; k < 3; ++k)
            for (int off = 16; off > 0; off >>= 1) s[k] += __shfl_down_sync(0xffffffffu, s[k], off);
        if (lane == 0) {
            SolverState *st = outer_level ? pr.out : pr.in;
            SolverState loc;
            for (int w = 0; w < STATE_WORDS; ++w) ((double *)&loc)[w] = __ldcg((const double *)st + w);
            loc.sum[0] = s[0];
            loc.sum[1] = s[1];
            loc.sum[2] = s[2];
            loc.sum[3] = 0.0;
            finalize(op, &loc);
            for (int w = 0; w < STATE_WORDS; ++w) __stcg((double *)st + w, ((double *)&loc)[w]);
            __threadfence();
        }
    }
}

__device__ void inner_start(const BatchArgs &A)
{
    // fresh unit-norm Alg. 2 state for every live problem
    for (int pi = blockIdx.x * blockDim.x + threadIdx.x; pi < A.nprob; pi += gridDim.x * blockDim.x) {
        const BProb &pr = A.probs[pi];
        if (__ldcg(&pr.out->done)) continue;
        SolverState s = {};
        s.tol2 = A.inner_tol2;
        s.maxit = A.inner_maxit;
        s.bd_eps = 1e-12;
        s.rho0[0] = 1.0;
        s.rr = 1.0;
        s.rt2 = 1.0;
        s.norm2[1] = 1.0;
        *pr.in = s;
    }
}

__device__ void inner_account(const BatchArgs &A)
{
    // accumulate the inner iterations and D^ counts of this half-step
    for (int pi = blockIdx.x * blockDim.x + threadIdx.x; pi < A.nprob; pi += gridDim.x * blockDim.x) {
        const BProb &pr = A.probs[pi];
        if (__ldcg(&pr.out->done)) continue;
        const int it = __ldcg(&pr.in->iter), eh = __ldcg(&pr.in->exit_half);
        __stcg(&pr.out->pad[0], __ldcg(&pr.out->pad[0]) + it);
        __stcg(&pr.out->pad[1], __ldcg(&pr.out->pad[1]) + 2 * it - eh);
    }
}

// One outer half-step is two cooperative launches: the inner FP32 solve
// (Alg. 2) of every live problem, with the conversions between the levels,
// at FP32-kernel occupancy; then the outer D^ and updates (Alg. 1) in PO,
// whose float-pair or FP64 arithmetic needs about twice the registers.
#define QCD_SYNC()                    \
    do {                              \
        if (!grid_barrier(A)) return; \
    } while (0)
template <int PO>
__global__ void __launch_bounds__(TILE, 3) batched_inner(BatchArgs A)
{
    inner_start(A);
    run_phase<PO, PO, false>(A, PH_INIT);
    QCD_SYNC();
    for (int it = 0; it <= A.inner_maxit; ++it) {
        run_phase<PO, PO, false>(A, PH_MULT_P);
        QCD_SYNC();
        run_phase<PO, PO, false>(A, PH_DHAT_Q);
        QCD_SYNC();
        run_finalise(A, PH_DHAT_Q);
        QCD_SYNC();
        run_phase<PO, PO, false>(A, PH_S);
        QCD_SYNC();
        run_finalise(A, PH_S);
        QCD_SYNC();
        run_phase<PO, PO, false>(A, PH_MULT_S);
        QCD_SYNC();
        run_phase<PO, PO, false>(A, PH_DHAT_T);
        QCD_SYNC();
        run_finalise(A, PH_DHAT_T);
        QCD_SYNC();
        run_phase<PO, PO, false>(A, PH_X);
        QCD_SYNC();
        run_finalise(A, PH_X);
        QCD_SYNC();
        run_phase<PO, PO, false>(A, PH_P);
        QCD_SYNC();
        bool any = false;
        for (int pi = 0; pi < A.nprob && !any; ++pi)
            any = !__ldcg(&A.probs[pi].out->done) && !__ldcg(&A.probs[pi].in->done);
        if (!any) break;
    }
    inner_account(A);
    run_phase<PO, PO, false>(A, PH_LIFT);
}

template <int PO, int PX>
__global__ void __launch_bounds__(TILE) batched_outer(BatchArgs A)
{
    run_phase<PO, PX, true>(A, PH_OMULT);
    QCD_SYNC();
    run_phase<PO, PX, true>(A, PH_ODHAT);
    QCD_SYNC();
    run_finalise(A, PH_ODHAT);
    QCD_SYNC();
    run_phase<PO, PX, true>(A, PH_OUPD);
    QCD_SYNC();
    run_finalise(A, PH_OUPD);
    if (A.half == 1) {
        QCD_SYNC();
        run_phase<PO, PX, true>(A, PH_OP);
        QCD_SYNC();
        run_finalise(A, PH_OP);
    }
}
#undef QCD_SYNC

SpinorPtr sp(const HVec &v) { return v.sp(); }

}  // namespace

int batched_solve(qcd_ctx **ctxs, int n, const void *const *b, void *const *x, const double *tol,
                  const qcd_solve_opts &o, qcd_solve_info *infos, long long spin_limit, int use_graph)
{
    qcd_ctx *c0 = ctxs[0];
    cudaStream_t user = c0->stream;
    // the outer level's precisions as in the single solve (outer_df64):
    // PO for the outer D^ and recursions, PX for x_e, b^_e and x_o; the true
    // residual is FP64 in every mode
    const int mode = o.outer_df64;
    const int PO = mode ? QCD_DF64 : QCD_F64;
    const int PX = mode == 2 ? QCD_DF64 : QCD_F64;
    void (*kin)(BatchArgs) = mode ? batched_inner<CDF> : batched_inner<C64>;
    void (*kout)(BatchArgs) = mode == 0   ? batched_outer<C64, C64>
                              : mode == 1 ? batched_outer<CDF, C64>
                                          : batched_outer<CDF, CDF>;
    std::vector<BProb> host(n);
    int tiles = 0;
    // ---- per problem: b^_e, |b|^2, and the outer start (same steps as the single solve)
    for (int i = 0; i < n; ++i) {
        qcd_ctx *c = ctxs[i];
        if (c->device != c0->device) {
            set_error_message("batched problems must live on one device");
            return QCD_EINVAL;
        }
        if (!c->have_clover) {
            set_error_message("problem %d: no clover term", i);
            return QCD_ESTATE;
        }
        // FP64 b_e, b_o (norms, true residual); b^_e and x_e in PX; the
        // outer iteration's vectors in PO
        HVec be, bo, beX, boX, bh, bh0, XX, tmpX, LO[8], L32[8];
        int rc;
        if ((rc = get_work(c, QCD_F64, S64_BE, &be)) || (rc = get_work(c, QCD_F64, S64_BO, &bo)) ||
            (rc = get_work(c, PX, S64_BE, &beX)) || (rc = get_work(c, PX, S64_BO, &boX)) ||
            (rc = get_work(c, PX, S64_BHAT, &bh)) || (rc = get_work(c, PO, S64_BHAT, &bh0)) ||
            (rc = get_work(c, PX, S64_LEVEL, &XX)))
            return rc;
        for (int k = 0; k < 8; ++k)
            if ((rc = get_work(c, PO, S64_LEVEL + k, &LO[k])) || (rc = get_work(c, QCD_F32, S32_LEVEL + k, &L32[k])))
                return rc;
        tmpX = LO[7];
        if (PX != PO && (rc = get_work(c, QCD_F64, S64_RE, &tmpX))) return rc;
        SolverState *outer = c->states + ST_OUTER, *inner = c->states + ST_MID, *aux = c->states + ST_AUX;
        const int nn = c->g.Vh_pad;
        cudaStream_t keep = c->stream;
        c->stream = user;
        rc = canon_to_half(c, QCD_F64, 0, b[i], 0, be, 1, 0);
        if (!rc) rc = canon_to_half(c, QCD_F64, 0, b[i], 1, bo, 1, 0);
        if (!rc) rc = state_init(c, aux, 0.0, 0.0, 0, 0.0, 0);
        if (!rc) rc = blas_norm2(c, QCD_F64, nn, be, aux, FIN_SETN + 0);
        if (!rc) rc = blas_norm2(c, QCD_F64, nn, bo, aux, FIN_ADDN + 0);
        if (!rc && PX != QCD_F64) rc = convert_half(c, be, beX);
        if (!rc && PX != QCD_F64) rc = convert_half(c, bo, boX);
        if (!rc) rc = clover_apply_half(c, PX, 1, 1, boX, tmpX, 1, 0);
        if (!rc) {
            StencilCall s;
            s.prec = PX;
            s.mode = M_SRC;
            s.out_par = 0;
            s.out = bh;
            s.in = tmpX;
            s.y = beX;
            s.a = 1.0;
            s.cc = c->kappa;
            rc = launch_stencil(c, s);
        }
        if (!rc && PX != PO) rc = convert_half(c, bh, bh0);
        if (!rc) rc = state_init(c, outer, 0.0, 0.0, o.max_outer, 1e-30, 0);
        if (!rc) rc = set_tol2(c, outer, aux, 0, 0.25 * tol[i] * tol[i]);
        // x_e = 0 (a zero complex has the same bits in FP64 and DF64)
        if (!rc) rc = blas_init(c, PO, nn, bh0, LO[1], LO[2], LO[3], XX, 1, outer, FIN_INIT);
        c->stream = keep;
        if (rc) return rc;
        BProb &pr = host[i];
        pr.g = c->g;
        pr.k2 = c->kappa * c->kappa;
        pr.k2f = (float)pr.k2;
        for (int par = 0; par < 2; ++par) {
            pr.U32.a[par] = c->U32[par];
            pr.U32.b[par] = nullptr;
            pr.UO.a[par] = PO == QCD_DF64 ? (const void *)c->UDF[par] : (const void *)c->U64[par];
            pr.UO.b[par] = nullptr;
            pr.Ci32.p[par] = c->Ci[QCD_F32][par];
            pr.CiO.p[par] = c->Ci[PO][par];
        }
        pr.x = sp(L32[0]); pr.r = sp(L32[1]); pr.rt = sp(L32[2]); pr.p = sp(L32[3]);
        pr.q = sp(L32[4]); pr.t = sp(L32[5]); pr.tmp = sp(L32[7]);
        pr.X = sp(XX); pr.R = sp(LO[1]); pr.RT = sp(LO[2]); pr.P = sp(LO[3]);
        pr.Q = sp(LO[4]); pr.T = sp(LO[5]); pr.Vv = sp(LO[6]); pr.TMP = sp(LO[7]);
        pr.in = inner;
        pr.out = outer;
        pr.partials = c->partials;
        pr.tile0 = tiles;
        pr.ntiles = (int)nblocks(c->g.Vh_pad, TILE);
        if (pr.ntiles > c->partial_blocks) {
            set_error_message("problem %d: too many tiles for its partials buffer", i);
            return QCD_EINVAL;
        }
        tiles += pr.ntiles;
    }
    // ---- device descriptors and barrier words, kept by the first context
    const size_t pbytes = sizeof(BProb) * n;
    const size_t need = ((pbytes + 63) / 64) * 64 + 256;
    int rc;
    if (c0->batch_bytes < need) {
        if (c0->batch_buf) {
            cudaStreamSynchronize(user);
            cudaFree(c0->batch_buf);
            for (auto &p : c0->pool)
                if (p == c0->batch_buf) p = nullptr;
            c0->batch_buf = nullptr;
            c0->batch_bytes = 0;
        }
        if ((rc = dev_alloc(c0, &c0->batch_buf, need))) return rc;
        c0->batch_bytes = need;
    }
    void *dev = c0->batch_buf;
    BProb *dprobs = (BProb *)dev;
    unsigned *bar = (unsigned *)((char *)dev + ((pbytes + 63) / 64) * 64);
    QCD_CUDA_CHECK(cudaMemcpyAsync(dprobs, host.data(), pbytes, cudaMemcpyHostToDevice, user));
    QCD_CUDA_CHECK(cudaMemsetAsync(bar, 0, 64, user));

    // cooperative grids: every block of a launch resident at once
    int per_in = 0, per_out = 0;
    QCD_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_in, kin, TILE, 0));
    QCD_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_out, kout, TILE, 0));
    if (per_in < 1 || per_out < 1) {
        set_error_message("the batched kernels cannot be resident");
        return QCD_ECUDA;
    }
    const int grid_in = std::max(1, std::min(tiles, per_in * c0->num_sms));
    const int grid_out = std::max(1, std::min(tiles, per_out * c0->num_sms));
    BatchArgs A[2];
    for (int h = 0; h < 2; ++h) {
        A[h].probs = dprobs;
        A[h].nprob = n;
        A[h].total_tiles = tiles;
        A[h].half = h;
        A[h].inner_maxit = o.max_inner[0];
        A[h].inner_tol2 = o.inner_tol[0] * o.inner_tol[0];
        A[h].bar_count = bar;
        A[h].bar_gen = bar + 1;
        A[h].err = (int *)(bar + 2);
        A[h].spin_limit = spin_limit;
    }
    // a stream of our own: graph capture is not possible on the legacy stream.
    // The stream, the event and the graph are released on every return path;
    // the user stream waits for the private one before they go.
    struct Res {
        cudaStream_t user, s = nullptr;
        cudaEvent_t ev = nullptr;
        cudaGraphExec_t exec = nullptr;
        ~Res()
        {
            if (exec) cudaGraphExecDestroy(exec);
            if (s && ev && cudaEventRecord(ev, s) == cudaSuccess) cudaStreamWaitEvent(user, ev, 0);
            if (ev) cudaEventDestroy(ev);
            if (s) cudaStreamDestroy(s);
        }
    } res;
    res.user = user;
    QCD_CUDA_CHECK(cudaStreamCreateWithFlags(&res.s, cudaStreamNonBlocking));
    QCD_CUDA_CHECK(cudaEventCreateWithFlags(&res.ev, cudaEventDisableTiming));
    cudaStream_t s = res.s;
    QCD_CUDA_CHECK(cudaEventRecord(res.ev, user));
    QCD_CUDA_CHECK(cudaStreamWaitEvent(s, res.ev, 0));
    auto launch1 = [&](void (*k)(BatchArgs), int grid, int h) -> cudaError_t {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(TILE);
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, k, A[h]);
    };
    auto launch = [&](int h) -> cudaError_t {
        const cudaError_t e = launch1(kin, grid_in, h);
        return e != cudaSuccess ? e : launch1(kout, grid_out, h);
    };
    cudaGraphExec_t &exec = res.exec;
    int graph_used = 0;
    if (use_graph) {
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            cudaError_t e0 = launch(0), e1 = launch(1);
            cudaError_t ee = cudaStreamEndCapture(s, &graph);
            if (e0 == cudaSuccess && e1 == cudaSuccess && ee == cudaSuccess &&
                cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess)
                graph_used = 1;
            if (graph) cudaGraphDestroy(graph);
        }
        cudaGetLastError();
    }
    std::vector<SolverState> st(n);
    int status = QCD_OK;
    int outer_done = 0;
    for (int it = 0; it < o.max_outer && !outer_done; ++it) {
        c0->launches += 4;
        if (graph_used) {
            QCD_CUDA_CHECK(cudaGraphLaunch(exec, s));
        } else {
            QCD_CUDA_CHECK(launch(0));
            QCD_CUDA_CHECK(launch(1));
        }
        int err = 0;
        QCD_CUDA_CHECK(cudaMemcpyAsync(&err, bar + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
        QCD_CUDA_CHECK(cudaStreamSynchronize(s));
        if (err) {
            status = err;
            set_error_message("a grid barrier of the batched kernel gave up waiting");
            break;
        }
        outer_done = 1;
        for (int i = 0; i < n; ++i) {
            QCD_CUDA_CHECK(cudaMemcpyAsync(&st[i], ctxs[i]->states + ST_OUTER, sizeof(SolverState),
                                           cudaMemcpyDeviceToHost, s));
        }
        QCD_CUDA_CHECK(cudaStreamSynchronize(s));
        for (int i = 0; i < n; ++i) outer_done &= st[i].done;
    }
    // the finishing steps below run on the user stream, after the batch
    QCD_CUDA_CHECK(cudaEventRecord(res.ev, s));
    QCD_CUDA_CHECK(cudaStreamWaitEvent(user, res.ev, 0));
    if (status != QCD_OK) return status;
    // ---- per problem: x_o, the true residual, a single-solve restart if needed
    for (int i = 0; i < n; ++i) {
        qcd_ctx *c = ctxs[i];
        cudaStream_t keep = c->stream;
        c->stream = user;
        // x_o = F_oo^-1 (b_o + kappa H_oe x_e) in the solution's precision,
        // then x rounded to FP64 (if it is not FP64) for the FP64 true residual
        HVec be, bo, xo, re, ro, X, XX, xoX, boX;
        int r = QCD_OK;
        if ((r = get_work(c, QCD_F64, S64_BE, &be)) || (r = get_work(c, QCD_F64, S64_BO, &bo)) ||
            (r = get_work(c, QCD_F64, S64_XO, &xo)) || (r = get_work(c, QCD_F64, S64_RE, &re)) ||
            (r = get_work(c, QCD_F64, S64_RO, &ro)) || (r = get_work(c, QCD_F64, S64_LEVEL, &X)) ||
            (r = get_work(c, PX, S64_LEVEL, &XX)) || (r = get_work(c, PX, S64_XO, &xoX)) ||
            (r = get_work(c, PX, S64_BO, &boX))) {
            c->stream = keep;
            return r;
        }
        // (with an FP64 solution the reconstruction pass also yields the odd
        // rows of the true residual, as in the single solve)
        StencilCall sx;
        sx.prec = PX;
        sx.mode = PX == QCD_F64 ? M_RECON : M_SRC;
        sx.out_par = 1;
        sx.out = xoX;
        sx.in = XX;
        sx.y = boX;
        sx.a = 1.0;
        sx.cc = c->kappa;
        if (PX == QCD_F64) {
            sx.red = R_NORM;
            sx.red_args = RedArgs{c->partials, c->counters, c->states + ST_AUX, FIN_SETN + 2};
        }
        r = launch_stencil(c, sx);
        if (!r && PX != QCD_F64) r = convert_half(c, XX, X);
        if (!r && PX != QCD_F64) r = convert_half(c, xoX, xo);
        const int npar = PX == QCD_F64 ? 1 : 2;  // the even rows (and the odd ones unless fused above)
        for (int par = 0; par < npar && !r; ++par) {
            StencilCall sr;
            sr.prec = QCD_F64;
            sr.mode = M_FULL;
            sr.out_par = par;
            sr.out = par ? ro : re;
            sr.in = par ? X : xo;
            sr.y = par ? xo : X;
            sr.a = -1.0;
            sr.cc = c->kappa;
            sr.z = par ? bo : be;
            sr.d = 1.0;
            sr.red = R_NORM;
            sr.red_args = RedArgs{c->partials, c->counters, c->states + ST_AUX,
                                  (par || PX == QCD_F64) ? FIN_ADDN + 2 : FIN_SETN + 2};
            r = launch_stencil(c, sr);
        }
        if (!r) r = half_to_canon(c, QCD_F64, 0, X, x[i], 0, 1, 0);
        if (!r) r = half_to_canon(c, QCD_F64, 0, xo, x[i], 1, 1, 0);
        SolverState ha;
        if (!r) {
            if (cudaMemcpyAsync(&ha, c->states + ST_AUX, sizeof(ha), cudaMemcpyDeviceToHost, user) != cudaSuccess ||
                cudaStreamSynchronize(user) != cudaSuccess)
                r = QCD_ECUDA;
        }
        c->stream = keep;
        if (r) return r;
        qcd_solve_info inf = {};
        inf.outer_iters = st[i].iter;
        inf.inner_iters[0] = st[i].pad[0];
        inf.dhat_applies[QCD_F32] = st[i].pad[1];
        inf.dhat_applies[QCD_F64] = 2L * st[i].iter - (st[i].exit_half && st[i].done ? 1 : 0);
        const double b2 = ha.norm2[0], r2 = ha.norm2[2];
        inf.true_resid = (b2 > 0 && std::isfinite(b2) && std::isfinite(r2)) ? std::sqrt(r2 / b2) : (b2 == 0 ? 0.0 : NAN);
        inf.status = QCD_OK;
        if (!(inf.true_resid <= tol[i])) {
            // restart this problem alone from its current solution
            qcd_solve_opts o2 = o;
            o2.use_x0 = 1;
            qcd_solve_info i2;
            cudaStream_t keep2 = c->stream;
            c->stream = user;
            const int rs = solve(c, b[i], x[i], tol[i], o2, &i2);
            c->stream = keep2;
            inf.restarts = 1 + i2.restarts;
            inf.outer_iters += i2.outer_iters;
            inf.inner_iters[0] += i2.inner_iters[0];
            for (int k = 0; k < 3; ++k) inf.dhat_applies[k] += i2.dhat_applies[k];
            inf.true_resid = i2.true_resid;
            inf.status = rs;
            if (rs != QCD_OK && status == QCD_OK) status = rs;
        }
        if (infos) infos[i] = inf;
    }
    (void)graph_used;
    return status;
}

}  // namespace qcd
