// Single-pass grid reduction with a deterministic order, and the BiCGStab
// scalar updates that its last block performs.
//
// Each block reduces its threads' values (warp shuffles, then one warp over
// the warp sums, the other warps leaving through a non-blocking barrier
// arrival) and writes one partial per block; all blocks but the last count
// themselves with a release add and retire, and the highest-indexed block
// (dispatched last) waits, bounded, for that count, adds the partials in
// block order and runs the finaliser on the solver state.  The sum order
// depends only on the launch shape, so results repeat bit for bit from run
// to run.  This replaces the paper's MPI_Allreduce of every dot product and
// norm (Sec. IV-B).
#pragma once

#include "ctx.cuh"

namespace qcd {

__device__ __forceinline__ bool finite_d(double x) { return isfinite(x); }

// The scalar recurrences of BiCGStab (Alg. 2, with alpha = rho0/<r~|q> and
// beta = (rho1/rho0)(alpha/omega), the standard reading of the printed
// formulas), run by one thread at the end of a grid reduction, on the
// critical path between two kernels: each quotient takes one FP64 division
// (a long dependent sequence on GB300, whose FP64 rate is 1/64 of FP32) and
// the breakdown test compares squares instead of taking square roots.
__device__ inline void finalize(int op, SolverState *st)
{
    const double *s = st->sum;
    switch (op) {
    case FIN_ALPHA: {
        const double dr = s[0], di = s[1];
        const double den = dr * dr + di * di;
        st->iter += 1;
        if (!(den > 0.0) || !finite_d(den)) {
            st->done = 1;
            st->status = finite_d(den) ? QCD_EBREAKDOWN : QCD_ENONFINITE;
            break;
        }
        const double inv = 1.0 / den;
        st->alpha[0] = (st->rho0[0] * dr + st->rho0[1] * di) * inv;
        st->alpha[1] = (st->rho0[1] * dr - st->rho0[0] * di) * inv;
        break;
    }
    case FIN_S:
        st->rr = s[0];
        if (!finite_d(s[0])) {
            st->done = 1;
            st->status = QCD_ENONFINITE;
        } else if (s[0] < st->tol2) {
            st->done = 1;
            st->status = QCD_OK;
            st->exit_half = 1;
        }
        break;
    case FIN_OMEGA: {
        const double tt = s[2];
        if (!(tt > 0.0) || !finite_d(tt) || !finite_d(s[0]) || !finite_d(s[1])) {
            st->done = 1;
            st->status = finite_d(tt) ? QCD_EBREAKDOWN : QCD_ENONFINITE;
            st->exit_half = 1;
            break;
        }
        const double inv = 1.0 / tt;
        st->omega[0] = s[0] * inv;
        st->omega[1] = s[1] * inv;
        if (st->omega[0] == 0.0 && st->omega[1] == 0.0) {
            st->done = 1;
            st->status = QCD_EBREAKDOWN;
            st->exit_half = 1;
        }
        break;
    }
    case FIN_X: {
        const double rr = s[0], r1r = s[1], r1i = s[2];
        st->rr = rr;
        st->exit_half = 0;
        if (!finite_d(rr) || !finite_d(r1r) || !finite_d(r1i)) {
            st->done = 1;
            st->status = QCD_ENONFINITE;
        } else if (rr < st->tol2) {
            st->done = 1;
            st->status = QCD_OK;
        } else if (st->bd_eps >= 0.0 && r1r * r1r + r1i * r1i <= st->bd_eps * st->bd_eps * (st->rt2 * rr)) {
            st->done = 1;
            st->status = QCD_EBREAKDOWN;
        } else if (st->iter >= st->maxit) {
            st->done = 1;
            st->status = QCD_ENOTCONV;
        } else {
            // beta = (rho1/rho0) * (alpha/omega) = (rho1 alpha) / (rho0 omega)
            const double nr = r1r * st->alpha[0] - r1i * st->alpha[1];
            const double ni = r1r * st->alpha[1] + r1i * st->alpha[0];
            const double dr = st->rho0[0] * st->omega[0] - st->rho0[1] * st->omega[1];
            const double di = st->rho0[0] * st->omega[1] + st->rho0[1] * st->omega[0];
            const double inv = 1.0 / (dr * dr + di * di);
            st->beta[0] = (nr * dr + ni * di) * inv;
            st->beta[1] = (ni * dr - nr * di) * inv;
            st->rho0[0] = r1r;
            st->rho0[1] = r1i;
        }
        break;
    }
    case FIN_INIT:
    case FIN_RESTART:
        // r = r~ = p = b: rho0 = |b|^2; a zero right-hand side is converged
        if (op == FIN_INIT && st->tol2_rel > 0.0) st->tol2 = st->tol2_rel * s[0];
        st->norm2[1] = s[0];
        st->rr = s[0];
        st->rt2 = s[0];
        st->rho0[0] = s[0];
        st->rho0[1] = 0.0;
        st->exit_half = 0;
        if (!finite_d(s[0])) {
            st->done = 1;
            st->status = QCD_ENONFINITE;
        } else if (s[0] <= st->tol2 || s[0] == 0.0) {
            st->done = 1;
            st->status = QCD_OK;
        } else {
            st->done = 0;
            st->status = QCD_OK;
        }
        break;
    default:
        if (op >= FIN_SETN && op < FIN_SETN + 4) st->norm2[op - FIN_SETN] = s[0];
        else if (op >= FIN_ADDN && op < FIN_ADDN + 4) st->norm2[op - FIN_ADDN] += s[0];
        break;
    }
    for (int k = 0; k < 2; ++k) {
        st->coef[k] = (float)st->alpha[k];
        st->coef[2 + k] = (float)st->omega[k];
        st->coef[4 + k] = (float)st->beta[k];
    }
}

// Reduce N values over the grid; blocks may be 1-D or 2-D.  The per-thread
// values and the warp stage are in the accumulator type A (float for the
// FP32 and FP16 levels, whose sums feed FP32 recurrences: GB300's FP64 rate
// is 1/64 of its FP32 rate, and per-thread FP64 adds slowed those kernels
// in proportion to their size); warp sums and everything after are FP64.
// bidx / nblk: the block's index among the nblk blocks of this reduction
// (blockIdx.x / gridDim.x, or another grid dimension when several
// reductions share one launch); the block with index nblk - 1 is dispatched
// after every other block of its reduction.
template <int N, class A>
__device__ __forceinline__ void grid_reduce_ex(A v[N], const RedArgs &ra, int bidx, int nblk)
{
    __shared__ double sh[32][4];
    __shared__ int last;
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int nthr = blockDim.x * blockDim.y;
    const int lane = tid & 31, wid = tid >> 5, nw = (nthr + 31) >> 5;
#pragma unroll
    for (int k = 0; k < N; ++k)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < N; ++k) sh[wid][k] = (double)v[k];
    if (bidx != nblk - 1) {
        // Every block but the last: warps 1.. post their sums and leave at
        // once (bar.arrive does not wait; their output stores proceed), warp
        // 0 waits for them (bar.sync on the same named barrier), adds the
        // sums in warp order, writes the block's partial and counts it.
        // Nothing holds a block at a full-block barrier.
        if (wid != 0) {
            asm volatile("bar.arrive 1, %0;" ::"r"(nthr) : "memory");
            return;
        }
        asm volatile("bar.sync 1, %0;" ::"r"(nthr) : "memory");
        double bsum[N];
#pragma unroll
        for (int k = 0; k < N; ++k) {
            double t = lane < nw ? sh[lane][k] : 0.0;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
            bsum[k] = t;
        }
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < N; ++k) ra.partials[(size_t)bidx * 4 + k] = bsum[k];
            // the partial ordered before the count; no reply awaited
            asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(ra.counter) : "memory");
        }
        return;
    }
    __syncthreads();
    if (wid == 0) {
        double bsum[N];
#pragma unroll
        for (int k = 0; k < N; ++k) {
            double t = lane < nw ? sh[lane][k] : 0.0;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
            bsum[k] = t;
        }
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < N; ++k) ra.partials[(size_t)bidx * 4 + k] = bsum[k];
            // the highest-indexed block is dispatched last: it waits
            // (bounded) until every other block has counted
            const unsigned want = (unsigned)nblk - 1;
            long long n = 0;
            unsigned got;
            for (;;) {
                asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(got) : "l"(ra.counter) : "memory");
                if (got >= want || ++n > (1ll << 26)) break;
                __nanosleep(32);
            }
            last = got >= want ? 1 : 0;
        }
    }
    __syncthreads();
    if (!last) {  // the other blocks never all counted: report, do not hang
        if (tid == 0) {
            ra.st->status = QCD_ETIMEOUT;
            ra.st->done = 1;
            *ra.counter = 0u;
            __threadfence();
        }
        return;
    }
    double s[N];
#pragma unroll
    for (int k = 0; k < N; ++k) s[k] = 0.0;
    // eight independent loads in flight per thread, the last batch
    // predicated: the partials arrive in ceil(G / 8 nthr) L2 round trips
    const int G = nblk;
    for (int b0 = tid; b0 < G; b0 += 8 * nthr) {
        double t[8][N];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int b = b0 + u * nthr;
#pragma unroll
            for (int k = 0; k < N; ++k) t[u][k] = b < G ? __ldcg(ra.partials + (size_t)b * 4 + k) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int k = 0; k < N; ++k) s[k] += t[u][k];
    }
#pragma unroll
    for (int k = 0; k < N; ++k)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s[k] += __shfl_down_sync(0xffffffffu, s[k], off);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < N; ++k) sh[wid][k] = s[k];
    __syncthreads();
    if (tid == 0) {
        for (int k = 0; k < N; ++k) {
            double t = 0.0;
            for (int w = 0; w < nw; ++w) t += sh[w][k];
            ra.st->sum[k] = t;
        }
        for (int k = N; k < 4; ++k) ra.st->sum[k] = 0.0;
        finalize(ra.op, ra.st);
        // no fence: the kernel ends here, and its completion publishes the
        // state and the counter to the next kernel in stream order
        *ra.counter = 0u;
    }
}

template <int N, class A>
__device__ __forceinline__ void grid_reduce(A v[N], const RedArgs &ra)
{
    grid_reduce_ex<N, A>(v, ra, (int)blockIdx.x, (int)gridDim.x);
}

}  // namespace qcd
