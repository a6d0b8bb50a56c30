// Pion two-point function from point-source propagators: the observable the
// solutions of Eq. 1 are computed for (Sec. II-A: expectation values of
// observables made of quarks).  With S the 12 spin-colour columns of the
// propagator from a point source, gamma5-hermiticity (D^dag = g5 D g5) turns
// the pion correlator sum_x Tr[g5 S(x) g5 g5 S(x)^dag g5] into
//
//   C(t) = sum_columns sum_{x in timeslice t} sum_{spin, colour} |S(x)|^2.
//
// One block sums a fixed share of one timeslice's elements over all
// columns; a second kernel adds the shares of each timeslice in order, so
// the result repeats bit for bit.
#include "blas.cuh"

namespace qcd {

namespace {

constexpr int CORR_THREADS = 256;

__device__ __forceinline__ double block_sum_d(double v)
{
    __shared__ double sh[CORR_THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < CORR_THREADS / 32; ++w) s += sh[w];
    return s;
}

// block (ch, t): elements ch*256 + k*chunks*256 + tid of timeslice t, all columns
__global__ void __launch_bounds__(CORR_THREADS) k_corr_partial(const double2 *__restrict__ S, long V, long V3,
                                                               int ncol, int chunks, double *partials)
{
    const int t = blockIdx.y, ch = blockIdx.x;
    const long n = V3 * 12;  // complex elements of one timeslice of one column
    double acc = 0.0;
    for (int col = 0; col < ncol; ++col) {
        const double2 *base = S + ((size_t)col * V + (size_t)t * V3) * 12;
        for (long i = (long)ch * CORR_THREADS + threadIdx.x; i < n; i += (long)chunks * CORR_THREADS) {
            const double2 z = __ldcs(base + i);
            acc = ::fma(z.x, z.x, acc);
            acc = ::fma(z.y, z.y, acc);
        }
    }
    const double s = block_sum_d(acc);
    if (threadIdx.x == 0) partials[(size_t)t * chunks + ch] = s;
}

__global__ void k_corr_final(const double *partials, int chunks, double *C)
{
    if (threadIdx.x != 0) return;
    const int t = blockIdx.x;
    double s = 0.0;
    for (int ch = 0; ch < chunks; ++ch) s += partials[(size_t)t * chunks + ch];
    C[t] = s;
}

}  // namespace

int pion_correlator(qcd_ctx *c, const void *S, int ncol, int on_device, double *C_host)
{
    const long V = (long)c->g.L[0] * c->g.L[1] * c->g.L[2] * c->g.L[3];
    const int Lt = c->g.L[3];
    const long V3 = V / Lt;
    const long n = V3 * 12;
    int chunks = (4 * c->num_sms + Lt - 1) / Lt;
    const long cap = (n + CORR_THREADS - 1) / CORR_THREADS;
    if (chunks > cap) chunks = (int)cap;
    if (chunks < 1) chunks = 1;
    const size_t col_bytes = (size_t)V * 12 * sizeof(double2);
    // device scratch: the per-block partials and C, after one column's
    // staging area when S is in host memory
    const size_t scratch = ((size_t)Lt * chunks + Lt) * sizeof(double);
    const size_t stage = on_device ? 0 : col_bytes;
    int rc;
    if ((rc = ensure_staging(c, stage + scratch))) return rc;
    char *base = (char *)c->staging;
    double *partials = (double *)(base + stage);
    double *Cd = partials + (size_t)Lt * chunks;
    ProfScope prof(c, QCD_K_OTHER, (double)ncol * col_bytes);
    if (on_device) {
        k_corr_partial<<<dim3(chunks, Lt), CORR_THREADS, 0, c->stream>>>((const double2 *)S, V, V3, ncol, chunks,
                                                                           partials);
        QCD_CUDA_CHECK(cudaGetLastError());
        k_corr_final<<<Lt, 32, 0, c->stream>>>(partials, chunks, Cd);
        QCD_CUDA_CHECK(cudaGetLastError());
        QCD_CUDA_CHECK(cudaMemcpyAsync(C_host, Cd, Lt * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        QCD_CUDA_CHECK(cudaStreamSynchronize(c->stream));
        return QCD_OK;
    }
    // host columns: copy one at a time, accumulate C on the host in column order
    std::vector<double> acc(Lt, 0.0), part(Lt);
    for (int col = 0; col < ncol; ++col) {
        QCD_CUDA_CHECK(cudaMemcpyAsync(base, (const char *)S + (size_t)col * col_bytes, col_bytes,
                                       cudaMemcpyHostToDevice, c->stream));
        k_corr_partial<<<dim3(chunks, Lt), CORR_THREADS, 0, c->stream>>>((const double2 *)base, V, V3, 1, chunks,
                                                                           partials);
        QCD_CUDA_CHECK(cudaGetLastError());
        k_corr_final<<<Lt, 32, 0, c->stream>>>(partials, chunks, Cd);
        QCD_CUDA_CHECK(cudaGetLastError());
        QCD_CUDA_CHECK(cudaMemcpyAsync(part.data(), Cd, Lt * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        QCD_CUDA_CHECK(cudaStreamSynchronize(c->stream));
        for (int t = 0; t < Lt; ++t) acc[t] += part[t];
    }
    for (int t = 0; t < Lt; ++t) C_host[t] = acc[t];
    return QCD_OK;
}

}  // namespace qcd
