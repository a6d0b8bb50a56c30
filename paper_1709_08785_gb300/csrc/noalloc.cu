// qcd_dslash_eo_noalloc: the hopping term on one parity, like qcd_dslash_eo,
// for callers that must not allocate device memory during the call.
//
// qcd_dslash_eo converts its canonical input into the library's internal
// site-blocked layout and its result back, through a staging buffer that the
// context allocates on first use.  Code that cannot call cudaMalloc at that
// point -- a real-time or serving loop whose allocator must stay untouched
// after start-up, a caller holding a memory budget that was fixed in advance,
// or a host thread that is not allowed to synchronise the device (cudaMalloc
// and cudaFree can) -- uses this entry point instead.  Its staging lives in a
// file-scope device array that the CUDA runtime creates when the library's
// module is loaded onto a device, so the call itself allocates nothing.
#include <mutex>

#include "blas.cuh"

namespace qcd {

// 24 MiB: room for the input and the output of one half-lattice vector in
// FP64 (384 bytes per site of one parity), i.e. Vh <= 65536 sites, a full
// lattice of up to 131072 sites (16^3 x 32).  Every device that loads the
// library holds this array until the process exits.
constexpr size_t NOALLOC_SCRATCH_BYTES = 24u << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int MAX_DEVICES = 64;
std::mutex g_mutex;
void *g_scratch_ptr[MAX_DEVICES] = {};

// Device address of the scratch array on the current device.  In host code
// g_noalloc_scratch names a host-side shadow, not device memory, so the
// address is looked up once per device with that device current.
int scratch_address(int device, void **out)
{
    if (device < 0 || device >= MAX_DEVICES) {
        set_error_message("device ordinal %d out of range", device);
        return QCD_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)", __FILE__, __LINE__);
            return QCD_ECUDA;
        }
        g_scratch_ptr[device] = p;
    }
    *out = g_scratch_ptr[device];
    return QCD_OK;
}

}  // namespace
}  // namespace qcd

using namespace qcd;

extern "C" int qcd_dslash_eo_noalloc(qcd_ctx *c, void *out, const void *in, int out_parity, int dagger, int prec)
{
    if (!c || !out || !in) {
        set_error_message("null argument");
        return QCD_EINVAL;
    }
    if (prec < QCD_F64 || prec > QCD_DF64 || (out_parity != 0 && out_parity != 1)) {
        set_error_message("bad precision %d or parity %d", prec, out_parity);
        return QCD_EINVAL;
    }
    if (!c->have_gauge) {
        set_error_message("no gauge field loaded");
        return QCD_ESTATE;
    }
    const size_t hb = hvec_bytes(c->g, prec);
    const size_t nb = prec == QCD_F16 ? (size_t)c->g.Vh_pad * sizeof(float) : 0;
    const size_t need = 2 * (hb + nb);
    if (need > NOALLOC_SCRATCH_BYTES) {
        set_error_message("lattice too large for qcd_dslash_eo_noalloc: needs %zu bytes of scratch, the limit is %zu "
                          "(at most %zu sites per parity in FP64)",
                          need, NOALLOC_SCRATCH_BYTES, NOALLOC_SCRATCH_BYTES / 384);
        return QCD_EINVAL;
    }
    // the array's address is per device and is looked up with the device
    // current; the kernels run on the context's stream, i.e. its device
    int dev = -1;
    QCD_CUDA_CHECK(cudaGetDevice(&dev));
    if (dev != c->device) {
        set_error_message("qcd_dslash_eo_noalloc: the context lives on device %d but device %d is current; make the "
                          "context's device current before the call",
                          c->device, dev);
        return QCD_EINVAL;
    }
    void *base = nullptr;
    int rc = scratch_address(dev, &base);
    if (rc) return rc;
    HVec vin, vout;
    vin.prec = vout.prec = prec;
    vin.p = base;
    vout.p = (char *)base + hb;
    if (nb) {
        vin.norm = (float *)((char *)base + 2 * hb);
        vout.norm = (float *)((char *)base + 2 * hb + nb);
    }
    // timing events are created on demand by the profiler: keep it off here
    const bool prof = c->profiling;
    c->profiling = false;
    const int f32io = prec == QCD_F32 || prec == QCD_F16;  // QCD_DF64 takes complex128, as QCD_F64
    rc = canon_to_half(c, prec, f32io, in, -1, vin, 1, 0);
    if (rc == QCD_OK) {
        StencilCall s;
        s.prec = prec;
        s.mode = M_HOP;
        s.dagger = dagger ? 1 : 0;
        s.out_par = out_parity;
        s.out = vout;
        s.in = vin;
        rc = launch_stencil(c, s);
    }
    if (rc == QCD_OK) rc = half_to_canon(c, prec, f32io, vout, out, -1, 1, 0);
    c->profiling = prof;
    return rc;
}
