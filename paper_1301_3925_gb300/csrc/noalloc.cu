// adlbr_step_explicit_noalloc: the explicit step with its scratch buffer in a
// fixed device array of this library instead of caller- or library-allocated
// memory (see include/adlbr.h for who needs it and its limits).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "internal.cuh"

namespace adlbr {

namespace {

// 16 MiB: the FP32 accumulator of up to 4,194,304 points, or the FP64 one of
// up to 2,097,152 points.  Every GPU that loads the library holds it until the
// process exits.
constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
struct Cached {
    CUcontext ctx = nullptr;   // the context the address belongs to
    void *addr = nullptr;
};
Cached g_cache[kMaxDevices];

// The calling thread's current context (driver entry point looked up once);
// nullptr if the driver entry point is unavailable.
CUcontext current_context() {
    static PFN_cuCtxGetCurrent_v4000 get = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(fn);
    });
    CUcontext c = nullptr;
    if (get) get(&c);
    return c;
}

// Device address of g_noalloc_scratch on the current device (the host-side
// name is only a stand-in, never a device address).  Looked up with the
// device current and cached per device together with the context it was
// taken in; a different current context (after a device reset, say) makes
// the next call look it up again.
adlbr_status scratch_address(int dev, void **out) {
    if (dev < 0 || dev >= kMaxDevices) return fail(ADLBR_E_ARG, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_mu);
    const CUcontext ctx = current_context();
    Cached &c = g_cache[dev];
    if (!c.addr || c.ctx != ctx) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        c.addr = p;
        c.ctx = current_context();   // the lookup may have made the primary context current
    }
    *out = c.addr;
    return ADLBR_OK;
}

size_t max_points(adlbr_dtype u_t) {
    return kNoAllocScratchBytes / (u_t == ADLBR_F64 ? sizeof(double) : sizeof(float));
}

}  // namespace

}  // namespace adlbr

using namespace adlbr;

extern "C" adlbr_status adlbr_step_explicit_noalloc(const adlbr_stencils *s, void *u,
                                                    adlbr_dtype u_t, double dt, int nsteps,
                                                    cudaStream_t stream) {
    if (adlbr_status st = check_handle(s)) return st;
    if (!u) return fail(ADLBR_E_ARG, "null buffer");
    if (nsteps < 0 || !(dt >= 0.0)) return fail(ADLBR_E_ARG, "bad dt / nsteps");
    if (u_t < ADLBR_F64 || u_t > ADLBR_BF16) return fail(ADLBR_E_ARG, "bad u dtype");
    const size_t limit = max_points(u_t);
    if ((size_t)s->N > limit)
        return fail(ADLBR_E_SHAPE,
                    "grid of %lld points exceeds the %zu-point limit of the allocation-free step "
                    "(%zu MiB static scratch); use adlbr_step_explicit with caller scratch",
                    (long long)s->N, limit, kNoAllocScratchBytes >> 20);
    int dev = -1;
    ADLBR_CUDA(cudaGetDevice(&dev));
    if (dev != s->device)
        return fail(ADLBR_E_ARG, "current device %d is not the handle's device %d", dev, s->device);
    // the set-up (the array's address on this device) happens on every
    // device's first call, also one with nsteps == 0
    void *acc = nullptr;
    if (adlbr_status st = scratch_address(dev, &acc)) return st;
    if (nsteps == 0) return ADLBR_OK;
    // per step: clear the accumulator, accumulate dt A u, subtract it
    const size_t bytes = (size_t)s->N * (u_t == ADLBR_F64 ? sizeof(double) : sizeof(float));
    for (int k = 0; k < nsteps; ++k) {
        ADLBR_CUDA(cudaMemsetAsync(acc, 0, bytes, stream));
        if (adlbr_status st = launch_accumulate(s, u, acc, u_t, dt, nullptr, stream)) return st;
        if (adlbr_status st = launch_finalize(s, u, acc, u_t, stream)) return st;
    }
    return ADLBR_OK;
}
