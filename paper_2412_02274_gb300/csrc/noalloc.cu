// noalloc.cu -- gres_compute_static: gres_compute with the library's own fixed
// scratch area instead of a caller-provided workspace.
//
// Who needs it: callers that cannot allocate device memory at the moment they
// want a result. Examples: a plugin running on another framework's stream
// whose caching allocator already owns the free device memory (a cudaMalloc
// there fails or breaks that framework's accounting); a latency-critical
// loop where cudaMalloc / cudaFree are ruled out because they can
// synchronize the whole device; a deployment that fixes its device footprint
// at start-up. Such callers still pass their input and output buffers; only
// the scratch comes from here.
//
// The scratch is one file-scope __device__ array of kStaticScratchBytes. Every
// GPU on which this library's kernels are loaded holds it until the process
// exits. In host code the array's name is only a host-side stand-in, so its
// device address is looked up with cudaGetSymbolAddress (with that device
// current) and cached per device together with the id of the CUDA context it
// belongs to; the first call on a device does that lookup, and so does the
// first call after the context changed (a cudaDeviceReset destroys the
// context, and the array's address with it). A lookup is refused inside a
// stream capture, which is why the first call should happen before any
// capture. All calls share the array: it keeps the previous call's contents
// (every call re-initialises what must start at zero before using it), and
// calls that overlap on the GPU -- two streams, or two host threads without
// ordering -- race on it and must be serialised by the caller.
#include "gres_internal.cuh"

#include <cuda.h>   // CUcontext / CUresult only: the two driver calls are fetched at run time

#include <cstdio>
#include <mutex>

namespace {

constexpr size_t kStaticScratchBytes = size_t(16) << 20;   // 16 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

struct ScratchAddr {
    void *addr = nullptr;
    unsigned long long ctx = 0;   // id of the context the address belongs to (0: unknown)
};
ScratchAddr g_scratch[kMaxDevices];
std::mutex g_scratch_mu;

using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);

// Unique id of the calling thread's current context, or 0 when there is none
// (or the driver cannot say). A context created after a device reset gets a
// new id. Neither driver call queues work or allocates, so this is safe
// inside a stream capture.
unsigned long long current_context_id() {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(p);
        cudaGetLastError();
    });
    if (!get_current || !get_id) return 0;
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of g_static_scratch on the current device: the cached one
// while the context is unchanged, else looked up again (not inside a stream
// capture: *capturing is set and cudaErrorStreamCaptureUnsupported returned).
cudaError_t scratch_address(cudaStream_t st, void **out, bool *capturing) {
    *capturing = false;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    const unsigned long long ctx = current_context_id();
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    ScratchAddr &c = g_scratch[dev];
    if (c.addr && ctx != 0 && c.ctx == ctx) {
        *out = c.addr;
        return cudaSuccess;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
        // no lookup inside a capture; without a context id the cached address is kept
        if (c.addr && ctx == 0) {
            *out = c.addr;
            return cudaSuccess;
        }
        *capturing = true;
        return cudaErrorStreamCaptureUnsupported;
    }
    cudaGetLastError();
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    c.addr = p;
    c.ctx = current_context_id();   // the lookup made the context current if it was not
    *out = p;
    return cudaSuccess;
}

}  // namespace

extern "C" {

size_t gres_static_scratch_bytes(void) { return kStaticScratchBytes; }

gres_status gres_compute_static(const uint32_t *d_data, int64_t n, int32_t d, int32_t dir,
                                const uint32_t *h_steps, int32_t k, const gres_plan_cfg *cfg,
                                int64_t *d_sky_idx, int32_t *d_step_idx,
                                int64_t *d_sky_count, int64_t *h_sky_count, void *stream) {
    size_t need = 0;
    gres_status s = gres_workspace_size(n, d, k, &need);   // validates n, d, k
    if (s != GRES_OK) return s;
    if (need > kStaticScratchBytes) {
        char msg[224];
        std::snprintf(msg, sizeof(msg),
                      "gres_compute_static: n=%lld, d=%d, k=%d needs %zu bytes of scratch but the "
                      "static scratch holds %zu; use gres_compute with a caller workspace",
                      (long long)n, (int)d, (int)k, need, kStaticScratchBytes);
        return gres::set_error(GRES_EINVAL, msg);
    }
    void *scratch = nullptr;
    bool capturing = false;
    cudaError_t e = scratch_address(static_cast<cudaStream_t>(stream), &scratch, &capturing);
    if (capturing)
        return gres::set_error(GRES_EINVAL,
                               "gres_compute_static: the first call on a device (or after a device reset) "
                               "must come before any stream capture");
    if (e != cudaSuccess) {
        char msg[160];
        std::snprintf(msg, sizeof(msg), "gres_compute_static: cudaGetSymbolAddress: %s",
                      cudaGetErrorString(e));
        return gres::set_error(GRES_ECUDA, msg);
    }
    return gres_compute(d_data, n, d, dir, h_steps, k, cfg, scratch, kStaticScratchBytes,
                        d_sky_idx, d_step_idx, d_sky_count, h_sky_count, nullptr, stream);
}

}  // extern "C"
