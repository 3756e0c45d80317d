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
// device address is looked up once per device with cudaGetSymbolAddress (with
// that device current) and cached; the first call on a device does that
// lookup, which is why the first call should happen before any stream
// capture. All calls share the array: it keeps the previous call's contents
// (every call re-initialises what must start at zero before using it), and
// calls that overlap on the GPU -- two streams, or two host threads without
// ordering -- race on it and must be serialised by the caller.
#include "gres_internal.cuh"

#include <cstdio>
#include <mutex>

namespace {

constexpr size_t kStaticScratchBytes = size_t(16) << 20;   // 16 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

void *g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Device address of g_static_scratch on the current device (looked up once).
cudaError_t scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (g_scratch_addr[dev] == nullptr) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
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
    cudaError_t e = scratch_address(&scratch);
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
