// cluster.cuh -- device helpers for kernels that run as ONE thread-block
// cluster of kClCTAs CTAs x kClThreads threads: CTA-wide scans, cluster-wide
// offsets and reductions through distributed shared memory, and a stable LSD
// radix sort. Stages that need every CTA's results are separated by the
// hardware cluster barrier (barrier.cluster arrive.release / wait.acquire):
// writes made before it -- to global or shared memory -- are visible to every
// CTA of the cluster after it. Nothing spins.
//
// These kernels serve the small, latency-bound part of the pipeline (after
// the representative filter the survivors and the skyline are a few
// thousand to a few ten thousand rows): one launch replaces a chain of small
// grid-wide kernels.
#pragma once

#include <cooperative_groups.h>

#include "gres_internal.cuh"

namespace gres {

namespace cg = cooperative_groups;

constexpr int kClCTAs = 16;         // CTAs per cluster (above the portable 8: opted in at launch)
constexpr int kClThreads = 1024;
constexpr int kClWarps = kClThreads / 32;
// dynamic shared memory of the radix sort, in words
constexpr int kClSortWords = 512 + kClWarps + 2 * kClWarps * 256;
constexpr size_t kClSortBytes = sizeof(uint32_t) * kClSortWords;

// Exclusive scan of v over the CTA; *total = the CTA's sum. wsum: kClWarps
// words of shared memory. Every thread of the CTA must call it.
__device__ __forceinline__ uint32_t cta_scan(uint32_t v, uint32_t *total, uint32_t *wsum) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t incl = v;
    #pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    uint32_t before = 0, all = 0;
    #pragma unroll 8
    for (int j = 0; j < kClWarps; j++) {
        const uint32_t x = wsum[j];
        before += j < w ? x : 0u;
        all += x;
    }
    __syncthreads();
    *total = all;
    return before + incl - v;
}

// This CTA's exclusive offset among the CTAs of the cluster: every CTA puts
// its count in *slot (shared), then after a cluster barrier reads the slots
// of all CTAs. *total = the cluster's sum. *slot must not be rewritten before
// the next cluster barrier.
__device__ __forceinline__ uint32_t cluster_offset(cg::cluster_group &cl, uint32_t *slot, uint32_t count,
                                                   uint32_t *total) {
    if (threadIdx.x == 0) *slot = count;
    cl.sync();
    const int r = (int)cl.block_rank();
    uint32_t before = 0, all = 0;
    #pragma unroll
    for (int q = 0; q < kClCTAs; q++) {
        const uint32_t c = *cl.map_shared_rank(slot, q);
        before += q < r ? c : 0u;
        all += c;
    }
    *total = all;
    return before;
}

// Per-attribute minimum / maximum over the cluster: each CTA has reduced its
// own values into lo_s / hi_s (shared, D words each); after a cluster barrier
// every thread reads all CTAs' arrays.
template <int D>
__device__ __forceinline__ void cluster_range(cg::cluster_group &cl, uint32_t *lo_s, uint32_t *hi_s,
                                              uint32_t (&lo)[D], uint32_t (&hi)[D]) {
    cl.sync();
    #pragma unroll
    for (int q = 0; q < D; q++) { lo[q] = 0xFFFFFFFFu; hi[q] = 0u; }
    #pragma unroll
    for (int c = 0; c < kClCTAs; c++) {
        const uint32_t *rl = cl.map_shared_rank(lo_s, c);
        const uint32_t *rh = cl.map_shared_rank(hi_s, c);
        #pragma unroll
        for (int q = 0; q < D; q++) { lo[q] = min(lo[q], rl[q]); hi[q] = max(hi[q], rh[q]); }
    }
}

// Warp-reduced min / max of D values into shared arrays (atomics).
template <int D>
__device__ __forceinline__ void cta_range_add(const uint32_t (&lo)[D], const uint32_t (&hi)[D], uint32_t *lo_s,
                                              uint32_t *hi_s) {
    #pragma unroll
    for (int q = 0; q < D; q++) {
        uint32_t a = lo[q], b = hi[q];
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a = min(a, __shfl_xor_sync(0xffffffffu, a, o));
            b = max(b, __shfl_xor_sync(0xffffffffu, b, o));
        }
        if ((threadIdx.x & 31) == 0 && a <= b) {
            atomicMin(&lo_s[q], a);
            atomicMax(&hi_s[q], b);
        }
    }
}

// Key range over the cluster (each CTA reduced its keys into kr[0] = min,
// kr[1] = max in shared memory); includes a cluster barrier.
__device__ __forceinline__ void cluster_key_range(cg::cluster_group &cl, unsigned long long *kr,
                                                  unsigned long long *kmin, unsigned long long *kmax) {
    cl.sync();
    unsigned long long a = ~0ull, b = 0ull;
    #pragma unroll
    for (int c = 0; c < kClCTAs; c++) {
        const unsigned long long *x = cl.map_shared_rank(kr, c);
        a = x[0] < a ? x[0] : a;
        b = x[1] > b ? x[1] : b;
    }
    *kmin = a;
    *kmax = b;
}

__device__ __forceinline__ void cta_key_add(unsigned long long kmn, unsigned long long kmx, unsigned long long *kr) {
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long a = __shfl_xor_sync(0xffffffffu, kmn, o);
        const unsigned long long b = __shfl_xor_sync(0xffffffffu, kmx, o);
        kmn = a < kmn ? a : kmn;
        kmx = b > kmx ? b : kmx;
    }
    if ((threadIdx.x & 31) == 0 && kmn <= kmx) {
        atomicMin(&kr[0], kmn);
        atomicMax(&kr[1], kmx);
    }
}

// Digit passes for keys in [kmin, kmax] (8-bit digits of key - kmin).
__device__ __forceinline__ int key_passes(unsigned long long kmin, unsigned long long kmax) {
    const unsigned long long range = kmax >= kmin ? kmax - kmin : 0ull;
    const int bits = range ? 64 - __clzll((long long)range) : 0;
    return (bits + 7) >> 3;
}

// Stable LSD radix sort of (k0[i], v0[i]), i < n, by key - kmin over
// `passes` 8-bit digits, inside the cluster; the result is in buffer
// passes & 1 (k0/v0 or k1/v1). CTA r owns the contiguous range
// [r c, (r + 1) c) (c = ceil(n / C) rounded up to 32), so stability only needs
// ranks in index order inside each CTA. Per pass: a shared-memory histogram
// of the CTA's range; a cluster barrier; each CTA reads every CTA's histogram
// (distributed shared memory) and takes, per digit, the items of all smaller
// digits plus those of its digit in lower-ranked CTAs as its base; then it
// scatters its range in rounds of kClThreads items (warp match_any ranks, a
// per-digit prefix over the warps, a running per-digit base); a cluster
// barrier ends the pass. sm: kClSortWords words of shared memory. Every thread
// of every CTA calls it with the same arguments.
__device__ __forceinline__ void cluster_radix_sort(cg::cluster_group &cl, uint32_t *sm, unsigned long long *k0,
                                                   uint32_t *v0, unsigned long long *k1, uint32_t *v1, long long n,
                                                   unsigned long long kmin, int passes) {
    uint32_t *hist = sm;                      // 256
    uint32_t *base = sm + 256;                // 256
    uint32_t *wsum = sm + 512;                // kClWarps
    uint32_t *wcnt = sm + 512 + kClWarps;     // kClWarps x 256
    uint32_t *woff = wcnt + kClWarps * 256;   // kClWarps x 256
    const int C = (int)cl.num_blocks();
    const int r = (int)cl.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const long long chunk = (((n + C - 1) / C) + 31) & ~31LL;
    const long long b0 = min(n, (long long)r * chunk), b1 = min(n, b0 + chunk);
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int pass = 0; pass < passes; pass++) {
        const unsigned long long *kin = (pass & 1) ? k1 : k0;
        const uint32_t *vin = (pass & 1) ? v1 : v0;
        unsigned long long *kout = (pass & 1) ? k0 : k1;
        uint32_t *vout = (pass & 1) ? v0 : v1;
        const int shift = 8 * pass;
        if (tid < 256) hist[tid] = 0;
        for (int j = tid; j < kClWarps * 256; j += kClThreads) wcnt[j] = 0;
        __syncthreads();
        for (long long i = b0 + tid; i < b1; i += kClThreads)
            atomicAdd(&hist[(uint32_t)(((kin[i] - kmin) >> shift) & 255ull)], 1u);
        cl.sync();
        if (tid < 256) {
            uint32_t tot = 0, pre = 0;
            #pragma unroll
            for (int q = 0; q < kClCTAs; q++) {   // independent remote loads, all in flight
                const uint32_t c = cl.map_shared_rank(hist, q)[tid];
                tot += c;
                pre += q < r ? c : 0u;
            }
            uint32_t incl = tot;
            #pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (lane == 31) wsum[w] = incl;
            asm volatile("bar.sync 1, 256;" ::: "memory");
            uint32_t before = 0;
            #pragma unroll
            for (int j = 0; j < 8; j++) before += j < w ? wsum[j] : 0u;
            base[tid] = before + incl - tot + pre;
        }
        __syncthreads();
        for (long long r0 = b0; r0 < b1; r0 += kClThreads) {
            const long long i = r0 + tid;
            const bool valid = i < b1;
            unsigned long long key = 0;
            uint32_t val = 0;
            uint32_t dg = 256;  // invalid items share a digit no real item has
            if (valid) {
                key = kin[i];
                val = vin[i];
                dg = (uint32_t)(((key - kmin) >> shift) & 255ull);
            }
            const unsigned peers = __match_any_sync(0xffffffffu, dg);
            const uint32_t rank = __popc(peers & lt_mask);
            if (valid && rank == 0) wcnt[w * 256 + dg] = __popc(peers);
            __syncthreads();
            if (tid < 256) {
                uint32_t run = base[tid];
                #pragma unroll 8
                for (int j = 0; j < kClWarps; j++) {
                    const uint32_t c = wcnt[j * 256 + tid];
                    wcnt[j * 256 + tid] = 0;
                    woff[j * 256 + tid] = run;
                    run += c;
                }
                base[tid] = run;
            }
            __syncthreads();
            if (valid) {
                const uint32_t pos = woff[w * 256 + dg] + rank;
                kout[pos] = key;
                vout[pos] = val;
            }
        }
        cl.sync();
    }
}

// ---- the same sort with the data in the cluster's shared memory -------------
// For n <= kClCTAs * kClSmemCap items with 32-bit keys. CTA r holds positions
// [r c, r c + c) of the current order (c = ceil(n / C) rounded up to 32) in
// its buffers kb[cur] / vb[cur]; a pass scatters each item straight into the
// buffer of the CTA that owns its new position (distributed shared memory), so
// the passes touch no global memory. Ranks, bases and barriers as in
// cluster_radix_sort. Returns the buffer (0 / 1) holding the result.
constexpr int kClSmemCap = 8192;
// dynamic shared memory: the sort's words plus two (key, value) buffers
constexpr size_t kClSmemBytes = kClSortBytes + sizeof(uint32_t) * 4 * (size_t)kClSmemCap;
static_assert((int64_t)kClCTAs * kClSmemCap >= kClusterSortMax,
              "the shared-memory sort must hold every input the cluster path takes");

__device__ __forceinline__ long long cluster_chunk(long long n) {
    return (((n + kClCTAs - 1) / kClCTAs) + 31) & ~31LL;
}

__device__ __forceinline__ int cluster_radix_sort_smem(cg::cluster_group &cl, uint32_t *sm, uint32_t *kb0,
                                                       uint32_t *vb0, uint32_t *kb1, uint32_t *vb1, long long n,
                                                       uint32_t kmin, int passes, int cur) {
    uint32_t *hist = sm;                      // 256
    uint32_t *base = sm + 256;                // 256
    uint32_t *wsum = sm + 512;                // kClWarps
    uint32_t *wcnt = sm + 512 + kClWarps;     // kClWarps x 256
    uint32_t *woff = wcnt + kClWarps * 256;   // kClWarps x 256
    const int r = (int)cl.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const long long c = cluster_chunk(n);
    const long long b0 = min(n, (long long)r * c);
    const int cnt = (int)(min(n, b0 + c) - b0);
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int pass = 0; pass < passes; pass++) {
        const uint32_t *kin = cur ? kb1 : kb0, *vin = cur ? vb1 : vb0;
        const int shift = 8 * pass;
        if (tid < 256) hist[tid] = 0;
        for (int j = tid; j < kClWarps * 256; j += kClThreads) wcnt[j] = 0;
        __syncthreads();
        for (int i = tid; i < cnt; i += kClThreads) atomicAdd(&hist[((kin[i] - kmin) >> shift) & 255u], 1u);
        cl.sync();
        if (tid < 256) {
            uint32_t tot = 0, pre = 0;
            #pragma unroll
            for (int q = 0; q < kClCTAs; q++) {
                const uint32_t v = cl.map_shared_rank(hist, q)[tid];
                tot += v;
                pre += q < r ? v : 0u;
            }
            uint32_t incl = tot;
            #pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (lane == 31) wsum[w] = incl;
            asm volatile("bar.sync 1, 256;" ::: "memory");
            uint32_t before = 0;
            #pragma unroll
            for (int j = 0; j < 8; j++) before += j < w ? wsum[j] : 0u;
            base[tid] = before + incl - tot + pre;
        }
        __syncthreads();
        uint32_t *kout = cur ? kb0 : kb1, *vout = cur ? vb0 : vb1;
        for (int r0 = 0; r0 < cnt; r0 += kClThreads) {
            const int i = r0 + tid;
            const bool valid = i < cnt;
            uint32_t key = 0, val = 0, dg = 256;  // invalid items share a digit no real item has
            if (valid) {
                key = kin[i];
                val = vin[i];
                dg = ((key - kmin) >> shift) & 255u;
            }
            const unsigned peers = __match_any_sync(0xffffffffu, dg);
            const uint32_t rank = __popc(peers & lt_mask);
            if (valid && rank == 0) wcnt[w * 256 + dg] = __popc(peers);
            __syncthreads();
            if (tid < 256) {
                uint32_t run = base[tid];
                #pragma unroll 8
                for (int j = 0; j < kClWarps; j++) {
                    const uint32_t v = wcnt[j * 256 + tid];
                    wcnt[j * 256 + tid] = 0;
                    woff[j * 256 + tid] = run;
                    run += v;
                }
                base[tid] = run;
            }
            __syncthreads();
            if (valid) {
                const uint32_t pos = woff[w * 256 + dg] + rank;
                const int owner = (int)(pos / (uint32_t)c);
                const uint32_t li = pos - (uint32_t)owner * (uint32_t)c;
                cl.map_shared_rank(kout, owner)[li] = key;
                cl.map_shared_rank(vout, owner)[li] = val;
            }
        }
        cl.sync();
        cur ^= 1;
    }
    return cur;
}

// Launches a cluster kernel: one cluster of kClCTAs CTAs (the helpers above
// assume exactly that many), kClThreads threads,
// `smem` bytes of dynamic shared memory (the kernel's limit is raised on first
// use).
template <typename... KArgs, typename... Args>
cudaError_t launch_cluster(void (*kernel)(KArgs...), size_t smem, bool *configured, cudaStream_t st,
                           Args... args) {
    if (!*configured) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        if (kClCTAs > 8) {
            e = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            if (e != cudaSuccess) return e;
        }
        *configured = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kClCTAs, 1, 1);
    cfg.blockDim = dim3(kClThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kClCTAs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, args...);
    note_launch();
    return e;
}

}  // namespace gres
