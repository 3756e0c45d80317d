// radix.cuh -- stable LSD radix sort of (uint64 key, uint32 value) pairs inside one
// cooperative launch (every block resident), for the survivor and skyline sorts of
// inputs above kClusterSortMax rows.
//
// Sorts ws.keys[0]/ws.vals[0] (n pairs) by key - key_min, 8-bit digits, for the
// passes the key range in the header needs (at most max_passes): pass p reads
// buffer p & 1 and writes buffer (p + 1) & 1. Each pass has three phases
// separated by grid-wide barriers: per-tile digit histograms (tiles of 1024 items,
// blocks take tiles in turn), a per-digit exclusive scan over the tiles (blocks
// take digits in turn), and a stable scatter in which each tile ranks its items
// per digit in input order (warp match_any for ranks within a warp, a per-digit
// prefix over warps, a running per-digit carry over the tile's rounds).
//
// The grid-wide barrier waits a bounded time: a block that waits too long sets
// kStatusTimeout in the header and the kernel returns (the host reports
// GRES_ETIMEOUT); every block then leaves at its next barrier.
#pragma once

#include "gres_internal.cuh"

namespace gres {

constexpr int kRxThreads = 256;                 // threads per block of a cooperative sort kernel
constexpr int kRxItems = 4;
constexpr int kRxTile = kRxThreads * kRxItems;  // 1024 items per tile (sort_blocks counts these)
constexpr int kRxWarps = kRxThreads / 32;
constexpr unsigned kBarrierSpins = 1u << 20;    // polls of 128 ns sleep plus a load: about a second at most

struct RadixShared {
    uint32_t cnt[256];
    uint32_t base[256];
    uint32_t wcnt[kRxWarps][256];
    uint32_t woff[kRxWarps][256];
    uint32_t wsum[kRxWarps];
    int ok;
};

// Grid-wide barrier of a cooperative launch: bar[0] counts arrivals, bar[1] is the
// generation (both in the workspace header; bar[0] is 0 between barriers). Returns
// false, in every thread of the block, if the wait ran out.
__device__ __forceinline__ bool grid_barrier(unsigned *bar, unsigned *status, int *ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = bar + 1;
        const unsigned g = *gen;   // cannot move on before this block has arrived
        __threadfence();
        *ok = 1;
        if (atomicAdd(bar, 1u) == gridDim.x - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            unsigned spins = 0;
            while (*gen == g) {
                if (++spins > kBarrierSpins) {
                    atomicOr(status, kStatusTimeout);
                    *ok = 0;
                    break;
                }
                __nanosleep(128);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *ok != 0;
}

// Digit counts of tile `tile` into hist[digit * G + tile].
__device__ __forceinline__ void rx_hist_tile(const unsigned long long *keys_in, uint32_t *hist, long long n,
                                             long long G, long long tile, unsigned long long kmin, int shift,
                                             RadixShared &s) {
    s.cnt[threadIdx.x] = 0;
    __syncthreads();
    const long long b0 = tile * kRxTile;
    const long long b1 = min(b0 + kRxTile, n);
    for (long long i = b0 + threadIdx.x; i < b1; i += kRxThreads)
        atomicAdd(&s.cnt[(uint32_t)(((keys_in[i] - kmin) >> shift) & 255ull)], 1u);
    __syncthreads();
    hist[(long long)threadIdx.x * G + tile] = s.cnt[threadIdx.x];
    __syncthreads();
}

// Exclusive scan of hist[digit * G .. + G) in place; the digit's total to dtot[digit].
__device__ __forceinline__ void rx_scan_digit(uint32_t *hist, uint32_t *dtot, long long G, int digit,
                                              RadixShared &s) {
    uint32_t *row = hist + (long long)digit * G;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t carry = 0;
    for (long long c0 = 0; c0 < G; c0 += kRxThreads) {
        const long long i = c0 + threadIdx.x;
        const uint32_t v = i < G ? row[i] : 0u;
        uint32_t incl = v;
        #pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s.wsum[w] = incl;
        __syncthreads();
        uint32_t before = 0, all = 0;
        #pragma unroll
        for (int j = 0; j < kRxWarps; j++) {
            before += j < w ? s.wsum[j] : 0u;
            all += s.wsum[j];
        }
        if (i < G) row[i] = carry + before + incl - v;
        carry += all;
        __syncthreads();
    }
    if (threadIdx.x == 0) dtot[digit] = carry;
}

// Stable scatter of tile `tile` by the digit at `shift`.
__device__ __forceinline__ void rx_scatter_tile(const unsigned long long *keys_in, const uint32_t *vals_in,
                                                unsigned long long *keys_out, uint32_t *vals_out,
                                                const uint32_t *hist, const uint32_t *dtot, long long n,
                                                long long G, long long tile, unsigned long long kmin, int shift,
                                                RadixShared &s) {
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    {
        // digit offsets: exclusive scan of the 256 digit totals, plus this tile's offset
        // inside the digit
        const uint32_t v = dtot[tid];
        uint32_t incl = v;
        #pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s.wsum[w] = incl;
        __syncthreads();
        uint32_t before = 0;
        #pragma unroll
        for (int j = 0; j < kRxWarps; j++) before += j < w ? s.wsum[j] : 0u;
        s.base[tid] = before + incl - v + hist[(long long)tid * G + tile];
    }
    for (int j = 0; j < kRxWarps; j++) s.wcnt[j][tid] = 0;
    __syncthreads();
    const long long b0 = tile * kRxTile;
    const long long b1 = min(b0 + kRxTile, n);
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int r = 0; r < kRxItems; r++) {
        const long long i = b0 + (long long)r * kRxThreads + tid;
        const bool valid = i < b1;
        unsigned long long key = 0;
        uint32_t val = 0;
        uint32_t dg = 256;   // invalid items share a digit no real item has
        if (valid) {
            key = keys_in[i];
            val = vals_in[i];
            dg = (uint32_t)(((key - kmin) >> shift) & 255ull);
        }
        const unsigned peers = __match_any_sync(0xffffffffu, dg);
        const uint32_t rank = __popc(peers & lt_mask);
        if (valid && rank == 0) s.wcnt[w][dg] = __popc(peers);
        __syncthreads();
        {
            uint32_t run = s.base[tid];
            #pragma unroll
            for (int j = 0; j < kRxWarps; j++) {
                const uint32_t c = s.wcnt[j][tid];
                s.wcnt[j][tid] = 0;
                s.woff[j][tid] = run;
                run += c;
            }
            s.base[tid] = run;
        }
        __syncthreads();
        if (valid) {
            const uint32_t pos = s.woff[w][dg] + rank;
            keys_out[pos] = key;
            vals_out[pos] = val;
        }
        __syncthreads();
    }
}

// The whole sort, every block of the cooperative grid taking part (blockDim.x ==
// kRxThreads). The key range (h->key_min, h->key_max) is final on entry. Returns
// the buffer holding the result (also written to h->sorted_sel), or -1 if a
// barrier wait ran out. Ends with a barrier.
__device__ __forceinline__ int rx_sort_coop(const Workspace &ws, long long n, int max_passes, RadixShared &s) {
    WsHeader *h = ws.hdr;
    const long long G = (n + kRxTile - 1) / kRxTile;
    const unsigned long long kmin = h->key_min;
    const int passes = min(radix_passes(h), max_passes);
    for (int p = 0; p < passes; p++) {
        const int in = p & 1, out = in ^ 1;
        for (long long t = blockIdx.x; t < G; t += gridDim.x)
            rx_hist_tile(ws.keys[in], ws.hist, n, G, t, kmin, 8 * p, s);
        if (!grid_barrier(h->bar, &h->status, &s.ok)) return -1;
        for (int dg = blockIdx.x; dg < 256; dg += gridDim.x) rx_scan_digit(ws.hist, ws.dtot, G, dg, s);
        if (!grid_barrier(h->bar, &h->status, &s.ok)) return -1;
        for (long long t = blockIdx.x; t < G; t += gridDim.x)
            rx_scatter_tile(ws.keys[in], ws.vals[in], ws.keys[out], ws.vals[out], ws.hist, ws.dtot, n, G, t, kmin,
                            8 * p, s);
        if (!grid_barrier(h->bar, &h->status, &s.ok)) return -1;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) h->sorted_sel = (unsigned)(passes & 1);
    return passes & 1;
}

// Block-reduced key range into the header (every thread calls it once per key).
__device__ __forceinline__ void rx_key_range(unsigned long long kmin, unsigned long long kmax, WsHeader *h) {
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long a = __shfl_xor_sync(0xffffffffu, kmin, o);
        const unsigned long long b = __shfl_xor_sync(0xffffffffu, kmax, o);
        kmin = a < kmin ? a : kmin;
        kmax = b > kmax ? b : kmax;
    }
    if ((threadIdx.x & 31) == 0 && kmin <= kmax) {
        atomicMin(&h->key_min, kmin);
        atomicMax(&h->key_max, kmax);
    }
}

// Grid size of a cooperative sort kernel: blocks that fit on the device at once
// (at most two per SM), queried once per kernel.
template <typename Kernel>
cudaError_t coop_blocks(Kernel kernel, int *out) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kRxThreads, 0);
    if (e != cudaSuccess) return e;
    *out = sms * (per_sm < 2 ? (per_sm < 1 ? 1 : per_sm) : 2);
    return per_sm >= 1 ? cudaSuccess : cudaErrorInvalidConfiguration;
}

// Queues a cooperative launch of `kernel` (kRxThreads threads per block).
template <typename... KArgs, typename... Args>
cudaError_t launch_coop(void (*kernel)(KArgs...), int blocks, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks, 1, 1);
    cfg.blockDim = dim3(kRxThreads, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, args...);
    note_launch();
    return e;
}

}  // namespace gres
