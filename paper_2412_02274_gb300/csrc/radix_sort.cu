// radix_sort.cu -- stable LSD radix sort of (uint64 key, uint32 value) pairs.
//
// Sorts ws.keys[0]/ws.vals[0] by key. The element count and the key range
// (hdr->key_min, hdr->key_max) live on the device, so the number of 8-bit
// digit passes that do any work, E = ceil(bits(key_max - key_min) / 8), is
// decided on the device: passes p >= E return at once. Pass p reads buffer
// p & 1 and writes buffer (p + 1) & 1, so the result is in buffer E & 1,
// which the first kernel records in hdr->sorted_sel. Digits are taken from
// key - key_min.
//
// Each pass is three kernels: per-block digit histograms, a per-digit scan
// over the blocks (one block per digit, with the digit totals), and a stable
// scatter in which each block takes its digit offsets from the totals and
// ranks its items per digit in input order (warp match_any for ranks within a
// warp, a per-digit prefix over warps for the block, a running per-digit carry
// across the block's rounds).
#include "gres_internal.cuh"

namespace gres {

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 4;
constexpr int kTile = kThreads * kItems;   // 1024 items per block
constexpr int kWarps = kThreads / 32;
constexpr long long kScanFreeBlocks = 64;   // up to this many blocks, scatter blocks scan for themselves

__global__ void __launch_bounds__(kThreads)
k_hist(WsHeader *h, const unsigned long long *keys_in, uint32_t *hist, const long long *d_n, int pass) {
    if (pass == 0 && blockIdx.x == 0 && threadIdx.x == 0) h->sorted_sel = (unsigned)(radix_passes(h) & 1);
    if (pass >= radix_passes(h)) return;
    const long long n = *d_n;
    const long long G = (n + kTile - 1) / kTile;
    if ((long long)blockIdx.x >= G) return;
    __shared__ uint32_t sh[256];
    sh[threadIdx.x] = 0;
    __syncthreads();
    const unsigned long long kmin = h->key_min;
    const int shift = 8 * pass;
    const long long b0 = (long long)blockIdx.x * kTile;
    const long long b1 = min(b0 + kTile, n);
    for (long long i = b0 + threadIdx.x; i < b1; i += kThreads) {
        uint32_t dg = (uint32_t)(((keys_in[i] - kmin) >> shift) & 255ull);
        atomicAdd(&sh[dg], 1u);
    }
    __syncthreads();
    hist[(long long)threadIdx.x * G + blockIdx.x] = sh[threadIdx.x];
}

// Per-digit exclusive scan over the blocks: block d scans hist[d*G .. d*G+G)
// in place and writes the digit's total to dtot[d].
constexpr int kScanThreads = 256;
__global__ void __launch_bounds__(kScanThreads)
k_scan(WsHeader *h, uint32_t *hist, uint32_t *dtot, const long long *d_n, int pass) {
    if (pass >= radix_passes(h)) return;
    const long long n = *d_n;
    const long long G = (n + kTile - 1) / kTile;
    if (G <= kScanFreeBlocks) return;
    uint32_t *row = hist + (long long)blockIdx.x * G;
    __shared__ uint32_t warp_tot[kScanThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t carry = 0;
    for (long long c0 = 0; c0 < G; c0 += kScanThreads) {
        const long long i = c0 + threadIdx.x;
        const uint32_t v = i < G ? row[i] : 0u;
        uint32_t incl = v;
        #pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) warp_tot[w] = incl;
        __syncthreads();
        uint32_t before = 0, all = 0;
        #pragma unroll
        for (int j = 0; j < kScanThreads / 32; j++) {
            before += j < w ? warp_tot[j] : 0u;
            all += warp_tot[j];
        }
        if (i < G) row[i] = carry + before + incl - v;
        carry += all;
        __syncthreads();
    }
    if (threadIdx.x == 0) dtot[blockIdx.x] = carry;
}

__global__ void __launch_bounds__(kThreads)
k_scatter(WsHeader *h, const unsigned long long *keys_in, const uint32_t *vals_in,
          unsigned long long *keys_out, uint32_t *vals_out, const uint32_t *hist,
          const uint32_t *dtot, const long long *d_n, int pass) {
    if (pass >= radix_passes(h)) return;
    const long long n = *d_n;
    const long long G = (n + kTile - 1) / kTile;
    if ((long long)blockIdx.x >= G) return;
    __shared__ uint32_t base[256];
    __shared__ uint32_t wcnt[kWarps][256];
    __shared__ uint32_t woff[kWarps][256];
    __shared__ uint32_t wsum[kWarps];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    {
        // digit offsets: exclusive scan of the 256 digit totals. With few blocks the
        // totals and this block's offset inside the digit come straight from the
        // per-block counts (no separate scan kernel).
        uint32_t v, inner;
        if (G <= kScanFreeBlocks) {
            const uint32_t *row = hist + (long long)tid * G;
            uint32_t tot = 0, pre = 0;
            for (long long b = 0; b < G; b++) {
                const uint32_t c = row[b];
                pre += b < (long long)blockIdx.x ? c : 0u;
                tot += c;
            }
            v = tot;
            inner = pre;
        } else {
            v = dtot[tid];
            inner = hist[(long long)tid * G + blockIdx.x];
        }
        uint32_t incl = v;
        #pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) wsum[w] = incl;
        __syncthreads();
        uint32_t before = 0;
        #pragma unroll
        for (int j = 0; j < kWarps; j++) before += j < w ? wsum[j] : 0u;
        base[tid] = before + incl - v + inner;
    }
    for (int j = 0; j < kWarps; j++) wcnt[j][tid] = 0;
    __syncthreads();
    const unsigned long long kmin = h->key_min;
    const int shift = 8 * pass;
    const long long b0 = (long long)blockIdx.x * kTile;
    const long long b1 = min(b0 + kTile, n);
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int r = 0; r < kItems; r++) {
        const long long i = b0 + (long long)r * kThreads + tid;
        const bool valid = i < b1;
        unsigned long long key = 0;
        uint32_t val = 0;
        uint32_t dg = 256;  // invalid items share a digit no real item has
        if (valid) {
            key = keys_in[i];
            val = vals_in[i];
            dg = (uint32_t)(((key - kmin) >> shift) & 255ull);
        }
        const unsigned peers = __match_any_sync(0xffffffffu, dg);
        const uint32_t rank = __popc(peers & lt_mask);
        if (valid && rank == 0) wcnt[w][dg] = __popc(peers);
        __syncthreads();
        {
            uint32_t run = base[tid];
            #pragma unroll
            for (int j = 0; j < kWarps; j++) {
                uint32_t c = wcnt[j][tid];
                wcnt[j][tid] = 0;
                woff[j][tid] = run;
                run += c;
            }
            base[tid] = run;
        }
        __syncthreads();
        if (valid) {
            const uint32_t pos = woff[w][dg] + rank;
            keys_out[pos] = key;
            vals_out[pos] = val;
        }
        __syncthreads();
    }
}

}  // namespace

int64_t sort_blocks(int64_t n) { return (n + kTile - 1) / kTile; }

// Queues up to `max_passes` digit passes on ws.keys[0]/ws.vals[0] (count in
// *d_n, at most n_max). The sorted data ends in buffer hdr->sorted_sel.
cudaError_t launch_radix_sort(Workspace &ws, int64_t n_max, const long long *d_n,
                              int max_passes, cudaStream_t st) {
    if (n_max <= 0) return cudaSuccess;
    const int64_t G = sort_blocks(n_max);
    if (G > 0) {
        for (int p = 0; p < max_passes; p++) {
            const int in = p & 1, out = (p + 1) & 1;
            k_hist<<<(unsigned)G, kThreads, 0, st>>>(ws.hdr, ws.keys[in], ws.hist, d_n, p); note_launch();
            if (G > kScanFreeBlocks) {
                k_scan<<<256, kScanThreads, 0, st>>>(ws.hdr, ws.hist, ws.dtot, d_n, p); note_launch();
            }
            k_scatter<<<(unsigned)G, kThreads, 0, st>>>(ws.hdr, ws.keys[in], ws.vals[in], ws.keys[out],
                                                        ws.vals[out], ws.hist, ws.dtot, d_n, p); note_launch();
        }
    }
    return cudaGetLastError();
}

}  // namespace gres
