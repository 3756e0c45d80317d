// gres_stage.cu -- grid resistance of every skyline tuple (Def. 2, Algorithm 1).
//
// Inputs: the canonical skyline rows (smaller is better) from skyline.cu. By
// the stability of gres (Sec. 3.2) the candidate dominators are the skyline
// itself.
//
// For a target t and a width delta, the projection of t is the cell with
// lowest corner Lv = floor(t / delta) * delta (Sec. 2). On the original
// values, floor(s/delta) <= floor(t/delta) iff s <= Uv = Lv + delta - 1, and
// floor(s/delta) < floor(t/delta) iff s < Lv. So s's projection dominates
// t's (Def. 1 on projections) iff s <= U in every attribute and s < L in one,
// where (U, L) = (Uv, Lv) for smaller-is-better and, on canonical values
// ~v, (U, L) = (~Lv, ~Uv) for larger-is-better. The kernel therefore never
// projects candidates: one division per (t, step, attribute) gives the
// bounds, and each (candidate, step) test is 2d unsigned compares.
//
// Pruning (speed only; results do not depend on it):
//   * candidates are grouped into 32-row tiles after a Grid / Angular /
//     Sliced partitioning (Sec. 3.1) so that tiles are spatially tight;
//   * s can dominate t at width delta only if delta > max_i (s_i - t_i)^+
//     (a worse attribute must share t's cell), so with the tile minimum
//     tmin a tile is irrelevant for every step with delta <= e_tile =
//     max_i (tmin_i - t_i)^+, and for every step if no tmin_i < t_i;
//   * tiles are visited in ascending order of their first relevant step,
//     and the scan of a target stops at the first step that has a
//     dominator (the minimum over steps, Def. 2); steps are never bisected
//     since membership is not monotone in the width.
//
//   * inside a tile, each row s gets its own first relevant step
//     (delta > max_i (s_i - t_i)^+); rows whose first relevant step is not
//     before the best step found so far are never tested, and the others are
//     tested only from that step on, in ascending order of it.
//
// Mapping: one warp per target tuple (dynamic queue). Lanes scan 32 tiles at
// a time, then the 32 rows of a chosen tile. Lane l holds the bounds of steps
// w0 + 32 j + l (j < SLOTS) in registers, computed on first use of slot j; a
// row to test is shuffled to all lanes; a ballot per slot and __ffs give the
// first dominated step. The candidate rows and tile minima are staged in
// shared memory with cp.async when they fit (they do for skylines up to
// about 6,900 rows at d = 6), otherwise read through L1.
#include "cluster.cuh"
#include "radix.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

namespace gres {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// ---- steps: widths and Granlund-Montgomery constants, passed by value -------
constexpr int kStepChunk = 2000;
struct StepChunk {
    int off;
    int count;
    uint4 e[kStepChunk];   // (m, s1, s2, delta)
};

// Division constants of K widths on the device (Granlund & Montgomery; the
// same constants as udiv_magic): magic[4j .. 4j+3] = (m, s1, s2, delta).
__device__ __forceinline__ uint4 magic_of(uint32_t delta) {
    int l = 0;
    while (l < 32 && (1ull << l) < (unsigned long long)delta) l++;
    const unsigned long long num = (1ull << 32) * ((1ull << l) - (unsigned long long)delta);
    return make_uint4((uint32_t)(num / delta + 1ull), l < 1 ? (uint32_t)l : 1u, l > 1 ? (uint32_t)(l - 1) : 0u, delta);
}

// Raw steps passed by value: a small chunk for the usual step lists (1 KB of
// kernel parameters), a large one (32 KB) for long lists.
template <int CAP>
struct RawSteps {
    int off;
    int count;
    uint32_t e[CAP];
};
constexpr int kRawSmall = 256;
constexpr int kRawLarge = 8000;

// Steps into device memory: division constants (m, s1, s2, divisor), made
// here, and the widths the pruning compares excesses with. Widths mode: the
// width itself. Grid-parameter mode (gbits = B): the divisor is g and the
// width is floor((2^B - 1) / g) + 1, the widest cell of floor(v g / 2^B)
// (clamped to 2^32 - 1; that only happens at g = 1, B = 32, where every value
// falls in one cell and nothing dominates).
template <int CAP>
__global__ void k_upload_steps(RawSteps<CAP> c, uint32_t *steps, uint32_t *magic, WsHeader *h, long long n,
                               unsigned *zero, int gbits, uint32_t *sel) {
    if (h) init_header(h, n);
    clear_sel_hist(sel);
    if (zero && threadIdx.x == 0) *zero = 0u;
    for (int i = threadIdx.x; i < c.count; i += blockDim.x) {
        const uint32_t v = c.e[i];
        unsigned long long w = v;
        if (gbits) w = ((1ull << gbits) - 1ull) / v + 1ull;
        steps[c.off + i] = w > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)w;
        reinterpret_cast<uint4 *>(magic)[c.off + i] = magic_of(v);
    }
}

// Queues the uploads of k steps (the first launch also resets the header h
// and/or clears *zero when given).
cudaError_t upload_steps(const uint32_t *h_steps, int k, uint32_t *steps, uint32_t *magic, WsHeader *h,
                         long long n, unsigned *zero, int gbits, uint32_t *sel, cudaStream_t st) {
    if (k <= kRawSmall) {
        RawSteps<kRawSmall> c;
        c.off = 0;
        c.count = k;
        std::memcpy(c.e, h_steps, sizeof(uint32_t) * (size_t)k);
        k_upload_steps<kRawSmall><<<1, 256, 0, st>>>(c, steps, magic, h, n, zero, gbits, sel); note_launch();
        return cudaGetLastError();
    }
    // 32 KB: not on the stack; one per host thread, so concurrent callers do not wait
    // for each other (launch arguments are copied when the launch is queued)
    thread_local RawSteps<kRawLarge> c;
    for (int off = 0; off < k; off += kRawLarge) {
        c.off = off;
        c.count = std::min(kRawLarge, k - off);
        std::memcpy(c.e, h_steps + off, sizeof(uint32_t) * (size_t)c.count);
        k_upload_steps<kRawLarge><<<1, 256, 0, st>>>(c, steps, magic, off == 0 ? h : nullptr, n,
                                                     off == 0 ? zero : nullptr, gbits,
                                                     off == 0 ? sel : nullptr); note_launch();
    }
    return cudaGetLastError();
}

template <int D>
__device__ __forceinline__ void ld_row(const uint32_t *base, long long r, uint32_t (&x)[D]) {
    constexpr int DP = padded_dims(D);
    const uint4 *p = reinterpret_cast<const uint4 *>(base + r * DP);
    uint4 a = p[0];
    x[0] = a.x;
    if (D > 1) x[1 < D ? 1 : 0] = a.y;
    if (D > 2) x[2 < D ? 2 : 0] = a.z;
    if (D > 3) x[3 < D ? 3 : 0] = a.w;
    if (DP == 8) {
        uint4 b = p[1];
        if (D > 4) x[4 < D ? 4 : 0] = b.x;
        if (D > 5) x[5 < D ? 5 : 0] = b.y;
        if (D > 6) x[6 < D ? 6 : 0] = b.z;
        if (D > 7) x[7 < D ? 7 : 0] = b.w;
    }
}

template <int D>
__device__ __forceinline__ void ldg_row(const uint32_t *base, long long r, uint32_t (&x)[D]) {
    constexpr int DP = padded_dims(D);
    const uint4 *p = reinterpret_cast<const uint4 *>(base + r * DP);
    uint4 a = __ldg(p);
    x[0] = a.x;
    if (D > 1) x[1 < D ? 1 : 0] = a.y;
    if (D > 2) x[2 < D ? 2 : 0] = a.z;
    if (D > 3) x[3 < D ? 3 : 0] = a.w;
    if (DP == 8) {
        uint4 b = __ldg(p + 1);
        if (D > 4) x[4 < D ? 4 : 0] = b.x;
        if (D > 5) x[5 < D ? 5 : 0] = b.y;
        if (D > 6) x[6 < D ? 6 : 0] = b.z;
        if (D > 7) x[7 < D ? 7 : 0] = b.w;
    }
}

struct PartArgs {
    int scheme;      // gres_part
    int m;           // GRID / ANGULAR slices
    int p;           // SLICED partitions
    int dim;         // SLICED attribute
    int bpa;         // bits per attribute of the order inside a partition
    int obits;       // bpa * D: the key is partition << obits | order
    int key32;       // every key fits 32 bits (the sort can stay in shared memory)
    unsigned long long thr[64];   // ANGULAR: tan^2(j pi / 2m) * 2^32, j = 1 .. m-1
};

template <int D>
__device__ __forceinline__ uint32_t pick(const uint32_t (&x)[D], int q) {
    uint32_t v = 0;
    #pragma unroll
    for (int i = 0; i < D; i++) v = i == q ? x[i] : v;
    return v;
}

// Order inside a partition: a Morton code (bpa bits per attribute) so that 32
// consecutive rows of a partition are spatially tight. The partition number
// and the code share one sort key of at most 16 bits where the partition
// count allows (two 8-bit radix passes).
template <int D>
__device__ __forceinline__ unsigned long long interleave(const uint32_t (&q)[D], int bpa) {
    unsigned long long key = 0;
    for (int b = bpa - 1; b >= 0; b--) {
        #pragma unroll
        for (int i = 0; i < D; i++) key = (key << 1) | ((q[i] >> b) & 1u);
    }
    return key;
}

// Over the skyline's range: x = v - lo quantized to bpa bits per attribute.
template <int D>
__device__ __forceinline__ unsigned long long morton_range(const uint32_t (&x)[D], const WsHeader *h, int bpa) {
    uint32_t q[D];
    #pragma unroll
    for (int i = 0; i < D; i++) {
        const unsigned long long span = (unsigned long long)(h->hi[i] - h->lo[i]) + 1ull;
        q[i] = (uint32_t)(((unsigned long long)x[i] << bpa) / span);
    }
    return interleave<D>(q, bpa);
}

// Partition numbers (Sec. 3.1) on coordinates x = v - lo (canonical):
//   GRID:    c_i = floor(x_i m / (hi_i - lo_i + 1)), p = sum_i c_i m^i
//   ANGULAR: phi_i = atan2(sqrt(sum_{j>i} x_j^2), x_i); bin_i = number of
//            thresholds j pi / 2m reached, decided exactly as
//            (Y << 32) >= X * thr_j in 128-bit integers (Eq. 1)
//   SLICED:  first pass keys on x_dim; the slice comes from the rank.
// Sort key = partition << obits | order inside the partition, value = row.
// GRID orders a cell by the Morton code of the position inside the cell,
// x_i m - c_i span_i in [0, span_i); the others by the code over the range.
template <int D>
__device__ __forceinline__ unsigned long long part_key(const uint32_t *sky_rows, long long j, const WsHeader *h,
                                                       const PartArgs &a) {
    uint32_t x[D];
    ld_row<D>(sky_rows, j, x);
    #pragma unroll
    for (int i = 0; i < D; i++) x[i] -= h->lo[i];
    unsigned long long pid = 0;
    if (a.scheme == GRES_PART_GRID) {
        unsigned long long w = 1;
        uint32_t q[D];
        #pragma unroll
        for (int i = 0; i < D; i++) {
            const unsigned long long span = (unsigned long long)(h->hi[i] - h->lo[i]) + 1ull;
            const unsigned long long xm = (unsigned long long)x[i] * (unsigned long long)a.m;
            const unsigned long long c = xm / span;
            pid += c * w;
            w *= (unsigned long long)a.m;
            q[i] = (uint32_t)(((xm - c * span) << a.bpa) / span);
        }
        return (pid << a.obits) | interleave<D>(q, a.bpa);
    }
    if (a.scheme == GRES_PART_ANGULAR) {
        unsigned long long w = 1;
        #pragma unroll
        for (int i = 0; i + 1 < D; i++) {
            const unsigned __int128 X = (unsigned __int128)x[i] * x[i];
            unsigned __int128 Y = 0;
            #pragma unroll
            for (int q = i + 1; q < D; q++) Y += (unsigned __int128)x[q] * x[q];
            int bin = 0;
            if (!(X == 0 && Y == 0)) {
                for (int t = 1; t < a.m; t++)
                    if ((Y << 32) >= X * (unsigned __int128)a.thr[t]) bin = t;
            }
            pid += (unsigned long long)bin * w;
            w *= (unsigned long long)a.m;
        }
        return (pid << a.obits) | morton_range<D>(x, h, a.bpa);
    }
    return pick<D>(x, a.dim);   // SLICED, first pass
}

// SLICED second pass key of the row of rank r (its row j read from the
// sorted values): slice floor(r p / S) << obits | Morton code over the range.
template <int D>
__device__ __forceinline__ unsigned long long sliced_key(const uint32_t *sky_rows, uint32_t j, long long r,
                                                         long long S, const WsHeader *h, const PartArgs &a) {
    uint32_t x[D];
    ld_row<D>(sky_rows, j, x);
    const unsigned long long slice = (unsigned long long)r * (unsigned long long)a.p / (unsigned long long)S;
    #pragma unroll
    for (int q = 0; q < D; q++) x[q] -= h->lo[q];
    return (slice << a.obits) | morton_range<D>(x, h, a.bpa);
}

// Candidate rows in partition order, padded to whole 32-row tiles with
// sentinel rows (all ones: never dominate), each tile's per-attribute minimum
// (tmin) and each 1024-row super-tile's minimum (smin). One block of 1024
// threads per super-tile; warp w builds tile w of it.
// Super-tile sup of the candidate layout, by one 1024-thread block; warp w
// builds tile w of it. wm: 32 x DP words of shared memory.
template <int D>
__device__ __forceinline__ void permute_super(const uint32_t *sky_rows, const uint32_t *vals, int identity,
                                              long long S, long long sup, uint32_t *cand, uint32_t *tmin,
                                              uint32_t *smin, uint32_t *perm, uint32_t (*wm)[padded_dims(D)]) {
    constexpr int DP = padded_dims(D);
    const long long T = (S + kTileRows - 1) / kTileRows;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long tile = sup * 32 + w;
    const long long i = tile * kTileRows + lane;
    uint32_t x[DP];
    if (i < S) {
        const uint32_t j = identity ? (uint32_t)i : vals[i];
        perm[i] = j;
        const uint4 *p = reinterpret_cast<const uint4 *>(sky_rows + (long long)j * DP);
        uint4 a = p[0];
        x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
        if (DP == 8) { uint4 b = p[1]; x[4 % DP] = b.x; x[5 % DP] = b.y; x[6 % DP] = b.z; x[7 % DP] = b.w; }
    } else {
        #pragma unroll
        for (int q = 0; q < DP; q++) x[q] = kSentinel;
    }
    if (tile < T) {
        uint4 *dst = reinterpret_cast<uint4 *>(cand + i * DP);
        dst[0] = make_uint4(x[0], x[1], x[2], x[3]);
        if (DP == 8) dst[1] = make_uint4(x[4 % DP], x[5 % DP], x[6 % DP], x[7 % DP]);
    }
    #pragma unroll
    for (int q = 0; q < DP; q++) {
        uint32_t v = x[q];
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(kFull, v, o));
        if (lane == 0) {
            wm[w][q] = v;
            if (tile < T) tmin[tile * DP + q] = v;
        }
    }
    __syncthreads();
    if (w == 0) {
        #pragma unroll
        for (int q = 0; q < DP; q++) {
            uint32_t v = wm[lane][q];
            #pragma unroll
            for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(kFull, v, o));
            if (lane == 0) smin[sup * DP + q] = v;
        }
    }
    __syncthreads();
}

// The partitioning of a skyline of more than kClusterSortMax rows, as one
// cooperative launch: the partition keys (partition number << obits | order
// inside the partition), the stable radix sort (for SLICED: by the chosen
// attribute, then by (slice, order) with slice floor(rank p / S), Sec. 3.1),
// then the candidate layout -- rows in that order in 32-row tiles padded with
// sentinel rows, tile and super-tile minima, perm (partition position ->
// skyline position). Returns at once (every block) for at most
// kClusterSortMax skyline rows: k_part_cluster partitions those. The key range
// was cleared by k_compact_sky.
template <int D>
__global__ void __launch_bounds__(kRxThreads)
k_part_coop(const uint32_t *sky_rows, Workspace ws, PartArgs a, int passes1, int passes2) {
    constexpr int DP = padded_dims(D);
    __shared__ RadixShared s;
    WsHeader *h = ws.hdr;
    const long long S = h->n_sky;
    if (S <= kClusterSortMax) return;
    const long long stride = (long long)gridDim.x * kRxThreads;
    const long long gt = (long long)blockIdx.x * kRxThreads + threadIdx.x;
    const bool none = a.scheme == GRES_PART_NONE;
    int sel = 0;
    if (!none) {
        unsigned long long kmn = ~0ull, kmx = 0ull;
        for (long long j = gt; j < S; j += stride) {
            const unsigned long long key = part_key<D>(sky_rows, j, h, a);
            ws.keys[0][j] = key;
            ws.vals[0][j] = (uint32_t)j;
            kmn = key < kmn ? key : kmn;
            kmx = key > kmx ? key : kmx;
        }
        rx_key_range(kmn, kmx, h);
        if (!grid_barrier(h->bar, &h->status, &s.ok)) return;
        sel = rx_sort_coop(ws, S, passes1, s);
        if (sel < 0) return;
        if (a.scheme == GRES_PART_SLICED) {
            // rank r -> slice floor(r p / S); the new keys order rows by (slice, order)
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                h->key_min = ~0ull;
                h->key_max = 0ull;
            }
            if (!grid_barrier(h->bar, &h->status, &s.ok)) return;
            const uint32_t *vs = ws.vals[sel];
            kmn = ~0ull;
            kmx = 0ull;
            for (long long r = gt; r < S; r += stride) {
                const uint32_t j = vs[r];
                const unsigned long long key = sliced_key<D>(sky_rows, j, r, S, h, a);
                ws.keys[0][r] = key;   // in place when the sorted buffer is buffer 0
                ws.vals[0][r] = j;
                kmn = key < kmn ? key : kmn;
                kmx = key > kmx ? key : kmx;
            }
            rx_key_range(kmn, kmx, h);
            if (!grid_barrier(h->bar, &h->status, &s.ok)) return;
            sel = rx_sort_coop(ws, S, passes2, s);
            if (sel < 0) return;
        }
    }
    // candidate layout: one warp per tile
    const uint32_t *vals = ws.vals[sel];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long T = (S + kTileRows - 1) / kTileRows;
    for (long long tile = (long long)blockIdx.x * kRxWarps + w; tile < T; tile += (long long)gridDim.x * kRxWarps) {
        const long long i = tile * kTileRows + lane;
        uint32_t x[DP];
        if (i < S) {
            const uint32_t j = none ? (uint32_t)i : vals[i];
            ws.perm[i] = j;
            const uint4 *p = reinterpret_cast<const uint4 *>(sky_rows + (long long)j * DP);
            const uint4 a0 = p[0];
            x[0] = a0.x; x[1] = a0.y; x[2] = a0.z; x[3] = a0.w;
            if (DP == 8) { const uint4 b = p[1]; x[4 % DP] = b.x; x[5 % DP] = b.y; x[6 % DP] = b.z; x[7 % DP] = b.w; }
        } else {
            #pragma unroll
            for (int q = 0; q < DP; q++) x[q] = kSentinel;
        }
        uint4 *dst = reinterpret_cast<uint4 *>(ws.cand + i * DP);
        dst[0] = make_uint4(x[0], x[1], x[2], x[3]);
        if (DP == 8) dst[1] = make_uint4(x[4 % DP], x[5 % DP], x[6 % DP], x[7 % DP]);
        #pragma unroll
        for (int q = 0; q < DP; q++) {
            uint32_t m = x[q];
            #pragma unroll
            for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_xor_sync(kFull, m, o));
            if (lane == 0) ws.tmin[tile * DP + q] = m;
        }
    }
    if (!grid_barrier(h->bar, &h->status, &s.ok)) return;
    const long long T2 = (T + 31) / 32;
    for (long long k = gt; k < T2 * DP; k += stride) {
        const long long sup = k / DP;
        const int q = (int)(k % DP);
        uint32_t m = kSentinel;
        for (long long t = sup * 32; t < min(T, sup * 32 + 32); t++) m = min(m, ws.tmin[t * DP + q]);
        ws.smin[sup * DP + q] = m;
    }
}

// The whole partitioning of a skyline of at most kClusterSortMax rows as one
// cluster launch: keys, the stable sort (two for SLICED: by the chosen
// attribute, then by slice and Morton code), and the candidate layout -- what
// the cooperative partition kernel (k_part_coop) computes for larger skylines.
// Returns at once (every CTA) for a larger skyline.
template <int D>
__global__ void __launch_bounds__(kClThreads)
k_part_cluster(const uint32_t *sky_rows, WsHeader *h, PartArgs a, unsigned long long *k0, uint32_t *v0,
               unsigned long long *k1, uint32_t *v1, uint32_t *cand, uint32_t *tmin, uint32_t *smin,
               uint32_t *perm) {
    constexpr int DP = padded_dims(D);
    extern __shared__ uint32_t sm[];
    __shared__ unsigned long long kr[2];
    __shared__ uint32_t wm[32][DP];
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks(), r = (int)cl.block_rank();
    const long long tt = (long long)C * kClThreads, gt = (long long)r * kClThreads + threadIdx.x;
    const long long S = h->n_sky;
    if (S > kClusterSortMax) return;   // k_part_coop partitions it (every CTA returns here)
    const bool none = a.scheme == GRES_PART_NONE;
    int sel = 0;
    if (!none && a.key32) {
        // keys of at most 32 bits: the (key, skyline position) pairs stay in the cluster's
        // shared memory, CTA r holding positions [b0, b0 + cnt)
        uint32_t *kb0 = sm + kClSortWords, *vb0 = kb0 + kClSmemCap, *kb1 = vb0 + kClSmemCap, *vb1 = kb1 + kClSmemCap;
        const long long c = cluster_chunk(S);
        const long long b0 = min(S, (long long)r * c);
        const int cnt = (int)(min(S, b0 + c) - b0);
        if (threadIdx.x == 0) { kr[0] = ~0ull; kr[1] = 0ull; }
        __syncthreads();
        unsigned long long kmn = ~0ull, kmx = 0ull;
        for (int i = threadIdx.x; i < cnt; i += kClThreads) {
            const unsigned long long key = part_key<D>(sky_rows, b0 + i, h, a);
            kb0[i] = (uint32_t)key;
            vb0[i] = (uint32_t)(b0 + i);
            kmn = key < kmn ? key : kmn;
            kmx = key > kmx ? key : kmx;
        }
        cta_key_add(kmn, kmx, kr);
        unsigned long long kmin, kmax;
        cluster_key_range(cl, kr, &kmin, &kmax);
        int cur = cluster_radix_sort_smem(cl, sm, kb0, vb0, kb1, vb1, S, (uint32_t)kmin, key_passes(kmin, kmax), 0);
        if (a.scheme == GRES_PART_SLICED) {
            // rank q -> slice floor(q p / S); re-key in place, sort again
            __shared__ unsigned long long kr2[2];
            if (threadIdx.x == 0) { kr2[0] = ~0ull; kr2[1] = 0ull; }
            __syncthreads();
            uint32_t *kc = cur ? kb1 : kb0;
            const uint32_t *vc = cur ? vb1 : vb0;
            kmn = ~0ull;
            kmx = 0ull;
            for (int i = threadIdx.x; i < cnt; i += kClThreads) {
                const unsigned long long key = sliced_key<D>(sky_rows, vc[i], b0 + i, S, h, a);
                kc[i] = (uint32_t)key;
                kmn = key < kmn ? key : kmn;
                kmx = key > kmx ? key : kmx;
            }
            cta_key_add(kmn, kmx, kr2);
            cluster_key_range(cl, kr2, &kmin, &kmax);
            cur = cluster_radix_sort_smem(cl, sm, kb0, vb0, kb1, vb1, S, (uint32_t)kmin, key_passes(kmin, kmax), cur);
        }
        // the order (and keys) to global memory for the candidate layout
        const uint32_t *kf = cur ? kb1 : kb0, *vf = cur ? vb1 : vb0;
        for (int i = threadIdx.x; i < cnt; i += kClThreads) {
            k0[b0 + i] = kf[i];
            v0[b0 + i] = vf[i];
        }
        cl.sync();
    } else if (!none) {
        // first key: partition number << obits | order (SLICED: the chosen attribute)
        if (threadIdx.x == 0) { kr[0] = ~0ull; kr[1] = 0ull; }
        __syncthreads();
        unsigned long long kmn = ~0ull, kmx = 0ull;
        for (long long j = gt; j < S; j += tt) {
            const unsigned long long key = part_key<D>(sky_rows, j, h, a);
            k0[j] = key;
            v0[j] = (uint32_t)j;
            kmn = key < kmn ? key : kmn;
            kmx = key > kmx ? key : kmx;
        }
        cta_key_add(kmn, kmx, kr);
        unsigned long long kmin, kmax;
        cluster_key_range(cl, kr, &kmin, &kmax);
        int passes = key_passes(kmin, kmax);
        cluster_radix_sort(cl, sm, k0, v0, k1, v1, S, kmin, passes);
        sel = passes & 1;
        if (a.scheme == GRES_PART_SLICED) {
            // rank r -> slice floor(r p / S); re-key in place into buffer 0, sort again
            const uint32_t *vs = sel ? v1 : v0;
            __shared__ unsigned long long kr2[2];
            if (threadIdx.x == 0) { kr2[0] = ~0ull; kr2[1] = 0ull; }
            __syncthreads();
            kmn = ~0ull;
            kmx = 0ull;
            for (long long q = gt; q < S; q += tt) {
                const uint32_t j = vs[q];
                const unsigned long long key = sliced_key<D>(sky_rows, j, q, S, h, a);
                k0[q] = key;
                v0[q] = j;
                kmn = key < kmn ? key : kmn;
                kmx = key > kmx ? key : kmx;
            }
            cta_key_add(kmn, kmx, kr2);
            cluster_key_range(cl, kr2, &kmin, &kmax);
            passes = key_passes(kmin, kmax);
            cluster_radix_sort(cl, sm, k0, v0, k1, v1, S, kmin, passes);
            sel = passes & 1;
        }
    }
    const long long T = (S + kTileRows - 1) / kTileRows;
    const long long T2 = (T + 31) / 32;
    for (long long sup = r; sup < T2; sup += C)
        permute_super<D>(sky_rows, sel ? v1 : v0, none ? 1 : 0, S, sup, cand, tmin, smin, perm, wm);
    if (r == 0 && threadIdx.x == 0) h->sorted_sel = (unsigned)sel;
    cl.sync();   // no CTA leaves while another may still read its shared memory
}

// gres_partition: the caller's rows, canonical and padded, as the candidate
// set; their per-attribute range into lo/hi and S = n.
template <int D>
__global__ void k_load_candidates(const uint32_t *rows, int dir, long long n, uint32_t *sky_rows,
                                  WsHeader *h) {
    constexpr int DP = padded_dims(D);
    if (blockIdx.x == 0 && threadIdx.x == 0) h->n_sky = n;
    uint32_t lo[D], hi[D];
    #pragma unroll
    for (int q = 0; q < D; q++) { lo[q] = 0xFFFFFFFFu; hi[q] = 0u; }
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride) {
        uint32_t y[DP];
        #pragma unroll
        for (int q = 0; q < DP; q++) y[q] = q < D ? canon(rows[j * D + (q < D ? q : 0)], dir) : 0u;
        #pragma unroll
        for (int q = 0; q < D; q++) { lo[q] = min(lo[q], y[q]); hi[q] = max(hi[q], y[q]); }
        uint4 *dst = reinterpret_cast<uint4 *>(sky_rows + j * DP);
        dst[0] = make_uint4(y[0], y[1], y[2], y[3]);
        if (DP == 8) dst[1] = make_uint4(y[4 % DP], y[5 % DP], y[6 % DP], y[7 % DP]);
    }
    #pragma unroll
    for (int q = 0; q < D; q++) {
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo[q] = min(lo[q], __shfl_xor_sync(kFull, lo[q], o));
            hi[q] = max(hi[q], __shfl_xor_sync(kFull, hi[q], o));
        }
        if ((threadIdx.x & 31) == 0 && lo[q] <= hi[q]) {
            atomicMin(&h->lo[q], lo[q]);
            atomicMax(&h->hi[q], hi[q]);
        }
    }
}

// gres_partition outputs: partition number by row (the sort key's high bits),
// the tile order, and the tile minima with d words per tile.
template <int D>
__global__ void k_partition_out(const WsHeader *h, const unsigned long long *keys0,
                                const unsigned long long *keys1, const uint32_t *perm,
                                const uint32_t *tmin, int scheme, int obits, long long n, int64_t *part,
                                uint32_t *order, uint32_t *tile_min) {
    constexpr int DP = padded_dims(D);
    const unsigned long long *keys = h->sorted_sel ? keys1 : keys0;
    const long long T = (n + kTileRows - 1) / kTileRows;
    const long long total = n > T * D ? n : T * D;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < total; r += stride) {
        if (r < n) {
            const uint32_t j = perm[r];
            order[r] = j;
            part[j] = scheme == GRES_PART_NONE ? 0 : (int64_t)(keys[r] >> obits);
        }
        if (r < T * D) tile_min[r] = tmin[(r / D) * DP + r % D];
    }
}

// Partition number per partition position (GRES_FLAG_COUNT_PARTS): the high
// bits of the final sort key (the cluster path's keys when S <= kClusterSortMax,
// with obits_small order bits, the cooperative path's above, with obits_large);
// 0 without partitioning; ~0 for the padding rows of the last tile.
__global__ void k_part_ids(const WsHeader *h, const unsigned long long *keys0, const unsigned long long *keys1,
                           int none, int obits_small, int obits_large, uint32_t *pid) {
    const long long S = h->n_sky;
    const long long lim = (S + kTileRows - 1) / kTileRows * kTileRows;
    const unsigned long long *keys = h->sorted_sel ? keys1 : keys0;
    const int obits = S <= kClusterSortMax ? obits_small : obits_large;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < lim;
         i += (long long)gridDim.x * blockDim.x)
        pid[i] = i >= S ? 0xFFFFFFFFu : none ? 0u : (uint32_t)(keys[i] >> obits);
}

// ---- the pairwise grid-dominance kernel ------------------------------------
struct DomArgs {
    DomQuery q;
    PartCount pc;
    unsigned *counter;        // work counter (zeroed before the launch)
    unsigned long long *tests;
    int smem_words;           // dynamic shared memory, in words
};

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem_src) : "memory");
}

// Threads per block of the grid-dominance kernels (one block per SM). A target's
// search is one long chain of dependent warp operations, so the kernels run as
// many warps per SM as the registers allow: the cell bounds of a target are
// made on the fly for each slot test instead of being kept in registers.
template <int D, int SLOTS, bool GM = false>
__host__ __device__ constexpr int dom_threads() {
    return GM ? (D <= 4 ? 768 : 640) : 1024;
}

constexpr uint32_t kNoTile = 0xFFFFFFFFu;

// Raw cell [lv, uv] of raw value v at one step (mg = the step's division
// constants and divisor). Widths: [floor(v / w) w, + w - 1] cut at 2^32 - 1.
// Grid parameter g over v / 2^B: with v g = c 2^B + r, [v - floor(r / g),
// v + floor((2^B - 1 - r) / g)] cut at 2^32 - 1.
__device__ __forceinline__ void raw_cell(uint32_t v, uint4 mg, int gbits, uint32_t &lv, uint32_t &uv) {
    if (gbits) {
        const unsigned long long mask = (1ull << gbits) - 1ull;
        const uint32_t r = (uint32_t)(((unsigned long long)v * mg.w) & mask);
        lv = v - udiv(r, mg.x, mg.y, mg.z);
        const unsigned long long u = (unsigned long long)v + udiv((uint32_t)(mask - r), mg.x, mg.y, mg.z);
        uv = u > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)u;
    } else {
        const uint32_t delta = mg.w;
        lv = udiv(v, mg.x, mg.y, mg.z) * delta;
        uv = lv > 0xFFFFFFFFu - (delta - 1u) ? 0xFFFFFFFFu : lv + (delta - 1u);
    }
}

// Representative Filtering in the gres stage (GRES_FLAG_GRES_REPS): for the
// target at partition position i, the first step at which one of the 32
// representatives' projections dominates the target's (K if none), as a
// bound for the search. One warp per target, lanes over 32 steps at a time.
template <int D>
__global__ void __launch_bounds__(256)
k_rep_bound(const uint32_t *cand, const uint32_t *greps, const long long *n_sky, const uint32_t *magic,
            int K, int dir, int gbits, int32_t *ub, unsigned long long *tests) {
    constexpr int DP = padded_dims(D);
    __shared__ uint32_t rs[32 * DP];
    for (int j = threadIdx.x; j < 32 * DP; j += blockDim.x) rs[j] = greps[j];
    __syncthreads();
    const long long S = *n_sky;
    const int lane = threadIdx.x & 31;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    unsigned long long n_tests = 0;
    for (long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < S; i += nw) {
        uint32_t t[D];
        ld_row<D>(cand, i, t);
        int result = K;
        for (int w0 = 0; w0 < K && result == K; w0 += 32) {
            const int k = w0 + lane;
            const bool live = k < K;
            const uint4 mg = live ? __ldg(reinterpret_cast<const uint4 *>(magic) + k) : make_uint4(1u, 0u, 0u, 1u);
            uint32_t lo[D], hi[D];
            #pragma unroll
            for (int q = 0; q < D; q++) {
                uint32_t lv, uv;
                raw_cell(dir ? ~t[q] : t[q], mg, gbits, lv, uv);
                hi[q] = live ? (dir ? ~lv : uv) : 0u;
                lo[q] = live ? (dir ? ~uv : lv) : 0u;
            }
            bool hit = false;
            for (int r = 0; r < 32; r++) {
                bool le = true, lt = false;
                #pragma unroll
                for (int q = 0; q < D; q++) {
                    const uint32_t sv = rs[r * DP + q];
                    le &= sv <= hi[q];
                    lt |= sv < lo[q];
                }
                hit |= le & lt;
            }
            n_tests += 32 * 32;
            const unsigned msk = __ballot_sync(kFull, hit);
            if (msk) result = w0 + __ffs(msk) - 1;
        }
        if (lane == 0) ub[i] = result;
    }
    if (tests && lane == 0 && n_tests) atomicAdd(tests, n_tests);
}

// Canonical row r of a candidate set, DP words apart: staged in shared memory
// (RES) or read through L1.
template <int D, bool RES>
__device__ __forceinline__ void ld_cand(const uint32_t *base, long long r, uint32_t (&x)[D]) {
    if (RES) ld_row<D>(base, r, x); else ldg_row<D>(base, r, x);
}

// Per attribute, the largest canonical value s with s - t < wl (wl >= 1):
// min(t + wl - 1, 2^32 - 1). A candidate row's excess max_i (s_i - t_i)^+ is
// below wl exactly when every s_i is at most this bound.
template <int D>
__device__ __forceinline__ void excess_bounds(const uint32_t (&t)[D], uint32_t wl, uint32_t (&thr)[D]) {
    #pragma unroll
    for (int q = 0; q < D; q++) thr[q] = min(t[q], 0xFFFFFFFFu - (wl - 1u)) + (wl - 1u);
}

// Grid resistance of the target at partition position i of query q (one
// warp; every lane returns it): the first step at which some candidate's
// projection dominates the target's projection, else K. CNT: count the
// lane-tests and pruning checks (GRES_FLAG_COUNT_TESTS / _PARTS); the search
// is the same either way. PAIR: load the rows of the next tile in key order
// together with the current tile's (the same tiles are looked at, in the same
// order; it needs D more registers).
template <int D, int SLOTS, bool RES, bool GM, bool CNT, bool PAIR>
__device__ __forceinline__ int dom_target(const DomQuery &qy, const uint32_t *cand, const uint32_t *tmin,
                                           const uint32_t *smin, long long T, unsigned i, uint32_t *wsteps,
                                           unsigned long long &n_tests, unsigned long long &n_checks,
                                           const PartCount &pc) {
    constexpr int WS = 32 * SLOTS;
    const int lane = threadIdx.x & 31;
    const int K = qy.K;
    uint32_t t[D];
    ld_cand<D, RES>(cand, i, t);
    int result = K;
    for (int w0 = 0; w0 < K; w0 += WS) {
        const int wcount = min(WS, K - w0);
        // this window's widths in shared memory
        #pragma unroll
        for (int j = 0; j < SLOTS; j++) {
            const int k = w0 + 32 * j + lane;
            wsteps[32 * j + lane] = k < K ? __ldg(qy.steps + k) : 0xFFFFFFFFu;
        }
        __syncwarp();
        int best = wcount;
        // The target's cell at the widths of one slot (canonical bounds per attribute).
        // With the grid parameter g they cost two divisions per attribute, so the g
        // form keeps the last slot's bounds (its step lists are short: usually one
        // slot); with widths they are made for every test, which keeps the kernel at 64
        // registers and 32 warps per SM.
        uint32_t chi[D], clo[D];
        int cj = -1;
        if (qy.ub) {
            // a known exit step (GRES_FLAG_GRES_REPS): only earlier steps are searched
            const int b = qy.ub[i];
            if (b >= w0 && b - w0 < wcount) best = b - w0;
        }
        // keys hold excesses >> qshift; only excesses below the window's widest width matter
        const uint32_t wmax = wsteps[wcount - 1];
        const int qshift = wmax >> 24 ? 32 - __clz(wmax) - 24 : 0;
        // wl: the width of step best - 1 (excesses at or above it cannot matter);
        // wlq: the largest key whose excess can be below wl ((wl - 1) >> qshift; with
        // qshift = 0 every key up to wlq is below wl, above 0 the keys equal to wlq
        // are checked exactly); thr: the excess bounds of wl
        uint32_t wl = best > 0 ? wsteps[best - 1] : 1u;
        uint32_t wlq = min((wl - 1u) >> qshift, 0x7FFFFFFu);
        uint32_t thr[D];
        excess_bounds<D>(t, wl, thr);
        // lane j < SLOTS - 1 holds the widest width of slot j (for the first slot that can matter)
        const uint32_t slot_top = (lane < SLOTS - 1 && 32 * lane + 31 < wcount) ? wsteps[32 * lane + 31] : 0xFFFFFFFFu;
        // Best-first over two levels -- 1024-row super-tiles, then 32-row tiles --
        // each visited in ascending order of its lower bound on the excess
        // max_i (s_i - t_i)^+ (keys hold it >> qshift, 27 bits), then the rows of a
        // tile whose excess is below delta[best - 1]. Anything whose bound reaches
        // delta[best - 1] is skipped.
        const long long T2 = (T + 31) / 32;
        for (long long s0 = 0; s0 < T2 && best > 0; s0 += 32) {
            uint32_t skey = kNoTile, sex = 0xFFFFFFFFu;
            if (s0 + lane < T2) {
                uint32_t mn[D];
                if (RES) ld_row<D>(smin, s0 + lane, mn); else ldg_row<D>(smin, s0 + lane, mn);
                uint32_t emax = 0;
                bool can = false;
                #pragma unroll
                for (int q = 0; q < D; q++) {
                    emax = max(emax, mn[q] > t[q] ? mn[q] - t[q] : 0u);
                    can |= mn[q] < t[q];
                }
                if (can && emax < wl) {
                    sex = emax;
                    skey = (min(emax >> qshift, 0x7FFFFFFu) << 5) | (uint32_t)lane;
                }
            }
            if (CNT) n_checks += 32;
            for (;;) {
                const uint32_t mk = __reduce_min_sync(kFull, skey);
                if (mk == kNoTile || (mk >> 5) > wlq) break;   // every super-tile left is too far
                const int sl = (int)(mk & 31u);
                if (lane == sl) skey = kNoTile;
                if (qshift && (mk >> 5) == wlq && __shfl_sync(kFull, sex, sl) >= wl) continue;
                const long long sup = s0 + sl;
                // tile level inside the super-tile: lane = tile
                uint32_t tkey = kNoTile, tex = 0xFFFFFFFFu;
                const long long tile = sup * 32 + lane;
                if (tile < T) {
                    uint32_t mn[D];
                    if (RES) ld_row<D>(tmin, tile, mn); else ldg_row<D>(tmin, tile, mn);
                    uint32_t emax = 0;
                    bool can = false;
                    #pragma unroll
                    for (int q = 0; q < D; q++) {
                        emax = max(emax, mn[q] > t[q] ? mn[q] - t[q] : 0u);
                        can |= mn[q] < t[q];
                    }
                    if (can && emax < wl) {
                        tex = emax;
                        tkey = (min(emax >> qshift, 0x7FFFFFFu) << 5) | (uint32_t)lane;
                    }
                }
                if (CNT) n_checks += 32;
                // The rows of one tile (s: this lane's row, r0: the tile's first row) against
                // the target; tests the rows that can matter and updates best.
                auto row_look = [&](const uint32_t (&s)[D], long long r0) {
                    // row level: lane r looks at row r of the tile; a row can dominate t
                    // only if some attribute is below t's and its excess is below wl (every
                    // attribute within the excess bounds): only a width wider than the
                    // excess, and before best, can make it dominate
                    bool le = true, lt = false;
                    #pragma unroll
                    for (int q = 0; q < D; q++) {
                        le &= s[q] <= thr[q];
                        lt |= s[q] < t[q];
                    }
                    if (CNT) {
                        n_checks += 32;
                        if (pc.pcnt) {
                            // per-partition split: rows of the target's partition, and the others
                            const uint32_t pt = __ldg(pc.pid + i);
                            const unsigned loc = __popc(__ballot_sync(kFull, __ldg(pc.pid + r0 + lane) == pt));
                            if (lane == 0 && pt < pc.nparts) {
                                atomicAdd(pc.pcnt + 2 + 4ull * pt + 1, (unsigned long long)loc);
                                atomicAdd(pc.pcnt + 2 + 4ull * pt + 3, (unsigned long long)(32 - loc));
                            }
                        }
                    }
                    // rows taken in tile order; best only shrinks, so a row is skipped once
                    // its excess reaches the current delta[best - 1]
                    unsigned elig = __ballot_sync(kFull, le & lt);
                    while (elig) {
                        const int c = __ffs(elig) - 1;
                        elig &= elig - 1;
                        uint32_t cv[D];   // the row, read by every lane (broadcast), and its excess
                        ld_cand<D, RES>(cand, r0 + c, cv);
                        uint32_t ec = 0;
                        #pragma unroll
                        for (int q = 0; q < D; q++) ec = max(ec, cv[q] > t[q] ? cv[q] - t[q] : 0u);
                        if (ec >= wl) continue;
                        // first slot holding a width wider than ec
                        const int jlo = __popc(__ballot_sync(kFull, slot_top <= ec));
                        const int jhi = (best - 1) >> 5;
                        for (int j = jlo; j <= jhi; j++) {
                            // the target's cell at this lane's width, canonical [lo, hi];
                            // lanes past K never match
                            const int k = w0 + 32 * j + lane;
                            const bool live = k < K;
                            if (GM ? cj != j : true) {
                                const uint4 mg = live ? __ldg(reinterpret_cast<const uint4 *>(qy.magic) + k)
                                                      : make_uint4(1u, 0u, 0u, 1u);
                                #pragma unroll
                                for (int q = 0; q < D; q++) {
                                    uint32_t lv, uv;
                                    raw_cell(qy.dir ? ~t[q] : t[q], mg, GM ? qy.gbits : 0, lv, uv);
                                    chi[q] = live ? (qy.dir ? ~lv : uv) : 0u;
                                    clo[q] = live ? (qy.dir ? ~uv : lv) : 0u;
                                }
                                cj = j;
                            }
                            bool dle = true, dlt = false;
                            #pragma unroll
                            for (int q = 0; q < D; q++) {
                                dle &= cv[q] <= chi[q];
                                dlt |= cv[q] < clo[q];
                            }
                            if (CNT) {
                                n_tests += 32;
                                if (pc.pcnt && lane == 0 && __ldg(pc.pid + i) < pc.nparts) {
                                    const uint32_t pt = __ldg(pc.pid + i);
                                    atomicAdd(pc.pcnt + 2 + 4ull * pt + (__ldg(pc.pid + r0 + c) == pt ? 0 : 2), 32ull);
                                }
                            }
                            const unsigned msk = __ballot_sync(kFull, dle & dlt);
                            if (msk) {
                                best = min(best, 32 * j + __ffs(msk) - 1);
                                if (best > 0) {
                                    wl = wsteps[best - 1];
                                    wlq = min((wl - 1u) >> qshift, 0x7FFFFFFu);
                                    excess_bounds<D>(t, wl, thr);
                                }
                                break;
                            }
                        }
                        if (best == 0) break;
                    }
                };
                for (;;) {
                    const uint32_t tk = __reduce_min_sync(kFull, tkey);
                    if (tk == kNoTile || (tk >> 5) > wlq) break;   // every tile left is too far
                    const int tl = (int)(tk & 31u);
                    if (lane == tl) tkey = kNoTile;
                    if (qshift && (tk >> 5) == wlq && __shfl_sync(kFull, tex, tl) >= wl) continue;
                    const long long r0 = (sup * 32 + tl) * kTileRows;
                    uint32_t s[D];
                    if (!PAIR) {
                        ld_cand<D, RES>(cand, r0 + lane, s);
                        row_look(s, r0);
                        if (best == 0) break;
                        continue;
                    }
                    // PAIR: the tile the search takes next (the keys only lose entries) is
                    // popped now, so that both tiles' rows load together; it is looked at
                    // after this one only if it still can matter then
                    const uint32_t tk2 = __reduce_min_sync(kFull, tkey);
                    const bool have2 = tk2 != kNoTile && (tk2 >> 5) <= wlq;
                    const int tl2 = (int)(tk2 & 31u);
                    if (have2 && lane == tl2) tkey = kNoTile;
                    const long long r02 = (sup * 32 + tl2) * kTileRows;
                    uint32_t s2[D];
                    ld_cand<D, RES>(cand, r0 + lane, s);
                    if (have2) ld_cand<D, RES>(cand, r02 + lane, s2);
                    row_look(s, r0);
                    if (best == 0 || !have2) break;
                    if ((tk2 >> 5) > wlq) break;   // best moved: every tile left is too far
                    if (qshift && (tk2 >> 5) == wlq && __shfl_sync(kFull, tex, tl2) >= wl) continue;
                    row_look(s2, r02);
                    if (best == 0) break;
                }
                if (best == 0) break;
            }
        }
        __syncwarp();
        if (best < wcount) { result = w0 + best; break; }
    }
    return result;
}

// Tile pairs in the single-query kernel up to d = 6: above that (and in the
// batched kernel, which holds its query's descriptor too) the extra row does
// not fit in the 64 registers and spills.
template <int D>
constexpr bool kPairTiles = D <= 6;

template <int D, int SLOTS, bool GM, bool CNT>
__global__ void __launch_bounds__(dom_threads<D, SLOTS, GM>(), 1)
k_dominance(DomArgs a) {
    constexpr int DP = padded_dims(D);
    constexpr int WS = 32 * SLOTS;
    extern __shared__ __align__(16) uint32_t sm[];
    const long long S = *a.q.n_sky;
    if (S == 0) return;
    const long long T = (S + kTileRows - 1) / kTileRows;
    const int nwarps = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t *wsteps = sm + warp * WS;
    uint32_t *stage = sm + nwarps * WS;
    const long long T2 = (T + 31) / 32;
    const long long cand_words = T * kTileRows * DP;
    const long long need = cand_words + T * DP + T2 * DP;
    const bool resident = need <= (long long)a.smem_words - (long long)nwarps * WS;
    if (resident) {
        const long long n16a = cand_words / 4, n16b = (T * DP) / 4, n16c = (T2 * DP) / 4;
        for (long long v = threadIdx.x; v < n16a; v += blockDim.x) cp_async16(stage + 4 * v, a.q.cand + 4 * v);
        for (long long v = threadIdx.x; v < n16b; v += blockDim.x)
            cp_async16(stage + cand_words + 4 * v, a.q.tmin + 4 * v);
        for (long long v = threadIdx.x; v < n16c; v += blockDim.x)
            cp_async16(stage + cand_words + T * DP + 4 * v, a.q.smin + 4 * v);
        asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
        __syncthreads();
    }
    unsigned long long n_tests = 0, n_checks = 0;
    if (resident) {
        for (;;) {
            unsigned i = 0;
            if (lane == 0) i = atomicAdd(a.counter, 1u);
            i = __shfl_sync(kFull, i, 0);
            if ((long long)i >= S) break;
            const int r = dom_target<D, SLOTS, true, GM, CNT, kPairTiles<D>>(a.q, stage, stage + cand_words,
                                                              stage + cand_words + T * DP, T, i, wsteps, n_tests,
                                                              n_checks, a.pc);
            if (lane == 0) a.q.out[a.q.perm[i]] = r;
        }
    } else {
        for (;;) {
            unsigned i = 0;
            if (lane == 0) i = atomicAdd(a.counter, 1u);
            i = __shfl_sync(kFull, i, 0);
            if ((long long)i >= S) break;
            const int r = dom_target<D, SLOTS, false, GM, CNT, kPairTiles<D>>(a.q, a.q.cand, a.q.tmin, a.q.smin, T, i, wsteps,
                                                               n_tests, n_checks, a.pc);
            if (lane == 0) a.q.out[a.q.perm[i]] = r;
        }
    }
    if (CNT && a.tests && lane == 0 && (n_tests | n_checks)) {
        atomicAdd(a.tests, n_tests);
        atomicAdd(a.tests + 1, n_checks);
    }
}

// Many queries (same D) in one launch: work items are the (query, target)
// pairs of all queries, handed out by one counter; candidates are read through
// L1 (each query has its own candidate set). A query with iperm set takes
// only its target range (see DomQuery).
constexpr int kMaxBatch = 256;
struct DomBatch {
    int count;
    unsigned *counter;        // zeroed before the launch
    DomQuery q[kMaxBatch];
};

template <int D, int SLOTS>
__global__ void __launch_bounds__(dom_threads<D, SLOTS>(), 1)
k_dominance_batch(const __grid_constant__ DomBatch b) {
    constexpr int WS = 32 * SLOTS;
    __shared__ unsigned long long first[kMaxBatch + 1];   // prefix sums of the targets
    extern __shared__ __align__(16) uint32_t sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t *wsteps = sm + warp * WS;
    if (threadIdx.x == 0) {
        unsigned long long run = 0;
        for (int j = 0; j < b.count; j++) {
            first[j] = run;
            run += b.q[j].iperm ? (unsigned long long)b.q[j].tn : (unsigned long long)*b.q[j].n_sky;
        }
        first[b.count] = run;
    }
    __syncthreads();
    const unsigned long long total = first[b.count];
    unsigned long long n_tests = 0, n_checks = 0;
    for (;;) {
        unsigned g = 0;
        if (lane == 0) g = atomicAdd(b.counter, 1u);
        g = __shfl_sync(kFull, g, 0);
        if (g >= total) break;
        int lo = 0, hi = b.count - 1;   // query j with first[j] <= g < first[j + 1]
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (first[mid] <= g) lo = mid; else hi = mid - 1;
        }
        // a copy: the search reads its fields often, and indexed reads of the
        // launch parameters go through the constant cache, shared by all queries
        const DomQuery q = b.q[lo];
        const long long S = *q.n_sky;
        const long long T = (S + kTileRows - 1) / kTileRows;
        const unsigned local = (unsigned)(g - first[lo]);
        const unsigned i = q.iperm ? __ldg(q.iperm + q.t0 + local) : local;
        const int r = dom_target<D, SLOTS, false, false, false, false>(q, q.cand, q.tmin, q.smin, T, i, wsteps, n_tests,
                                                                    n_checks, PartCount());
        if (lane == 0) q.out[q.iperm ? local : q.perm[i]] = r;
    }
}

__global__ void k_invert_perm(const uint32_t *perm, long long S, uint32_t *iperm) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < S; i += stride)
        iperm[perm[i]] = (uint32_t)i;
}

constexpr int kMaxMagicJobs = 256;
struct MagicBatch {
    int count;
    MagicJob j[kMaxMagicJobs];
};

__global__ void k_make_magic(const __grid_constant__ MagicBatch b) {
    for (int jb = blockIdx.x; jb < b.count; jb += gridDim.x) {
        const MagicJob &job = b.j[jb];
        if (job.zero && threadIdx.x == 0) *job.zero = 0u;
        for (int k = threadIdx.x; k < job.K; k += blockDim.x)
            reinterpret_cast<uint4 *>(job.magic)[k] = magic_of(job.steps[k]);
    }
}

__global__ void k_gproj(const uint32_t *v, long long count, StepChunk c, uint32_t *out) {
    const long long total = count * c.count;
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < total;
         x += (long long)gridDim.x * blockDim.x) {
        const long long j = x / count, i = x - j * count;
        const uint4 mg = c.e[j];
        out[(c.off + j) * count + i] = udiv(v[i], mg.x, mg.y, mg.z);
    }
}

int g_sm_count = 0;
int g_smem_optin = 0;

cudaError_t device_props() {
    if (g_sm_count) return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    return cudaDeviceGetAttribute(&g_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
}

template <int D, int SLOTS, bool GM, bool CNT>
cudaError_t launch_dom(DomArgs a, cudaStream_t st) {
    static bool configured = false;
    const int smem = g_smem_optin;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_dominance<D, SLOTS, GM, CNT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    a.smem_words = smem / 4;
    k_dominance<D, SLOTS, GM, CNT><<<g_sm_count, dom_threads<D, SLOTS, GM>(), smem, st>>>(a); note_launch();
    return cudaGetLastError();
}

template <int D, int SLOTS, bool GM>
cudaError_t launch_dom_counted(DomArgs a, cudaStream_t st) {
    return a.tests ? launch_dom<D, SLOTS, GM, true>(a, st) : launch_dom<D, SLOTS, GM, false>(a, st);
}

template <int D, int SLOTS>
cudaError_t launch_dom_batch(const DomBatch &b, cudaStream_t st) {
    const int smem = (dom_threads<D, SLOTS>() / 32) * 32 * SLOTS * 4;
    k_dominance_batch<D, SLOTS><<<g_sm_count, dom_threads<D, SLOTS>(), smem, st>>>(b); note_launch();
    return cudaGetLastError();
}

// Key widths, known on the host: partition number (pbits bits) << obits |
// order, with obits = bpa * d the order bits that the partition number leaves
// below a budget (at least one per attribute). The budget is 16 bits (two
// radix passes) for the single-cluster path, where the sort is a good part of
// the stage, and 32 bits above it, where the grid-dominance time dominates and
// finer tiles pay (ANT N=1M d=6: 25% less dominance time than with 16 bits).
// Returns obits.
int order_bits(const gres_plan_cfg &cfg, int d, int64_t n, int *pbits, int *bpa) {
    const int budget = n <= kClusterSortMax ? 16 : 32;
    unsigned long long cells = 1;
    if (cfg.scheme == GRES_PART_GRID || cfg.scheme == GRES_PART_ANGULAR)
        for (int i = 0; i < (cfg.scheme == GRES_PART_GRID ? d : d - 1); i++) cells *= (unsigned long long)cfg.m;
    if (cfg.scheme == GRES_PART_SLICED) cells = (unsigned long long)cfg.p;
    int b = 0;
    for (unsigned long long v = cells - 1; v; v >>= 1) b++;
    *pbits = b;
    *bpa = std::max(1, (budget - b) / d);
    return *bpa * d;
}

template <int D>
cudaError_t partition_d(const gres_plan_cfg &cfg, int64_t n, Workspace &ws, cudaStream_t st) {
    const int scheme = cfg.scheme;
    PartArgs pa;
    std::memset(&pa, 0, sizeof(pa));
    pa.scheme = scheme;
    pa.m = cfg.m;
    pa.p = cfg.p;
    pa.dim = cfg.slice_dim;
    if (scheme == GRES_PART_ANGULAR) {
        const double pi = 3.14159265358979323846;
        for (int j = 1; j < cfg.m && j < 64; j++) {
            const double t = std::tan((double)j * pi / (2.0 * (double)cfg.m));
            pa.thr[j] = (unsigned long long)std::llround(t * t * 4294967296.0);
        }
    }
    auto passes = [&](int bits) { return (bits + 7) / 8; };
    // A skyline of at most kClusterSortMax rows is partitioned in one cluster launch
    // (16-bit keys), a larger one in one cooperative launch (32-bit keys). S is known on
    // the device only: for inputs above kClusterSortMax rows both are queued and each
    // returns at once for the other size.
    PartArgs ps = pa;
    int pbits_s = 0;
    ps.obits = order_bits(cfg, D, std::min<int64_t>(n, kClusterSortMax), &pbits_s, &ps.bpa);
    ps.key32 = pbits_s + ps.obits <= 32 ? 1 : 0;   // SLICED's first key is one 32-bit value
    static bool configured = false;
    cudaError_t e = launch_cluster(k_part_cluster<D>, kClSmemBytes, &configured, st, (const uint32_t *)ws.sky_rows,
                                   ws.hdr, ps, ws.keys[0], ws.vals[0], ws.keys[1], ws.vals[1], ws.cand, ws.tmin,
                                   ws.smin, ws.perm);
    if (e != cudaSuccess || n <= kClusterSortMax) return e;
    int pbits = 0;
    pa.obits = order_bits(cfg, D, n, &pbits, &pa.bpa);
    pa.key32 = pbits + pa.obits <= 32 ? 1 : 0;
    static int coop = 0;
    if (!coop && (e = coop_blocks(k_part_coop<D>, &coop)) != cudaSuccess) return e;
    e = launch_coop(k_part_coop<D>, coop, st, (const uint32_t *)ws.sky_rows, ws, pa,
                    passes(scheme == GRES_PART_SLICED ? 32 : pa.obits + pbits), passes(pa.obits + pbits));
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <int D>
cudaError_t dominance_d(int slots, const DomQuery &q, unsigned *counter, unsigned long long *tests,
                        cudaStream_t st, const PartCount &pc) {
    DomArgs a;
    a.q = q;
    a.pc = pc;
    a.counter = counter;
    a.tests = tests;
    a.smem_words = 0;
    if (q.gbits) return slots == 4 ? launch_dom_counted<D, 4, true>(a, st) : launch_dom_counted<D, 8, true>(a, st);
    return slots == 4 ? launch_dom_counted<D, 4, false>(a, st) : launch_dom_counted<D, 8, false>(a, st);
}

template <int D>
cudaError_t dominance_batch_d(int slots, const DomQuery *qs, int count, unsigned *counter, cudaStream_t st) {
    DomBatch b;
    b.count = count;
    b.counter = counter;
    for (int i = 0; i < count; i++) b.q[i] = qs[i];
    return slots == 4 ? launch_dom_batch<D, 4>(b, st) : launch_dom_batch<D, 8>(b, st);
}

#define GRES_DISPATCH_D(d, call)                \
    switch (d) {                                \
        case 1: return call(1);                 \
        case 2: return call(2);                 \
        case 3: return call(3);                 \
        case 4: return call(4);                 \
        case 5: return call(5);                 \
        case 6: return call(6);                 \
        case 7: return call(7);                 \
        case 8: return call(8);                 \
        default: return cudaErrorInvalidValue;  \
    }

}  // namespace

cudaError_t launch_upload_steps(uint32_t *d_steps, uint32_t *d_magic, unsigned *zero, const uint32_t *h_steps,
                                int k, cudaStream_t st) {
    return upload_steps(h_steps, k, d_steps, d_magic, nullptr, 0, zero, 0, nullptr, st);
}

cudaError_t launch_init_steps(Workspace &ws, int64_t n, const uint32_t *h_steps, int k, cudaStream_t st,
                              int gbits) {
    return upload_steps(h_steps, k, ws.steps, ws.magic, ws.hdr, (long long)n, nullptr, gbits, ws.sel_hist, st);
}

cudaError_t launch_partition(int d, const gres_plan_cfg &cfg, int64_t n, Workspace &ws, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    cudaError_t e = device_props();
    if (e != cudaSuccess) return e;
#define GRES_PART(D) partition_d<D>(cfg, n, ws, st)
    GRES_DISPATCH_D(d, GRES_PART)
#undef GRES_PART
}

cudaError_t launch_invert_perm(const uint32_t *perm, int64_t S, uint32_t *iperm, cudaStream_t st) {
    if (S == 0) return cudaSuccess;
    cudaError_t e = device_props();
    if (e != cudaSuccess) return e;
    const int blocks = (int)std::min<int64_t>((S + 255) / 256, (int64_t)g_sm_count * 4);
    k_invert_perm<<<blocks, 256, 0, st>>>(perm, (long long)S, iperm); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_load_candidates(const uint32_t *d_rows, int64_t n, int d, int dir, Workspace &ws,
                                   cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    cudaError_t e = device_props();
    if (e != cudaSuccess) return e;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)g_sm_count * 4);
#define GRES_LOAD(D) (k_load_candidates<D><<<blocks, 256, 0, st>>>(d_rows, dir, (long long)n, ws.sky_rows, ws.hdr), \
                      note_launch(), cudaGetLastError())
    GRES_DISPATCH_D(d, GRES_LOAD)
#undef GRES_LOAD
}

cudaError_t launch_partition_out(int d, const gres_plan_cfg &cfg, int64_t n, Workspace &ws, int64_t *d_part,
                                 uint32_t *d_order, uint32_t *d_tile_min, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const int scheme = cfg.scheme;
    int pbits = 0, bpa = 0;
    const int obits = order_bits(cfg, d, n, &pbits, &bpa);
    const int64_t total = std::max<int64_t>(n, (n + kTileRows - 1) / kTileRows * d);
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)g_sm_count * 4);
#define GRES_OUT(D) (k_partition_out<D><<<blocks, 256, 0, st>>>(ws.hdr, ws.keys[0], ws.keys[1], ws.perm, \
                     ws.tmin, scheme, obits, (long long)n, d_part, d_order, d_tile_min), note_launch(), cudaGetLastError())
    GRES_DISPATCH_D(d, GRES_OUT)
#undef GRES_OUT
}

cudaError_t launch_dominance(int d, int slots, const DomQuery &q, unsigned *counter,
                             unsigned long long *tests, cudaStream_t st, const PartCount &pc) {
    cudaError_t e = device_props();
    if (e != cudaSuccess) return e;
#define GRES_DOM(D) dominance_d<D>(slots, q, counter, tests, st, pc)
    GRES_DISPATCH_D(d, GRES_DOM)
#undef GRES_DOM
}

cudaError_t launch_dominance_batch(int d, int slots, const DomQuery *qs, int count, unsigned *counter,
                                   cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    if (count > kMaxBatch) return cudaErrorInvalidValue;
    cudaError_t e = device_props();
    if (e != cudaSuccess) return e;
#define GRES_DOMB(D) dominance_batch_d<D>(slots, qs, count, counter, st)
    GRES_DISPATCH_D(d, GRES_DOMB)
#undef GRES_DOMB
}

cudaError_t launch_make_magic(const MagicJob *jobs, int count, cudaStream_t st) {
    for (int off = 0; off < count; off += kMaxMagicJobs) {
        MagicBatch b;
        b.count = std::min(kMaxMagicJobs, count - off);
        for (int i = 0; i < b.count; i++) b.j[i] = jobs[off + i];
        k_make_magic<<<b.count, 256, 0, st>>>(b); note_launch();
    }
    return cudaGetLastError();
}

cudaError_t launch_rep_bound(int d, int64_t n, Workspace &ws, int k, int dir, int gbits,
                             unsigned long long *tests, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    cudaError_t e = device_props();
    if (e != cudaSuccess) return e;
    const int blocks = (int)std::min<int64_t>((n * 32 + 255) / 256, (int64_t)g_sm_count * 8);
#define GRES_RB(D) (k_rep_bound<D><<<blocks, 256, 0, st>>>(ws.cand, ws.greps, &ws.hdr->n_sky, ws.magic, k, dir, \
                    gbits, ws.res, tests), note_launch(), cudaGetLastError())
    GRES_DISPATCH_D(d, GRES_RB)
#undef GRES_RB
}

int64_t plan_partitions(const gres_plan_cfg &cfg, int d) {
    if (cfg.scheme == GRES_PART_SLICED) return cfg.p;
    if (cfg.scheme == GRES_PART_GRID || cfg.scheme == GRES_PART_ANGULAR) {
        int64_t cells = 1;
        for (int i = 0; i < (cfg.scheme == GRES_PART_GRID ? d : d - 1); i++) cells *= cfg.m;
        return cells;
    }
    return 1;
}

cudaError_t launch_gres_stage(const uint32_t * /*d_data*/, int64_t n, int d, int dir, int k,
                              const gres_plan_cfg &cfg, Workspace &ws,
                              const int64_t * /*d_sky_idx*/, int32_t *d_step_idx,
                              unsigned long long *d_tests, cudaStream_t st, int gbits) {
    if (n == 0) return cudaSuccess;
    stage_begin(kStagePartition, st);
    cudaError_t e = launch_partition(d, cfg, n, ws, st);
    stage_end(kStagePartition, st);
    if (e != cudaSuccess) return e;
    DomQuery q;
    q.cand = ws.cand;
    q.tmin = ws.tmin;
    q.smin = ws.smin;
    q.perm = ws.perm;
    q.n_sky = &ws.hdr->n_sky;
    q.magic = ws.magic;
    q.steps = ws.steps;
    q.out = d_step_idx;
    q.K = k;
    q.dir = dir;
    q.gbits = gbits;
    unsigned long long *counts = (cfg.flags & GRES_FLAG_COUNT_TESTS) ? d_tests : nullptr;
    PartCount pc;
    if ((cfg.flags & GRES_FLAG_COUNT_PARTS) && d_tests) {
        if ((e = device_props()) != cudaSuccess) return e;
        int pb = 0, bpa = 0;
        const int ob_s = order_bits(cfg, d, std::min<int64_t>(n, kClusterSortMax), &pb, &bpa);
        const int ob_l = order_bits(cfg, d, n, &pb, &bpa);
        const int blocks = (int)std::min<int64_t>((n + kTileRows + 255) / 256, (int64_t)g_sm_count * 4);
        k_part_ids<<<blocks, 256, 0, st>>>(ws.hdr, ws.keys[0], ws.keys[1], cfg.scheme == GRES_PART_NONE ? 1 : 0,
                                           ob_s, ob_l, ws.pid); note_launch();
        pc.pid = ws.pid;
        pc.pcnt = d_tests;
        pc.nparts = (unsigned)std::min<int64_t>(plan_partitions(cfg, d), 0xFFFFFFFFll);
    }
    stage_begin(kStageDominance, st);   // the representative bound pass counts as grid-dominance work
    if (cfg.flags & GRES_FLAG_GRES_REPS) {
        q.ub = ws.res;
        e = launch_rep_bound(d, n, ws, k, dir, gbits, counts, st);
        if (e != cudaSuccess) {
            stage_end(kStageDominance, st);
            return e;
        }
    }
    e = launch_dominance(d, cfg.slots, q, &ws.hdr->work_next,
                         (cfg.flags & GRES_FLAG_COUNT_TESTS) ? d_tests : nullptr, st, pc);
    stage_end(kStageDominance, st);
    return e;
}

cudaError_t launch_gproj(const uint32_t *d_values, int64_t count, const uint32_t *h_steps, int k,
                         uint32_t *d_out, cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    cudaError_t e = device_props();
    if (e != cudaSuccess) return e;
    StepChunk c;
    for (int off = 0; off < k; off += kStepChunk) {
        c.off = off;
        c.count = std::min(kStepChunk, k - off);
        for (int i = 0; i < c.count; i++) {
            uint32_t m, s1, s2;
            udiv_magic(h_steps[off + i], &m, &s1, &s2);
            c.e[i] = make_uint4(m, s1, s2, h_steps[off + i]);
        }
        const long long total = (long long)count * c.count;
        const int blocks = (int)std::min<long long>((total + 255) / 256, (long long)g_sm_count * 8);
        k_gproj<<<blocks, 256, 0, st>>>(d_values, (long long)count, c, d_out); note_launch();
    }
    return cudaGetLastError();
}

void udiv_magic(uint32_t delta, uint32_t *m, uint32_t *s1, uint32_t *s2) {
    int l = 0;
    while (l < 32 && (1ull << l) < (unsigned long long)delta) l++;   // l = ceil(log2 delta)
    const unsigned long long two32 = 1ull << 32;
    const unsigned long long num = two32 * ((1ull << l) - (unsigned long long)delta);
    *m = (uint32_t)(num / delta + 1ull);
    *s1 = l < 1 ? (uint32_t)l : 1u;
    *s2 = l > 1 ? (uint32_t)(l - 1) : 0u;
}

}  // namespace gres
