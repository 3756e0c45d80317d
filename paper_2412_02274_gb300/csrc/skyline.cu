// skyline.cu -- Sky(r) (Def. 1) by a sort-by-sum pass with block dominance filters.
//
// Pipeline (all sizes after n live in the workspace header):
//   1. keys:    canonical rows (smaller is better; GRES_MAX reads ~v) and the
//               key f(t) = sum of the canonical values. f is monotone, so s
//               dominates t implies f(s) < f(t).
//   2. select:  the representatives of Representative Filtering (Sec. 3.1):
//               the rows with the smallest f, found by a selection (a
//               range-free histogram of f by its leading bits, then 4,096
//               sub-buckets of the boundary bucket, give a threshold leaving
//               at most R rows below it), then ordered by the Morton code of
//               their rows so that runs of 32 are spatially tight.
//               Representatives dominated by another one stay: by
//               transitivity the filter drops the same rows either way.
//   3. filter:  a first pass, one row per thread, against 32 of the
//               representatives (one per spatial run: the one dominating the
//               largest part of the data's box); then every row it leaves
//               against all the representatives.
//   4. group:   the survivors in a spatial order (a Morton code over their
//               bounding box: 16 bits, or at least 4 bits per attribute when
//               more than 131,072 rows survive) in 32-row tiles with
//               per-tile and per-1024-row minima.
//   5. final:   each survivor against the survivors of every tile whose
//               minimum is <= it in every attribute; it is in the skyline iff
//               none dominates it. (If t is dominated, a skyline tuple
//               dominates it, and skyline tuples always survive step 3.)
//   6. flags by original row -> ascending row numbers, plus the canonical
//      skyline rows for the gres stage.
#include "cluster.cuh"
#include "radix.cuh"

#include <algorithm>

namespace gres {

namespace {

constexpr int kCT = 256;            // threads per compaction block
constexpr int kPer = 32;            // consecutive rows per compaction thread
constexpr int kCB = kCT * kPer;     // rows per compaction block (and per k_final segment count)
static_assert(kCB <= 65536, "row offsets inside a compaction block are 16-bit");
constexpr int kTriThreads = 256;

template <int D>
__device__ __forceinline__ void load_canon(const uint32_t *data, long long row, int dir, uint32_t (&x)[D]) {
    const uint32_t *p = data + row * D;
    #pragma unroll
    for (int i = 0; i < D; i++) x[i] = canon(p[i], dir);
}

template <int D>
__device__ __forceinline__ void load_row(const uint32_t *base, long long r, uint32_t (&x)[D]) {
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
__device__ __forceinline__ void store_row(uint32_t *base, long long r, const uint32_t (&x)[D]) {
    constexpr int DP = padded_dims(D);
    uint32_t y[DP];
    #pragma unroll
    for (int i = 0; i < DP; i++) y[i] = i < D ? x[i < D ? i : 0] : 0u;
    uint4 *p = reinterpret_cast<uint4 *>(base + r * DP);
    p[0] = make_uint4(y[0], y[1], y[2], y[3]);
    if (DP == 8) p[1] = make_uint4(y[4 % DP], y[5 % DP], y[6 % DP], y[7 % DP]);
}

// Def. 1 on canonical rows: s dominates t.
template <int D>
__device__ __forceinline__ bool dominates(const uint32_t (&s)[D], const uint32_t (&t)[D]) {
    bool le = true, lt = false;
    #pragma unroll
    for (int i = 0; i < D; i++) {
        le &= s[i] <= t[i];
        lt |= s[i] < t[i];
    }
    return le && lt;
}

// Smallest row sum over the warp's rows (~0 for lanes without a row): a tile
// can hold a dominator of x only if some row sums to less than x (Def. 1 on
// canonical values implies a strictly smaller sum).
template <int D, int DP>
__device__ __forceinline__ unsigned long long warp_min_sum(const uint32_t (&x)[DP], bool valid) {
    unsigned long long v = 0;
    #pragma unroll
    for (int q = 0; q < D; q++) v += x[q];
    if (!valid) v = ~0ull;
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, v, o);
        v = y < v ? y : v;
    }
    return v;
}

// Morton code of x - lo over `bits` bits per attribute (D * bits <= 32):
// coordinate i is quantized to floor((x_i - lo_i) 2^bits / (hi_i - lo_i + 1)).
template <int D>
__device__ __forceinline__ uint32_t morton(const uint32_t (&x)[D], const uint32_t *lo, const uint32_t *hi, int bits) {
    uint32_t q[D];
    #pragma unroll
    for (int i = 0; i < D; i++) {
        const unsigned long long span = (unsigned long long)(hi[i] - lo[i]) + 1ull;
        q[i] = (uint32_t)(((unsigned long long)(x[i] - lo[i]) << bits) / span);
    }
    uint32_t key = 0;
    for (int b = bits - 1; b >= 0; b--) {
        #pragma unroll
        for (int i = 0; i < D; i++) key = (key << 1) | ((q[i] >> b) & 1u);
    }
    return key;
}

// Exclusive scan over a kCT-thread block; *total gets the block sum.
__device__ __forceinline__ uint32_t block_scan(uint32_t v, uint32_t *total) {
    __shared__ uint32_t wsum[kCT / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t incl = v;
    #pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    uint32_t before = 0, all = 0;
    #pragma unroll
    for (int j = 0; j < kCT / 32; j++) {
        uint32_t x = wsum[j];
        before += j < w ? x : 0u;
        all += x;
    }
    __syncthreads();
    *total = all;
    return before + incl - v;
}

__global__ void k_init(WsHeader *h, long long n, uint32_t *sel) {
    init_header(h, n);
    clear_sel_hist(sel);
}


// ---- representative selection ------------------------------------------------
// The representatives are the rows of smallest f (at most R of them, Sec. 3.1),
// found by two histogram levels. Level 1 buckets f without knowing its range:
// f < 128 exactly, larger f by its leading bit and the 6 bits below it (1,920
// buckets, monotone in f, relative width 1/64). Level 2 splits the bucket
// where the running count passes R into up to 4,096 equal sub-buckets.
constexpr int kSelBuckets = 4096;
static_assert(2 * kSelBuckets == kSelHistWords, "two histogram levels in the workspace's counters");

__device__ __forceinline__ uint32_t fbucket(unsigned long long f) {
    if (f < 128ull) return (uint32_t)f;
    const int e = 63 - __clzll((long long)f);                  // leading bit, 7 .. 34
    return 128u + (uint32_t)(e - 7) * 64u + (uint32_t)((f >> (e - 6)) & 63ull);
}

// Lowest value of level-1 bucket b and log2 of its width.
__device__ __forceinline__ void fbucket_range(uint32_t b, unsigned long long *lo, int *wbits) {
    if (b < 128u) { *lo = b; *wbits = 0; return; }
    const int e = 7 + (int)((b - 128u) / 64u);
    const unsigned long long m = (b - 128u) % 64u;
    *wbits = e - 6;
    *lo = (64ull + m) << (e - 6);
}

// Run by the last block (1024 threads) of a histogram kernel: the first bucket
// at which the running count (plus `base`) exceeds R, as (bucket << 32 |
// count below it); ~0 when every row fits.
__device__ __forceinline__ unsigned long long sel_find(const uint32_t *hist, uint32_t base, int R) {
    __shared__ uint32_t wsum[32];
    __shared__ unsigned long long found;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) found = ~0ull;
    uint32_t c[4], local = 0;
    #pragma unroll
    for (int q = 0; q < 4; q++) { c[q] = hist[4 * tid + q]; local += c[q]; }
    uint32_t incl = local;
    #pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    uint32_t before = 0;
    for (int j = 0; j < 32; j++) before += j < w ? wsum[j] : 0u;
    uint32_t run = base + before + incl - local;
    #pragma unroll
    for (int q = 0; q < 4; q++) {
        if (run + c[q] > (uint32_t)R) {
            atomicMin(&found, ((unsigned long long)(4 * tid + q) << 32) | run);
            break;
        }
        run += c[q];
    }
    __syncthreads();
    return found;
}

// Sum keys f = sum_i c_i (A2) and the level-1 histogram; the last block picks
// the level-1 bucket b1 (sel_b1 = kSelBuckets when all rows fit in R).
template <int D>
__global__ void __launch_bounds__(1024)
k_keys(const uint32_t *data, long long n, int dir, unsigned long long *keys, WsHeader *h, uint32_t *hist, int R) {
    __shared__ uint32_t sh[kSelBuckets];
    __shared__ uint32_t blo[D], bhi[D];
    for (int b = threadIdx.x; b < kSelBuckets; b += blockDim.x) sh[b] = 0;
    if (threadIdx.x < D) { blo[threadIdx.x] = 0xFFFFFFFFu; bhi[threadIdx.x] = 0u; }
    __syncthreads();
    uint32_t lo[D], hi[D];
    #pragma unroll
    for (int j = 0; j < D; j++) { lo[j] = 0xFFFFFFFFu; hi[j] = 0u; }
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        uint32_t x[D];
        load_canon<D>(data, i, dir, x);
        unsigned long long k = 0;
        #pragma unroll
        for (int j = 0; j < D; j++) {
            k += x[j];
            lo[j] = min(lo[j], x[j]);
            hi[j] = max(hi[j], x[j]);
        }
        keys[i] = k;
        atomicAdd(&sh[fbucket(k)], 1u);
    }
    // the data's per-attribute range (dlo / dhi: the first filter pass ranks its
    // representatives by the part of that box they dominate)
    #pragma unroll
    for (int j = 0; j < D; j++) {
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo[j] = min(lo[j], __shfl_xor_sync(0xffffffffu, lo[j], o));
            hi[j] = max(hi[j], __shfl_xor_sync(0xffffffffu, hi[j], o));
        }
        if ((threadIdx.x & 31) == 0 && lo[j] <= hi[j]) { atomicMin(&blo[j], lo[j]); atomicMax(&bhi[j], hi[j]); }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kSelBuckets; b += blockDim.x)
        if (sh[b]) atomicAdd(&hist[b], sh[b]);
    if (threadIdx.x < D && blo[threadIdx.x] <= bhi[threadIdx.x]) {
        atomicMin(&h->dlo[threadIdx.x], blo[threadIdx.x]);
        atomicMax(&h->dhi[threadIdx.x], bhi[threadIdx.x]);
    }
    if (last_block_done(&h->done[0])) {
        const unsigned long long found = sel_find(hist, 0u, R);
        if (threadIdx.x == 0) {
            if (found == ~0ull) { h->sel_b1 = kSelBuckets; h->sel_below = 0; }
            else { h->sel_b1 = (uint32_t)(found >> 32); h->sel_below = (uint32_t)found; }
        }
    }
}

// Bitonic sort of one value per thread over a block of kMaxReps threads
// (compare-exchange partners under 32 apart through warp shuffles, the others
// through shared memory sk); returns this thread's value of the ascending
// order.
__device__ __forceinline__ unsigned long long block_bitonic(unsigned long long v, unsigned long long *sk) {
    const int tid = threadIdx.x;
    for (int size = 2; size <= kMaxReps; size <<= 1) {
        const bool asc = (tid & size) == 0;
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            unsigned long long other;
            if (stride >= 32) {
                sk[tid] = v;
                __syncthreads();
                other = sk[tid ^ stride];
                __syncthreads();
            } else {
                other = __shfl_xor_sync(0xffffffffu, v, stride);
            }
            const bool lower = (tid & stride) == 0;
            const unsigned long long mn = other < v ? other : v, mx = other < v ? v : other;
            v = (asc == lower) ? mn : mx;
        }
    }
    return v;
}

// Orders the representatives spatially -- by the Morton code of their rows
// over their bounding box, then by row -- with a bitonic sort in one block,
// and writes their canonical rows to `rows` in that order. Spatially tight
// runs of 32 representatives let the filter skip whole runs. Representatives
// dominated by another representative stay: by transitivity the filter drops
// exactly the same rows with or without them. Also clears the per-segment
// skyline counts that k_final fills (nb of them). greps (may be NULL): also the 32
// candidates of smallest f, canonical rows padded with sentinel rows, for the
// gres stage's representatives. Run by one block of kMaxReps threads (all of
// them); nc = the number of candidates in rep_idx; sk, xs, lo, hi: shared
// arrays of kMaxReps, D * kMaxReps, D and D words.
template <int D>
__device__ __forceinline__ void rep_sort_block(const uint32_t *data, int dir, const uint32_t *rep_idx, int nc,
                                               WsHeader *h, uint32_t *rows, uint32_t *blocksum, long long nb,
                                               uint32_t *greps, uint32_t *kill, unsigned long long *sk,
                                               uint32_t *xs, uint32_t *lo, uint32_t *hi) {
    const int tid = threadIdx.x;
    for (long long j = tid; j < nb; j += kMaxReps) blocksum[j] = 0u;
    if (tid < D) { lo[tid] = 0xFFFFFFFFu; hi[tid] = 0u; }
    __syncthreads();
    uint32_t x[D];
    const uint32_t idx = tid < nc ? __ldcg(rep_idx + tid) : 0xFFFFFFFFu;
    if (tid < nc) load_canon<D>(data, idx, dir, x);
    else {
        #pragma unroll
        for (int q = 0; q < D; q++) x[q] = 0u;
    }
    #pragma unroll
    for (int q = 0; q < D; q++) {
        xs[q * kMaxReps + tid] = tid < nc ? x[q] : 0u;
        uint32_t a = tid < nc ? x[q] : 0xFFFFFFFFu, b = tid < nc ? x[q] : 0u;
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a = min(a, __shfl_xor_sync(0xffffffffu, a, o));
            b = max(b, __shfl_xor_sync(0xffffffffu, b, o));
        }
        if ((tid & 31) == 0 && a <= b) { atomicMin(&lo[q], a); atomicMax(&hi[q], b); }
    }
    __syncthreads();
    if (greps) {
        // f < 2^35 and tid < 2^10: (f, candidate) in one 64-bit key
        unsigned long long f = 0;
        #pragma unroll
        for (int q = 0; q < D; q++) f += tid < nc ? x[q] : 0u;
        const unsigned long long g = block_bitonic(tid < nc ? (f << 10) | (unsigned long long)tid : ~0ull, sk);
        __syncthreads();
        if (tid < 32) {
            constexpr int DP = padded_dims(D);
            uint32_t y[D];
            if (g != ~0ull) {
                const int c = (int)(g & 1023ull);
                #pragma unroll
                for (int q = 0; q < D; q++) y[q] = xs[q * kMaxReps + c];
                store_row<D>(greps, tid, y);
            } else {
                #pragma unroll
                for (int q = 0; q < DP; q++) greps[tid * DP + q] = kSentinel;
            }
        }
    }
    // sort key: Morton code (22 / D bits per attribute) | row (31 bits) | slot
    // (10 bits): ordered by code then row, and the slot finds the shared copy
    const int bits = 22 / D;
    unsigned long long v = tid < nc ? ((unsigned long long)morton<D>(x, lo, hi, bits) << 41) |
                                          ((unsigned long long)idx << 10) | (unsigned long long)tid
                                    : ~0ull;
    v = block_bitonic(v, sk);
    if (tid < nc) {
        const int c = (int)(v & 1023ull);
        #pragma unroll
        for (int q = 0; q < D; q++) x[q] = xs[q * kMaxReps + c];
        store_row<D>(rows, tid, x);
    }
    {
        // The first filter pass's representatives: one per run of 32 in this spatial
        // order (kKillers = 32 runs at most), the one whose dominated region covers
        // the largest part of the data's box (score: the sum of log2(dhi_q - x_q + 1),
        // the log of the box volume above x; ties to the first), then ordered by
        // that score, strongest first. Spread over the runs, they cover different
        // parts of the data. A speed-only choice: correctness never depends on it.
        // Sentinel rows stand in for missing runs. sk is free after the sort.
        static_assert(kKillers == kMaxReps / 32, "one first-pass representative per run");
        constexpr int DP = padded_dims(D);
        const int lane = tid & 31, w = tid >> 5;
        unsigned long long key = 0;
        if (tid < nc) {
            float sc = 0.f;
            #pragma unroll
            for (int q = 0; q < D; q++) sc += __log2f((float)(h->dhi[q] - min(x[q], h->dhi[q])) + 1.f);
            key = (1ull << 63) | ((unsigned long long)__float_as_uint(sc) << 32) | (unsigned)(31 - lane);
        }
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long other = __shfl_xor_sync(0xffffffffu, key, o);
            key = other > key ? other : key;
        }
        const int src = 31 - (int)(key & 31ull);
        uint32_t y[D];
        #pragma unroll
        for (int q = 0; q < D; q++) y[q] = __shfl_sync(0xffffffffu, x[q], src);
        unsigned long long *kkey = sk;                              // per run: score | run
        uint32_t *krow = reinterpret_cast<uint32_t *>(sk + 32);     // per run: its row
        if (lane == 0) {
            kkey[w] = key ? ((key >> 32) << 32) | (unsigned long long)w : 0ull;
            #pragma unroll
            for (int q = 0; q < D; q++) krow[w * D + q] = y[q];
        }
        __syncthreads();
        if (w == 0) {
            // strongest first: a bitonic sort of the 32 run keys, descending
            unsigned long long v2 = kkey[lane];
            for (int size = 2; size <= 32; size <<= 1) {
                for (int stride = size >> 1; stride > 0; stride >>= 1) {
                    const unsigned long long other = __shfl_xor_sync(0xffffffffu, v2, stride);
                    const bool up = (lane & size) == 0, lower = (lane & stride) == 0;
                    const unsigned long long mn = other < v2 ? other : v2, mx = other < v2 ? v2 : other;
                    v2 = (up == lower) ? mx : mn;
                }
            }
            if (v2) {
                const int rw = (int)(v2 & 31ull);
                uint32_t z[D];
                #pragma unroll
                for (int q = 0; q < D; q++) z[q] = krow[rw * D + q];
                store_row<D>(kill, lane, z);
            } else {
                #pragma unroll
                for (int q = 0; q < DP; q++) kill[lane * DP + q] = kSentinel;
            }
        }
    }
    if (tid == 0) {
        h->n_cand = nc;
        h->n_reps = nc;
    }
}

// Level 2 and the gather in one pass: rows below bucket b1 are representatives
// at once; rows in b1 are counted per sub-bucket and listed (boundary list,
// capacity n). The last block finds the sub-bucket threshold, adds the listed
// rows under it (at most R rows in all), and then orders the representatives
// (rep_sort_block), so no separate launch is needed for that.
template <int D>
__global__ void __launch_bounds__(kMaxReps)
k_sel_l2(const unsigned long long *keys, long long n, WsHeader *h, uint32_t *hist, int R,
         unsigned long long *bnd, uint32_t *rep_idx, const uint32_t *data, int dir, uint32_t *rows,
         uint32_t *blocksum, long long nb, uint32_t *greps, uint32_t *kill) {
    // the level-2 histogram, and in the last block the representative sort's arrays
    constexpr size_t kHistBytes = sizeof(uint32_t) * kSelBuckets;
    constexpr size_t kRepBytes = sizeof(unsigned long long) * kMaxReps + sizeof(uint32_t) * (D * kMaxReps + 2 * D);
    __shared__ __align__(16) unsigned char raw[kHistBytes > kRepBytes ? kHistBytes : kRepBytes];
    __shared__ unsigned nc_s;
    uint32_t *sh = reinterpret_cast<uint32_t *>(raw);
    for (int b = threadIdx.x; b < kSelBuckets; b += blockDim.x) sh[b] = 0;
    __syncthreads();
    const uint32_t b1 = h->sel_b1;
    unsigned long long lo = 0;
    int wbits = 0;
    if (b1 < (uint32_t)kSelBuckets) fbucket_range(b1, &lo, &wbits);
    const int sh2 = wbits > 12 ? wbits - 12 : 0;
    unsigned *n_cand = reinterpret_cast<unsigned *>(&h->n_cand);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const unsigned long long f = keys[i];
        const uint32_t b = fbucket(f);
        if (b < b1) {
            const unsigned pos = atomicAdd(n_cand, 1u);
            if (pos < (unsigned)kMaxReps) rep_idx[pos] = (uint32_t)i;
        } else if (b == b1) {
            const uint32_t sb = (uint32_t)((f - lo) >> sh2);
            atomicAdd(&sh[sb], 1u);
            bnd[atomicAdd(&h->n_bnd, 1u)] = ((unsigned long long)sb << 32) | (unsigned long long)i;
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kSelBuckets; b += blockDim.x)
        if (sh[b]) atomicAdd(&hist[b], sh[b]);
    if (!last_block_done(&h->done[1])) return;
    if (b1 < (uint32_t)kSelBuckets) {   // else every row is a representative already
        const unsigned long long found = sel_find(hist, h->sel_below, R);
        const unsigned long long thr = found == ~0ull ? ~0ull : (found >> 32);
        const unsigned nbnd = h->n_bnd;
        for (unsigned j = threadIdx.x; j < nbnd; j += blockDim.x) {
            const unsigned long long v = bnd[j];
            if ((v >> 32) < thr) {
                const unsigned pos = atomicAdd(n_cand, 1u);
                if (pos < (unsigned)kMaxReps) rep_idx[pos] = (uint32_t)(v & 0xFFFFFFFFull);
            }
        }
    }
    __syncthreads();   // this block's gather (atomics, rep_idx stores) is done; sh is dead
    if (threadIdx.x == 0) nc_s = atomicAdd(n_cand, 0u);
    __syncthreads();
    unsigned long long *sk = reinterpret_cast<unsigned long long *>(raw);
    uint32_t *xs = reinterpret_cast<uint32_t *>(raw + sizeof(unsigned long long) * kMaxReps);
    rep_sort_block<D>(data, dir, rep_idx, (int)min(nc_s, (unsigned)kMaxReps), h, rows, blocksum, nb, greps, kill,
                      sk, xs, xs + D * kMaxReps, xs + D * kMaxReps + D);
}

// First filter pass, one row per thread: every row against the kKillers
// representatives that dominate the largest part of the data's box. A row one
// of them dominates is not a skyline tuple (Def. 1): its flag is set to 0.
// The other rows go, in no particular order, to the list that the warp filter
// (k_filter) works through. On uniform data this drops most rows for a few
// compares each; on anticorrelated data it drops few and adds a few percent
// to the filter's cost.
constexpr int kPreThreads = 256;
constexpr int kPreRows = 4;                             // rows per thread and chunk
constexpr int kPreChunk = kPreThreads * kPreRows;       // rows per block and chunk
constexpr int kPreA = 4;                                // representatives tested on every row
template <int D>
__device__ __forceinline__ void kill_row(const uint4 *ks, int k, uint32_t (&sv)[D]) {
    constexpr int DP = padded_dims(D);
    const uint4 a = ks[k * (DP / 4)];
    sv[0] = a.x;
    if (D > 1) sv[1 < D ? 1 : 0] = a.y;
    if (D > 2) sv[2 < D ? 2 : 0] = a.z;
    if (D > 3) sv[3 < D ? 3 : 0] = a.w;
    if (DP == 8) {
        const uint4 b = ks[k * (DP / 4) + (DP == 8 ? 1 : 0)];
        if (D > 4) sv[4 < D ? 4 : 0] = b.x;
        if (D > 5) sv[5 < D ? 5 : 0] = b.y;
        if (D > 6) sv[6 < D ? 6 : 0] = b.z;
        if (D > 7) sv[7 < D ? 7 : 0] = b.w;
    }
}

// Appends row i (when live) to the block's list lst (counter *cnt) with one
// shared atomic per warp.
__device__ __forceinline__ void block_append(bool live, uint32_t i, uint32_t *lst, unsigned *cnt) {
    const int lane = threadIdx.x & 31;
    const unsigned m = __ballot_sync(0xffffffffu, live);
    unsigned pos = 0;
    if (lane == 0 && m) pos = atomicAdd(cnt, (unsigned)__popc(m));
    pos = __shfl_sync(0xffffffffu, pos, 0);
    if (live) lst[pos + __popc(m & ((1u << lane) - 1u))] = i;
}

// Blocks take chunks of kPreChunk rows: every row against the kPreA strongest
// representatives, then the rows left against the others (compacted, one per
// thread); the chunk's surviving rows go to the list with one global atomic.
template <int D>
__global__ void __launch_bounds__(kPreThreads)
k_prefilter(const uint32_t *data, int dir, long long n, const uint32_t *kill, WsHeader *h, uint32_t *flags,
            uint32_t *alive) {
    constexpr int DP = padded_dims(D);
    __shared__ uint4 ks[kKillers * DP / 4];
    __shared__ uint32_t lst[kPreChunk];   // rows left by the first kPreA representatives
    __shared__ uint32_t buf[kPreChunk];   // the chunk's surviving rows
    __shared__ unsigned cnt_a, cnt, base;
    for (int j = threadIdx.x; j < kKillers * DP / 4; j += blockDim.x) ks[j] = reinterpret_cast<const uint4 *>(kill)[j];
    if (blockIdx.x == 0 && threadIdx.x == 0) {   // the sort-key range, cleared for the survivor sort
        h->key_min = ~0ull;
        h->key_max = 0ull;
    }
    for (long long c0 = (long long)blockIdx.x * kPreChunk; c0 < n; c0 += (long long)gridDim.x * kPreChunk) {
        if (threadIdx.x == 0) { cnt_a = 0; cnt = 0; }
        __syncthreads();
        #pragma unroll 1
        for (int r = 0; r < kPreRows; r++) {
            const long long i = c0 + (long long)r * kPreThreads + threadIdx.x;
            const bool valid = i < n;
            bool live = valid;
            if (valid) {
                uint32_t x[D];
                load_canon<D>(data, i, dir, x);
                #pragma unroll
                for (int k = 0; k < kPreA; k++) {
                    uint32_t sv[D];
                    kill_row<D>(ks, k, sv);
                    live = live && !dominates<D>(sv, x);
                }
                if (!live) flags[i] = 0u;
            }
            block_append(live, (uint32_t)i, lst, &cnt_a);
        }
        __syncthreads();
        const unsigned na = cnt_a;
        for (unsigned j0 = 0; j0 < na; j0 += kPreThreads) {
            const unsigned j = j0 + threadIdx.x;
            const bool valid = j < na;
            const uint32_t i = valid ? lst[j] : 0u;
            uint32_t x[D];
            if (valid) load_canon<D>(data, i, dir, x);
            else {
                #pragma unroll
                for (int q = 0; q < D; q++) x[q] = 0u;
            }
            bool live = valid;
            for (int k = kPreA; k < kKillers; k++) {
                if (!__any_sync(0xffffffffu, live)) break;
                uint32_t sv[D];
                kill_row<D>(ks, k, sv);
                live = live && !dominates<D>(sv, x);
            }
            if (valid && !live) flags[i] = 0u;
            block_append(live, i, buf, &cnt);
        }
        __syncthreads();
        if (threadIdx.x == 0) base = cnt ? atomicAdd(&h->n_alive, cnt) : 0u;
        __syncthreads();
        for (unsigned j = threadIdx.x; j < cnt; j += kPreThreads) alive[base + j] = buf[j];
        __syncthreads();
    }
}

// The rows the first pass left (alive, h->n_alive of them, in any order)
// against all the representatives. Survivors (rows no representative
// dominates) are listed, in no particular order, as canonical rows
// (surv_rows), original row numbers (surv_orig) and their count (n_surv),
// with their per-attribute range (slo / shi) for the spatial order; the
// flags of all the rows looked at are set to 0 (k_final sets the skyline
// rows' flags). The
// representatives sit in shared memory (attribute-major) in runs of 32 with
// each run's per-attribute minimum; a run can hold a dominator of x only if
// its minimum is <= x in every attribute. Each lane keeps the minimum of run
// `lane` in registers. A warp takes kFilterRowsPerWarp rows and checks them
// one at a time: the lanes test the run minima, then the rows of each
// possible run, stopping at the first dominator. Blocks stay resident and
// step through kFilterChunk-row chunks of the list, so the representatives
// are staged once per block and short per-warp chains keep many warps in
// flight.
constexpr int kFilterThreads = 512;
constexpr int kFilterRowsPerWarp = 4;
constexpr int kFilterChunk = (kFilterThreads / 32) * kFilterRowsPerWarp;
template <int D>
__global__ void __launch_bounds__(kFilterThreads)
k_filter(const uint32_t *data, int dir, const uint32_t *alive, const uint32_t *reps, WsHeader *h,
         uint32_t *flags, uint32_t *surv_rows, uint32_t *surv_orig) {
    constexpr int DP = padded_dims(D);
    __shared__ uint32_t rs[D * kMaxReps];
    __shared__ uint32_t rmin[D * (kMaxReps / 32)];
    __shared__ uint32_t srow[kFilterChunk];        // the chunk's survivors, listed at once
    __shared__ uint32_t sx[kFilterChunk * DP];
    __shared__ unsigned scnt;
    __shared__ unsigned long long sbase;
    __shared__ uint32_t blo[D], bhi[D];
    if (threadIdx.x < D) { blo[threadIdx.x] = 0xFFFFFFFFu; bhi[threadIdx.x] = 0u; }
    const int nr = (int)h->n_reps;
    const int nruns = (nr + 31) / 32;
    const long long na = h->n_alive;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int j = threadIdx.x; j < nruns * 32; j += kFilterThreads) {
        uint32_t x[D];
        if (j < nr) load_row<D>(reps, j, x);
        else {
            #pragma unroll
            for (int q = 0; q < D; q++) x[q] = kSentinel;
        }
        #pragma unroll
        for (int q = 0; q < D; q++) {
            rs[q * kMaxReps + j] = x[q];
            uint32_t m = x[q];
            #pragma unroll
            for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_xor_sync(0xffffffffu, m, o));
            if ((j & 31) == 0) rmin[q * (kMaxReps / 32) + (j >> 5)] = m;
        }
    }
    __syncthreads();
    uint32_t mn[D];   // minimum of run `lane`
    #pragma unroll
    for (int q = 0; q < D; q++) mn[q] = lane < nruns ? rmin[q * (kMaxReps / 32) + lane] : 0xFFFFFFFFu;
    const bool run_ok = lane < nruns;
    uint32_t lo[D], hi[D];
    #pragma unroll
    for (int q = 0; q < D; q++) { lo[q] = 0xFFFFFFFFu; hi[q] = 0u; }
    for (long long c0 = (long long)blockIdx.x * kFilterChunk; c0 < na; c0 += (long long)gridDim.x * kFilterChunk) {
        if (threadIdx.x == 0) scnt = 0;
        __syncthreads();
        const long long g0 = c0 + (long long)warp * kFilterRowsPerWarp;
        if (g0 < na) {
            const int lim = (int)min((long long)kFilterRowsPerWarp, na - g0);
            uint32_t x[D];
            const uint32_t row = lane < lim ? __ldcg(alive + g0 + lane) : 0u;
            if (lane < lim) load_canon<D>(data, row, dir, x);
            else {
                #pragma unroll
                for (int q = 0; q < D; q++) x[q] = 0u;
            }
            unsigned alive_mask = 0;
            for (int l = 0; l < lim; l++) {
                uint32_t xs[D];
                #pragma unroll
                for (int q = 0; q < D; q++) xs[q] = __shfl_sync(0xffffffffu, x[q], l);
                bool maybe = run_ok;
                #pragma unroll
                for (int q = 0; q < D; q++) maybe &= mn[q] <= xs[q];
                unsigned runs = __ballot_sync(0xffffffffu, maybe);
                bool dom = false;
                while (runs && !dom) {
                    const int rr = __ffs(runs) - 1;
                    runs &= runs - 1;
                    const int j = rr * 32 + lane;
                    uint32_t sv[D];
                    #pragma unroll
                    for (int q = 0; q < D; q++) sv[q] = rs[q * kMaxReps + j];
                    dom = __any_sync(0xffffffffu, j < nr && dominates<D>(sv, xs));
                }
                if (!dom) alive_mask |= 1u << l;
            }
            if (lane < lim) flags[row] = 0u;
            const bool keep = lane < lim && ((alive_mask >> lane) & 1u);
            const unsigned m = __ballot_sync(0xffffffffu, keep);
            unsigned pos = 0;
            if (lane == 0 && m) pos = atomicAdd(&scnt, (unsigned)__popc(m));
            pos = __shfl_sync(0xffffffffu, pos, 0);
            if (keep) {
                const unsigned slot = pos + __popc(m & ((1u << lane) - 1u));
                srow[slot] = row;
                #pragma unroll
                for (int q = 0; q < DP; q++) sx[slot * DP + q] = q < D ? x[q < D ? q : 0] : 0u;
                #pragma unroll
                for (int q = 0; q < D; q++) { lo[q] = min(lo[q], x[q]); hi[q] = max(hi[q], x[q]); }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0 && scnt)
            sbase = atomicAdd(reinterpret_cast<unsigned long long *>(&h->n_surv), (unsigned long long)scnt);
        __syncthreads();
        for (unsigned j = threadIdx.x; j < scnt; j += kFilterThreads) {
            surv_orig[sbase + j] = srow[j];
            #pragma unroll
            for (int q = 0; q < DP; q++) surv_rows[(sbase + j) * DP + q] = sx[j * DP + q];
        }
        __syncthreads();
    }
    // the survivors' range
    #pragma unroll
    for (int q = 0; q < D; q++) {
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo[q] = min(lo[q], __shfl_xor_sync(0xffffffffu, lo[q], o));
            hi[q] = max(hi[q], __shfl_xor_sync(0xffffffffu, hi[q], o));
        }
        if (lane == 0 && lo[q] <= hi[q]) { atomicMin(&blo[q], lo[q]); atomicMax(&bhi[q], hi[q]); }
    }
    __syncthreads();
    if (threadIdx.x < D && blo[threadIdx.x] <= bhi[threadIdx.x]) {
        atomicMin(&h->slo[threadIdx.x], blo[threadIdx.x]);
        atomicMax(&h->shi[threadIdx.x], bhi[threadIdx.x]);
    }
}

// Bits per attribute of the survivors' Morton code when more than
// kClusterSortMax rows survive: at least 4, so that at d >= 5 the final
// check's tiles stay tight when many survivors are not skyline rows. Fewer
// survivors keep 16 / D bits (a 16-bit code): there an extra digit pass costs
// more than it saves.
constexpr int surv_fine_bits(int D) { return 16 / D > 4 ? 16 / D : 4; }
constexpr int surv_sort_passes(int D) { return (D * surv_fine_bits(D) + 7) / 8; }

// The survivor sort above kClusterSortMax survivors, as one cooperative launch:
// the survivors' Morton keys over their range (surv_fine_bits bits per
// attribute), the stable radix sort (the passes the key range needs), then the
// survivors in that order in 32-row tiles padded with sentinel rows (all ones:
// never dominate), with each tile's per-attribute minimum (tmin) and each
// 1024-row super-tile's minimum (smin); perm gets the original row numbers.
// Returns at once (every block) when at most kClusterSortMax rows survive:
// k_surv_cluster sorts those. The key range was cleared by k_filter.
template <int D>
__global__ void __launch_bounds__(kRxThreads)
k_surv_sort_coop(Workspace ws) {
    constexpr int DP = padded_dims(D);
    __shared__ RadixShared s;
    WsHeader *h = ws.hdr;
    const long long M = h->n_surv;
    if (M <= kClusterSortMax) return;
    const int bits = surv_fine_bits(D);
    const long long stride = (long long)gridDim.x * kRxThreads;
    const long long gt = (long long)blockIdx.x * kRxThreads + threadIdx.x;
    unsigned long long kmn = ~0ull, kmx = 0ull;
    for (long long r = gt; r < M; r += stride) {
        uint32_t x[D];
        load_row<D>(ws.surv_rows, r, x);
        const unsigned long long k = morton<D>(x, h->slo, h->shi, bits);
        ws.keys[0][r] = k;
        ws.vals[0][r] = (uint32_t)r;
        kmn = k < kmn ? k : kmn;
        kmx = k > kmx ? k : kmx;
    }
    rx_key_range(kmn, kmx, h);
    if (!grid_barrier(h->bar, &h->status, &s.ok)) return;
    const int sel = rx_sort_coop(ws, M, surv_sort_passes(D), s);
    if (sel < 0) return;
    const uint32_t *vals = ws.vals[sel];
    // tiles: one warp per tile
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long T = (M + kTileRows - 1) / kTileRows;
    for (long long tile = (long long)blockIdx.x * kRxWarps + w; tile < T; tile += (long long)gridDim.x * kRxWarps) {
        const long long r = tile * kTileRows + lane;
        uint32_t x[DP];
        if (r < M) {
            const uint32_t j = vals[r];
            const uint4 *src = reinterpret_cast<const uint4 *>(ws.surv_rows + (long long)j * DP);
            const uint4 a = src[0];
            x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
            if (DP == 8) { const uint4 b = src[1]; x[4 % DP] = b.x; x[5 % DP] = b.y; x[6 % DP] = b.z; x[7 % DP] = b.w; }
            ws.perm[r] = ws.surv_orig[j];
        } else {
            #pragma unroll
            for (int q = 0; q < DP; q++) x[q] = kSentinel;
        }
        uint4 *dst = reinterpret_cast<uint4 *>(ws.cand + r * DP);
        dst[0] = make_uint4(x[0], x[1], x[2], x[3]);
        if (DP == 8) dst[1] = make_uint4(x[4 % DP], x[5 % DP], x[6 % DP], x[7 % DP]);
        #pragma unroll
        for (int q = 0; q < DP; q++) {
            uint32_t m = x[q];
            #pragma unroll
            for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_xor_sync(0xffffffffu, m, o));
            if (lane == 0) ws.tmin[tile * DP + q] = m;
        }
        const unsigned long long ms = warp_min_sum<D>(x, r < M);
        if (lane == 0) ws.tsum[tile] = ms;
    }
    if (!grid_barrier(h->bar, &h->status, &s.ok)) return;
    // super-tile minima: one thread per super-tile and attribute word
    const long long T2 = (T + 31) / 32;
    for (long long k = gt; k < T2 * DP; k += stride) {
        const long long sup = k / DP;
        const int q = (int)(k % DP);
        uint32_t m = kSentinel;
        for (long long t = sup * 32; t < min(T, sup * 32 + 32); t++) m = min(m, ws.tmin[t * DP + q]);
        ws.smin[sup * DP + q] = m;
    }
    for (long long sup = gt; sup < T2; sup += stride) {
        unsigned long long m = ~0ull;
        for (long long t = sup * 32; t < min(T, sup * 32 + 32); t++) m = min(m, ws.tsum[t]);
        ws.ssum[sup] = m;
    }
}

// Final filter over the survivors in spatial order: survivor x is a skyline
// tuple iff no survivor dominates it (Def. 1). A tile (32 rows) or super-tile
// (1024 rows) can hold a dominator only if its minimum is <= x in every
// attribute -- the grid-dominance pruning of Sec. 3.1 on tiles -- and if
// its smallest row sum is below x's sum (a dominator's sum is smaller). One warp per
// survivor: lanes test 32 super-tile minima, then the 32 tile minima of each
// possible super-tile, then the 32 rows of each possible tile, stopping at the
// first dominator. Sets skyflag[original row] and, with segcount, counts the
// skyline rows of each kCB-row segment.
template <int D>
__global__ void __launch_bounds__(kTriThreads)
k_final(const uint32_t *rows, const uint32_t *orig, const uint32_t *tmin, const uint32_t *smin,
        const unsigned long long *tsum, const unsigned long long *ssum, const WsHeader *h, uint32_t *skyflag,
        uint32_t *segcount) {
    const long long M = h->n_surv;
    const long long T = (M + kTileRows - 1) / kTileRows;
    const long long T2 = (T + 31) / 32;
    const int lane = threadIdx.x & 31;
    const long long wid = ((long long)blockIdx.x * kTriThreads + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * kTriThreads) >> 5;
    for (long long q = wid; q < M; q += nw) {
        uint32_t x[D];
        load_row<D>(rows, q, x);
        unsigned long long xsum = 0;
        #pragma unroll
        for (int i = 0; i < D; i++) xsum += x[i];
        bool dom = false;
        for (long long s0 = 0; s0 < T2 && !dom; s0 += 32) {
            bool maybe = false;
            if (s0 + lane < T2) {
                uint32_t m[D];
                load_row<D>(smin, s0 + lane, m);
                maybe = __ldg(ssum + s0 + lane) < xsum;
                #pragma unroll
                for (int i = 0; i < D; i++) maybe &= m[i] <= x[i];
            }
            unsigned supers = __ballot_sync(0xffffffffu, maybe);
            while (supers && !dom) {
                const long long sup = s0 + __ffs(supers) - 1;
                supers &= supers - 1;
                const long long tile = sup * 32 + lane;
                bool tmaybe = false;
                if (tile < T) {
                    uint32_t m[D];
                    load_row<D>(tmin, tile, m);
                    tmaybe = __ldg(tsum + tile) < xsum;
                    #pragma unroll
                    for (int i = 0; i < D; i++) tmaybe &= m[i] <= x[i];
                }
                unsigned tiles = __ballot_sync(0xffffffffu, tmaybe);
                while (tiles && !dom) {
                    const long long t = sup * 32 + __ffs(tiles) - 1;
                    tiles &= tiles - 1;
                    uint32_t sv[D];
                    load_row<D>(rows, t * kTileRows + lane, sv);
                    dom = __any_sync(0xffffffffu, dominates<D>(sv, x));
                }
            }
        }
        if (!dom && lane == 0) {
            const uint32_t o = orig[q];
            skyflag[o] = 1u;
            atomicAdd(&segcount[o / kCB], 1u);
        }
    }
}

// Skyline rows in ascending row order: row numbers, canonical rows, and the
// skyline's per-attribute range (lo / hi) for the partitioning; the sort-key
// range is cleared for the partition sort.
template <int D>
__global__ void __launch_bounds__(kCT)
k_compact_sky(const uint32_t *data, int dir, long long n, const uint32_t *skyflag,
              const uint32_t *blocksum, int64_t *sky_idx, uint32_t *sky_rows, WsHeader *h, long long nb) {
    __shared__ uint32_t blo[D], bhi[D];
    if (threadIdx.x < D) { blo[threadIdx.x] = 0xFFFFFFFFu; bhi[threadIdx.x] = 0u; }
    if (blockIdx.x == 0 && threadIdx.x == 0) { h->key_min = ~0ull; h->key_max = 0ull; }
    uint32_t lo[D], hi[D];
    #pragma unroll
    for (int q = 0; q < D; q++) { lo[q] = 0xFFFFFFFFu; hi[q] = 0u; }
    // segments without skyline rows have nothing to do (block 0 still writes S)
    if (blockIdx.x != 0 && blocksum[blockIdx.x] == 0u) return;
    // raw per-segment counts (from k_final): this block's offset is the sum of the
    // counts before it, S the sum of all
    uint32_t run;
    {
        uint32_t before = 0, all = 0;
        for (long long j = threadIdx.x; j < nb; j += kCT) {
            const uint32_t c = blocksum[j];
            before += j < (long long)blockIdx.x ? c : 0u;
            all += c;
        }
        uint32_t tb, ta;
        block_scan(before, &tb);
        block_scan(all, &ta);
        run = tb;
        if (blockIdx.x == 0 && threadIdx.x == 0) h->n_sky = ta;
    }
    // thread t reads the flags of rows [p0, p0 + kPer) (all loads at once); one scan of
    // the per-thread counts lists the block's skyline rows in order in shared memory,
    // then the block copies them, one row per thread
    __shared__ uint16_t lst[kCB];
    const long long b0 = (long long)blockIdx.x * kCB;
    const long long p0 = b0 + (long long)threadIdx.x * kPer;
    uint32_t f[kPer];
    if (p0 + kPer <= n && (reinterpret_cast<uintptr_t>(skyflag) & 15u) == 0) {
        const uint4 *fp = reinterpret_cast<const uint4 *>(skyflag + p0);
        #pragma unroll
        for (int k = 0; k < kPer / 4; k++) {
            const uint4 v = fp[k];
            f[4 * k] = v.x; f[4 * k + 1] = v.y; f[4 * k + 2] = v.z; f[4 * k + 3] = v.w;
        }
    } else {
        #pragma unroll
        for (int k = 0; k < kPer; k++) f[k] = p0 + k < n ? skyflag[p0 + k] : 0u;
    }
    uint32_t c = 0;
    #pragma unroll
    for (int k = 0; k < kPer; k++) c += f[k] ? 1u : 0u;
    uint32_t tot;
    uint32_t e = block_scan(c, &tot);
    #pragma unroll
    for (int k = 0; k < kPer; k++)
        if (f[k]) lst[e++] = (uint16_t)(threadIdx.x * kPer + k);
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < tot; j += kCT) {
        const long long p = b0 + lst[j];
        sky_idx[run + j] = p;
        uint32_t x[D];
        load_canon<D>(data, p, dir, x);
        store_row<D>(sky_rows, run + j, x);
        #pragma unroll
        for (int q = 0; q < D; q++) { lo[q] = min(lo[q], x[q]); hi[q] = max(hi[q], x[q]); }
    }
    #pragma unroll
    for (int q = 0; q < D; q++) {
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo[q] = min(lo[q], __shfl_xor_sync(0xffffffffu, lo[q], o));
            hi[q] = max(hi[q], __shfl_xor_sync(0xffffffffu, hi[q], o));
        }
        if ((threadIdx.x & 31) == 0 && lo[q] <= hi[q]) { atomicMin(&blo[q], lo[q]); atomicMax(&bhi[q], hi[q]); }
    }
    __syncthreads();
    if (threadIdx.x < D && blo[threadIdx.x] <= bhi[threadIdx.x]) {
        atomicMin(&h->lo[threadIdx.x], blo[threadIdx.x]);
        atomicMax(&h->hi[threadIdx.x], bhi[threadIdx.x]);
    }
}

// ---- the survivor sort as a single cluster launch ------------------------
// For inputs of at most kClusterSortMax rows the O(survivors) stages between
// the survivor compaction and the final check run as one cluster launch
// (cluster.cuh) instead of a chain of small kernels, computing exactly what
// the chain computes. The O(n) compactions stay grid-wide.

// The survivors' 16-bit Morton keys over their range, the stable sort by
// key, and the survivor tiles in that order (rows, original row numbers, tile
// and super-tile minima) -- the work of k_surv_keys, the radix sort and
// k_gather_tiles, for the M survivors k_filter listed.
template <int D>
__global__ void __launch_bounds__(kClThreads)
k_surv_cluster(Workspace ws) {
    constexpr int DP = padded_dims(D);
    extern __shared__ uint32_t sm[];
    __shared__ unsigned long long kr[2];
    __shared__ uint32_t wm[32][DP];
    __shared__ unsigned long long wsm[32];
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks(), r = (int)cl.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    WsHeader *h = ws.hdr;
    const long long M = h->n_surv;
    if (M > kClusterSortMax) return;   // k_surv_sort_coop sorts them (every CTA returns here)
    if (tid == 0) { kr[0] = ~0ull; kr[1] = 0ull; }
    __syncthreads();
    // this CTA's positions [b0, b0 + cnt) of the (key, survivor) pairs, in shared memory
    uint32_t *kb0 = sm + kClSortWords, *vb0 = kb0 + kClSmemCap, *kb1 = vb0 + kClSmemCap, *vb1 = kb1 + kClSmemCap;
    const long long c = cluster_chunk(M);
    const long long b0 = min(M, (long long)r * c);
    const int cnt = (int)(min(M, b0 + c) - b0);
    const int bits = 16 / D;
    unsigned long long kmn = ~0ull, kmx = 0ull;
    for (int i = tid; i < cnt; i += kClThreads) {
        uint32_t x[D];
        load_row<D>(ws.surv_rows, b0 + i, x);
        const uint32_t k = morton<D>(x, h->slo, h->shi, bits);
        kb0[i] = k;
        vb0[i] = (uint32_t)(b0 + i);
        kmn = k < kmn ? k : kmn;
        kmx = k > kmx ? k : kmx;
    }
    cta_key_add(kmn, kmx, kr);
    unsigned long long kmin, kmax;
    cluster_key_range(cl, kr, &kmin, &kmax);
    const int fin = cluster_radix_sort_smem(cl, sm, kb0, vb0, kb1, vb1, M, (uint32_t)kmin, key_passes(kmin, kmax), 0);
    // the sorted survivor numbers to global memory for the tile gather
    const uint32_t *vf = fin ? vb1 : vb0;
    for (int i = tid; i < cnt; i += kClThreads) ws.vals[0][b0 + i] = vf[i];
    cl.sync();
    const uint32_t *vals = ws.vals[0];
    // survivor tiles in key order: one super-tile per CTA and round, warp w builds its tile w
    const long long T = (M + kTileRows - 1) / kTileRows;
    const long long T2 = (T + 31) / 32;
    for (long long sup = r; sup < T2; sup += C) {
        const long long tile = sup * 32 + w;
        const long long row = tile * kTileRows + lane;
        uint32_t x[DP];
        if (row < M) {
            const uint32_t j = vals[row];
            const uint4 *src = reinterpret_cast<const uint4 *>(ws.surv_rows + (long long)j * DP);
            const uint4 a = src[0];
            x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
            if (DP == 8) { const uint4 b = src[1]; x[4 % DP] = b.x; x[5 % DP] = b.y; x[6 % DP] = b.z; x[7 % DP] = b.w; }
            ws.perm[row] = ws.surv_orig[j];
        } else {
            #pragma unroll
            for (int q = 0; q < DP; q++) x[q] = kSentinel;
        }
        if (tile < T) {
            uint4 *dst = reinterpret_cast<uint4 *>(ws.cand + row * DP);
            dst[0] = make_uint4(x[0], x[1], x[2], x[3]);
            if (DP == 8) dst[1] = make_uint4(x[4 % DP], x[5 % DP], x[6 % DP], x[7 % DP]);
        }
        #pragma unroll
        for (int q = 0; q < DP; q++) {
            uint32_t m = x[q];
            #pragma unroll
            for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_xor_sync(0xffffffffu, m, o));
            if (lane == 0) {
                wm[w][q] = m;
                if (tile < T) ws.tmin[tile * DP + q] = m;
            }
        }
        const unsigned long long ms = warp_min_sum<D>(x, row < M);
        if (lane == 0) {
            wsm[w] = ms;
            if (tile < T) ws.tsum[tile] = ms;
        }
        __syncthreads();
        if (w == 0) {
            #pragma unroll
            for (int q = 0; q < DP; q++) {
                uint32_t m = wm[lane][q];
                #pragma unroll
                for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_xor_sync(0xffffffffu, m, o));
                if (lane == 0) ws.smin[sup * DP + q] = m;
            }
            unsigned long long m = wsm[lane];
            #pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long y = __shfl_xor_sync(0xffffffffu, m, o);
                m = y < m ? y : m;
            }
            if (lane == 0) ws.ssum[sup] = m;
        }
        __syncthreads();
    }
    if (r == 0 && tid == 0) h->sorted_sel = 0u;
    cl.sync();   // no CTA leaves while another may still read its shared memory
}

template <int D>
cudaError_t skyline_d(const uint32_t *d_data, int64_t n, int dir, int reps, Workspace &ws,
                      int64_t *d_sky_idx, cudaStream_t st, bool gres_reps) {
    const long long nb = (n + kCB - 1) / kCB;
    cudaError_t e = cudaSuccess;   // the selection histograms were zeroed with the header
    const int hb = (int)std::min<long long>((n + 1023) / 1024, 152LL * 2);
    k_keys<D><<<hb, 1024, 0, st>>>(d_data, n, dir, ws.keys[0], ws.hdr, ws.sel_hist, reps); note_launch();
    k_sel_l2<D><<<hb, kMaxReps, 0, st>>>(ws.keys[0], n, ws.hdr, ws.sel_hist + kSelBuckets, reps, ws.keys[1],
                                         ws.rep_idx, d_data, dir, ws.reps, ws.blocksum, nb,
                                         gres_reps ? ws.greps : nullptr, ws.kill); note_launch();
    static int filter_blocks = 0;   // resident blocks of k_filter<D> on this GPU
    if (filter_blocks == 0) {
        int per_sm = 0, dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_filter<D>, kFilterThreads, 0);
        filter_blocks = std::max(1, per_sm) * std::max(1, sms);
    }
    const long long fchunks = (n + kFilterChunk - 1) / kFilterChunk;
    const int fb = (int)std::min<long long>(fchunks, (long long)filter_blocks);
    const int pb = (int)std::min<long long>((n + kPreChunk - 1) / kPreChunk, 152LL * 8);
    k_prefilter<D><<<pb, kPreThreads, 0, st>>>(d_data, dir, n, ws.kill, ws.hdr, ws.flags, ws.vals[1]); note_launch();
    k_filter<D><<<fb, kFilterThreads, 0, st>>>(d_data, dir, ws.vals[1], ws.reps, ws.hdr, ws.flags, ws.surv_rows,
                                               ws.surv_orig);
    note_launch();
    // The survivor sort: in one cluster up to kClusterSortMax survivors, else with the
    // cooperative kernel. The survivor count is known on the device only, so above
    // that many input rows both are queued and each returns at once for the other size.
    static bool configured = false;
    e = launch_cluster(k_surv_cluster<D>, kClSmemBytes, &configured, st, ws);
    if (e != cudaSuccess) return e;
    if (n > kClusterSortMax) {
        static int coop = 0;
        if (!coop && (e = coop_blocks(k_surv_sort_coop<D>, &coop)) != cudaSuccess) return e;
        e = launch_coop(k_surv_sort_coop<D>, coop, st, ws);
        if (e != cudaSuccess) return e;
    }
    k_final<D><<<(unsigned)std::min<int64_t>((n + 7) / 8, 152LL * 16), kTriThreads, 0, st>>>(
        ws.cand, ws.perm, ws.tmin, ws.smin, ws.tsum, ws.ssum, ws.hdr, ws.flags, ws.blocksum); note_launch();
    k_compact_sky<D><<<(unsigned)nb, kCT, 0, st>>>(d_data, dir, n, ws.flags, ws.blocksum, d_sky_idx,
                                                    ws.sky_rows, ws.hdr, nb); note_launch();
    return cudaGetLastError();
}

}  // namespace

int64_t scan_blocks(int64_t n) { return (n + kCB - 1) / kCB; }

cudaError_t launch_init(Workspace &ws, int64_t n, cudaStream_t st) {
    k_init<<<1, 256, 0, st>>>(ws.hdr, (long long)n, ws.sel_hist); note_launch();
    return cudaGetLastError();
}

cudaError_t launch_skyline(const uint32_t *d_data, int64_t n, int d, int dir, int reps,
                           Workspace &ws, int64_t *d_sky_idx, cudaStream_t st, bool gres_reps) {
    if (n == 0) return cudaSuccess;
    switch (d) {
        case 1: return skyline_d<1>(d_data, n, dir, reps, ws, d_sky_idx, st, gres_reps);
        case 2: return skyline_d<2>(d_data, n, dir, reps, ws, d_sky_idx, st, gres_reps);
        case 3: return skyline_d<3>(d_data, n, dir, reps, ws, d_sky_idx, st, gres_reps);
        case 4: return skyline_d<4>(d_data, n, dir, reps, ws, d_sky_idx, st, gres_reps);
        case 5: return skyline_d<5>(d_data, n, dir, reps, ws, d_sky_idx, st, gres_reps);
        case 6: return skyline_d<6>(d_data, n, dir, reps, ws, d_sky_idx, st, gres_reps);
        case 7: return skyline_d<7>(d_data, n, dir, reps, ws, d_sky_idx, st, gres_reps);
        case 8: return skyline_d<8>(d_data, n, dir, reps, ws, d_sky_idx, st, gres_reps);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gres
