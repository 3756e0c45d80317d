// gres_internal.cuh -- shared declarations of libgres (device helpers, workspace
// layout, kernel launchers). Not part of the public ABI (see include/gres.h).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/gres.h"

namespace gres {

constexpr int kMaxD = 8;
constexpr int kTileRows = 32;          // candidate rows per pruning tile
constexpr int kMaxReps = 1024;         // skyline pre-filter representatives
constexpr int kKillers = 32;           // representatives of the first, one-row-per-thread filter pass
constexpr uint32_t kSentinel = 0xFFFFFFFFu;  // padding row value: never dominates

// Rows of canonical values are stored padded to DP words (16-byte multiples).
__host__ __device__ constexpr int padded_dims(int d) { return d <= 4 ? 4 : 8; }

// Status bits written by kernels into the workspace header.
enum : uint32_t {
    kStatusTimeout = 1u,   // a bounded device-side wait ran out
    kStatusInternal = 2u,  // an internal capacity or consistency check failed
};

// ---------------------------------------------------------------------------
// Workspace: one caller-owned device buffer, carved into 256-byte aligned
// regions. The header holds device-side sizes so that nothing after the input
// size needs the host (the whole call can be captured into a CUDA graph).
struct WsHeader {
    unsigned long long key_min;   // key range of the current sort
    unsigned long long key_max;
    long long n_rows;             // input rows n
    long long n_surv;             // rows left after the representative filter
    long long n_sky;              // skyline size S
    long long n_reps;             // representatives kept (mutually non-dominated)
    long long n_cand;             // representative candidates (smallest keys)
    unsigned int sel_b1;          // level-1 selection bucket
    unsigned int sel_below;       // rows under bucket sel_b1
    unsigned int work_next;       // dynamic work counter of the gres kernel
    unsigned int status;          // kStatus* bits
    unsigned int sorted_sel;      // buffer (0/1) holding the last radix sort's result
    unsigned int done[4];         // block tickets of the last-block-done fusions
    unsigned int lo[kMaxD];       // per-attribute canonical minimum over the skyline
    unsigned int hi[kMaxD];       // per-attribute canonical maximum over the skyline
    unsigned int slo[kMaxD];      // per-attribute canonical minimum over the survivors
    unsigned int shi[kMaxD];      // per-attribute canonical maximum over the survivors
    unsigned int n_bnd;           // rows in the selection's boundary bucket
    unsigned int n_alive;         // rows left by the one-row-per-thread filter pass
    unsigned int dlo[kMaxD];      // per-attribute canonical minimum over all rows
    unsigned int dhi[kMaxD];      // per-attribute canonical maximum over all rows
    unsigned int bar[2];          // grid-wide barrier of the cooperative sorts: arrivals, generation
};

// Digit passes that do work in the radix sort of the current key range; the
// sorted data is in buffer (passes & 1), recorded in sorted_sel once the
// sort is done.
__device__ __forceinline__ int radix_passes(const WsHeader *h) {
    unsigned long long range = h->key_max >= h->key_min ? h->key_max - h->key_min : 0ull;
    int bits = range ? 64 - __clzll((long long)range) : 0;
    return (bits + 7) >> 3;
}

struct Workspace {
    WsHeader *hdr;
    unsigned long long *keys[2];  // radix sort key ping-pong, n each
    uint32_t *vals[2];            // radix sort value ping-pong, n each
    uint32_t *hist;               // 256 * sort_blocks(n)
    uint32_t *dtot;               // 256 digit totals of the current pass
    uint32_t *blocksum;           // skyline rows per kCB-row segment of the input (compaction offsets)
    uint32_t *flags;              // n
    uint32_t *surv_rows;          // n * DP canonical rows, sum order
    uint32_t *surv_orig;          // n original row numbers, sum order
    uint32_t *reps;               // kMaxReps * DP
    uint32_t *sel_hist;           // kSelHistWords selection histogram counters (zeroed with the header)
    uint32_t *rep_idx;            // kMaxReps representative candidate rows
    uint32_t *sky_rows;           // (n + tile) * DP canonical rows, skyline order
    uint32_t *cand;               // (n + tile) * DP canonical rows, partition order
    uint32_t *tmin;               // tiles * DP per-tile minima
    uint32_t *smin;               // super-tiles (1024 rows) * DP minima
    unsigned long long *tsum;     // per survivor tile: its smallest row sum (sentinel tiles: ~0)
    unsigned long long *ssum;     // per survivor super-tile: its smallest row sum
    uint32_t *perm;               // n: partition position -> skyline position
    int32_t *res;                 // n: per partition position, a bound on the result (GRES_FLAG_GRES_REPS)
    uint32_t *greps;              // 32 * DP: the gres-stage representatives (GRES_FLAG_GRES_REPS)
    uint32_t *kill;               // kKillers * DP: the first filter pass's representatives
    uint32_t *pid;                // n + tile: partition number per partition position (GRES_FLAG_COUNT_PARTS)
    uint32_t *steps;              // K widths
    uint32_t *magic;              // K * 4 multiply-high constants (m, s1, s2, delta)
    size_t bytes;
};

int64_t sort_blocks(int64_t n);
int64_t scan_blocks(int64_t n);
size_t workspace_layout(int64_t n, int d, int k, void *base, Workspace *ws);

// Counters of the representative selection's two histogram levels (4,096 each).
constexpr int kSelHistWords = 2 * 4096;

// Zeroes the selection histograms (one thread block); done by the kernel that
// resets the header, so no separate memset precedes the skyline pass.
__device__ __forceinline__ void clear_sel_hist(uint32_t *sel) {
    if (sel)
        for (int i = threadIdx.x; i < kSelHistWords; i += blockDim.x) sel[i] = 0u;
}

// Resets the per-call header fields (one thread block, >= 32 threads).
__device__ __forceinline__ void init_header(WsHeader *h, long long n) {
    if (threadIdx.x == 0) {
        h->key_min = ~0ull;
        h->key_max = 0ull;
        h->n_rows = n;
        h->n_surv = 0;
        h->n_sky = 0;
        h->n_reps = 0;
        h->n_cand = 0;
        h->n_bnd = 0;
        h->n_alive = 0;
        h->bar[0] = 0;
        h->work_next = 0;
        h->status = 0;
        h->sorted_sel = 0;
    }
    if (threadIdx.x < 4) h->done[threadIdx.x] = 0;
    if (threadIdx.x < kMaxD) {
        h->lo[threadIdx.x] = 0xFFFFFFFFu;
        h->hi[threadIdx.x] = 0u;
        h->slo[threadIdx.x] = 0xFFFFFFFFu;
        h->shi[threadIdx.x] = 0u;
        h->dlo[threadIdx.x] = 0xFFFFFFFFu;
        h->dhi[threadIdx.x] = 0u;
    }
}

// Last-block-done: every block calls this once at its end (all threads); it
// returns true in exactly one block, the last to arrive, after which the
// writes of every other block are visible to it. The ticket is reset for the
// next launch. No block waits on another.
__device__ __forceinline__ bool last_block_done(unsigned int *ticket) {
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned t = atomicAdd(ticket, 1u);
        last = t == gridDim.x * gridDim.y * gridDim.z - 1;
        if (last) *ticket = 0;
    }
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// Exclusive scan of a[0 .. count) in place by one block (blockDim.x a
// multiple of 32, <= 1024); returns the total (in every thread).
__device__ __forceinline__ uint32_t block_scan_inplace(uint32_t *a, long long count) {
    __shared__ uint32_t wsum[32];
    const int nt = blockDim.x;
    const long long chunk = (count + nt - 1) / nt;
    const long long c0 = (long long)threadIdx.x * chunk;
    const long long c1 = c0 + chunk < count ? c0 + chunk : count;
    uint32_t local = 0;
    for (long long i = c0; i < c1; i++) local += a[i];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t incl = local;
    #pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    uint32_t before = 0, all = 0;
    for (int j = 0; j < (nt >> 5); j++) {
        before += j < w ? wsum[j] : 0u;
        all += wsum[j];
    }
    uint32_t run = before + incl - local;
    for (long long i = c0; i < c1; i++) {
        const uint32_t c = a[i];
        a[i] = run;
        run += c;
    }
    __syncthreads();
    return all;
}

// Granlund & Montgomery (1994), unsigned division by a run-time invariant
// divisor (their Fig. 4.1): with l = ceil(log2 delta),
// m = floor(2^32 (2^l - delta) / delta) + 1, s1 = min(l, 1), s2 = max(l - 1, 0),
// floor(v / delta) = (t + ((v - t) >> s1)) >> s2 where t = mulhi(m, v).
void udiv_magic(uint32_t delta, uint32_t *m, uint32_t *s1, uint32_t *s2);

__device__ __forceinline__ uint32_t udiv(uint32_t v, uint32_t m, uint32_t s1, uint32_t s2) {
    uint32_t t = __umulhi(m, v);
    return (t + ((v - t) >> s1)) >> s2;
}

// Canonical value: smaller is better after this map (GRES_MAX reads ~v).
__device__ __forceinline__ uint32_t canon(uint32_t v, int dir) { return dir ? ~v : v; }

// Sets the calling thread's gres_last_error() message; returns s.
gres_status set_error(gres_status s, const char *msg);

// Counts kernel launches queued by the library (gres_launch_count()).
void note_launch();

// Optional per-stage timing with CUDA events on the launching stream
// (gres_timing_enable / gres_timing_read). Stage ids:
enum Stage { kStageSkyline = 0, kStagePartition = 1, kStageDominance = 2, kStageCount = 3 };
void stage_begin(int stage, cudaStream_t st);
void stage_end(int stage, cudaStream_t st);

// One gres query on one prepared candidate set.
struct DomQuery {
    const uint32_t *cand;     // T*32 rows, DP words each (partition order, sentinel-padded)
    const uint32_t *tmin;     // T rows, DP words each
    const uint32_t *smin;     // ceil(T / 32) super-tile rows, DP words each
    const uint32_t *perm;     // partition position -> skyline position
    const long long *n_sky;   // S (device)
    const uint32_t *magic;    // K * 4: (m, s1, s2, delta)
    const uint32_t *steps;    // K widths
    int32_t *out;             // result per skyline position
    int K;
    int dir;
    // Target range (resident datasets): when iperm is set, the targets are the
    // skyline positions t0 .. t0 + tn - 1 (iperm: skyline -> partition
    // position) and the result of position j goes to out[j - t0].
    const uint32_t *iperm = nullptr;
    unsigned t0 = 0, tn = 0;
    // Grid parameter mode (the paper's g): 0 = integer widths; B = steps are
    // intervals g over values read as v / 2^B, projection floor(v g / 2^B)
    // (magic holds g's division constants, steps the pruning widths).
    int gbits = 0;
    // Optional bound per partition position (GRES_FLAG_GRES_REPS): a step at
    // which the target is known to leave; the search looks only below it.
    const int32_t *ub = nullptr;
};

// Optional per-partition counts of one query (GRES_FLAG_COUNT_PARTS): the
// partition number of every partition position (padding positions: ~0) and
// the counters (see include/gres.h), indexed from pcnt[2].
struct PartCount {
    const uint32_t *pid = nullptr;
    unsigned long long *pcnt = nullptr;
    unsigned nparts = 0;      // partitions: targets of a larger number are not counted
};

// Division constants to make on the device for one query (k_make_magic).
struct MagicJob {
    const uint32_t *steps;
    uint32_t *magic;
    int K;
    unsigned *zero;           // a counter to clear (may be null)
};
// ---- kernel launchers (each queues on `st`, returns the launch error) -------
cudaError_t launch_init(Workspace &ws, int64_t n, cudaStream_t st);
// Uploads the widths and their division constants and resets the header.
cudaError_t launch_init_steps(Workspace &ws, int64_t n, const uint32_t *h_steps, int k, cudaStream_t st,
                              int gbits = 0);
// Survivor sets and skylines of at most kClusterSortMax rows are sorted inside
// one thread-block cluster per sort (cluster.cuh); larger ones in one
// cooperative launch (radix.cuh). The counts are known on the device only: for
// inputs above kClusterSortMax rows both are queued and each returns at once
// when the count is not its size.
constexpr int64_t kClusterSortMax = 131072;
cudaError_t launch_skyline(const uint32_t *d_data, int64_t n, int d, int dir, int reps,
                           Workspace &ws, int64_t *d_sky_idx, cudaStream_t st, bool gres_reps = false);
cudaError_t launch_gres_stage(const uint32_t *d_data, int64_t n, int d, int dir, int k,
                              const gres_plan_cfg &cfg, Workspace &ws,
                              const int64_t *d_sky_idx, int32_t *d_step_idx,
                              unsigned long long *d_tests, cudaStream_t st, int gbits = 0);
// Per target, the first step at which one of the 32 gres-stage representatives
// (ws.greps) dominates, into ws.res (GRES_FLAG_GRES_REPS); after the partitioning.
cudaError_t launch_rep_bound(int d, int64_t n, Workspace &ws, int k, int dir, int gbits,
                             unsigned long long *tests, cudaStream_t st);
// Partitions of a checked plan for d attributes (GRID m^d, ANGULAR m^(d-1),
// SLICED p, NONE 1).
int64_t plan_partitions(const gres_plan_cfg &cfg, int d);
// The candidate partitioning of the skyline in ws (cand, tmin, perm).
cudaError_t launch_partition(int d, const gres_plan_cfg &cfg, int64_t n, Workspace &ws, cudaStream_t st);
// The caller's rows as the candidate set (canonical padded rows into
// sky_rows, their range into lo/hi, S = n), for gres_partition.
cudaError_t launch_load_candidates(const uint32_t *d_rows, int64_t n, int d, int dir, Workspace &ws,
                                   cudaStream_t st);
// Partition numbers by row, the tile order and the tile minima (d words per
// tile) after launch_partition.
cudaError_t launch_partition_out(int d, const gres_plan_cfg &cfg, int64_t n, Workspace &ws, int64_t *d_part,
                                 uint32_t *d_order, uint32_t *d_tile_min, cudaStream_t st);
// The grid-dominance kernel for one query; *counter must be 0.
cudaError_t launch_dominance(int d, int slots, const DomQuery &q, unsigned *counter,
                             unsigned long long *tests, cudaStream_t st, const PartCount &pc = PartCount());
// One launch for up to 256 queries of the same d; *counter must be 0.
cudaError_t launch_dominance_batch(int d, int slots, const DomQuery *qs, int count, unsigned *counter,
                                   cudaStream_t st);
// iperm[perm[i]] = i for i < S (the inverse of a dataset's tile order).
cudaError_t launch_invert_perm(const uint32_t *perm, int64_t S, uint32_t *iperm, cudaStream_t st);
// Device-side division constants (and counter resets) for many queries.
cudaError_t launch_make_magic(const MagicJob *jobs, int count, cudaStream_t st);
// Widths from the host into d_steps / d_magic; zeroes *zero when given.
cudaError_t launch_upload_steps(uint32_t *d_steps, uint32_t *d_magic, unsigned *zero, const uint32_t *h_steps,
                                int k, cudaStream_t st);
cudaError_t launch_gproj(const uint32_t *d_values, int64_t count, const uint32_t *h_steps, int k,
                         uint32_t *d_out, cudaStream_t st);
// The dominance-test peak probe (probe.cu); *lane_ops = its compare lane-ops.
cudaError_t launch_test_peak(int d, int iters, int blocks, unsigned long long *sink, cudaStream_t st,
                             double *lane_ops);

}  // namespace gres

// A prepared dataset: the skyline and the candidate tiles, on the device
// (gres_dataset_create). One device allocation holds every array.
struct gres_dataset {
    int device;
    int64_t n;
    int32_t d;
    int32_t dir;
    int32_t slots;
    int64_t S;
    void *mem;
    size_t bytes;
    int64_t *sky_idx;     // S: skyline rows, ascending
    uint32_t *perm;       // S: partition position -> skyline position
    uint32_t *iperm;      // S: skyline position -> partition position
    uint32_t *cand;       // T*32 rows of DP words (partition order, sentinel-padded)
    uint32_t *tmin;       // T rows of DP words
    uint32_t *smin;       // ceil(T / 32) rows of DP words
    long long *n_sky;     // S on the device
};
