/*
 * gres.h -- C ABI of libgres: skyline and grid resistance (gres) on one GPU.
 *
 * What is computed (Martinenghi, "Parallelizing the Computation of Robustness
 * for Measuring the Strength of Tuples"):
 *   - dominance and the skyline Sky(r):  Def. 1 (Sec. 2);
 *   - the grid projection gproj(t, g), the lowest corner of the grid cell
 *     holding t:                          Sec. 2;
 *   - grid resistance gres(t; r), the finest grid at which gproj(t) leaves
 *     the skyline of gproj(r); 1 if it never leaves: Def. 2 (Sec. 2) and
 *     Algorithm 1 (Sec. 3.2); gres depends on skyline tuples only (its
 *     stability, Sec. 3.2), so candidates are the skyline;
 *   - Grid / Angular / Sliced partitioning:  Sec. 3.1 (used here to group
 *     candidate tuples into tiles that can be skipped; speed only).
 *
 * Fixed point. A relation r is n rows of d attributes, uint32, row-major
 * (row i at data[i*d .. i*d+d-1]); a value v stands for the real v / 2^B.
 * A grid is given by its integer cell width delta: a value projects to
 * floor(v / delta). The paper's g intervals on [0,1) are the width
 * delta = 2^B / g. A step list is K strictly ascending widths
 * delta_0 < ... < delta_{K-1} (finest grid first, i.e. the paper's scan
 * g = g_bar, ..., 2). The result for a skyline tuple is the index k of the
 * first width at which some tuple's projection dominates its projection, or
 * K when that never happens (the paper's gres = 1). The paper's value is
 * delta_k / 2^B (k < K) or 1 (k = K).
 *
 * Direction: GRES_MIN = smaller is better (the paper's convention); GRES_MAX
 * = larger is better (the opposite convention the paper allows). With
 * GRES_MAX the projection is still floor(v / delta); only comparisons flip.
 *
 * Conventions for every call:
 *   - Ownership: the caller owns every buffer (host or device). The library
 *     allocates no device memory in these calls; scratch space comes from the
 *     caller through (d_ws, ws_bytes), sized by gres_workspace_size(). The
 *     server object (gres_serve_*) owns the device memory it was given a
 *     budget for and frees it in gres_serve_destroy().
 *   - Streams: work is queued on the caller's CUDA stream (cudaStream_t
 *     passed as void*; NULL = legacy default stream). A call returns after
 *     queueing unless it writes a host count (h_sky_count != NULL), in which
 *     case it waits for the stream.
 *   - Results: skyline indices are original row numbers in ascending order;
 *     d_step_idx[j] is the result of row d_sky_idx[j].
 *   - Errors: every call returns a gres_status; no C++ exception crosses the
 *     ABI. gres_last_error() returns a message for the calling thread's last
 *     failure. GRES_EINVAL: a bad argument (nothing is launched).
 *     GRES_ECUDA: a CUDA launch or copy failed (the message has the CUDA
 *     error string). GRES_ETIMEOUT: a bounded device-side wait ran out.
 *   - Limits: 1 <= d <= 8, 0 <= n < 2^31, 1 <= K <= 2^20.
 */
#ifndef GRES_H
#define GRES_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GRES_OK = 0,
    GRES_EINVAL = 1,
    GRES_ENOMEM = 2,
    GRES_EAGAIN = 3,
    GRES_ETIMEOUT = 4,
    GRES_ECUDA = 5,
    GRES_EINTERNAL = 6
} gres_status;

typedef enum { GRES_MIN = 0, GRES_MAX = 1 } gres_dir;

/* Candidate grouping for tile skipping (Sec. 3.1). Results never depend on it. */
typedef enum {
    GRES_PART_NONE = 0,     /* skyline order as found (ascending row index)            */
    GRES_PART_GRID = 1,     /* m slices per attribute, p = m^d cells                  */
    GRES_PART_ANGULAR = 2,  /* m slices per hyperspherical angle, p = m^(d-1) (Eq. 1)  */
    GRES_PART_SLICED = 3    /* p equal slices of the order on one attribute            */
} gres_part;

/* Plan for gres_compute. A NULL plan (or zero fields) means: GRID with m
 * chosen so that m^d is about 256 cells, 1024 representatives, 8 slots. */
typedef struct {
    int32_t scheme;       /* gres_part                                                  */
    int32_t m;            /* GRID / ANGULAR slices per dimension (0: auto)              */
    int32_t p;            /* SLICED partitions (0: auto = 64)                           */
    int32_t slice_dim;    /* SLICED attribute (0 .. d-1)                                */
    int32_t reps;         /* skyline pre-filter representatives, 1..1024 (0: 1024)      */
    int32_t slots;        /* gres kernel step slots per lane: 4 or 8 (0: 8)             */
    int32_t flags;        /* GRES_FLAG_*                                                */
    int32_t reserved;     /* must be 0                                                  */
} gres_plan_cfg;

/* Count the dominance tests and pruning checks the gres kernel evaluates into
 * d_tests (see gres_compute). For accounting only. */
#define GRES_FLAG_COUNT_TESTS 1
/* Representative Filtering in the gres stage (Sec. 3.1, applied to gres; the
 * paper reports it of little use there): before its search, every skyline
 * tuple is tested at every step against the 32 rows of smallest f (sum of the
 * values; by stability any rows of r may serve as candidates), and the first
 * step at which one of them dominates bounds the search. Results are
 * unchanged. Honoured by gres_compute, gres_compute_g and gres_batch
 * (rejected by the dataset and server calls). With GRES_FLAG_COUNT_TESTS the
 * representative tests are counted in d_tests[0] too. */
#define GRES_FLAG_GRES_REPS 2
/* The paper's accounting of dominance tests by phase (Sec. 4: the parallel
 * phase costs what its heaviest partition costs, the final phase what it
 * tests across partitions), on this kernel's search: with this flag (and
 * GRES_FLAG_COUNT_TESTS) d_tests holds 2 + 4 * P uint64, P =
 * gres_plan_partitions(cfg, d), and for every target tuple in partition p the
 * kernel adds to d_tests[2 + 4p + 0] its lane-tests against candidates of
 * partition p, [+1] its row checks (one per candidate row looked at, per lane)
 * of candidates of partition p, [+2] and [+3] the same against candidates of
 * other partitions (padding rows of the last tile count there). Tile and
 * super-tile bounding-box checks are not split: they stay in d_tests[1] only.
 * Local work of a partition runs in parallel with the other partitions'; the
 * cross-partition work is what the paper's final phase does. Honoured by
 * gres_compute and gres_compute_g only (with GRES_FLAG_GRES_REPS the
 * representative tests are not split either). */
#define GRES_FLAG_COUNT_PARTS 4

/* The number of partitions P of a plan for d attributes (after the defaults of
 * gres_plan_cfg are applied): m^d for GRID, m^(d-1) for ANGULAR, p for SLICED,
 * 1 for NONE -- the size of the per-partition counts of GRES_FLAG_COUNT_PARTS.
 * cfg may be NULL (the default plan). GRES_EINVAL for a bad plan or d. */
gres_status gres_plan_partitions(const gres_plan_cfg *cfg, int32_t d, int64_t *out);

/* Thread-local message for the calling thread's most recent failed call
 * ("" if none). The pointer stays valid until the next call on that thread. */
const char *gres_last_error(void);

/* Library version string. */
const char *gres_version(void);

/* Bytes of device scratch that sky_compute / gres_compute need for n rows of
 * d attributes and K steps. Writes *bytes. GRES_EINVAL for out-of-range
 * arguments. Pure host computation. */
gres_status gres_workspace_size(int64_t n, int32_t d, int32_t k, size_t *bytes);

/* Skyline of r (Def. 1) by a sort-by-sum pass with block dominance filters.
 *   d_data       device, n*d uint32, row-major (read only)
 *   dir          gres_dir
 *   d_ws         device scratch, >= gres_workspace_size(n, d, 1) bytes,
 *                256-byte aligned
 *   d_sky_idx    device, capacity n int64: skyline row numbers, ascending
 *   d_sky_count  device int64 (may be NULL): the skyline size S
 *   h_sky_count  host int64 (may be NULL): S; waits for the stream
 * Duplicated rows do not dominate each other: all copies of a skyline row
 * are in the skyline. */
gres_status sky_compute(const uint32_t *d_data, int64_t n, int32_t d, int32_t dir,
                        void *d_ws, size_t ws_bytes,
                        int64_t *d_sky_idx, int64_t *d_sky_count, int64_t *h_sky_count,
                        void *stream);

/* Grid resistance of every skyline tuple (Def. 2, Algorithm 1): the skyline
 * (as sky_compute), then for each skyline tuple t the first step k at which
 * some skyline tuple's projection dominates t's projection.
 *   h_steps      host, k uint32 widths, strictly ascending, >= 1
 *   cfg          plan (may be NULL); see gres_plan_cfg
 *   d_ws         device scratch, >= gres_workspace_size(n, d, k) bytes
 *   d_sky_idx    device, capacity n int64: skyline rows, ascending
 *   d_step_idx   device, capacity n int32: result per skyline row, in [0, k]
 *   d_sky_count  device int64 (may be NULL): S
 *   h_sky_count  host int64 (may be NULL): S; waits for the stream
 *   d_tests      device uint64[2] (may be NULL): with GRES_FLAG_COUNT_TESTS,
 *                [0] += (candidate, step) tests evaluated by the grid-dominance
 *                kernel, counted per lane (32 per warp-wide test of one
 *                candidate row at 32 steps), [1] += pruning checks (one per
 *                tile bounding box or candidate row looked at, per lane)
 * With h_sky_count == NULL nothing waits on the host, so the call can be
 * captured into a CUDA graph (all sizes after the skyline live on the device). */
gres_status gres_compute(const uint32_t *d_data, int64_t n, int32_t d, int32_t dir,
                         const uint32_t *h_steps, int32_t k, const gres_plan_cfg *cfg,
                         void *d_ws, size_t ws_bytes,
                         int64_t *d_sky_idx, int32_t *d_step_idx,
                         int64_t *d_sky_count, int64_t *h_sky_count,
                         unsigned long long *d_tests, void *stream);

/* Host-buffer form of gres_compute: copies h_data to the device, computes,
 * and copies the S results back, then waits; later work on `stream` is
 * ordered after it.
 *   h_data       host, n*d uint32 row-major (pinned memory copies faster)
 *   d_ws         device scratch, >= gres_workspace_size_host(n, d, k) bytes
 *   h_sky_idx    host, capacity n int64
 *   h_step_idx   host, capacity n int32
 *   h_sky_count  host int64 (required)
 * With pinned h_data the calling thread keeps up to 4 captured CUDA graphs,
 * keyed by (h_data, n, d, dir, widths, plan, d_ws, h_sky_idx, h_step_idx,
 * device). A call matching one replays it on a library stream: one graph
 * launch instead of a dozen kernel launches. The replay reads h_data's
 * current contents. If h_sky_idx and h_step_idx are pinned too, the graph
 * also copies the first S0 results back, S0 being the skyline size of the
 * call that captured it: a replay with S <= S0 then waits once, and one with
 * S > S0 copies the rest and waits again. Positions S .. S0-1 of the result
 * buffers (inside their capacity n) may then be overwritten with stale values.
 * Kernels replayed this way are counted once by gres_launch_count, at
 * capture. */
gres_status gres_workspace_size_host(int64_t n, int32_t d, int32_t k, size_t *bytes);
gres_status gres_compute_host(const uint32_t *h_data, int64_t n, int32_t d, int32_t dir,
                              const uint32_t *h_steps, int32_t k, const gres_plan_cfg *cfg,
                              void *d_ws, size_t ws_bytes,
                              int64_t *h_sky_idx, int32_t *h_step_idx, int64_t *h_sky_count,
                              void *stream);

/* ---- resident datasets and repeated queries --------------------------------
 * The skyline and its candidate tiles depend only on the data (Def. 1; gres
 * is stable, Sec. 3.2), so a dataset prepared once answers any number of gres
 * queries, each with its own step list, with the grid-dominance kernel alone. */
typedef struct gres_dataset gres_dataset;

/* Prepares `data` (n*d uint32 row-major; on the host when data_on_host != 0,
 * else on the device) with plan `cfg` (may be NULL): computes the skyline and
 * the candidate tiles on `stream`, waits for them, and keeps them in device
 * memory owned by the handle (gres_dataset_info reports its size). Until
 * gres_dataset_destroy the input may be freed. GRES_ENOMEM if the device
 * memory runs out. */
gres_status gres_dataset_create(const uint32_t *data, int64_t n, int32_t d, int32_t dir,
                                const gres_plan_cfg *cfg, int32_t data_on_host, void *stream,
                                gres_dataset **out);
gres_status gres_dataset_destroy(gres_dataset *ds);
/* n, d, skyline size S and the handle's device bytes (any output may be NULL). */
gres_status gres_dataset_info(const gres_dataset *ds, int64_t *n, int32_t *d, int64_t *sky_count,
                              size_t *device_bytes);
/* The S skyline row numbers (ascending) into `out` (host if out_on_host, waits). */
gres_status gres_dataset_sky_idx(const gres_dataset *ds, int64_t *out, int32_t out_on_host, void *stream);

/* Device scratch bytes of one query with k widths. */
gres_status gres_query_workspace_size(int32_t k, size_t *bytes);
/* gres of every skyline tuple of a prepared dataset for the widths h_steps
 * (host, k, strictly ascending, >= 1): d_step_idx[j] (device, S int32) is the
 * result of skyline row j (same order as gres_dataset_sky_idx). d_qws: device
 * scratch of gres_query_workspace_size(k) bytes, 256-byte aligned; queries
 * that overlap on the GPU need distinct scratch. Queues on `stream`. */
gres_status gres_query(const gres_dataset *ds, const uint32_t *h_steps, int32_t k, void *d_qws,
                       size_t qws_bytes, int32_t *d_step_idx, void *stream);

/* ---- many independent instances in one call ----------------------------------
 * Each instance is a whole gres_compute problem. Skyline and partitioning run
 * per instance on a pool of internal streams forked from and joined back to
 * `stream`; then the grid-dominance kernel runs once per dimensionality (and
 * slots setting) over the targets of all those instances. Nothing waits on the
 * host: the call can be captured into one CUDA graph. */
typedef struct {
    const uint32_t *d_data;   /* device, n*d uint32 row-major                    */
    int64_t n;
    int32_t d;
    int32_t dir;
    const uint32_t *d_steps;  /* device, k widths, strictly ascending, >= 1 (not
                                 checked on the host in this call)               */
    int32_t k;
    gres_plan_cfg cfg;        /* plan (zero fields: defaults)                    */
    int64_t *d_sky_idx;       /* device, capacity n: skyline rows, ascending     */
    int32_t *d_step_idx;      /* device, capacity n: result per skyline row      */
    int64_t *d_sky_count;     /* device (may be NULL): S                         */
} gres_instance;

/* Device scratch bytes for the instances (sum of their gres_compute needs plus
 * a small head). */
gres_status gres_batch_workspace_size(const gres_instance *inst, int32_t n_inst, size_t *bytes);
gres_status gres_batch(const gres_instance *inst, int32_t n_inst, void *d_ws, size_t ws_bytes, void *stream);

/* ---- serving: resident datasets, continuous batching -------------------------
 * A server keeps prepared datasets in device memory within an HBM budget and
 * answers gres queries (a dataset and a step list) submitted from any thread.
 * A scheduler thread keeps up to max_inflight batches on the GPU; whenever a
 * slot frees up it takes up to max_batch queued queries (arrival order) and
 * runs them as one batch: one copy of their widths, one kernel for their
 * division constants, one grid-dominance launch per dimensionality over all
 * their targets, one copy of the results. A query on a skyline larger than
 * chunk_targets is answered in pieces of at most chunk_targets targets, one
 * piece per batch, after which the query goes to the back of the queue:
 * batches stay short and queries on small skylines do not wait behind a
 * large one. Queries that arrive while batches run are admitted as slots
 * free up. Results are identical to gres_query / gres_compute (the kernels
 * are deterministic per target). */
typedef struct gres_server gres_server;
typedef struct {
    int32_t max_batch;       /* queries per batch, 1..256 (0: 64)                   */
    int32_t max_inflight;    /* batches on the GPU at once, 1..16 (0: 2)            */
    int32_t queue_capacity;  /* queued queries before GRES_EAGAIN (0: 65536)        */
    int32_t max_k;           /* longest step list accepted (0: 4096)                */
    int32_t start_paused;    /* nonzero: queue queries but start no batch until
                                gres_serve_resume (admission control, tests)        */
    int32_t chunk_targets;   /* targets per piece of a query (0: 16384; < 0: whole
                                queries, no pieces)                                 */
} gres_serve_cfg;

/* Creates a server on the current device. hbm_budget_bytes bounds the device
 * memory it holds (datasets and batch buffers); GRES_ENOMEM if it cannot even
 * hold the batch buffers. cfg may be NULL. */
gres_status gres_serve_create(size_t hbm_budget_bytes, const gres_serve_cfg *cfg, gres_server **out);
/* Prepares and keeps a dataset (as gres_dataset_create); *out_id names it.
 * GRES_ENOMEM (and nothing kept) if it would exceed the budget. */
gres_status gres_serve_add_dataset(gres_server *sv, const uint32_t *data, int64_t n, int32_t d, int32_t dir,
                                   const gres_plan_cfg *plan, int32_t data_on_host, int32_t *out_id);
/* Drops a dataset; GRES_EAGAIN while queries on it are unfinished. */
gres_status gres_serve_remove_dataset(gres_server *sv, int32_t id);
/* Queues a query (widths copied; host, k, strictly ascending, >= 1, k <=
 * max_k). GRES_EAGAIN if the queue is full. */
gres_status gres_serve_submit(gres_server *sv, int32_t dataset_id, const uint32_t *h_steps, int32_t k,
                              uint64_t *out_ticket);
/* Waits up to timeout_us (0: do not wait; < 0: no limit) for a query; then
 * writes its S results (skyline order of the dataset) to h_step_idx (capacity
 * cap), S to h_sky_count and the submit-to-completion time to h_latency_ns
 * (either may be NULL), and forgets the ticket. GRES_EAGAIN if it is not
 * finished in time (the ticket stays valid). */
gres_status gres_serve_poll(gres_server *sv, uint64_t ticket, int32_t *h_step_idx, int64_t cap,
                            int64_t *h_sky_count, int64_t *h_latency_ns, int64_t timeout_us);
/* The skyline row numbers of a served dataset, ascending (Def. 1): position j
 * of every gres_serve_poll result on it is the tuple h_sky_idx[j]. Writes S
 * to h_sky_count (may be NULL) and the S row numbers to h_sky_idx (host,
 * capacity cap; GRES_EINVAL if cap < S). Waits for the copy. */
gres_status gres_serve_sky_idx(gres_server *sv, int32_t dataset_id, int64_t *h_sky_idx, int64_t cap,
                               int64_t *h_sky_count);
/* Starts batches again after start_paused (or gres_serve_pause). */
gres_status gres_serve_resume(gres_server *sv);
/* Stops starting new batches (running ones finish; queries keep queueing). */
gres_status gres_serve_pause(gres_server *sv);
/* Withdraws a query: dropped if still queued, results discarded if running. */
gres_status gres_serve_cancel(gres_server *sv, uint64_t ticket);
/* Batches run, queries answered, kernels launched, device bytes held. */
gres_status gres_serve_stats(gres_server *sv, uint64_t *batches, uint64_t *queries, uint64_t *launches,
                             size_t *device_bytes);
/* Stops the scheduler (queued queries are dropped, running batches finish)
 * and frees everything the server holds. */
gres_status gres_serve_destroy(gres_server *sv);

/* Partitioning of a candidate set (Sec. 3.1) into the tile layout that the
 * grid-dominance kernel reads: the same kernels gres_compute runs on the
 * skyline, here on the caller's rows as they are (no skyline step).
 *   d_rows      device, n*d uint32, row-major (not modified).
 *   cfg         scheme GRID / ANGULAR / SLICED / NONE with m, p, slice_dim
 *               (NULL: GRID with about 256 cells); reps, slots, flags unused.
 *   d_part      device, n int64: partition number of each row on canonical
 *               coordinates x = c - min c (c = v for GRES_MIN, 2^32-1-v for
 *               GRES_MAX; min and max over the n rows, per attribute):
 *                 GRID     sum_i floor(x_i m / (max_i - min_i + 1)) m^i;
 *                 ANGULAR  sum_{i<d-1} b_i m^i with b_i the number of angles
 *                          j pi / 2m (j = 1 .. m-1) that
 *                          phi_i = atan2(sqrt(x_{i+1}^2 + ... + x_{d-1}^2), x_i)
 *                          reaches (Eq. 1), decided exactly as
 *                          Y 2^32 >= X round(tan^2(j pi / 2m) 2^32);
 *                 SLICED   floor(r p / n), r the rank of the row in the order
 *                          of x_{slice_dim} (ties: lower row first);
 *                 NONE     0.
 *   d_order     device, n uint32: the rows in tile order (position -> row);
 *               partition numbers never decrease along it.
 *   d_tile_min  device, ceil(n/32)*d uint32: per 32-row tile of that order,
 *               the per-attribute minimum of the canonical values c.
 * Workspace: gres_workspace_size(n, d, 1). The order inside a partition
 * (a spatial order) is unspecified. GRES_EINVAL on bad arguments before
 * anything is queued. */
gres_status gres_partition(const uint32_t *d_rows, int64_t n, int32_t d, int32_t dir,
                           const gres_plan_cfg *cfg, void *d_ws, size_t ws_bytes,
                           int64_t *d_part, uint32_t *d_order, uint32_t *d_tile_min, void *stream);

/* gres_compute with the paper's grid parameter (Def. 2, Algorithm 1 with its
 * g from g_bar down to 2): values are read as fixed point v / 2^bits and the
 * grid projection at g is floor(v g / 2^bits) -- cells of slightly different
 * widths when g does not divide 2^bits. Results are indices into h_g: the
 * first g (in the order given) at which the tuple leaves the skyline, k if
 * none (the paper's gres = 1); the paper's value is 1 / h_g[index].
 *   bits   1 .. 32 (values may exceed 2^bits - 1; the projection stays exact)
 *   h_g    host, k uint32 grid parameters, strictly descending, >= 1
 * Other arguments as gres_compute; workspace gres_workspace_size(n, d, k). */
gres_status gres_compute_g(const uint32_t *d_data, int64_t n, int32_t d, int32_t dir, int32_t bits,
                           const uint32_t *h_g, int32_t k, const gres_plan_cfg *cfg,
                           void *d_ws, size_t ws_bytes,
                           int64_t *d_sky_idx, int32_t *d_step_idx,
                           int64_t *d_sky_count, int64_t *h_sky_count,
                           unsigned long long *d_tests, void *stream);

/* Grid projection (Sec. 2) of `count` values at each of k widths:
 * d_out[j*count + i] = floor(d_values[i] / h_steps[j]) (the paper's
 * floor(t[i] g) numerator with delta = 2^B / g). Division by a run-time
 * invariant divisor uses multiply-high constants (Granlund & Montgomery,
 * PLDI 1994), exact for every uint32 value.
 *   d_values  device, count uint32;  d_out  device, k*count uint32. */
gres_status gres_gproj(const uint32_t *d_values, int64_t count, const uint32_t *h_steps,
                       int32_t k, uint32_t *d_out, void *stream);

/* Number of CUDA kernels this library has queued since it was loaded (all
 * threads). For accounting in benchmarks. */
unsigned long long gres_launch_count(void);

/* Per-stage device timing for benchmarks. While enabled on the calling
 * thread, sky_compute and gres_compute record a pair of CUDA events on the
 * caller's stream around each stage: 0 = skyline pass, 1 = candidate
 * partitioning (range, partition keys, sort, tiles), 2 = the grid-dominance
 * kernel. gres_timing_enable(on) turns recording on or off and clears the
 * record. gres_timing_read waits for the recorded events and writes, for
 * stages 0 .. nstages-1, the summed milliseconds ms[i] and the number of
 * timed intervals launches[i], then clears the record. Events are created on
 * first use (do a warm-up call before timing) and reused afterwards. Inside a
 * stream capture the records become graph nodes: each replay of the graph
 * re-records that call's events. */
gres_status gres_timing_enable(int32_t on);
gres_status gres_timing_read(double *ms, int64_t *launches, int32_t nstages);

/* gres_compute without a caller workspace. The paper has no counterpart: this
 * exists for callers that cannot allocate device memory when they need a
 * result -- e.g. a plugin on another framework's stream whose allocator owns
 * the free memory, or a latency-critical loop that must not call cudaMalloc
 * (it can synchronize the device) -- and so cannot provide d_ws.
 * Same arguments and results as gres_compute, minus d_ws/ws_bytes/d_tests.
 * Scratch: one static device array of gres_static_scratch_bytes() bytes
 * (16 MiB: about 177,000 rows at d <= 4, 116,000 at d = 8, with up to 4,096
 * widths) inside the library, held on every GPU that loads the library until
 * the process exits. Sizes whose gres_workspace_size exceeds it give
 * GRES_EINVAL and nothing is launched. The call allocates nothing (no
 * cudaMalloc / cudaFree); keep gres_timing_enable off, since stage timing
 * creates CUDA events on first use. The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress, with that device current);
 * make that first call before any stream capture: a call that needs the
 * lookup inside a capture gets GRES_EINVAL. The address is kept per device
 * with the id of its CUDA context, and looked up again after the context
 * changed (cudaDeviceReset). All calls share the array:
 * each call re-initialises what it needs, and calls that overlap on the GPU
 * (different streams or unsynchronised threads) race on it -- serialise them. */
gres_status gres_compute_static(const uint32_t *d_data, int64_t n, int32_t d, int32_t dir,
                                const uint32_t *h_steps, int32_t k, const gres_plan_cfg *cfg,
                                int64_t *d_sky_idx, int32_t *d_step_idx,
                                int64_t *d_sky_count, int64_t *h_sky_count, void *stream);
size_t gres_static_scratch_bytes(void);

/* Measurement helper: the peak rate of the dominance test (Def. 1) on this
 * GPU, the denominator of the grid-dominance kernel's roofline. Queues one
 * kernel on `stream` in which every thread holds 16 candidate rows in
 * registers and tests each against a target cell [lo, hi] that moves every
 * iteration, for `iters` iterations; a test is d "<=" and d "<" comparisons
 * folded into one predicate, the 2d compare lane-ops per test that the
 * grid-dominance kernel counts as its work. *lane_ops receives the compare
 * lane-ops of the launch (blocks x 256 threads x iters x 16 x 2d); time the
 * launch with CUDA events on `stream` for lane-ops/s.
 *   d       1..8;  iters >= 1;  blocks: grid size, 0 = one full wave (as
 *           many blocks as are resident on all SMs at once).
 *   d_sink  device, one uint64: written only if a count reaches a value it
 *           cannot reach (it keeps the tests from being optimised away).
 * Errors: GRES_EINVAL for d outside [1, 8], iters < 1, blocks < 0, or a NULL
 * pointer; GRES_ECUDA if the launch fails. */
gres_status gres_test_peak_probe(int32_t d, int32_t iters, int32_t blocks, unsigned long long *d_sink,
                                 void *stream, double *lane_ops);

/* Check of the bounded grid-wide wait that the cooperative sorts (inputs above
 * 131,072 rows) use between their phases; the paper has no counterpart. One
 * cooperative launch of one block per SM waits at a grid-wide barrier, except
 * block `absent` (-1: none), which leaves at once. The waiting blocks give up
 * after about a second, set the timeout bit in the status word and return, so
 * the GPU context stays usable. d_words: device, 3 uint32 (arrival count,
 * generation, status), zeroed by the call; *h_status gets the status word
 * (bit 0: a wait ran out). Waits for the launch.
 * Returns GRES_OK, GRES_ETIMEOUT if a wait ran out, GRES_EINVAL for NULL
 * pointers, GRES_ECUDA if a CUDA call fails. */
gres_status gres_barrier_probe(int32_t absent, unsigned *d_words, void *stream, uint32_t *h_status);

/* Host helper: the multiply-high constants gres_gproj uses for divisor
 * `delta` (>= 1): floor(v / delta) = (t + ((v - t) >> s1)) >> s2 with
 * t = mulhi(m, v). Exposed so the constants can be checked without a GPU. */
gres_status gres_udiv_magic(uint32_t delta, uint32_t *m, uint32_t *s1, uint32_t *s2);

#ifdef __cplusplus
}
#endif

#endif /* GRES_H */
