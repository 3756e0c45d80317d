// api.cu -- the extern "C" entry points of libgres (include/gres.h): argument
// validation, workspace layout, stream handling and error reporting. All
// computation is queued as CUDA kernels (skyline.cu, radix_sort.cu,
// gres_stage.cu; the test-rate probe in probe.cu); nothing here computes a
// result on the host.
#include "gres_internal.cuh"

#include <atomic>
#include <cstdio>
#include <cstring>
#include <string>
#include <algorithm>
#include <vector>

namespace {

thread_local std::string g_last_error;
std::atomic<unsigned long long> g_launches{0};

// Per-thread stage timer: CUDA event pairs recorded on the launching stream.
struct StageTimer {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    struct Pair { int stage; cudaEvent_t a, b; };
    std::vector<Pair> pairs;
    cudaEvent_t open[gres::kStageCount] = {};
    cudaEvent_t next() {
        if (used == pool.size()) {
            cudaEvent_t e = nullptr;
            if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
            pool.push_back(e);
        }
        return pool[used++];
    }
};
thread_local StageTimer g_timer;

gres_status fail(gres_status s, const std::string &msg) {
    g_last_error = msg;
    return s;
}

gres_status cuda_fail(cudaError_t e, const char *where) {
    g_last_error = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return GRES_ECUDA;
}

gres_status check_dims(int64_t n, int32_t d) {
    if (d < 1 || d > gres::kMaxD) return fail(GRES_EINVAL, "d must be in [1, 8]");
    if (n < 0 || n >= (int64_t(1) << 31)) return fail(GRES_EINVAL, "n must be in [0, 2^31)");
    return GRES_OK;
}

gres_status check_steps(const uint32_t *h_steps, int32_t k) {
    if (k < 1 || k > (1 << 20)) return fail(GRES_EINVAL, "k must be in [1, 2^20]");
    if (!h_steps) return fail(GRES_EINVAL, "h_steps is NULL");
    if (h_steps[0] < 1) return fail(GRES_EINVAL, "steps must be >= 1");
    for (int32_t i = 1; i < k; i++)
        if (h_steps[i] <= h_steps[i - 1]) return fail(GRES_EINVAL, "steps must be strictly ascending");
    return GRES_OK;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

gres_status check_plan(const gres_plan_cfg *cfg, int32_t d, gres_plan_cfg *out) {
    gres_plan_cfg c;
    std::memset(&c, 0, sizeof(c));
    if (cfg) c = *cfg;
    if (cfg == nullptr) c.scheme = GRES_PART_GRID;
    if (c.scheme < GRES_PART_NONE || c.scheme > GRES_PART_SLICED)
        return fail(GRES_EINVAL, "cfg.scheme must be a gres_part");
    if (c.reserved != 0) return fail(GRES_EINVAL, "cfg.reserved must be 0");
    if (c.flags & ~(GRES_FLAG_COUNT_TESTS | GRES_FLAG_GRES_REPS | GRES_FLAG_COUNT_PARTS))
        return fail(GRES_EINVAL, "unknown cfg.flags bits");
    if ((c.flags & GRES_FLAG_COUNT_PARTS) && !(c.flags & GRES_FLAG_COUNT_TESTS))
        return fail(GRES_EINVAL, "GRES_FLAG_COUNT_PARTS needs GRES_FLAG_COUNT_TESTS");
    if (c.reps == 0) c.reps = gres::kMaxReps;
    if (c.reps < 1 || c.reps > gres::kMaxReps) return fail(GRES_EINVAL, "cfg.reps must be in [1, 1024]");
    if (c.slots == 0) c.slots = 8;
    if (c.slots != 4 && c.slots != 8) return fail(GRES_EINVAL, "cfg.slots must be 4 or 8");
    if (c.scheme == GRES_PART_GRID || c.scheme == GRES_PART_ANGULAR) {
        const int dims = c.scheme == GRES_PART_GRID ? d : d - 1;
        if (c.m == 0) {
            // about 256 cells
            int m = 2;
            while (dims > 0) {
                double cells = 1.0;
                for (int i = 0; i < dims; i++) cells *= (m + 1);
                if (cells > 256.0 * 1.5) break;
                m++;
            }
            c.m = dims > 0 ? m : 1;
            if (c.scheme == GRES_PART_ANGULAR && c.m > 64) c.m = 64;
        }
        if (c.m < 1) return fail(GRES_EINVAL, "cfg.m must be >= 1");
        double cells = 1.0;
        for (int i = 0; i < dims; i++) cells *= c.m;
        if (cells > 4294967295.0) return fail(GRES_EINVAL, "cfg.m^d must be < 2^32");
        if (c.scheme == GRES_PART_ANGULAR && c.m > 64) return fail(GRES_EINVAL, "ANGULAR m must be <= 64");
    }
    if (c.scheme == GRES_PART_SLICED) {
        if (c.p == 0) c.p = 64;
        if (c.p < 1) return fail(GRES_EINVAL, "cfg.p must be >= 1");
        if (c.slice_dim < 0 || c.slice_dim >= d) return fail(GRES_EINVAL, "cfg.slice_dim must be in [0, d)");
    }
    *out = c;
    return GRES_OK;
}

bool ws_ok(void *d_ws, size_t ws_bytes, size_t need) {
    return d_ws != nullptr && ws_bytes >= need && (reinterpret_cast<uintptr_t>(d_ws) & 255u) == 0;
}

gres_status read_status(gres::Workspace &ws, cudaStream_t st) {
    unsigned int status = 0;
    cudaError_t e = cudaMemcpyAsync(&status, &ws.hdr->status, sizeof(status), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(e, "status copy");
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    if (status & gres::kStatusTimeout) return fail(GRES_ETIMEOUT, "a bounded device wait ran out");
    if (status & gres::kStatusInternal) return fail(GRES_EINTERNAL, "internal device check failed");
    return GRES_OK;
}

gres_status finish_counts(gres::Workspace &ws, int64_t *d_sky_count, int64_t *h_sky_count, cudaStream_t st) {
    cudaError_t e;
    if (d_sky_count) {
        e = cudaMemcpyAsync(d_sky_count, &ws.hdr->n_sky, sizeof(int64_t), cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "count copy");
    }
    if (h_sky_count) {
        long long s = 0;
        e = cudaMemcpyAsync(&s, &ws.hdr->n_sky, sizeof(s), cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return cuda_fail(e, "count copy");
        gres_status r = read_status(ws, st);
        if (r != GRES_OK) return r;
        *h_sky_count = s;
    }
    return GRES_OK;
}

}  // namespace

namespace gres {

gres_status set_error(gres_status s, const char *msg) { return fail(s, msg); }

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// Records e on st; inside a stream capture as an external event node, which
// re-records the event at every replay of the graph.
void record_stage_event(cudaEvent_t e, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
    else
        cudaEventRecord(e, st);
}

void stage_begin(int stage, cudaStream_t st) {
    if (!g_timer.on) return;
    cudaEvent_t e = g_timer.next();
    if (!e) return;
    record_stage_event(e, st);
    g_timer.open[stage] = e;
}

void stage_end(int stage, cudaStream_t st) {
    if (!g_timer.on || !g_timer.open[stage]) return;
    cudaEvent_t e = g_timer.next();
    if (!e) return;
    record_stage_event(e, st);
    g_timer.pairs.push_back({stage, g_timer.open[stage], e});
    g_timer.open[stage] = nullptr;
}

size_t workspace_layout(int64_t n, int d, int k, void *base, Workspace *ws) {
    const int DP = padded_dims(d);
    const int64_t nn = n > 0 ? n : 1;
    const int64_t rows_pad = nn + kTileRows;
    const int64_t tiles = rows_pad / kTileRows + 1;
    size_t off = 0;
    char *b = static_cast<char *>(base);
    auto take = [&](size_t bytes) -> void * {
        void *p = b ? b + off : nullptr;
        off += align256(bytes);
        return p;
    };
    Workspace w;
    w.hdr = static_cast<WsHeader *>(take(sizeof(WsHeader)));
    w.keys[0] = static_cast<unsigned long long *>(take(8 * nn));
    w.keys[1] = static_cast<unsigned long long *>(take(8 * nn));
    w.vals[0] = static_cast<uint32_t *>(take(4 * nn));
    w.vals[1] = static_cast<uint32_t *>(take(4 * nn));
    w.hist = static_cast<uint32_t *>(take(4 * 256 * (sort_blocks(nn) + 1)));
    w.dtot = static_cast<uint32_t *>(take(4 * 256));
    w.blocksum = static_cast<uint32_t *>(take(4 * (scan_blocks(nn) + 1)));
    w.flags = static_cast<uint32_t *>(take(4 * nn));
    w.surv_rows = static_cast<uint32_t *>(take(4 * DP * nn));
    w.surv_orig = static_cast<uint32_t *>(take(4 * nn));
    w.reps = static_cast<uint32_t *>(take(4 * DP * kMaxReps));
    w.sel_hist = static_cast<uint32_t *>(take(sizeof(uint32_t) * gres::kSelHistWords));
    w.rep_idx = static_cast<uint32_t *>(take(4 * kMaxReps));
    w.sky_rows = static_cast<uint32_t *>(take(4 * DP * rows_pad));
    w.cand = static_cast<uint32_t *>(take(4 * DP * rows_pad));
    w.tmin = static_cast<uint32_t *>(take(4 * DP * tiles));
    w.smin = static_cast<uint32_t *>(take(4 * DP * (tiles / 32 + 1)));
    w.tsum = static_cast<unsigned long long *>(take(8 * (size_t)tiles));
    w.ssum = static_cast<unsigned long long *>(take(8 * (size_t)(tiles / 32 + 1)));
    w.perm = static_cast<uint32_t *>(take(4 * nn));
    w.res = static_cast<int32_t *>(take(4 * nn));
    w.greps = static_cast<uint32_t *>(take(4 * DP * 32));
    w.kill = static_cast<uint32_t *>(take(4 * DP * kKillers));
    w.pid = static_cast<uint32_t *>(take(4 * (size_t)rows_pad));
    w.steps = static_cast<uint32_t *>(take(4 * (size_t)(k > 0 ? k : 1)));
    w.magic = static_cast<uint32_t *>(take(16 * (size_t)(k > 0 ? k : 1)));
    w.bytes = off;
    if (ws) *ws = w;
    return off;
}

}  // namespace gres

extern "C" {

const char *gres_last_error(void) { return g_last_error.c_str(); }

const char *gres_version(void) { return "libgres 0.1 (sm_103a)"; }

unsigned long long gres_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

gres_status gres_timing_enable(int32_t on) {
    g_timer.on = on != 0;
    g_timer.pairs.clear();
    g_timer.used = 0;
    for (auto &e : g_timer.open) e = nullptr;
    return GRES_OK;
}

gres_status gres_timing_read(double *ms, int64_t *launches, int32_t nstages) {
    if (!ms || !launches || nstages < 1) return fail(GRES_EINVAL, "bad timing outputs");
    for (int i = 0; i < nstages; i++) { ms[i] = 0.0; launches[i] = 0; }
    for (const auto &p : g_timer.pairs) {
        cudaError_t e = cudaEventSynchronize(p.b);
        if (e != cudaSuccess) return cuda_fail(e, "timing event");
        float t = 0.f;
        e = cudaEventElapsedTime(&t, p.a, p.b);
        if (e != cudaSuccess) return cuda_fail(e, "timing event");
        if (p.stage < nstages) { ms[p.stage] += t; launches[p.stage] += 1; }
    }
    g_timer.pairs.clear();
    g_timer.used = 0;
    return GRES_OK;
}

gres_status gres_workspace_size(int64_t n, int32_t d, int32_t k, size_t *bytes) {
    if (!bytes) return fail(GRES_EINVAL, "bytes is NULL");
    gres_status s = check_dims(n, d);
    if (s != GRES_OK) return s;
    if (k < 1 || k > (1 << 20)) return fail(GRES_EINVAL, "k must be in [1, 2^20]");
    *bytes = gres::workspace_layout(n, d, k, nullptr, nullptr);
    return GRES_OK;
}

gres_status gres_workspace_size_host(int64_t n, int32_t d, int32_t k, size_t *bytes) {
    gres_status s = gres_workspace_size(n, d, k, bytes);
    if (s != GRES_OK) return s;
    const int64_t nn = n > 0 ? n : 1;
    *bytes += align256(4 * (size_t)nn * d) + align256(8 * (size_t)nn) + align256(4 * (size_t)nn) + 256;
    return GRES_OK;
}

gres_status gres_plan_partitions(const gres_plan_cfg *cfg, int32_t d, int64_t *out) {
    if (!out) return fail(GRES_EINVAL, "out is NULL");
    if (d < 1 || d > gres::kMaxD) return fail(GRES_EINVAL, "d must be in [1, 8]");
    gres_plan_cfg c;
    gres_status s = check_plan(cfg, d, &c);
    if (s != GRES_OK) return s;
    *out = gres::plan_partitions(c, d);
    return GRES_OK;
}

gres_status sky_compute(const uint32_t *d_data, int64_t n, int32_t d, int32_t dir,
                        void *d_ws, size_t ws_bytes,
                        int64_t *d_sky_idx, int64_t *d_sky_count, int64_t *h_sky_count,
                        void *stream) {
    gres_status s = check_dims(n, d);
    if (s != GRES_OK) return s;
    if (dir != GRES_MIN && dir != GRES_MAX) return fail(GRES_EINVAL, "dir must be GRES_MIN or GRES_MAX");
    if (n > 0 && (!d_data || !d_sky_idx)) return fail(GRES_EINVAL, "d_data / d_sky_idx is NULL");
    const size_t need = gres::workspace_layout(n, d, 1, nullptr, nullptr);
    if (!ws_ok(d_ws, ws_bytes, need)) return fail(GRES_EINVAL, "workspace too small, NULL or not 256-byte aligned");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    gres::Workspace ws;
    gres::workspace_layout(n, d, 1, d_ws, &ws);
    cudaError_t e = gres::launch_init(ws, n, st);
    if (e != cudaSuccess) return cuda_fail(e, "init");
    gres::stage_begin(gres::kStageSkyline, st);
    e = gres::launch_skyline(d_data, n, d, dir, gres::kMaxReps, ws, d_sky_idx, st);
    gres::stage_end(gres::kStageSkyline, st);
    if (e != cudaSuccess) return cuda_fail(e, "skyline");
    return finish_counts(ws, d_sky_count, h_sky_count, st);
}

gres_status gres_compute(const uint32_t *d_data, int64_t n, int32_t d, int32_t dir,
                         const uint32_t *h_steps, int32_t k, const gres_plan_cfg *cfg,
                         void *d_ws, size_t ws_bytes,
                         int64_t *d_sky_idx, int32_t *d_step_idx,
                         int64_t *d_sky_count, int64_t *h_sky_count,
                         unsigned long long *d_tests, void *stream) {
    gres_status s = check_dims(n, d);
    if (s != GRES_OK) return s;
    if (dir != GRES_MIN && dir != GRES_MAX) return fail(GRES_EINVAL, "dir must be GRES_MIN or GRES_MAX");
    s = check_steps(h_steps, k);
    if (s != GRES_OK) return s;
    gres_plan_cfg plan;
    s = check_plan(cfg, d, &plan);
    if (s != GRES_OK) return s;
    if (n > 0 && (!d_data || !d_sky_idx || !d_step_idx))
        return fail(GRES_EINVAL, "d_data / d_sky_idx / d_step_idx is NULL");
    const size_t need = gres::workspace_layout(n, d, k, nullptr, nullptr);
    if (!ws_ok(d_ws, ws_bytes, need)) return fail(GRES_EINVAL, "workspace too small, NULL or not 256-byte aligned");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    gres::Workspace ws;
    gres::workspace_layout(n, d, k, d_ws, &ws);
    cudaError_t e = gres::launch_init_steps(ws, n, h_steps, k, st);
    if (e != cudaSuccess) return cuda_fail(e, "init");
    gres::stage_begin(gres::kStageSkyline, st);
    e = gres::launch_skyline(d_data, n, d, dir, plan.reps, ws, d_sky_idx, st,
                             (plan.flags & GRES_FLAG_GRES_REPS) != 0);
    gres::stage_end(gres::kStageSkyline, st);
    if (e != cudaSuccess) return cuda_fail(e, "skyline");
    e = gres::launch_gres_stage(d_data, n, d, dir, k, plan, ws, d_sky_idx, d_step_idx, d_tests, st);
    if (e != cudaSuccess) return cuda_fail(e, "gres stage");
    return finish_counts(ws, d_sky_count, h_sky_count, st);
}

gres_status gres_compute_g(const uint32_t *d_data, int64_t n, int32_t d, int32_t dir, int32_t bits,
                           const uint32_t *h_g, int32_t k, const gres_plan_cfg *cfg,
                           void *d_ws, size_t ws_bytes,
                           int64_t *d_sky_idx, int32_t *d_step_idx,
                           int64_t *d_sky_count, int64_t *h_sky_count,
                           unsigned long long *d_tests, void *stream) {
    gres_status s = check_dims(n, d);
    if (s != GRES_OK) return s;
    if (dir != GRES_MIN && dir != GRES_MAX) return fail(GRES_EINVAL, "dir must be GRES_MIN or GRES_MAX");
    if (bits < 1 || bits > 32) return fail(GRES_EINVAL, "bits must be in [1, 32]");
    if (k < 1 || k > (1 << 20)) return fail(GRES_EINVAL, "k must be in [1, 2^20]");
    if (!h_g) return fail(GRES_EINVAL, "h_g is NULL");
    if (h_g[k - 1] < 1) return fail(GRES_EINVAL, "grid parameters must be >= 1");
    for (int32_t i = 1; i < k; i++)
        if (h_g[i] >= h_g[i - 1]) return fail(GRES_EINVAL, "grid parameters must be strictly descending");
    gres_plan_cfg plan;
    s = check_plan(cfg, d, &plan);
    if (s != GRES_OK) return s;
    if (n > 0 && (!d_data || !d_sky_idx || !d_step_idx))
        return fail(GRES_EINVAL, "d_data / d_sky_idx / d_step_idx is NULL");
    const size_t need = gres::workspace_layout(n, d, k, nullptr, nullptr);
    if (!ws_ok(d_ws, ws_bytes, need)) return fail(GRES_EINVAL, "workspace too small, NULL or not 256-byte aligned");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    gres::Workspace ws;
    gres::workspace_layout(n, d, k, d_ws, &ws);
    cudaError_t e = gres::launch_init_steps(ws, n, h_g, k, st, bits);
    if (e != cudaSuccess) return cuda_fail(e, "init");
    gres::stage_begin(gres::kStageSkyline, st);
    e = gres::launch_skyline(d_data, n, d, dir, plan.reps, ws, d_sky_idx, st,
                             (plan.flags & GRES_FLAG_GRES_REPS) != 0);
    gres::stage_end(gres::kStageSkyline, st);
    if (e != cudaSuccess) return cuda_fail(e, "skyline");
    e = gres::launch_gres_stage(d_data, n, d, dir, k, plan, ws, d_sky_idx, d_step_idx, d_tests, st, bits);
    if (e != cudaSuccess) return cuda_fail(e, "gres stage");
    return finish_counts(ws, d_sky_count, h_sky_count, st);
}

namespace {

// gres_compute_host keeps one CUDA graph per (input buffer, shape, widths,
// plan, workspace, device) for pinned inputs: the input copy, the whole
// computation and the copy of S and the status word back. A repeated call
// with the same arguments replays it -- one graph launch instead of a dozen
// kernel launches -- and then copies the S results. The first call of a key
// runs directly (which also sets every kernel's launch attributes outside any
// capture) and captures the graph afterwards without running it.
struct HostGraph {
    const uint32_t *h_data = nullptr;
    int64_t n = 0;
    int32_t d = 0, dir = 0;
    std::vector<uint32_t> steps;
    gres_plan_cfg cfg;
    void *d_ws = nullptr;
    int device = -1;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    int64_t *h_out = nullptr;     // pinned: [0] S, [1] the header's status word (low 32 bits)
    int64_t *h_sky = nullptr;     // the caller's result buffers the graph copies into
    int32_t *h_step = nullptr;
    int64_t spec = 0;             // results the graph copies (the capturing call's S; 0 if unpinned)
    unsigned long long used = 0;
};
constexpr size_t kHostGraphs = 4;
thread_local std::vector<HostGraph> g_host_graphs;
thread_local unsigned long long g_host_clock = 0;

void host_graph_free(HostGraph &g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.ev) cudaEventDestroy(g.ev);
    if (g.st) cudaStreamDestroy(g.st);
    if (g.h_out) cudaFreeHost(g.h_out);
    g = HostGraph();
}

}  // namespace

gres_status gres_compute_host(const uint32_t *h_data, int64_t n, int32_t d, int32_t dir,
                              const uint32_t *h_steps, int32_t k, const gres_plan_cfg *cfg,
                              void *d_ws, size_t ws_bytes,
                              int64_t *h_sky_idx, int32_t *h_step_idx, int64_t *h_sky_count,
                              void *stream) {
    gres_status s = check_dims(n, d);
    if (s != GRES_OK) return s;
    if (!h_sky_count) return fail(GRES_EINVAL, "h_sky_count is NULL");
    if (n > 0 && (!h_data || !h_sky_idx || !h_step_idx))
        return fail(GRES_EINVAL, "h_data / h_sky_idx / h_step_idx is NULL");
    size_t need = 0;
    s = gres_workspace_size_host(n, d, k > 0 ? k : 1, &need);
    if (s != GRES_OK) return s;
    if (!ws_ok(d_ws, ws_bytes, need)) return fail(GRES_EINVAL, "workspace too small, NULL or not 256-byte aligned");
    const size_t core = gres::workspace_layout(n, d, k, nullptr, nullptr);
    const int64_t nn = n > 0 ? n : 1;
    char *extra = static_cast<char *>(d_ws) + core;
    uint32_t *d_data = reinterpret_cast<uint32_t *>(extra);
    int64_t *d_sky = reinterpret_cast<int64_t *>(extra + align256(4 * (size_t)nn * d));
    int32_t *d_res = reinterpret_cast<int32_t *>(extra + align256(4 * (size_t)nn * d) + align256(8 * (size_t)nn));
    int64_t *d_count = reinterpret_cast<int64_t *>(reinterpret_cast<char *>(d_res) + align256(4 * (size_t)nn));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    gres_plan_cfg plan_key;
    std::memset(&plan_key, 0, sizeof(plan_key));
    if (cfg) plan_key = *cfg;
    int device = 0;
    if ((e = cudaGetDevice(&device)) != cudaSuccess) return cuda_fail(e, "device");
    cudaPointerAttributes pa;
    const bool pinned = n > 0 && cudaPointerGetAttributes(&pa, h_data) == cudaSuccess && pa.type == cudaMemoryTypeHost;
    cudaGetLastError();   // clear a lookup error on unregistered memory
    HostGraph *hit = nullptr;
    if (pinned && k >= 1 && h_steps) {
        for (HostGraph &g : g_host_graphs)
            if (g.exec && g.h_data == h_data && g.n == n && g.d == d && g.dir == dir && g.d_ws == d_ws &&
                g.h_sky == h_sky_idx && g.h_step == h_step_idx &&
                g.device == device && std::memcmp(&g.cfg, &plan_key, sizeof(plan_key)) == 0 &&
                g.steps.size() == (size_t)k && std::memcmp(g.steps.data(), h_steps, 4 * (size_t)k) == 0)
                hit = &g;
        if (hit && hit->spec > 0) {
            // the graph copies results straight into the caller's buffers: they must still be
            // pinned (a freed pinned buffer may come back as pageable memory at the same address)
            cudaPointerAttributes ra, rb;
            const bool out_pinned = cudaPointerGetAttributes(&ra, h_sky_idx) == cudaSuccess &&
                                    ra.type == cudaMemoryTypeHost &&
                                    cudaPointerGetAttributes(&rb, h_step_idx) == cudaSuccess &&
                                    rb.type == cudaMemoryTypeHost;
            cudaGetLastError();
            if (!out_pinned) {
                const size_t at = (size_t)(hit - g_host_graphs.data());
                host_graph_free(*hit);
                g_host_graphs.erase(g_host_graphs.begin() + (std::ptrdiff_t)at);
                hit = nullptr;
            }
        }
    }
    int64_t S = 0;
    if (hit) {
        hit->used = ++g_host_clock;
        if ((e = cudaEventRecord(hit->ev, st)) != cudaSuccess) return cuda_fail(e, "host graph");
        if ((e = cudaStreamWaitEvent(hit->st, hit->ev, 0)) != cudaSuccess) return cuda_fail(e, "host graph");
        if ((e = cudaGraphLaunch(hit->exec, hit->st)) != cudaSuccess) return cuda_fail(e, "host graph");
        if ((e = cudaStreamSynchronize(hit->st)) != cudaSuccess) return cuda_fail(e, "stream synchronize");
        const unsigned status = (unsigned)hit->h_out[1];
        if (status & gres::kStatusTimeout) return fail(GRES_ETIMEOUT, "a bounded device wait ran out");
        if (status & gres::kStatusInternal) return fail(GRES_EINTERNAL, "internal device check failed");
        S = hit->h_out[0];
        st = hit->st;
    } else {
        if (n > 0) {
            e = cudaMemcpyAsync(d_data, h_data, 4 * (size_t)n * d, cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) return cuda_fail(e, "input copy");
        }
        s = gres_compute(d_data, n, d, dir, h_steps, k, cfg, d_ws, core, d_sky, d_res, nullptr, &S, nullptr, stream);
        if (s != GRES_OK) return s;
        if (pinned) {
            // capture the same work for the next call with these arguments
            HostGraph g;
            g.h_data = h_data;
            g.n = n;
            g.d = d;
            g.dir = dir;
            g.steps.assign(h_steps, h_steps + k);
            g.cfg = plan_key;
            g.d_ws = d_ws;
            g.device = device;
            g.h_sky = h_sky_idx;
            g.h_step = h_step_idx;
            // with pinned result buffers the graph also copies the first S results (S of this call)
            cudaPointerAttributes ra, rb;
            const bool out_pinned = cudaPointerGetAttributes(&ra, h_sky_idx) == cudaSuccess &&
                                    ra.type == cudaMemoryTypeHost &&
                                    cudaPointerGetAttributes(&rb, h_step_idx) == cudaSuccess &&
                                    rb.type == cudaMemoryTypeHost;
            cudaGetLastError();
            g.spec = out_pinned ? S : 0;
            bool ok = cudaStreamCreateWithFlags(&g.st, cudaStreamNonBlocking) == cudaSuccess &&
                      cudaEventCreateWithFlags(&g.ev, cudaEventDisableTiming) == cudaSuccess &&
                      cudaMallocHost(&g.h_out, 2 * sizeof(int64_t)) == cudaSuccess;
            cudaGraph_t graph = nullptr;
            if (ok) ok = cudaStreamBeginCapture(g.st, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (ok) {
                bool body = cudaMemcpyAsync(d_data, h_data, 4 * (size_t)n * d, cudaMemcpyHostToDevice, g.st) ==
                            cudaSuccess;
                if (body) body = gres_compute(d_data, n, d, dir, h_steps, k, cfg, d_ws, core, d_sky, d_res, d_count,
                                              nullptr, nullptr, g.st) == GRES_OK;
                if (body) body = cudaMemcpyAsync(g.h_out, d_count, sizeof(int64_t), cudaMemcpyDeviceToHost,
                                                 g.st) == cudaSuccess;
                if (body) body = cudaMemcpyAsync(g.h_out + 1, &reinterpret_cast<gres::WsHeader *>(d_ws)->status,
                                                 sizeof(unsigned), cudaMemcpyDeviceToHost, g.st) == cudaSuccess;
                if (body && g.spec > 0)
                    body = cudaMemcpyAsync(h_sky_idx, d_sky, 8 * (size_t)g.spec, cudaMemcpyDeviceToHost, g.st) ==
                               cudaSuccess &&
                           cudaMemcpyAsync(h_step_idx, d_res, 4 * (size_t)g.spec, cudaMemcpyDeviceToHost, g.st) ==
                               cudaSuccess;
                ok = cudaStreamEndCapture(g.st, &graph) == cudaSuccess && body;
            }
            if (ok) ok = cudaGraphInstantiate(&g.exec, graph, 0) == cudaSuccess;
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            if (ok) {
                g.h_out[1] = 0;
                g.used = ++g_host_clock;
                if (g_host_graphs.size() >= kHostGraphs) {
                    auto old = std::min_element(g_host_graphs.begin(), g_host_graphs.end(),
                                                [](const HostGraph &a, const HostGraph &b) { return a.used < b.used; });
                    host_graph_free(*old);
                    g_host_graphs.erase(old);
                }
                g_host_graphs.push_back(std::move(g));
            } else {
                host_graph_free(g);
            }
        }
    }
    // results the replayed graph has not copied already
    const int64_t from = hit ? std::min(S, hit->spec) : 0;
    if (S > from) {
        cudaError_t e = cudaMemcpyAsync(h_sky_idx + from, d_sky + from, 8 * (size_t)(S - from),
                                        cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return cuda_fail(e, "result copy");
        e = cudaMemcpyAsync(h_step_idx + from, d_res + from, 4 * (size_t)(S - from), cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return cuda_fail(e, "result copy");
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    }
    if (hit) {
        // later work on the caller's stream comes after the graph's
        cudaEventRecord(hit->ev, hit->st);
        cudaStreamWaitEvent(static_cast<cudaStream_t>(stream), hit->ev, 0);
    }
    *h_sky_count = S;
    return GRES_OK;
}

gres_status gres_partition(const uint32_t *d_rows, int64_t n, int32_t d, int32_t dir,
                           const gres_plan_cfg *cfg, void *d_ws, size_t ws_bytes,
                           int64_t *d_part, uint32_t *d_order, uint32_t *d_tile_min, void *stream) {
    gres_status s = check_dims(n, d);
    if (s != GRES_OK) return s;
    if (dir != GRES_MIN && dir != GRES_MAX) return fail(GRES_EINVAL, "dir must be GRES_MIN or GRES_MAX");
    gres_plan_cfg plan;
    s = check_plan(cfg, d, &plan);
    if (s != GRES_OK) return s;
    if (n > 0 && (!d_rows || !d_part || !d_order || !d_tile_min))
        return fail(GRES_EINVAL, "d_rows / d_part / d_order / d_tile_min is NULL");
    const size_t need = gres::workspace_layout(n, d, 1, nullptr, nullptr);
    if (!ws_ok(d_ws, ws_bytes, need)) return fail(GRES_EINVAL, "workspace too small, NULL or not 256-byte aligned");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    gres::Workspace ws;
    gres::workspace_layout(n, d, 1, d_ws, &ws);
    cudaError_t e = gres::launch_init(ws, n, st);
    if (e != cudaSuccess) return cuda_fail(e, "init");
    e = gres::launch_load_candidates(d_rows, n, d, dir, ws, st);
    if (e != cudaSuccess) return cuda_fail(e, "load");
    e = gres::launch_partition(d, plan, n, ws, st);
    if (e != cudaSuccess) return cuda_fail(e, "partition");
    e = gres::launch_partition_out(d, plan, n, ws, d_part, d_order, d_tile_min, st);
    if (e != cudaSuccess) return cuda_fail(e, "partition output");
    return GRES_OK;
}

gres_status gres_gproj(const uint32_t *d_values, int64_t count, const uint32_t *h_steps,
                       int32_t k, uint32_t *d_out, void *stream) {
    if (count < 0) return fail(GRES_EINVAL, "count must be >= 0");
    gres_status s = check_steps(h_steps, k);
    if (s != GRES_OK) return s;
    if (count > 0 && (!d_values || !d_out)) return fail(GRES_EINVAL, "d_values / d_out is NULL");
    cudaError_t e = gres::launch_gproj(d_values, count, h_steps, k, d_out, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "gproj");
    return GRES_OK;
}

gres_status gres_test_peak_probe(int32_t d, int32_t iters, int32_t blocks, unsigned long long *d_sink,
                                 void *stream, double *lane_ops) {
    if (d < 1 || d > gres::kMaxD) return fail(GRES_EINVAL, "d must be in [1, 8]");
    if (iters < 1 || blocks < 0) return fail(GRES_EINVAL, "iters must be >= 1 and blocks >= 0");
    if (!d_sink || !lane_ops) return fail(GRES_EINVAL, "d_sink / lane_ops is NULL");
    cudaError_t e = gres::launch_test_peak(d, iters, blocks, d_sink, static_cast<cudaStream_t>(stream), lane_ops);
    if (e != cudaSuccess) return cuda_fail(e, "test peak probe");
    return GRES_OK;
}

gres_status gres_udiv_magic(uint32_t delta, uint32_t *m, uint32_t *s1, uint32_t *s2) {
    if (delta < 1 || !m || !s1 || !s2) return fail(GRES_EINVAL, "delta must be >= 1, outputs non-NULL");
    gres::udiv_magic(delta, m, s1, s2);
    return GRES_OK;
}

}  // extern "C"
