// batch.cu -- resident datasets, per-query gres, and many instances per call.
//
// The skyline and its candidate tiles depend only on the data (Def. 1 and the
// stability of gres, Sec. 3.2): a dataset prepared once answers any number of
// gres queries, each with its own step list, with just the grid-dominance
// kernel. gres_batch runs many independent instances: their skyline and
// partitioning stages on a pool of forked streams, then the grid-dominance
// kernel once for all instances of a dimensionality (one work queue over all
// their targets). Every call queues on the caller's stream and is
// capturable into a CUDA graph.
#include "gres_internal.cuh"

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

namespace {

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

gres_status fail(gres_status s, const std::string &msg) { return gres::set_error(s, msg.c_str()); }

gres_status cuda_fail(cudaError_t e, const char *where) {
    return fail(GRES_ECUDA, std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

// Forked streams and their fork / join events, per device, created on first use.
constexpr int kPoolStreams = 16;
struct StreamPool {
    bool ready = false;
    cudaStream_t s[kPoolStreams];
    cudaEvent_t fork, join[kPoolStreams];
};
constexpr int kMaxDevices = 64;
StreamPool g_pools[kMaxDevices];
std::mutex g_pool_mu;

cudaError_t stream_pool(StreamPool **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_pool_mu);
    StreamPool &p = g_pools[dev];
    if (!p.ready) {
        for (int i = 0; i < kPoolStreams; i++) {
            if ((e = cudaStreamCreateWithFlags(&p.s[i], cudaStreamNonBlocking)) != cudaSuccess) return e;
            if ((e = cudaEventCreateWithFlags(&p.join[i], cudaEventDisableTiming)) != cudaSuccess) return e;
        }
        if ((e = cudaEventCreateWithFlags(&p.fork, cudaEventDisableTiming)) != cudaSuccess) return e;
        p.ready = true;
    }
    *out = &p;
    return cudaSuccess;
}

gres_status check_common(int64_t n, int32_t d, int32_t dir) {
    if (d < 1 || d > gres::kMaxD) return fail(GRES_EINVAL, "d must be in [1, 8]");
    if (n < 0 || n >= (int64_t(1) << 31)) return fail(GRES_EINVAL, "n must be in [0, 2^31)");
    if (dir != GRES_MIN && dir != GRES_MAX) return fail(GRES_EINVAL, "dir must be GRES_MIN or GRES_MAX");
    return GRES_OK;
}

gres_status normalize_plan(const gres_plan_cfg *cfg, int32_t d, gres_plan_cfg *out, bool allow_reps = false) {
    // the same defaults and limits as gres_compute
    gres_plan_cfg c;
    std::memset(&c, 0, sizeof(c));
    if (cfg) c = *cfg; else c.scheme = GRES_PART_GRID;
    if (c.scheme < GRES_PART_NONE || c.scheme > GRES_PART_SLICED) return fail(GRES_EINVAL, "cfg.scheme must be a gres_part");
    if (c.reserved != 0) return fail(GRES_EINVAL, "cfg.reserved must be 0");
    const int allowed = GRES_FLAG_COUNT_TESTS | (allow_reps ? GRES_FLAG_GRES_REPS : 0);
    if (c.flags & ~allowed) return fail(GRES_EINVAL, "cfg.flags: flag not supported by this call");
    if (c.reps == 0) c.reps = gres::kMaxReps;
    if (c.reps < 1 || c.reps > gres::kMaxReps) return fail(GRES_EINVAL, "cfg.reps must be in [1, 1024]");
    if (c.slots == 0) c.slots = 8;
    if (c.slots != 4 && c.slots != 8) return fail(GRES_EINVAL, "cfg.slots must be 4 or 8");
    if (c.scheme == GRES_PART_GRID || c.scheme == GRES_PART_ANGULAR) {
        const int dims = c.scheme == GRES_PART_GRID ? d : d - 1;
        if (c.m == 0) {
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

}  // namespace

extern "C" {

gres_status gres_dataset_create(const uint32_t *data, int64_t n, int32_t d, int32_t dir,
                                const gres_plan_cfg *cfg, int32_t data_on_host, void *stream,
                                gres_dataset **out) {
    if (!out) return fail(GRES_EINVAL, "out is NULL");
    *out = nullptr;
    gres_status s = check_common(n, d, dir);
    if (s != GRES_OK) return s;
    if (n > 0 && !data) return fail(GRES_EINVAL, "data is NULL");
    gres_plan_cfg plan;
    if ((s = normalize_plan(cfg, d, &plan)) != GRES_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t nn = n > 0 ? n : 1;
    const size_t ws_bytes = gres::workspace_layout(n, d, 1, nullptr, nullptr);
    const size_t tmp_bytes = ws_bytes + align256(8 * (size_t)nn) + (data_on_host ? align256(4 * (size_t)nn * d) : 0);
    void *tmp = nullptr;
    cudaError_t e = cudaMallocAsync(&tmp, tmp_bytes, st);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? fail(GRES_ENOMEM, "dataset: out of device memory")
                                                                 : cuda_fail(e, "dataset scratch");
    gres::Workspace ws;
    gres::workspace_layout(n, d, 1, tmp, &ws);
    char *extra = static_cast<char *>(tmp) + ws_bytes;
    int64_t *tmp_sky = reinterpret_cast<int64_t *>(extra);
    const uint32_t *d_data = data;
    if (data_on_host && n > 0) {
        uint32_t *dd = reinterpret_cast<uint32_t *>(extra + align256(8 * (size_t)nn));
        e = cudaMemcpyAsync(dd, data, 4 * (size_t)n * d, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) { cudaFreeAsync(tmp, st); return cuda_fail(e, "dataset upload"); }
        d_data = dd;
    }
    long long S = 0;
    e = gres::launch_init(ws, n, st);
    if (e == cudaSuccess) e = gres::launch_skyline(d_data, n, d, dir, plan.reps, ws, tmp_sky, st);
    if (e == cudaSuccess) e = gres::launch_partition(d, plan, n, ws, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&S, &ws.hdr->n_sky, sizeof(S), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { cudaFreeAsync(tmp, st); return cuda_fail(e, "dataset prepare"); }
    const int DP = gres::padded_dims(d);
    const int64_t T = (S + gres::kTileRows - 1) / gres::kTileRows;
    const size_t b_sky = align256(8 * (size_t)(S > 0 ? S : 1));
    const size_t b_perm = align256(4 * (size_t)(S > 0 ? S : 1));
    const size_t b_cand = align256(4 * (size_t)DP * (size_t)(T > 0 ? T : 1) * gres::kTileRows);
    const size_t b_tmin = align256(4 * (size_t)DP * (size_t)(T > 0 ? T : 1));
    const int64_t T2 = (T + 31) / 32;
    const size_t b_smin = align256(4 * (size_t)DP * (size_t)(T2 > 0 ? T2 : 1));
    const size_t bytes = b_sky + 2 * b_perm + b_cand + b_tmin + b_smin + 256;
    void *mem = nullptr;
    e = cudaMalloc(&mem, bytes);
    if (e != cudaSuccess) {
        cudaFreeAsync(tmp, st);
        cudaStreamSynchronize(st);
        return e == cudaErrorMemoryAllocation ? fail(GRES_ENOMEM, "dataset: out of device memory")
                                              : cuda_fail(e, "dataset allocation");
    }
    gres_dataset *ds = new gres_dataset;
    cudaGetDevice(&ds->device);
    ds->n = n;
    ds->d = d;
    ds->dir = dir;
    ds->slots = plan.slots;
    ds->S = S;
    ds->mem = mem;
    ds->bytes = bytes;
    char *m = static_cast<char *>(mem);
    ds->sky_idx = reinterpret_cast<int64_t *>(m);
    ds->perm = reinterpret_cast<uint32_t *>(m + b_sky);
    ds->iperm = reinterpret_cast<uint32_t *>(m + b_sky + b_perm);
    m += b_perm;
    ds->cand = reinterpret_cast<uint32_t *>(m + b_sky + b_perm);
    ds->tmin = reinterpret_cast<uint32_t *>(m + b_sky + b_perm + b_cand);
    ds->smin = reinterpret_cast<uint32_t *>(m + b_sky + b_perm + b_cand + b_tmin);
    ds->n_sky = reinterpret_cast<long long *>(m + b_sky + b_perm + b_cand + b_tmin + b_smin);
    e = cudaMemcpyAsync(ds->n_sky, &ws.hdr->n_sky, sizeof(long long), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && S > 0) {
        e = cudaMemcpyAsync(ds->sky_idx, tmp_sky, 8 * (size_t)S, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(ds->perm, ws.perm, 4 * (size_t)S, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = gres::launch_invert_perm(ds->perm, S, ds->iperm, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ds->cand, ws.cand, 4 * (size_t)DP * T * gres::kTileRows, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ds->tmin, ws.tmin, 4 * (size_t)DP * T, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ds->smin, ws.smin, 4 * (size_t)DP * T2, cudaMemcpyDeviceToDevice, st);
    }
    cudaFreeAsync(tmp, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaFree(mem);
        delete ds;
        return cuda_fail(e, "dataset copy");
    }
    *out = ds;
    return GRES_OK;
}

gres_status gres_dataset_destroy(gres_dataset *ds) {
    if (!ds) return GRES_OK;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != ds->device) cudaSetDevice(ds->device);
    cudaError_t e = cudaFree(ds->mem);
    if (cur != ds->device) cudaSetDevice(cur);
    delete ds;
    return e == cudaSuccess ? GRES_OK : cuda_fail(e, "dataset free");
}

gres_status gres_dataset_info(const gres_dataset *ds, int64_t *n, int32_t *d, int64_t *sky_count,
                              size_t *device_bytes) {
    if (!ds) return fail(GRES_EINVAL, "dataset is NULL");
    if (n) *n = ds->n;
    if (d) *d = ds->d;
    if (sky_count) *sky_count = ds->S;
    if (device_bytes) *device_bytes = ds->bytes;
    return GRES_OK;
}

gres_status gres_dataset_sky_idx(const gres_dataset *ds, int64_t *out, int32_t out_on_host, void *stream) {
    if (!ds || (!out && ds->S > 0)) return fail(GRES_EINVAL, "dataset / out is NULL");
    if (ds->S == 0) return GRES_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(out, ds->sky_idx, 8 * (size_t)ds->S,
                                    out_on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && out_on_host) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? GRES_OK : cuda_fail(e, "sky_idx copy");
}

gres_status gres_query_workspace_size(int32_t k, size_t *bytes) {
    if (!bytes) return fail(GRES_EINVAL, "bytes is NULL");
    if (k < 1 || k > (1 << 20)) return fail(GRES_EINVAL, "k must be in [1, 2^20]");
    *bytes = align256(4 * (size_t)k) + align256(16 * (size_t)k) + 256;
    return GRES_OK;
}

gres_status gres_query(const gres_dataset *ds, const uint32_t *h_steps, int32_t k, void *d_qws, size_t qws_bytes,
                       int32_t *d_step_idx, void *stream) {
    if (!ds) return fail(GRES_EINVAL, "dataset is NULL");
    size_t need = 0;
    gres_status s = gres_query_workspace_size(k, &need);
    if (s != GRES_OK) return s;
    if (!h_steps) return fail(GRES_EINVAL, "h_steps is NULL");
    if (h_steps[0] < 1) return fail(GRES_EINVAL, "steps must be >= 1");
    for (int32_t i = 1; i < k; i++)
        if (h_steps[i] <= h_steps[i - 1]) return fail(GRES_EINVAL, "steps must be strictly ascending");
    if (!d_qws || qws_bytes < need || (reinterpret_cast<uintptr_t>(d_qws) & 255u))
        return fail(GRES_EINVAL, "query workspace too small, NULL or not 256-byte aligned");
    if (ds->S > 0 && !d_step_idx) return fail(GRES_EINVAL, "d_step_idx is NULL");
    if (ds->S == 0) return GRES_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char *q = static_cast<char *>(d_qws);
    uint32_t *steps = reinterpret_cast<uint32_t *>(q);
    uint32_t *magic = reinterpret_cast<uint32_t *>(q + align256(4 * (size_t)k));
    unsigned *counter = reinterpret_cast<unsigned *>(q + align256(4 * (size_t)k) + align256(16 * (size_t)k));
    cudaError_t e = gres::launch_upload_steps(steps, magic, counter, h_steps, k, st);
    if (e != cudaSuccess) return cuda_fail(e, "query steps");
    gres::DomQuery dq;
    dq.cand = ds->cand;
    dq.tmin = ds->tmin;
    dq.smin = ds->smin;
    dq.perm = ds->perm;
    dq.n_sky = ds->n_sky;
    dq.magic = magic;
    dq.steps = steps;
    dq.out = d_step_idx;
    dq.K = k;
    dq.dir = ds->dir;
    e = gres::launch_dominance(ds->d, ds->slots, dq, counter, nullptr, st);
    return e == cudaSuccess ? GRES_OK : cuda_fail(e, "query");
}

// ---- many instances ------------------------------------------------------------
namespace {

struct InstLayout {
    size_t ws_off, ws_bytes;
};

gres_status batch_layout(const gres_instance *inst, int32_t n_inst, std::vector<InstLayout> *lay,
                         size_t *head, size_t *total) {
    if (n_inst < 0 || (n_inst > 0 && !inst)) return fail(GRES_EINVAL, "bad instance list");
    // head: one work counter per dominance launch (at most one per (d, slots) and 256 instances)
    const size_t h = align256(sizeof(unsigned) * (size_t)(16 + 2 * (n_inst / 256 + 1) * 16));
    size_t off = h;
    if (lay) lay->resize((size_t)n_inst);
    for (int32_t i = 0; i < n_inst; i++) {
        const gres_instance &x = inst[i];
        gres_status s = check_common(x.n, x.d, x.dir);
        if (s != GRES_OK) return fail(s, "instance " + std::to_string(i) + ": " + gres_last_error());
        if (x.k < 1 || x.k > (1 << 20)) return fail(GRES_EINVAL, "instance " + std::to_string(i) + ": k out of range");
        const size_t b = gres::workspace_layout(x.n, x.d, x.k, nullptr, nullptr);
        if (lay) (*lay)[(size_t)i] = {off, b};
        off += align256(b);
    }
    if (head) *head = h;
    *total = off;
    return GRES_OK;
}

}  // namespace

gres_status gres_batch_workspace_size(const gres_instance *inst, int32_t n_inst, size_t *bytes) {
    if (!bytes) return fail(GRES_EINVAL, "bytes is NULL");
    return batch_layout(inst, n_inst, nullptr, nullptr, bytes);
}

gres_status gres_batch(const gres_instance *inst, int32_t n_inst, void *d_ws, size_t ws_bytes, void *stream) {
    std::vector<InstLayout> lay;
    size_t head = 0, total = 0;
    gres_status s = batch_layout(inst, n_inst, &lay, &head, &total);
    if (s != GRES_OK) return s;
    if (n_inst == 0) return GRES_OK;
    if (!d_ws || ws_bytes < total || (reinterpret_cast<uintptr_t>(d_ws) & 255u))
        return fail(GRES_EINVAL, "batch workspace too small, NULL or not 256-byte aligned");
    std::vector<gres_plan_cfg> plans((size_t)n_inst);
    for (int32_t i = 0; i < n_inst; i++) {
        const gres_instance &x = inst[i];
        if ((s = normalize_plan(&x.cfg, x.d, &plans[(size_t)i], true)) != GRES_OK) return s;
        if (x.n > 0 && (!x.d_data || !x.d_steps || !x.d_sky_idx || !x.d_step_idx))
            return fail(GRES_EINVAL, "instance " + std::to_string(i) + ": NULL buffer");
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    StreamPool *pool = nullptr;
    cudaError_t e = stream_pool(&pool);
    if (e != cudaSuccess) return cuda_fail(e, "stream pool");
    char *base = static_cast<char *>(d_ws);
    unsigned *counters = reinterpret_cast<unsigned *>(base);
    std::vector<gres::Workspace> ws((size_t)n_inst);
    for (int32_t i = 0; i < n_inst; i++)
        gres::workspace_layout(inst[i].n, inst[i].d, inst[i].k, base + lay[(size_t)i].ws_off, &ws[(size_t)i]);
    // 1. counters and division constants for every instance, on the caller's stream
    e = cudaMemsetAsync(counters, 0, head, st);
    if (e != cudaSuccess) return cuda_fail(e, "batch counters");
    std::vector<gres::MagicJob> jobs;
    for (int32_t i = 0; i < n_inst; i++) {
        if (inst[i].n == 0) continue;
        jobs.push_back({inst[i].d_steps, ws[(size_t)i].magic, inst[i].k, nullptr});
    }
    e = gres::launch_make_magic(jobs.data(), (int)jobs.size(), st);
    if (e != cudaSuccess) return cuda_fail(e, "batch constants");
    // 2. skyline and partitioning per instance, on the forked streams
    if ((e = cudaEventRecord(pool->fork, st)) != cudaSuccess) return cuda_fail(e, "fork");
    for (int j = 0; j < kPoolStreams; j++)
        if ((e = cudaStreamWaitEvent(pool->s[j], pool->fork, 0)) != cudaSuccess) return cuda_fail(e, "fork");
    for (int32_t i = 0; i < n_inst; i++) {
        const gres_instance &x = inst[i];
        cudaStream_t si = pool->s[i % kPoolStreams];
        gres::Workspace &w = ws[(size_t)i];
        e = gres::launch_init(w, x.n, si);
        const bool greps = (plans[(size_t)i].flags & GRES_FLAG_GRES_REPS) != 0;
        if (e == cudaSuccess)
            e = gres::launch_skyline(x.d_data, x.n, x.d, x.dir, plans[(size_t)i].reps, w, x.d_sky_idx, si, greps);
        if (e == cudaSuccess) e = gres::launch_partition(x.d, plans[(size_t)i], x.n, w, si);
        if (e == cudaSuccess && greps) e = gres::launch_rep_bound(x.d, x.n, w, x.k, x.dir, 0, nullptr, si);
        if (e == cudaSuccess && x.d_sky_count)
            e = cudaMemcpyAsync(x.d_sky_count, &w.hdr->n_sky, sizeof(int64_t), cudaMemcpyDeviceToDevice, si);
        if (e != cudaSuccess) return cuda_fail(e, "batch skyline");
    }
    for (int j = 0; j < kPoolStreams; j++) {
        if ((e = cudaEventRecord(pool->join[j], pool->s[j])) != cudaSuccess) return cuda_fail(e, "join");
        if ((e = cudaStreamWaitEvent(st, pool->join[j], 0)) != cudaSuccess) return cuda_fail(e, "join");
    }
    // 3. the grid-dominance kernel: one launch per (d, slots) over all those instances
    int launch = 0;
    for (int d = 1; d <= gres::kMaxD; d++) {
        for (int slots : {4, 8}) {
            std::vector<gres::DomQuery> qs;
            for (int32_t i = 0; i < n_inst; i++) {
                const gres_instance &x = inst[i];
                if (x.d != d || plans[(size_t)i].slots != slots || x.n == 0) continue;
                gres::DomQuery q;
                q.cand = ws[(size_t)i].cand;
                q.tmin = ws[(size_t)i].tmin;
                q.smin = ws[(size_t)i].smin;
                q.perm = ws[(size_t)i].perm;
                q.n_sky = &ws[(size_t)i].hdr->n_sky;
                q.magic = ws[(size_t)i].magic;
                q.steps = x.d_steps;
                q.out = x.d_step_idx;
                q.K = x.k;
                q.dir = x.dir;
                if (plans[(size_t)i].flags & GRES_FLAG_GRES_REPS) q.ub = ws[(size_t)i].res;
                qs.push_back(q);
            }
            for (size_t off = 0; off < qs.size(); off += 256) {
                const int cnt = (int)std::min<size_t>(256, qs.size() - off);
                e = gres::launch_dominance_batch(d, slots, qs.data() + off, cnt, counters + 16 + launch, st);
                if (e != cudaSuccess) return cuda_fail(e, "batch dominance");
                launch++;
            }
        }
    }
    return GRES_OK;
}

}  // extern "C"
