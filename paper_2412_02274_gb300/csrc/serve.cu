// serve.cu -- a gres query server: resident datasets, continuous batching.
//
// Datasets are prepared once (skyline + candidate tiles, see batch.cu) and stay
// in device memory within an HBM budget. Queries (a dataset and a step list)
// queue on the host. A scheduler thread keeps up to `max_inflight` batches on
// the GPU: whenever a slot is free it takes up to `max_batch` pending queries
// in queue order and runs them as one batch on the slot's stream -- one copy
// of all their widths, one kernel for their division constants, one
// grid-dominance launch per dimensionality over all their targets, and one
// copy of all results back. A query contributes one piece to a batch: at most
// `chunk_targets` of its targets (a range of skyline positions); if targets
// are left it goes to the back of the queue, so a query on a very large
// skyline is spread over many short batches instead of holding up everything
// queued behind it. Queries that arrive while batches run are admitted as soon
// as a slot frees up, so their work overlaps with the batches already on the
// device. Completion is detected with cudaEventQuery and host condition
// variables: nothing waits on the device.
#include "gres_internal.cuh"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

namespace {

using Clock = std::chrono::steady_clock;

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
gres_status fail(gres_status s, const std::string &m) { return gres::set_error(s, m.c_str()); }
gres_status cuda_fail(cudaError_t e, const char *where) {
    return fail(GRES_ECUDA, std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

struct Query {
    uint64_t ticket = 0;
    int32_t dataset = -1;
    std::vector<uint32_t> steps;
    int64_t S = 0;
    std::vector<int32_t> result;   // S entries, filled piece by piece
    int64_t next = 0;              // first target not yet handed to a batch
    int outstanding = 0;           // pieces on the GPU
    uint64_t last_batch = 0;       // the batch that took its latest piece
    bool queued = false;           // in the pending queue
    bool done = false;
    bool cancelled = false;
    gres_status status = GRES_OK;
    Clock::time_point t_submit, t_done;
};

// Targets [t0, t0 + tn) of a query, in one batch.
struct Piece {
    std::shared_ptr<Query> q;
    int64_t t0 = 0, tn = 0;
};

struct DatasetEntry {
    gres_dataset *ds = nullptr;
    int32_t d = 0, dir = 0, slots = 8;
    int64_t S = 0;
    size_t bytes = 0;
    int pending = 0;        // queries referencing it that are not finished
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    // device buffers
    void *dev = nullptr;    // steps | magic | counters | results
    size_t dev_bytes = 0;
    size_t res_cap = 0;     // int32 results capacity
    // pinned host buffers
    uint32_t *h_steps = nullptr;
    int32_t *h_res = nullptr;
    size_t h_res_cap = 0;
    std::vector<Piece> batch;
    std::vector<size_t> res_off;
};

}  // namespace

struct gres_server {
    int device = 0;
    size_t budget = 0;
    size_t used = 0;        // device bytes in use (datasets + slot buffers)
    gres_serve_cfg cfg;
    std::mutex mu;
    std::condition_variable cv_work;    // scheduler: new queries or stop
    std::condition_variable cv_done;    // pollers: queries finished
    std::deque<std::shared_ptr<Query>> pending;
    std::unordered_map<uint64_t, std::shared_ptr<Query>> tickets;
    std::map<int32_t, DatasetEntry> datasets;
    int32_t next_dataset = 0;
    uint64_t next_ticket = 1;
    std::vector<Slot> slots;
    std::thread worker;
    bool stop = false;
    bool paused = false;
    gres_status worker_error = GRES_OK;
    std::string worker_message;
    uint64_t next_batch = 1;
    // statistics
    unsigned long long n_batches = 0, n_queries = 0, n_launches = 0;
};

namespace {

// Slot buffer layout for `cap_res` result entries.
size_t slot_dev_bytes(const gres_serve_cfg &c, size_t cap_res) {
    const size_t steps = align256(4 * (size_t)c.max_batch * c.max_k);
    const size_t magic = align256(16 * (size_t)c.max_batch * c.max_k);
    const size_t counters = align256(4 * 64);
    return steps + magic + counters + align256(4 * (cap_res ? cap_res : 1));
}

// Grows a free slot's result buffers to `cap` entries (scheduler thread, lock held).
gres_status slot_reserve(gres_server *sv, Slot &sl, size_t cap) {
    if (cap <= sl.res_cap && sl.dev) return GRES_OK;
    const size_t bytes = slot_dev_bytes(sv->cfg, cap);
    if (sv->used - sl.dev_bytes + bytes > sv->budget) return fail(GRES_ENOMEM, "serve: results exceed the HBM budget");
    if (sl.dev) cudaFree(sl.dev);
    sv->used -= sl.dev_bytes;
    sl.dev = nullptr;
    sl.dev_bytes = 0;
    sl.res_cap = 0;
    cudaError_t e = cudaMalloc(&sl.dev, bytes);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? fail(GRES_ENOMEM, "serve: out of device memory")
                                                                 : cuda_fail(e, "serve slot");
    sl.dev_bytes = bytes;
    sl.res_cap = cap;
    sv->used += bytes;
    if (sl.h_res_cap < cap) {
        if (sl.h_res) cudaFreeHost(sl.h_res);
        e = cudaMallocHost(&sl.h_res, 4 * cap);
        if (e != cudaSuccess) { sl.h_res = nullptr; sl.h_res_cap = 0; return cuda_fail(e, "serve pinned results"); }
        sl.h_res_cap = cap;
    }
    return GRES_OK;
}

// Launches the slot's batch (scheduler thread, lock NOT held).
gres_status launch_batch(gres_server *sv, Slot &sl, const std::vector<DatasetEntry> &dsv) {
    const gres_serve_cfg &c = sv->cfg;
    char *base = static_cast<char *>(sl.dev);
    uint32_t *d_steps = reinterpret_cast<uint32_t *>(base);
    uint32_t *d_magic = reinterpret_cast<uint32_t *>(base + align256(4 * (size_t)c.max_batch * c.max_k));
    unsigned *d_count = reinterpret_cast<unsigned *>(base + align256(4 * (size_t)c.max_batch * c.max_k) +
                                                     align256(16 * (size_t)c.max_batch * c.max_k));
    int32_t *d_res = reinterpret_cast<int32_t *>(reinterpret_cast<char *>(d_count) + align256(4 * 64));
    // widths, packed
    std::vector<size_t> soff(sl.batch.size());
    size_t total_k = 0, total_s = 0;
    sl.res_off.assign(sl.batch.size(), 0);
    for (size_t i = 0; i < sl.batch.size(); i++) {
        const Query &qq = *sl.batch[i].q;
        soff[i] = total_k;
        std::memcpy(sl.h_steps + total_k, qq.steps.data(), 4 * qq.steps.size());
        total_k += qq.steps.size();
        sl.res_off[i] = total_s;
        total_s += (size_t)sl.batch[i].tn;
    }
    cudaError_t e = cudaMemcpyAsync(d_steps, sl.h_steps, 4 * total_k, cudaMemcpyHostToDevice, sl.stream);
    if (e != cudaSuccess) return cuda_fail(e, "serve steps");
    e = cudaMemsetAsync(d_count, 0, 4 * 64, sl.stream);
    if (e != cudaSuccess) return cuda_fail(e, "serve counters");
    std::vector<gres::MagicJob> jobs(sl.batch.size());
    for (size_t i = 0; i < sl.batch.size(); i++)
        jobs[i] = {d_steps + soff[i], d_magic + 4 * soff[i], (int)sl.batch[i].q->steps.size(), nullptr};
    e = gres::launch_make_magic(jobs.data(), (int)jobs.size(), sl.stream);
    if (e != cudaSuccess) return cuda_fail(e, "serve constants");
    sv->n_launches += 1 + (jobs.size() + 255) / 256;
    int launch = 0;
    for (int d = 1; d <= gres::kMaxD; d++) {
        for (int slots : {4, 8}) {
            std::vector<gres::DomQuery> qs;
            for (size_t i = 0; i < sl.batch.size(); i++) {
                const DatasetEntry &de = dsv[i];
                if (de.d != d || de.slots != slots || sl.batch[i].tn == 0) continue;
                const gres_dataset *ds = de.ds;
                gres::DomQuery q;
                q.cand = ds->cand;
                q.tmin = ds->tmin;
                q.smin = ds->smin;
                q.perm = ds->perm;
                q.n_sky = ds->n_sky;
                q.magic = d_magic + 4 * soff[i];
                q.steps = d_steps + soff[i];
                q.out = d_res + sl.res_off[i];
                q.K = (int)sl.batch[i].q->steps.size();
                q.dir = de.dir;
                q.iperm = ds->iperm;
                q.t0 = (unsigned)sl.batch[i].t0;
                q.tn = (unsigned)sl.batch[i].tn;
                qs.push_back(q);
            }
            for (size_t off = 0; off < qs.size(); off += 256) {
                if (launch >= 64) return fail(GRES_EINTERNAL, "serve: too many launches in one batch");
                const int cnt = (int)std::min<size_t>(256, qs.size() - off);
                e = gres::launch_dominance_batch(d, slots, qs.data() + off, cnt, d_count + launch, sl.stream);
                if (e != cudaSuccess) return cuda_fail(e, "serve dominance");
                launch++;
                sv->n_launches++;
            }
        }
    }
    if (total_s) {
        e = cudaMemcpyAsync(sl.h_res, d_res, 4 * total_s, cudaMemcpyDeviceToHost, sl.stream);
        if (e != cudaSuccess) return cuda_fail(e, "serve results");
    }
    e = cudaEventRecord(sl.done, sl.stream);
    return e == cudaSuccess ? GRES_OK : cuda_fail(e, "serve event");
}

// Marks a query finished (lock held).
void complete(gres_server *sv, Query &q, gres_status st) {
    q.status = q.cancelled ? GRES_EINVAL : st;
    q.done = true;
    q.t_done = Clock::now();
    auto it = sv->datasets.find(q.dataset);
    if (it != sv->datasets.end()) it->second.pending--;
    if (q.cancelled) sv->tickets.erase(q.ticket);
    sv->n_queries++;
}

// Removes a query from the pending queue (lock held).
void unqueue(gres_server *sv, const std::shared_ptr<Query> &q) {
    for (auto p = sv->pending.begin(); p != sv->pending.end(); ++p)
        if (*p == q) { sv->pending.erase(p); break; }
    q->queued = false;
}

void finish_batch(gres_server *sv, Slot &sl, gres_status st) {
    // lock held
    for (size_t i = 0; i < sl.batch.size(); i++) {
        Piece &pc = sl.batch[i];
        Query &q = *pc.q;
        q.outstanding--;
        if (q.done) continue;
        if (st != GRES_OK && q.status == GRES_OK) q.status = st;
        if (q.status == GRES_OK && !q.cancelled && pc.tn > 0)
            std::memcpy(q.result.data() + pc.t0, sl.h_res + sl.res_off[i], 4 * (size_t)pc.tn);
        // a failed piece fails the query and a cancelled query takes no more
        // pieces; either ends when its last piece in flight comes back
        const bool ended = q.status != GRES_OK || q.cancelled;
        if (ended && q.queued) unqueue(sv, pc.q);
        if (q.outstanding == 0 && (ended || q.next == q.S)) complete(sv, q, q.status);
    }
    sv->n_batches++;
    sl.batch.clear();
    sl.busy = false;
}

void worker_main(gres_server *sv) {
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lock(sv->mu);
    for (;;) {
        // retire finished batches
        bool any_busy = false;
        for (Slot &sl : sv->slots) {
            if (!sl.busy) continue;
            const cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaSuccess) {
                finish_batch(sv, sl, GRES_OK);
                sv->cv_done.notify_all();
            } else if (q != cudaErrorNotReady) {
                finish_batch(sv, sl, GRES_ECUDA);
                sv->worker_error = GRES_ECUDA;
                sv->worker_message = cudaGetErrorString(q);
                sv->cv_done.notify_all();
            } else {
                any_busy = true;
            }
        }
        // start batches on free slots
        for (Slot &sl : sv->slots) {
            if (sl.busy || sv->paused) continue;
            while (!sv->pending.empty() && sv->pending.front()->cancelled) sv->pending.pop_front();
            if (sv->pending.empty()) break;
            std::vector<DatasetEntry> dsv;
            size_t need = 0;
            const uint64_t bid = sv->next_batch++;
            while (!sv->pending.empty() && (int)sl.batch.size() < sv->cfg.max_batch) {
                auto q = sv->pending.front();
                if (q->last_batch == bid) break;   // the queue came round: one piece per query per batch
                sv->pending.pop_front();
                q->queued = false;
                if (q->cancelled) continue;
                const DatasetEntry &de = sv->datasets.at(q->dataset);
                const int64_t left = q->S - q->next;
                const int64_t tn = sv->cfg.chunk_targets > 0 ? std::min<int64_t>(left, sv->cfg.chunk_targets) : left;
                sl.batch.push_back(Piece{q, q->next, tn});
                dsv.push_back(de);
                q->next += tn;
                q->outstanding++;
                q->last_batch = bid;
                need += (size_t)tn;
                if (q->next < q->S) {
                    sv->pending.push_back(q);
                    q->queued = true;
                }
            }
            if (sl.batch.empty()) break;
            gres_status st = slot_reserve(sv, sl, std::max<size_t>(need, 1));
            if (st == GRES_OK) {
                sl.busy = true;
                lock.unlock();
                st = launch_batch(sv, sl, dsv);
                lock.lock();
            }
            if (st != GRES_OK) {
                sl.busy = true;
                finish_batch(sv, sl, st);
                sv->cv_done.notify_all();
            } else {
                any_busy = true;
            }
        }
        if (sv->stop && !any_busy) break;
        if (any_busy) {
            // batches on the GPU: look again shortly (or when new work arrives)
            sv->cv_work.wait_for(lock, std::chrono::microseconds(20));
        } else if (!sv->stop && (sv->pending.empty() || sv->paused)) {
            sv->cv_work.wait(lock, [&] { return sv->stop || (!sv->pending.empty() && !sv->paused); });
        }
    }
}

}  // namespace

extern "C" {

gres_status gres_serve_create(size_t hbm_budget_bytes, const gres_serve_cfg *cfg, gres_server **out) {
    if (!out) return fail(GRES_EINVAL, "out is NULL");
    *out = nullptr;
    gres_serve_cfg c;
    std::memset(&c, 0, sizeof(c));
    if (cfg) c = *cfg;
    if (c.max_batch == 0) c.max_batch = 64;
    if (c.max_inflight == 0) c.max_inflight = 2;
    if (c.queue_capacity == 0) c.queue_capacity = 1 << 16;
    if (c.max_k == 0) c.max_k = 4096;
    if (c.chunk_targets == 0) c.chunk_targets = 16384;
    if (c.max_batch < 1 || c.max_batch > 256) return fail(GRES_EINVAL, "max_batch must be in [1, 256]");
    if (c.max_inflight < 1 || c.max_inflight > 16) return fail(GRES_EINVAL, "max_inflight must be in [1, 16]");
    if (c.queue_capacity < 1) return fail(GRES_EINVAL, "queue_capacity must be >= 1");
    if (c.max_k < 1 || c.max_k > (1 << 20)) return fail(GRES_EINVAL, "max_k must be in [1, 2^20]");
    const size_t slot_min = slot_dev_bytes(c, 1);
    if (hbm_budget_bytes < slot_min * (size_t)c.max_inflight)
        return fail(GRES_ENOMEM, "serve: the HBM budget does not cover the batch slots");
    auto sv = std::make_unique<gres_server>();
    cudaError_t e = cudaGetDevice(&sv->device);
    if (e != cudaSuccess) return cuda_fail(e, "serve device");
    sv->budget = hbm_budget_bytes;
    sv->cfg = c;
    sv->paused = c.start_paused != 0;
    sv->slots.resize((size_t)c.max_inflight);
    for (Slot &sl : sv->slots) {
        if ((e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking)) != cudaSuccess) break;
        if ((e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming)) != cudaSuccess) break;
        if ((e = cudaMallocHost(&sl.h_steps, 4 * (size_t)c.max_batch * c.max_k)) != cudaSuccess) break;
        gres_status st = slot_reserve(sv.get(), sl, 1);
        if (st != GRES_OK) { gres_serve_destroy(sv.release()); return st; }
    }
    if (e != cudaSuccess) { gres_serve_destroy(sv.release()); return cuda_fail(e, "serve setup"); }
    sv->worker = std::thread(worker_main, sv.get());
    *out = sv.release();
    return GRES_OK;
}

gres_status gres_serve_add_dataset(gres_server *sv, const uint32_t *data, int64_t n, int32_t d, int32_t dir,
                                   const gres_plan_cfg *plan, int32_t data_on_host, int32_t *out_id) {
    if (!sv || !out_id) return fail(GRES_EINVAL, "server / out_id is NULL");
    // Prepared on a private stream; the budget counts the handle's bytes plus the
    // results room its queries need in every slot.
    cudaStream_t st = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "serve stream");
    gres_dataset *ds = nullptr;
    gres_status s = gres_dataset_create(data, n, d, dir, plan, data_on_host, st, &ds);
    cudaStreamDestroy(st);
    if (s != GRES_OK) return s;
    std::lock_guard<std::mutex> lock(sv->mu);
    const int64_t piece = sv->cfg.chunk_targets > 0 ? std::min<int64_t>(ds->S, sv->cfg.chunk_targets) : ds->S;
    const size_t extra = 4 * (size_t)piece * (size_t)sv->cfg.max_batch * sv->slots.size();
    if (sv->used + ds->bytes + extra > sv->budget) {
        gres_dataset_destroy(ds);
        return fail(GRES_ENOMEM, "serve: dataset exceeds the HBM budget");
    }
    DatasetEntry de;
    de.ds = ds;
    de.d = ds->d;
    de.dir = ds->dir;
    de.slots = ds->slots;
    de.S = ds->S;
    de.bytes = ds->bytes;
    sv->used += ds->bytes;
    const int32_t id = sv->next_dataset++;
    sv->datasets[id] = de;
    *out_id = id;
    return GRES_OK;
}

gres_status gres_serve_remove_dataset(gres_server *sv, int32_t id) {
    if (!sv) return fail(GRES_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> lock(sv->mu);
    auto it = sv->datasets.find(id);
    if (it == sv->datasets.end()) return fail(GRES_EINVAL, "no such dataset");
    if (it->second.pending > 0) return fail(GRES_EAGAIN, "dataset has queries in progress");
    sv->used -= it->second.bytes;
    gres_dataset_destroy(it->second.ds);
    sv->datasets.erase(it);
    return GRES_OK;
}

gres_status gres_serve_submit(gres_server *sv, int32_t dataset_id, const uint32_t *h_steps, int32_t k,
                              uint64_t *out_ticket) {
    if (!sv || !out_ticket) return fail(GRES_EINVAL, "server / out_ticket is NULL");
    if (!h_steps || k < 1) return fail(GRES_EINVAL, "empty step list");
    if (k > sv->cfg.max_k) return fail(GRES_EINVAL, "step list longer than the server's max_k");
    if (h_steps[0] < 1) return fail(GRES_EINVAL, "steps must be >= 1");
    for (int32_t i = 1; i < k; i++)
        if (h_steps[i] <= h_steps[i - 1]) return fail(GRES_EINVAL, "steps must be strictly ascending");
    auto q = std::make_shared<Query>();
    q->steps.assign(h_steps, h_steps + k);
    q->dataset = dataset_id;
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        if (sv->worker_error != GRES_OK) return fail(sv->worker_error, "serve: " + sv->worker_message);
        auto it = sv->datasets.find(dataset_id);
        if (it == sv->datasets.end()) return fail(GRES_EINVAL, "no such dataset");
        if ((int64_t)sv->pending.size() >= sv->cfg.queue_capacity) return fail(GRES_EAGAIN, "serve: queue full");
        q->S = it->second.S;
        q->result.assign((size_t)q->S, 0);
        q->ticket = sv->next_ticket++;
        q->t_submit = Clock::now();
        it->second.pending++;
        sv->tickets[q->ticket] = q;
        sv->pending.push_back(q);
        q->queued = true;
        *out_ticket = q->ticket;
    }
    sv->cv_work.notify_one();
    return GRES_OK;
}

gres_status gres_serve_poll(gres_server *sv, uint64_t ticket, int32_t *h_step_idx, int64_t cap,
                            int64_t *h_sky_count, int64_t *h_latency_ns, int64_t timeout_us) {
    if (!sv) return fail(GRES_EINVAL, "server is NULL");
    std::unique_lock<std::mutex> lock(sv->mu);
    auto it = sv->tickets.find(ticket);
    if (it == sv->tickets.end()) return fail(GRES_EINVAL, "unknown ticket");
    std::shared_ptr<Query> q = it->second;
    if (q->cancelled) return fail(GRES_EINVAL, "query was cancelled");
    if (!q->done && timeout_us != 0) {
        auto pred = [&] { return q->done; };
        if (timeout_us < 0) sv->cv_done.wait(lock, pred);
        else sv->cv_done.wait_for(lock, std::chrono::microseconds(timeout_us), pred);
    }
    if (!q->done) return fail(GRES_EAGAIN, "query not finished");
    if (q->status != GRES_OK) {
        sv->tickets.erase(ticket);
        return fail(q->status, "query failed");
    }
    if (h_sky_count) *h_sky_count = q->S;
    if (h_latency_ns)
        *h_latency_ns = std::chrono::duration_cast<std::chrono::nanoseconds>(q->t_done - q->t_submit).count();
    if (q->S > 0) {
        if (!h_step_idx || cap < q->S) return fail(GRES_EINVAL, "result buffer too small (need sky_count)");
        std::memcpy(h_step_idx, q->result.data(), 4 * (size_t)q->S);
    }
    sv->tickets.erase(ticket);
    return GRES_OK;
}

gres_status gres_serve_sky_idx(gres_server *sv, int32_t dataset_id, int64_t *h_sky_idx, int64_t cap,
                               int64_t *h_sky_count) {
    if (!sv) return fail(GRES_EINVAL, "server is NULL");
    const gres_dataset *ds = nullptr;
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        auto it = sv->datasets.find(dataset_id);
        if (it == sv->datasets.end()) return fail(GRES_EINVAL, "no such dataset");
        ds = it->second.ds;
        if (h_sky_count) *h_sky_count = it->second.S;
        if (it->second.S > 0 && (!h_sky_idx || cap < it->second.S))
            return fail(GRES_EINVAL, "index buffer too small (need sky_count)");
        if (it->second.S == 0) return GRES_OK;
        // the copy runs outside the lock; the caller keeps the dataset (no remove) meanwhile
        it->second.pending++;
    }
    cudaStream_t st = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    gres_status r = e == cudaSuccess ? gres_dataset_sky_idx(ds, h_sky_idx, 1, st) : cuda_fail(e, "serve stream");
    if (st) cudaStreamDestroy(st);
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        auto it = sv->datasets.find(dataset_id);
        if (it != sv->datasets.end()) it->second.pending--;
    }
    return r;
}

gres_status gres_serve_resume(gres_server *sv) {
    if (!sv) return fail(GRES_EINVAL, "server is NULL");
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        sv->paused = false;
    }
    sv->cv_work.notify_all();
    return GRES_OK;
}

gres_status gres_serve_pause(gres_server *sv) {
    if (!sv) return fail(GRES_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> lock(sv->mu);
    sv->paused = true;
    return GRES_OK;
}

gres_status gres_serve_cancel(gres_server *sv, uint64_t ticket) {
    if (!sv) return fail(GRES_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> lock(sv->mu);
    auto it = sv->tickets.find(ticket);
    if (it == sv->tickets.end()) return fail(GRES_EINVAL, "unknown ticket");
    std::shared_ptr<Query> q = it->second;
    if (q->done) return fail(GRES_EINVAL, "query already finished");
    q->cancelled = true;
    // nothing on the GPU: drop it now; pieces in flight: it ends with the last one
    if (q->queued) unqueue(sv, q);
    if (q->outstanding == 0) complete(sv, *q, GRES_EINVAL);
    sv->cv_done.notify_all();
    return GRES_OK;
}

gres_status gres_serve_stats(gres_server *sv, uint64_t *batches, uint64_t *queries, uint64_t *launches,
                             size_t *device_bytes) {
    if (!sv) return fail(GRES_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> lock(sv->mu);
    if (batches) *batches = sv->n_batches;
    if (queries) *queries = sv->n_queries;
    if (launches) *launches = sv->n_launches;
    if (device_bytes) *device_bytes = sv->used;
    return GRES_OK;
}

gres_status gres_serve_destroy(gres_server *sv) {
    if (!sv) return GRES_OK;
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        sv->stop = true;
        for (auto &q : sv->pending) q->cancelled = true;
        sv->pending.clear();
    }
    sv->cv_work.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    for (Slot &sl : sv->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.dev) cudaFree(sl.dev);
        if (sl.h_steps) cudaFreeHost(sl.h_steps);
        if (sl.h_res) cudaFreeHost(sl.h_res);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    for (auto &kv : sv->datasets) gres_dataset_destroy(kv.second.ds);
    delete sv;
    return GRES_OK;
}

}  // extern "C"
