// kc_server: continuous-batching k-clique query server behind the C ABI (declared in
// include/kclique.h).  Host code: threads, queues, admission; every count, listing and
// prepare it runs is a call of this library's own GPU entry points (or of a caller's
// stand-in backend, for testing the scheduling without a GPU).
//
// Threads:
//   * the query worker runs every count request waiting when the previous batch ended
//     as ONE kclique_count_batch call (continuous batching, at most max_batch per call);
//   * list workers (list_workers of them, each with its own CUDA stream and device row
//     buffer) write the rows of listing requests with KC_ROWS_ONLY; a listing whose buffer
//     filled gets its exact totals from a count entry that joins the next batch;
//   * upload workers (upload_workers of them, each with its own stream) prepare uploaded
//     graphs, after admitting them against the HBM budget (least-recently-used unpinned
//     graphs that no request waits on are released to make room; an upload that still
//     does not fit is rejected).
// Counts, listings and prepares run on different streams, so their work overlaps on the
// device where the SMs have room.  A batch's persistent kernels fill every SM until its
// slowest query ends, so short work goes first: while uploads or listings are queued or
// running, the next batch waits for them (at most yield_ms).  Prepared graphs stay
// resident across requests.  There is no result cache.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "kc_internal.cuh"

namespace {

double now_s() {
    using namespace std::chrono;
    return duration_cast<duration<double>>(steady_clock::now().time_since_epoch()).count();
}

// ------------------------------------------------------------------ the GPU backend
struct GpuBackend {
    int device = 0;
    cudaStream_t qstream = nullptr;
    kc_params params;
};

// per list- or upload-worker thread: a stream and a device row buffer, freed when the
// thread ends
struct WorkerState {
    int device = -1;
    cudaStream_t stream = nullptr;
    uint32_t *d_rows = nullptr;
    uint64_t bytes = 0;
    ~WorkerState() {
        if (device >= 0) {
            cudaSetDevice(device);
            if (d_rows) cudaFree(d_rows);
            if (stream) cudaStreamDestroy(stream);
        }
    }
};
thread_local WorkerState t_worker;

// the calling worker thread's stream, created on first use
kc_status worker_stream(const GpuBackend *b, cudaStream_t *s) {
    WorkerState &w = t_worker;
    if (w.device < 0) {
        KC_CUDA(cudaStreamCreateWithFlags(&w.stream, cudaStreamNonBlocking));
        w.device = b->device;
    }
    *s = w.stream;
    return KC_OK;
}

kc_status gpu_prepare(void *ctx, const uint32_t *row_ptr, const uint32_t *col, uint32_t n, uint64_t nnz,
                      void **graph, uint64_t *bytes) {
    GpuBackend *b = (GpuBackend *)ctx;
    KC_CUDA(cudaSetDevice(b->device));
    cudaStream_t s;
    kc_status st = worker_stream(b, &s);
    if (st != KC_OK) return st;
    kc_graph *g = nullptr;
    st = kclique_prepare(row_ptr, col, n, nnz, 0, (kc_stream)s, &g);
    if (st != KC_OK) return st;
    *graph = g;
    *bytes = g->resident_bytes;
    return KC_OK;
}

kc_status gpu_count_batch(void *ctx, void *const *graphs, const uint32_t *ks, const kc_params *qp, uint32_t nq,
                          kc_result *results) {
    GpuBackend *b = (GpuBackend *)ctx;
    KC_CUDA(cudaSetDevice(b->device));
    kc_params p = b->params;
    p.flags |= KC_CHECKSUM;
    return kclique_count_batch_tuned((const kc_graph *const *)graphs, ks, qp, nq, &p, (kc_stream)b->qstream,
                                     results);
}

kc_status gpu_list(void *ctx, void *graph, uint32_t k, uint32_t *rows, uint64_t cap, kc_result *r) {
    GpuBackend *b = (GpuBackend *)ctx;
    KC_CUDA(cudaSetDevice(b->device));
    cudaStream_t s;
    kc_status st0 = worker_stream(b, &s);
    if (st0 != KC_OK) return st0;
    WorkerState &w = t_worker;
    const uint64_t need = sizeof(uint32_t) * (uint64_t)k * (cap ? cap : 1);
    if (need > w.bytes) {
        if (w.d_rows) KC_CUDA(cudaFree(w.d_rows));
        w.d_rows = nullptr;
        w.bytes = 0;
        KC_CUDA(cudaMalloc(&w.d_rows, need));
        w.bytes = need;
    }
    kc_params p = b->params;
    p.flags |= KC_ROWS_ONLY;
    kc_status st = kclique_list((const kc_graph *)graph, k, w.d_rows, cap, &p, (kc_stream)w.stream, r);
    if (st != KC_OK && st != KC_TRUNCATED) return st;
    if (rows && r->written) {
        KC_CUDA(cudaMemcpyAsync(rows, w.d_rows, sizeof(uint32_t) * (uint64_t)k * r->written, cudaMemcpyDeviceToHost,
                                w.stream));
        KC_CUDA(cudaStreamSynchronize(w.stream));
    }
    return st;
}

void gpu_release(void *ctx, void *graph) {
    GpuBackend *b = (GpuBackend *)ctx;
    cudaSetDevice(b->device);
    kclique_release((kc_graph *)graph);
}

// ------------------------------------------------------------------ server state
struct Req {
    uint64_t ticket = 0;
    kc_request r;
    std::vector<uint32_t> rp, col;  // upload: the CSR, copied at submit
    double t_submit = 0;
    bool totals = false;             // the totals entry of a truncated listing
    kc_completion partial;           // ... and the listing's own completion so far
};

struct Graph {
    void *h = nullptr;
    uint64_t bytes = 0;
    bool pinned = false;
    bool ready = false;
    uint32_t waiting = 0;            // requests queued, parked or running on it
    uint64_t lru = 0;                // last-use stamp
    std::vector<Req *> parked;       // requests that arrived before its upload finished
};

}  // namespace

struct kc_server {
    kc_server_config cfg;
    kc_server_backend be;
    GpuBackend gpu;
    bool own_gpu = false;

    std::mutex mu;
    std::condition_variable cv;       // work arrived / state changed
    std::condition_variable done_cv;  // a completion arrived
    std::deque<Req *> countq, listq, uploadq;
    std::deque<kc_completion> done;
    std::unordered_map<uint64_t, Graph> graphs;
    uint64_t next_ticket = 1, next_graph = 1, lru_clock = 0;
    uint64_t reserved = 0;            // estimated bytes of uploads being prepared
    uint64_t inflight = 0;            // submitted, not yet completed
    uint32_t short_running = 0;       // uploads and listings on the GPU now
    bool stop = false;
    kc_server_counters st;
    std::vector<std::thread> threads;

    uint64_t resident() const {
        uint64_t b = reserved;
        for (const auto &kv : graphs) b += kv.second.bytes;
        return b;
    }
};

namespace {

void complete_locked(kc_server *sv, const kc_completion &c) {
    sv->done.push_back(c);
    sv->st.completed++;
    sv->inflight--;
    sv->done_cv.notify_all();
    sv->cv.notify_all();
}

kc_completion base_completion(const Req *q) {
    kc_completion c;
    memset(&c, 0, sizeof(c));
    c.ticket = q->ticket;
    c.graph = q->r.graph;
    c.kind = q->r.kind;
    c.k = q->r.k;
    c.t_submit = q->t_submit;
    return c;
}

void finish_locked(kc_server *sv, Req *q, kc_status status, const kc_result *r) {
    kc_completion c = q->totals ? q->partial : base_completion(q);
    if (r) {
        c.count_lo = r->count_lo;
        c.count_hi = r->count_hi;
        c.checksum = r->checksum;
        if (!q->totals) c.written = r->written;
    }
    if (status != KC_OK || !q->totals) c.status = status;
    c.t_done = now_s();
    complete_locked(sv, c);
    delete q;
}

// a query on a ready graph goes to its queue (lock held)
void enqueue_ready_locked(kc_server *sv, Req *q) {
    if (q->r.kind == KC_REQ_LIST) sv->listq.push_back(q);
    else sv->countq.push_back(q);
    sv->cv.notify_all();
}

// release LRU unpinned graphs nobody waits on until `need` more bytes fit (lock held);
// nothing is released when even releasing all of them would not make room
bool evict_for_locked(kc_server *sv, uint64_t need) {
    const uint64_t budget = sv->cfg.hbm_budget_bytes;
    uint64_t freeable = 0;
    for (auto &kv : sv->graphs)
        if (!kv.second.pinned && kv.second.ready && kv.second.waiting == 0) freeable += kv.second.bytes;
    if (sv->resident() + need > budget + freeable) return false;
    while (sv->resident() + need > budget) {
        uint64_t victim = 0, best = ~0ull;
        for (auto &kv : sv->graphs) {
            const Graph &g = kv.second;
            if (!g.pinned && g.ready && g.waiting == 0 && g.lru < best) { best = g.lru; victim = kv.first; }
        }
        if (!victim) return false;
        Graph g = sv->graphs[victim];
        sv->graphs.erase(victim);
        sv->st.evictions++;
        sv->be.release(sv->be.ctx, g.h);
    }
    return true;
}

uint64_t estimate_bytes(uint32_t n, uint64_t nnz) {
    // resident arrays (CSR, per-slot ids and rounds, per-edge arrays, VSet) with a
    // triangle allowance of 4 per edge, plus the prepare temporaries
    return 4ull * (n + 1) + 12ull * nnz + 28ull * (nnz / 2) + 16ull * nnz;
}

void upload_worker(kc_server *sv) {
    std::unique_lock<std::mutex> lk(sv->mu);
    while (true) {
        sv->cv.wait(lk, [&] { return sv->stop || !sv->uploadq.empty(); });
        if (sv->uploadq.empty()) return;
        Req *q = sv->uploadq.front();
        sv->uploadq.pop_front();
        const uint64_t gid = q->r.graph;
        const uint64_t need = estimate_bytes(q->r.n, q->r.nnz);
        if (!evict_for_locked(sv, need)) {
            sv->st.rejected++;
            Graph g = sv->graphs[gid];
            sv->graphs.erase(gid);
            for (Req *p : g.parked) finish_locked(sv, p, KC_ERR_OOM, nullptr);
            finish_locked(sv, q, KC_ERR_OOM, nullptr);
            continue;
        }
        sv->reserved += need;
        sv->short_running++;
        lk.unlock();
        const double t0 = now_s();
        void *h = nullptr;
        uint64_t bytes = 0;
        kc_status st = sv->be.prepare(sv->be.ctx, q->rp.data(), q->col.data(), q->r.n, q->r.nnz, &h, &bytes);
        lk.lock();
        sv->short_running--;
        sv->st.busy_upload_s += now_s() - t0;
        sv->reserved -= need;
        Graph &g = sv->graphs[gid];
        std::vector<Req *> parked;
        parked.swap(g.parked);
        if (st != KC_OK) {
            sv->graphs.erase(gid);
            for (Req *p : parked) finish_locked(sv, p, st, nullptr);
        } else {
            g.h = h;
            g.bytes = bytes;
            g.ready = true;
            g.lru = ++sv->lru_clock;
            for (Req *p : parked) enqueue_ready_locked(sv, p);
        }
        finish_locked(sv, q, st, nullptr);
    }
}

void query_worker(kc_server *sv) {
    std::unique_lock<std::mutex> lk(sv->mu);
    std::vector<Req *> batch;
    std::vector<void *> hs;
    std::vector<uint32_t> ks;
    std::vector<kc_params> qp;
    std::vector<kc_result> res;
    while (true) {
        sv->cv.wait(lk, [&] { return !sv->countq.empty() || (sv->stop && sv->inflight == 0); });
        if (sv->countq.empty()) return;
        if (sv->cfg.yield_ms != KC_SERVER_NO_YIELD) {
            // short work first (uploads, listings): for a while, they take the SMs first
            const auto until = std::chrono::steady_clock::now() + std::chrono::milliseconds(sv->cfg.yield_ms);
            sv->cv.wait_until(lk, until, [&] {
                return sv->short_running == 0 && sv->uploadq.empty() && sv->listq.empty();
            });
        }
        batch.clear();
        hs.clear();
        ks.clear();
        qp.clear();
        while (!sv->countq.empty() && batch.size() < sv->cfg.max_batch) {
            Req *q = sv->countq.front();
            sv->countq.pop_front();
            Graph &g = sv->graphs[q->r.graph];
            g.lru = ++sv->lru_clock;
            batch.push_back(q);
            hs.push_back(g.h);
            ks.push_back(q->r.k);
            kc_params c;
            memset(&c, 0, sizeof(c));
            c.t_max = q->r.t_max ? q->r.t_max : sv->cfg.params.t_max;
            c.split_min = q->r.split_min ? q->r.split_min : sv->cfg.params.split_min;
            c.width_min = q->r.width_min ? q->r.width_min : sv->cfg.params.width_min;
            qp.push_back(c);
        }
        sv->st.batches++;
        sv->st.batched_queries += batch.size();
        sv->st.max_batch_seen = std::max<uint64_t>(sv->st.max_batch_seen, batch.size());
        lk.unlock();
        res.assign(batch.size(), kc_result());
        const double t0 = now_s();
        kc_status st =
            sv->be.count_batch(sv->be.ctx, hs.data(), ks.data(), qp.data(), (uint32_t)batch.size(), res.data());
        lk.lock();
        sv->st.busy_count_s += now_s() - t0;
        for (size_t i = 0; i < batch.size(); i++) {
            Graph &g = sv->graphs[batch[i]->r.graph];
            g.waiting--;
            finish_locked(sv, batch[i], st, st == KC_OK ? &res[i] : nullptr);
        }
    }
}

void list_worker(kc_server *sv) {
    std::unique_lock<std::mutex> lk(sv->mu);
    while (true) {
        sv->cv.wait(lk, [&] { return !sv->listq.empty() || (sv->stop && sv->inflight == 0); });
        if (sv->listq.empty()) return;
        Req *q = sv->listq.front();
        sv->listq.pop_front();
        Graph &g = sv->graphs[q->r.graph];
        g.lru = ++sv->lru_clock;
        void *h = g.h;
        sv->short_running++;
        lk.unlock();
        kc_result r;
        memset(&r, 0, sizeof(r));
        const double t0 = now_s();
        kc_status st = sv->be.list(sv->be.ctx, h, q->r.k, q->r.rows, q->r.cap, &r);
        lk.lock();
        sv->short_running--;
        sv->st.busy_list_s += now_s() - t0;
        if (st == KC_TRUNCATED && r.written >= q->r.cap) {
            // the buffer filled before the pass ended: the exact totals come from a count
            // entry in the next batch; the graph stays held until then
            q->partial = base_completion(q);
            q->partial.written = r.written;
            q->partial.status = KC_TRUNCATED;
            q->totals = true;
            sv->countq.push_back(q);
            sv->cv.notify_all();
            continue;
        }
        sv->graphs[q->r.graph].waiting--;
        if (st == KC_OK && r.written > q->r.cap) r.written = q->r.cap;
        finish_locked(sv, q, st, (st == KC_OK || st == KC_TRUNCATED) ? &r : nullptr);
    }
}

}  // namespace

extern "C" {

kc_status kc_server_create(const kc_server_config *cfg, kc_server **out) {
    if (!out) return KC_ERR_INVALID_ARG;
    *out = nullptr;
    kc_server *sv = new kc_server();
    memset(&sv->cfg, 0, sizeof(sv->cfg));
    if (cfg) sv->cfg = *cfg;
    if (!sv->cfg.hbm_budget_bytes) sv->cfg.hbm_budget_bytes = 120ull << 30;
    if (!sv->cfg.max_batch) sv->cfg.max_batch = 512;
    if (!sv->cfg.list_workers) sv->cfg.list_workers = 4;
    if (!sv->cfg.upload_workers) sv->cfg.upload_workers = 4;
    if (!sv->cfg.yield_ms) sv->cfg.yield_ms = 1000;
    if (sv->cfg.params.d_edge_count || sv->cfg.params.d_edge_checksum || sv->cfg.params.d_edge_cycles) {
        delete sv;
        return KC_ERR_INVALID_ARG;
    }
    memset(&sv->st, 0, sizeof(sv->st));
    if (cfg && cfg->backend) {
        sv->be = *cfg->backend;
        if (!sv->be.prepare || !sv->be.count_batch || !sv->be.list || !sv->be.release) {
            delete sv;
            return KC_ERR_INVALID_ARG;
        }
    } else {
        int dev = sv->cfg.device;
        if (dev < 0) {
            cudaError_t e = cudaGetDevice(&dev);
            if (e != cudaSuccess) {
                kc_set_last_cuda_error(e, "cudaGetDevice", __FILE__, __LINE__);
                delete sv;
                return KC_ERR_CUDA;
            }
        }
        sv->gpu.device = dev;
        sv->gpu.params = sv->cfg.params;
        cudaError_t e = cudaSetDevice(dev);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sv->gpu.qstream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            kc_set_last_cuda_error(e, "kc_server_create streams", __FILE__, __LINE__);
            delete sv;
            return KC_ERR_CUDA;
        }
        sv->own_gpu = true;
        sv->be.ctx = &sv->gpu;
        sv->be.prepare = gpu_prepare;
        sv->be.count_batch = gpu_count_batch;
        sv->be.list = gpu_list;
        sv->be.release = gpu_release;
    }
    for (uint32_t i = 0; i < sv->cfg.upload_workers; i++) sv->threads.emplace_back(upload_worker, sv);
    sv->threads.emplace_back(query_worker, sv);
    for (uint32_t i = 0; i < sv->cfg.list_workers; i++) sv->threads.emplace_back(list_worker, sv);
    *out = sv;
    return KC_OK;
}

kc_status kc_server_adopt(kc_server *sv, void *graph, uint64_t resident_bytes, int pin, uint64_t *graph_id) {
    if (!sv || !graph || !graph_id) return KC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(sv->mu);
    const uint64_t gid = sv->next_graph++;
    Graph &g = sv->graphs[gid];
    g.h = graph;
    g.bytes = (sv->own_gpu && !resident_bytes) ? ((kc_graph *)graph)->resident_bytes : resident_bytes;
    g.pinned = pin != 0;
    g.ready = true;
    g.lru = ++sv->lru_clock;
    *graph_id = gid;
    return KC_OK;
}

kc_status kc_server_submit(kc_server *sv, const kc_request *req, uint64_t *ticket, uint64_t *graph_id) {
    if (!sv || !req || !ticket) return KC_ERR_INVALID_ARG;
    *ticket = 0;
    if (graph_id) *graph_id = 0;
    if (req->kind > KC_REQ_UPLOAD) return KC_ERR_INVALID_ARG;
    if (req->kind != KC_REQ_UPLOAD && (req->k < 3 || req->k > KC_MAX_K)) return KC_ERR_INVALID_ARG;
    if (req->kind == KC_REQ_UPLOAD && (!req->row_ptr || (req->nnz && !req->col))) return KC_ERR_INVALID_ARG;
    Req *q = new Req();
    q->r = *req;
    q->t_submit = now_s();
    if (req->kind == KC_REQ_UPLOAD) {
        q->rp.assign(req->row_ptr, req->row_ptr + (size_t)req->n + 1);
        if (req->nnz) q->col.assign(req->col, req->col + req->nnz);
        else q->col.assign(1, 0u);
        q->r.row_ptr = nullptr;
        q->r.col = nullptr;
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    q->ticket = sv->next_ticket++;
    *ticket = q->ticket;
    sv->st.submitted++;
    sv->inflight++;
    if (req->kind == KC_REQ_UPLOAD) {
        const uint64_t gid = sv->next_graph++;
        q->r.graph = gid;
        if (graph_id) *graph_id = gid;
        Graph &g = sv->graphs[gid];
        g.pinned = req->pin != 0;
        sv->uploadq.push_back(q);
        sv->cv.notify_all();
        return KC_OK;
    }
    auto it = sv->graphs.find(req->graph);
    if (it == sv->graphs.end()) {
        finish_locked(sv, q, KC_ERR_INVALID_ARG, nullptr);  // unknown graph: completes at once
        return KC_OK;
    }
    if (graph_id) *graph_id = req->graph;
    it->second.waiting++;
    if (it->second.ready) enqueue_ready_locked(sv, q);
    else it->second.parked.push_back(q);
    return KC_OK;
}

uint32_t kc_server_poll(kc_server *sv, kc_completion *out, uint32_t max, int32_t wait_ms) {
    if (!sv || !out || !max) return 0;
    std::unique_lock<std::mutex> lk(sv->mu);
    if (sv->done.empty() && wait_ms != 0) {
        auto ready = [&] { return !sv->done.empty(); };
        if (wait_ms < 0) sv->done_cv.wait(lk, ready);
        else sv->done_cv.wait_for(lk, std::chrono::milliseconds(wait_ms), ready);
    }
    uint32_t n = 0;
    while (n < max && !sv->done.empty()) {
        out[n++] = sv->done.front();
        sv->done.pop_front();
    }
    return n;
}

kc_status kc_server_stats(kc_server *sv, kc_server_counters *st) {
    if (!sv || !st) return KC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(sv->mu);
    *st = sv->st;
    st->resident_bytes = sv->resident();
    st->graphs = sv->graphs.size();
    st->inflight = sv->inflight;
    return KC_OK;
}

void kc_server_destroy(kc_server *sv) {
    if (!sv) return;
    {
        std::unique_lock<std::mutex> lk(sv->mu);
        sv->cv.wait(lk, [&] { return sv->inflight == 0; });  // queued work finishes first
        sv->stop = true;
        sv->cv.notify_all();
    }
    for (auto &t : sv->threads) t.join();
    for (auto &kv : sv->graphs)
        if (kv.second.h) sv->be.release(sv->be.ctx, kv.second.h);
    if (sv->own_gpu) {
        cudaSetDevice(sv->gpu.device);
        cudaStreamDestroy(sv->gpu.qstream);
    }
    delete sv;
}

}  // extern "C"
