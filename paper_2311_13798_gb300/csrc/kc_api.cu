// C ABI of libkclique (declared in include/kclique.h).
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <vector>

#include "kc_internal.cuh"

static thread_local char g_last_error[512];

void kc_set_last_cuda_error(cudaError_t e, const char *what, const char *file, int line) {
    snprintf(g_last_error, sizeof(g_last_error), "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
}

extern "C" const char *kclique_last_error(void) { return g_last_error; }

void kc_set_last_error_msg(const char *msg) { snprintf(g_last_error, sizeof(g_last_error), "%s", msg); }

static std::atomic<unsigned long long> g_launches{0};

void kc_note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

extern "C" unsigned long long kclique_launch_count(int reset) {
    return reset ? g_launches.exchange(0) : g_launches.load();
}

#ifndef KC_KERNEL_REV
#define KC_KERNEL_REV "unknown"
#endif
extern "C" const char *kclique_kernel_rev(void) { return KC_KERNEL_REV; }

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

// Early-termination threshold: the caller's t_max, or 0 for the paper's rule, which
// the launch code resolves per query from k and tau (kc_pick_t)
u32 pick_t(const kc_params *p) { return p ? p->t_max : 0u; }

kc_status map_device_status(unsigned st) {
    if (st & KC_DEV_ERR_OVERFLOW) return KC_ERR_OVERFLOW;
    if (st & KC_DEV_ERR_WIDTH) return KC_ERR_UNSUPPORTED;
    if (st & KC_DEV_ERR_TIMEOUT) return KC_ERR_TIMEOUT;
    if (st) return KC_ERR_CUDA;
    return KC_OK;
}

u64 suffix_of(const kc_graph *g, u64 x) { return x > g->tau ? 0ull : g->h_size_suffix[x]; }

kc_status check_width(const kc_graph *g, u32 k) {
    u64 lo = std::max<u64>(KC_MAX_BRANCH + 1, (u64)k - 2);
    return suffix_of(g, lo) ? KC_ERR_UNSUPPORTED : KC_OK;
}

kc_status run_one(const kc_graph *g, u32 k, const kc_params *p, cudaStream_t s, kc_result *r, int list, u32 *d_out,
                  u64 cap) {
    if (!g || !r) return KC_ERR_INVALID_ARG;
    memset(r, 0, sizeof(*r));
    if (k < 3 || k > KC_MAX_K) return KC_ERR_INVALID_ARG;
    if (list && cap && !d_out) return KC_ERR_INVALID_ARG;
    const bool truss_inner = p && (p->flags & KC_TRUSS_INNER);
    if (truss_inner && (list || p->d_edge_count || p->d_edge_checksum || p->d_edge_cycles)) return KC_ERR_INVALID_ARG;
    DeviceGuard dg(g->device);
    r->ms_prepare = g->ms_prepare;
    if (p && p->d_edge_count) KC_CUDA(cudaMemsetAsync(p->d_edge_count, 0, sizeof(u64) * (g->m ? g->m : 1), s));
    if (p && p->d_edge_checksum) KC_CUDA(cudaMemsetAsync(p->d_edge_checksum, 0, sizeof(u64) * (g->m ? g->m : 1), s));
    if (p && p->d_edge_cycles) KC_CUDA(cudaMemsetAsync(p->d_edge_cycles, 0, sizeof(u64) * (g->m ? g->m : 1), s));
    if ((u64)k > (u64)g->tau + 2) {  // omega <= tau + 2: no k-clique
        KC_CUDA(cudaStreamSynchronize(s));
        return KC_OK;
    }
    kc_status st = check_width(g, k);
    if (st != KC_OK) return st;
    kc_query q;
    q.g = g;
    q.k = k;
    q.ticket_begin = 0;
    q.ticket_end = 0;
    kc_run_cfg cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.t_max = pick_t(p);
    cfg.flags = p ? p->flags : 0u;
    cfg.warps_per_block = p ? p->warps_per_block : 0u;
    cfg.blocks = p ? p->blocks : 0u;
    cfg.list = list;
    cfg.d_out = d_out;
    cfg.cap = cap;
    cfg.d_edge_count = p ? p->d_edge_count : nullptr;
    cfg.d_edge_checksum = p ? p->d_edge_checksum : nullptr;
    cfg.d_edge_cycles = p ? p->d_edge_cycles : nullptr;
    cfg.split_min = p ? p->split_min : 0u;
    cfg.width_min = p ? p->width_min : 0u;
    cfg.ticket_begin = p ? p->ticket_begin : 0ull;
    cfg.ticket_end = p ? p->ticket_end : 0ull;
    kc_dev_acc acc;
    memset(&acc, 0, sizeof(acc));
    float ms = 0.f, msb = 0.f;
    // listing: one pass writes rows and, when every clique fits, also yields the exact
    // totals; once the buffer is full it stops, and the totals come from a count with
    // checksum instead (which may split heavy sub-branches; a listing pass cannot)
    cfg.stop_full = list;
    st = truss_inner ? kc_run_ebbkc_t(g, k, &cfg, s, &acc, &ms, &msb) : kc_run_queries(&q, 1, &cfg, s, &acc, &ms, &msb);
    if (st != KC_OK) return st;
    st = map_device_status(acc.status);
    if (st != KC_OK) return st;
    const u64 written = acc.written;
    u64 extra_ops = 0, extra_nodes = 0, extra_pairs = 0;
    const bool rows_only = p && (p->flags & KC_ROWS_ONLY);
    if (list && written >= cap && !rows_only) {
        extra_ops = acc.word_ops;
        extra_nodes = acc.nodes;
        extra_pairs = acc.pair_tests;
        kc_run_cfg cc = cfg;
        cc.list = 0;
        cc.stop_full = 0;
        cc.d_out = nullptr;
        cc.cap = 0;
        cc.flags |= KC_CHECKSUM;
        float ms2 = 0.f, msb2 = 0.f;
        memset(&acc, 0, sizeof(acc));
        st = kc_run_queries(&q, 1, &cc, s, &acc, &ms2, &msb2);
        if (st != KC_OK) return st;
        st = map_device_status(acc.status);
        if (st != KC_OK) return st;
        ms += ms2;
        msb += msb2;
    }
    const bool no_totals = list && written >= cap && rows_only;
    r->count_lo = no_totals ? 0ull : acc.count_lo;
    r->count_hi = no_totals ? 0ull : acc.count_hi;
    r->checksum = (list || (cfg.flags & KC_CHECKSUM)) && !no_totals ? acc.checksum : 0ull;
    r->written = list ? std::min<u64>(written, cap) : 0ull;
    r->edge_branches = acc.branches;
    r->nodes = acc.nodes + extra_nodes;
    r->et_hits = acc.et_hits;
    r->word_ops = acc.word_ops + extra_ops;
    r->pair_tests = acc.pair_tests + extra_pairs;
    r->ms_count = ms;
    r->ms_branch = msb;
    if (no_totals) return KC_TRUNCATED;  // the buffer filled: totals unknown
    if (list && (acc.count_hi != 0 || acc.count_lo > cap)) return KC_TRUNCATED;
    return KC_OK;
}

// The queries of a batch that can have cliques (k <= tau + 2) and their indices; the
// others keep zero results.
kc_status batch_queries(const kc_graph *const *graphs, const uint32_t *ks, const kc_params *qp, uint32_t nq,
                        kc_result *results, std::vector<kc_query> &qv, std::vector<u32> &idx, int *dev) {
    memset(results, 0, sizeof(kc_result) * nq);
    for (u32 i = 0; i < nq; i++) {
        if (!graphs[i] || ks[i] < 3 || ks[i] > KC_MAX_K) return KC_ERR_INVALID_ARG;
        if (*dev < 0) *dev = graphs[i]->device;
        if (graphs[i]->device != *dev) return KC_ERR_INVALID_ARG;
        results[i].ms_prepare = graphs[i]->ms_prepare;
        if ((u64)ks[i] > (u64)graphs[i]->tau + 2) continue;
        kc_status st = check_width(graphs[i], ks[i]);
        if (st != KC_OK) return st;
        kc_query q;
        q.g = graphs[i];
        q.k = ks[i];
        q.ticket_begin = 0;
        q.ticket_end = 0;
        if (qp) {
            q.t_max = qp[i].t_max;
            q.split_min = qp[i].split_min;
            q.width_min = qp[i].width_min;
        }
        qv.push_back(q);
        idx.push_back(i);
    }
    return KC_OK;
}

kc_run_cfg batch_cfg(const kc_params *p) {
    kc_run_cfg cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.t_max = pick_t(p);
    cfg.flags = p ? p->flags : 0u;
    cfg.warps_per_block = p ? p->warps_per_block : 0u;
    cfg.blocks = p ? p->blocks : 0u;
    cfg.split_min = p ? p->split_min : 0u;
    cfg.width_min = p ? p->width_min : 0u;
    return cfg;
}

// the accumulators of the run queries into their results; the worst device status
kc_status batch_results(const std::vector<kc_dev_acc> &acc, const std::vector<u32> &idx, u32 flags, float ms,
                        float msb, kc_result *results) {
    kc_status worst = KC_OK;
    for (size_t j = 0; j < idx.size(); j++) {
        kc_result &r = results[idx[j]];
        kc_status sj = map_device_status(acc[j].status);
        if (sj != KC_OK) worst = sj;
        r.count_lo = acc[j].count_lo;
        r.count_hi = acc[j].count_hi;
        r.checksum = (flags & KC_CHECKSUM) ? acc[j].checksum : 0ull;
        r.edge_branches = acc[j].branches;
        r.nodes = acc[j].nodes;
        r.et_hits = acc[j].et_hits;
        r.word_ops = acc[j].word_ops;
        r.pair_tests = acc[j].pair_tests;
        r.ms_count = ms;
        r.ms_branch = msb;
    }
    return worst;
}

}  // namespace

extern "C" {

kc_status kclique_prepare(const uint32_t *row_ptr, const uint32_t *col, uint32_t n, uint64_t nnz, int on_device,
                          kc_stream s, kc_graph **out) {
    if (!out) return KC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!row_ptr || (nnz && !col)) return KC_ERR_INVALID_ARG;
    return kc_prepare_impl(row_ptr, col, n, nnz, on_device, KC_ORDER_TRUSS, (cudaStream_t)s, out);
}

kc_status kclique_prepare_ordered(const uint32_t *row_ptr, const uint32_t *col, uint32_t n, uint64_t nnz,
                                  int on_device, uint32_t ordering, kc_stream s, kc_graph **out) {
    if (!out) return KC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!row_ptr || (nnz && !col) || ordering > KC_ORDER_COLOUR) return KC_ERR_INVALID_ARG;
    return kc_prepare_impl(row_ptr, col, n, nnz, on_device, ordering, (cudaStream_t)s, out);
}

kc_status kclique_count(const kc_graph *g, uint32_t k, const kc_params *p, kc_stream s, kc_result *r) {
    return run_one(g, k, p, (cudaStream_t)s, r, 0, nullptr, 0);
}

kc_status kclique_list(const kc_graph *g, uint32_t k, uint32_t *d_out, uint64_t cap, const kc_params *p,
                       kc_stream s, kc_result *r) {
    return run_one(g, k, p, (cudaStream_t)s, r, 1, d_out, cap);
}

kc_status kclique_info(const kc_graph *g, kc_info *info) {
    if (!g || !info) return KC_ERR_INVALID_ARG;
    memset(info, 0, sizeof(*info));
    info->n = g->n;
    info->m = g->m;
    info->triangles = g->triangles;
    info->tau = g->tau;
    info->max_degree = g->max_degree;
    info->rounds = g->rounds;
    info->resident_bytes = g->resident_bytes;
    return KC_OK;
}

kc_status kclique_edge_data(const kc_graph *g, uint32_t *eu, uint32_t *ev, uint32_t *level, uint32_t *round,
                            uint32_t *vset_size, kc_stream sv) {
    if (!g) return KC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)sv;
    DeviceGuard dg(g->device);
    const u64 m = g->m;
    if (m == 0) return KC_OK;
    if (eu) KC_CUDA(cudaMemcpyAsync(eu, g->eu, sizeof(u32) * m, cudaMemcpyDeviceToHost, s));
    if (ev) KC_CUDA(cudaMemcpyAsync(ev, g->ev, sizeof(u32) * m, cudaMemcpyDeviceToHost, s));
    if (level) KC_CUDA(cudaMemcpyAsync(level, g->level, sizeof(u32) * m, cudaMemcpyDeviceToHost, s));
    if (round) KC_CUDA(cudaMemcpyAsync(round, g->round, sizeof(u32) * m, cudaMemcpyDeviceToHost, s));
    if (vset_size) {
        std::vector<u64> ptr(m + 1);
        KC_CUDA(cudaMemcpyAsync(ptr.data(), g->vset_ptr, sizeof(u64) * (m + 1), cudaMemcpyDeviceToHost, s));
        KC_CUDA(cudaStreamSynchronize(s));
        for (u64 i = 0; i < m; i++) vset_size[i] = (u32)(ptr[i + 1] - ptr[i]);
    }
    KC_CUDA(cudaStreamSynchronize(s));
    return KC_OK;
}

void kclique_release(kc_graph *g) { kc_free_graph(g); }

const char *kclique_status_string(kc_status st) {
    switch (st) {
        case KC_OK: return "ok";
        case KC_TRUNCATED: return "list buffer full: count and checksum cover all cliques";
        case KC_ERR_INVALID_ARG: return "invalid argument";
        case KC_ERR_INVALID_GRAPH: return "invalid graph (row_ptr not monotone, column id >= n, or too many entries)";
        case KC_ERR_OOM: return "device out of memory";
        case KC_ERR_CUDA: return "CUDA error";
        case KC_ERR_TIMEOUT: return "bounded device wait timed out";
        case KC_ERR_OVERFLOW: return "count reached 2^128";
        case KC_ERR_UNSUPPORTED: return "sub-branch wider than the supported maximum";
    }
    return "unknown status";
}

kc_status kclique_count_batch(const kc_graph *const *graphs, const uint32_t *ks, uint32_t nq, const kc_params *p,
                              kc_stream sv, kc_result *results) {
    return kclique_count_batch_tuned(graphs, ks, nullptr, nq, p, sv, results);
}

kc_status kclique_count_batch_tuned(const kc_graph *const *graphs, const uint32_t *ks, const kc_params *qp,
                                    uint32_t nq, const kc_params *p, kc_stream sv, kc_result *results) {
    if (!graphs || !ks || !results) return KC_ERR_INVALID_ARG;
    if (p && (p->d_edge_count || p->d_edge_checksum || p->d_edge_cycles)) return KC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)sv;
    std::vector<kc_query> qv;
    std::vector<u32> idx;
    int dev = -1;
    kc_status st = batch_queries(graphs, ks, qp, nq, results, qv, idx, &dev);
    if (st != KC_OK || qv.empty()) return st;
    DeviceGuard dg(dev);
    const kc_run_cfg cfg = batch_cfg(p);
    std::vector<kc_dev_acc> acc(qv.size());
    float ms = 0.f, msb = 0.f;
    st = kc_run_queries(qv.data(), (u32)qv.size(), &cfg, s, acc.data(), &ms, &msb);
    if (st != KC_OK) return st;
    return batch_results(acc, idx, cfg.flags, ms, msb, results);
}

}  // extern "C"

struct kc_batch_plan {
    kc_plan *plan = nullptr;         // null when no query can have cliques
    int device = 0;
    u32 nq = 0;
    u32 flags = 0;
    std::vector<u32> idx;            // the run queries' indices
    std::vector<float> ms_prepare;   // per query
};

extern "C" {

kc_status kclique_batch_plan_create(const kc_graph *const *graphs, const uint32_t *ks, const kc_params *qp,
                                    uint32_t nq, const kc_params *p, kc_stream sv, kc_batch_plan **out) {
    if (!graphs || !ks || !out) return KC_ERR_INVALID_ARG;
    *out = nullptr;
    if (p && (p->d_edge_count || p->d_edge_checksum || p->d_edge_cycles)) return KC_ERR_INVALID_ARG;
    std::vector<kc_result> res(nq ? nq : 1);
    std::vector<kc_query> qv;
    kc_batch_plan *bp = new kc_batch_plan();
    int dev = -1;
    kc_status st = batch_queries(graphs, ks, qp, nq, res.data(), qv, bp->idx, &dev);
    if (st != KC_OK) {
        delete bp;
        return st;
    }
    bp->nq = nq;
    bp->flags = p ? p->flags : 0u;
    for (u32 i = 0; i < nq; i++) bp->ms_prepare.push_back(res[i].ms_prepare);
    if (!qv.empty()) {
        bp->device = dev;
        DeviceGuard dg(dev);
        const kc_run_cfg cfg = batch_cfg(p);
        st = kc_plan_create(qv.data(), (u32)qv.size(), &cfg, (cudaStream_t)sv, &bp->plan);
        if (st != KC_OK) {
            delete bp;
            return st;
        }
    }
    *out = bp;
    return KC_OK;
}

kc_status kclique_batch_plan_run(kc_batch_plan *bp, kc_stream sv, kc_result *results) {
    if (!bp || !results) return KC_ERR_INVALID_ARG;
    memset(results, 0, sizeof(kc_result) * bp->nq);
    for (u32 i = 0; i < bp->nq; i++) results[i].ms_prepare = bp->ms_prepare[i];
    if (!bp->plan) return KC_OK;
    DeviceGuard dg(bp->device);
    std::vector<kc_dev_acc> acc(bp->idx.size());
    float ms = 0.f;
    kc_status st = kc_plan_run(bp->plan, (cudaStream_t)sv, acc.data(), &ms);
    if (st != KC_OK) return st;
    return batch_results(acc, bp->idx, bp->flags, ms, ms, results);
}

void kclique_batch_plan_release(kc_batch_plan *bp) {
    if (!bp) return;
    kc_plan_free(bp->plan);
    delete bp;
}

}  // extern "C"
