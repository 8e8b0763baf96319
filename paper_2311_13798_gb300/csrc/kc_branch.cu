// Branch engine, host side: the launches of the per-edge sub-branches of EBBkC-H
// (paper Alg. 5 with EBBkC-C_Rec of Alg. 4 and the early termination of
// Sec. 5).  The kernels are in kc_branch_dev.cuh, instantiated per bitset width in
// kc_branch_w<W>.cu; this file builds the per-query descriptors, runs the width classes
// and reads the results back, and holds the binomial table and the integer-peak probe.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "kc_branch_dev.cuh"

namespace {
using namespace kcb;

kc_status launch_width(int W, int mode, const Args &a, const std::vector<QDesc> &qs, u64 tickets,
                       const kc_run_cfg *cfg, cudaStream_t s, QDesc *d_qs, u64 *d_qstart, unsigned long long *d_ctr,
                       SplitBufs *sb) {
    switch (W) {
        case 1: return launch_width_1(mode, a, qs, tickets, cfg, s, d_qs, d_qstart, d_ctr, sb);
        case 2: return launch_width_2(mode, a, qs, tickets, cfg, s, d_qs, d_qstart, d_ctr, sb);
        case 4: return launch_width_4(mode, a, qs, tickets, cfg, s, d_qs, d_qstart, d_ctr, sb);
        case 8: return launch_width_8(mode, a, qs, tickets, cfg, s, d_qs, d_qstart, d_ctr, sb);
        case 16: return launch_width_16(mode, a, qs, tickets, cfg, s, d_qs, d_qstart, d_ctr, sb);
        case 32: return launch_width_32(mode, a, qs, tickets, cfg, s, d_qs, d_qstart, d_ctr, sb);
    }
    return KC_ERR_UNSUPPORTED;
}

kc_status launch_fixed_width(int W, int mode, const Args &a, const QDesc *qs, u32 nqs, const kc_run_cfg *cfg,
                             cudaStream_t s, QDesc *d_qs, u64 *d_qstart, unsigned long long *d_ctr) {
    switch (W) {
        case 1: return launch_fixed_width_1(mode, a, qs, nqs, cfg, s, d_qs, d_qstart, d_ctr);
        case 2: return launch_fixed_width_2(mode, a, qs, nqs, cfg, s, d_qs, d_qstart, d_ctr);
        case 4: return launch_fixed_width_4(mode, a, qs, nqs, cfg, s, d_qs, d_qstart, d_ctr);
        case 8: return launch_fixed_width_8(mode, a, qs, nqs, cfg, s, d_qs, d_qstart, d_ctr);
        case 16: return launch_fixed_width_16(mode, a, qs, nqs, cfg, s, d_qs, d_qstart, d_ctr);
        case 32: return launch_fixed_width_32(mode, a, qs, nqs, cfg, s, d_qs, d_qstart, d_ctr);
    }
    return KC_ERR_UNSUPPORTED;
}

#if KC_DEBUG_BOUNDS
unsigned long long debug_flags() {
    unsigned long long f = 0;
    for (unsigned long long x : {debug_flag_width_1(), debug_flag_width_2(), debug_flag_width_4(),
                                 debug_flag_width_8(), debug_flag_width_16(), debug_flag_width_32()})
        if (!f) f = x;
    return f;
}
#endif

// ---------------------------------------------------------------- binomials
__global__ void binom_kernel(u128 *T) {
    int r = threadIdx.x;
    for (int n = 0; n < BINOM_N; n++) {
        if (r < BINOM_R) {
            u128 v;
            if (r == 0) v = 1;
            else if (r > n) v = 0;
            else {
                u128 a = T[(n - 1) * BINOM_R + r - 1];
                u128 b = (r <= n - 1) ? T[(n - 1) * BINOM_R + r] : 0;
                u128 sum = a + b;
                v = (a == SAT128 || b == SAT128 || sum < a) ? SAT128 : sum;
            }
            T[n * BINOM_R + r] = v;
        }
        __syncthreads();
    }
}

// binomial tables, one per device; created once under g_tables_mu (the library may
// be entered from several host threads, e.g. a server's worker pool)
constexpr int KC_MAX_DEVICES = 64;
u128 *g_tables[KC_MAX_DEVICES] = {};
std::mutex g_tables_mu;
}  // namespace

// early-termination threshold of one query: the caller's t_max (at most 3: the kernels
// hold closed forms for cliques, 2-plexes and 3-plexes), or the paper's rule (Sec. 6.1
// "Baselines and Metrics": t = 2 when k <= tau / 2, else t = 3)
u32 kc_pick_t(u32 t_max, u32 k, u32 tau) {
    if (t_max) return std::min<u32>(t_max, 3u);
    return 2ull * k <= (u64)tau ? 2u : 3u;
}

kc_status kc_ensure_tables(cudaStream_t s) {
    int dev = 0;
    KC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= KC_MAX_DEVICES) return KC_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_tables_mu);
    if (!g_tables[dev]) {
        // keep stream-ordered scratch (split buffers, prepare temporaries) cached in the pool
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t thr = ~0ull;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
        u128 *T = nullptr;
        KC_CUDA(cudaMalloc(&T, sizeof(u128) * BINOM_N * BINOM_R));
        binom_kernel<<<1, 64, 0, s>>>(T);
        kc_note_launch();
        KC_CUDA(cudaGetLastError());
        KC_CUDA(cudaStreamSynchronize(s));
        g_tables[dev] = T;
    }
    return KC_OK;
}

namespace {
using namespace kcb;

// number of edges of g with |VSet| >= x (tickets are sorted by |VSet| descending)
u64 suffix_count(const kc_graph *g, u64 x) { return x > g->tau ? 0ull : g->h_size_suffix[x]; }

// the width class (a power of two, 1..32) that a requested width_min selects
u32 width_floor(u32 wmin) {
    u32 w = 1;
    while (w < wmin && w < 32) w <<= 1;
    return w;
}

// smallest sub-branch size of width class W for queries at k; classes narrower than
// wmin are empty and class wmin takes every smaller sub-branch
u64 class_low(int W, u32 k, u32 wmin = 1) {
    u64 s_lo = (W == 1 || (u32)W == width_floor(wmin)) ? 0ull : 16ull * W + 1;
    return s_lo < (u64)k - 2 ? (u64)k - 2 : s_lo;
}

// The tickets [b, en) of one query whose sub-branches fit width class W.
void class_range(const kc_graph *g, u32 k, int W, const kc_run_cfg *cfg, u64 *b, u64 *en, u32 wmin = 1) {
    auto suffix = [&](u64 x) -> u64 { return suffix_count(g, x); };
    const u64 s_hi = 32ull * W;
    const u64 s_lo = class_low(W, k, wmin);
    *b = *en = 0;
    if ((u32)W < width_floor(wmin) || s_lo > s_hi) return;
    u64 bb = suffix(s_hi + 1), ee = suffix(s_lo);
    if (cfg && cfg->ticket_end > cfg->ticket_begin) {  // shard
        bb = std::max<u64>(bb, cfg->ticket_begin);
        ee = std::min<u64>(ee, cfg->ticket_end);
    }
    if (ee > bb) { *b = bb; *en = ee; }
}

QDesc make_desc(const kc_graph *g, u32 k, u32 t_max, u64 b, u64 en, kc_dev_acc *acc) {
    QDesc d;
    memset(&d, 0, sizeof(d));
    d.row_ptr = g->row_ptr; d.col = g->col; d.pos_eid = g->pos_eid; d.pos_round = g->pos_round;
    d.eu = g->eu; d.ev = g->ev; d.round = g->round; d.vset = g->vset; d.tickets = g->tickets;
    d.vset_ptr = g->vset_ptr;
    d.k = k;
    d.t_max = kc_pick_t(t_max, k, g->tau);
    d.t0 = b;
    d.nt = en - b;
    d.acc = acc;
    return d;
}

u64 align256(u64 x) { return (x + 255ull) & ~255ull; }

// one persistent launch (plus its item launch) per group
struct Group {
    int W, mode;
    std::vector<QDesc> qs;
    std::vector<u64> qstart;
    u64 off_qs = 0, off_qstart = 0, off_ctr = 0;
};

// The launch groups of a set of queries, and the layout of the device buffer they share.
struct Batch {
    std::vector<Group> groups;
    u64 bytes = 0;
};

void plan_batch(const kc_query *qv, u32 nq, const kc_run_cfg *cfg, Batch *bt) {
    const int base_mode = cfg->list ? (MODE_LIST | MODE_CHECKSUM) : ((cfg->flags & KC_CHECKSUM) ? MODE_CHECKSUM : 0);
    const int widths[6] = {32, 16, 8, 4, 2, 1};
    for (int wi = 0; wi < 6; wi++) {
        const int W = widths[wi];
        for (int par = 0; par < (cfg->list ? 1 : 2); par++) {
            Group gr;
            gr.W = W;
            gr.mode = cfg->list ? base_mode : (base_mode | (par == 0 ? MODE_ODD : MODE_EVEN));
            for (u32 i = 0; i < nq; i++) {
                const kc_graph *g = qv[i].g;
                const u32 k = qv[i].k;
                if (!cfg->list && (int)(k & 1u) != (par == 0 ? 1 : 0)) continue;
                // per-query choices override the run's
                const u32 t_max = qv[i].t_max ? qv[i].t_max : cfg->t_max;
                const u32 split_min = qv[i].split_min ? qv[i].split_min : cfg->split_min;
                const u32 wmin = qv[i].width_min ? qv[i].width_min : (cfg->width_min ? cfg->width_min : 1u);
                u64 b, en;
                class_range(g, k, W, cfg, &b, &en, wmin);
                if (en <= b) continue;
                QDesc d = make_desc(g, k, t_max, b, en, nullptr);
                d.acc = (kc_dev_acc *)(uintptr_t)i;  // index for now: the device address is set below
                // split the heavy tickets (|VSet| >= split_min) of k >= 7 queries (A12)
                const u64 smin = split_min ? split_min : 64ull;
                if (k >= 7 && split_min != ~0u && !cfg->list) {
                    const u64 hb = suffix_count(g, std::max<u64>(smin, class_low(W, k, wmin)));
                    d.nheavy = hb > b ? std::min<u64>(hb - b, d.nt) : 0ull;
                }
                d.edge_count = cfg->d_edge_count;
                d.edge_checksum = cfg->d_edge_checksum;
                d.edge_cycles = cfg->d_edge_cycles;
                gr.qs.push_back(d);
            }
            if (gr.qs.empty()) continue;
            gr.qstart.assign(gr.qs.size() + 1, 0);
            for (size_t i = 0; i < gr.qs.size(); i++) gr.qstart[i + 1] = gr.qstart[i] + gr.qs[i].nt;
            bt->groups.push_back(std::move(gr));
        }
    }
    // one device buffer: accumulators, then per group its descriptors, prefix and counters
    u64 bytes = align256(sizeof(kc_dev_acc) * (nq ? nq : 1));
    for (Group &gr : bt->groups) {
        gr.off_qs = bytes;
        bytes += align256(sizeof(QDesc) * gr.qs.size());
        gr.off_qstart = bytes;
        bytes += align256(sizeof(u64) * gr.qstart.size());
        gr.off_ctr = bytes;
        bytes += align256(4 * sizeof(unsigned long long));
    }
    bt->bytes = bytes;
}

// The host image of the device buffer at dbuf: zeroed accumulators and counters, each
// group's descriptors (accumulator pointers into dbuf) and ticket prefix.
void batch_image(const Batch &bt, unsigned char *dbuf, unsigned char *host) {
    memset(host, 0, bt.bytes);
    kc_dev_acc *d_acc = (kc_dev_acc *)dbuf;
    for (const Group &gr : bt.groups) {
        std::vector<QDesc> qs = gr.qs;
        for (QDesc &d : qs) d.acc = d_acc + (uintptr_t)d.acc;
        memcpy(host + gr.off_qs, qs.data(), sizeof(QDesc) * qs.size());
        memcpy(host + gr.off_qstart, gr.qstart.data(), sizeof(u64) * gr.qstart.size());
    }
}

Args batch_args(const kc_run_cfg *cfg, int dev) {
    Args a;
    memset(&a, 0, sizeof(a));
    a.t_max = cfg->t_max;
    a.flags = cfg->flags;
    a.d_out = cfg->d_out;
    a.cap = cfg->cap;
    a.stop_full = cfg->list && cfg->stop_full ? 1u : 0u;
    a.binom = g_tables[dev];
    return a;
}

// The groups' launches on s, back to back (ev: two events per group, or null).
kc_status launch_batch(const Batch &bt, const Args &a, const kc_run_cfg *cfg, cudaStream_t s, unsigned char *dbuf,
                       SplitBufs *sb, cudaEvent_t *ev) {
    kc_status st = KC_OK;
    for (size_t gi = 0; gi < bt.groups.size() && st == KC_OK; gi++) {
        const Group &gr = bt.groups[gi];
        if (ev) KC_CUDA(cudaEventRecord(ev[2 * gi], s));
        st = launch_width(gr.W, gr.mode, a, gr.qs, gr.qstart.back(), cfg, s, (QDesc *)(dbuf + gr.off_qs),
                          (u64 *)(dbuf + gr.off_qstart), (unsigned long long *)(dbuf + gr.off_ctr), sb);
        if (ev) KC_CUDA(cudaEventRecord(ev[2 * gi + 1], s));
    }
    return st;
}

}  // namespace

// Run queries: the tickets of each query are split into width classes, and the queries
// of one class and one parity of k form a launch group (the kernels are compiled per
// parity).  Every group's descriptors, ticket prefix and counters are written to one
// device buffer by one copy, so the groups launch back to back on the stream with no
// host synchronisation between them; the host waits once, for the results.
kc_status kc_run_queries(const kc_query *qv, u32 nq, const kc_run_cfg *cfg, cudaStream_t s, kc_dev_acc *h_acc,
                         float *ms, float *ms_branch) {
    kc_status st = kc_ensure_tables(s);
    if (st != KC_OK) return st;
    int dev = 0;
    KC_CUDA(cudaGetDevice(&dev));
    Batch bt;
    plan_batch(qv, nq, cfg, &bt);
    std::vector<Group> &groups = bt.groups;
    const u64 bytes = bt.bytes;
    unsigned char *dbuf = nullptr;
    KC_CUDA(cudaMallocAsync(&dbuf, bytes, s));
    kc_dev_acc *d_acc = (kc_dev_acc *)dbuf;
    std::vector<unsigned char> host(bytes);
    batch_image(bt, dbuf, host.data());
    SplitBufs sb;
    Args a = batch_args(cfg, dev);
    a.prof = (KC_SECTION_PROFILE && getenv("KC_PROFILE")) ? 1u : 0u;
    if (a.prof) {
        KC_CUDA(cudaMallocAsync(&a.l3hist, 64 * sizeof(unsigned long long), s));
        KC_CUDA(cudaMemsetAsync(a.l3hist, 0, 64 * sizeof(unsigned long long), s));
    }
    std::vector<cudaEvent_t> ev(2 * groups.size() + 2);
    for (cudaEvent_t &e : ev) KC_CUDA(cudaEventCreate(&e));
    KC_CUDA(cudaEventRecord(ev[0], s));
    // the copy reads pageable memory: it is staged before this call returns, and it is
    // ordered on the stream before the launches
    KC_CUDA(cudaMemcpyAsync(dbuf, host.data(), bytes, cudaMemcpyHostToDevice, s));
    if (cfg->d_edge_count)
        KC_CUDA(cudaMemsetAsync(cfg->d_edge_count, 0, sizeof(u64) * (nq ? qv[0].g->m : 0), s));
    if (cfg->d_edge_checksum)
        KC_CUDA(cudaMemsetAsync(cfg->d_edge_checksum, 0, sizeof(u64) * (nq ? qv[0].g->m : 0), s));
    if (cfg->d_edge_cycles)
        KC_CUDA(cudaMemsetAsync(cfg->d_edge_cycles, 0, sizeof(u64) * (nq ? qv[0].g->m : 0), s));
    const bool profile = getenv("KC_PROFILE") != nullptr;
    st = launch_batch(bt, a, cfg, s, dbuf, &sb, ev.data() + 2);
    KC_CUDA(cudaEventRecord(ev[1], s));
    if (st == KC_OK) KC_CUDA(cudaMemcpyAsync(h_acc, d_acc, sizeof(kc_dev_acc) * nq, cudaMemcpyDeviceToHost, s));
    cudaStreamSynchronize(s);
    *ms_branch = 0.f;
    for (size_t gi = 0; gi < groups.size() && st == KC_OK; gi++) {
        float bm = 0.f;
        cudaEventElapsedTime(&bm, ev[2 + 2 * gi], ev[3 + 2 * gi]);
        *ms_branch += bm;
        if (profile) {
            u64 nt = 0;
            for (const QDesc &d : groups[gi].qs) nt += d.nt;
            fprintf(stderr, "[kclique] class W=%d queries=%zu tickets=%llu mode=%d %.3f ms\n", groups[gi].W,
                    groups[gi].qs.size(), (unsigned long long)nt, groups[gi].mode, bm);
        }
    }
#if KC_DEBUG_BOUNDS
    {
        const unsigned long long dbg = debug_flags();
        if (dbg)
            fprintf(stderr, "[kclique] bounds check failed: line %llu index %llu bound %llu\n", dbg >> 40,
                    (dbg >> 20) & 0xFFFFFull, dbg & 0xFFFFFull);
    }
#endif
    if (profile && st == KC_OK) {
        const char *names[6] = {"extract", "colour", "et(l>=4)", "l3-frames", "generate", "evaluate"};
        for (int i = 0; i < 6; i++) {
            unsigned long long t = 0;
            for (u32 j = 0; j < nq; j++) t += h_acc[j].sec[i];
            fprintf(stderr, "[kclique] section %-10s %.3e warp-cycles\n", names[i], (double)t);
        }
        unsigned long long hh[64];
        if (a.l3hist && cudaMemcpy(hh, a.l3hist, sizeof(hh), cudaMemcpyDeviceToHost) == cudaSuccess) {
            const char *bn[7] = {"<=8", "<=16", "<=32", "<=64", "<=128", "<=256", ">256"};
            for (int i = 0; i < 7; i++)
                fprintf(stderr, "[kclique] l3 frames %-5s %12llu  %.3e warp-cycles\n", bn[i], hh[i], (double)hh[8 + i]);
            for (int i = 0; i <= 10; i++)
                fprintf(stderr, "[kclique] l3 density %2d/10 %12llu  %.3e warp-cycles  mean size %.1f\n", i, hh[16 + i],
                        (double)hh[27 + i], hh[16 + i] ? (double)hh[38 + i] / (double)hh[16 + i] : 0.0);
        }
    }
    if (a.l3hist) cudaFreeAsync(a.l3hist, s);
    cudaEventElapsedTime(ms, ev[0], ev[1]);
    for (cudaEvent_t &e : ev) cudaEventDestroy(e);
    cudaFreeAsync(dbuf, s);
    if (sb.slots) cudaFreeAsync(sb.slots, s);
    cudaStreamSynchronize(s);
    if (st == KC_OK) {
        cudaError_t ce = cudaGetLastError();
        if (ce != cudaSuccess) {
            kc_set_last_cuda_error(ce, "branch kernels", __FILE__, __LINE__);
            return KC_ERR_CUDA;
        }
    }
    return st;
}

// ---------------------------------------------------------------- integer peak probe
// Sustained rate of the inner mix of the branch kernel: for every 32-bit word, two ANDs
// and a POPC (fused by the compiler into LOP3 + POPC + IADD), 8 independent chains per
// thread.  Counts 3 lane-ops per word, the accounting used for word_ops.
__global__ void int_peak_kernel(u32 seed, int iters, unsigned long long *sink) {
    u32 a[8], b[8], c[8];
    u32 acc = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) {
        a[i] = seed * (threadIdx.x + 1 + i) ^ blockIdx.x;
        b[i] = seed + 0x9E3779B9u * (i + 1) + threadIdx.x;
        c[i] = ~a[i] ^ (b[i] << 7);
    }
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int i = 0; i < 8; i++) {
            u32 x = a[i] & b[i] & c[i];
            acc += __popc(x);
            a[i] = b[i];
            b[i] = c[i];
            c[i] = x ^ (u32)it;
        }
    }
    if (acc == 0x7FFFFFFFu) atomicAdd(sink, 1ull);  // keeps the loop alive
}

extern "C" KC_API kc_status kclique_int_peak(double *lane_ops_per_s, int *sms, kc_stream sv) {
    if (!lane_ops_per_s) return KC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)sv;
    int dev = 0, nsm = 0;
    KC_CUDA(cudaGetDevice(&dev));
    KC_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    unsigned long long *sink = nullptr;
    KC_CUDA(cudaMalloc(&sink, sizeof(unsigned long long)));
    const int threads = 256, blocks = nsm * 8, iters = 1 << 14;
    int_peak_kernel<<<blocks, threads, 0, s>>>(12345u, iters / 16, sink);  // warm-up
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 5; rep++) {
        cudaEventRecord(e0, s);
        int_peak_kernel<<<blocks, threads, 0, s>>>(12345u + rep, iters, sink);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    KC_CUDA(cudaGetLastError());
    *lane_ops_per_s = 3.0 * 8.0 * (double)iters * threads * blocks / (best * 1e-3);
    if (sms) *sms = nsm;
    return KC_OK;
}

// ---------------------------------------------------------------- no-allocation path
// The same persistent kernels, launched for callers that cannot allocate device memory:
// the query table, accumulators and counters live in caller-supplied scratch, the
// binomial table is caller-supplied, sub-branches are not split (no split buffers), and
// host-side bookkeeping uses fixed arrays.
static_assert(KC_BINOM_ENTRIES == BINOM_N * BINOM_R, "binomial table size");

// Every kernel instance the no-allocation path can launch, loaded at its set-up.
kc_status kc_preload_fixed_kernels() {
    kc_status st = KC_OK;
    for (kc_status (*f)() : {preload_width_1, preload_width_2, preload_width_4, preload_width_8, preload_width_16,
                             preload_width_32})
        if (st == KC_OK) st = f();
    if (st == KC_OK) {
        cudaFuncAttributes fa;
        KC_CUDA(cudaFuncGetAttributes(&fa, binom_kernel));
    }
    return st;
}

kc_status kc_fill_binom(u128 *table, cudaStream_t s) {
    binom_kernel<<<1, 64, 0, s>>>(table);
    kc_note_launch();
    KC_CUDA(cudaGetLastError());
    KC_CUDA(cudaStreamSynchronize(s));
    return KC_OK;
}

u64 kc_scratch_bytes_for(u32 nq) {
    return align256(sizeof(kc_dev_acc) * (u64)nq) + align256(sizeof(QDesc) * (u64)nq) +
           align256(sizeof(u64) * ((u64)nq + 1)) + align256(4 * sizeof(unsigned long long));
}

kc_status kc_run_queries_in_scratch(const kc_query *qv, u32 nq, const kc_run_cfg *cfg, cudaStream_t s,
                                    unsigned char *d_scratch, u64 scratch_bytes, const u128 *d_binom,
                                    kc_dev_acc *h_acc) {
    const u32 t_max = cfg->t_max, flags = cfg->flags;
    if (nq == 0) return KC_OK;
    if (nq > kNoallocMaxQ || kc_scratch_bytes_for(nq) > scratch_bytes) return KC_ERR_INVALID_ARG;
    unsigned char *p = d_scratch;
    kc_dev_acc *d_acc = (kc_dev_acc *)p;
    p += align256(sizeof(kc_dev_acc) * (u64)nq);
    QDesc *d_qs = (QDesc *)p;
    p += align256(sizeof(QDesc) * (u64)nq);
    u64 *d_qstart = (u64 *)p;
    p += align256(sizeof(u64) * ((u64)nq + 1));
    unsigned long long *d_ctr = (unsigned long long *)p;
    // the scratch keeps the previous call's contents: the accumulators start at zero
    KC_CUDA(cudaMemsetAsync(d_acc, 0, sizeof(kc_dev_acc) * nq, s));
    Args a;
    memset(&a, 0, sizeof(a));
    a.t_max = t_max;
    a.flags = flags;
    a.binom = d_binom;
    const int base_mode = (flags & KC_CHECKSUM) ? MODE_CHECKSUM : 0;
    const int widths[6] = {32, 16, 8, 4, 2, 1};
    kc_status st = KC_OK;
    for (int wi = 0; wi < 6 && st == KC_OK; wi++) {
        const int W = widths[wi];
        for (int par = 0; par < 2 && st == KC_OK; par++) {
            QDesc qs[kNoallocMaxQ];
            u32 nqs = 0;
            for (u32 i = 0; i < nq; i++) {
                const kc_graph *g = qv[i].g;
                const u32 k = qv[i].k;
                if ((int)(k & 1u) != (par == 0 ? 1 : 0)) continue;
                u64 b, en;
                class_range(g, k, W, nullptr, &b, &en);
                if (en <= b) continue;
                qs[nqs++] = make_desc(g, k, t_max, b, en, d_acc + i);
            }
            if (!nqs) continue;
            st = launch_fixed_width(W, base_mode | (par == 0 ? MODE_ODD : MODE_EVEN), a, qs, nqs, cfg, s, d_qs,
                                    d_qstart, d_ctr);
            // the query table in scratch is rewritten for the next group
            if (st == KC_OK) KC_CUDA(cudaStreamSynchronize(s));
        }
    }
    if (st != KC_OK) return st;
    KC_CUDA(cudaMemcpyAsync(h_acc, d_acc, sizeof(kc_dev_acc) * nq, cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaStreamSynchronize(s));
    return KC_OK;
}


// ---------------------------------------------------------------- batch plans
// One batch's work captured once as a CUDA graph: the copy of the buffer image (which
// also zeroes the accumulators and counters), the launch groups and the copy of the
// results back to pinned host memory.  A run replays it.
struct kc_plan {
    int device = 0;
    u32 nq = 0;
    u32 launches = 0;                          // kernel launches per run
    kc_run_cfg cfg;
    Batch bt;
    unsigned char *dbuf = nullptr;             // device buffer
    unsigned char *hbuf = nullptr;             // its pinned host image
    kc_dev_acc *h_acc = nullptr;               // pinned copy of the accumulators
    SplitBufs sb;
    cudaStream_t cs = nullptr;                 // the stream the graph was captured on
    cudaGraphExec_t exec = nullptr;
};

void kc_plan_free(kc_plan *p) {
    if (!p) return;
    cudaSetDevice(p->device);
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->cs) {
        if (p->sb.slots) cudaFreeAsync(p->sb.slots, p->cs);
        cudaStreamSynchronize(p->cs);
        cudaStreamDestroy(p->cs);
    }
    if (p->dbuf) cudaFree(p->dbuf);
    if (p->hbuf) cudaFreeHost(p->hbuf);
    if (p->h_acc) cudaFreeHost(p->h_acc);
    delete p;
}

kc_status kc_plan_create(const kc_query *qv, u32 nq, const kc_run_cfg *cfg, cudaStream_t s, kc_plan **out) {
    *out = nullptr;
    if (cfg->list || cfg->d_edge_count || cfg->d_edge_checksum || cfg->d_edge_cycles) return KC_ERR_INVALID_ARG;
    kc_status st = kc_ensure_tables(s);
    if (st != KC_OK) return st;
    kc_plan *p = new kc_plan();
    auto fail = [&](kc_status e) { kc_plan_free(p); return e; };
    auto cuda = [&](cudaError_t e, const char *what) {
        if (e == cudaSuccess) return KC_OK;
        kc_set_last_cuda_error(e, what, __FILE__, __LINE__);
        return e == cudaErrorMemoryAllocation ? KC_ERR_OOM : KC_ERR_CUDA;
    };
    if ((st = cuda(cudaGetDevice(&p->device), "cudaGetDevice")) != KC_OK) return fail(st);
    p->nq = nq;
    p->cfg = *cfg;
    plan_batch(qv, nq, cfg, &p->bt);
    if ((st = cuda(cudaMalloc(&p->dbuf, p->bt.bytes), "cudaMalloc")) != KC_OK) return fail(st);
    if ((st = cuda(cudaMallocHost(&p->hbuf, p->bt.bytes), "cudaMallocHost")) != KC_OK) return fail(st);
    if ((st = cuda(cudaMallocHost(&p->h_acc, sizeof(kc_dev_acc) * (nq ? nq : 1)), "cudaMallocHost")) != KC_OK)
        return fail(st);
    batch_image(p->bt, p->dbuf, p->hbuf);
    if ((st = cuda(cudaStreamCreateWithFlags(&p->cs, cudaStreamNonBlocking), "cudaStreamCreate")) != KC_OK)
        return fail(st);
    // the caller's stream's earlier work (the graphs' preparation) comes first
    cudaEvent_t dep;
    if ((st = cuda(cudaEventCreateWithFlags(&dep, cudaEventDisableTiming), "cudaEventCreate")) != KC_OK) return fail(st);
    cudaEventRecord(dep, s);
    cudaStreamWaitEvent(p->cs, dep, 0);
    cudaEventDestroy(dep);
    const Args a = batch_args(cfg, p->device);
    // an ordinary first run sizes the buffers of split sub-branches, so the captured
    // launches allocate nothing
    if ((st = cuda(cudaMemcpyAsync(p->dbuf, p->hbuf, p->bt.bytes, cudaMemcpyHostToDevice, p->cs), "cudaMemcpyAsync")) !=
        KC_OK)
        return fail(st);
    if ((st = launch_batch(p->bt, a, cfg, p->cs, p->dbuf, &p->sb, nullptr)) != KC_OK) return fail(st);
    if ((st = cuda(cudaStreamSynchronize(p->cs), "first run")) != KC_OK) return fail(st);
    // capture (relaxed: the launch code queries occupancy and sets kernel attributes)
    const unsigned long long n0 = kclique_launch_count(0);
    if ((st = cuda(cudaStreamBeginCapture(p->cs, cudaStreamCaptureModeRelaxed), "cudaStreamBeginCapture")) != KC_OK)
        return fail(st);
    cudaError_t ce = cudaMemcpyAsync(p->dbuf, p->hbuf, p->bt.bytes, cudaMemcpyHostToDevice, p->cs);
    kc_status lst = ce == cudaSuccess ? launch_batch(p->bt, a, cfg, p->cs, p->dbuf, &p->sb, nullptr) : KC_ERR_CUDA;
    if (ce == cudaSuccess && lst == KC_OK)
        ce = cudaMemcpyAsync(p->h_acc, p->dbuf, sizeof(kc_dev_acc) * nq, cudaMemcpyDeviceToHost, p->cs);
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(p->cs, &graph);  // always ends the capture
    p->launches = (u32)(kclique_launch_count(0) - n0);
    if (lst != KC_OK) {
        if (graph) cudaGraphDestroy(graph);
        return fail(lst);
    }
    if ((st = cuda(ce != cudaSuccess ? ce : ee, "stream capture")) != KC_OK) {
        if (graph) cudaGraphDestroy(graph);
        return fail(st);
    }
    const cudaError_t ie = cudaGraphInstantiate(&p->exec, graph, 0);
    cudaGraphDestroy(graph);
    if ((st = cuda(ie, "cudaGraphInstantiate")) != KC_OK) return fail(st);
    *out = p;
    return KC_OK;
}

kc_status kc_plan_run(kc_plan *p, cudaStream_t s, kc_dev_acc *h_acc, float *ms) {
    int cur = 0;
    KC_CUDA(cudaGetDevice(&cur));
    if (cur != p->device) KC_CUDA(cudaSetDevice(p->device));
    cudaEvent_t ev[2];
    KC_CUDA(cudaEventCreate(&ev[0]));
    KC_CUDA(cudaEventCreate(&ev[1]));
    KC_CUDA(cudaEventRecord(ev[0], s));
    const cudaError_t le = cudaGraphLaunch(p->exec, s);
    KC_CUDA(cudaEventRecord(ev[1], s));
    const cudaError_t se = cudaStreamSynchronize(s);
    *ms = 0.f;
    cudaEventElapsedTime(ms, ev[0], ev[1]);
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (cur != p->device) cudaSetDevice(cur);
    KC_CUDA(le);
    KC_CUDA(se);
    for (u32 i = 0; i < p->launches; i++) kc_note_launch();
    memcpy(h_acc, p->h_acc, sizeof(kc_dev_acc) * p->nq);
    return KC_OK;
}
