// kclique_count_batch_noalloc: batched k-clique counting that allocates no device memory.
//
// Who needs it: code that cannot call cudaMalloc at the moment it counts -- for example
// a host that hands the GPU out under a fixed memory pool or a pre-reserved arena, a
// callback running on a driver thread where allocation is not allowed, or a process that
// has reached its device-memory limit and must still answer queries on graphs it already
// prepared.  The regular kclique_count / kclique_count_batch allocate their per-call
// scratch (query table, accumulators, counters, split buffers) with cudaMallocAsync; this
// entry point instead takes that scratch from one file-scope static __device__ array of
// a fixed size, so it calls no cudaMalloc, cudaFree or allocating library routine.
//
// Limits and behaviour:
//   * at most KC_NOALLOC_MAX_QUERIES queries per call (scratch is sized for that many);
//     a larger batch is rejected with KC_ERR_INVALID_ARG and a kclique_last_error text;
//   * sub-branches are not split across warps (splitting needs buffers proportional to
//     the graph), so very heavy k >= 7 queries run slower than through kclique_count;
//   * per-edge outputs of kc_params are not supported (rejected as KC_ERR_INVALID_ARG);
//   * the first call on a device does a one-time set-up with that device current: it
//     looks up the device addresses of the static arrays (cudaGetSymbolAddress), loads
//     the code of every kernel this path can launch (module loading is lazy by default,
//     and loading a kernel takes device memory) and fills the static binomial table
//     with one kernel.  Make that first call early -- before any stream capture, and
//     before the process is at its device-memory limit;
//   * the set-up is kept per device index for the life of the process: after a
//     cudaDeviceReset (or any teardown of the device's primary context) the cached
//     addresses are stale, so the entry point must not be used across a reset;
//   * kc_params.warps_per_block and .blocks act as for kclique_count_batch; the
//     timings ms_count and ms_branch are left at 0 (timing would need events);
//   * every call on a device shares the same scratch array, which keeps the previous
//     call's contents (the accumulators are cleared at the start of each call).  Calls
//     that overlap on the GPU -- from different host threads or streams -- race on it;
//     the caller must serialise them.
#include <cuda_runtime.h>
#include <string.h>

#include <mutex>

#include "kc_internal.cuh"

#define KC_NOALLOC_MAX_QUERIES 64u
#define KC_NOALLOC_SCRATCH_BYTES (32u << 10)

// Scratch of the no-allocation path (every GPU that loads the library holds it until exit).
static __device__ __align__(256) unsigned char kc_noalloc_scratch[KC_NOALLOC_SCRATCH_BYTES];
// Binomial table C(n, r), n < 1025, r < 33 (saturating 128-bit), filled once per device.
static __device__ __align__(256) u128 kc_noalloc_binom[KC_BINOM_ENTRIES];

namespace {

struct NoallocDevice {
    bool ready = false;
    unsigned char *scratch = nullptr;  // device address of kc_noalloc_scratch
    u128 *binom = nullptr;             // device address of kc_noalloc_binom
};

std::mutex g_noalloc_mu;
NoallocDevice g_noalloc_dev[64];

// One-time set-up per device (the device must be current).  In host code the names of
// the static arrays are host-side stand-ins, not device addresses: the addresses come
// from cudaGetSymbolAddress.
kc_status noalloc_setup(int dev, cudaStream_t s, NoallocDevice **out) {
    if (dev < 0 || dev >= 64) return KC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    NoallocDevice &d = g_noalloc_dev[dev];
    if (!d.ready) {
        void *sc = nullptr, *bt = nullptr;
        KC_CUDA(cudaGetSymbolAddress(&sc, kc_noalloc_scratch));
        KC_CUDA(cudaGetSymbolAddress(&bt, kc_noalloc_binom));
        kc_status st = kc_preload_fixed_kernels();
        if (st != KC_OK) return st;
        st = kc_fill_binom((u128 *)bt, s);
        if (st != KC_OK) return st;
        d.scratch = (unsigned char *)sc;
        d.binom = (u128 *)bt;
        d.ready = true;
    }
    *out = &d;
    return KC_OK;
}

kc_status status_of(unsigned st) {
    if (st & KC_DEV_ERR_OVERFLOW) return KC_ERR_OVERFLOW;
    if (st & KC_DEV_ERR_WIDTH) return KC_ERR_UNSUPPORTED;
    if (st & KC_DEV_ERR_TIMEOUT) return KC_ERR_TIMEOUT;
    if (st) return KC_ERR_CUDA;
    return KC_OK;
}

}  // namespace

extern "C" KC_API kc_status kclique_count_batch_noalloc(const kc_graph *const *graphs, const uint32_t *ks,
                                                         uint32_t nq, const kc_params *p, kc_stream sv,
                                                         kc_result *results) {
    if (!graphs || !ks || !results) return KC_ERR_INVALID_ARG;
    if (nq > KC_NOALLOC_MAX_QUERIES) {
        kc_set_last_error_msg("kclique_count_batch_noalloc: more queries than KC_NOALLOC_MAX_QUERIES (64) in one call");
        return KC_ERR_INVALID_ARG;
    }
    if (p && (p->d_edge_count || p->d_edge_checksum || p->d_edge_cycles)) {
        kc_set_last_error_msg("kclique_count_batch_noalloc: per-edge outputs are not supported");
        return KC_ERR_INVALID_ARG;
    }
    memset(results, 0, sizeof(kc_result) * nq);
    if (nq == 0) return KC_OK;
    cudaStream_t s = (cudaStream_t)sv;
    const int dev = graphs[0] ? graphs[0]->device : -1;
    kc_query qv[KC_NOALLOC_MAX_QUERIES];
    u32 idx[KC_NOALLOC_MAX_QUERIES];
    u32 nrun = 0;
    for (u32 i = 0; i < nq; i++) {
        const kc_graph *g = graphs[i];
        if (!g || ks[i] < 3 || ks[i] > KC_MAX_K || g->device != dev) return KC_ERR_INVALID_ARG;
        results[i].ms_prepare = g->ms_prepare;
        if ((u64)ks[i] > (u64)g->tau + 2) continue;  // omega <= tau + 2: no k-clique
        const u64 lo = (u64)KC_MAX_BRANCH + 1 > (u64)ks[i] - 2 ? (u64)KC_MAX_BRANCH + 1 : (u64)ks[i] - 2;
        if (lo <= g->tau && g->h_size_suffix[lo]) return KC_ERR_UNSUPPORTED;
        qv[nrun].g = g;
        qv[nrun].k = ks[i];
        qv[nrun].ticket_begin = 0;
        qv[nrun].ticket_end = 0;
        idx[nrun++] = i;
    }
    if (!nrun) return KC_OK;
    int prev = -1;
    KC_CUDA(cudaGetDevice(&prev));
    if (prev != dev) KC_CUDA(cudaSetDevice(dev));
    NoallocDevice *nd = nullptr;
    kc_status st = noalloc_setup(dev, s, &nd);
    kc_run_cfg cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.t_max = p ? p->t_max : 0u;  // 0: the paper's rule per query
    cfg.flags = p ? p->flags : 0u;
    cfg.warps_per_block = p ? p->warps_per_block : 0u;
    cfg.blocks = p ? p->blocks : 0u;
    kc_dev_acc acc[KC_NOALLOC_MAX_QUERIES];
    if (st == KC_OK)
        st = kc_run_queries_in_scratch(qv, nrun, &cfg, s, nd->scratch, KC_NOALLOC_SCRATCH_BYTES, nd->binom, acc);
    if (prev != dev) cudaSetDevice(prev);
    if (st != KC_OK) return st;
    kc_status worst = KC_OK;
    for (u32 j = 0; j < nrun; j++) {
        kc_result &r = results[idx[j]];
        kc_status sj = status_of(acc[j].status);
        if (sj != KC_OK) worst = sj;
        r.count_lo = acc[j].count_lo;
        r.count_hi = acc[j].count_hi;
        r.checksum = (p && (p->flags & KC_CHECKSUM)) ? acc[j].checksum : 0ull;
        r.edge_branches = acc[j].branches;
        r.nodes = acc[j].nodes;
        r.et_hits = acc[j].et_hits;
        r.word_ops = acc[j].word_ops;
        r.pair_tests = acc[j].pair_tests;
    }
    return worst;
}
