/*
 * kclique.h -- C ABI of libkclique: exact k-clique counting and listing on one
 * NVIDIA GB300 (sm_103a) with the edge-oriented branch-and-bound method EBBkC
 * (Wang, Yu & Long, "Efficient k-Clique Listing: An Edge-Oriented Branching
 * Strategy", SIGMOD 2024, arXiv 2311.13798).
 *
 * Problem (paper Sec. 2, Def. "k-clique" and Problem "k-clique listing"): given
 * a simple undirected graph G = (V, E) and k >= 3, find every set of k vertices
 * whose pairs are all edges.
 *
 * Method (paper Sec. 4.4, Alg. 5 "EBBkC-H", with the early termination of Sec. 5):
 *   kclique_prepare  builds the symmetric CSR, the truss-based edge ordering
 *                    (Sec. 4.2, Eq. 6) by level-synchronous peeling, and for every
 *                    edge e the vertex set VSet(e) of its sub-branch (Eq. 2);
 *   kclique_count /  run, for every edge e whose |VSet(e)| >= k-2, the sub-branch
 *   kclique_list     g_e: greedy colouring, colour-ordered DAG (Sec. 4.3), edge
 *                    branching with pruning Rules (1) and (2), leaves at l = 1 and
 *                    l = 2 (Alg. 2), and early termination on cliques and 2-plexes
 *                    (Sec. 5, Alg. 6).
 *
 * Conventions
 *   - Vertex ids are uint32 in [0, n).  The input CSR may be non-symmetric and may
 *     hold duplicates and self-loops; directions, duplicates and loops are dropped
 *     (paper Sec. 6.1, "Datasets").
 *   - Edge ids number the undirected edges (u < v) in lexicographic order.
 *   - Counts are exact unsigned 128-bit integers (count_lo + 2^64 count_hi).
 *   - checksum = sum over listed cliques Q of prod_{v in Q} z(v) mod 2^64, with
 *     z(v) = splitmix64(v) | 1 (SplitMix64 output step, Steele-Lea-Flood 2014).
 *     The paper defines no checksum; this one is order independent.
 *   - Every call enqueues its GPU work on the caller's stream `s` (0 = legacy
 *     default stream) and returns after that work has finished, with the result
 *     in host memory.  A graph handle is read-only after prepare: concurrent
 *     count/list calls on one handle from different streams are allowed.
 *   - Errors are returned as kc_status; on error, output structs are zeroed and
 *     no handle is created.  The library never aborts the process and never traps
 *     the GPU: device-side failures (bounds, bounded waits) set a status word that
 *     the host reads back.
 */
#ifndef KCLIQUE_H
#define KCLIQUE_H

#include <stdint.h>

#if defined(__GNUC__)
#define KC_API __attribute__((visibility("default")))
#else
#define KC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *kc_stream; /* a cudaStream_t */

typedef enum {
    KC_OK = 0,
    KC_TRUNCATED = 1,          /* list buffer full: count/checksum still cover all cliques */
    KC_ERR_INVALID_ARG = -1,   /* bad pointer, k < 3, k > KC_MAX_K, ... */
    KC_ERR_INVALID_GRAPH = -2, /* row_ptr not monotone, column id >= n, nnz >= 2^32 */
    KC_ERR_OOM = -3,           /* device allocation failed */
    KC_ERR_CUDA = -4,          /* a CUDA runtime call failed */
    KC_ERR_TIMEOUT = -5,       /* a bounded device wait gave up */
    KC_ERR_OVERFLOW = -6,      /* the count reached 2^128 */
    KC_ERR_UNSUPPORTED = -7    /* a sub-branch wider than KC_MAX_BRANCH vertices survives */
} kc_status;

#define KC_MAX_K 32          /* largest k accepted */
#define KC_MAX_BRANCH 1024   /* largest |VSet(e)| a kernel holds in shared memory */

/* kc_params.flags */
#define KC_NO_ET 0x1u        /* disable early termination (Sec. 5) */
#define KC_NO_RULE2 0x2u     /* disable pruning Rule (2) (Sec. 4.3) */
#define KC_CHECKSUM 0x4u     /* also compute the checksum in kclique_count */
#define KC_NO_RULE1 0x8u     /* disable pruning Rule (1) (Sec. 4.3) */
#define KC_ROWS_ONLY 0x10u   /* kclique_list: rows only; see kclique_list for the totals */

typedef struct kc_graph kc_graph; /* opaque, device resident, immutable after prepare */

typedef struct {
    uint32_t t_max;            /* early termination on t-plexes, t <= t_max (1 or 2); 0 = paper's rule */
    uint32_t warps_per_block;  /* 0 = library default */
    uint32_t blocks;           /* persistent grid size; 0 = (SMs x resident blocks) */
    uint32_t flags;            /* KC_NO_ET | KC_NO_RULE2 | KC_CHECKSUM | KC_NO_RULE1 */
    uint64_t *d_edge_count;    /* optional device [m]: k-cliques whose first edge is e (mod 2^64) */
    uint64_t *d_edge_checksum; /* optional device [m]: their checksum */
    uint64_t *d_edge_cycles;   /* optional device [m]: SM clock cycles the warps spent on e's sub-branch */
    uint32_t split_min;        /* k >= 7: sub-branches with |VSet| >= split_min are split across warps,
                                  one work item per top-frame vertex (0 = 64; 0xFFFFFFFF = never) */
    uint32_t pad;
    uint64_t ticket_begin;     /* run only the top-level edges [ticket_begin, ticket_end) of the order by */
    uint64_t ticket_end;       /* |VSet| descending (0, 0 = all): a shard for one of several GPUs */
} kc_params;

typedef struct {
    uint64_t count_lo, count_hi; /* exact number of k-cliques */
    uint64_t checksum;           /* see conventions (0 unless requested or listing) */
    uint64_t written;            /* rows written to the list buffer (<= cap) */
    uint64_t edge_branches;      /* top-level sub-branches run (|VSet(e)| >= k-2) */
    uint64_t nodes;              /* branch frames expanded */
    uint64_t et_hits;            /* frames closed by early termination */
    uint64_t word_ops;           /* algorithmic bitset lane-ops: 3 per 32-bit word of every
                                    candidate-set intersection (AND, AND, POPC), 2 per word of
                                    every degree test (AND, POPC) */
    uint64_t pair_tests;         /* adjacency tests made while extracting sub-branches */
    float ms_prepare;            /* device time of the prepare call that built the graph */
    float ms_count;              /* device time of this call */
    float ms_branch;             /* device time of the branch kernels alone */
    float pad;
} kc_result;

typedef struct {
    uint32_t n;
    uint64_t m;              /* undirected edges after cleaning */
    uint64_t triangles;      /* = sum_e |VSet(e)| */
    uint32_t tau;            /* max |VSet(e)| = largest truss level (Eq. 7) */
    uint32_t max_degree;
    uint64_t rounds;         /* peeling rounds */
    uint64_t resident_bytes; /* device bytes held by the handle */
} kc_info;

/*
 * kclique_prepare -- clean the graph and build the truss-based edge ordering and
 * the per-edge sub-branch vertex sets (paper Alg. 5 line 1; Sec. 4.2 Eq. 6;
 * Alg. 3 lines 2-4 VSet/ESet).
 *   row_ptr[n+1], col[nnz]: CSR of uint32; on_device != 0 means both are device
 *     pointers, else host pointers (copied in).  Caller keeps ownership.
 *   out: receives a new handle owned by the caller (free with kclique_release).
 * Errors: KC_ERR_INVALID_ARG (null pointers), KC_ERR_INVALID_GRAPH, KC_ERR_OOM,
 *   KC_ERR_CUDA.
 */
KC_API kc_status kclique_prepare(const uint32_t *row_ptr, const uint32_t *col, uint32_t n, uint64_t nnz,
                          int on_device, kc_stream s, kc_graph **out);

/*
 * kclique_count -- exact number of k-cliques of a prepared graph (paper Alg. 5
 * lines 2-6 with EBBkC-C_Rec of Alg. 4, pruning Rules (1)-(2) of Sec. 4.3 and
 * early termination of Sec. 5).  p may be NULL (defaults).  r is written on
 * KC_OK.  k < 3 or k > KC_MAX_K: KC_ERR_INVALID_ARG.  k > tau + 2: count 0.
 */
KC_API kc_status kclique_count(const kc_graph *g, uint32_t k, const kc_params *p, kc_stream s, kc_result *r);

/*
 * kclique_list -- list the k-cliques into d_out, a caller-owned DEVICE buffer of
 * cap * k uint32: row-major, each row one clique in ascending original ids, row
 * order unspecified.  If more than cap cliques exist, the first cap found are
 * written, KC_TRUNCATED is returned, r->written = cap, and r->count /
 * r->checksum still cover all cliques.  The checksum is always computed.
 * The listing pass stops once the buffer is full; the totals then come from a
 * second pass, a count with checksum (r->ms_* and the work counters cover both).
 * With KC_ROWS_ONLY in p->flags that second pass is skipped: once the buffer is
 * full (r->written == cap) the call returns KC_TRUNCATED with r->count and
 * r->checksum 0 (the caller counts separately); otherwise they are the exact
 * totals as always.
 */
KC_API kc_status kclique_list(const kc_graph *g, uint32_t k, uint32_t *d_out, uint64_t cap,
                       const kc_params *p, kc_stream s, kc_result *r);

/* kclique_info -- sizes and statistics of a prepared graph (host struct). */
KC_API kc_status kclique_info(const kc_graph *g, kc_info *info);

/*
 * kclique_edge_data -- copy per-edge arrays of a prepared graph to host buffers
 * (any may be NULL): endpoints eu/ev [m] (u < v), truss level [m], peel round
 * [m], |VSet(e)| [m].  The edge order used by the method is (round, edge id).
 */
KC_API kc_status kclique_edge_data(const kc_graph *g, uint32_t *eu, uint32_t *ev, uint32_t *level,
                            uint32_t *round, uint32_t *vset_size, kc_stream s);

/* kclique_release -- free a handle (NULL is ignored). */
KC_API void kclique_release(kc_graph *g);

/* kclique_status_string -- static text for a status code. */
KC_API const char *kclique_status_string(kc_status st);

/* kclique_last_error -- text of the last failed CUDA call on this thread ("" if none). */
KC_API const char *kclique_last_error(void);

/*
 * kclique_count_batch -- many independent queries (graph, k) in one persistent
 * launch per width class; results[i] corresponds to (graphs[i], ks[i]).  The
 * per-query counts equal those of kclique_count on the same inputs.
 */
KC_API kc_status kclique_count_batch(const kc_graph *const *graphs, const uint32_t *ks, uint32_t nq,
                              const kc_params *p, kc_stream s, kc_result *results);

/*
 * kclique_count_batch_noalloc -- the batched count of kclique_count_batch for callers
 * that cannot allocate device memory when they count (a fixed pre-reserved pool, a
 * driver-thread callback, a process at its memory limit).  The paper has no
 * counterpart; this is an integration aid.  Per-call scratch comes from one static
 * device array of 32 KiB inside the library, so the call makes no cudaMalloc /
 * cudaFree and no allocating library call.  Arguments and results as for
 * kclique_count_batch, with these limits:
 *   - nq <= 64 queries per call, else KC_ERR_INVALID_ARG (kclique_last_error says why);
 *   - no per-edge outputs in p; sub-branches are never split across warps;
 *   - the first call on a device sets up that device (looks up the static arrays and
 *     fills a static binomial table); make it before any stream capture;
 *   - all calls on a device share the static scratch: calls that overlap on the GPU
 *     race, so the caller serialises them.
 */
KC_API kc_status kclique_count_batch_noalloc(const kc_graph *const *graphs, const uint32_t *ks, uint32_t nq,
                                             const kc_params *p, kc_stream s, kc_result *results);

/*
 * kclique_int_peak -- measurement utility (no counterpart in the paper): the sustained
 * rate of the branch kernel's inner operation mix, AND + AND + POPC on 32-bit words held
 * in registers, on the current device, in lane-ops per second (3 per word), with the SM
 * count.  Used as the denominator of the integer roofline.
 */
KC_API kc_status kclique_int_peak(double *lane_ops_per_s, int *sms, kc_stream s);

/* kclique_launch_count -- measurement utility: GPU kernels this library has launched in
 * this process (reset != 0: return the count and restart it at zero). */
KC_API unsigned long long kclique_launch_count(int reset);

/* kclique_kernel_rev -- measurement utility: a hash of the kernel sources this library
 * was built from, to tell whether stored profiler counters still describe it. */
KC_API const char *kclique_kernel_rev(void);

#ifdef __cplusplus
}
#endif

#endif /* KCLIQUE_H */
