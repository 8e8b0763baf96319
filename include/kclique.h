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
 *                    l = 2 (Alg. 2), and early termination on cliques, 2-plexes
 *                    and 3-plexes (Sec. 5, Alg. 6 and Alg. 7).
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
#define KC_TRUSS_INNER 0x20u /* kclique_count: EBBkC-T (Alg. 3), every level of the branching in the
                                global truss-based edge order instead of the colour order inside the
                                sub-branches; no colouring, no Rules (1)-(2), no early termination (the
                                ordering ablation of Sec. 6.2).  Not with kclique_list or per-edge outputs:
                                KC_ERR_INVALID_ARG */

typedef struct kc_graph kc_graph; /* opaque, device resident, immutable after prepare */

typedef struct {
    uint32_t t_max;            /* early termination on t-plexes, t <= t_max (1, 2 or 3; larger = 3);
                                  0 = the paper's rule (Sec. 6.1): t = 2 if k <= tau/2, else 3 */
    uint32_t warps_per_block;  /* warps per persistent block, 1..4 (0 or larger = 4) */
    uint32_t blocks;           /* persistent grid size; 0 = (SMs x resident blocks) */
    uint32_t flags;            /* KC_NO_ET | KC_NO_RULE2 | KC_CHECKSUM | KC_NO_RULE1 */
    uint64_t *d_edge_count;    /* optional device [m]: k-cliques whose first edge is e (mod 2^64) */
    uint64_t *d_edge_checksum; /* optional device [m]: their checksum */
    uint64_t *d_edge_cycles;   /* optional device [m]: SM clock cycles the warps spent on e's sub-branch */
    uint32_t split_min;        /* k >= 7: sub-branches with |VSet| >= split_min are split across warps,
                                  one work item per top-frame vertex (0 = 64; 0xFFFFFFFF = never) */
    uint32_t width_min;        /* bitset width class: sub-branches of fewer than 32 * width_min vertices
                                  run in the kernels for width_min words (1, 2, 4, 8, 16, 32; 0 = the
                                  narrowest that holds them) */
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
 * the per-edge sub-branch vertex sets (paper Alg. 5; Sec. 4.2 Eq. 6;
 * Alg. 3 VSet/ESet).
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
 * with EBBkC-C_Rec of Alg. 4, pruning Rules (1)-(2) of Sec. 4.3 and
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

/*
 * kclique_prepare_ordered -- kclique_prepare with a choice of the top-level edge order:
 *   KC_ORDER_TRUSS  the truss-based ordering (Sec. 4.2, Eq. 6): EBBkC-H, the default;
 *   KC_ORDER_COLOUR the colour-based ordering (Sec. 4.3, Alg. 4): a greedy
 *                   colouring of G in decreasing (degree, id) order, vertices sorted by
 *                   non-increasing colour (ties by id), each edge branching on the common
 *                   out-neighbours of its endpoints (EBBkC-C; the ablation of Sec. 6).
 * Every order gives the same counts, checksums and cliques; only the work changes.
 * KC_ERR_UNSUPPORTED if (colours + 1) * n does not fit 32 bits.
 */
#define KC_ORDER_TRUSS 0u
#define KC_ORDER_COLOUR 1u
KC_API kc_status kclique_prepare_ordered(const uint32_t *row_ptr, const uint32_t *col, uint32_t n, uint64_t nnz,
                                         int on_device, uint32_t ordering, kc_stream s, kc_graph **out);

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
 * kclique_count_batch_tuned -- kclique_count_batch with per-query choices: qp[i] (when qp
 * is not NULL) gives t_max, split_min and width_min of query i (an autotuner's picks);
 * flags, blocks and warps_per_block come from p.  Results as for kclique_count_batch.
 */
KC_API kc_status kclique_count_batch_tuned(const kc_graph *const *graphs, const uint32_t *ks, const kc_params *qp,
                                           uint32_t nq, const kc_params *p, kc_stream s, kc_result *results);

/*
 * Batch plans -- a batch that is counted again and again (the same graphs, ks and
 * parameters) as one CUDA graph: kclique_batch_plan_create builds the batch's launch
 * groups and their device buffer, runs the batch once (which sizes every buffer), then
 * captures the copy of the buffer image, the persistent launches and the copy of the
 * results back as one graph.  kclique_batch_plan_run replays it on stream s, waits for it
 * and writes results[0..nq) exactly as kclique_count_batch_tuned would (ms_count: the
 * replay's time).  Arguments of create as for kclique_count_batch_tuned; the graphs must
 * outlive the plan, and no per-edge outputs may be set in p.  The plan owns its device
 * and pinned host buffers until kclique_batch_plan_release.  One run of a plan at a time
 * (runs of different plans may overlap on different streams).  Errors: as for the batch;
 * a failure inside the capture releases everything made so far and returns KC_ERR_CUDA.
 * The batching layer of the serving/batching design (no counterpart in the paper).
 */
typedef struct kc_batch_plan kc_batch_plan;
KC_API kc_status kclique_batch_plan_create(const kc_graph *const *graphs, const uint32_t *ks, const kc_params *qp,
                                           uint32_t nq, const kc_params *p, kc_stream s, kc_batch_plan **out);
KC_API kc_status kclique_batch_plan_run(kc_batch_plan *plan, kc_stream s, kc_result *results);
KC_API void kclique_batch_plan_release(kc_batch_plan *plan);

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
 * ---- Serving: a continuous-batching query server (no counterpart in the paper; the
 * serving layer around the exact method, whose arithmetic it does not change) ----
 *
 * Requests -- count (graph, k), list (graph, k, rows), upload (a host CSR) -- are
 * submitted at any time and complete asynchronously; kc_server_poll returns their
 * completions.  Inside, one thread runs every count request waiting when the previous
 * batch ended as ONE kclique_count_batch call (continuous batching); list_workers
 * threads write listing rows, each on its own stream (a listing whose buffer filled
 * gets its exact totals from a count entry that joins the next batch); an upload
 * thread prepares uploaded graphs on its own stream.  Their work overlaps on the GPU.
 * Prepared graphs stay resident across requests.  Uploads are admitted against an HBM
 * budget: the resident bytes of all graphs (kc_info.resident_bytes) plus an estimate
 * for graphs being prepared may not exceed it; least-recently-used unpinned graphs
 * that no request waits on are released to make room, and an upload that still does
 * not fit completes with KC_ERR_OOM.  Each result equals that of the same call made
 * alone (integer results: exactly).
 */
typedef struct kc_server kc_server;

/* The calls the server makes.  NULL in kc_server_config = this library on the GPU
 * (kclique_prepare / kclique_count_batch with KC_CHECKSUM / kclique_list with
 * KC_ROWS_ONLY into a device buffer copied to `rows` / kclique_release).  count_batch's
 * qp[i] holds the per-request choices of kc_request (t_max, split_min, width_min; 0 =
 * the server's kc_server_config.params).  A caller may
 * pass stand-ins to exercise the scheduling without a GPU.  Graph handles are opaque
 * to the server.  list: write up to cap rows of k ids to the HOST buffer rows (may be
 * NULL) and return KC_TRUNCATED with r->written == cap when the buffer filled (totals
 * then unknown), else KC_OK with the exact totals. */
typedef struct {
    void *ctx;
    kc_status (*prepare)(void *ctx, const uint32_t *row_ptr, const uint32_t *col, uint32_t n, uint64_t nnz,
                         void **graph, uint64_t *resident_bytes);
    kc_status (*count_batch)(void *ctx, void *const *graphs, const uint32_t *ks, const kc_params *qp, uint32_t nq,
                             kc_result *results);
    kc_status (*list)(void *ctx, void *graph, uint32_t k, uint32_t *rows, uint64_t cap, kc_result *r);
    void (*release)(void *ctx, void *graph);
} kc_server_backend;

typedef struct {
    uint64_t hbm_budget_bytes;         /* 0 = 120 GiB */
    uint32_t max_batch;                /* count requests per batched call; 0 = 512 */
    uint32_t list_workers;             /* listings in flight at once; 0 = 4 */
    int32_t device;                    /* CUDA device of the GPU backend; -1 = the current one */
    uint32_t upload_workers;           /* uploads prepared at once; 0 = 4 */
    uint32_t yield_ms;                 /* short work first: a count batch waits while uploads or
                                          listings are queued or running, at most this many
                                          milliseconds; 0 = 1000, KC_SERVER_NO_YIELD = never waits */
    uint32_t pad;
    kc_params params;                  /* for every count batch and listing (per-edge outputs must be NULL) */
    const kc_server_backend *backend;  /* NULL = the GPU */
} kc_server_config;

#define KC_SERVER_NO_YIELD 0xFFFFFFFFu

#define KC_REQ_COUNT 0u
#define KC_REQ_LIST 1u
#define KC_REQ_UPLOAD 2u

typedef struct {
    uint32_t kind;            /* KC_REQ_COUNT | KC_REQ_LIST | KC_REQ_UPLOAD */
    uint32_t k;               /* count / list */
    uint64_t graph;           /* count / list: a graph id (from kc_server_adopt or an upload) */
    uint64_t cap;             /* list: rows wanted */
    uint32_t *rows;           /* list: caller-owned HOST buffer of cap * k uint32 (or NULL), written
                                 before the completion is posted; keep it alive until then */
    const uint32_t *row_ptr;  /* upload: host CSR, copied by kc_server_submit */
    const uint32_t *col;
    uint32_t n;
    uint32_t pin;             /* upload: never evicted */
    uint64_t nnz;
    uint32_t t_max, split_min, width_min;  /* count: this request's choices (an autotuner's picks);
                                              0 = the server's params */
    uint32_t pad;
} kc_request;

typedef struct {
    uint64_t ticket;          /* as returned by kc_server_submit */
    uint64_t graph;
    uint32_t kind, k;
    int32_t status;           /* kc_status; a listing whose rows were cut at cap: KC_TRUNCATED with exact
                                 totals; a request on an unknown graph: KC_ERR_INVALID_ARG */
    uint32_t pad;
    uint64_t count_lo, count_hi, checksum;
    uint64_t written;         /* list: rows in rows[] */
    double t_submit, t_done;  /* seconds on the server's monotonic clock */
} kc_completion;

typedef struct {
    uint64_t submitted, completed, rejected, evictions;
    uint64_t batches, batched_queries, max_batch_seen;
    uint64_t resident_bytes, graphs, inflight;
    double busy_count_s, busy_list_s, busy_upload_s;  /* seconds inside backend calls */
} kc_server_counters;

/* kc_server_create -- start a server (threads, streams).  cfg may be NULL (defaults). */
KC_API kc_status kc_server_create(const kc_server_config *cfg, kc_server **out);

/* kc_server_adopt -- hand a prepared graph to the server (it releases it when evicted or
 * destroyed); resident_bytes 0 = take kc_info.resident_bytes (GPU backend).  pin != 0:
 * never evicted.  *graph_id receives its id. */
KC_API kc_status kc_server_adopt(kc_server *sv, void *graph, uint64_t resident_bytes, int pin, uint64_t *graph_id);

/* kc_server_submit -- queue a request; *ticket identifies its completion.  graph_id
 * (may be NULL) receives the graph's id; for an upload it is the new graph's id, and
 * requests on it may be submitted at once (they wait for its prepare).  Invalid
 * requests (k < 3, k > KC_MAX_K, null upload arrays) return KC_ERR_INVALID_ARG. */
KC_API kc_status kc_server_submit(kc_server *sv, const kc_request *req, uint64_t *ticket, uint64_t *graph_id);

/* kc_server_poll -- move up to max completions to out; waits up to wait_ms ms for the
 * first one (0: no wait, < 0: no limit).  Returns the number moved. */
KC_API uint32_t kc_server_poll(kc_server *sv, kc_completion *out, uint32_t max, int32_t wait_ms);

KC_API kc_status kc_server_stats(kc_server *sv, kc_server_counters *st);

/* kc_server_destroy -- finish every submitted request, stop the threads, release the
 * graphs it holds.  Completions not yet polled are dropped. */
KC_API void kc_server_destroy(kc_server *sv);

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
