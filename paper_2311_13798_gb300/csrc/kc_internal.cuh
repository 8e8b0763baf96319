// Internal declarations of libkclique (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/kclique.h"

typedef unsigned __int128 u128;
typedef uint64_t u64;
typedef uint32_t u32;

#define KC_CUDA(call)                                                   \
    do {                                                                \
        cudaError_t _e = (call);                                        \
        if (_e != cudaSuccess) {                                        \
            kc_set_last_cuda_error(_e, #call, __FILE__, __LINE__);      \
            return (_e == cudaErrorMemoryAllocation) ? KC_ERR_OOM : KC_ERR_CUDA; \
        }                                                               \
    } while (0)

void kc_set_last_cuda_error(cudaError_t e, const char *what, const char *file, int line);

// host-side count of kernel launches made by the library (for the bench's launch count)
void kc_note_launch();

// device-side status word bits (set by kernels, read by the host)
#define KC_DEV_ERR_BOUNDS 0x1u
#define KC_DEV_ERR_OVERFLOW 0x2u
#define KC_DEV_ERR_WIDTH 0x4u
#define KC_DEV_ERR_TIMEOUT 0x8u
#define KC_DEV_ERR_GRAPH 0x10u

// The checksum's key of vertex v: the first output of SplitMix64 seeded with v, made odd.
__device__ __forceinline__ u64 zkey(u64 v) {
    u64 x = v + 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    x = x ^ (x >> 31);
    return x | 1ull;
}

// Device-resident prepared graph.
struct kc_graph {
    int device;
    u32 n;
    u64 m;        // undirected edges
    u64 nnz;      // 2m
    u64 triangles;
    u32 tau;
    u32 max_degree;
    u64 rounds;
    u64 resident_bytes;
    float ms_prepare;
    // CSR (symmetric, sorted, deduplicated, loop free)
    u32 *row_ptr;     // [n+1]
    u32 *col;         // [2m]
    u32 *pos_eid;     // [2m] edge id of each CSR slot
    u32 *pos_round;   // [2m] peel round of each CSR slot's edge
    // edges
    u32 *eu, *ev;     // [m] endpoints u < v
    u32 *level;       // [m] truss level (trussness - 2)
    u32 *round;       // [m] peel round; edge order = (round, id)
    // sub-branch vertex sets (Eq. 2), ascending ids
    u64 *vset_ptr;    // [m+1]
    u32 *vset;        // [triangles]
    // tickets: edge ids sorted by |VSet| descending
    u32 *tickets;     // [m]
    // host copy: number of edges with |VSet| >= s, for s = 0..tau+1
    u64 *h_size_suffix; // [tau + 2]
    // scratch owned by the handle for count/list calls (reused, guarded by the stream order)
};

// ---- prepare (kc_prepare.cu)
kc_status kc_prepare_impl(const u32 *row_ptr, const u32 *col, u32 n, u64 nnz, int on_device, u32 ordering,
                          cudaStream_t s, kc_graph **out);
void kc_free_graph(kc_graph *g);

// ---- branch engine (kc_branch.cu)
struct kc_query {
    const kc_graph *g;
    u32 k;
    u64 ticket_begin;   // range of g->tickets to run
    u64 ticket_end;
    // per-query choices (0: the run's kc_run_cfg values)
    u32 t_max = 0, split_min = 0, width_min = 0;
};

struct kc_run_cfg {
    u32 t_max;          // 0: the paper's rule per query (kc_pick_t); else at most 3
    u32 flags;
    u32 warps_per_block;
    u32 blocks;
    int list;           // 1 = write cliques
    int stop_full;      // list: end the pass once the buffer is full (totals then partial)
    u32 *d_out;
    u64 cap;
    u64 *d_edge_count;
    u64 *d_edge_checksum;
    u64 *d_edge_cycles;
    u32 split_min;      // 0: default; ~0u: never split
    u32 width_min;      // 0: the narrowest width class that holds a sub-branch
    u64 ticket_begin, ticket_end;  // shard of the ticket order (0, 0 = all)
};

// Accumulators in device memory (one per query).
struct kc_dev_acc {
    unsigned long long count_lo, count_hi;
    unsigned long long checksum;
    unsigned long long written;   // rows reserved (may exceed cap)
    unsigned long long nodes;
    unsigned long long et_hits;
    unsigned long long branches;
    unsigned long long word_ops;
    unsigned long long pair_tests;
    unsigned long long sec[6];    // profiling only: SM cycles per section (lane 0 of each warp)
    unsigned int status;
    unsigned int pad;
};

kc_status kc_run_queries(const kc_query *q, u32 nq, const kc_run_cfg *cfg, cudaStream_t s,
                         kc_dev_acc *h_acc, float *ms, float *ms_branch);

// Batch plans (kc_branch.cu): the launches of one batch of queries captured once as a
// CUDA graph and replayed per run (one run of a plan at a time)
struct kc_plan;
kc_status kc_plan_create(const kc_query *qv, u32 nq, const kc_run_cfg *cfg, cudaStream_t s, kc_plan **out);
kc_status kc_plan_run(kc_plan *p, cudaStream_t s, kc_dev_acc *h_acc, float *ms);
void kc_plan_free(kc_plan *p);

// EBBkC-T (Alg. 3, kc_branch_t.cu): one count of g at k with every level of the branching
// in the global truss-based edge order; cfg's flags (KC_CHECKSUM) and ticket shard apply
kc_status kc_run_ebbkc_t(const kc_graph *g, u32 k, const kc_run_cfg *cfg, cudaStream_t s, kc_dev_acc *h_acc,
                         float *ms, float *ms_branch);

// early-termination threshold t of one query (0 = the paper's rule)
u32 kc_pick_t(u32 t_max, u32 k, u32 tau);

// binomial table on the device (saturating u128), built on first use per device
kc_status kc_ensure_tables(cudaStream_t s);

// entries of the binomial table: C(n, r) for n < 1025, r < 33
#define KC_BINOM_ENTRIES (1025 * 33)

// ---- no-allocation count path (kc_noalloc.cu): scratch and table supplied by the caller
kc_status kc_fill_binom(u128 *table, cudaStream_t s);
u64 kc_scratch_bytes_for(u32 nq);
kc_status kc_run_queries_in_scratch(const kc_query *q, u32 nq, const kc_run_cfg *cfg, cudaStream_t s,
                                    unsigned char *d_scratch, u64 scratch_bytes, const u128 *d_binom,
                                    kc_dev_acc *h_acc);
kc_status kc_preload_fixed_kernels();
void kc_set_last_error_msg(const char *msg);

// ---- small host helpers
static inline u64 kc_div_up(u64 a, u64 b) { return (a + b - 1) / b; }
