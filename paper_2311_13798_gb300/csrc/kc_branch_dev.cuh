// Branch engine, device side: the per-edge sub-branches of EBBkC-H (paper Alg. 5,
// EBBkC-C_Rec of Alg. 4) with early termination (Sec. 5), on one GB300.
//
// Work unit = one top-level edge e (a "ticket"), tickets sorted by |VSet(e)|
// descending and handed out by an atomic counter to persistent warps.  One warp
// owns a ticket end to end:
//   A5  extraction: bitset adjacency of g_e on VSet(e), keeping a pair (w, x) only
//       if (w, x) is an edge that comes after e in the (round, id) order -- the
//       suffix-graph edges of Eq. 2;
//   A6  greedy colouring (first fit in non-increasing local degree order, Sec. 4.3)
//       and renumbering so that positions run in non-increasing colour; the DAG of
//       Alg. 4 is implicit (out-neighbours = neighbours at larger positions);
//   A7  edge branching with an explicit per-depth stack; each batch of up to 32
//       child edges (u -> v) is evaluated lane-per-child: C' = C & N(u) & N(v) &
//       {positions > v}; Rule (1) limits u and v to colour prefixes, Rule (2)
//       counts the distinct colours of C' with one carry-propagating add per word;
//   A8  leaves l = 1 (|C'|) and l = 2 (edges of g[C']) (Alg. 2);
//   A9  early termination at every frame with l >= 3: a t-plex test on the minimum
//       degree, then C(|C|, l) for cliques and the kC2Plex count of Alg. 6 in
//       closed form, sum_j C(|F|, l-j) C(p, j) 2^j, for 2-plexes;
//   A10 exact 128-bit accumulation (per-lane partials, warp totals, one atomic
//       add with carry per warp) and the order-independent checksum;
//   A11 list emission with warp-aggregated slot reservation.
// Integer work only (AND, POPC, FFS); no tensor cores.
#pragma once
// This header holds the kernels and their launch templates; each kc_branch_w<W>.cu
// instantiates them for one bitset width W (words of 32 bits per adjacency row), so the
// widths compile in parallel, and kc_branch.cu drives the launches.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <vector>

#include "kc_internal.cuh"

// build-time tuning knobs (same results for every value)
#ifndef KC_SCAN_RATIO  // extraction scans a row when its length <= ratio x candidates left
#define KC_SCAN_RATIO 4
#endif
#ifndef KC_MINB8        // resident blocks per SM asked of the compiler, ticket kernel, W = 8
#define KC_MINB8 4      // (shared memory allows 3; 3 and 4 measured the same on k = 5 and 7)
#endif
#ifndef KC_ITEM_MINB8  // resident blocks per SM asked of the compiler, item kernel, W = 8
#define KC_ITEM_MINB8 6   // (6: 80 registers; 8 % faster than 4 on the power-law k = 7 run)
#endif
#ifndef KC_LANE_L3       // W <= 8: l = 3 children whose complement has at most
#define KC_LANE_L3 2      // KC_LANE_L3 * |C'| missing pairs are counted in their lane (0: off)
#endif
#ifndef KC_LANE_ET_MAX  // l = 3 children up to this size get the in-lane plex test; larger ones
#define KC_LANE_ET_MAX 1024  // go to the warp routine, which tests them too
#endif
#ifndef KC_SECTION_PROFILE  // 1: per-section cycle counters (KC_PROFILE=1 at run time)
#define KC_SECTION_PROFILE 0
#endif
#ifndef KC_DEBUG_BOUNDS  // 1: self-checking build (bounds of computed shared-memory indices)
#define KC_DEBUG_BOUNDS 0
#endif
#ifndef KC_ROW_PAD     // words of padding after each adjacency row (odd stride: no bank conflicts)
#define KC_ROW_PAD 1
#endif
#ifndef KC_COLD_NOINLINE  // 1: routines run once per sub-branch or per frame of l >= 4 stay
#define KC_COLD_NOINLINE 1  // out of line (one copy per kernel, a smaller hot loop)
#endif
#if KC_COLD_NOINLINE
#define KC_COLD __noinline__
#else
#define KC_COLD
#endif
#ifndef KC_PRECHECK    // per-u plex pre-check masks for l = 3 children (count mode); off:
#define KC_PRECHECK 0  // on the power-law workload the masks cost more than they saved
#endif


// types shared by the translation units of the branch engine
namespace kcb {
constexpr u32 kNoallocMaxQ = 64;  // queries per call of the no-allocation path

constexpr int WARPS_PER_BLOCK_DEFAULT = 4;
constexpr int BINOM_N = 1025;  // C(n, r) for n < BINOM_N
constexpr int BINOM_R = 33;    //            and r < BINOM_R
constexpr int MODE_CHECKSUM = 1;
constexpr int MODE_LIST = 2;
// count modes are compiled per parity of k: frames hold l = k - 2 - 2 d, so a kernel for
// odd k never meets the l = 2 leaves and one for even k never meets l = 3 frames
constexpr int MODE_ODD = 4;
constexpr int MODE_EVEN = 8;

const u128 SAT128 = ~(u128)0;

struct QDesc {
    const u32 *row_ptr, *col, *pos_eid, *pos_round, *eu, *ev, *round, *vset, *tickets;
    const u64 *vset_ptr;
    u32 k;
    u32 t_max;        // early termination on t-plexes, t <= t_max (0: none)
    u64 t0;           // first ticket (index into tickets) of this launch's range
    u64 nt;           // tickets in range
    u64 nheavy;       // the first nheavy tickets of the range are split (k >= 7)
    kc_dev_acc *acc;
    u64 *edge_count;
    u64 *edge_checksum;
    u64 *edge_cycles;
};

struct Args {
    const QDesc *qs;
    const u64 *qstart;  // [nq+1] prefix of nt
    u32 nq;
    u32 D;              // depth slots in the shared-memory layout
    u32 warp_bytes;
    u32 t_max;
    u32 flags;
    u32 prof;           // 1: accumulate per-section cycles (KC_PROFILE)
    unsigned long long *ticket_ctr;
    // splitting of heavy sub-branches (A12)
    unsigned char *slots;           // [slot_cap] published sub-branches (nullptr: no splitting)
    unsigned long long *slot_ctr;
    u64 slot_cap;
    unsigned long long *slot_next;  // slots taken by branch_items_kernel blocks
    u32 *d_out;
    u64 cap;
    u32 stop_full;      // list: leave once the buffer is full
    u32 pad_;
    const u128 *binom;
    unsigned long long *l3hist;  // profiling only: [2][8] l = 3 frames and their cycles by size
};

// device buffers of the split path, grown on demand and reused across classes
struct SplitBufs {
    unsigned char *slots = nullptr;
    u64 slot_bytes_cap = 0;
};

// per-width entry points (defined by KC_BRANCH_WIDTH in kc_branch_w<W>.cu)
#define KC_BRANCH_DECLARE(W)                                                                                      \
    kc_status launch_width_##W(int mode, const Args &a, const std::vector<QDesc> &qs, u64 tickets,                \
                               const kc_run_cfg *cfg, cudaStream_t s, QDesc *d_qs, u64 *d_qstart,                 \
                               unsigned long long *d_ctr, SplitBufs *sb);                                         \
    kc_status launch_fixed_width_##W(int mode, const Args &a, const QDesc *qs, u32 nqs, const kc_run_cfg *cfg,    \
                                     cudaStream_t s, QDesc *d_qs, u64 *d_qstart, unsigned long long *d_ctr);      \
    kc_status preload_width_##W();                                                                                \
    unsigned long long debug_flag_width_##W();
KC_BRANCH_DECLARE(1)
KC_BRANCH_DECLARE(2)
KC_BRANCH_DECLARE(4)
KC_BRANCH_DECLARE(8)
KC_BRANCH_DECLARE(16)
KC_BRANCH_DECLARE(32)
#undef KC_BRANCH_DECLARE
}  // namespace kcb

#ifdef KC_BRANCH_INSTANTIATE
namespace {
using namespace kcb;

// ---------------------------------------------------------------- helpers
#if KC_DEBUG_BOUNDS
// first violation: (source line << 40) | (index & 0xFFFFF) << 20 | (bound & 0xFFFFF)
__device__ unsigned long long g_kc_dbg;
__device__ __noinline__ bool kc_dbg_ok(long long i, long long n, int line) {
    if (i >= 0 && i < n) return true;
    atomicCAS(&g_kc_dbg, 0ull, ((unsigned long long)line << 40) | ((unsigned long long)(i & 0xFFFFF) << 20) |
                                   (unsigned long long)(n & 0xFFFFF));
    return false;
}
#define KC_OK(i, n) kc_dbg_ok((long long)(i), (long long)(n), __LINE__)
// the first violation recorded by this translation unit's kernels (cleared on read)
unsigned long long read_debug_flag() {
    unsigned long long dbg = 0, zero = 0;
    if (cudaMemcpyFromSymbol(&dbg, g_kc_dbg, sizeof(dbg)) == cudaSuccess && dbg)
        cudaMemcpyToSymbol(g_kc_dbg, &zero, sizeof(zero));
    return dbg;
}
#else
#define KC_OK(i, n) true
unsigned long long read_debug_flag() { return 0; }
#endif

__device__ __forceinline__ u128 add_sat(u128 a, u128 b) {
    u128 s = a + b;
    return (a == SAT128 || b == SAT128 || s < a) ? SAT128 : s;
}

__device__ __forceinline__ u128 mul_sat(u128 a, u128 b) {
    if (a == 0 || b == 0) return 0;
    if (a == SAT128 || b == SAT128) return SAT128;
    u64 ah = (u64)(a >> 64), bh = (u64)(b >> 64);
    if (ah == 0 && bh == 0) {
        u64 al = (u64)a, bl = (u64)b;
        return ((u128)__umul64hi(al, bl) << 64) | (u128)(al * bl);
    }
    if (ah != 0 && bh != 0) return SAT128;
    if (a > SAT128 / b) return SAT128;
    return a * b;
}

__device__ __forceinline__ u128 binom(const u128 *T, int n, int r) {
    if (r < 0 || r > n) return 0;
    if (n >= BINOM_N || r >= BINOM_R) return SAT128;
    return T[n * BINOM_R + r];
}

// mask of positions > p inside word w
__device__ __forceinline__ u32 gt_mask(int p, int w) {
    int pw = p >> 5;
    if (w < pw) return 0u;
    if (w > pw) return 0xFFFFFFFFu;
    int b = p & 31;
    return b == 31 ? 0u : (0xFFFFFFFFu << (b + 1));
}

// mask of positions < lim inside word w
__device__ __forceinline__ u32 lt_mask(int lim, int w) {
    int lw = lim >> 5;
    if (w < lw) return 0xFFFFFFFFu;
    if (w > lw) return 0u;
    int b = lim & 31;
    return b == 0 ? 0u : (0xFFFFFFFFu >> (32 - b));
}

__device__ __forceinline__ u64 warp_sum_u64(u64 x) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

__device__ __forceinline__ u128 warp_sum_u128(u64 x) {
    // sum of 32 u64 values without overflow: split into halves
    u64 lo = x & 0xFFFFFFFFull, hi = x >> 32;
    lo = warp_sum_u64(lo);
    hi = warp_sum_u64(hi);
    return ((u128)hi << 32) + (u128)lo;
}

// ---------------------------------------------------------------- smem layout
struct Lay {
    u32 *A;          // [S][W + KC_ROW_PAD] adjacency rows (undirected, positions); an odd
                     // row stride puts word w of 32 different rows in 32 different banks
    u32 *C0;         // [W] top frame
    u32 *vid;        // [S] vertex id per position
    u64 *z;          // [S] key per position
    uint16_t *col;   // [S] colour per position
    uint16_t *aux;   // [S] scratch (degree / order / class index)
    uint16_t *aux2;  // [S] scratch (positions list)
    uint16_t *lim;   // [S+2] number of positions with colour >= c
    u32 *J, *E;      // [W] colour segment masks
    u32 *V;          // [D][W] generator: remaining v candidates
    int *cur;        // [D] generator: current u
    int *nchild;     // [D]
    int *nextc;      // [D]
    int *slot;       // [D]
    u32 *childC;     // [D][32][W]
    u64 *childP;     // [D][32]
    u32 *childUV;    // [D][32]
    u32 *path;       // [2D+4]
    uint16_t *bu, *bv;  // [32]
    uint8_t *bs;        // [32] ring slot of each batch entry's u (plex pre-check)
    u32 *Bm, *M1;       // [4][W] per-u masks of the last 4 u's (plex pre-check; only the one
                        // depth whose frames have l = 5 uses them)
    int *rn;            // [D] u's entered into the ring so far
    u32 *tmpW;       // [W]
    u32 *tmpW2;      // [W]
};

template <int W>
__host__ __device__ constexpr u32 align16(u32 x) { return (x + 15u) & ~15u; }

// The frame of a sub-branch (adjacency, ids, keys, colours, Rule 1/2 tables) is read-only
// once extracted and coloured; the item kernel keeps one copy per block, shared by its
// warps.  Everything else is per-warp DFS state.
template <int W>
__host__ __device__ u32 frame_bytes(bool sum) {
    const u32 S = 32u * W;
    u32 b = 0;
    b += align16<W>(4u * S * (W + KC_ROW_PAD)); // A
    b += align16<W>(4u * S);           // vid
    b += sum ? align16<W>(8u * S) : 0u;  // z (checksum / listing only)
    b += align16<W>(2u * S);           // col
    b += align16<W>(2u * (S + 2));     // lim
    b += align16<W>(8u * W);           // J, E
    return b;
}

// per-warp bytes; shared_frame: the frame lives elsewhere (one per block)
template <int W>
__host__ __device__ u32 lay_bytes(u32 D, bool sum, bool shared_frame = false) {
    const u32 S = 32u * W;
    u32 b = shared_frame ? 0u : frame_bytes<W>(sum);
    b += align16<W>(4u * W);           // C0
    b += align16<W>(2u * S);           // aux
    b += align16<W>(2u * S);           // aux2
    b += align16<W>(4u * D * W);       // V
    b += align16<W>(16u * D);          // cur, nchild, nextc, slot
    b += align16<W>(4u * D * 32 * W);  // childC
    b += sum ? align16<W>(8u * D * 32) : 0u;  // childP (checksum / listing only)
    b += align16<W>(4u * D * 32);      // childUV
    b += align16<W>(4u * (2 * D + 4)); // path
    b += align16<W>(2u * 64);          // bu, bv
    b += align16<W>(32u);              // bs
    b += KC_PRECHECK ? align16<W>(2u * 4u * 4 * W) : 0u;  // Bm, M1
    b += align16<W>(4u * D);           // rn
    b += align16<W>(8u * W);           // tmpW, tmpW2
    return b;
}

// p: this warp's bytes; frame: the shared frame (nullptr: the frame is at the start of p)
template <int W>
__host__ __device__ Lay make_lay(unsigned char *p, u32 D, bool sum, unsigned char *frame = nullptr) {
    const u32 S = 32u * W;
    Lay L;
    unsigned char *f = frame ? frame : p;
    u32 o = 0;
    L.A = (u32 *)(f + o); o += align16<W>(4u * S * (W + KC_ROW_PAD));
    L.vid = (u32 *)(f + o); o += align16<W>(4u * S);
    L.z = (u64 *)(f + o); o += sum ? align16<W>(8u * S) : 0u;
    L.col = (uint16_t *)(f + o); o += align16<W>(2u * S);
    L.lim = (uint16_t *)(f + o); o += align16<W>(2u * (S + 2));
    L.J = (u32 *)(f + o); L.E = L.J + W; o += align16<W>(8u * W);
    if (frame) o = 0;
    L.C0 = (u32 *)(p + o); o += align16<W>(4u * W);
    L.aux = (uint16_t *)(p + o); o += align16<W>(2u * S);
    L.aux2 = (uint16_t *)(p + o); o += align16<W>(2u * S);
    L.V = (u32 *)(p + o); o += align16<W>(4u * D * W);
    L.cur = (int *)(p + o); L.nchild = L.cur + D; L.nextc = L.nchild + D; L.slot = L.nextc + D;
    o += align16<W>(16u * D);
    L.childC = (u32 *)(p + o); o += align16<W>(4u * D * 32 * W);
    L.childP = (u64 *)(p + o); o += sum ? align16<W>(8u * D * 32) : 0u;
    L.childUV = (u32 *)(p + o); o += align16<W>(4u * D * 32);
    L.path = (u32 *)(p + o); o += align16<W>(4u * (2 * D + 4));
    L.bu = (uint16_t *)(p + o); L.bv = L.bu + 32; o += align16<W>(2u * 64);
    L.bs = (uint8_t *)(p + o); o += align16<W>(32u);
    L.Bm = (u32 *)(p + o); L.M1 = L.Bm + 4 * W; o += KC_PRECHECK ? align16<W>(2u * 4u * 4 * W) : 0u;
    L.rn = (int *)(p + o); o += align16<W>(4u * D);
    L.tmpW = (u32 *)(p + o); L.tmpW2 = L.tmpW + W; o += align16<W>(8u * W);
    return L;
}

// ---------------------------------------------------------------- warp primitives
template <int W>
__device__ __forceinline__ int warp_popc(const u32 *X, int lane) {
    int c = lane < W ? __popc(X[lane]) : 0;
    return __reduce_add_sync(0xffffffffu, (unsigned)c);
}

// smallest set bit position >= from, or -1
template <int W>
__device__ __forceinline__ int warp_first_from(const u32 *X, int from, int lane) {
    u32 x = 0;
    if (lane < W) x = X[lane] & ~lt_mask(from, lane);
    unsigned bal = __ballot_sync(0xffffffffu, x != 0);
    if (!bal) return -1;
    int fl = __ffs(bal) - 1;
    u32 wv = __shfl_sync(0xffffffffu, x, fl);
    return fl * 32 + __ffs(wv) - 1;
}

// position of the i-th set bit (i from 0) of a W-word set held in registers
template <int W>
__device__ __forceinline__ int select_bit(const u32 (&cw)[W], int i) {
    int before = 0, pos = -1;
#pragma unroll
    for (int w = 0; w < W; w++) {
        const int p = __popc(cw[w]);
        if (pos < 0 && i < before + p) pos = w * 32 + (int)__fns(cw[w], 0u, i - before + 1);
        before += p;
    }
    return pos;
}

// positions of the set bits of a W-word set held in registers, in increasing order, to
// out[0 .. popc): one ballot-free pass per word (lane j stores bit j of the word at its
// rank among the word's set bits)
template <int W>
__device__ __forceinline__ void compact_positions(const u32 (&cw)[W], uint16_t *out, int lane) {
    int base = 0;
    const u32 below = (1u << lane) - 1u;
#pragma unroll
    for (int w = 0; w < W; w++) {
        const u32 word = cw[w];
        if ((word >> lane) & 1u) out[base + __popc(word & below)] = (uint16_t)(w * 32 + lane);
        base += __popc(word);
    }
    __syncwarp();
}

// permute positions: new position r holds old position ord[r] (ord in L.aux2), rows and columns,
// plus vid / z / extra u16 array (optional)
// Returns false (and leaves A partly permuted) if ord is not a permutation.
template <int W>
__device__ KC_COLD bool permute(const Lay &L, int s, int lane, uint16_t *extra16) {
    const uint16_t *ord = L.aux2;
    // columns, row by row (each row is read fully before it is written)
    int src[W];
#pragma unroll
    for (int w = 0; w < W; w++) {
        int r = 32 * w + lane;
        src[w] = r < s ? ord[r] : -1;
    }
    for (int r = 0; r < s; r++) {
        u32 *row = L.A + r * (W + KC_ROW_PAD);
        u32 mine = 0;
#pragma unroll
        for (int w = 0; w < W; w++) {
            int sp = src[w];
            bool bit = sp >= 0 && KC_OK(sp, s) && ((row[sp >> 5] >> (sp & 31)) & 1u);
            u32 bal = __ballot_sync(0xffffffffu, bit);
            if (lane == w) mine = bal;
        }
        __syncwarp();
        if (lane < W) row[lane] = mine;
        __syncwarp();
    }
    // rows: follow the cycles of ord (visited bits in tmpW2)
    if (lane < W) L.tmpW2[lane] = 0;
    __syncwarp();
    int steps = 0;
    for (int st = 0; st < s; st++) {
        // lane 0 sets visited bits below; every lane takes lane 0's reading (the shuffle
        // also orders all lanes' reads before lane 0's next write)
        const int vis = __shfl_sync(0xffffffffu, (int)((L.tmpW2[st >> 5] >> (st & 31)) & 1u), 0);
        if (vis) continue;
        u32 keep = lane < W ? L.A[st * (W + KC_ROW_PAD) + lane] : 0;
        int j = st;
        while (true) {
            if (++steps > s) return false;  // not a permutation: bounded, reported by the caller
            int sp = ord[j];
            if (!KC_OK(sp, s) || !KC_OK(j, s)) return false;
            if (lane == 0) L.tmpW2[j >> 5] |= 1u << (j & 31);
            if (sp == st) {
                __syncwarp();
                if (lane < W) L.A[j * (W + KC_ROW_PAD) + lane] = keep;
                __syncwarp();
                break;
            }
            u32 t = lane < W ? L.A[sp * (W + KC_ROW_PAD) + lane] : 0;
            __syncwarp();
            if (lane < W) L.A[j * (W + KC_ROW_PAD) + lane] = t;
            __syncwarp();
            j = sp;
        }
    }
    // per-position arrays, gathered through shared scratch (the child-frame buffers,
    // unused while a sub-branch is being renumbered); keys are recomputed from ids
    u32 *tmp = L.childC;
    for (int r = lane; r < s; r += 32) tmp[r] = KC_OK(ord[r], s) ? L.vid[ord[r]] : 0u;
    __syncwarp();
    for (int r = lane; r < s; r += 32) L.vid[r] = tmp[r];
    __syncwarp();
    if (extra16) {
        for (int r = lane; r < s; r += 32) tmp[r] = extra16[ord[r]];
        __syncwarp();
        for (int r = lane; r < s; r += 32) extra16[r] = (uint16_t)tmp[r];
        __syncwarp();
    }
    return true;
}

// ---------------------------------------------------------------- state
struct Acc {
    u64 leaf;       // per lane: leaf counts of the current ticket
    u64 csum;       // per lane: checksum (mod 2^64)
    u128 cf;        // warp-uniform: closed-form counts of the current ticket
    u64 cf_csum;    // warp-uniform: closed-form checksum of the current ticket
    u64 nodes, et;  // per lane (lane 0 counts)
    u64 ops;        // per lane: algorithmic word-ops (3 per word of an intersection, 2 per degree word)
    u64 pairs;      // per lane: adjacency tests during extraction
#if KC_SECTION_PROFILE
    u64 sec[6];     // lane 0, profiling: extract, colour, ET (l >= 4), l=3 frames, generate, evaluate
#endif
    u32 status;
};

// ---------------------------------------------------------------- A5 extraction
template <int W>
__device__ __forceinline__ void extract_body(const Lay &L, const QDesc &q, int s, u32 e, u32 re, int lane, Acc &acc) {
    constexpr int RS = W + KC_ROW_PAD;
    for (int i = lane; i < s * RS; i += 32) L.A[i] = 0;
    __syncwarp();
    const u32 vmax = L.vid[s - 1];
    // rows in batches of 32: lane r restricts row ib + r to its columns in (x, vmax] (two
    // binary searches, 32 rows in flight at once), then the warp runs over the batch's
    // (row, item) pairs as one flat list, so short and long rows share the lanes evenly
    for (int ib = 0; ib + 1 < s; ib += 32) {
        const int i = ib + lane;
        u32 xb = 0, xe = 0;
        int work = 0, scan = 1;
        if (i + 1 < s) {
            const u32 x = L.vid[i];
            const u32 rb = q.row_ptr[x], re_ = q.row_ptr[x + 1];
            u32 lo = rb, hi = re_;
            while (lo < hi) { u32 mid = (lo + hi) >> 1; if (q.col[mid] <= x) lo = mid + 1; else hi = mid; }
            xb = lo;
            hi = re_;
            while (lo < hi) { u32 mid = (lo + hi) >> 1; if (q.col[mid] <= vmax) lo = mid + 1; else hi = mid; }
            xe = lo;
            const int rem = s - 1 - i;
            // scan the row (coalesced loads, binary search in shared vid) unless it is much
            // longer than the candidates; then search each candidate in the row instead
            scan = (xe - xb) <= (u32)KC_SCAN_RATIO * (u32)rem;
            work = scan ? (int)(xe - xb) : rem;
        }
        int off = work;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, off, o);
            if (lane >= o) off += y;
        }
        const int total = __shfl_sync(0xffffffffu, off, 31);
        off -= work;  // exclusive prefix
        for (int t0 = 0; t0 < total; t0 += 32) {
            const int t = t0 + lane;
            // the row of item t: the last lane r with off_r <= t (it has work_r > t - off_r)
            int r = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int o2 = __shfl_sync(0xffffffffu, off, r + step);
                if (o2 <= t) r += step;
            }
            const u32 xb_r = __shfl_sync(0xffffffffu, xb, r);
            const u32 xe_r = __shfl_sync(0xffffffffu, xe, r);
            const int scan_r = __shfl_sync(0xffffffffu, scan, r);
            const int k = t - __shfl_sync(0xffffffffu, off, r);
            if (t >= total) continue;
            const int ir = ib + r;
            acc.pairs++;
            int j = -1;
            u32 p = 0;
            if (scan_r) {
                p = xb_r + (u32)k;
                const u32 y = q.col[p];
                int lo = ir + 1, hi = s;
                while (lo < hi) { int mid = (lo + hi) >> 1; if (L.vid[mid] < y) lo = mid + 1; else hi = mid; }
                if (lo < s && L.vid[lo] == y) j = lo;
            } else {
                const int jj = ir + 1 + k;
                const u32 y = L.vid[jj];
                u32 lo = xb_r, hi = xe_r;
                while (lo < hi) { u32 mid = (lo + hi) >> 1; if (q.col[mid] < y) lo = mid + 1; else hi = mid; }
                if (lo < xe_r && q.col[lo] == y) { j = jj; p = lo; }
            }
            if (j >= 0) {
                const u32 rr = q.pos_round[p], ee = q.pos_eid[p];
                if ((rr > re || (rr == re && ee > e)) && KC_OK(ir, s) && KC_OK(j, s)) {
                    atomicOr(&L.A[ir * RS + (j >> 5)], 1u << (j & 31));
                    atomicOr(&L.A[j * RS + (ir >> 5)], 1u << (ir & 31));
                }
            }
        }
    }
    __syncwarp();
}

#ifndef KC_EXTRACT_NOINLINE  // 1: extraction out of line as well (measured slower at k = 5)
#define KC_EXTRACT_NOINLINE 0
#endif
#if KC_EXTRACT_NOINLINE
#define KC_EXTRACT_ATTR __noinline__
#else
#define KC_EXTRACT_ATTR __forceinline__
#endif
template <int W>
__device__ KC_EXTRACT_ATTR void extract(const Lay &L, const QDesc &q, int s, u32 e, u32 re, int lane, Acc &acc) {
    extract_body<W>(L, q, s, e, re, lane, acc);
}

// ---------------------------------------------------------------- A6 colouring
// Returns the number of colours.  Afterwards positions run in non-increasing
// colour; L.col[p] is the colour of position p; L.lim[c] = #positions with colour >= c.
template <int W>
__device__ KC_COLD int colour_and_order(const Lay &L, int s, int lane) {  // -1: internal error
    for (int i = lane; i < 32 * W + 2; i += 32) L.lim[i] = 0;
    // degrees in g_e
    for (int i = lane; i < s; i += 32) {
        int d = 0;
#pragma unroll
        for (int w = 0; w < W; w++) d += __popc(L.A[i * (W + KC_ROW_PAD) + w]);
        L.aux[i] = (uint16_t)d;
    }
    __syncwarp();
    // order by (degree desc, position asc)
    for (int i = lane; i < s; i += 32) {
        int di = L.aux[i], r = 0;
        for (int j = 0; j < s; j++) {
            int dj = L.aux[j];
            r += (dj > di) || (dj == di && j < i);
        }
        if (KC_OK(r, s)) L.aux2[r] = (uint16_t)i;
    }
    __syncwarp();
    if (!permute<W>(L, s, lane, nullptr)) return -1;
    // first-fit colouring in position order, one colour class at a time: class c is
    // the greedy independent set of the still uncoloured positions (identical to
    // giving each vertex, in order, the least colour unused by earlier neighbours)
    u32 R = 0;
    if (lane < W) R = lt_mask(s, lane);
    int c = 0;
    while (__any_sync(0xffffffffu, R != 0)) {
        c++;
        u32 S = R;
        int k = 0;
        while (true) {
            unsigned bal = __ballot_sync(0xffffffffu, S != 0);
            if (!bal) break;
            int fl = __ffs(bal) - 1;
            u32 wv = __shfl_sync(0xffffffffu, S, fl);
            int x = fl * 32 + __ffs(wv) - 1;
            if (lane == 0 && KC_OK(x, s)) { L.col[x] = (uint16_t)c; L.aux[x] = (uint16_t)k; }
            k++;
            if (lane == fl) { R &= ~(1u << (x & 31)); S &= ~(1u << (x & 31)); }
            if (lane < W) S &= ~L.A[x * (W + KC_ROW_PAD) + lane];
        }
        if (lane == 0 && KC_OK(c, 32 * W + 2)) L.lim[c] = (uint16_t)k;  // class size for now
    }
    const int ncol = c;
    __syncwarp();
    // class sizes -> lim[c] = #positions with colour >= c (suffix sums)
    if (lane == 0) {
        int acc = 0;
        for (int cc = ncol; cc >= 1; cc--) { acc += L.lim[cc]; L.lim[cc] = (uint16_t)acc; }
        L.lim[ncol + 1] = 0;
        L.lim[0] = (uint16_t)s;
    }
    __syncwarp();
    // final position of x: positions of colours > col(x), then index within its class
    for (int x = lane; x < s; x += 32) {
        int cx = L.col[x];
        int np = L.lim[cx + 1] + L.aux[x];
        if (KC_OK(np, s)) L.aux2[np] = (uint16_t)x;
    }
    __syncwarp();
    if (!permute<W>(L, s, lane, L.col)) return -1;
    // segment masks for Rule (2): E = last position of each colour class
    if (lane < W) { L.E[lane] = 0; L.J[lane] = lt_mask(s, lane); }
    __syncwarp();
    if (lane == 0) {
        for (int cc = 1; cc <= ncol; cc++) {
            int last = L.lim[cc] - 1;  // classes of colour >= cc end here
            L.E[last >> 5] |= 1u << (last & 31);
        }
        for (int w = 0; w < W; w++) L.J[w] &= ~L.E[w];
    }
    __syncwarp();
    return ncol;
}

// number of distinct colours in X (Rule 2), one carry-propagating add per word
template <int W>
__device__ __forceinline__ int distinct_colours(const u32 (&X)[W], const u32 *J, const u32 *E) {
    int d = 0;
    u32 carry = 0;
#pragma unroll
    for (int w = 0; w < W; w++) {
        u32 j = J[w];
        u64 t = (u64)(X[w] & j) + (u64)j + carry;
        carry = (u32)(t >> 32);
        d += __popc(((u32)t | X[w]) & E[w]);
    }
    return d;
}

// ---------------------------------------------------------------- listing
__device__ void write_clique(u32 *out, u64 slot, u32 k, const u32 *ids, int nids) {
    u32 q[KC_MAX_K];
    for (int i = 0; i < nids; i++) q[i] = ids[i];
    for (int i = 1; i < nids; i++) {
        u32 x = q[i];
        int j = i - 1;
        while (j >= 0 && q[j] > x) { q[j + 1] = q[j]; j--; }
        q[j + 1] = x;
    }
    u32 *dst = out + slot * k;
    if (!KC_OK(nids, (int)k + 1)) return;
    for (int i = 0; i < nids; i++) dst[i] = q[i];
}


// ---------------------------------------------------------------- A9 early termination
// kCtPlex for t = 3 (Sec. 5.2, Alg. 7) in closed form.  In a 3-plex every vertex of C
// misses at most two others, so the inverse graph H (the missing pairs) has maximum
// degree 2: a disjoint union of isolated vertices (the universal ones), paths and
// cycles.  The l-cliques of g[C] are the independent l-sets of H, so their number is
// the x^l coefficient of H's independence polynomial, the product over its components;
// with a weight z_v per vertex the same coefficient is the checksum sum over those
// cliques of prod z_v.  Alg. 7 reaches the same sets by branching on the inverse graph
// (the I-set combinations times the branches on the non-universal vertices); the
// product form counts them without enumerating.
//
// The warp evaluates the polynomial lane per coefficient (lane j holds x^j; l <= 30)
// with one dynamic-programming step per vertex, walking H component by component:
// a = sets of the vertices seen so far whose last vertex is not taken, b = last taken;
// a vertex v of weight z: a' = a + b, b' = z * x * (a, or a + b when v starts a new
// component).  A cycle v1..vm runs two tracks (v1 out / v1 in) and drops the sets
// that take both v1 and vm.  Counts use z = 1 in saturating 128-bit arithmetic,
// the checksum uses the keys mod 2^64.
struct Poly2 {
    u128 ca, cb;  // counts
    u64 sa, sb;   // key-weighted sums
};

__device__ __forceinline__ u128 shfl_up_u128(u128 v, int lane) {
    const u64 lo = __shfl_up_sync(0xffffffffu, (u64)v, 1);
    const u64 hi = __shfl_up_sync(0xffffffffu, (u64)(v >> 64), 1);
    return lane == 0 ? (u128)0 : (((u128)hi << 64) | (u128)lo);
}

// one vertex of weight z; fresh: v starts a new component (no edge to the previous vertex)
template <bool SUM>
__device__ __forceinline__ void poly_step(Poly2 &p, u64 z, bool fresh, int lane) {
    const u128 tot = add_sat(p.ca, p.cb);
    const u128 sh = shfl_up_u128(fresh ? tot : p.ca, lane);
    p.ca = tot;
    p.cb = sh;
    if (SUM) {
        const u64 st = p.sa + p.sb;
        const u64 ss = __shfl_up_sync(0xffffffffu, fresh ? st : p.sa, 1);
        p.sa = st;
        p.sb = lane == 0 ? 0ull : ss * z;
    }
}

// returns false if the walk met an inconsistent partner table (bounded; reported)
template <int W, bool SUM>
__device__ KC_COLD bool plex3_poly(const Lay &L, const u32 (&cw)[W], int cnt, int l, int lane, uint16_t *pr, u128 *cnt_l,
                           u64 *sum_l) {
    constexpr int RS = W + KC_ROW_PAD;
    u32 *D1 = L.tmpW, *NU = L.tmpW2;  // D1: one missing partner; NU: at least one
    if (lane < W) { D1[lane] = 0; NU[lane] = 0; }
    __syncwarp();
    // partners of every vertex of C (at most two), by position
    for (int base = 0; base < cnt; base += 32) {
        const int i = base + lane;
        if (i < cnt) {
            const int x = L.aux2[i];
            int p1 = 0xFFFF, p2 = 0xFFFF;
            if (L.aux[i] < cnt - 1) {
#pragma unroll
                for (int w = 0; w < W; w++) {
                    u32 nb = cw[w] & ~L.A[x * RS + w] & ~((w == (x >> 5)) ? (1u << (x & 31)) : 0u);
                    while (nb) {
                        const int y = w * 32 + __ffs(nb) - 1;
                        nb &= nb - 1;
                        if (p1 == 0xFFFF) p1 = y; else if (p2 == 0xFFFF) p2 = y;
                    }
                }
                if (KC_OK(x >> 5, W)) {
                    atomicOr(&NU[x >> 5], 1u << (x & 31));
                    if (p2 == 0xFFFF) atomicOr(&D1[x >> 5], 1u << (x & 31));
                }
            }
            if (KC_OK(x, 32 * W)) { pr[2 * x] = (uint16_t)p1; pr[2 * x + 1] = (uint16_t)p2; }
        }
    }
    __syncwarp();
    u32 uni = 0, d1 = 0;  // this lane's word of the universal and the path-end vertices
    if (lane < W) { uni = cw[lane] & ~NU[lane]; d1 = D1[lane]; }
    __syncwarp();
    u32 *Vis = L.tmpW2;  // visited non-universal vertices
    if (lane < W) Vis[lane] = uni;
    __syncwarp();
    Poly2 p;
    p.ca = lane == 0 ? (u128)1 : (u128)0;
    p.cb = 0;
    p.sa = lane == 0 ? 1ull : 0ull;
    p.sb = 0;
    int steps = 0;
    // isolated vertices of H (universal in g[C]), one component each
    while (true) {
        const unsigned bal = __ballot_sync(0xffffffffu, uni != 0);
        if (!bal) break;
        const int fl = __ffs(bal) - 1;
        const u32 wv = __shfl_sync(0xffffffffu, uni, fl);
        const int v = fl * 32 + __ffs(wv) - 1;
        if (lane == fl) uni &= uni - 1;
        poly_step<SUM>(p, SUM ? L.z[v] : 0ull, true, lane);
        if (++steps > cnt) return false;
    }
    // paths, each walked from an end vertex; then the cycles (what is left)
    for (int pass = 0; pass < 2; pass++) {
        while (true) {
            u32 cand = 0;
            if (lane < W) cand = cw[lane] & ~Vis[lane] & (pass == 0 ? d1 : 0xFFFFFFFFu);
            const unsigned bal = __ballot_sync(0xffffffffu, cand != 0);
            if (!bal) break;
            const int fl = __ffs(bal) - 1;
            const u32 wv = __shfl_sync(0xffffffffu, cand, fl);
            int v = fl * 32 + __ffs(wv) - 1;
            if (pass == 0) {  // a path from its end v
                int prev = -1;
                bool fresh = true;
                while (v >= 0) {
                    if (!KC_OK(v, 32 * W)) return false;
                    __syncwarp();
                    if (lane == 0) Vis[v >> 5] |= 1u << (v & 31);
                    poly_step<SUM>(p, SUM ? L.z[v] : 0ull, fresh, lane);
                    fresh = false;
                    if (++steps > cnt) return false;
                    const int q1 = pr[2 * v], q2 = pr[2 * v + 1];
                    int nx = (q1 != prev) ? q1 : q2;
                    if (nx == 0xFFFF) nx = -1;
                    prev = v;
                    v = nx;
                }
                __syncwarp();
                continue;
            }
            // a cycle v1 = v, v2, ..., vm (every vertex has two partners)
            const u64 z1 = SUM ? L.z[v] : 0ull;
            Poly2 t1;  // the track with v1 taken
            {
                const u128 tot = add_sat(p.ca, p.cb);
                t1.ca = 0;
                t1.cb = shfl_up_u128(tot, lane);
                p.ca = tot;
                p.cb = 0;
                t1.sa = 0;
                t1.sb = 0;
                if (SUM) {
                    const u64 st = p.sa + p.sb;
                    const u64 ss = __shfl_up_sync(0xffffffffu, st, 1);
                    t1.sb = lane == 0 ? 0ull : ss * z1;
                    p.sa = st;
                    p.sb = 0;
                }
            }
            __syncwarp();
            if (lane == 0) Vis[v >> 5] |= 1u << (v & 31);
            if (++steps > cnt) return false;
            const int v1 = v;
            int prev = v1, cur = pr[2 * v1];
            while (cur != v1) {
                if (cur == 0xFFFF || !KC_OK(cur, 32 * W)) return false;
                __syncwarp();
                if (lane == 0) Vis[cur >> 5] |= 1u << (cur & 31);
                const u64 zc = SUM ? L.z[cur] : 0ull;
                poly_step<SUM>(p, zc, false, lane);
                poly_step<SUM>(t1, zc, false, lane);
                if (++steps > cnt) return false;
                const int q1 = pr[2 * cur], q2 = pr[2 * cur + 1];
                const int nx = (q1 != prev) ? q1 : q2;
                prev = cur;
                cur = nx;
            }
            __syncwarp();
            // drop the sets holding both v1 and vm (t1.cb); fold into a fresh state
            p.ca = add_sat(add_sat(p.ca, p.cb), t1.ca);
            p.cb = 0;
            if (SUM) {
                p.sa = p.sa + p.sb + t1.sa;
                p.sb = 0;
            }
        }
    }
    const u128 c = add_sat(p.ca, p.cb);
    const u64 lo = __shfl_sync(0xffffffffu, (u64)c, l), hi = __shfl_sync(0xffffffffu, (u64)(c >> 64), l);
    *cnt_l = ((u128)hi << 64) | (u128)lo;
    *sum_l = SUM ? __shfl_sync(0xffffffffu, p.sa + p.sb, l) : 0ull;
    return steps == cnt;
}

// the largest x in [m-1, xm) with C(x, m) <= r (C(x, m) grows with x): binary search
__device__ __forceinline__ int colex_largest(const u128 *T, int m, int xm, u128 r) {
    int lo = m - 1, hi = xm - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (binom(T, mid, m) <= r) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Listing with early termination (Sec. 5.1, Alg. 6 in listing form): the l-cliques of a
// clique or 2-plex frame are written without branching.  F = the universal vertices, P =
// the missing pairs (a, b); a clique takes j pairs (one end of each) and l - j vertices
// of F, so the rows number sum_j C(|F|, l-j) C(|P|, j) 2^j.  The warp reserves them in
// one step and each lane writes the rows of its ranks: rank -> (j; an (l-j)-subset of F;
// a j-subset of P; the ends, one bit per pair), each subset by the combinatorial number
// system (the largest x with C(x, m) <= rank picks the m-th element).  aux2 / aux hold the
// frame's positions and degrees; sc is scratch for the F and P lists (2 x 32W u16).
template <int W>
__device__ void list_plex(const Lay &L, const Args &a, const QDesc &q, const u32 *C, int cnt, int l, int d,
                          int lane, uint16_t *sc, u128 rows) {
    uint16_t *Fl = sc, *Pl = sc + 32 * W;  // F positions; pairs as (a, b) in Pl[2i], Pl[2i+1]
    int nf = 0, np = 0;
    for (int base = 0; base < cnt; base += 32) {
        const int i = base + lane;
        int x = -1, y = -1;
        bool isf = false, isp = false;
        if (i < cnt) {
            x = L.aux2[i];
            isf = L.aux[i] == cnt - 1;
            if (!isf) {
#pragma unroll
                for (int w = 0; w < W; w++) {
                    const u32 nb = C[w] & ~L.A[x * (W + KC_ROW_PAD) + w] & ~((w == (x >> 5)) ? (1u << (x & 31)) : 0u);
                    if (y < 0 && nb) y = w * 32 + __ffs(nb) - 1;
                }
                isp = y > x;
            }
        }
        const unsigned bf = __ballot_sync(0xffffffffu, isf), bp = __ballot_sync(0xffffffffu, isp);
        const unsigned below = (1u << lane) - 1u;
        if (isf && KC_OK(nf + __popc(bf & below), 32 * W)) Fl[nf + __popc(bf & below)] = (uint16_t)x;
        if (isp && KC_OK(np + __popc(bp & below), 16 * W)) {
            Pl[2 * (np + __popc(bp & below))] = (uint16_t)x;
            Pl[2 * (np + __popc(bp & below)) + 1] = (uint16_t)y;
        }
        nf += __popc(bf);
        np += __popc(bp);
    }
    __syncwarp();
    // reserve the rows (rows past the buffer are counted, not written)
    const u64 want = rows > (u128)(1ull << 62) ? (1ull << 62) : (u64)rows;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&q.acc->written, (unsigned long long)want);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= a.cap) return;
    const u64 nrow = min((u64)want, (u64)(a.cap - base));
    const int npath = 2 * (d + 1);
    for (u64 r0 = 0; r0 < nrow; r0 += 32) {
        const u64 r = r0 + (u64)lane;
        if (r >= nrow) continue;
        u32 ids[KC_MAX_K];
        for (int i = 0; i < npath; i++) ids[i] = L.path[i];
        // j: the number of pairs the clique takes
        u128 rem = r;
        int j = 0;
        u128 cj = 0;
        for (; j <= l && j <= np; j++) {
            cj = mul_sat(mul_sat(binom(a.binom, nf, l - j), binom(a.binom, np, j)), (u128)1 << j);
            if (rem < cj) break;
            rem -= cj;
        }
        if (j > l || j > np) continue;  // not reached: r < rows
        const u64 ends = (u64)(rem & (((u128)1 << j) - 1));
        rem >>= j;
        const u128 cp = binom(a.binom, np, j);
        u128 iB = rem % cp, iA = rem / cp;
        int o = npath;
        // (l - j)-subset of F: colex unranking, largest element first
        int xm = nf;
        for (int m = l - j; m >= 1; m--) {
            const int x = colex_largest(a.binom, m, xm, iA);
            iA -= binom(a.binom, x, m);
            ids[o++] = L.vid[Fl[x]];
            xm = x;
        }
        int pm = np, bit = 0;
        for (int m = j; m >= 1; m--) {
            const int x = colex_largest(a.binom, m, pm, iB);
            iB -= binom(a.binom, x, m);
            ids[o++] = L.vid[Pl[2 * x + (int)((ends >> bit) & 1ull)]];
            bit++;
            pm = x;
        }
        write_clique(a.d_out, base + r, q.k, ids, o);
    }
}

// Returns true if the frame is closed (pruned by size or counted in closed form).
// pr: scratch of 2 x 32W u16 (a free child slot of the next depth) for the t = 3 form
template <int W, int MODE>
__device__ KC_COLD bool early_terminate(const Lay &L, const Args &a, const u32 *C, int l, u64 P, int lane, Acc &acc,
                                bool et_allowed, int ws, uint16_t *pr, int tmax, const QDesc &q, int d,
                                bool list_rows) {
    u32 cw[W];
    int cnt = 0;
#pragma unroll
    for (int w = 0; w < W; w++) {
        cw[w] = C[w];
        cnt += __popc(cw[w]);
    }
    if (cnt < l) return true;
    if (!et_allowed) return false;
    // degrees inside C, lane per vertex (early exit as soon as some vertex is too sparse)
    int mind = cnt;
    compact_positions<W>(cw, L.aux2, lane);
    for (int base = 0; base < cnt; base += 32) {
        int i = base + lane;
        int d = cnt;
        if (i < cnt) {
            int x = L.aux2[i];
            d = 0;
#pragma unroll
            for (int w = 0; w < W; w++) d += __popc(L.A[x * (W + KC_ROW_PAD) + w] & cw[w]);
            L.aux[i] = (uint16_t)d;
            acc.ops += 2u * (u32)ws;
        }
        d = __reduce_min_sync(0xffffffffu, (unsigned)d);
        mind = min(mind, d);
        if (mind < cnt - tmax) return false;
    }
    __syncwarp();
    const int t = cnt - mind;  // 1: clique, 2: 2-plex, 3: 3-plex
    u128 add = 0;
    u64 csum = 0;
    const bool want_sum = (MODE & (MODE_CHECKSUM | MODE_LIST)) != 0;
    if ((MODE & MODE_LIST) && list_rows && t >= 3) return false;  // listed by branching
    if (t >= 3) {
        u64 s3 = 0;
        if (!plex3_poly<W, (MODE & (MODE_CHECKSUM | MODE_LIST)) != 0>(L, cw, cnt, l, lane, pr, &add, &s3)) {
            acc.status |= KC_DEV_ERR_BOUNDS;
            return true;
        }
        if (add == SAT128) acc.status |= KC_DEV_ERR_OVERFLOW;
        acc.cf = add_sat(acc.cf, add);
        acc.cf_csum += want_sum ? s3 * P : 0ull;
        if (lane == 0) acc.et++;
        return true;
    }
    if (t <= 1) {
        add = binom(a.binom, cnt, l);
    } else {
        // F = universal vertices, p = missing pairs (Sec. 5.1, Alg. 6)
        int nf = 0;
        for (int base = 0; base < cnt; base += 32) {
            int i = base + lane;
            bool f = i < cnt && L.aux[i] == cnt - 1;
            nf += __popc(__ballot_sync(0xffffffffu, f));
        }
        int p = (cnt - nf) / 2;
        for (int j = 0; j <= p && j <= l; j++) {
            u128 term = mul_sat(mul_sat(binom(a.binom, nf, l - j), binom(a.binom, p, j)), (u128)1 << j);
            add = add_sat(add, term);
        }
    }
    if (want_sum) {
        // coefficient of x^l in prod (1 + c_i x): c = z_f for universal f, z_a + z_b per missing pair
        u64 e = lane == 0 ? 1ull : 0ull;
        for (int i = 0; i < cnt; i++) {
            int x = L.aux2[i];
            u64 c;
            if (t <= 1 || L.aux[i] == cnt - 1) {
                c = L.z[x];
            } else {
                // partner: the one non-neighbour of x inside C
                u32 nb = 0;
                if (lane < W) nb = C[lane] & ~L.A[x * (W + KC_ROW_PAD) + lane] & ~((lane == (x >> 5)) ? (1u << (x & 31)) : 0u);
                unsigned bal = __ballot_sync(0xffffffffu, nb != 0);
                int fl = __ffs(bal) - 1;
                u32 wv = __shfl_sync(0xffffffffu, nb, fl);
                int y = fl * 32 + __ffs(wv) - 1;
                if (y < x) continue;
                c = L.z[x] + L.z[y];
            }
            u64 prev = __shfl_up_sync(0xffffffffu, e, 1);
            if (lane >= 1 && lane <= l) e += c * prev;
        }
        csum = __shfl_sync(0xffffffffu, e, l) * P;
    }
    if (add == SAT128) acc.status |= KC_DEV_ERR_OVERFLOW;
    if ((MODE & MODE_LIST) && list_rows) list_plex<W>(L, a, q, C, cnt, l, d, lane, pr, add);
    acc.cf = add_sat(acc.cf, add);
    acc.cf_csum += csum;
    if (lane == 0) acc.et++;
    return true;
}

// ---------------------------------------------------------------- l = 3 frames
// The 3-cliques of g[C]: a lane per vertex x of C computes deg(x) in C; then, whichever
// side is sparser, either the triangles directly,
//     sum_x sum_{y in N(x) & C, y > x} |N(x) & N(y) & C & {> y}|,
// or by inclusion-exclusion over the missing pairs M of C (an exact identity),
//     C(c,3) - |M| (c-2) + sum_x C(dbar(x), 2) - T(complement),
// with dbar the missing degree and T(complement) the triples with no edge.  A
// clique or 2-plex (Sec. 5 test, t <= t_max) is closed by the Alg. 6 count instead.
// SUM: also the checksum P * sum over triangles of z_a z_b z_c -- for plexes the x^3
// coefficient of prod (1 + c x) (c = z_f for a universal vertex, z_a + z_b per missing
// pair), for the complement side the same identity with weights:
//     e3(z_C) - sum_{ab in M} z_a z_b (Z - z_a - z_b) + sum_x z_x e2(z of non-nbrs of x) - T_z.

// product of two truncated polynomials (1 + a1 x + a2 x^2 + a3 x^3)(1 + b1 x + ...)
__device__ __forceinline__ void poly3_mul(u64 &a1, u64 &a2, u64 &a3, u64 b1, u64 b2, u64 b3) {
    const u64 c3 = a3 + b3 + a1 * b2 + a2 * b1;
    const u64 c2 = a2 + b2 + a1 * b1;
    a1 += b1;
    a2 = c2;
    a3 = c3;
}

__device__ __forceinline__ void poly3_warp_product(u64 &p1, u64 &p2, u64 &p3) {
    for (int o = 16; o > 0; o >>= 1) {
        const u64 b1 = __shfl_xor_sync(0xffffffffu, p1, o);
        const u64 b2 = __shfl_xor_sync(0xffffffffu, p2, o);
        const u64 b3 = __shfl_xor_sync(0xffffffffu, p3, o);
        poly3_mul(p1, p2, p3, b1, b2, b3);
    }
}

template <int W, bool SUM>
// prof_bin (profiling builds): the density decile of the frame (10 = closed as a plex)
__device__ void frame_l3_count(const Lay &L, const u32 *C, int lane, Acc &acc, int tmax, bool use_et, int ws, u64 P,
                               int *prof_bin = nullptr) {
    u32 cw[W];
    int cnt = 0;
#pragma unroll
    for (int w = 0; w < W; w++) {
        cw[w] = C[w];
        cnt += __popc(cw[w]);
    }
    if (cnt < 3) return;
    u64 sumdeg = 0, sc2 = 0;
    int mind = cnt, nuni = 0;
    u64 Z = 0, q1 = 0, q2 = 0, q3 = 0;  // SUM: sum of keys, lane's part of prod (1 + z x)
    compact_positions<W>(cw, L.aux2, lane);
    for (int base = 0; base < cnt; base += 32) {
        const int i = base + lane;
        if (i < cnt) {
            const int x = L.aux2[i];
            int d = 0;
#pragma unroll
            for (int w = 0; w < W; w++) d += __popc(L.A[x * (W + KC_ROW_PAD) + w] & cw[w]);
            L.aux[i] = (uint16_t)d;
            const int db = cnt - 1 - d;
            sumdeg += (u64)d;
            sc2 += (u64)db * (u64)(db - 1) / 2;
            mind = min(mind, d);
            nuni += (db == 0);
            acc.ops += 2u * (u32)ws;
            if (SUM) {
                const u64 z = L.z[x];
                Z += z;
                poly3_mul(q1, q2, q3, z, 0ull, 0ull);
            }
        }
    }
    __syncwarp();
    sumdeg = warp_sum_u64(sumdeg);
    sc2 = warp_sum_u64(sc2);
    if (SUM) Z = warp_sum_u64(Z);  // the key sum over all of C
    mind = (int)__reduce_min_sync(0xffffffffu, (unsigned)mind);
    nuni = (int)__reduce_add_sync(0xffffffffu, (unsigned)nuni);
    const u64 c = (u64)cnt;
    const u64 tri_all = c * (c - 1) * (c - 2) / 6;
    const u64 E = sumdeg / 2, M = c * (c - 1) / 2 - E;
    if (use_et && mind >= cnt - tmax) {
        // clique: C(c,3); 2-plex: sum_j C(|F|, 3-j) C(p, j) 2^j (Alg. 6 count)
        u64 add;
        if (mind == cnt - 1) {
            add = tri_all;
        } else {
            const u64 f = (u64)nuni, pp = (c - f) / 2;
            add = f * (f - 1) * (f - 2) / 6 + (f * (f - 1) / 2) * pp * 2 + f * (pp * (pp - 1) / 2) * 4 +
                  (pp * (pp - 1) * (pp - 2) / 6) * 8;
        }
        if (SUM) {
            u64 p1 = 0, p2 = 0, p3 = 0;
            for (int base = 0; base < cnt; base += 32) {
                const int i = base + lane;
                if (i < cnt) {
                    const int x = L.aux2[i];
                    if (L.aux[i] == cnt - 1) {
                        poly3_mul(p1, p2, p3, L.z[x], 0ull, 0ull);
                    } else {  // its one missing partner y; the pair's factor once, from min(x, y)
                        int y = -1;
#pragma unroll
                        for (int w = 0; w < W; w++) {
                            const u32 nb = cw[w] & ~L.A[x * (W + KC_ROW_PAD) + w] & ~((w == (x >> 5)) ? (1u << (x & 31)) : 0u);
                            if (y < 0 && nb) y = w * 32 + __ffs(nb) - 1;
                        }
                        if (y > x) poly3_mul(p1, p2, p3, L.z[x] + L.z[y], 0ull, 0ull);
                    }
                }
            }
            poly3_warp_product(p1, p2, p3);
            if (lane == 0) acc.csum += P * p3;
        }
        if (lane == 0) { acc.leaf += add; acc.et++; }
        return;
    }
    if (KC_SECTION_PROFILE && prof_bin) *prof_bin = (int)((10 * E) / (c * (c - 1) / 2 + 1));
    const bool comp = M < E;
    const u32 cm = comp ? 0xFFFFFFFFu : 0u;  // rows are read as A ^ cm: the complement side flips them
    u64 t = 0, zsum = 0;
    for (int base = 0; base < cnt; base += 32) {
        const int i = base + lane;
        if (i < cnt) {
            const int x = L.aux2[i];
            u32 row[W];
            u32 words = 0;  // words of this row's intersections (from y's word on)
#pragma unroll
            for (int w = 0; w < W; w++) row[w] = (L.A[x * (W + KC_ROW_PAD) + w] ^ cm) & cw[w] & gt_mask(x, w);
            const u64 zx = SUM ? L.z[x] : 0ull;
            if (SUM && comp) {
                // z_x e2(keys of all non-neighbours of x in C)
                u64 f1 = 0, f2 = 0;
#pragma unroll (W <= 8 ? W : 1)
                for (int w = 0; w < W; w++) {
                    u32 nb = cw[w] & ~L.A[x * (W + KC_ROW_PAD) + w] & ~((w == (x >> 5)) ? (1u << (x & 31)) : 0u);
                    while (nb) {
                        const u64 z = L.z[w * 32 + __ffs(nb) - 1];
                        nb &= nb - 1;
                        f2 += f1 * z;
                        f1 += z;
                    }
                }
                zsum += zx * f2;
            }
            // y runs over row in increasing order and leaves it as it goes, so row holds
            // exactly the candidates z > y and no word below y's has any left
#pragma unroll (W <= 8 ? W : 1)
            for (int w = 0; w < W; w++) {
                while (row[w]) {
                    const int y = w * 32 + __ffs(row[w]) - 1;
                    row[w] &= row[w] - 1;
                    int tc = 0;
                    u64 zw = 0;
#pragma unroll
                    for (int w2 = 0; w2 < W; w2++) {
                        if (w2 < w) continue;
                        u32 tb = row[w2] & (L.A[y * (W + KC_ROW_PAD) + w2] ^ cm);
                        tc += __popc(tb);
                        if (SUM) {
                            while (tb) { zw += L.z[w2 * 32 + __ffs(tb) - 1]; tb &= tb - 1; }
                        }
                    }
                    t += (u64)tc;
                    if (SUM) {
                        const u64 zy = L.z[y];
                        if (comp) zsum -= zx * zy * (Z - zx - zy) + zx * zy * zw;  // missing pair, complement triangles
                        else zsum += zx * zy * zw;
                    }
                    words += (u32)(ws - (y >> 5));
                }
            }
            acc.ops += 3u * words;
        }
    }
    if (SUM) {
        // warp-wide: e3 of all keys (complement side), the lanes' weighted terms
        if (comp) {
            u64 p1 = q1, p2 = q2, p3 = q3;
            poly3_warp_product(p1, p2, p3);
            zsum = warp_sum_u64(zsum);
            if (lane == 0) acc.csum += P * (p3 + zsum);
        } else {
            acc.csum += P * zsum;
        }
    }
    if (!comp) {
        acc.leaf += t;
    } else {
        t = warp_sum_u64(t);
        if (lane == 0) acc.leaf += tri_all - M * (c - 2) + sc2 - t;
    }
}

// ---------------------------------------------------------------- l = 4 frames
// The 4-cliques of g[C] through its complement H (the missing pairs of C).  A 4-set of C
// is a clique iff it spans no edge of H, so by inclusion-exclusion over the edge sets F
// of H that span at most 4 vertices (sign (-1)^|F|, times the C(c-|V(F)|, 4-|V(F)|) ways
// to complete V(F) to a 4-set):
//   K4 = C(c,4) - M C(c-2,2) + (P3 - T)(c-3) + 2K2 - P4 - S3 + C4 + paw - diamond + K4(H)
// over the subgraph types of H: M edges, P3 = sum_x C(dbar_x, 2) paths of two edges,
// T triangles, 2K2 = C(M,2) - P3 pairs of disjoint edges, P4 = sum_{xa in H}
// (dbar_x - 1)(dbar_a - 1) - 3T paths of three edges, S3 = sum_x C(dbar_x, 3) stars,
// C4 = (1/2) sum_{x<y} C(codeg(x,y), 2) 4-cycles, paw = sum_x (dbar_x - 2) T_x (T_x
// the triangles at x), diamond = sum_{xa in H} C(t_xa, 2) (t_xa the triangles on xa),
// and the 4-cliques of H.
// SUM: the checksum P * sum over 4-cliques of z_a z_b z_c z_d, by the same expansion
// with every F weighted by the keys of V(F) times e_{4-|V(F)|} of the keys of C - V(F),
// written without division (mod 2^64): with Z, e2, e4 the elementary symmetric sums of
// C's keys, S1(x) and e_j(N(x)) those of x's H-neighbours, p_j their power sums, and
// Q(x) = sum over H-edges ab inside N(x) of z_a z_b,
//   e4 - sum_{xa in H} z_x z_a e2(C - {x, a}) + sum_x z_x ((Z - z_x) e2(N(x)) - (p1 p2 - p3))
//   - Z T_z + sum_x z_x^2 Q(x) + [e2 over H-edges of z_x z_a - sum_x z_x^2 e2(N(x))]
//   - P4_z - sum_x z_x e3(N(x)) + C4_z + sum_x (z_x S1(x) - 2 z_x^2) Q(x) - diamond_z + K4(H)_z
// with T_z = sum over triangles of H of their key products, P4_z = sum_{xa in H} z_x z_a
// ((S1(x) - z_a)(S1(a) - z_x) - sum_{b in N(x) & N(a)} z_b^2), C4_z = sum_{x<y} z_x z_y
// e2(keys of N(x) & N(y) & {> x}) (each 4-cycle once, through its least vertex and the
// one opposite), diamond_z = sum_{xa in H} z_x z_a e2(keys of N(x) & N(a)).
// Lane per vertex x; its row of H is C & ~N(x) without x.  The cost is O(c^2 W) word
// operations (the pairs of C4) plus work on the edges of H, against O(|E| c W) for
// branching on the frame's edges, so it is taken only when H is sparse
// (M <= E / KC_L4_DENSE); it returns false, and the frame branches, otherwise.
#ifndef KC_L4  // count dense l = 4 frames whole (even k)
#define KC_L4 1
#endif
#ifndef KC_L4_DENSE
#define KC_L4_DENSE 3
#endif

__device__ __forceinline__ void poly4_mul(u64 &a1, u64 &a2, u64 &a3, u64 &a4, u64 b1, u64 b2, u64 b3, u64 b4) {
    const u64 c4 = a4 + b4 + a1 * b3 + a2 * b2 + a3 * b1;
    const u64 c3 = a3 + b3 + a1 * b2 + a2 * b1;
    const u64 c2 = a2 + b2 + a1 * b1;
    a1 += b1;
    a2 = c2;
    a3 = c3;
    a4 = c4;
}

__device__ __forceinline__ void poly4_warp_product(u64 &p1, u64 &p2, u64 &p3, u64 &p4) {
    for (int o = 16; o > 0; o >>= 1) {
        const u64 b1 = __shfl_xor_sync(0xffffffffu, p1, o);
        const u64 b2 = __shfl_xor_sync(0xffffffffu, p2, o);
        const u64 b3 = __shfl_xor_sync(0xffffffffu, p3, o);
        const u64 b4 = __shfl_xor_sync(0xffffffffu, p4, o);
        poly4_mul(p1, p2, p3, p4, b1, b2, b3, b4);
    }
}

// the H-row of vertex y in C: C & ~N(y) without y
template <int W>
__device__ __forceinline__ u32 hrow_word(const Lay &L, const u32 *cw, int y, int w) {
    return cw[w] & ~L.A[y * (W + KC_ROW_PAD) + w] & ~((w == (y >> 5)) ? (1u << (y & 31)) : 0u);
}

template <int W, bool SUM>
__device__ __noinline__ bool frame_l4_count(const Lay &L, const u32 *C, int lane, Acc &acc, int ws, u64 P) {
    u32 cw[W];
    int cnt = 0;
#pragma unroll
    for (int w = 0; w < W; w++) {
        cw[w] = C[w];
        cnt += __popc(cw[w]);
    }
    if (cnt < 4) return true;  // no 4-set
    compact_positions<W>(cw, L.aux2, lane);
    u64 sdb = 0;
    u64 e1 = 0, e2 = 0, e3 = 0, e4 = 0;  // SUM: the lane's part of prod (1 + z x) over C
    for (int base = 0; base < cnt; base += 32) {
        const int i = base + lane;
        if (i < cnt) {
            const int x = L.aux2[i];
            int db = -1;  // x itself is not in N(x)
#pragma unroll
            for (int w = 0; w < W; w++) db += __popc(cw[w] & ~L.A[x * (W + KC_ROW_PAD) + w]);
            L.aux[x] = (uint16_t)db;  // by vertex
            sdb += (u64)db;
            acc.ops += 2u * (u32)ws;
            if (SUM) poly4_mul(e1, e2, e3, e4, L.z[x], 0ull, 0ull, 0ull);
        }
    }
    sdb = warp_sum_u64(sdb);
    const u64 c = (u64)cnt, M = sdb / 2, E = c * (c - 1) / 2 - M;
    if (M * KC_L4_DENSE > E) return false;
    if (SUM) poly4_warp_product(e1, e2, e3, e4);  // e1 = Z: every lane holds the sums over C
    __syncwarp();
    // The count's terms folded per element, each element of H visited once: a vertex x
    // adds C(dbar_x, 2)(c - 4) - C(dbar_x, 3); an H-edge x < a adds -(dbar_x - 1)(dbar_a - 1)
    // - C(t_xa, 2); a triangle x < a < b of H adds dbar_x + dbar_a + dbar_b - c (its parts of
    // -T(c-3) + 3T + paw); a 4-cycle (counted at its least vertex x and the vertex y
    // opposite) and a 4-clique of H add 1.  SUM: zs collects every weighted term but the
    // e2 over H-edge weights, whose lane parts are ew1, ew2.
    u64 kc = 0, zs = 0, ew1 = 0, ew2 = 0;
    u32 words = 0;
    for (int base = 0; base < cnt; base += 32) {
        const int i = base + lane;
        if (i >= cnt) continue;
        const int x = L.aux2[i];
        const u64 dx = L.aux[x];
        kc += dx * (dx - 1) / 2 * (c - 4) - dx * (dx - 1) * (dx - 2) / 6;
        u32 hx[W];
#pragma unroll
        for (int w = 0; w < W; w++) hx[w] = hrow_word<W>(L, cw, x, w);
        const u64 zx = SUM ? L.z[x] : 0ull;
        u64 s1 = 0, qx = 0;  // SUM: S1(x), Q(x)
        if (SUM && dx) {
            u64 q2 = 0, q3 = 0, n2 = 0, n3 = 0;
#pragma unroll (W <= 8 ? W : 1)
            for (int w = 0; w < W; w++) {
                u32 nb = hx[w];
                while (nb) {
                    const u64 za = L.z[w * 32 + __ffs(nb) - 1];
                    nb &= nb - 1;
                    n3 += n2 * za;
                    n2 += s1 * za;
                    s1 += za;
                    const u64 za2 = za * za;
                    q2 += za2;
                    q3 += za2 * za;
                }
            }
            // paths of two edges, stars, pairs of H-edges that share x
            zs += zx * ((e1 - zx) * n2 - (s1 * q2 - q3)) - zx * n3 - zx * zx * n2;
        }
        if (dx) {
#pragma unroll (W <= 8 ? W : 1)
            for (int w = 0; w < W; w++) {
                u32 nb = hx[w];
                while (nb) {
                    const int a = w * 32 + __ffs(nb) - 1;
                    nb &= nb - 1;
                    if (!SUM && a < x) continue;
                    u32 cm[W];  // common H-neighbours of x and a
                    int t = 0;
#pragma unroll
                    for (int w2 = 0; w2 < W; w2++) {
                        cm[w2] = hx[w2] & hrow_word<W>(L, cw, a, w2);
                        t += __popc(cm[w2]);
                    }
                    words += (u32)W;
                    u64 za = 0, zc_gt = 0, cz2 = 0, ce2 = 0;
                    if (SUM) {
                        za = L.z[a];
                        u64 ce1 = 0;
#pragma unroll (W <= 8 ? W : 1)
                        for (int w2 = 0; w2 < W; w2++) {
                            u32 bb = cm[w2];
                            while (bb) {
                                const int b = w2 * 32 + __ffs(bb) - 1;
                                bb &= bb - 1;
                                const u64 zb = L.z[b];
                                if (b > a) zc_gt += zb;
                                cz2 += zb * zb;
                                ce2 += ce1 * zb;
                                ce1 += zb;
                            }
                        }
                        qx += za * zc_gt;
                    }
                    if (a < x) continue;
                    const u64 da = L.aux[a];
                    kc -= (dx - 1) * (da - 1) + (u64)t * (u64)(t - 1) / 2;
                    if (SUM) {
                        const u64 wt = zx * za;
                        u64 s1a = 0;
#pragma unroll (W <= 8 ? W : 1)
                        for (int w2 = 0; w2 < W; w2++) {
                            u32 bb = hrow_word<W>(L, cw, a, w2);
                            while (bb) { s1a += L.z[w2 * 32 + __ffs(bb) - 1]; bb &= bb - 1; }
                        }
                        words += (u32)W;
                        ew2 += ew1 * wt;
                        ew1 += wt;
                        // single edge (e2 of C - {x, a}), triangles on it above a, P4_z, diamond_z
                        zs -= wt * (e2 - (zx + za) * (e1 - zx - za) - wt) + e1 * wt * zc_gt +
                              wt * ((s1 - za) * (s1a - zx) - cz2) + wt * ce2;
                    }
                    // triangles x < a < b, and the 4-cliques of H whose least vertices are x < a
#pragma unroll
                    for (int w2 = 0; w2 < W; w2++) cm[w2] &= gt_mask(a, w2);
                    if (t) {
#pragma unroll (W <= 8 ? W : 1)
                        for (int w2 = 0; w2 < W; w2++) {
                            u32 bb = cm[w2];
                            while (bb) {
                                const int b = w2 * 32 + __ffs(bb) - 1;
                                bb &= bb - 1;
                                kc += dx + da + (u64)L.aux[b] - c;
                                int q = 0;
                                u64 zq = 0;
#pragma unroll
                                for (int w3 = 0; w3 < W; w3++) {
                                    u32 qq = cm[w3] & ~L.A[b * (W + KC_ROW_PAD) + w3] & gt_mask(b, w3);
                                    q += __popc(qq);
                                    if (SUM) {
                                        while (qq) { zq += L.z[w3 * 32 + __ffs(qq) - 1]; qq &= qq - 1; }
                                    }
                                }
                                kc += (u64)q;
                                if (SUM) zs += zx * za * L.z[b] * zq;
                                words += (u32)W;
                            }
                        }
                    }
                }
            }
        }
        if (SUM) zs += zx * qx * (s1 - zx);  // triangle and paw terms
        // 4-cycles with least vertex x and opposite vertex y: common H-neighbours above x
        if (dx >= 2) {
            for (int j = i + 1; j < cnt; j++) {
                const int y = L.aux2[j];
                if (L.aux[y] < 2) continue;
                // y is in hx & ~N(y) when xy is an H-edge (y is not its own neighbour): drop it
                const u32 ybit = 1u << (y & 31);
                const int yw = y >> 5;
                u32 cn[W];
                int cg = 0;
#pragma unroll
                for (int w = 0; w < W; w++) {
                    cn[w] = hx[w] & ~L.A[y * (W + KC_ROW_PAD) + w] & gt_mask(x, w) & ~(w == yw ? ybit : 0u);
                    cg += __popc(cn[w]);
                }
                kc += (u64)cg * (u64)(cg - 1) / 2;
                words += (u32)W;
                if (SUM && cg >= 2) {
                    u64 f1 = 0, f2 = 0;  // e1, e2 of their keys
#pragma unroll (W <= 8 ? W : 1)
                    for (int w = 0; w < W; w++) {
                        u32 bb = cn[w];
                        while (bb) {
                            const u64 zb = L.z[w * 32 + __ffs(bb) - 1];
                            bb &= bb - 1;
                            f2 += f1 * zb;
                            f1 += zb;
                        }
                    }
                    zs += zx * L.z[y] * f2;
                }
            }
        }
    }
    acc.ops += 2u * words;
    kc = warp_sum_u64(kc);
    if (SUM) {
        // e2 over all H-edge weights: the lanes' own e2 plus the products across lanes
        u64 pre = ew1;
        for (int o = 1; o < 32; o <<= 1) {
            const u64 y = __shfl_up_sync(0xffffffffu, pre, o);
            if (lane >= o) pre += y;
        }
        pre -= ew1;  // key-weight sum of the lanes below
        zs += ew2 + ew1 * pre;
        zs = warp_sum_u64(zs);
    }
    if (lane == 0) {
        const u64 cc4 = c * (c - 1) * (c - 2) * (c - 3) / 24;
        const u64 cc2 = (c - 2) * (c - 3) / 2;
        // unsigned arithmetic wraps consistently; the true value lies in [0, 2^64)
        acc.leaf += cc4 - M * cc2 + M * (M - 1) / 2 + kc;
        if (SUM) acc.csum += P * (e4 + zs);
    }
    return true;
}

// ---------------------------------------------------------------- kernels
// resident blocks per SM targeted by the register allocator, per bitset width
template <int W>
struct MinBlocks {
    static constexpr int value = W <= 4 ? 6 : (W <= 8 ? KC_MINB8 : (W <= 16 ? 2 : 1));
};

// A heavy sub-branch published for splitting (A12): the coloured, renumbered
// adjacency of g_e plus what a helper warp needs to rebuild its frames.
struct SlotHdr {
    u32 e, s, qi, limu;  // edge, |VSet|, query, top-frame vertices u to branch on (Rule 1)
    u64 P0, pad2;
};

template <int W>
__host__ __device__ constexpr u32 slot_bytes() {
    return 32u + 4u * (32u * W) * W + 4u * (32u * W) + 2u * (32u * W) + ((2u * (32u * W + 2) + 15u) & ~15u) +
           8u * W;
}

struct WarpTotals {
    u128 q_total;   // warp-uniform: count of the current query
    u64 q_csum;     // warp-uniform: checksum of the current query
    u64 branches;
    int cur_q;
};

template <int MODE>
__device__ void flush_query(const Args &a, Acc &acc, WarpTotals &wt, int lane, bool prof) {
    constexpr bool SUM = (MODE & (MODE_CHECKSUM | MODE_LIST)) != 0;
    if (wt.cur_q < 0) return;
    const QDesc &q = a.qs[wt.cur_q];
    const u64 ops = warp_sum_u64(acc.ops), pairs = warp_sum_u64(acc.pairs);
    const u64 nodes = warp_sum_u64(acc.nodes), ets = warp_sum_u64(acc.et);
    if (lane == 0) {
        atomicAdd(&q.acc->word_ops, (unsigned long long)ops);
        atomicAdd(&q.acc->pair_tests, (unsigned long long)pairs);
#if KC_SECTION_PROFILE
        if (prof)
            for (int i = 0; i < 6; i++) atomicAdd(&q.acc->sec[i], (unsigned long long)acc.sec[i]);
#endif
        u64 lo = (u64)wt.q_total, hi = (u64)(wt.q_total >> 64);
        if (lo | hi) {
            unsigned long long old = atomicAdd(&q.acc->count_lo, (unsigned long long)lo);
            unsigned long long carry = (old + lo < old) ? 1ull : 0ull;
            if (hi + carry) atomicAdd(&q.acc->count_hi, (unsigned long long)(hi + carry));
        }
        if (SUM) atomicAdd(&q.acc->checksum, (unsigned long long)wt.q_csum);
        atomicAdd(&q.acc->nodes, (unsigned long long)nodes);
        atomicAdd(&q.acc->et_hits, (unsigned long long)ets);
        atomicAdd(&q.acc->branches, (unsigned long long)wt.branches);
        if (acc.status) atomicOr(&q.acc->status, acc.status);
    }
    wt.q_total = 0; wt.q_csum = 0; wt.branches = 0;
    acc.nodes = 0; acc.et = 0; acc.status = 0; acc.ops = 0; acc.pairs = 0;
#if KC_SECTION_PROFILE
    for (int i = 0; i < 6; i++) acc.sec[i] = 0;
#endif
}

__device__ __forceinline__ void reset_unit(Acc &acc) {
    acc.leaf = 0; acc.csum = 0; acc.cf = 0; acc.cf_csum = 0;
}

// end of a unit of work (a whole sub-branch, or one split item) of edge e: fold the
// unit's count into the warp totals and add it to the optional per-edge outputs
template <int MODE>
__device__ void finish_unit(const QDesc &q, u32 e, Acc &acc, WarpTotals &wt, int lane, long long t_start) {
    constexpr bool SUM = (MODE & (MODE_CHECKSUM | MODE_LIST)) != 0;
    u128 leaf = warp_sum_u128(acc.leaf);
    u64 cs = SUM ? warp_sum_u64(acc.csum) + acc.cf_csum : 0ull;
    u128 tot = leaf + acc.cf;
    if (tot < leaf || acc.cf == SAT128) acc.status |= KC_DEV_ERR_OVERFLOW;
    u128 nt = wt.q_total + tot;
    if (nt < wt.q_total) acc.status |= KC_DEV_ERR_OVERFLOW;
    wt.q_total = nt;
    wt.q_csum += cs;
    if (lane == 0) {
        if (q.edge_count && tot) atomicAdd((unsigned long long *)&q.edge_count[e], (unsigned long long)(u64)tot);
        if (q.edge_checksum && cs) atomicAdd((unsigned long long *)&q.edge_checksum[e], (unsigned long long)cs);
        if (q.edge_cycles) atomicAdd((unsigned long long *)&q.edge_cycles[e], (unsigned long long)(clock64() - t_start));
    }
}

#if KC_SECTION_PROFILE
#define KC_SEC_ADD(i) \
    if (prof && lane == 0) acc.sec[i] += (u64)(clock64() - tsec)
#else
#define KC_SEC_ADD(i) (void)tsec
#endif
#define KC_SEC_BEGIN() \
    if (KC_SECTION_PROFILE && prof) tsec = clock64()
#define KC_SEC_END(i) \
    KC_SEC_ADD(i)

// A7-A9: depth-first search over the frames of one sub-branch whose coloured,
// renumbered adjacency is in L.  The top frame is C0 = {0..s-1} with l = l0; its
// child edges (u, v) are restricted to u in [u_lo, u_hi).  top_et: run the early
// termination test on the top frame (false when a split item resumes it).
template <int W, int MODE>
__device__ void run_dfs(const Lay &L, const Args &a, const QDesc &q, int s, int l0, u64 P0, int lane, Acc &acc,
                        int Ws, int u_lo, int u_hi, bool top_et, bool prof) {
    constexpr bool SUM = (MODE & (MODE_CHECKSUM | MODE_LIST)) != 0;
    constexpr bool LIST = (MODE & MODE_LIST) != 0;
    constexpr bool ODD = (MODE & MODE_ODD) != 0, EVEN = (MODE & MODE_EVEN) != 0;
    const bool use_rule1 = !(a.flags & KC_NO_RULE1);
    const bool use_rule2 = !(a.flags & KC_NO_RULE2);
    const int tq = (int)q.t_max;
    const bool use_et = !(a.flags & KC_NO_ET) && tq >= 1;
    const u32 k = q.k;
    long long tsec = 0;
    if (lane < W) L.C0[lane] = lt_mask(s, lane);
    if (lane == 0) { L.cur[0] = u_lo - 1; L.slot[0] = 0; L.rn[0] = 0; }
    if (lane < W) L.V[lane] = 0;
    __syncwarp();
    int d = 0;
    int phase = top_et ? 0 : 1;  // 0 start frame, 1 generate, 2 descend into children, 3 frame done
    bool full = LIST && (*(volatile unsigned long long *)&q.acc->written >= a.cap);
    while (true) {
        const int l = l0 - 2 * d;
        const u32 *C = d == 0 ? L.C0 : L.childC + ((size_t)(d * 32 + L.slot[d])) * W;
        const u64 P = SUM ? (d == 0 ? P0 : L.childP[d * 32 + L.slot[d]]) : 0ull;
        if (phase == 0) {
            if (lane == 0) acc.nodes++;
            if (LIST) full = *(volatile unsigned long long *)&q.acc->written >= a.cap;
            // rows only: the totals come from a separate count
            if (LIST && a.stop_full && __shfl_sync(0xffffffffu, (int)full, 0)) break;
            if (!EVEN && l == 3 && (!LIST || full)) {
                const long long tf = (KC_SECTION_PROFILE && prof) ? clock64() : 0;
                KC_SEC_BEGIN();
                int dbin = 10;
                frame_l3_count<W, SUM>(L, C, lane, acc, min(tq, 2), use_et, Ws, P, &dbin);
                KC_SEC_END(3);
                if (KC_SECTION_PROFILE && prof && a.l3hist) {
                    const int c = warp_popc<W>(C, lane);
                    if (lane == 0) {
                        const int b = c <= 8 ? 0 : c <= 16 ? 1 : c <= 32 ? 2 : c <= 64 ? 3 : c <= 128 ? 4 : c <= 256 ? 5 : 6;
                        const unsigned long long dt = (unsigned long long)(clock64() - tf);
                        atomicAdd(&a.l3hist[b], 1ull);
                        atomicAdd(&a.l3hist[8 + b], dt);
                        // by edge density decile (10: closed as a plex): frames, cycles, vertices
                        atomicAdd(&a.l3hist[16 + dbin], 1ull);
                        atomicAdd(&a.l3hist[27 + dbin], dt);
                        atomicAdd(&a.l3hist[38 + dbin], (unsigned long long)c);
                    }
                }
                phase = 3;
                continue;
            }
            KC_SEC_BEGIN();
            // listing: a clique or 2-plex frame writes its rows directly (Alg. 6 listing)
            const bool closed = early_terminate<W, MODE>(L, a, C, l, P, lane, acc, use_et, Ws,
                                                         (uint16_t *)(L.childC + (size_t)((d + 1) * 32) * W), tq, q, d,
                                                         LIST && !full);
            KC_SEC_END(2);
            if (closed) { phase = 3; continue; }
            // even k, count and checksum modes: a dense l = 4 frame is counted whole through its complement
            if (KC_L4 && EVEN && l == 4 && frame_l4_count<W, SUM>(L, C, lane, acc, Ws, P)) { phase = 3; continue; }
            if (lane == 0) { L.cur[d] = d == 0 ? u_lo - 1 : -1; L.rn[d] = 0; }
            if (lane < W) L.V[d * W + lane] = 0;
            __syncwarp();
            phase = 1;
            continue;
        }
        if (phase == 1) {
            KC_SEC_BEGIN();
            // fill a batch of up to 32 child edges (u, v); Rule (1) as colour prefixes
            int limu = use_rule1 ? (int)L.lim[min(l, 32 * W + 1)] : s;
            if (d == 0) limu = min(limu, u_hi);
            const int limv = use_rule1 ? (int)L.lim[min(l - 1, 32 * W + 1)] : s;
            int nb = 0;
            u32 *V = L.V + d * W;
            int u = L.cur[d];
            // plex pre-check for l = 3 children (count mode): masks of the current u
            const bool pre = KC_PRECHECK && !SUM && l == 5 && use_et;
            int nuniq = 0;  // distinct u's in this batch (at most 4: the ring)
            if (pre) {
                u32 vw0 = lane < W ? V[lane] : 0u;
                nuniq = __any_sync(0xffffffffu, vw0 != 0) ? 1 : 0;
            }
            while (nb < 32) {
                u32 vw = lane < W ? V[lane] : 0u;
                int c = __popc(vw);
                int tot = __reduce_add_sync(0xffffffffu, (unsigned)c);
                if (tot == 0) {
                    if (u == -2) break;  // generator exhausted
                    if (pre && nuniq == 4) break;  // ring full: evaluate this batch first
                    int nu = warp_first_from<W>(C, u + 1, lane);
                    if (nu < 0 || nu >= limu) { u = -2; break; }
                    u = nu;
                    if (!KC_OK(u, s)) { u = -2; break; }
                    u32 nv = 0;
                    if (lane < W) nv = L.A[u * (W + KC_ROW_PAD) + lane] & C[lane] & gt_mask(u, lane) & lt_mask(limv, lane);
                    if (lane < W) V[lane] = nv;
                    if (pre && __any_sync(0xffffffffu, nv != 0)) {
                        // over Cu = C & N(u) & {> u}: B = vertices with >= t_max non-neighbours
                        // in Cu, M1 = vertices with >= 1; every child set of u lies inside Cu
                        const int slot = L.rn[d] & 3;
                        u32 cu[W];
                        int ncu = 0;
#pragma unroll
                        for (int w = 0; w < W; w++) {
                            cu[w] = C[w] & L.A[u * (W + KC_ROW_PAD) + w] & gt_mask(u, w);
                            ncu += __popc(cu[w]);
                        }
                        u32 *Bm = L.Bm + slot * W, *M1 = L.M1 + slot * W;
                        if (lane < W) { Bm[lane] = 0; M1[lane] = 0; }
                        __syncwarp();
                        const int tm = min(tq, 2);
                        for (int base = 0; base < ncu; base += 32) {
                            const int i = base + lane;
                            if (i < ncu) {
                                const int x = select_bit<W>(cu, i);
                                int md = -1;  // x itself is not in N(x)
#pragma unroll
                                for (int w = 0; w < W; w++) md += __popc(cu[w] & ~L.A[x * (W + KC_ROW_PAD) + w]);
                                if (md >= tm) atomicOr(&Bm[x >> 5], 1u << (x & 31));
                                if (md >= 1) atomicOr(&M1[x >> 5], 1u << (x & 31));
                                acc.ops += 2u * (u32)Ws;
                            }
                        }
                        __syncwarp();
                        if (lane == 0) L.rn[d] = L.rn[d] + 1;
                        nuniq++;
                    }
                    __syncwarp();
                    continue;
                }
                int off = c;
                for (int o = 1; o < 32; o <<= 1) {
                    int y = __shfl_up_sync(0xffffffffu, off, o);
                    if (lane >= o) off += y;
                }
                off -= c;
                int room = 32 - nb;
                int take = max(0, min(c, room - off));
                const uint8_t rs = pre ? (uint8_t)((L.rn[d] - 1) & 3) : (uint8_t)0;
                for (int i = 0; i < take; i++) {
                    int b = __ffs(vw) - 1;
                    vw &= vw - 1;
                    if (!KC_OK(nb + off + i, 32) || !KC_OK(lane * 32 + b, s)) continue;
                    L.bu[nb + off + i] = (uint16_t)u;
                    L.bv[nb + off + i] = (uint16_t)(lane * 32 + b);
                    L.bs[nb + off + i] = rs;
                }
                if (lane < W) V[lane] = vw;
                nb += min(tot, room);
                __syncwarp();
            }
            if (lane == 0) L.cur[d] = u;
            __syncwarp();
            KC_SEC_END(4);
            if (nb == 0) { phase = 3; continue; }
            KC_SEC_BEGIN();
            // evaluate the batch, lane per child
            const int l2 = l - 2;
            const int cu0 = lane < nb ? L.bu[lane] : 0;
            const int cv0 = lane < nb ? L.bv[lane] : 0;
            const bool has = lane < nb && KC_OK(cu0, s) && KC_OK(cv0, s);
            const int cu = has ? cu0 : 0;
            const int cv = has ? cv0 : 0;
            u32 cw[W];
            int cc = 0;
#pragma unroll
            for (int w = 0; w < W; w++) {
                u32 x = (has && w >= (cv >> 5)) ? (C[w] & L.A[cu * (W + KC_ROW_PAD) + w] & L.A[cv * (W + KC_ROW_PAD) + w] & gt_mask(cv, w)) : 0u;
                cw[w] = x;
                cc += __popc(x);
            }
            const u64 Pc = SUM ? P * L.z[cu] * L.z[cv] : 0ull;
            if (has) acc.ops += 3u * (u32)(Ws - (cv >> 5));
            bool push = false;
            if (!ODD && !EVEN && l2 == 1) {  // listing only: count modes close l = 3 frames whole
                acc.leaf += (u64)cc;
                if (SUM && cc) {
                    u64 zs = 0;
#pragma unroll (W <= 8 ? W : 1)
                    for (int w = 0; w < W; w++) {
                        u32 x = cw[w];
                        while (x) { int b = __ffs(x) - 1; x &= x - 1; zs += L.z[w * 32 + b]; }
                    }
                    acc.csum += Pc * zs;
                }
                if (LIST && !full) {
                    unsigned long long base = 0;
                    int off2 = cc;
                    for (int o = 1; o < 32; o <<= 1) {
                        int y = __shfl_up_sync(0xffffffffu, off2, o);
                        if (lane >= o) off2 += y;
                    }
                    int tot2 = __shfl_sync(0xffffffffu, off2, 31);
                    off2 -= cc;
                    if (lane == 0 && tot2) base = atomicAdd(&q.acc->written, (unsigned long long)tot2);
                    base = __shfl_sync(0xffffffffu, base, 0);
                    u32 ids[KC_MAX_K];
                    int np = 2 * (d + 1);
                    for (int i = 0; i < np; i++) ids[i] = L.path[i];
                    ids[np] = L.vid[cu];
                    ids[np + 1] = L.vid[cv];
                    int idx = 0;
#pragma unroll (W <= 8 ? W : 1)
                    for (int w = 0; w < W; w++) {
                        u32 x = cw[w];
                        while (x) {
                            int b = __ffs(x) - 1;
                            x &= x - 1;
                            if (base + off2 + idx < a.cap) {
                                ids[np + 2] = L.vid[w * 32 + b];
                                write_clique(a.d_out, base + off2 + idx, k, ids, np + 3);
                            }
                            idx++;
                        }
                    }
                }
            } else if (!ODD && l2 == 2) {
                if (cc >= 2) {
                    u64 ec = 0, zs = 0;
                    u32 rest[W];  // cw without the positions visited so far (all <= xp)
#pragma unroll
                    for (int w = 0; w < W; w++) rest[w] = cw[w];
                    // SUM: zr = key sum over rest; a vertex's key sum over its neighbours in
                    // rest is summed directly or, when its non-neighbours there are fewer
                    // (dense frames), as zr minus the keys of those non-neighbours
                    u64 zr = 0;
                    if (SUM) {
#pragma unroll (W <= 8 ? W : 1)
                        for (int w = 0; w < W; w++) {
                            u32 x = cw[w];
                            while (x) { int b = __ffs(x) - 1; x &= x - 1; zr += L.z[w * 32 + b]; }
                        }
                    }
#pragma unroll (W <= 8 ? W : 1)
                    for (int w = 0; w < W; w++) {
                        while (rest[w]) {
                            int b = __ffs(rest[w]) - 1;
                            rest[w] &= rest[w] - 1;
                            const int xp = w * 32 + b;
                            acc.ops += 3u * (u32)(Ws - (xp >> 5));
                            int dn = 0, dm = 0;
#pragma unroll
                            for (int w2 = 0; w2 < W; w2++) {
                                if (w2 < w) continue;
                                const u32 row = L.A[xp * (W + KC_ROW_PAD) + w2];
                                dn += __popc(row & rest[w2]);
                                if (SUM) dm += __popc(rest[w2] & ~row);
                            }
                            ec += (u64)dn;
                            if (SUM) {
                                const u64 zx = L.z[xp];
                                zr -= zx;
                                const bool miss = dm < dn;
                                u64 zin = 0;
                                if (dn && dm) {
#pragma unroll
                                    for (int w2 = 0; w2 < W; w2++) {
                                        if (w2 < w) continue;
                                        const u32 row = L.A[xp * (W + KC_ROW_PAD) + w2];
                                        u32 y = rest[w2] & (miss ? ~row : row);
                                        while (y) { int b2 = __ffs(y) - 1; y &= y - 1; zin += L.z[w2 * 32 + b2]; }
                                    }
                                }
                                zs += zx * (dm == 0 ? zr : miss ? zr - zin : zin);
                            }
                        }
                    }
                    acc.leaf += ec;
                    if (SUM) acc.csum += Pc * zs;
                    if (LIST && !full && ec) {
                        unsigned long long base = atomicAdd(&q.acc->written, (unsigned long long)ec);
                        u32 ids[KC_MAX_K];
                        int np = 2 * (d + 1);
                        for (int i = 0; i < np; i++) ids[i] = L.path[i];
                        ids[np] = L.vid[cu];
                        ids[np + 1] = L.vid[cv];
                        u64 idx = 0;
                        for (int w = 0; w < W; w++) {
                            u32 x = cw[w];
                            while (x) {
                                int b = __ffs(x) - 1;
                                x &= x - 1;
                                const int xp = w * 32 + b;
                                for (int w2 = 0; w2 < W; w2++) {
                                    u32 y = L.A[xp * (W + KC_ROW_PAD) + w2] & cw[w2] & gt_mask(xp, w2);
                                    while (y) {
                                        int b2 = __ffs(y) - 1;
                                        y &= y - 1;
                                        if (base + idx < a.cap) {
                                            ids[np + 2] = L.vid[xp];
                                            ids[np + 3] = L.vid[w2 * 32 + b2];
                                            write_clique(a.d_out, base + idx, k, ids, np + 4);
                                        }
                                        idx++;
                                    }
                                }
                            }
                        }
                    }
                }
            } else {
                bool closed = false;
                if (KC_PRECHECK && !SUM && l2 == 3 && has && cc >= 3 && use_et) {
                    // pre-check against the masks of this child's u: no vertex of C' has
                    // t_max non-neighbours even in the larger set Cu => C' is a t-plex
                    const int slot = L.bs[lane];
                    const u32 *Bm = L.Bm + slot * W, *M1 = L.M1 + slot * W;
                    bool bad = false, any1 = false;
#pragma unroll
                    for (int w = 0; w < W; w++) {
                        bad |= (cw[w] & Bm[w]) != 0u;
                        any1 |= (cw[w] & M1[w]) != 0u;
                    }
                    if (!bad) {
                        const u64 c = (u64)cc;
                        u64 nonuni = 0;
                        if (any1) {  // count the vertices with a non-neighbour inside C'
#pragma unroll (W <= 8 ? W : 1)
                            for (int w = 0; w < W; w++) {
                                u32 bits = cw[w] & M1[w];
                                while (bits) {
                                    const int x = w * 32 + __ffs(bits) - 1;
                                    bits &= bits - 1;
                                    bool nb = false;
#pragma unroll
                                    for (int w2 = 0; w2 < W; w2++)
                                        nb |= (cw[w2] & ~L.A[x * (W + KC_ROW_PAD) + w2] & ~((w2 == (x >> 5)) ? (1u << (x & 31)) : 0u)) != 0u;
                                    nonuni += nb;
                                }
                            }
                        }
                        const u64 f = c - nonuni, pp = nonuni / 2;
                        acc.leaf += f * (f - 1) * (f - 2) / 6 + (f * (f - 1) / 2) * pp * 2 + f * (pp * (pp - 1) / 2) * 4 +
                                    (pp * (pp - 1) * (pp - 2) / 6) * 8;
                        acc.ops += 2u * (u32)(Ws - (cv >> 5));
                        acc.et++;
                        acc.nodes++;
                        closed = true;
                    }
                }
                if (KC_LANE_L3 > 0 && W <= 8 && !EVEN && !closed && l2 == 3 && has && cc >= 3 && (!LIST || full)) {
                    // l = 3 child counted in this lane through its complement H (exact for any
                    // child): with dbar(x) the non-neighbours of x in C', M = sum dbar / 2 the
                    // missing pairs and T the triangles of H,
                    //     #triangles = C(c,3) - M (c-2) + sum_x C(dbar(x), 2) - T,
                    // and with keys (SUM) the same identity weighted:
                    //     e3(z_C') - sum_{ab in M} z_a z_b (Z - z_a - z_b)
                    //              + sum_x z_x e2(z of x's non-neighbours) - T_z.
                    // The lane gives up once M passes KC_LANE_L3 * |C'| (a dense complement:
                    // the child goes to the warp routine).  A child whose H has maximum degree
                    // <= t_max - 1 is a t-plex: the paper's early termination (Sec. 5).
                    const int w0 = cv >> 5;  // the child's set has no bits below v's word
                    const u32 budget = 2u * (u32)KC_LANE_L3 * (u32)cc;
                    u32 msum = 0, visited = 0;
                    u64 s2 = 0;
                    u64 e1 = 0, e2 = 0, e3 = 0;  // SUM: elementary symmetric sums of the keys
                    int maxdb = 0;
                    u32 dm[W];  // vertices with missing partners (SUM: one or more; else two or more)
#pragma unroll
                    for (int w = 0; w < W; w++) dm[w] = 0u;
#pragma unroll
                    for (int w = 0; w < W; w++) {
                        u32 bits = cw[w];
                        while (bits && msum <= budget) {
                            const int b = __ffs(bits) - 1;
                            bits &= bits - 1;
                            const int x = w * 32 + b;
                            int dg = 0;
#pragma unroll
                            for (int w2 = 0; w2 < W; w2++)
                                if (w2 >= w0) dg += __popc(L.A[x * (W + KC_ROW_PAD) + w2] & cw[w2]);
                            const int db = cc - 1 - dg;
                            msum += (u32)db;
                            s2 += (u64)(db * (db - 1) / 2);
                            maxdb = max(maxdb, db);
                            if (db >= (SUM ? 1 : 2)) dm[w] |= 1u << b;
                            if (SUM) {
                                const u64 z = L.z[x];
                                e3 += e2 * z;
                                e2 += e1 * z;
                                e1 += z;
                            }
                            visited++;
                        }
                    }
                    acc.ops += 2u * (u32)(Ws - w0) * visited;
                    if (msum <= budget) {
                        // pairs of H (x, y > x) and its triangles x < y < z
                        u64 tc = 0, zpair = 0, znb = 0, ztri = 0;
                        u32 words = 0;
#pragma unroll
                        for (int w = 0; w < W; w++) {
                            while (dm[w]) {
                                const int x = w * 32 + __ffs(dm[w]) - 1;
                                dm[w] &= dm[w] - 1;
                                const u64 zx = SUM ? L.z[x] : 0ull;
                                u32 r[W];  // missing partners of x above x
                                u64 f1 = 0, f2 = 0;
#pragma unroll
                                for (int w2 = 0; w2 < W; w2++) {
                                    const u32 nb = (w2 >= w0) ? (cw[w2] & ~L.A[x * (W + KC_ROW_PAD) + w2] &
                                                                 ~((w2 == w) ? (1u << (x & 31)) : 0u)) : 0u;
                                    r[w2] = nb & gt_mask(x, w2);
                                    if (SUM) {  // e2 of the keys of all of x's missing partners
                                        u32 t = nb;
                                        while (t) {
                                            const u64 z = L.z[w2 * 32 + __ffs(t) - 1];
                                            t &= t - 1;
                                            f2 += f1 * z;
                                            f1 += z;
                                        }
                                    }
                                }
                                if (SUM) znb += zx * f2;
#pragma unroll
                                for (int wy = 0; wy < W; wy++) {
                                    while (r[wy]) {
                                        const int y = wy * 32 + __ffs(r[wy]) - 1;
                                        r[wy] &= r[wy] - 1;
                                        const u64 zy = SUM ? L.z[y] : 0ull;
                                        u64 zw = 0;
#pragma unroll
                                        for (int w2 = 0; w2 < W; w2++) {
                                            if (w2 < wy) continue;
                                            u32 tb = r[w2] & ~L.A[y * (W + KC_ROW_PAD) + w2];
                                            tc += __popc(tb);
                                            if (SUM)
                                                while (tb) { zw += L.z[w2 * 32 + __ffs(tb) - 1]; tb &= tb - 1; }
                                        }
                                        if (SUM) {
                                            zpair += zx * zy * (e1 - zx - zy);
                                            ztri += zx * zy * zw;
                                        }
                                        words += (u32)(Ws - wy);
                                    }
                                }
                            }
                        }
                        acc.ops += 3u * words;
                        const u64 c = (u64)cc, m = (u64)(msum / 2);
                        acc.leaf += c * (c - 1) * (c - 2) / 6 - m * (c - 2) + s2 - tc;
                        if (SUM) acc.csum += Pc * (e3 - zpair + znb - ztri);
                        if (use_et && maxdb <= tq - 1) acc.et++;
                        acc.nodes++;
                        closed = true;
                    }
                }
                if (!EVEN && !closed && l2 == 3 && has && cc >= 3 && cc <= KC_LANE_ET_MAX && use_et &&
                    (!LIST || full) && (KC_LANE_L3 == 0 || W > 8)) {
                    // l = 3 child: the t-plex test and the Alg. 6 count in this lane (a lane
                    // leaves the test at its first vertex of too small degree); SUM: the x^3
                    // coefficient of prod (1 + c x), c = z_f (universal) or z_a + z_b (pair)
                    const int tmax = min(tq, 2);  // the in-lane forms cover t <= 2
                    const int w0 = cv >> 5;  // the child's set has no bits below v's word
                    int nuni = 0;
                    bool plex = true;
                    u64 p1 = 0, p2 = 0, p3 = 0;
#pragma unroll (W <= 8 ? W : 1)
                    for (int w = 0; w < W; w++) {
                        u32 bits = plex ? cw[w] : 0u;
                        while (bits) {
                            const int x = w * 32 + __ffs(bits) - 1;
                            bits &= bits - 1;
                            int dg = 0;
#pragma unroll
                            for (int w2 = 0; w2 < W; w2++)
                                if (w2 >= w0) dg += __popc(L.A[x * (W + KC_ROW_PAD) + w2] & cw[w2]);
                            if (dg < cc - tmax) { plex = false; bits = 0; }
                            nuni += (dg == cc - 1);
                            if (SUM && plex) {
                                if (dg == cc - 1) {
                                    poly3_mul(p1, p2, p3, L.z[x], 0ull, 0ull);
                                } else {
                                    int y = -1;
#pragma unroll
                                    for (int w2 = 0; w2 < W; w2++) {
                                        const u32 nb = (w2 >= w0) ? (cw[w2] & ~L.A[x * (W + KC_ROW_PAD) + w2] &
                                                                     ~((w2 == (x >> 5)) ? (1u << (x & 31)) : 0u)) : 0u;
                                        if (y < 0 && nb) y = w2 * 32 + __ffs(nb) - 1;
                                    }
                                    if (y > x) poly3_mul(p1, p2, p3, L.z[x] + L.z[y], 0ull, 0ull);
                                }
                            }
                        }
                    }
                    acc.ops += 2u * (u32)(Ws - w0) * (u32)cc;  // (the test may stop early)
                    if (plex) {
                        const u64 c = (u64)cc, f = (u64)nuni, pp = (c - f) / 2;
                        acc.leaf += f * (f - 1) * (f - 2) / 6 + (f * (f - 1) / 2) * pp * 2 + f * (pp * (pp - 1) / 2) * 4 +
                                    (pp * (pp - 1) * (pp - 2) / 6) * 8;
                        if (SUM) acc.csum += Pc * p3;
                        acc.et++;
                        acc.nodes++;
                        closed = true;
                    }
                }
                push = has && !closed && cc >= l2 && (!use_rule2 || distinct_colours<W>(cw, L.J, L.E) >= l2);
            }
            const unsigned pb = __ballot_sync(0xffffffffu, push);
            if (pb) {
                const int slotc = __popc(pb & ((1u << lane) - 1));
                const int dn = d + 1;
                if (push && KC_OK(dn, a.D)) {
                    u32 *dst = L.childC + ((size_t)(dn * 32 + slotc)) * W;
#pragma unroll
                    for (int w = 0; w < W; w++) dst[w] = cw[w];
                    if (SUM) L.childP[dn * 32 + slotc] = Pc;
                    L.childUV[dn * 32 + slotc] = (u32)cu | ((u32)cv << 16);
                }
                if (lane == 0) { L.nchild[dn] = __popc(pb); L.nextc[dn] = 0; }
                __syncwarp();
                phase = 2;
            }
            KC_SEC_END(5);
            continue;
        }
        if (phase == 2) {
            const int dn = d + 1;
            const int nx = L.nextc[dn];
            const int nch = L.nchild[dn];
            __syncwarp();  // every lane has read nextc before lane 0 advances it
            if (nx < nch) {
                if (lane == 0) {
                    L.nextc[dn] = nx + 1;
                    L.slot[dn] = nx;
                    if (LIST) {
                        u32 uv = L.childUV[dn * 32 + nx];
                        L.path[2 * dn] = L.vid[uv & 0xFFFFu];
                        L.path[2 * dn + 1] = L.vid[uv >> 16];
                    }
                }
                __syncwarp();
                d = dn;
                phase = 0;
            } else {
                phase = 1;
            }
            continue;
        }
        // phase 3: frame done
        if (d == 0) break;
        d--;
        phase = 2;
    }
}

// A5-A12, one warp per ticket.  Tickets of the split list (heavy sub-branches, k >= 7)
// are extracted and coloured here, then published with one work item per top-frame
// vertex u for branch_items_kernel; all other tickets run to completion here.
template <int W, int MODE>
__global__ void __launch_bounds__(32 * WARPS_PER_BLOCK_DEFAULT, MinBlocks<W>::value)
branch_kernel(Args a) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr bool SUM = (MODE & (MODE_CHECKSUM | MODE_LIST)) != 0;
    constexpr bool LIST = (MODE & MODE_LIST) != 0;
    constexpr bool ODD = (MODE & MODE_ODD) != 0, EVEN = (MODE & MODE_EVEN) != 0;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const Lay L = make_lay<W>(smem + (size_t)wib * a.warp_bytes, a.D, SUM);
    const bool use_rule1 = !(a.flags & KC_NO_RULE1);
    const bool prof = KC_SECTION_PROFILE && a.prof != 0;
    long long tsec = 0;
    Acc acc;
    reset_unit(acc);
    acc.nodes = 0; acc.et = 0; acc.status = 0; acc.ops = 0; acc.pairs = 0;
#if KC_SECTION_PROFILE
    for (int i = 0; i < 6; i++) acc.sec[i] = 0;
#endif
    WarpTotals wt;
    wt.q_total = 0; wt.q_csum = 0; wt.branches = 0; wt.cur_q = -1;

    while (true) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(a.ticket_ctr, 1ull);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= a.qstart[a.nq]) break;
        int lo = 0, hi = (int)a.nq - 1;
        while (lo < hi) { int mid = (lo + hi + 1) >> 1; if (a.qstart[mid] <= t) lo = mid; else hi = mid - 1; }
        const int qi = lo;
        if (qi != wt.cur_q) { flush_query<MODE>(a, acc, wt, lane, prof); wt.cur_q = qi; }
        const QDesc &q = a.qs[qi];
        const u32 k = q.k;
        const int l0 = (int)k - 2;
        const bool use_et = !(a.flags & KC_NO_ET) && q.t_max >= 1;
        const u64 tq = t - a.qstart[qi];
        const u32 e = q.tickets[q.t0 + tq];
        const long long t_start = clock64();
        const u64 vb = q.vset_ptr[e];
        const int s = (int)(q.vset_ptr[e + 1] - vb);
        if (s < l0) continue;
        if (s > 32 * W) { acc.status |= KC_DEV_ERR_WIDTH; continue; }
        wt.branches++;
        const int Ws = (s + 31) >> 5;  // words a sub-branch of s vertices needs
        const u32 eu = q.eu[e], ev = q.ev[e];
        const u64 P0 = SUM ? zkey(eu) * zkey(ev) : 0ull;
        for (int i = lane; i < s; i += 32) {
            u32 v = q.vset[vb + i];
            L.vid[i] = v;
            if (SUM) L.z[i] = zkey(v);
        }
        if (lane == 0) { L.path[0] = eu; L.path[1] = ev; }
        __syncwarp();
        reset_unit(acc);
        const bool full0 = LIST && (*(volatile unsigned long long *)&q.acc->written >= a.cap);
        if (LIST && a.stop_full && __shfl_sync(0xffffffffu, (int)full0, 0)) break;

        if (!EVEN && l0 == 1) {
            acc.leaf += (lane == 0) ? (u64)s : 0ull;
            if (SUM) {
                u64 zs = 0;
                for (int i = lane; i < s; i += 32) zs += L.z[i];
                acc.csum += P0 * zs;
            }
            if (LIST && !full0) {
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(&q.acc->written, (unsigned long long)s);
                base = __shfl_sync(0xffffffffu, base, 0);
                for (int i = lane; i < s; i += 32) {
                    if (base + i < a.cap) {
                        u32 ids[3] = {eu, ev, L.vid[i]};
                        write_clique(a.d_out, base + i, k, ids, 3);
                    }
                }
            }
        } else {
            KC_SEC_BEGIN();
            extract<W>(L, q, s, e, q.round[e], lane, acc);
            KC_SEC_END(0);
            if (!ODD && l0 == 2) {
                // edges of g_e
                for (int i = lane; i < s; i += 32) {
                    u32 c = 0;
                    u64 zs = 0;
#pragma unroll (W <= 8 ? W : 1)
                    for (int w = 0; w < W; w++) {
                        u32 x = L.A[i * (W + KC_ROW_PAD) + w] & gt_mask(i, w);
                        c += __popc(x);
                        if (SUM) {
                            while (x) { int b = __ffs(x) - 1; x &= x - 1; zs += L.z[w * 32 + b]; }
                        }
                    }
                    acc.leaf += c;
                    acc.ops += 2u * (u32)(Ws - (i >> 5));
                    if (SUM) acc.csum += P0 * L.z[i] * zs;
                    if (LIST && !full0 && c) {
                        unsigned long long base = atomicAdd(&q.acc->written, (unsigned long long)c);
                        u32 idx = 0;
                        for (int w = 0; w < W; w++) {
                            u32 x = L.A[i * (W + KC_ROW_PAD) + w] & gt_mask(i, w);
                            while (x) {
                                int b = __ffs(x) - 1;
                                x &= x - 1;
                                if (base + idx < a.cap) {
                                    u32 ids[4] = {eu, ev, L.vid[i], L.vid[w * 32 + b]};
                                    write_clique(a.d_out, base + idx, k, ids, 4);
                                }
                                idx++;
                            }
                        }
                    }
                }
            } else if (!EVEN && l0 == 3 && (!LIST || full0)) {
                // k = 5 counting: the triangles of g_e need no colours (Rules 1 and 2 only
                // prune deeper branching), so the frame is counted in extraction order
                if (lane < W) L.C0[lane] = lt_mask(s, lane);
                __syncwarp();
                if (lane == 0) acc.nodes++;
                KC_SEC_BEGIN();
                frame_l3_count<W, SUM>(L, L.C0, lane, acc, min((int)q.t_max, 2), use_et, Ws, P0);
                KC_SEC_END(3);
            } else {
                // even k: a top frame with l = 4 (k = 6) is tested and, when dense, counted
                // whole in extraction order: neither the closed forms nor the l = 4 identity
                // depend on the vertex order, so the colouring is done only for a frame that
                // branches
                const bool tested4 = KC_L4 && EVEN && l0 == 4;
                if (tested4) {
                    if (lane < W) L.C0[lane] = lt_mask(s, lane);
                    __syncwarp();
                    if (lane == 0) acc.nodes++;
                    KC_SEC_BEGIN();
                    const bool closed = early_terminate<W, MODE>(L, a, L.C0, 4, P0, lane, acc, use_et, Ws,
                                                                 (uint16_t *)(L.childC + (size_t)32 * W),
                                                                 (int)q.t_max, q, 0, false) ||
                                        frame_l4_count<W, SUM>(L, L.C0, lane, acc, Ws, P0);
                    KC_SEC_END(2);
                    if (closed) {
                        finish_unit<MODE>(q, e, acc, wt, lane, t_start);
                        continue;
                    }
                }
                KC_SEC_BEGIN();
                const int ncol_ok = colour_and_order<W>(L, s, lane);
                KC_SEC_END(1);
                if (ncol_ok < 0) {
                    acc.status |= KC_DEV_ERR_BOUNDS;
                    continue;
                }
                if (SUM) {
                    for (int i = lane; i < s; i += 32) L.z[i] = zkey(L.vid[i]);
                    __syncwarp();
                }
                const bool heavy = !LIST && a.slots != nullptr && l0 >= 5 && tq < q.nheavy;
                bool done = false;
                if (heavy) {
                    // top frame test here, once; the item kernel resumes at its child edges
                    if (lane < W) L.C0[lane] = lt_mask(s, lane);
                    __syncwarp();
                    if (lane == 0) acc.nodes++;
                    KC_SEC_BEGIN();
                    const bool closed = early_terminate<W, MODE>(L, a, L.C0, l0, P0, lane, acc, use_et, Ws,
                                                                 (uint16_t *)(L.childC + (size_t)32 * W),
                                                                 (int)q.t_max, q, 0, false);
                    KC_SEC_END(2);
                    const int limu = min(s, use_rule1 ? (int)L.lim[min(l0, 32 * W + 1)] : s);
                    if (closed || limu <= 0) {
                        done = true;
                    } else {
                        unsigned long long sl = 0;
                        if (lane == 0) sl = atomicAdd(a.slot_ctr, 1ull);
                        sl = __shfl_sync(0xffffffffu, sl, 0);
                        if (sl < a.slot_cap) {
                            unsigned char *gs = a.slots + sl * (u64)slot_bytes<W>();
                            if (lane == 0) {
                                SlotHdr h;
                                h.e = e; h.s = (u32)s; h.qi = (u32)qi; h.limu = (u32)limu; h.P0 = P0; h.pad2 = 0;
                                *(SlotHdr *)gs = h;
                            }
                            u32 *gA = (u32 *)(gs + 32);
                            u32 *gvid = gA + (32 * W) * W;
                            uint16_t *gcol = (uint16_t *)(gvid + 32 * W);
                            uint16_t *glim = gcol + 32 * W;
                            u32 *gJ = (u32 *)((unsigned char *)glim + ((2u * (32u * W + 2) + 15u) & ~15u));
                            for (int i = lane; i < s * W; i += 32) gA[i] = L.A[(i / W) * (W + KC_ROW_PAD) + (i % W)];
                            for (int i = lane; i < s; i += 32) { gvid[i] = L.vid[i]; gcol[i] = L.col[i]; }
                            for (int i = lane; i < 32 * W + 2; i += 32) glim[i] = L.lim[i];
                            if (lane < W) { gJ[lane] = L.J[lane]; gJ[W + lane] = L.E[lane]; }
                            done = true;
                        }
                        // else: no room left, run the sub-branch here (below)
                    }
                }
                if (!done) run_dfs<W, MODE>(L, a, q, s, l0, P0, lane, acc, Ws, 0, s, !heavy && !tested4, prof);
            }
        }
        finish_unit<MODE>(q, e, acc, wt, lane, t_start);
    }
    flush_query<MODE>(a, acc, wt, lane, prof);
}

// A12 split sub-branches: a block takes one work unit at a time -- a published sub-branch
// (slot), or with few slots a stride class of one slot's top-frame vertices -- loads the
// slot's frame into shared memory unless it holds it already, and its warps take the
// unit's vertices u from a block counter; each u runs the child edges (u, v) of the top
// frame and everything below them.  Vertices are handed out in increasing u, the
// costliest first, so the block's wait for its last warp is short.
template <int W>
struct ItemMinBlocks {
    static constexpr int value = W <= 4 ? 6 : (W <= 8 ? KC_ITEM_MINB8 : (W <= 16 ? 2 : 1));
};

template <int W, int MODE>
__global__ void __launch_bounds__(32 * WARPS_PER_BLOCK_DEFAULT, ItemMinBlocks<W>::value)
branch_items_kernel(Args a) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr bool SUM = (MODE & (MODE_CHECKSUM | MODE_LIST)) != 0;
    constexpr int RS = W + KC_ROW_PAD;
    __shared__ unsigned long long s_slot;
    __shared__ int s_unext;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    unsigned char *frame = smem;
    const Lay L = make_lay<W>(smem + frame_bytes<W>(SUM) + (size_t)wib * a.warp_bytes, a.D, SUM, frame);
    const bool prof = KC_SECTION_PROFILE && a.prof != 0;
    Acc acc;
    reset_unit(acc);
    acc.nodes = 0; acc.et = 0; acc.status = 0; acc.ops = 0; acc.pairs = 0;
#if KC_SECTION_PROFILE
    for (int i = 0; i < 6; i++) acc.sec[i] = 0;
#endif
    WarpTotals wt;
    wt.q_total = 0; wt.q_csum = 0; wt.branches = 0; wt.cur_q = -1;
    const u64 n_slots = min((u64)*(volatile unsigned long long *)a.slot_ctr, a.slot_cap);
    // with few slots, several blocks share one: a work unit is (slot, c), c < cps, and takes
    // the vertices u = c, c + cps, c + 2 cps, ... (a mix of costly low u and cheap high u)
    const u64 want_units = 8ull * gridDim.x;
    const u32 cps = n_slots >= want_units ? 1u : (u32)min((u64)((want_units + n_slots - 1) / (n_slots ? n_slots : 1)), (u64)64);
    const u64 n_units = n_slots * cps;
    long long loaded = -1;  // slot whose frame this block holds
    while (true) {
        if (threadIdx.x == 0) {
            s_slot = atomicAdd(a.slot_next, 1ull);
            s_unext = 0;
        }
        __syncthreads();
        const u64 unit = s_slot;
        if (unit >= n_units) break;
        const u64 sl = unit / cps;
        const u32 c0 = (u32)(unit % cps);
        const unsigned char *gs = a.slots + sl * (u64)slot_bytes<W>();
        const SlotHdr h = *(const SlotHdr *)gs;
        const int s = KC_OK(h.s, 32 * W + 1) ? (int)h.s : 0;
        const int limu = KC_OK(h.limu, s + 1) ? (int)h.limu : 0;
        if ((long long)sl != loaded) {
            const u32 *gA = (const u32 *)(gs + 32);
            const u32 *gvid = gA + (32 * W) * W;
            const uint16_t *gcol = (const uint16_t *)(gvid + 32 * W);
            const uint16_t *glim = gcol + 32 * W;
            const u32 *gJ = (const u32 *)((const unsigned char *)glim + ((2u * (32u * W + 2) + 15u) & ~15u));
            for (int i = threadIdx.x; i < s * W; i += blockDim.x) L.A[(i / W) * RS + (i % W)] = gA[i];
            for (int i = threadIdx.x; i < s; i += blockDim.x) {
                const u32 v = gvid[i];
                L.vid[i] = v;
                L.col[i] = gcol[i];
                if (SUM) L.z[i] = zkey(v);
            }
            for (int i = threadIdx.x; i < 32 * W + 2; i += blockDim.x) L.lim[i] = glim[i];
            if (threadIdx.x < W) { L.J[threadIdx.x] = gJ[threadIdx.x]; L.E[threadIdx.x] = gJ[W + threadIdx.x]; }
            loaded = (long long)sl;
        }
        __syncthreads();
        const int qi = (int)h.qi;
        if (qi != wt.cur_q) { flush_query<MODE>(a, acc, wt, lane, prof); wt.cur_q = qi; }
        const QDesc &q = a.qs[qi];
        const int l0 = (int)q.k - 2;
        const int Ws = (s + 31) >> 5;
        while (true) {
            int j = 0;
            if (lane == 0) j = atomicAdd(&s_unext, 1);
            j = __shfl_sync(0xffffffffu, j, 0);
            const long long uu = (long long)c0 + (long long)cps * j;
            if (uu >= limu) break;
            const int u = (int)uu;
            const long long t_start = clock64();
            if (lane == 0) { L.path[0] = q.eu[h.e]; L.path[1] = q.ev[h.e]; }
            __syncwarp();
            reset_unit(acc);
            run_dfs<W, MODE>(L, a, q, s, l0, h.P0, lane, acc, Ws, u, u + 1, false, prof);
            finish_unit<MODE>(q, h.e, acc, wt, lane, t_start);
        }
        __syncthreads();  // every warp is done with this frame before the next one loads
    }
    flush_query<MODE>(a, acc, wt, lane, prof);
}
#undef KC_SEC_BEGIN
#undef KC_SEC_END

// ---------------------------------------------------------------- host-side launch code
// launch geometry for a persistent kernel: (blocks, warps per block, shared bytes)
// block_bytes: dynamic shared memory per block on top of warp_bytes per warp
template <typename K>
kc_status geometry(K kern, u32 warp_bytes, u64 work, const kc_run_cfg *cfg, u64 *blocks, int *wpb_out, size_t *smem_out,
                   u32 block_bytes = 0) {
    // warps per block: the caller's choice within the kernels' launch bound, else the default
    int wpb = (cfg->warps_per_block >= 1 && cfg->warps_per_block <= (u32)WARPS_PER_BLOCK_DEFAULT)
                  ? (int)cfg->warps_per_block : WARPS_PER_BLOCK_DEFAULT;
    int dev = 0, max_optin = 0, nsm = 0;
    KC_CUDA(cudaGetDevice(&dev));
    KC_CUDA(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    KC_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    cudaFuncAttributes fa;
    KC_CUDA(cudaFuncGetAttributes(&fa, kern));
    const size_t dyn_max = (size_t)max_optin - fa.sharedSizeBytes;  // minus static __shared__
    size_t smem = (size_t)block_bytes + (size_t)warp_bytes * wpb;
    while (smem > dyn_max && wpb > 1) { wpb--; smem = (size_t)block_bytes + (size_t)warp_bytes * wpb; }
    if (smem > dyn_max) return KC_ERR_UNSUPPORTED;
    // the attribute is per kernel and process-wide: always the same value (the opt-in
    // maximum), so launches of one kernel with different sizes from several host
    // threads cannot invalidate each other's launch configuration
    KC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_max));
    int per_sm = 0;
    KC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * wpb, smem));
    if (per_sm < 1) per_sm = 1;
    u64 bl = (u64)nsm * per_sm;
    if (cfg->blocks) bl = cfg->blocks;
    u64 need = kc_div_up(work, (u64)wpb);
    if (bl > need) bl = need;
    if (bl < 1) bl = 1;
    *blocks = bl;
    *wpb_out = wpb;
    *smem_out = smem;
    return KC_OK;
}


// one launch group: the queries of one width class (and parity of k), whose descriptors
// d_qs[nq], ticket prefix d_qstart[nq + 1] (total tickets: `tickets`) and zeroed counters
// d_ctr[4] the caller has placed on the device, stream-ordered before this launch
template <int W, int MODE>
kc_status launch_class(const Args &a0, const std::vector<QDesc> &qs, u64 tickets, const kc_run_cfg *cfg,
                       cudaStream_t s, QDesc *d_qs, u64 *d_qstart, unsigned long long *d_ctr, SplitBufs *sb) {
    Args a = a0;
    u32 D = 1;
    u64 nheavy = 0;
    for (const QDesc &q : qs) {
        int l0 = (int)q.k - 2;
        u32 dq = l0 >= 3 ? (u32)((l0 - 3) / 2 + 1) + 1 : 1;
        D = std::max(D, dq);
        nheavy += q.nheavy;
    }
    a.D = D;
    a.warp_bytes = lay_bytes<W>(D, (MODE & (MODE_CHECKSUM | MODE_LIST)) != 0);
    a.qs = d_qs;
    a.qstart = d_qstart;
    a.nq = (u32)qs.size();
    a.ticket_ctr = d_ctr;
    a.slots = nullptr;
    if (nheavy && !(MODE & MODE_LIST)) {
        const u64 need_slots = nheavy * (u64)slot_bytes<W>();
        if (sb->slot_bytes_cap < need_slots) {
            if (sb->slots) KC_CUDA(cudaFreeAsync(sb->slots, s));
            sb->slots = nullptr;
            KC_CUDA(cudaMallocAsync(&sb->slots, need_slots, s));
            sb->slot_bytes_cap = need_slots;
        }
        a.slots = sb->slots;
        a.slot_cap = nheavy;
        a.slot_ctr = d_ctr + 1;
        a.slot_next = d_ctr + 2;
    }
    u64 blocks = 1;
    int wpb = 1;
    size_t smem = 0;
    kc_status st = geometry(branch_kernel<W, MODE>, a.warp_bytes, tickets, cfg, &blocks, &wpb, &smem);
    if (st != KC_OK) return st;
    branch_kernel<W, MODE><<<(unsigned)blocks, 32 * wpb, smem, s>>>(a);
    kc_note_launch();
    KC_CUDA(cudaGetLastError());
    if constexpr (!(MODE & MODE_LIST)) {  // listing passes never split
    if (a.slots) {
        // the item count is only known on the device: size the grid for a full machine
        constexpr bool sum = (MODE & (MODE_CHECKSUM | MODE_LIST)) != 0;
        Args ai = a;
        ai.warp_bytes = lay_bytes<W>(D, sum, true);
        st = geometry(branch_items_kernel<W, MODE>, ai.warp_bytes, ~0ull >> 8, cfg, &blocks, &wpb, &smem,
                      frame_bytes<W>(sum));
        if (st != KC_OK) return st;
        branch_items_kernel<W, MODE><<<(unsigned)blocks, 32 * wpb, smem, s>>>(ai);
        kc_note_launch();
        KC_CUDA(cudaGetLastError());
    }
    }
    return KC_OK;
}

template <int W, int MODE>
kc_status launch_class_fixed(const Args &a0, const QDesc *qs, u32 nqs, const kc_run_cfg *cfg, cudaStream_t s,
                             QDesc *d_qs, u64 *d_qstart, unsigned long long *d_ctr) {
    Args a = a0;
    u32 D = 1;
    for (u32 i = 0; i < nqs; i++) {
        int l0 = (int)qs[i].k - 2;
        u32 dq = l0 >= 3 ? (u32)((l0 - 3) / 2 + 1) + 1 : 1;
        D = std::max(D, dq);
    }
    a.D = D;
    a.warp_bytes = lay_bytes<W>(D, (MODE & (MODE_CHECKSUM | MODE_LIST)) != 0);
    u64 qstart[kNoallocMaxQ + 1];
    qstart[0] = 0;
    for (u32 i = 0; i < nqs; i++) qstart[i + 1] = qstart[i] + qs[i].nt;
    KC_CUDA(cudaMemcpyAsync(d_qs, qs, sizeof(QDesc) * nqs, cudaMemcpyHostToDevice, s));
    KC_CUDA(cudaMemcpyAsync(d_qstart, qstart, sizeof(u64) * (nqs + 1), cudaMemcpyHostToDevice, s));
    KC_CUDA(cudaMemsetAsync(d_ctr, 0, 4 * sizeof(unsigned long long), s));
    a.qs = d_qs;
    a.qstart = d_qstart;
    a.nq = nqs;
    a.ticket_ctr = d_ctr;
    a.slots = nullptr;
    u64 blocks = 1;
    int wpb = 1;
    size_t smem = 0;
    kc_status st = geometry(branch_kernel<W, MODE>, a.warp_bytes, qstart[nqs], cfg, &blocks, &wpb, &smem);
    if (st != KC_OK) return st;
    branch_kernel<W, MODE><<<(unsigned)blocks, 32 * wpb, smem, s>>>(a);
    kc_note_launch();
    KC_CUDA(cudaGetLastError());
    return KC_OK;
}

// load the code of one kernel instance now (module loading is lazy by default: the
// first launch of an instance would otherwise load it, which takes device memory)
template <typename K>
kc_status preload(K kern) {
    cudaFuncAttributes fa;
    KC_CUDA(cudaFuncGetAttributes(&fa, kern));
    return KC_OK;
}
}  // namespace

// the entry points of one width
#define KC_BRANCH_WIDTH(W)                                                                                        \
    namespace kcb {                                                                                               \
    kc_status launch_width_##W(int mode, const Args &a, const std::vector<QDesc> &qs, u64 tickets,                \
                               const kc_run_cfg *cfg, cudaStream_t s, QDesc *d_qs, u64 *d_qstart,                 \
                               unsigned long long *d_ctr, SplitBufs *sb) {                                        \
        switch (mode) {                                                                                           \
            case MODE_ODD: return launch_class<W, MODE_ODD>(a, qs, tickets, cfg, s, d_qs, d_qstart, d_ctr, sb);   \
            case MODE_EVEN: return launch_class<W, MODE_EVEN>(a, qs, tickets, cfg, s, d_qs, d_qstart, d_ctr, sb); \
            case MODE_CHECKSUM | MODE_ODD:                                                                        \
                return launch_class<W, MODE_CHECKSUM | MODE_ODD>(a, qs, tickets, cfg, s, d_qs, d_qstart, d_ctr, sb); \
            case MODE_CHECKSUM | MODE_EVEN:                                                                       \
                return launch_class<W, MODE_CHECKSUM | MODE_EVEN>(a, qs, tickets, cfg, s, d_qs, d_qstart, d_ctr, sb); \
            case MODE_LIST | MODE_CHECKSUM:                                                                       \
                return launch_class<W, MODE_LIST | MODE_CHECKSUM>(a, qs, tickets, cfg, s, d_qs, d_qstart, d_ctr, sb); \
        }                                                                                                         \
        return KC_ERR_INVALID_ARG;                                                                                \
    }                                                                                                             \
    kc_status launch_fixed_width_##W(int mode, const Args &a, const QDesc *qs, u32 nqs, const kc_run_cfg *cfg,    \
                                     cudaStream_t s, QDesc *d_qs, u64 *d_qstart, unsigned long long *d_ctr) {     \
        switch (mode) {                                                                                           \
            case MODE_ODD: return launch_class_fixed<W, MODE_ODD>(a, qs, nqs, cfg, s, d_qs, d_qstart, d_ctr);     \
            case MODE_EVEN: return launch_class_fixed<W, MODE_EVEN>(a, qs, nqs, cfg, s, d_qs, d_qstart, d_ctr);   \
            case MODE_CHECKSUM | MODE_ODD:                                                                        \
                return launch_class_fixed<W, MODE_CHECKSUM | MODE_ODD>(a, qs, nqs, cfg, s, d_qs, d_qstart, d_ctr); \
            case MODE_CHECKSUM | MODE_EVEN:                                                                       \
                return launch_class_fixed<W, MODE_CHECKSUM | MODE_EVEN>(a, qs, nqs, cfg, s, d_qs, d_qstart, d_ctr); \
        }                                                                                                         \
        return KC_ERR_INVALID_ARG;                                                                                \
    }                                                                                                             \
    kc_status preload_width_##W() {                                                                               \
        kc_status st = preload(branch_kernel<W, MODE_ODD>);                                                       \
        if (st == KC_OK) st = preload(branch_kernel<W, MODE_EVEN>);                                               \
        if (st == KC_OK) st = preload(branch_kernel<W, MODE_CHECKSUM | MODE_ODD>);                                \
        if (st == KC_OK) st = preload(branch_kernel<W, MODE_CHECKSUM | MODE_EVEN>);                               \
        return st;                                                                                                \
    }                                                                                                             \
    unsigned long long debug_flag_width_##W() { return read_debug_flag(); }                                       \
    }
#endif  // KC_BRANCH_INSTANTIATE
