// EBBkC-T (paper Alg. 3, Sec. 4.2): edge-oriented branching in which every level, not
// only the top one, follows the global truss-based edge order pi_tau.  A frame is a
// vertex set V together with the key r (peel round, edge id) of the edge that made it;
// its edges are the edges of G between vertices of V whose key exceeds r (they lie in
// ESet of every edge on the path).  The child of a frame edge e' = (x, y) is
// V & VSet(e') -- the vertices w of V with both xw and yw after e' -- with key(e').
// Leaves: l = 1 counts |V|, l = 2 the frame's edges.  There is no colouring, no pruning
// rule beyond |V| >= l and no early termination: this is the ordering ablation against
// EBBkC-H (truss order at the top, colour order inside, Sec. 4.4).
//
// One warp per top-level sub-branch g_e.  Its adjacency (edges after e only) is a bitset
// in shared memory, and the keys of its edges form an s x s matrix in the warp's slice of
// a global scratch buffer; set operations run a word at a time, lane per bit, against
// a row of that matrix.  Count and checksum modes.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "kc_internal.cuh"

namespace {

constexpr int TD = KC_MAX_K / 2 + 1;  // frame stack depth

struct TArgs {
    const u32 *row_ptr, *col, *pos_eid, *pos_round, *eu, *ev, *round, *vset, *tickets;
    const u64 *vset_ptr;
    u64 t0, nt;                 // tickets [t0, t0 + nt)
    unsigned long long *ctr;    // ticket counter
    kc_dev_acc *acc;
    u64 *R;                     // per warp: S x S edge keys
    u32 k;
    u32 warp_bytes;             // shared memory per warp
};

__device__ __forceinline__ u64 tw_sum(u64 x) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// bits of the words above position p (exclusive) in word w
__device__ __forceinline__ u32 above(int p, int w) {
    const int pw = p >> 5;
    if (w < pw) return 0u;
    if (w > pw) return 0xFFFFFFFFu;
    const int b = p & 31;
    return b == 31 ? 0u : (0xFFFFFFFFu << (b + 1));
}

template <int W, bool SUM>
__global__ void __launch_bounds__(128) ebbkc_t_kernel(TArgs a) {
    constexpr int S = 32 * W;
    constexpr int RS = W + 1;  // odd row stride
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    unsigned char *base = smem + (size_t)wib * a.warp_bytes;
    u32 *A = (u32 *)base;                       // [S][RS]
    u32 *vid = A + S * RS;                      // [S]
    u32 *Vs = vid + S;                          // [TD][W] frame vertex sets
    u32 *Ys = Vs + TD * W;                      // [TD][W] the current x's remaining child ends y
    int *xs = (int *)(Ys + TD * W);             // [TD] current x
    u64 *rs = (u64 *)(((uintptr_t)(xs + TD) + 15) & ~(uintptr_t)15);  // [TD] frame keys
    u64 *Ps = rs + TD;                          // [TD] key products of the frame's path
    u64 *z = Ps + TD;                           // [S] keys (SUM)
    const u64 gw = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    u64 *R = a.R + gw * (u64)S * S;
    const int l0 = (int)a.k - 2;
    u64 cnt = 0, csum = 0, nodes = 0, branches = 0;  // lane parts
    unsigned status = 0;
    while (true) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(a.ctr, 1ull);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= a.nt) break;
        const u32 e = a.tickets[a.t0 + t];
        const u64 vb = a.vset_ptr[e];
        const int s = (int)(a.vset_ptr[e + 1] - vb);
        if (s < l0) continue;
        if (s > S) { status |= KC_DEV_ERR_WIDTH; continue; }
        branches++;
        const u32 eu = a.eu[e], ev = a.ev[e], re = a.round[e];
        const u64 ke = ((u64)re << 32) | e;
        const u64 P0 = SUM ? zkey(eu) * zkey(ev) : 0ull;
        for (int i = lane; i < s; i += 32) {
            vid[i] = a.vset[vb + i];
            if (SUM) z[i] = zkey(vid[i]);
        }
        if (l0 == 1) {  // k = 3: the triangles on e
            if (lane == 0) { cnt += (u64)s; nodes++; }
            if (SUM) {
                u64 zs = 0;
                for (int i = lane; i < s; i += 32) zs += z[i];
                csum += P0 * zs;
            }
            __syncwarp();
            continue;
        }
        // g_e: its edges (both ends in VSet(e), after e) as bits, their keys in R
        for (int i = lane; i < S * RS; i += 32) A[i] = 0u;
        __syncwarp();
        const u32 vmax = vid[s - 1];
        for (int i = 0; i + 1 < s; i++) {
            // row x restricted to (x, vmax] (two binary searches, alike in every lane); it is
            // scanned against VSet, or, when much longer, each candidate is searched in it
            const u32 x = vid[i];
            u32 lo = a.row_ptr[x], hi = a.row_ptr[x + 1];
            while (lo < hi) { const u32 mid = (lo + hi) >> 1; if (a.col[mid] <= x) lo = mid + 1; else hi = mid; }
            const u32 rb = lo;
            hi = a.row_ptr[x + 1];
            while (lo < hi) { const u32 mid = (lo + hi) >> 1; if (a.col[mid] <= vmax) lo = mid + 1; else hi = mid; }
            const u32 rend = lo;
            const int rem = s - 1 - i;
            const bool scan = rend - rb <= 4u * (u32)rem;
            const int items = scan ? (int)(rend - rb) : rem;
            for (int it = lane; it < items; it += 32) {
                int j = -1;
                u32 p = 0;
                if (scan) {
                    p = rb + (u32)it;
                    const u32 y = a.col[p];
                    int l2 = i + 1, h2 = s;
                    while (l2 < h2) { const int mid = (l2 + h2) >> 1; if (vid[mid] < y) l2 = mid + 1; else h2 = mid; }
                    if (l2 < s && vid[l2] == y) j = l2;
                } else {
                    const int jj = i + 1 + it;
                    const u32 y = vid[jj];
                    u32 l2 = rb, h2 = rend;
                    while (l2 < h2) { const u32 mid = (l2 + h2) >> 1; if (a.col[mid] < y) l2 = mid + 1; else h2 = mid; }
                    if (l2 < rend && a.col[l2] == y) { j = jj; p = l2; }
                }
                if (j < 0) continue;
                const u32 rr = a.pos_round[p], ee = a.pos_eid[p];
                if (rr > re || (rr == re && ee > e)) {
                    atomicOr(&A[i * RS + (j >> 5)], 1u << (j & 31));
                    atomicOr(&A[j * RS + (i >> 5)], 1u << (i & 31));
                    const u64 kk = ((u64)rr << 32) | ee;
                    R[(u64)i * S + j] = kk;
                    R[(u64)j * S + i] = kk;
                }
            }
        }
        __syncwarp();
        // frame 0: all of VSet(e) with key(e)
        if (lane < W) Vs[lane] = lane < (s >> 5) ? 0xFFFFFFFFu : (lane == (s >> 5) ? (1u << (s & 31)) - 1u : 0u);
        if (lane == 0) { xs[0] = -1; rs[0] = ke; Ps[0] = P0; }
        if (lane < W) Ys[lane] = 0u;
        __syncwarp();
        if (lane == 0) nodes++;
        int d = 0;
        if (l0 == 2) d = -1;  // k = 4: the edges of g_e, below
        if (l0 == 2) {
            // every edge of A is after e
            for (int i = lane; i < s; i += 32) {
                u64 zi = 0;
#pragma unroll
                for (int w = 0; w < W; w++) {
                    u32 m = A[i * RS + w] & above(i, w);
                    cnt += (u64)__popc(m);
                    if (SUM) while (m) { zi += z[w * 32 + __ffs(m) - 1]; m &= m - 1; }
                }
                if (SUM) csum += P0 * z[i] * zi;
            }
        }
        __syncwarp();
        while (d >= 0) {
            const int l = l0 - 2 * d;
            u32 *V = Vs + d * W, *Y = Ys + d * W;
            // the next child end y of the current x, else the next x
            u32 yw = lane < W ? Y[lane] : 0u;
            const unsigned hasy = __ballot_sync(0xffffffffu, yw != 0u);
            if (!hasy) {
                const int x0 = xs[d];
                u32 cand = 0u;
                if (lane < W) cand = V[lane] & above(x0, lane);
                const unsigned hc = __ballot_sync(0xffffffffu, cand != 0u);
                if (!hc) { d--; continue; }  // frame done
                const int wl = __ffs(hc) - 1;
                const u32 cw = __shfl_sync(0xffffffffu, cand, wl);
                const int x = wl * 32 + __ffs(cw) - 1;
                // its child ends: y in V, y > x, xy an edge after the frame's key
                const u64 r = rs[d];
                for (int w = 0; w < W; w++) {
                    const u32 c = V[w] & A[x * RS + w] & above(x, w);
                    const bool ok = ((c >> lane) & 1u) && R[(u64)x * S + w * 32 + lane] > r;
                    const unsigned b = __ballot_sync(0xffffffffu, ok);
                    if (lane == 0) Y[w] = b;
                }
                if (lane == 0) xs[d] = x;
                __syncwarp();
                continue;
            }
            const int wl = __ffs(hasy) - 1;
            const u32 yword = __shfl_sync(0xffffffffu, yw, wl);
            const int y = wl * 32 + __ffs(yword) - 1;
            const int x = xs[d];
            if (lane == wl) Y[wl] = yword & (yword - 1u);
            __syncwarp();
            const u64 kxy = R[(u64)x * S + y];
            // the child: w in V adjacent to x and y by edges after xy
            u32 cv = 0u;  // lane w's word of the child (lanes < W)
            int cc = 0;
            for (int w = 0; w < W; w++) {
                const u32 c = V[w] & A[x * RS + w] & A[y * RS + w];
                const int p = w * 32 + lane;
                const bool ok = ((c >> lane) & 1u) && R[(u64)x * S + p] > kxy && R[(u64)y * S + p] > kxy;
                const unsigned b = __ballot_sync(0xffffffffu, ok);
                if (lane == w) cv = b;
                cc += __popc(b);
            }
            if (lane == 0) nodes++;
            const int l2 = l - 2;
            if (cc < l2) continue;
            const u64 P = SUM ? Ps[d] * z[x] * z[y] : 0ull;
            if (l2 == 1) {
                if (lane == 0) cnt += (u64)cc;
                if (SUM) {
                    u64 zs = 0;
                    if (lane < W) {
                        u32 m = cv;
                        while (m) { zs += z[lane * 32 + __ffs(m) - 1]; m &= m - 1; }
                    }
                    csum += P * zs;
                }
                continue;
            }
            if (l2 == 2) {
                // the child's edges: pairs a < b of it, joined by an edge after xy
                u32 *C2 = Vs + (d + 1) * W;  // scratch: the child's set
                if (lane < W) C2[lane] = cv;
                __syncwarp();
                for (int w0 = 0; w0 < W; w0++) {
                    u32 m = C2[w0];
                    while (m) {
                        const int av = w0 * 32 + __ffs(m) - 1;
                        m &= m - 1;
                        u64 zb = 0;
                        for (int w = w0; w < W; w++) {
                            const u32 c = C2[w] & A[av * RS + w] & above(av, w);
                            const int p = w * 32 + lane;
                            const bool ok = ((c >> lane) & 1u) && R[(u64)av * S + p] > kxy;
                            if (ok) {
                                cnt++;
                                if (SUM) zb += z[p];
                            }
                        }
                        if (SUM) csum += P * z[av] * zb;
                    }
                }
                __syncwarp();
                continue;
            }
            // descend
            if (d + 1 >= TD) { status |= KC_DEV_ERR_BOUNDS; continue; }
            if (lane < W) { Vs[(d + 1) * W + lane] = cv; Ys[(d + 1) * W + lane] = 0u; }
            if (lane == 0) { xs[d + 1] = -1; rs[d + 1] = kxy; Ps[d + 1] = P; }
            __syncwarp();
            d++;
        }
        __syncwarp();
    }
    cnt = tw_sum(cnt);
    csum = tw_sum(csum);
    nodes = tw_sum(nodes);
    status = __reduce_or_sync(0xffffffffu, status);
    if (lane == 0) {
        const unsigned long long old = atomicAdd(&a.acc->count_lo, (unsigned long long)cnt);
        if (old + cnt < old) atomicAdd(&a.acc->count_hi, 1ull);
        if (SUM) atomicAdd(&a.acc->checksum, (unsigned long long)csum);
        atomicAdd(&a.acc->nodes, (unsigned long long)nodes);
        atomicAdd(&a.acc->branches, (unsigned long long)branches);
        if (status) atomicOr(&a.acc->status, status);
    }
}

template <int W>
u32 t_warp_bytes() {
    constexpr u32 S = 32u * W;
    u32 b = 4u * S * (W + 1) + 4u * S + 8u * TD * W + 4u * TD;
    b = (b + 15u) & ~15u;
    b += 16u * TD + 8u * S;
    return (b + 15u) & ~15u;
}

template <int W>
kc_status launch_t(const TArgs &a0, bool sum, int warps, int blocks, cudaStream_t s) {
    TArgs a = a0;
    a.warp_bytes = t_warp_bytes<W>();
    const size_t sh = (size_t)a.warp_bytes * warps;
    auto kern = sum ? ebbkc_t_kernel<W, true> : ebbkc_t_kernel<W, false>;
    KC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh));
    kern<<<blocks, 32 * warps, sh, s>>>(a);
    kc_note_launch();
    KC_CUDA(cudaGetLastError());
    return KC_OK;
}

u64 suffix_t(const kc_graph *g, u64 x) { return x > g->tau ? 0ull : g->h_size_suffix[x]; }

}  // namespace

kc_status kc_run_ebbkc_t(const kc_graph *g, u32 k, const kc_run_cfg *cfg, cudaStream_t s, kc_dev_acc *h_acc,
                         float *ms, float *ms_branch) {
    int dev = 0, nsm = 0;
    KC_CUDA(cudaGetDevice(&dev));
    KC_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const bool sum = (cfg->flags & KC_CHECKSUM) != 0;
    const int widths[6] = {32, 16, 8, 4, 2, 1};
    // one scratch for the largest class launched: per warp an S x S key matrix
    struct Launch { int W; u64 b, en; int warps, blocks; };
    std::vector<Launch> ls;
    u64 rbytes = 0;
    for (int W : widths) {
        const u64 s_hi = 32ull * W, s_lo = std::max<u64>(W == 1 ? 0ull : 16ull * W + 1, (u64)k - 2);
        if (s_lo > s_hi) continue;
        u64 b = suffix_t(g, s_hi + 1), en = suffix_t(g, s_lo);
        if (cfg->ticket_end > cfg->ticket_begin) {
            b = std::max<u64>(b, cfg->ticket_begin);
            en = std::min<u64>(en, cfg->ticket_end);
        }
        if (en <= b) continue;
        const int warps = W >= 32 ? 1 : (W >= 16 ? 2 : 4);
        const int blocks = nsm * (W >= 16 ? 1 : 2);
        ls.push_back({W, b, en, warps, blocks});
        rbytes = std::max<u64>(rbytes, (u64)warps * blocks * (32ull * W) * (32ull * W) * 8ull);
    }
    unsigned char *dbuf = nullptr;
    const u64 hdr = (sizeof(kc_dev_acc) + 8 * sizeof(unsigned long long) + 255) & ~255ull;
    KC_CUDA(cudaMallocAsync(&dbuf, hdr + rbytes, s));
    KC_CUDA(cudaMemsetAsync(dbuf, 0, hdr, s));
    TArgs a;
    memset(&a, 0, sizeof(a));
    a.row_ptr = g->row_ptr; a.col = g->col; a.pos_eid = g->pos_eid; a.pos_round = g->pos_round;
    a.eu = g->eu; a.ev = g->ev; a.round = g->round; a.vset = g->vset; a.tickets = g->tickets;
    a.vset_ptr = g->vset_ptr;
    a.k = k;
    a.acc = (kc_dev_acc *)dbuf;
    a.R = (u64 *)(dbuf + hdr);
    cudaEvent_t ev[2];
    KC_CUDA(cudaEventCreate(&ev[0]));
    KC_CUDA(cudaEventCreate(&ev[1]));
    KC_CUDA(cudaEventRecord(ev[0], s));
    kc_status st = KC_OK;
    for (size_t i = 0; i < ls.size() && st == KC_OK; i++) {
        const Launch &L = ls[i];
        a.t0 = L.b;
        a.nt = L.en - L.b;
        a.ctr = (unsigned long long *)(dbuf + sizeof(kc_dev_acc)) + i % 8;
        switch (L.W) {
            case 1: st = launch_t<1>(a, sum, L.warps, L.blocks, s); break;
            case 2: st = launch_t<2>(a, sum, L.warps, L.blocks, s); break;
            case 4: st = launch_t<4>(a, sum, L.warps, L.blocks, s); break;
            case 8: st = launch_t<8>(a, sum, L.warps, L.blocks, s); break;
            case 16: st = launch_t<16>(a, sum, L.warps, L.blocks, s); break;
            default: st = launch_t<32>(a, sum, L.warps, L.blocks, s); break;
        }
    }
    KC_CUDA(cudaEventRecord(ev[1], s));
    if (st == KC_OK) KC_CUDA(cudaMemcpyAsync(h_acc, dbuf, sizeof(kc_dev_acc), cudaMemcpyDeviceToHost, s));
    cudaFreeAsync(dbuf, s);
    KC_CUDA(cudaStreamSynchronize(s));
    cudaEventElapsedTime(ms, ev[0], ev[1]);
    *ms_branch = *ms;
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    return st;
}
