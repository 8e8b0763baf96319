// Graph preparation on the device (paper Alg. 5 and Alg. 3):
//   A1  clean symmetric CSR (drop directions, duplicates, self-loops; Sec. 6.1)
//   A2  edge ids, triangle listing on a degree orientation, per-edge triangle incidence
//   A3  truss-based edge ordering (Sec. 4.2, Eq. 6) by level-synchronous peeling:
//       at level s every remaining edge with support <= s is removed in one round,
//       supports of surviving edges drop once per destroyed triangle, rounds repeat
//       until none is <= s, then s rises to the least remaining support.  The edge
//       order is (round, edge id).
//   A4  VSet(e) = third vertices of the triangles whose first edge (in that order)
//       is e -- the vertex set of the sub-branch g_e of Eq. 2; |VSet(e)| <= level(e).
// All kernels are HBM/L2 bound integer work; no tensor cores.
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "kc_internal.cuh"

namespace {

constexpr int TPB = 256;

inline unsigned grid_for(u64 n, int tpb = TPB) {
    u64 b = (n + tpb - 1) / tpb;
    if (b < 1) b = 1;
    if (b > (1u << 30)) b = 1u << 30;
    return (unsigned)b;
}

// ------------------------------------------------------------ scans
// Exclusive prefix sum of n values of type TI into TO (out has n+1 entries: out[n] = total).
template <typename TI, typename TO>
__global__ void scan_block_kernel(const TI *__restrict__ in, TO *__restrict__ out, TO *__restrict__ block_sums, u64 n) {
    constexpr int PER = 4;
    __shared__ TO warp_tot[32];
    u64 base = (u64)blockIdx.x * blockDim.x * PER;
    TO v[PER];
    TO local = 0;
    for (int i = 0; i < PER; i++) {
        u64 idx = base + (u64)threadIdx.x * PER + i;
        v[i] = idx < n ? (TO)in[idx] : (TO)0;
        local += v[i];
    }
    // inclusive scan of `local` across the block
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    TO x = local;
    for (int o = 1; o < 32; o <<= 1) {
        TO y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int nw = blockDim.x >> 5;
        TO t = lane < nw ? warp_tot[lane] : (TO)0;
        for (int o = 1; o < 32; o <<= 1) {
            TO y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) warp_tot[lane] = t;
    }
    __syncthreads();
    TO excl = x - local + (wid > 0 ? warp_tot[wid - 1] : (TO)0);
    for (int i = 0; i < PER; i++) {
        u64 idx = base + (u64)threadIdx.x * PER + i;
        if (idx < n) out[idx] = excl;
        excl += v[i];
    }
    if (threadIdx.x == blockDim.x - 1) block_sums[blockIdx.x] = excl;
}

template <typename TO>
__global__ void scan_add_kernel(TO *__restrict__ out, const TO *__restrict__ offs, u64 n, int per_block) {
    u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += offs[i / per_block];
}

template <typename TO>
__global__ void set_total_kernel(TO *out, const TO *block_sums_scanned, const TO *block_sums, u64 nb, u64 n) {
    out[n] = block_sums_scanned[nb - 1] + block_sums[nb - 1];
}

template <typename TI, typename TO>
kc_status scan_excl(const TI *in, TO *out, u64 n, cudaStream_t s) {
    const int threads = 1024, per = threads * 4;
    if (n == 0) {
        KC_CUDA(cudaMemsetAsync(out, 0, sizeof(TO), s));
        return KC_OK;
    }
    u64 nb = kc_div_up(n, per);
    TO *bs = nullptr, *bss = nullptr;
    KC_CUDA(cudaMallocAsync(&bs, sizeof(TO) * (nb + 1), s));
    KC_CUDA(cudaMallocAsync(&bss, sizeof(TO) * (nb + 1), s));
    scan_block_kernel<TI, TO><<<(unsigned)nb, threads, 0, s>>>(in, out, bs, n);
    kc_note_launch();
    if (nb > 1) {
        kc_status st = scan_excl<TO, TO>(bs, bss, nb, s);
        if (st != KC_OK) return st;
        scan_add_kernel<TO><<<grid_for(n), TPB, 0, s>>>(out, bss, n, per);
        kc_note_launch();
        set_total_kernel<TO><<<1, 1, 0, s>>>(out, bss, bs, nb, n);
        kc_note_launch();
    } else {
        KC_CUDA(cudaMemcpyAsync(out + n, bs, sizeof(TO), cudaMemcpyDeviceToDevice, s));
    }
    KC_CUDA(cudaFreeAsync(bs, s));
    KC_CUDA(cudaFreeAsync(bss, s));
    return KC_OK;
}

// ------------------------------------------------------------ validation / cleaning
__global__ void validate_kernel(const u32 *__restrict__ rp, const u32 *__restrict__ col, u32 n, u64 nnz,
                                unsigned *status) {
    u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    u64 stride = (u64)gridDim.x * blockDim.x;
    for (u64 v = i; v < n; v += stride)
        if (rp[v] > rp[v + 1]) atomicOr(status, KC_DEV_ERR_GRAPH);
    if (i == 0 && (rp[0] != 0 || rp[n] != nnz)) atomicOr(status, KC_DEV_ERR_GRAPH);
    for (u64 p = i; p < nnz; p += stride)
        if (col[p] >= n) atomicOr(status, KC_DEV_ERR_GRAPH);
}

__device__ __forceinline__ u64 lower_bound_u32(const u32 *__restrict__ a, u64 lo, u64 hi, u32 x) {
    while (lo < hi) {
        u64 mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// already clean?  strictly increasing rows, no loops, symmetric
__global__ void clean_check_kernel(const u32 *__restrict__ rp, const u32 *__restrict__ col, u32 n, unsigned *bad) {
    u64 warp = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    u64 nwarps = ((u64)gridDim.x * blockDim.x) >> 5;
    for (u64 u = warp; u < n; u += nwarps) {
        u32 b = rp[u], e = rp[u + 1];
        for (u32 p = b + lane; p < e; p += 32) {
            u32 v = col[p];
            bool ok = v != u && (p == b || col[p - 1] < v);
            if (ok) {
                u64 q = lower_bound_u32(col, rp[v], rp[v + 1], (u32)u);
                ok = q < rp[v + 1] && col[q] == u;
            }
            if (!ok) atomicOr(bad, 1u);
        }
    }
}

__global__ void sym_count_kernel(const u32 *__restrict__ rp, const u32 *__restrict__ col, u32 n, u32 *cnt) {
    u64 warp = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    u64 nwarps = ((u64)gridDim.x * blockDim.x) >> 5;
    for (u64 u = warp; u < n; u += nwarps) {
        u32 b = rp[u], e = rp[u + 1];
        for (u32 p = b + lane; p < e; p += 32) {
            u32 v = col[p];
            if (v != u) { atomicAdd(&cnt[u], 1u); atomicAdd(&cnt[v], 1u); }
        }
    }
}

__global__ void sym_scatter_kernel(const u32 *__restrict__ rp, const u32 *__restrict__ col, u32 n,
                                   u64 *cursor, u32 *tcol) {
    u64 warp = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    u64 nwarps = ((u64)gridDim.x * blockDim.x) >> 5;
    for (u64 u = warp; u < n; u += nwarps) {
        u32 b = rp[u], e = rp[u + 1];
        for (u32 p = b + lane; p < e; p += 32) {
            u32 v = col[p];
            if (v != u) {
                tcol[atomicAdd((unsigned long long *)&cursor[u], 1ull)] = v;
                tcol[atomicAdd((unsigned long long *)&cursor[v], 1ull)] = (u32)u;
            }
        }
    }
}

// ------------------------------------------------------------ segmented sort
// Rows are sorted by one of three kernels chosen by length; bins hold row ids.
__global__ void bin_rows_kernel(const u64 *__restrict__ ptr, u64 nrows, u32 *bins, u32 *bin_cnt,
                                u32 lim_warp, u32 lim_block) {
    u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nrows) return;
    u64 len = ptr[i + 1] - ptr[i];
    if (len <= 1) return;
    int b = len <= lim_warp ? 0 : (len <= lim_block ? 1 : 2);
    u32 slot = atomicAdd(&bin_cnt[b], 1u);
    bins[(u64)b * nrows + slot] = (u32)i;
}

// one warp per row of length <= 32: register bitonic sort
__global__ void sort_rows_warp_kernel(const u64 *__restrict__ ptr, u32 *data, const u32 *__restrict__ rows,
                                      const u32 *__restrict__ nrows_p) {
    u64 warp = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    u64 nwarps = ((u64)gridDim.x * blockDim.x) >> 5;
    u32 nrows = *nrows_p;
    for (u64 r = warp; r < nrows; r += nwarps) {
        u32 row = rows[r];
        u64 b = ptr[row];
        u32 len = (u32)(ptr[row + 1] - b);
        u32 x = lane < (int)len ? data[b + lane] : 0xFFFFFFFFu;
        for (int k = 2; k <= 32; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                u32 y = __shfl_xor_sync(0xffffffffu, x, j);
                bool up = ((lane & k) == 0);
                bool lower = ((lane & j) == 0);
                x = (lower == up) ? min(x, y) : max(x, y);
            }
        if (lane < (int)len) data[b + lane] = x;
    }
}

// one block per row, shared-memory bitonic sort of up to `cap` (power of two) entries
__global__ void sort_rows_block_kernel(const u64 *__restrict__ ptr, u32 *data, const u32 *__restrict__ rows,
                                       const u32 *__restrict__ nrows_p, u32 cap) {
    extern __shared__ u32 sh[];
    u32 nrows = *nrows_p;
    for (u32 r = blockIdx.x; r < nrows; r += gridDim.x) {
        u32 row = rows[r];
        u64 b = ptr[row];
        u32 len = (u32)(ptr[row + 1] - b);
        u32 P = 1;
        while (P < len) P <<= 1;
        for (u32 i = threadIdx.x; i < P; i += blockDim.x) sh[i] = i < len ? data[b + i] : 0xFFFFFFFFu;
        __syncthreads();
        for (u32 k = 2; k <= P; k <<= 1)
            for (u32 j = k >> 1; j > 0; j >>= 1) {
                for (u32 i = threadIdx.x; i < P; i += blockDim.x) {
                    u32 q = i ^ j;
                    if (q > i) {
                        u32 a = sh[i], c = sh[q];
                        bool up = (i & k) == 0;
                        if ((a > c) == up) { sh[i] = c; sh[q] = a; }
                    }
                }
                __syncthreads();
            }
        for (u32 i = threadIdx.x; i < len; i += blockDim.x) data[b + i] = sh[i];
        __syncthreads();
    }
    (void)cap;
}

// one block per row, bitonic sort in a global scratch buffer (very long rows)
__global__ void sort_rows_global_kernel(const u64 *__restrict__ ptr, u32 *data, const u32 *__restrict__ rows,
                                        u32 nrows, u32 *scratch, u64 scratch_len) {
    for (u32 r = blockIdx.x; r < nrows; r += gridDim.x) {
        u32 row = rows[r];
        u64 b = ptr[row];
        u64 len = ptr[row + 1] - b;
        u64 P = 1;
        while (P < len) P <<= 1;
        if (P > scratch_len) continue;  // host sized the scratch for the longest row
        u32 *sh = scratch;
        for (u64 i = threadIdx.x; i < P; i += blockDim.x) sh[i] = i < len ? data[b + i] : 0xFFFFFFFFu;
        __syncthreads();
        for (u64 k = 2; k <= P; k <<= 1)
            for (u64 j = k >> 1; j > 0; j >>= 1) {
                for (u64 i = threadIdx.x; i < P; i += blockDim.x) {
                    u64 q = i ^ j;
                    if (q > i) {
                        u32 a = sh[i], c = sh[q];
                        bool up = (i & k) == 0;
                        if ((a > c) == up) { sh[i] = c; sh[q] = a; }
                    }
                }
                __syncthreads();
            }
        for (u64 i = threadIdx.x; i < len; i += blockDim.x) data[b + i] = sh[i];
        __syncthreads();
    }
}

kc_status sort_segments(const u64 *d_ptr, u32 *d_data, u64 nrows, cudaStream_t s) {
    if (nrows == 0) return KC_OK;
    const u32 lim_warp = 32, lim_block = 8192;
    u32 *bins = nullptr, *bin_cnt = nullptr;
    KC_CUDA(cudaMallocAsync(&bins, sizeof(u32) * nrows * 3, s));
    KC_CUDA(cudaMallocAsync(&bin_cnt, sizeof(u32) * 4, s));
    KC_CUDA(cudaMemsetAsync(bin_cnt, 0, sizeof(u32) * 4, s));
    bin_rows_kernel<<<grid_for(nrows), TPB, 0, s>>>(d_ptr, nrows, bins, bin_cnt, lim_warp, lim_block);
    kc_note_launch();
    u32 h_cnt[4];
    KC_CUDA(cudaMemcpyAsync(h_cnt, bin_cnt, sizeof(u32) * 4, cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaStreamSynchronize(s));
    if (h_cnt[0]) {
        sort_rows_warp_kernel<<<grid_for((u64)h_cnt[0] * 32), TPB, 0, s>>>(d_ptr, d_data, bins, bin_cnt);
        kc_note_launch();
    }
    if (h_cnt[1]) {
        size_t sm = sizeof(u32) * lim_block;
        KC_CUDA(cudaFuncSetAttribute(sort_rows_block_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        unsigned nb = h_cnt[1] < 65536 ? h_cnt[1] : 65536;
        sort_rows_block_kernel<<<nb, 512, sm, s>>>(d_ptr, d_data, bins + nrows, bin_cnt + 1, lim_block);
        kc_note_launch();
    }
    if (h_cnt[2]) {
        // longest row -> scratch size (one row at a time per block; use one block)
        std::vector<u32> rows(h_cnt[2]);
        KC_CUDA(cudaMemcpyAsync(rows.data(), bins + 2 * nrows, sizeof(u32) * h_cnt[2], cudaMemcpyDeviceToHost, s));
        std::vector<u64> hp(nrows + 1);
        KC_CUDA(cudaMemcpyAsync(hp.data(), d_ptr, sizeof(u64) * (nrows + 1), cudaMemcpyDeviceToHost, s));
        KC_CUDA(cudaStreamSynchronize(s));
        u64 maxlen = 0;
        for (u32 r : rows) maxlen = std::max<u64>(maxlen, hp[r + 1] - hp[r]);
        u64 P = 1;
        while (P < maxlen) P <<= 1;
        u32 *scratch = nullptr;
        KC_CUDA(cudaMallocAsync(&scratch, sizeof(u32) * P, s));
        sort_rows_global_kernel<<<1, 1024, 0, s>>>(d_ptr, d_data, bins + 2 * nrows, h_cnt[2], scratch, P);
        kc_note_launch();
        KC_CUDA(cudaFreeAsync(scratch, s));
    }
    KC_CUDA(cudaFreeAsync(bins, s));
    KC_CUDA(cudaFreeAsync(bin_cnt, s));
    return KC_OK;
}

__global__ void dedupe_count_kernel(const u64 *__restrict__ tptr, const u32 *__restrict__ tcol, u32 n, u32 *cnt) {
    u64 warp = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    u64 nwarps = ((u64)gridDim.x * blockDim.x) >> 5;
    for (u64 u = warp; u < n; u += nwarps) {
        u64 b = tptr[u], e = tptr[u + 1];
        u32 c = 0;
        for (u64 p = b + lane; p < e; p += 32) c += (p == b || tcol[p - 1] != tcol[p]);
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0) cnt[u] = c;
    }
}

__global__ void dedupe_write_kernel(const u64 *__restrict__ tptr, const u32 *__restrict__ tcol, u32 n,
                                    const u64 *__restrict__ optr, u32 *ocol) {
    u64 warp = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    u64 nwarps = ((u64)gridDim.x * blockDim.x) >> 5;
    for (u64 u = warp; u < n; u += nwarps) {
        u64 b = tptr[u], e = tptr[u + 1];
        u64 out = optr[u];
        for (u64 p0 = b; p0 < e; p0 += 32) {
            u64 p = p0 + lane;
            bool keep = p < e && (p == b || tcol[p - 1] != tcol[p]);
            unsigned bal = __ballot_sync(0xffffffffu, keep);
            if (keep) ocol[out + __popc(bal & ((1u << lane) - 1))] = tcol[p];
            out += __popc(bal);
        }
    }
}

__global__ void u64_to_u32_kernel(const u64 *__restrict__ in, u32 *__restrict__ out, u64 n) {
    u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (u32)in[i];
}

// ------------------------------------------------------------ edge ids
__global__ void upper_count_kernel(const u32 *__restrict__ rp, const u32 *__restrict__ col, u32 n,
                                   u32 *ucnt, u32 *ustart, u32 *maxdeg) {
    u64 u = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    u32 b = rp[u], e = rp[u + 1];
    u32 s = (u32)lower_bound_u32(col, b, e, (u32)u + 1);
    ustart[u] = s;
    ucnt[u] = e - s;
    atomicMax(maxdeg, e - b);
}

__global__ void edge_ids_upper_kernel(const u32 *__restrict__ rp, const u32 *__restrict__ col, u32 n,
                                      const u32 *__restrict__ ustart, const u64 *__restrict__ eoff,
                                      u32 *pos_eid, u32 *eu, u32 *ev) {
    u64 warp = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    u64 nwarps = ((u64)gridDim.x * blockDim.x) >> 5;
    for (u64 u = warp; u < n; u += nwarps) {
        u32 s = ustart[u], e = rp[u + 1];
        for (u32 p = s + lane; p < e; p += 32) {
            u32 id = (u32)(eoff[u] + (p - s));
            pos_eid[p] = id;
            eu[id] = (u32)u;
            ev[id] = col[p];
        }
    }
}

__global__ void edge_ids_lower_kernel(const u32 *__restrict__ rp, const u32 *__restrict__ col, u32 n,
                                      const u32 *__restrict__ ustart, u32 *pos_eid) {
    u64 warp = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    u64 nwarps = ((u64)gridDim.x * blockDim.x) >> 5;
    for (u64 u = warp; u < n; u += nwarps) {
        u32 b = rp[u], s = ustart[u];
        for (u32 p = b + lane; p < s; p += 32) {
            u32 v = col[p];
            u64 q = lower_bound_u32(col, ustart[v], rp[v + 1], (u32)u);
            pos_eid[p] = pos_eid[q];
        }
    }
}

// ------------------------------------------------------------ triangles
// degree orientation: u -> v iff (deg u, u) < (deg v, v)
__device__ __forceinline__ bool before(u32 du, u32 u, u32 dv, u32 v) { return du < dv || (du == dv && u < v); }

__global__ void orient_count_kernel(const u32 *__restrict__ rp, const u32 *__restrict__ col, u32 n, u32 *ocnt) {
    u64 warp = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    u64 nwarps = ((u64)gridDim.x * blockDim.x) >> 5;
    for (u64 u = warp; u < n; u += nwarps) {
        u32 b = rp[u], e = rp[u + 1], du = e - b, c = 0;
        for (u32 p = b + lane; p < e; p += 32) {
            u32 v = col[p];
            c += before(du, (u32)u, rp[v + 1] - rp[v], v);
        }
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0) ocnt[u] = c;
    }
}

__global__ void orient_write_kernel(const u32 *__restrict__ rp, const u32 *__restrict__ col,
                                    const u32 *__restrict__ pos_eid, u32 n, const u64 *__restrict__ optr,
                                    u32 *ocol, u32 *oeid) {
    u64 warp = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    u64 nwarps = ((u64)gridDim.x * blockDim.x) >> 5;
    for (u64 u = warp; u < n; u += nwarps) {
        u32 b = rp[u], e = rp[u + 1], du = e - b;
        u64 out = optr[u];
        for (u32 p0 = b; p0 < e; p0 += 32) {
            u32 p = p0 + lane;
            bool keep = false;
            u32 v = 0;
            if (p < e) { v = col[p]; keep = before(du, (u32)u, rp[v + 1] - rp[v], v); }
            unsigned bal = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                u64 q = out + __popc(bal & ((1u << lane) - 1));
                ocol[q] = v;
                oeid[q] = pos_eid[p];
            }
            out += __popc(bal);
        }
    }
}

// For every oriented edge u->v: common out-neighbours w (both lists sorted by id).
// MODE 0: add 1 to the support of the three edges.  MODE 1: append the other two
// edge ids to each edge's incidence list.
template <int MODE>
__global__ void triangles_kernel(const u32 *__restrict__ rp, const u32 *__restrict__ col, u32 n,
                                 const u64 *__restrict__ optr, const u32 *__restrict__ ocol,
                                 const u32 *__restrict__ oeid, u32 *sup, u64 *cursor, u64 *inc) {
    u64 warp = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    u64 nwarps = ((u64)gridDim.x * blockDim.x) >> 5;
    for (u64 u = warp; u < n; u += nwarps) {
        u64 ub = optr[u], ue = optr[u + 1];
        for (u64 a = ub; a < ue; a++) {
            u32 v = ocol[a], euv = oeid[a];
            u64 vb = optr[v], ve = optr[v + 1];
            // lanes stride over the shorter list, binary search the longer
            bool u_short = (ue - ub) <= (ve - vb);
            u64 sb = u_short ? ub : vb, se = u_short ? ue : ve;
            u64 lb = u_short ? vb : ub, le = u_short ? ve : ue;
            for (u64 p = sb + lane; p < se; p += 32) {
                u32 w = ocol[p];
                u64 q = lower_bound_u32(ocol, lb, le, w);
                if (q < le && ocol[q] == w) {
                    u32 e1 = oeid[p], e2 = oeid[q];  // (short-owner, w), (long-owner, w)
                    if (MODE == 0) {
                        atomicAdd(&sup[euv], 1u);
                        atomicAdd(&sup[e1], 1u);
                        atomicAdd(&sup[e2], 1u);
                    } else {
                        inc[atomicAdd((unsigned long long *)&cursor[euv], 1ull)] = ((u64)e1 << 32) | e2;
                        inc[atomicAdd((unsigned long long *)&cursor[e1], 1ull)] = ((u64)euv << 32) | e2;
                        inc[atomicAdd((unsigned long long *)&cursor[e2], 1ull)] = ((u64)euv << 32) | e1;
                    }
                }
            }
        }
    }
}

// ------------------------------------------------------------ peel
// st: 0 alive, 1 in the current frontier, 2 removed
__global__ void compact_alive_kernel(const u32 *__restrict__ alive, u32 nalive, const uint8_t *__restrict__ st,
                                     const u32 *__restrict__ sup, u32 *alive_out, u32 *cnt, u32 *minsup) {
    u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nalive) return;
    u32 e = alive[i];
    if (st[e] == 2) return;
    alive_out[atomicAdd(cnt, 1u)] = e;
    atomicMin(minsup, sup[e]);
}

__global__ void frontier_from_alive_kernel(const u32 *__restrict__ alive, u32 nalive, const u32 *__restrict__ sup,
                                           u32 s, u32 *F, u32 *fcnt) {
    u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nalive) return;
    u32 e = alive[i];
    if (sup[e] <= s) F[atomicAdd(fcnt, 1u)] = e;
}

__global__ void mark_frontier_kernel(const u32 *__restrict__ F, u32 nf, uint8_t *st, u32 *level, u32 *round,
                                     u32 s, u32 r) {
    u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    u32 e = F[i];
    st[e] = 1;
    level[e] = s;
    round[e] = r;
}

__global__ void peel_round_kernel(const u32 *__restrict__ F, u32 nf, const u64 *__restrict__ inc_ptr,
                                  const u64 *__restrict__ inc, const uint8_t *__restrict__ st, u32 *sup, u32 s,
                                  u32 *Fn, u32 *fncnt) {
    u64 warp = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    u64 nwarps = ((u64)gridDim.x * blockDim.x) >> 5;
    for (u64 i = warp; i < nf; i += nwarps) {
        u32 e = F[i];
        for (u64 p = inc_ptr[e] + lane; p < inc_ptr[e + 1]; p += 32) {
            u64 pr = inc[p];
            u32 e1 = (u32)(pr >> 32), e2 = (u32)pr;
            uint8_t s1 = st[e1], s2 = st[e2];
            if (s1 == 2 || s2 == 2) continue;          // triangle destroyed in an earlier round
            if ((s1 == 1 && e1 < e) || (s2 == 1 && e2 < e)) continue;  // another frontier edge owns it
            if (s1 == 0) { u32 old = atomicSub(&sup[e1], 1u); if (old == s + 1) Fn[atomicAdd(fncnt, 1u)] = e1; }
            if (s2 == 0) { u32 old = atomicSub(&sup[e2], 1u); if (old == s + 1) Fn[atomicAdd(fncnt, 1u)] = e2; }
        }
    }
}

__global__ void iota_kernel(u32 *a, u64 m) {
    u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) a[i] = (u32)i;
}

__global__ void retire_frontier_kernel(const u32 *__restrict__ F, u32 nf, uint8_t *st) {
    u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nf) st[F[i]] = 2;
}

// ------------------------------------------------------------ persistent peel
// The whole level-synchronous peel in one cooperative launch (all blocks resident),
// rounds separated by a software grid barrier.  Data written by other blocks inside the
// launch is read with volatile loads (bypassing the non-coherent L1).
struct PeelState {
    u32 ctr[4];        // [0] alive after compaction, [1] frontier size, [2] least support, [3] unused
    u32 cnt[3];        // next-frontier sizes, rotating by round (round r writes cnt[r % 3])
    unsigned bar[2];   // barrier arrivals, generation
    unsigned status;   // KC_DEV_ERR_* bits
    u32 rounds;
};

// A wait longer than 2^35 SM cycles (~17 s) sets KC_DEV_ERR_TIMEOUT and returns.
__device__ __forceinline__ void grid_sync(PeelState *ps) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = &ps->bar[1];
        const unsigned gen = *vgen;
        __threadfence();
        if (atomicAdd(&ps->bar[0], 1u) == gridDim.x - 1) {
            atomicExch(&ps->bar[0], 0u);
            __threadfence();
            atomicAdd(&ps->bar[1], 1u);
        } else {
            const long long t0 = clock64();
            while (*vgen == gen) {
                if (clock64() - t0 > (1ll << 35)) {
                    atomicOr(&ps->status, KC_DEV_ERR_TIMEOUT);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
}

// Block 0 finishes the peel alone (block barriers instead of grid barriers: a sparse
// core's many small rounds are barrier-bound) once at most KC_PEEL_SOLO edges remain and
// (remaining edges) x (least support + 1), a bound from below on the triangle work left,
// is at most KC_PEEL_SOLO_WORK (a dense core's few big rounds need the whole grid).
#ifndef KC_PEEL_SOLO
#define KC_PEEL_SOLO (1u << 15)
#endif
#ifndef KC_PEEL_SOLO_WORK
#define KC_PEEL_SOLO_WORK (1ull << 18)
#endif

#ifndef KC_PEEL_SMALL  // graphs with at most this many triangle incidences are peeled by one block
#define KC_PEEL_SMALL (1ull << 18)
#endif

__device__ __forceinline__ u32 vld(const u32 *p) { return *(const volatile u32 *)p; }
__device__ __forceinline__ uint8_t vld8(const uint8_t *p) { return *(const volatile uint8_t *)p; }

// Rounds take two grid barriers: (A) retire the previous frontier, mark the current one
// and clear the counter of the round after next | barrier | (B) remove the current
// frontier's triangles, collecting the next frontier | barrier.  The frontier buffer of
// round r - 1 is retired in (A) of round r and is then free for round r's next frontier.
// The next-frontier counters rotate over three slots, so a slot is cleared two barriers
// after every thread last read it.
__global__ void __launch_bounds__(256) peel_persistent_kernel(u64 m, const u64 *__restrict__ inc_ptr,
                                                              const u64 *__restrict__ inc, u32 *sup, uint8_t *st,
                                                              u32 *level, u32 *round, u32 *alive, u32 *alive2,
                                                              u32 *F, u32 *Fn, PeelState *ps) {
    u64 tid = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    u64 nthr = (u64)gridDim.x * blockDim.x;
    u64 warp = tid >> 5, nwarps = nthr >> 5;
    const int lane = threadIdx.x & 31;
    bool solo = false;  // block 0 alone: block barriers
    auto sync = [&]() {
        if (solo) __syncthreads();
        else grid_sync(ps);
    };
    u32 lvl = 0, r = 0, nf = 0, nfp = 0;
    u32 *Fp = Fn;  // previous frontier (to retire); its buffer takes the next frontier
    u64 nalive = m;
    for (u64 i = tid; i < m; i += nthr) alive[i] = (u32)i;
    grid_sync(ps);
    while (!(*(volatile unsigned *)&ps->status & KC_DEV_ERR_TIMEOUT)) {
        if (nf == 0) {
            for (u64 i = tid; i < nfp; i += nthr) st[vld(&Fp[i])] = 2;
            nfp = 0;
            if (nalive == 0) break;
            if (tid == 0) { ps->ctr[0] = 0; ps->ctr[2] = 0xFFFFFFFFu; }
            sync();
            for (u64 i = tid; i < nalive; i += nthr) {
                const u32 e = vld(&alive[i]);
                if (vld8(&st[e]) == 2) continue;
                alive2[atomicAdd(&ps->ctr[0], 1u)] = e;
                atomicMin(&ps->ctr[2], vld(&sup[e]));
            }
            sync();
            nalive = vld(&ps->ctr[0]);
            const u32 minsup = vld(&ps->ctr[2]);
            u32 *t = alive; alive = alive2; alive2 = t;
            if (nalive == 0) break;
            if (minsup > lvl) lvl = minsup;
            sync();  // all have read ctr[0..2]
            if (!solo && nalive <= KC_PEEL_SOLO && nalive * (u64)(lvl + 1) <= KC_PEEL_SOLO_WORK) {
                // every block took the same decision from the same nalive; the others leave
                // and take no further part in any barrier
                if (blockIdx.x != 0) return;
                solo = true;
                tid = threadIdx.x;
                nthr = blockDim.x;
                warp = tid >> 5;
                nwarps = nthr >> 5;
            }
            if (tid == 0) ps->ctr[1] = 0;
            sync();
            for (u64 i = tid; i < nalive; i += nthr) {
                const u32 e = vld(&alive[i]);
                if (vld(&sup[e]) <= lvl) F[atomicAdd(&ps->ctr[1], 1u)] = e;
            }
            sync();
            nf = vld(&ps->ctr[1]);
            if (nf == 0) {  // cannot happen: the least support is <= lvl
                if (tid == 0) atomicOr(&ps->status, KC_DEV_ERR_BOUNDS);
                break;
            }
        }
        // (A)
        for (u64 i = tid; i < nfp; i += nthr) st[vld(&Fp[i])] = 2;
        for (u64 i = tid; i < nf; i += nthr) {
            const u32 e = vld(&F[i]);
            st[e] = 1;
            level[e] = lvl;
            round[e] = r;
        }
        if (tid == 0) ps->cnt[(r + 1) % 3] = 0;
        sync();
        // (B): the next frontier goes to Fp's buffer (retired above)
        u32 *const Fnext = Fp;
        u32 *const cnt = &ps->cnt[r % 3];
        for (u64 i = warp; i < nf; i += nwarps) {
            const u32 e = vld(&F[i]);
            for (u64 p = inc_ptr[e] + lane; p < inc_ptr[e + 1]; p += 32) {
                const u64 pr = inc[p];
                const u32 e1 = (u32)(pr >> 32), e2 = (u32)pr;
                const uint8_t s1 = vld8(&st[e1]), s2 = vld8(&st[e2]);
                if (s1 == 2 || s2 == 2) continue;                       // destroyed in an earlier round
                if ((s1 == 1 && e1 < e) || (s2 == 1 && e2 < e)) continue;  // another frontier edge owns it
                if (s1 == 0) { u32 old = atomicSub(&sup[e1], 1u); if (old == lvl + 1) Fnext[atomicAdd(cnt, 1u)] = e1; }
                if (s2 == 0) { u32 old = atomicSub(&sup[e2], 1u); if (old == lvl + 1) Fnext[atomicAdd(cnt, 1u)] = e2; }
            }
        }
        sync();
        nfp = nf;
        nf = vld(cnt);
        Fp = F;
        F = Fnext;
        r++;
    }
    if (tid == 0 && blockIdx.x == 0) ps->rounds = r;
}

// ------------------------------------------------------------ colour-based ordering
// EBBkC-C's top level (Sec. 4.3, Alg. 4): a greedy colouring of G, vertices in
// non-increasing colour (ties by id), each edge oriented to its later endpoint.  Greedy in
// the order of decreasing (degree, id) is computed in rounds (Jones-Plassmann): a vertex
// whose uncoloured neighbours all come later in that order takes the least colour none of
// its coloured neighbours has.  Two such vertices are never adjacent, so a round's
// readers never see a colour change, and the result is the sequential greedy colouring.
// One warp per vertex; colours are found 1024 at a time in a shared bitmap.
__device__ __forceinline__ bool colour_before(u32 du, u32 u, u32 dv, u32 v) {
    return du > dv || (du == dv && u < v);
}

__global__ void max_kernel(const u32 *__restrict__ a, u64 n, u32 *mx) {
    const u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicMax(mx, a[i]);
}

__global__ void colour_round_kernel(const u32 *__restrict__ rp, const u32 *__restrict__ col, u32 n, u32 *colour,
                                    u32 *left) {
    __shared__ u32 bm[TPB / 32][32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const u64 nwarps = ((u64)gridDim.x * blockDim.x) >> 5;
    for (u64 v64 = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v64 < n; v64 += nwarps) {
        const u32 v = (u32)v64;
        if (colour[v]) continue;
        const u32 b = rp[v], e = rp[v + 1], dv = e - b;
        bool ready = true;
        for (u32 i = b + lane; i < e && ready; i += 32) {
            const u32 u = col[i];
            if (!colour[u] && colour_before(rp[u + 1] - rp[u], u, dv, v)) ready = false;
        }
        ready = __all_sync(0xffffffffu, ready);
        if (!ready) {
            if (lane == 0) atomicAdd(left, 1u);
            continue;
        }
        for (u32 base = 1;; base += 1024) {  // colours [base, base + 1024)
            bm[wib][lane] = 0;
            __syncwarp();
            for (u32 i = b + lane; i < e; i += 32) {
                const u32 c = colour[col[i]];
                if (c >= base && c < base + 1024) atomicOr(&bm[wib][(c - base) >> 5], 1u << ((c - base) & 31));
            }
            __syncwarp();
            const u32 freew = ~bm[wib][lane];
            const unsigned bal = __ballot_sync(0xffffffffu, freew != 0);
            if (bal) {
                const int fl = __ffs(bal) - 1;
                const u32 wv = __shfl_sync(0xffffffffu, freew, fl);
                if (lane == 0) colour[v] = base + 32u * (u32)fl + (u32)(__ffs(wv) - 1);
                __syncwarp();
                break;
            }
            __syncwarp();
        }
    }
}

// the edge order of the colour-based DAG: rank(a, b) = the later endpoint's position in
// (colour descending, id ascending); ties between edges with the same later endpoint go
// by edge id.  VSet(e) is then the common out-neighbours of e's endpoints (Alg. 4) and
// every pair inside it comes after e.
__global__ void colour_rank_kernel(const u32 *__restrict__ eu, const u32 *__restrict__ ev, const u32 *__restrict__ colour,
                                   u32 cmax, u32 n, u64 m, u32 *round) {
    const u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const u32 a = eu[i], b = ev[i];
    const u64 pa = (u64)(cmax - colour[a]) * n + a, pb = (u64)(cmax - colour[b]) * n + b;
    round[i] = (u32)(pa > pb ? pa : pb);
}

// ------------------------------------------------------------ VSet
__device__ __forceinline__ bool key_less(u32 ra, u32 ea, u32 rb, u32 eb) { return ra < rb || (ra == rb && ea < eb); }

template <int MODE>
__global__ void vset_kernel(u64 m, const u64 *__restrict__ inc_ptr, const u64 *__restrict__ inc,
                            const u32 *__restrict__ round, const u32 *__restrict__ eu, const u32 *__restrict__ ev,
                            u32 *vcnt, const u64 *__restrict__ vptr, u32 *vset) {
    u64 warp = ((u64)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    u64 nwarps = ((u64)gridDim.x * blockDim.x) >> 5;
    for (u64 e = warp; e < m; e += nwarps) {
        u32 re = round[e], a = eu[e], b = ev[e];
        u64 out = MODE ? vptr[e] : 0;
        u32 c = 0;
        for (u64 p0 = inc_ptr[e]; p0 < inc_ptr[e + 1]; p0 += 32) {
            u64 p = p0 + lane;
            bool keep = false;
            u32 w = 0;
            if (p < inc_ptr[e + 1]) {
                u64 pr = inc[p];
                u32 e1 = (u32)(pr >> 32), e2 = (u32)pr;
                keep = key_less(re, (u32)e, round[e1], e1) && key_less(re, (u32)e, round[e2], e2);
                if (keep && MODE) { u32 x = eu[e1], y = ev[e1]; w = (x == a || x == b) ? y : x; }
            }
            unsigned bal = __ballot_sync(0xffffffffu, keep);
            if (MODE && keep) vset[out + __popc(bal & ((1u << lane) - 1))] = w;
            out += __popc(bal);
            c += __popc(bal);
        }
        if (!MODE && lane == 0) vcnt[e] = c;
    }
}

__global__ void pos_round_kernel(const u32 *__restrict__ pos_eid, const u32 *__restrict__ round, u64 nnz, u32 *pos_round) {
    u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nnz) pos_round[i] = round[pos_eid[i]];
}

// tickets: counting sort of edges by |VSet| descending
__global__ void size_hist_kernel(const u32 *__restrict__ vcnt, u64 m, u32 *hist, u32 *maxs) {
    u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    atomicAdd(&hist[vcnt[i]], 1u);
    atomicMax(maxs, vcnt[i]);
}

__global__ void ticket_scatter_kernel(const u32 *__restrict__ vcnt, u64 m, u64 *cursor, u32 *tickets) {
    u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    tickets[atomicAdd((unsigned long long *)&cursor[vcnt[i]], 1ull)] = (u32)i;
}

struct Scratch {
    std::vector<void *> ptrs;
    cudaStream_t s;
    ~Scratch() {
        for (void *p : ptrs) cudaFreeAsync(p, s);
    }
};

// scratch (scr != nullptr): stream-ordered allocation freed at the end of prepare;
// resident arrays of the handle (scr == nullptr): plain cudaMalloc, freed by release
template <typename T>
kc_status dalloc(T **p, u64 count, cudaStream_t s, Scratch *scr) {
    if (count == 0) count = 1;
    cudaError_t e = scr ? cudaMallocAsync((void **)p, sizeof(T) * count, s) : cudaMalloc((void **)p, sizeof(T) * count);
    if (e != cudaSuccess) {
        kc_set_last_cuda_error(e, scr ? "cudaMallocAsync" : "cudaMalloc", __FILE__, __LINE__);
        *p = nullptr;
        return e == cudaErrorMemoryAllocation ? KC_ERR_OOM : KC_ERR_CUDA;
    }
    if (scr) scr->ptrs.push_back(*p);
    return KC_OK;
}

#define KC_TRY(...)                    \
    do {                               \
        kc_status _st = (__VA_ARGS__); \
        if (_st != KC_OK) return _st;  \
    } while (0)

// warp-per-row kernels use this many threads
inline unsigned warp_grid(u64 rows) {
    u64 b = kc_div_up(rows * 32, TPB);
    if (b > 4u * 152u * 16u) b = 4u * 152u * 16u;
    if (b < 1) b = 1;
    return (unsigned)b;
}

}  // namespace

void kc_free_graph(kc_graph *g) {
    if (!g) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(g->device);
    void *ps[] = {g->row_ptr, g->col, g->pos_eid, g->pos_round, g->eu, g->ev, g->level, g->round,
                  g->vset_ptr, g->vset, g->tickets};
    for (void *p : ps)
        if (p) cudaFree(p);
    free(g->h_size_suffix);
    cudaSetDevice(cur);
    delete g;
}

static kc_status prepare_body(const u32 *row_ptr_in, const u32 *col_in, u32 n, u64 nnz, int on_device, u32 ordering,
                              cudaStream_t s, kc_graph *g) {
    Scratch scr;
    scr.s = s;
    // ---- input on the device
    const u32 *rp = row_ptr_in, *ci = col_in;
    if (!on_device) {
        u32 *d_rp, *d_ci;
        KC_TRY(dalloc(&d_rp, (u64)n + 1, s, &scr));
        KC_TRY(dalloc(&d_ci, nnz, s, &scr));
        KC_CUDA(cudaMemcpyAsync(d_rp, row_ptr_in, sizeof(u32) * ((u64)n + 1), cudaMemcpyHostToDevice, s));
        if (nnz) KC_CUDA(cudaMemcpyAsync(d_ci, col_in, sizeof(u32) * nnz, cudaMemcpyHostToDevice, s));
        rp = d_rp;
        ci = d_ci;
    }
    unsigned *d_flags;
    KC_TRY(dalloc(&d_flags, 4, s, &scr));
    KC_CUDA(cudaMemsetAsync(d_flags, 0, sizeof(unsigned) * 4, s));
    validate_kernel<<<grid_for(std::max<u64>(n, nnz)), TPB, 0, s>>>(rp, ci, n, nnz, d_flags);
    kc_note_launch();
    if (n) {
        clean_check_kernel<<<warp_grid(n), TPB, 0, s>>>(rp, ci, n, d_flags + 1);
        kc_note_launch();
    }
    unsigned h_flags[4];
    KC_CUDA(cudaMemcpyAsync(h_flags, d_flags, sizeof(h_flags), cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaStreamSynchronize(s));
    if (h_flags[0]) return KC_ERR_INVALID_GRAPH;

    // ---- A1: clean CSR
    u32 *row_ptr = nullptr, *col = nullptr;
    u64 nnz2 = 0;
    KC_TRY(dalloc(&row_ptr, (u64)n + 1, s, nullptr));
    g->row_ptr = row_ptr;
    if (!h_flags[1]) {
        nnz2 = nnz;
        KC_TRY(dalloc(&col, nnz2, s, nullptr));
        g->col = col;
        KC_CUDA(cudaMemcpyAsync(row_ptr, rp, sizeof(u32) * ((u64)n + 1), cudaMemcpyDeviceToDevice, s));
        if (nnz2) KC_CUDA(cudaMemcpyAsync(col, ci, sizeof(u32) * nnz2, cudaMemcpyDeviceToDevice, s));
    } else {
        u32 *cnt;
        u64 *tptr, *cursor;
        KC_TRY(dalloc(&cnt, (u64)n + 1, s, &scr));
        KC_TRY(dalloc(&tptr, (u64)n + 1, s, &scr));
        KC_TRY(dalloc(&cursor, (u64)n + 1, s, &scr));
        KC_CUDA(cudaMemsetAsync(cnt, 0, sizeof(u32) * ((u64)n + 1), s));
        sym_count_kernel<<<warp_grid(n), TPB, 0, s>>>(rp, ci, n, cnt);
        kc_note_launch();
        KC_TRY(scan_excl<u32, u64>(cnt, tptr, n, s));
        u64 tot = 0;
        KC_CUDA(cudaMemcpyAsync(&tot, tptr + n, sizeof(u64), cudaMemcpyDeviceToHost, s));
        KC_CUDA(cudaStreamSynchronize(s));
        u32 *tcol;
        KC_TRY(dalloc(&tcol, tot, s, &scr));
        KC_CUDA(cudaMemcpyAsync(cursor, tptr, sizeof(u64) * ((u64)n + 1), cudaMemcpyDeviceToDevice, s));
        sym_scatter_kernel<<<warp_grid(n), TPB, 0, s>>>(rp, ci, n, cursor, tcol);
        kc_note_launch();
        KC_TRY(sort_segments(tptr, tcol, n, s));
        dedupe_count_kernel<<<warp_grid(n), TPB, 0, s>>>(tptr, tcol, n, cnt);
        kc_note_launch();
        u64 *optr;
        KC_TRY(dalloc(&optr, (u64)n + 1, s, &scr));
        KC_TRY(scan_excl<u32, u64>(cnt, optr, n, s));
        KC_CUDA(cudaMemcpyAsync(&nnz2, optr + n, sizeof(u64), cudaMemcpyDeviceToHost, s));
        KC_CUDA(cudaStreamSynchronize(s));
        if (nnz2 >= (1ull << 32)) return KC_ERR_INVALID_GRAPH;
        KC_TRY(dalloc(&col, nnz2, s, nullptr));
        g->col = col;
        dedupe_write_kernel<<<warp_grid(n), TPB, 0, s>>>(tptr, tcol, n, optr, col);
        kc_note_launch();
        u64_to_u32_kernel<<<grid_for((u64)n + 1), TPB, 0, s>>>(optr, row_ptr, (u64)n + 1);
        kc_note_launch();
    }
    g->nnz = nnz2;
    u64 m = nnz2 / 2;
    g->m = m;

    // ---- A2: edge ids
    u32 *ucnt, *ustart, *d_maxdeg;
    u64 *eoff;
    KC_TRY(dalloc(&ucnt, (u64)n + 1, s, &scr));
    KC_TRY(dalloc(&ustart, (u64)n + 1, s, &scr));
    KC_TRY(dalloc(&eoff, (u64)n + 1, s, &scr));
    KC_TRY(dalloc(&d_maxdeg, 1, s, &scr));
    KC_CUDA(cudaMemsetAsync(d_maxdeg, 0, sizeof(u32), s));
    KC_TRY(dalloc(&g->pos_eid, nnz2, s, nullptr));
    KC_TRY(dalloc(&g->pos_round, nnz2, s, nullptr));
    KC_TRY(dalloc(&g->eu, m, s, nullptr));
    KC_TRY(dalloc(&g->ev, m, s, nullptr));
    KC_TRY(dalloc(&g->level, m, s, nullptr));
    KC_TRY(dalloc(&g->round, m, s, nullptr));
    KC_TRY(dalloc(&g->vset_ptr, m + 1, s, nullptr));
    KC_TRY(dalloc(&g->tickets, m, s, nullptr));
    if (n) {
        upper_count_kernel<<<grid_for(n), TPB, 0, s>>>(row_ptr, col, n, ucnt, ustart, d_maxdeg);
        kc_note_launch();
        KC_TRY(scan_excl<u32, u64>(ucnt, eoff, n, s));
        edge_ids_upper_kernel<<<warp_grid(n), TPB, 0, s>>>(row_ptr, col, n, ustart, eoff, g->pos_eid, g->eu, g->ev);
        kc_note_launch();
        edge_ids_lower_kernel<<<warp_grid(n), TPB, 0, s>>>(row_ptr, col, n, ustart, g->pos_eid);
        kc_note_launch();
    }
    KC_CUDA(cudaMemcpyAsync(&g->max_degree, d_maxdeg, sizeof(u32), cudaMemcpyDeviceToHost, s));

    // ---- A2: triangles on the degree orientation -> support and incidence lists
    u32 *ocnt, *ocol, *oeid, *sup;
    u64 *optr2;
    KC_TRY(dalloc(&ocnt, (u64)n + 1, s, &scr));
    KC_TRY(dalloc(&optr2, (u64)n + 1, s, &scr));
    KC_TRY(dalloc(&ocol, m, s, &scr));
    KC_TRY(dalloc(&oeid, m, s, &scr));
    KC_TRY(dalloc(&sup, m, s, &scr));
    KC_CUDA(cudaMemsetAsync(sup, 0, sizeof(u32) * (m ? m : 1), s));
    if (n) {
        orient_count_kernel<<<warp_grid(n), TPB, 0, s>>>(row_ptr, col, n, ocnt);
        kc_note_launch();
        KC_TRY(scan_excl<u32, u64>(ocnt, optr2, n, s));
        orient_write_kernel<<<warp_grid(n), TPB, 0, s>>>(row_ptr, col, g->pos_eid, n, optr2, ocol, oeid);
        kc_note_launch();
        triangles_kernel<0><<<warp_grid(n), TPB, 0, s>>>(row_ptr, col, n, optr2, ocol, oeid, sup, nullptr, nullptr);
        kc_note_launch();
    }
    u64 *inc_ptr, *cursor2;
    KC_TRY(dalloc(&inc_ptr, m + 1, s, &scr));
    KC_TRY(dalloc(&cursor2, m + 1, s, &scr));
    KC_TRY(scan_excl<u32, u64>(sup, inc_ptr, m, s));
    u64 ninc = 0;
    KC_CUDA(cudaMemcpyAsync(&ninc, inc_ptr + m, sizeof(u64), cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaStreamSynchronize(s));
    u64 *inc;
    KC_TRY(dalloc(&inc, ninc, s, &scr));
    KC_CUDA(cudaMemcpyAsync(cursor2, inc_ptr, sizeof(u64) * (m + 1), cudaMemcpyDeviceToDevice, s));
    if (n) {
        triangles_kernel<1><<<warp_grid(n), TPB, 0, s>>>(row_ptr, col, n, optr2, ocol, oeid, nullptr, cursor2, inc);
        kc_note_launch();
    }
    g->triangles = ninc / 3;

    // ---- A3: level-synchronous peel
    uint8_t *st;
    u32 *alive, *alive2, *F, *Fn, *ctr;
    KC_TRY(dalloc(&st, m, s, &scr));
    KC_TRY(dalloc(&alive, m, s, &scr));
    KC_TRY(dalloc(&alive2, m, s, &scr));
    KC_TRY(dalloc(&F, m, s, &scr));
    KC_TRY(dalloc(&Fn, m, s, &scr));
    KC_TRY(dalloc(&ctr, 4, s, &scr));
    KC_CUDA(cudaMemsetAsync(st, 0, m ? m : 1, s));
    // host copies of the counters: pageable (a pinned allocation per call would cost more
    // than the few 4-byte reads, and freeing it waits for the whole device)
    u32 h_ctr[4] = {0, 0, 0, 0};
    if (m) {
        iota_kernel<<<grid_for(m), TPB, 0, s>>>(alive, m);
        kc_note_launch();
    }
    // one cooperative persistent launch when the device supports it (host-driven rounds otherwise);
    // a graph with few edges and triangles is peeled by one block from the start, in an ordinary launch
    // that needs no co-resident grid, so it starts as soon as one SM has room
    bool peeled = false;
    if (m > 0 && m <= KC_PEEL_SOLO && ninc <= KC_PEEL_SMALL) {
        PeelState *ps;
        KC_TRY(dalloc(&ps, 1, s, &scr));
        KC_CUDA(cudaMemsetAsync(ps, 0, sizeof(PeelState), s));
        peel_persistent_kernel<<<1, 256, 0, s>>>(m, inc_ptr, inc, sup, st, g->level, g->round, alive, alive2, F, Fn,
                                                  ps);
        kc_note_launch();
        PeelState h;
        KC_CUDA(cudaMemcpyAsync(&h, ps, sizeof(PeelState), cudaMemcpyDeviceToHost, s));
        KC_CUDA(cudaStreamSynchronize(s));
        if (h.status & KC_DEV_ERR_TIMEOUT) return KC_ERR_TIMEOUT;
        if (h.status) return KC_ERR_CUDA;
        g->rounds = h.rounds;
        peeled = true;
    }
    if (!peeled) {
        int dev = 0, coop = 0, nsm = 0, per_sm = 0;
        KC_CUDA(cudaGetDevice(&dev));
        KC_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
        KC_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        KC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, peel_persistent_kernel, 256, 0));
        if (coop && per_sm > 0 && m > 0) {
            PeelState *ps;
            KC_TRY(dalloc(&ps, 1, s, &scr));
            KC_CUDA(cudaMemsetAsync(ps, 0, sizeof(PeelState), s));
            u32 *lvl_p = g->level, *rnd_p = g->round;
            const u64 *incp = inc_ptr, *incc = inc;
            void *kargs[] = {(void *)&m, (void *)&incp, (void *)&incc, (void *)&sup, (void *)&st, (void *)&lvl_p,
                             (void *)&rnd_p, (void *)&alive, (void *)&alive2, (void *)&F, (void *)&Fn, (void *)&ps};
            // few blocks: a round's work is small next to its two grid barriers, whose cost
            // grows with the number of arriving blocks
            const unsigned grid = (unsigned)std::min<u64>((u64)nsm * std::min(per_sm, 2), kc_div_up(m, 256));
            KC_CUDA(cudaLaunchCooperativeKernel((void *)peel_persistent_kernel, dim3(grid), dim3(256), kargs, 0, s));
            kc_note_launch();
            PeelState h;
            KC_CUDA(cudaMemcpyAsync(&h, ps, sizeof(PeelState), cudaMemcpyDeviceToHost, s));
            KC_CUDA(cudaStreamSynchronize(s));
            if (h.status & KC_DEV_ERR_TIMEOUT) return KC_ERR_TIMEOUT;
            if (h.status) return KC_ERR_CUDA;
            g->rounds = h.rounds;
            peeled = true;
        }
    }
    u64 nalive = peeled ? 0 : m;
    u32 lvl = 0, r = 0;
    u32 nf = 0;
    while (!peeled) {
        if (nf == 0) {
            if (nalive == 0) break;
            KC_CUDA(cudaMemsetAsync(ctr, 0, sizeof(u32) * 2, s));
            KC_CUDA(cudaMemsetAsync(ctr + 2, 0xFF, sizeof(u32), s));
            compact_alive_kernel<<<grid_for(nalive), TPB, 0, s>>>(alive, (u32)nalive, st, sup, alive2, ctr, ctr + 2);
            kc_note_launch();
            KC_CUDA(cudaMemcpyAsync(h_ctr, ctr, sizeof(u32) * 4, cudaMemcpyDeviceToHost, s));
            KC_CUDA(cudaStreamSynchronize(s));
            nalive = h_ctr[0];
            std::swap(alive, alive2);
            if (nalive == 0) break;
            if (h_ctr[2] > lvl) lvl = h_ctr[2];
            KC_CUDA(cudaMemsetAsync(ctr + 1, 0, sizeof(u32), s));
            frontier_from_alive_kernel<<<grid_for(nalive), TPB, 0, s>>>(alive, (u32)nalive, sup, lvl, F, ctr + 1);
            kc_note_launch();
            KC_CUDA(cudaMemcpyAsync(h_ctr + 1, ctr + 1, sizeof(u32), cudaMemcpyDeviceToHost, s));
            KC_CUDA(cudaStreamSynchronize(s));
            nf = h_ctr[1];
            if (nf == 0) return KC_ERR_CUDA;  // cannot happen: the least support is <= lvl
        }
        mark_frontier_kernel<<<grid_for(nf), TPB, 0, s>>>(F, nf, st, g->level, g->round, lvl, r);
        kc_note_launch();
        KC_CUDA(cudaMemsetAsync(ctr + 3, 0, sizeof(u32), s));
        peel_round_kernel<<<warp_grid(nf), TPB, 0, s>>>(F, nf, inc_ptr, inc, st, sup, lvl, Fn, ctr + 3);
        kc_note_launch();
        retire_frontier_kernel<<<grid_for(nf), TPB, 0, s>>>(F, nf, st);
        kc_note_launch();
        KC_CUDA(cudaMemcpyAsync(h_ctr + 3, ctr + 3, sizeof(u32), cudaMemcpyDeviceToHost, s));
        KC_CUDA(cudaStreamSynchronize(s));
        nf = h_ctr[3];
        std::swap(F, Fn);
        r++;
    }
    if (!peeled) g->rounds = r;

    // ---- EBBkC-C: the colour-based edge order replaces the truss-based one
    if (ordering == KC_ORDER_COLOUR && m) {
        u32 *colour, *left;
        KC_TRY(dalloc(&colour, (u64)n + 1, s, &scr));
        KC_TRY(dalloc(&left, 1, s, &scr));
        KC_CUDA(cudaMemsetAsync(colour, 0, sizeof(u32) * ((u64)n + 1), s));
        for (u64 rounds = 0;; rounds++) {
            if (rounds > (u64)n + 1) return KC_ERR_CUDA;  // cannot happen: one vertex colours per round at least
            KC_CUDA(cudaMemsetAsync(left, 0, sizeof(u32), s));
            colour_round_kernel<<<warp_grid(n), TPB, 0, s>>>(g->row_ptr, g->col, n, colour, left);
            kc_note_launch();
            KC_CUDA(cudaMemcpyAsync(h_ctr, left, sizeof(u32), cudaMemcpyDeviceToHost, s));
            KC_CUDA(cudaStreamSynchronize(s));
            if (h_ctr[0] == 0) break;
        }
        // the largest colour: positions (cmax - colour) * n + v must fit 32 bits
        u32 *d_cmax;
        KC_TRY(dalloc(&d_cmax, 1, s, &scr));
        KC_CUDA(cudaMemsetAsync(d_cmax, 0, sizeof(u32), s));
        max_kernel<<<grid_for(n), TPB, 0, s>>>(colour, n, d_cmax);
        kc_note_launch();
        u32 cmax = 0;
        KC_CUDA(cudaMemcpyAsync(&cmax, d_cmax, sizeof(u32), cudaMemcpyDeviceToHost, s));
        KC_CUDA(cudaStreamSynchronize(s));
        if ((u64)(cmax + 1) * n > 0xFFFFFFFFull) return KC_ERR_UNSUPPORTED;
        colour_rank_kernel<<<grid_for(m), TPB, 0, s>>>(g->eu, g->ev, colour, cmax, n, m, g->round);
        kc_note_launch();
    }

    // ---- A4: VSet
    u32 *vcnt;
    KC_TRY(dalloc(&vcnt, m + 1, s, &scr));
    if (m) {
        vset_kernel<0><<<warp_grid(m), TPB, 0, s>>>(m, inc_ptr, inc, g->round, g->eu, g->ev, vcnt, nullptr, nullptr);
        kc_note_launch();
    }
    KC_TRY(scan_excl<u32, u64>(vcnt, g->vset_ptr, m, s));
    u64 tv = 0;
    KC_CUDA(cudaMemcpyAsync(&tv, g->vset_ptr + m, sizeof(u64), cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaStreamSynchronize(s));
    if (tv != g->triangles) return KC_ERR_CUDA;  // every triangle has exactly one first edge
    KC_TRY(dalloc(&g->vset, tv, s, nullptr));
    if (m) {
        vset_kernel<1><<<warp_grid(m), TPB, 0, s>>>(m, inc_ptr, inc, g->round, g->eu, g->ev, nullptr, g->vset_ptr, g->vset);
        kc_note_launch();
        KC_TRY(sort_segments(g->vset_ptr, g->vset, m, s));
    }
    if (nnz2) {
        pos_round_kernel<<<grid_for(nnz2), TPB, 0, s>>>(g->pos_eid, g->round, nnz2, g->pos_round);
        kc_note_launch();
    }

    // ---- tickets by |VSet| descending
    u32 *hist, *d_maxs;
    KC_TRY(dalloc(&d_maxs, 1, s, &scr));
    KC_CUDA(cudaMemsetAsync(d_maxs, 0, sizeof(u32), s));
    // max |VSet| <= max support < max degree
    u64 hsz = (u64)g->max_degree + 2;
    KC_TRY(dalloc(&hist, hsz, s, &scr));
    KC_CUDA(cudaMemsetAsync(hist, 0, sizeof(u32) * hsz, s));
    if (m) {
        size_hist_kernel<<<grid_for(m), TPB, 0, s>>>(vcnt, m, hist, d_maxs);
        kc_note_launch();
    }
    KC_CUDA(cudaMemcpyAsync(&g->tau, d_maxs, sizeof(u32), cudaMemcpyDeviceToHost, s));
    std::vector<u32> h_hist(hsz);
    KC_CUDA(cudaMemcpyAsync(h_hist.data(), hist, sizeof(u32) * hsz, cudaMemcpyDeviceToHost, s));
    KC_CUDA(cudaStreamSynchronize(s));
    // descending offsets
    std::vector<u64> h_off(hsz, 0);
    u64 acc = 0;
    for (u64 sz = hsz; sz-- > 0;) { h_off[sz] = acc; acc += h_hist[sz]; }
    g->h_size_suffix = (u64 *)malloc(sizeof(u64) * ((u64)g->tau + 2));
    {
        u64 suf = 0;
        // h_size_suffix[x] = #edges with |VSet| >= x
        std::vector<u64> tmp((u64)g->tau + 2, 0);
        for (u64 sz = (u64)g->tau + 1; sz-- > 0;) { suf += h_hist[sz]; tmp[sz] = suf; }
        tmp[(u64)g->tau + 1] = 0;
        memcpy(g->h_size_suffix, tmp.data(), sizeof(u64) * ((u64)g->tau + 2));
    }
    u64 *tcur;
    KC_TRY(dalloc(&tcur, hsz, s, &scr));
    KC_CUDA(cudaMemcpyAsync(tcur, h_off.data(), sizeof(u64) * hsz, cudaMemcpyHostToDevice, s));
    if (m) {
        ticket_scatter_kernel<<<grid_for(m), TPB, 0, s>>>(vcnt, m, tcur, g->tickets);
        kc_note_launch();
    }
    KC_CUDA(cudaGetLastError());
    KC_CUDA(cudaStreamSynchronize(s));
    g->resident_bytes = sizeof(u32) * ((u64)n + 1) + sizeof(u32) * nnz2 * 3 + sizeof(u32) * m * 7 +
                        sizeof(u64) * (m + 1) + sizeof(u32) * tv;
    return KC_OK;
}

kc_status kc_prepare_impl(const u32 *row_ptr, const u32 *col, u32 n, u64 nnz, int on_device, u32 ordering, cudaStream_t s,
                          kc_graph **out) {
    if (!out || (!row_ptr) || (nnz && !col)) return KC_ERR_INVALID_ARG;
    *out = nullptr;
    if (nnz >= (1ull << 31)) return KC_ERR_INVALID_GRAPH;
    kc_graph *g = new kc_graph();
    memset(g, 0, sizeof(*g));
    cudaGetDevice(&g->device);
    g->n = n;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, s);
    kc_status st = prepare_body(row_ptr, col, n, nnz, on_device, ordering, s, g);
    cudaEventRecord(e1, s);
    cudaStreamSynchronize(s);
    if (st == KC_OK) {
        cudaError_t ce = cudaGetLastError();
        if (ce != cudaSuccess) {
            kc_set_last_cuda_error(ce, "prepare kernels", __FILE__, __LINE__);
            st = KC_ERR_CUDA;
        }
    }
    cudaEventElapsedTime(&g->ms_prepare, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != KC_OK) {
        kc_free_graph(g);
        return st;
    }
    *out = g;
    return KC_OK;
}
