/*
 * Plain CPU oracle for exact k-clique counting and listing.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark may call this library; the GPU product path never does,
 * and the two share no code.
 *
 * What it computes (paper, Sec. 2, Def. "k-clique" and Problem "k-clique
 * listing"): for a simple undirected graph G and k >= 3, the set Q_k of k-vertex
 * subsets whose pairs are all edges.  It reports
 *   count    = |Q_k| as an unsigned 128-bit integer;
 *   checksum = sum over Q in Q_k of prod_{v in Q} z(v)   (mod 2^64),
 *              z(v) = splitmix64(v) | 1, splitmix64 being the published SplitMix64
 *              output step (Steele, Lea & Flood, OOPSLA 2014): add the golden
 *              gamma 0x9E3779B97F4A7C15, then xor-shift 30 / multiply
 *              0xBF58476D1CE4E5B9 / xor-shift 27 / multiply 0x94D049BB133111EB /
 *              xor-shift 31.  The paper does not define a checksum; this one is
 *              order independent and odd per clique, so a lost or doubled clique
 *              always changes it.
 *
 * Method: a degeneracy-ordered vertex-branching lister (the VBBkC family of
 * Sec. 3, Alg. 1, with the l = 1 leaf), written independently of the GPU code:
 * order vertices by Batagelj-Zaversnik bucket peeling, orient every edge from
 * the earlier to the later vertex, and for each vertex u recurse on the local
 * bitset adjacency of its out-neighbourhood.  An optional exact shortcut (a
 * textbook identity, not the paper's t-plex machinery) closes a branch whose
 * candidate set is complete: C(|C|, l) cliques, checksum P * e_l(z_C).
 *
 * It also computes the edge quantities the GPU preprocessing must reproduce:
 *   - the truss levels by level-synchronous peeling (Sec. 4.2 "truss-based edge
 *     ordering", Eq. 6, read as: at level s remove, all at once, every remaining
 *     edge with at most s common neighbours among the remaining edges, repeat
 *     until none is left, then raise s to the least remaining support; edges
 *     removed together form one round, and the edge order is (round, edge id));
 *   - a textbook one-edge-at-a-time truss peel (a pin for the levels above);
 *   - VSet(e) sizes and, for chosen edges e, the (k-2)-cliques of the
 *     sub-branch g_e of Eq. 2 (edges of the suffix graph only).
 * Edge ids number the undirected edges (u < v) in lexicographic order.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;
typedef uint64_t u64;
typedef uint32_t u32;

static int cmp_u32(const void *x, const void *y) {
    u32 a = *(const u32 *)x, b = *(const u32 *)y;
    return a < b ? -1 : a > b;
}

/* ------------------------------------------------------------------ keys */
u64 oc_key(u64 v) {
    u64 x = v + 0x9E3779B97F4A7C15ULL;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ULL;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBULL;
    x = x ^ (x >> 31);
    return x | 1ULL;
}

/* --------------------------------------------------- saturating binomials */
#define OC_MAXN 4096
#define OC_MAXR 64
static const u128 OC_SAT = ~(u128)0;
static u128 *g_binom = NULL; /* (OC_MAXN+1) x (OC_MAXR+1), Pascal's rule */

static void init_binom(void) {
    if (g_binom) return;
    u128 *b = (u128 *)calloc((size_t)(OC_MAXN + 1) * (OC_MAXR + 1), sizeof(u128));
    for (int n = 0; n <= OC_MAXN; n++) {
        b[(size_t)n * (OC_MAXR + 1)] = 1;
        for (int r = 1; r <= OC_MAXR && r <= n; r++) {
            u128 a = b[(size_t)(n - 1) * (OC_MAXR + 1) + r - 1];
            u128 c = (r <= n - 1) ? b[(size_t)(n - 1) * (OC_MAXR + 1) + r] : 0;
            u128 s = a + c;
            b[(size_t)n * (OC_MAXR + 1) + r] = (a == OC_SAT || c == OC_SAT || s < a) ? OC_SAT : s;
        }
    }
    g_binom = b;
}

static u128 binom(int n, int r) {
    if (r < 0 || r > n) return 0;
    return g_binom[(size_t)n * (OC_MAXR + 1) + r];
}

/* ------------------------------------------------------ per-thread state */
typedef struct {
    u128 count;
    u64 checksum;
    u64 nodes;
    int overflow;
    /* listing */
    u32 *out;
    u64 cap;
    u64 written;
    int k;
    u32 S[64];
    int depth;
} acc_t;

static void acc_add(acc_t *a, u128 c) {
    if (c == OC_SAT) { a->overflow = 1; return; }
    u128 s = a->count + c;
    if (s < a->count) a->overflow = 1;
    a->count = s;
}

/* ---------------------------------------------------- branch over bitsets */
typedef struct {
    int d;           /* local vertices */
    int W;           /* 64-bit words per row */
    const u64 *adj;  /* d x W: bit j of row i set iff j > i and (i, j) is an edge */
    const u64 *z;    /* key of each local vertex */
    const u32 *vid;  /* original id of each local vertex */
    int shortcut;
    int want_checksum;
    u64 *stack;      /* (levels) x W scratch */
} branch_t;

static int popc_set(const u64 *C, int W) {
    int c = 0;
    for (int w = 0; w < W; w++) c += __builtin_popcountll(C[w]);
    return c;
}

static void emit(acc_t *a, const u32 *extra, int ne) {
    if (!a->out) return;
    if (a->written >= a->cap) { a->written++; return; }
    u32 q[64];
    int t = 0;
    for (int i = 0; i < a->depth; i++) q[t++] = a->S[i];
    for (int i = 0; i < ne; i++) q[t++] = extra[i];
    /* insertion sort: rows are stored ascending */
    for (int i = 1; i < t; i++) {
        u32 x = q[i];
        int j = i - 1;
        while (j >= 0 && q[j] > x) { q[j + 1] = q[j]; j--; }
        q[j + 1] = x;
    }
    memcpy(a->out + a->written * (u64)a->k, q, sizeof(u32) * (size_t)t);
    a->written++;
}

/* is every pair of C adjacent?  (rows hold only later neighbours) */
static int is_complete(const branch_t *b, const u64 *C) {
    int W = b->W;
    int remaining = popc_set(C, W);
    for (int w = 0; w < W; w++) {
        u64 x = C[w];
        while (x) {
            int i = w * 64 + __builtin_ctzll(x);
            x &= x - 1;
            remaining--;
            int c = 0;
            const u64 *row = b->adj + (size_t)i * W;
            for (int t = 0; t < W; t++) c += __builtin_popcountll(row[t] & C[t]);
            if (c != remaining) return 0;
        }
    }
    return 1;
}

static void rec(const branch_t *b, acc_t *a, const u64 *C, int l, u64 P, int lvl) {
    int W = b->W;
    a->nodes++;
    int cnt = popc_set(C, W);
    if (cnt < l) return;
    if (l == 1) {
        acc_add(a, (u128)cnt);
        if (b->want_checksum || a->out) {
            u64 s = 0;
            for (int w = 0; w < W; w++) {
                u64 x = C[w];
                while (x) {
                    int i = w * 64 + __builtin_ctzll(x);
                    x &= x - 1;
                    s += b->z[i];
                    if (a->out) emit(a, &b->vid[i], 1);
                }
            }
            a->checksum += P * s;
        }
        return;
    }
    if (b->shortcut && !a->out && cnt <= OC_MAXN && l <= OC_MAXR && is_complete(b, C)) {
        acc_add(a, binom(cnt, l));
        if (b->want_checksum) {
            u64 e[OC_MAXR + 1];
            memset(e, 0, sizeof(e));
            e[0] = 1;
            for (int w = 0; w < W; w++) {
                u64 x = C[w];
                while (x) {
                    int i = w * 64 + __builtin_ctzll(x);
                    x &= x - 1;
                    for (int j = l; j >= 1; j--) e[j] += e[j - 1] * b->z[i];
                }
            }
            a->checksum += P * e[l];
        }
        return;
    }
    u64 *Cn = b->stack + (size_t)lvl * W;
    for (int w = 0; w < W; w++) {
        u64 x = C[w];
        while (x) {
            int i = w * 64 + __builtin_ctzll(x);
            x &= x - 1;
            const u64 *row = b->adj + (size_t)i * W;
            for (int t = 0; t < W; t++) Cn[t] = C[t] & row[t];
            if (a->out) a->S[a->depth++] = b->vid[i];
            rec(b, a, Cn, l - 1, P * b->z[i], lvl + 1);
            if (a->out) a->depth--;
        }
    }
}

/* ----------------------------------------------------- degeneracy order */
/* Batagelj-Zaversnik O(m) core ordering; returns order[] and pos[]. */
static void degeneracy_order(u32 n, const u64 *rp, const u32 *col, u32 *order, u32 *pos, u32 *degen) {
    u32 *deg = (u32 *)malloc(sizeof(u32) * (n + 1));
    u32 md = 0;
    for (u32 v = 0; v < n; v++) {
        deg[v] = (u32)(rp[v + 1] - rp[v]);
        if (deg[v] > md) md = deg[v];
    }
    u32 *bin = (u32 *)calloc(md + 2, sizeof(u32));
    for (u32 v = 0; v < n; v++) bin[deg[v]]++;
    u32 start = 0;
    for (u32 d = 0; d <= md; d++) { u32 c = bin[d]; bin[d] = start; start += c; }
    for (u32 v = 0; v < n; v++) { pos[v] = bin[deg[v]]; order[pos[v]] = v; bin[deg[v]]++; }
    for (u32 d = md + 1; d >= 1; d--) bin[d] = bin[d - 1];
    bin[0] = 0;
    u32 dg = 0;
    for (u32 i = 0; i < n; i++) {
        u32 v = order[i];
        if (deg[v] > dg) dg = deg[v];
        for (u64 p = rp[v]; p < rp[v + 1]; p++) {
            u32 u = col[p];
            if (deg[u] > deg[v]) {
                u32 du = deg[u], pu = pos[u], pw = bin[du], w = order[pw];
                if (u != w) { pos[u] = pw; order[pu] = w; pos[w] = pu; order[pw] = u; }
                bin[du]++;
                deg[u]--;
            }
        }
    }
    *degen = dg;
    free(deg);
    free(bin);
}

/* ------------------------------------------------------- whole-graph run */
/*
 * Count (and optionally list) the k-cliques of a clean symmetric CSR.
 * tops/ntops: if tops != NULL, only the branches of those top vertices are run
 * (a bounded sample for timing); otherwise all vertices.
 * Returns 0, or 1 if the count overflowed 2^128.
 */
int oc_count(u32 n, const u64 *rp, const u32 *col, int k, int shortcut, int want_checksum,
             int threads, const u32 *tops, u64 ntops,
             u64 *count_lo, u64 *count_hi, u64 *checksum, u64 *nodes, u32 *degen_out,
             u32 *out, u64 cap, u64 *written) {
    init_binom();
    if (k < 1 || k > 64) return 2;
    u32 *order = (u32 *)malloc(sizeof(u32) * (n ? n : 1));
    u32 *pos = (u32 *)malloc(sizeof(u32) * (n ? n : 1));
    u32 degen = 0;
    degeneracy_order(n, rp, col, order, pos, &degen);
    if (degen_out) *degen_out = degen;
    /* out-lists sorted by position */
    u64 *orp = (u64 *)calloc((size_t)n + 1, sizeof(u64));
    for (u32 u = 0; u < n; u++) {
        u64 c = 0;
        for (u64 p = rp[u]; p < rp[u + 1]; p++) c += pos[col[p]] > pos[u];
        orp[u + 1] = orp[u] + c;
    }
    u32 *ocol = (u32 *)malloc(sizeof(u32) * (orp[n] ? orp[n] : 1));
    for (u32 u = 0; u < n; u++) {
        u64 t = orp[u];
        for (u64 p = rp[u]; p < rp[u + 1]; p++)
            if (pos[col[p]] > pos[u]) ocol[t++] = col[p];
        /* sort by position (insertion sort on small lists, fine for an oracle) */
        for (u64 i = orp[u] + 1; i < orp[u + 1]; i++) {
            u32 x = ocol[i];
            u64 j = i;
            while (j > orp[u] && pos[ocol[j - 1]] > pos[x]) { ocol[j] = ocol[j - 1]; j--; }
            ocol[j] = x;
        }
    }
    u128 total = 0;
    u64 csum = 0, tnodes = 0, twritten = 0;
    int overflow = 0;
    u64 nt = tops ? ntops : n;
    if (threads <= 0) threads = 1;
    if (out) threads = 1; /* listing is sequential: rows in a deterministic order */
#pragma omp parallel num_threads(threads)
    {
        acc_t a;
        memset(&a, 0, sizeof(a));
        a.k = k;
        if (out) { a.out = out; a.cap = cap; }
        int32_t *loc = (int32_t *)malloc(sizeof(int32_t) * (n ? n : 1));
        memset(loc, 0, sizeof(int32_t) * (n ? n : 1));
        u64 *adj = NULL, *zz = NULL, *stk = NULL;
        u32 *vid = NULL;
        size_t adj_cap = 0, v_cap = 0;
#pragma omp for schedule(dynamic, 16)
        for (u64 ti = 0; ti < nt; ti++) {
            u32 u = tops ? tops[ti] : (u32)ti;
            int d = (int)(orp[u + 1] - orp[u]);
            if (d < k - 1) continue;
            int W = (d + 63) / 64;
            if ((size_t)d * W > adj_cap) {
                adj_cap = (size_t)d * W;
                adj = (u64 *)realloc(adj, sizeof(u64) * adj_cap);
            }
            if ((size_t)d > v_cap) {
                v_cap = d;
                zz = (u64 *)realloc(zz, sizeof(u64) * v_cap);
                vid = (u32 *)realloc(vid, sizeof(u32) * v_cap);
            }
            stk = (u64 *)realloc(stk, sizeof(u64) * (size_t)(k + 2) * W);
            memset(adj, 0, sizeof(u64) * (size_t)d * W);
            for (int i = 0; i < d; i++) {
                u32 x = ocol[orp[u] + i];
                loc[x] = i + 1;
                zz[i] = oc_key(x);
                vid[i] = x;
            }
            for (int i = 0; i < d; i++) {
                u32 x = vid[i];
                for (u64 p = orp[x]; p < orp[x + 1]; p++) {
                    int j = loc[ocol[p]];
                    if (j) { j--; adj[(size_t)i * W + j / 64] |= 1ULL << (j % 64); }
                }
            }
            branch_t b = {d, W, adj, zz, vid, shortcut, want_checksum, stk};
            u64 *C = (u64 *)calloc(W, sizeof(u64));
            for (int i = 0; i < d; i++) C[i / 64] |= 1ULL << (i % 64);
            if (out) a.S[a.depth++] = u;
            if (k == 1) {
                acc_add(&a, 1);
                a.checksum += oc_key(u);
            } else {
                rec(&b, &a, C, k - 1, oc_key(u), 0);
            }
            if (out) a.depth--;
            free(C);
            for (int i = 0; i < d; i++) loc[vid[i]] = 0;
        }
#pragma omp critical
        {
            u128 s = total + a.count;
            if (s < total || a.overflow) overflow = 1;
            total = s;
            csum += a.checksum;
            tnodes += a.nodes;
            twritten += a.written;
        }
        free(loc); free(adj); free(zz); free(vid); free(stk);
    }
    *count_lo = (u64)total;
    *count_hi = (u64)(total >> 64);
    *checksum = csum;
    if (nodes) *nodes = tnodes;
    if (written) *written = twritten;
    free(order); free(pos); free(orp); free(ocol);
    return overflow ? 1 : 0;
}

/* ------------------------------------------------------------ edge ids */
/* eid_of_pos[p] for every CSR slot; eu/ev endpoints (u < v) of each edge. */
static void edge_ids(u32 n, const u64 *rp, const u32 *col, u32 *eid_of_pos, u32 *eu, u32 *ev) {
    u64 e = 0;
    for (u32 u = 0; u < n; u++)
        for (u64 p = rp[u]; p < rp[u + 1]; p++)
            if (col[p] > u) { eid_of_pos[p] = (u32)e; eu[e] = u; ev[e] = col[p]; e++; }
    for (u32 u = 0; u < n; u++)
        for (u64 p = rp[u]; p < rp[u + 1]; p++)
            if (col[p] < u) {
                u32 v = col[p]; /* find u in row v by binary search */
                u64 lo = rp[v], hi = rp[v + 1];
                while (lo < hi) { u64 mid = (lo + hi) / 2; if (col[mid] < u) lo = mid + 1; else hi = mid; }
                eid_of_pos[p] = eid_of_pos[lo];
            }
}

/* position of x in row v, or ~0 */
static u64 find_pos(const u64 *rp, const u32 *col, u32 v, u32 x) {
    u64 lo = rp[v], hi = rp[v + 1];
    while (lo < hi) { u64 mid = (lo + hi) / 2; if (col[mid] < x) lo = mid + 1; else hi = mid; }
    return (lo < rp[v + 1] && col[lo] == x) ? lo : ~0ULL;
}

/* For edge (u,v): call f on every common neighbour w with the ids of (u,w), (v,w).
 * Scans the shorter row and binary-searches the longer one. */
#define FOR_TRIANGLES(u, v, ...)                                                        \
    do {                                                                                 \
        u32 _a = (u), _b = (v);                                                          \
        if (rp[_a + 1] - rp[_a] > rp[_b + 1] - rp[_b]) { u32 _t = _a; _a = _b; _b = _t; } \
        for (u64 _p = rp[_a]; _p < rp[_a + 1]; _p++) {                                   \
            u32 w = col[_p];                                                             \
            u64 _q = find_pos(rp, col, _b, w);                                           \
            if (_q == ~0ULL) continue;                                                   \
            u32 ea = eid_of_pos[_p], eb = eid_of_pos[_q];                                \
            __VA_ARGS__                                                                  \
        }                                                                                \
    } while (0)

/* --------------------------------------------- level-synchronous truss peel */
/* level[e], round[e] for every edge; returns the number of rounds. */
u64 oc_truss_peel(u32 n, const u64 *rp, const u32 *col, u64 m, u32 *level, u32 *round_out) {
    u32 *eid_of_pos = (u32 *)malloc(sizeof(u32) * (rp[n] ? rp[n] : 1));
    u32 *eu = (u32 *)malloc(sizeof(u32) * (m ? m : 1));
    u32 *ev = (u32 *)malloc(sizeof(u32) * (m ? m : 1));
    edge_ids(n, rp, col, eid_of_pos, eu, ev);
    u32 *sup = (u32 *)calloc(m ? m : 1, sizeof(u32));
    /* state: 0 alive, 1 in current frontier, 2 removed */
    uint8_t *st = (uint8_t *)calloc(m ? m : 1, 1);
    uint8_t *mark = (uint8_t *)calloc(m ? m : 1, 1);
#pragma omp parallel for schedule(dynamic, 1024)
    for (u64 e = 0; e < m; e++) {
        u32 c = 0;
        FOR_TRIANGLES(eu[e], ev[e], { (void)ea; (void)eb; (void)w; c++; });
        sup[e] = c;
    }
    u32 *F = (u32 *)malloc(sizeof(u32) * (m ? m : 1));
    u32 *Fn = (u32 *)malloc(sizeof(u32) * (m ? m : 1));
    u32 *alive = (u32 *)malloc(sizeof(u32) * (m ? m : 1));
    u64 nalive = m;
    for (u64 e = 0; e < m; e++) alive[e] = (u32)e;
    u32 s = 0;
    u64 r = 0;
    while (nalive > 0) {
        /* compact the alive list and find the frontier of this level */
        u64 na = 0, nf = 0;
        u32 minsup = 0xFFFFFFFFu;
        for (u64 i = 0; i < nalive; i++) {
            u32 e = alive[i];
            if (st[e] == 2) continue;
            alive[na++] = e;
            if (sup[e] < minsup) minsup = sup[e];
        }
        nalive = na;
        if (!nalive) break;
        if (minsup > s) s = minsup;
        for (u64 i = 0; i < nalive; i++)
            if (sup[alive[i]] <= s) F[nf++] = alive[i];
        while (nf > 0) {
            for (u64 i = 0; i < nf; i++) { st[F[i]] = 1; level[F[i]] = s; round_out[F[i]] = (u32)r; }
            u64 nn = 0;
            for (u64 i = 0; i < nf; i++) {
                u32 e = F[i];
                FOR_TRIANGLES(eu[e], ev[e], {
                    (void)w;
                    if (st[ea] == 2 || st[eb] == 2) continue; /* destroyed in an earlier round */
                    /* the frontier edge with the smallest id among this triangle's
                       frontier edges performs the decrements */
                    if (st[ea] == 1 && ea < e) continue;
                    if (st[eb] == 1 && eb < e) continue;
                    if (st[ea] == 0) { sup[ea]--; if (sup[ea] <= s && !mark[ea]) { mark[ea] = 1; Fn[nn++] = ea; } }
                    if (st[eb] == 0) { sup[eb]--; if (sup[eb] <= s && !mark[eb]) { mark[eb] = 1; Fn[nn++] = eb; } }
                });
            }
            for (u64 i = 0; i < nf; i++) st[F[i]] = 2;
            r++;
            /* next frontier, in edge-id order */
            for (u64 i = 0; i < nn; i++) mark[Fn[i]] = 0;
            /* sort Fn ascending (counting-free insertion would be slow; use qsort) */
            qsort(Fn, nn, sizeof(u32), cmp_u32);
            u32 *t = F; F = Fn; Fn = t;
            nf = nn;
        }
    }
    free(eid_of_pos); free(eu); free(ev); free(sup); free(st); free(mark);
    free(F); free(Fn); free(alive);
    return r;
}


/* --------------------------------------- textbook sequential truss peel */
/* One edge at a time, always an edge of least current support; level[e] is the
 * running maximum of the support at removal (= trussness - 2). */
void oc_truss_sequential(u32 n, const u64 *rp, const u32 *col, u64 m, u32 *level) {
    u32 *eid_of_pos = (u32 *)malloc(sizeof(u32) * (rp[n] ? rp[n] : 1));
    u32 *eu = (u32 *)malloc(sizeof(u32) * (m ? m : 1));
    u32 *ev = (u32 *)malloc(sizeof(u32) * (m ? m : 1));
    edge_ids(n, rp, col, eid_of_pos, eu, ev);
    u32 *sup = (u32 *)calloc(m ? m : 1, sizeof(u32));
    uint8_t *gone = (uint8_t *)calloc(m ? m : 1, 1);
    u32 maxs = 0;
    for (u64 e = 0; e < m; e++) {
        u32 c = 0;
        FOR_TRIANGLES(eu[e], ev[e], { (void)ea; (void)eb; (void)w; c++; });
        sup[e] = c;
        if (c > maxs) maxs = c;
    }
    /* bucket queue keyed by support */
    u32 *bin = (u32 *)calloc(maxs + 2, sizeof(u32));
    u32 *order = (u32 *)malloc(sizeof(u32) * (m ? m : 1));
    u32 *pos = (u32 *)malloc(sizeof(u32) * (m ? m : 1));
    for (u64 e = 0; e < m; e++) bin[sup[e]]++;
    u32 start = 0;
    for (u32 d = 0; d <= maxs; d++) { u32 c = bin[d]; bin[d] = start; start += c; }
    for (u64 e = 0; e < m; e++) { pos[e] = bin[sup[e]]; order[pos[e]] = (u32)e; bin[sup[e]]++; }
    for (u32 d = maxs + 1; d >= 1; d--) bin[d] = bin[d - 1];
    bin[0] = 0;
    u32 cur = 0;
    for (u64 i = 0; i < m; i++) {
        u32 e = order[i];
        if (sup[e] > cur) cur = sup[e];
        level[e] = cur;
        gone[e] = 1;
        FOR_TRIANGLES(eu[e], ev[e], {
            (void)w;
            if (gone[ea] || gone[eb]) continue;
            u32 ed[2] = {ea, eb};
            for (int t = 0; t < 2; t++) {
                u32 f = ed[t];
                if (sup[f] > sup[e]) { /* move f one bucket down */
                    u32 df = sup[f], pf = pos[f], pw = bin[df], g = order[pw];
                    if (f != g) { pos[f] = pw; order[pf] = g; pos[g] = pf; order[pw] = f; }
                    bin[df]++;
                    sup[f]--;
                }
            }
        });
    }
    free(eid_of_pos); free(eu); free(ev); free(sup); free(gone); free(bin); free(order); free(pos);
}

/* ------------------------------------------------ per-edge sub-branches */
/* For every edge: |VSet(e)| = #common neighbours w with both (u,w) and (v,w)
 * after e in the (round, id) order (Eq. 2 with the suffix graph). */
void oc_vset_sizes(u32 n, const u64 *rp, const u32 *col, u64 m, const u32 *round_of, u32 *sizes) {
    u32 *eid_of_pos = (u32 *)malloc(sizeof(u32) * (rp[n] ? rp[n] : 1));
    u32 *eu = (u32 *)malloc(sizeof(u32) * (m ? m : 1));
    u32 *ev = (u32 *)malloc(sizeof(u32) * (m ? m : 1));
    edge_ids(n, rp, col, eid_of_pos, eu, ev);
#pragma omp parallel for schedule(dynamic, 1024)
    for (u64 e = 0; e < m; e++) {
        u32 c = 0;
        FOR_TRIANGLES(eu[e], ev[e], {
            (void)w;
            int after_a = round_of[ea] > round_of[e] || (round_of[ea] == round_of[e] && ea > e);
            int after_b = round_of[eb] > round_of[e] || (round_of[eb] == round_of[e] && eb > e);
            c += after_a && after_b;
        });
        sizes[e] = c;
    }
    free(eid_of_pos); free(eu); free(ev);
}

/* For each chosen edge e: the (k-2)-cliques of g_e (Eq. 2), i.e. the k-cliques
 * whose first edge in the (round, id) order is e; count and checksum (which
 * includes z(u) z(v)).  Returns 0, or 1 on overflow. */
int oc_edge_counts(u32 n, const u64 *rp, const u32 *col, u64 m, const u32 *round_of, int k,
                   const u32 *edges, u64 ne, int shortcut, int threads,
                   u64 *cnt_lo, u64 *cnt_hi, u64 *csum) {
    init_binom();
    u32 *eid_of_pos = (u32 *)malloc(sizeof(u32) * (rp[n] ? rp[n] : 1));
    u32 *eu = (u32 *)malloc(sizeof(u32) * (m ? m : 1));
    u32 *ev = (u32 *)malloc(sizeof(u32) * (m ? m : 1));
    edge_ids(n, rp, col, eid_of_pos, eu, ev);
    int overflow = 0;
    if (threads <= 0) threads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads)
    for (u64 i = 0; i < ne; i++) {
        u32 e = edges[i];
        u32 u = eu[e], v = ev[e];
#define AFTER(f) (round_of[f] > round_of[e] || (round_of[f] == round_of[e] && (f) > e))
        /* VSet(e), ascending ids */
        u32 *vs = NULL;
        int d = 0, capd = 0;
        FOR_TRIANGLES(u, v, {
            if (AFTER(ea) && AFTER(eb)) {
                if (d == capd) { capd = capd ? 2 * capd : 64; vs = (u32 *)realloc(vs, sizeof(u32) * capd); }
                vs[d++] = w;
            }
        });
        /* sort ascending */
        qsort(vs, d, sizeof(u32), cmp_u32);
        acc_t a;
        memset(&a, 0, sizeof(a));
        int l = k - 2;
        if (l <= 0) {
            acc_add(&a, 1);
            a.checksum = oc_key(u) * oc_key(v);
        } else if (d >= l) {
            int W = (d + 63) / 64;
            u64 *adj = (u64 *)calloc((size_t)d * W, sizeof(u64));
            u64 *zz = (u64 *)malloc(sizeof(u64) * d);
            u64 *stk = (u64 *)malloc(sizeof(u64) * (size_t)(k + 2) * W);
            u64 *C = (u64 *)calloc(W, sizeof(u64));
            for (int x = 0; x < d; x++) { zz[x] = oc_key(vs[x]); C[x / 64] |= 1ULL << (x % 64); }
            for (int x = 0; x < d; x++)
                for (int y = x + 1; y < d; y++) {
                    u64 q = find_pos(rp, col, vs[x], vs[y]);
                    if (q == ~0ULL) continue;
                    u32 f = eid_of_pos[q];
                    if (AFTER(f)) adj[(size_t)x * W + y / 64] |= 1ULL << (y % 64);
                }
            branch_t b = {d, W, adj, zz, vs, shortcut, 1, stk};
            rec(&b, &a, C, l, oc_key(u) * oc_key(v), 0);
            free(adj); free(zz); free(stk); free(C);
        }
#undef AFTER
        cnt_lo[i] = (u64)a.count;
        cnt_hi[i] = (u64)(a.count >> 64);
        csum[i] = a.checksum;
        if (a.overflow) overflow = 1;
        free(vs);
    }
    free(eid_of_pos); free(eu); free(ev);
    return overflow;
}
