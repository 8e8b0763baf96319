"""Seeded synthetic graph generators shared by the oracle tests, the GPU tests and the bench.

This module holds no k-clique arithmetic: it only draws graphs.  Every random
number comes from a counter-based generator (the SplitMix64 output function of
Steele, Lea & Flood, OOPSLA 2014, applied to a (seed, stream, index) counter),
and every floating-point step uses only IEEE basic operations (+ - * / and
frexp/ldexp), so the same seed yields the same graph bit for bit on x86 and on
Arm, whatever the numpy version.  ``ln`` and ``exp`` below are series written
here for that reason (libm and numpy's SIMD kernels may differ by an ulp
between machines).

Graphs are returned as :class:`Graph` -- a symmetric, sorted, duplicate-free,
loop-free CSR of uint32 (``row_ptr[n+1]``, ``col[2m]``) -- the input form the
paper assumes after dropping directions and self-loops (Sec. 6.1, "Datasets").

Workload shapes (the paper's real graphs are not available; these stand in):
  * ``gnp``          Erdos-Renyi G(n, p) by geometric skipping over pair indices.
  * ``chung_lu``     power-law expected-degree graph (p_ij = min(1, w_i w_j / S)),
                     Miller-Hagberg skipping, plus planted cliques and a relabel.
  * ``sbm_2plex``    stochastic block model with dense blocks, some of them exact
                     2-plexes (K_b minus a matching), plus sparse inter-block edges.
  * ``batch_specs``  the parameters of a batch of many small uneven graphs.
  * small fixtures  complete, complete multipartite (Turan), 2-plex, t-plex,
                     complete bipartite, the 4-vertex example of Appendix B.
"""
from __future__ import annotations

import hashlib
import math
from dataclasses import dataclass

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GOLD = np.uint64(0x9E3779B97F4A7C15)
_C1 = np.uint64(0xBF58476D1CE4E5B9)
_C2 = np.uint64(0x94D049BB133111EB)
_LN2 = 0.6931471805599453


# --------------------------------------------------------------------------- RNG
def _mix(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (xor-shift / multiply finaliser), wrapping uint64."""
    x = x.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        x ^= x >> np.uint64(30)
        x *= _C1
        x ^= x >> np.uint64(27)
        x *= _C2
        x ^= x >> np.uint64(31)
    return x


def rand_u64(seed: int, stream, idx) -> np.ndarray:
    """Counter-based uint64 draws: one independent value per (seed, stream, idx)."""
    stream = np.asarray(stream, dtype=np.uint64)
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        key = _mix(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * _GOLD + np.uint64(0x632BE59BD9B4E019))
        s = _mix(key ^ (stream * _GOLD + _GOLD))
        return _mix(s + (idx + np.uint64(1)) * _GOLD)


def rand_unit(seed: int, stream, idx) -> np.ndarray:
    """Uniform doubles strictly inside (0, 1): (top 53 bits + 1/2) * 2^-53."""
    x = rand_u64(seed, stream, idx) >> np.uint64(11)
    return (x.astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def rand_int(seed: int, stream, idx, lo: int, hi: int) -> np.ndarray:
    """Integers uniform in [lo, hi] (inclusive) by multiply-shift on 32 random bits."""
    span = np.uint64(hi - lo + 1)
    x = rand_u64(seed, stream, idx) >> np.uint64(32)
    return (lo + ((x * span) >> np.uint64(32))).astype(np.int64)


# ------------------------------------------------- deterministic elementary math
def ln(x) -> np.ndarray:
    """Natural log from frexp and the atanh series (IEEE basic operations only)."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)
    small = m < 0.7071067811865476
    m = np.where(small, m * 2.0, m)
    e = np.where(small, e - 1, e).astype(np.float64)
    t = (m - 1.0) / (m + 1.0)
    t2 = t * t
    s = np.zeros_like(t)
    term = t.copy()
    for k in range(13):
        s = s + term / float(2 * k + 1)
        term = term * t2
    return 2.0 * s + e * _LN2


def exp(x) -> np.ndarray:
    """exp by range reduction x = q ln2 + r and a Taylor series for e^r."""
    x = np.asarray(x, dtype=np.float64)
    q = np.floor(x / _LN2 + 0.5)
    r = x - q * _LN2
    s = np.ones_like(r)
    term = np.ones_like(r)
    for k in range(1, 22):
        term = term * r / float(k)
        s = s + term
    return np.ldexp(s, q.astype(np.int64))


# -------------------------------------------------------------------- container
@dataclass
class Graph:
    n: int
    row_ptr: np.ndarray  # uint32 [n+1]
    col: np.ndarray      # uint32 [2m], each row sorted ascending

    @property
    def m(self) -> int:
        return int(self.col.size // 2)

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr.astype(np.int64))

    def edges(self) -> tuple[np.ndarray, np.ndarray]:
        """Undirected edges (u < v) in lexicographic order."""
        rows = np.repeat(np.arange(self.n, dtype=np.int64), self.degrees())
        c = self.col.astype(np.int64)
        keep = rows < c
        return rows[keep], c[keep]

    def fingerprint(self) -> str:
        h = hashlib.sha256()
        h.update(np.int64(self.n).tobytes())
        h.update(self.row_ptr.astype("<u4").tobytes())
        h.update(self.col.astype("<u4").tobytes())
        return h.hexdigest()[:16]


def from_edges(n: int, u, v) -> Graph:
    """Symmetric sorted CSR from an arbitrary edge list (duplicates and loops dropped)."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    keep = u != v
    u, v = u[keep], v[keep]
    key = np.sort(np.minimum(u, v) * np.int64(n) + np.maximum(u, v))
    if key.size:
        key = key[np.concatenate([[True], key[1:] != key[:-1]])]
    a = key // n
    b = key % n
    both = np.sort(np.concatenate([a * np.int64(n) + b, b * np.int64(n) + a]))
    src = both // n
    dst = both % n
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum(np.bincount(src, minlength=n))
    assert row_ptr[-1] < 2**32
    return Graph(n, row_ptr.astype(np.uint32), dst.astype(np.uint32))


def relabel(g: Graph, perm: np.ndarray) -> Graph:
    """Vertex i of ``g`` becomes ``perm[i]``."""
    u, v = g.edges()
    return from_edges(g.n, perm[u], perm[v])


def random_perm(n: int, seed: int, stream: int) -> np.ndarray:
    keys = rand_u64(seed, stream, np.arange(n, dtype=np.uint64))
    order = np.lexsort((np.arange(n), keys))
    perm = np.empty(n, dtype=np.int64)
    perm[order] = np.arange(n)
    return perm


def disjoint_union(graphs: list[Graph]) -> Graph:
    us, vs, off = [], [], 0
    for g in graphs:
        u, v = g.edges()
        us.append(u + off)
        vs.append(v + off)
        off += g.n
    return from_edges(off, np.concatenate(us) if us else [], np.concatenate(vs) if vs else [])


# ---------------------------------------------------------------- random models
def _pair_from_index(n: int, L: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Map linear indices over pairs i<j (row-major) to (i, j); exact integer fix-up."""
    L = L.astype(np.int64)
    # row i starts at S(i) = i*(2n-i-1)/2
    N2 = 2 * n - 1
    i = np.floor((N2 - np.sqrt(np.maximum(N2 * N2 - 8.0 * L, 0.0))) / 2.0).astype(np.int64)
    i = np.clip(i, 0, n - 2)

    def start(r):
        return r * (2 * n - r - 1) // 2

    for _ in range(3):
        i = np.where(start(i) > L, i - 1, i)
        i = np.where(start(i + 1) <= L, i + 1, i)
    j = L - start(i) + i + 1
    return i, j


def _skip_sample(total: int, p: float, seed: int, stream: int) -> np.ndarray:
    """Indices in [0, total) kept independently with probability p (geometric skips)."""
    if p <= 0 or total <= 0:
        return np.zeros(0, dtype=np.int64)
    if p >= 1:
        return np.arange(total, dtype=np.int64)
    lq = ln(np.array([1.0 - p]))[0]
    out = []
    pos = -1
    drawn = 0
    chunk = max(1024, int(total * p * 1.1) + 1024)
    while True:
        r = rand_unit(seed, stream, np.arange(drawn, drawn + chunk, dtype=np.uint64))
        drawn += chunk
        skips = np.floor(ln(r) / lq).astype(np.int64) + 1
        pos_arr = pos + np.cumsum(skips)
        inside = pos_arr < total
        out.append(pos_arr[inside])
        if not inside.all():
            break
        pos = int(pos_arr[-1])
    return np.concatenate(out)


def gnp(n: int, p: float, seed: int = 0, stream: int = 1) -> Graph:
    """G(n, p): every pair independently with probability p."""
    total = n * (n - 1) // 2
    L = _skip_sample(total, p, seed, stream)
    i, j = _pair_from_index(n, L)
    return from_edges(n, i, j)


def _distinct_draw(n: int, s: int, seed: int, stream: int) -> np.ndarray:
    """s distinct vertices of [0, n), uniform, in order of first draw."""
    s = min(s, n)
    got = np.zeros(0, dtype=np.int64)
    drawn = 0
    while got.size < s:
        c = rand_int(seed, stream, np.arange(drawn, drawn + 2 * s + 8, dtype=np.uint64), 0, n - 1)
        drawn += 2 * s + 8
        allv = np.concatenate([got, c])
        _, first = np.unique(allv, return_index=True)
        got = allv[np.sort(first)]
    return got[:s]


def _plant_cliques(n: int, sizes: list[int], seed: int, stream: int):
    us, vs = [], []
    for c, s in enumerate(sizes):
        verts = _distinct_draw(n, s, seed, stream * 1000003 + c)
        a, b = np.triu_indices(verts.size, 1)
        us.append(verts[a])
        vs.append(verts[b])
    if not us:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    return np.concatenate(us), np.concatenate(vs)


def chung_lu_weights(n: int, w_max: float, exponent: float, i0: float) -> np.ndarray:
    """w_i = w_max ((i + i0) / i0)^(-1/(exponent-1)), i = 0..n-1 (non-increasing)."""
    i = np.arange(n, dtype=np.float64)
    return w_max * exp(-ln((i + i0) / i0) / (exponent - 1.0))


def chung_lu(n: int = 1_000_000, w_max: float = 10_000.0, exponent: float = 2.1,
             i0: float = 147.844, planted: int = 200, planted_min: int = 30,
             planted_max: int = 60, seed: int = 0, relabel_ids: bool = True) -> Graph:
    """Chung-Lu expected-degree graph, p_ij = min(1, w_i w_j / S) with S = sum w.

    Pairs are drawn per row with the Miller-Hagberg skip over the weight-sorted
    vertices (rows advanced together, vectorised).  ``i0`` sets sum w: with the
    defaults sum w = 2.0e7 (average degree 20, about 1e7 edges) and 211 vertices
    have w >= sqrt(S), so they are mutually adjacent with probability 1.
    """
    w = chung_lu_weights(n, w_max, exponent, i0)
    S = math.fsum(w.tolist())
    rows = np.arange(n - 1, dtype=np.int64)
    j = rows + 1
    p = np.minimum(1.0, w[rows] * w[j] / S)
    draw = np.zeros(n - 1, dtype=np.uint64)
    eu, ev = [], []
    while rows.size:
        # geometric skip for rows whose current probability is below one
        r = rand_unit(seed, rows.astype(np.uint64) + np.uint64(7), draw)
        draw += np.uint64(1)
        lq = ln(np.where(p < 1.0, 1.0 - p, 0.5))
        skip = np.where(p < 1.0, np.floor(ln(r) / lq), 0.0)
        skip = np.minimum(skip, float(n)).astype(np.int64)
        j = j + skip
        ok = j < n
        rows, j, p, draw = rows[ok], j[ok], p[ok], draw[ok]
        if not rows.size:
            break
        q = np.minimum(1.0, w[rows] * w[j] / S)
        r2 = rand_unit(seed, rows.astype(np.uint64) + np.uint64(7), draw)
        draw += np.uint64(1)
        acc = r2 < q / p
        eu.append(rows[acc])
        ev.append(j[acc])
        p = q
        j = j + 1
        ok = (j < n) & (p > 0)
        rows, j, p, draw = rows[ok], j[ok], p[ok], draw[ok]
    u = np.concatenate(eu)
    v = np.concatenate(ev)
    if planted:
        sizes = rand_int(seed, 11, np.arange(planted, dtype=np.uint64), planted_min, planted_max).tolist()
        pu, pv = _plant_cliques(n, sizes, seed, 12)
        u = np.concatenate([u, pu])
        v = np.concatenate([v, pv])
    g = from_edges(n, u, v)
    if relabel_ids:
        g = relabel(g, random_perm(n, seed, 13))
    return g


def sbm_2plex(blocks: int = 200, block_size: int = 250, p_in: float = 0.9,
              p_out: float = 1e-4, two_plex_blocks: int = 50, seed: int = 0,
              relabel_ids: bool = True) -> tuple[Graph, dict]:
    """Stochastic block model with dense blocks; ``two_plex_blocks`` of them are exact
    2-plexes (K_b minus a random matching of M_b ~ U{1..b/2} pairs), the others G(b, p_in).

    Returns the graph and a dict with the block of every vertex (after relabel),
    the list of 2-plex blocks and their matching sizes.
    """
    b = block_size
    n = blocks * b
    sel_keys = rand_u64(seed, 21, np.arange(blocks, dtype=np.uint64))
    two_plex = np.sort(np.argsort(sel_keys, kind="stable")[:two_plex_blocks])
    is2 = np.zeros(blocks, dtype=bool)
    is2[two_plex] = True
    us, vs = [], []
    a_idx, b_idx = np.triu_indices(b, 1)
    matchings = {}
    for blk in range(blocks):
        base = blk * b
        if is2[blk]:
            M = int(rand_int(seed, 22, np.array([blk], dtype=np.uint64), 1, b // 2)[0])
            keys = rand_u64(seed, 23 + 1000 * blk, np.arange(b, dtype=np.uint64))
            order = np.argsort(keys, kind="stable")[: 2 * M]
            drop = set()
            for t in range(M):
                x, y = int(order[2 * t]), int(order[2 * t + 1])
                drop.add((min(x, y), max(x, y)))
            keep = np.array([(int(x), int(y)) not in drop for x, y in zip(a_idx, b_idx)])
            us.append(base + a_idx[keep])
            vs.append(base + b_idx[keep])
            matchings[blk] = M
        else:
            r = rand_unit(seed, 24 + 1000 * blk, np.arange(a_idx.size, dtype=np.uint64))
            keep = r < p_in
            us.append(base + a_idx[keep])
            vs.append(base + b_idx[keep])
    # inter-block pairs: sample over all pairs, drop the intra-block ones
    L = _skip_sample(n * (n - 1) // 2, p_out, seed, 25)
    i, j = _pair_from_index(n, L)
    inter = (i // b) != (j // b)
    us.append(i[inter])
    vs.append(j[inter])
    g = from_edges(n, np.concatenate(us), np.concatenate(vs))
    block_of = np.arange(n) // b
    if relabel_ids:
        perm = random_perm(n, seed, 26)
        g = relabel(g, perm)
        inv = np.empty(n, dtype=np.int64)
        inv[perm] = np.arange(n)
        block_of = block_of[inv]
    return g, {"block_of": block_of, "two_plex_blocks": two_plex.tolist(), "matching": matchings}


def batch_specs(count: int = 4096, seed: int = 0, n_lo: int = 64, n_hi: int = 4096,
                d_lo: float = 8.0, d_hi: float = 64.0, k_lo: int = 3, k_hi: int = 10):
    """Parameters of a batch of independent small graphs: (n, p, clique sizes, k, seed)."""
    idx = np.arange(count, dtype=np.uint64)
    ns = rand_int(seed, 31, idx, n_lo, n_hi)
    ds = d_lo + (d_hi - d_lo) * rand_unit(seed, 32, idx)
    nc = rand_int(seed, 33, idx, 1, 4)
    ks = rand_int(seed, 34, idx, k_lo, k_hi)
    specs = []
    for t in range(count):
        n = int(ns[t])
        p = min(1.0, float(ds[t]) / (n - 1))
        sizes = rand_int(seed, 35 + 17 * t, np.arange(int(nc[t]), dtype=np.uint64), 8, 24).tolist()
        specs.append({"n": n, "p": p, "cliques": [min(s, n) for s in sizes], "k": int(ks[t]),
                      "seed": seed * 1_000_003 + t})
    return specs


def batch_graph(spec: dict) -> Graph:
    g = gnp(spec["n"], spec["p"], spec["seed"], stream=41)
    pu, pv = _plant_cliques(spec["n"], spec["cliques"], spec["seed"], 42)
    u, v = g.edges()
    return from_edges(spec["n"], np.concatenate([u, pu]), np.concatenate([v, pv]))


# ------------------------------------------------------------------ fixtures
def complete(n: int) -> Graph:
    a, b = np.triu_indices(n, 1)
    return from_edges(n, a, b)


def complete_multipartite(parts: list[int]) -> Graph:
    lab = np.repeat(np.arange(len(parts)), parts)
    n = int(sum(parts))
    a, b = np.triu_indices(n, 1)
    keep = lab[a] != lab[b]
    return from_edges(n, a[keep], b[keep])


def complete_bipartite(p: int, q: int) -> Graph:
    return complete_multipartite([p, q])


def two_plex(f: int, pairs: int) -> Graph:
    """K_{f+2p} minus a perfect matching on its last 2p vertices (f universal vertices)."""
    n = f + 2 * pairs
    a, b = np.triu_indices(n, 1)
    miss = (a >= f) & (b == a + pairs) & (a < f + pairs)
    return from_edges(n, a[~miss], b[~miss])


def t_plex(n: int, t: int, seed: int = 0, density: float = 1.0) -> Graph:
    """Random t-plex: K_n minus a random graph of maximum degree t-1 (greedy, seeded)."""
    keys = rand_u64(seed, 51, np.arange(n * n, dtype=np.uint64))
    a, b = np.triu_indices(n, 1)
    order = np.argsort(keys[a * n + b], kind="stable")
    deg = np.zeros(n, dtype=np.int64)
    missing = np.zeros(a.size, dtype=bool)
    r = rand_unit(seed, 52, np.arange(a.size, dtype=np.uint64))
    for idx in order:
        x, y = a[idx], b[idx]
        if deg[x] < t - 1 and deg[y] < t - 1 and r[idx] < density:
            missing[idx] = True
            deg[x] += 1
            deg[y] += 1
    return from_edges(n, a[~missing], b[~missing])


def appendix_b() -> Graph:
    """Appendix B example: v1..v4 (ids 0..3), edges (v1,v3),(v1,v4),(v2,v3),(v2,v4),(v3,v4)."""
    return from_edges(4, [0, 0, 1, 1, 2], [2, 3, 2, 3, 3])


def config1(seed: int = 0) -> Graph:
    """Erdos-Renyi G(n=2000, p=0.01) (about 2e4 edges)."""
    return gnp(2000, 0.01, seed)
