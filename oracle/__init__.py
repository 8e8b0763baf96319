"""CPU oracle for exact k-clique counting / listing -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the GPU library
(``paper_2311_13798_gb300``) and never imports it.

The arithmetic lives in ``kc_oracle.c`` (plain C + OpenMP, 128-bit counts); this
module compiles it with gcc on first use and marshals numpy arrays.  Also here:
``brute_force`` (all k-subsets, pure Python, tiny graphs) and ``checksum_of``
(the checksum of an explicit clique list), both written from the definitions
(paper Sec. 2, Def. "k-clique"; checksum = sum over cliques of the product of
z(v) = splitmix64(v) | 1, mod 2^64).

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(brute force, complete graphs, Turan graphs, trace(A^3)/6, 2-plex closed forms,
the Appendix B example, complete bipartite graphs, disjoint unions, relabelings,
and a second truss-peel algorithm for the levels); ``sparse_complement_count`` is
pinned against ``count`` and brute force on 2- and 3-plexes and cocktail-party graphs.
"""
from __future__ import annotations

import ctypes as C
import itertools
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kc_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libkc_oracle.so")
_lib = None
_lock = threading.Lock()
MASK64 = (1 << 64) - 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2 -fopenmp); returns the library path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.POINTER
            u64p, u32p = P(C.c_uint64), P(C.c_uint32)
            lib.oc_key.restype = C.c_uint64
            lib.oc_key.argtypes = [C.c_uint64]
            lib.oc_count.restype = C.c_int
            lib.oc_count.argtypes = [C.c_uint32, u64p, u32p, C.c_int, C.c_int, C.c_int, C.c_int,
                                     u32p, C.c_uint64, u64p, u64p, u64p, u64p, u32p, u32p,
                                     C.c_uint64, u64p]
            lib.oc_truss_peel.restype = C.c_uint64
            lib.oc_truss_peel.argtypes = [C.c_uint32, u64p, u32p, C.c_uint64, u32p, u32p]
            lib.oc_truss_sequential.restype = None
            lib.oc_truss_sequential.argtypes = [C.c_uint32, u64p, u32p, C.c_uint64, u32p]
            lib.oc_vset_sizes.restype = None
            lib.oc_vset_sizes.argtypes = [C.c_uint32, u64p, u32p, C.c_uint64, u32p, u32p]
            lib.oc_edge_counts.restype = C.c_int
            lib.oc_edge_counts.argtypes = [C.c_uint32, u64p, u32p, C.c_uint64, u32p, C.c_int, u32p,
                                           C.c_uint64, C.c_int, C.c_int, u64p, u64p, u64p]
            _lib = lib
    return _lib


def _p(a, t):
    return a.ctypes.data_as(C.POINTER(t))


def threads_default() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


# ------------------------------------------------------------------ inputs
class CleanGraph:
    """Symmetric, sorted, duplicate- and loop-free CSR (64-bit offsets) of any input CSR.

    Directions, duplicates and self-loops are dropped (paper Sec. 6.1, "Datasets").
    """

    def __init__(self, n, row_ptr, col):
        n = int(n)
        rp = np.asarray(row_ptr, dtype=np.int64)
        c = np.asarray(col, dtype=np.int64)
        src = np.repeat(np.arange(n, dtype=np.int64), np.diff(rp))
        keep = src != c
        a = np.minimum(src[keep], c[keep])
        b = np.maximum(src[keep], c[keep])
        key = np.unique(a * n + b)
        a, b = key // n, key % n
        s2 = np.concatenate([a, b])
        d2 = np.concatenate([b, a])
        order = np.lexsort((d2, s2))
        s2, d2 = s2[order], d2[order]
        self.n = n
        self.row_ptr = np.zeros(n + 1, dtype=np.uint64)
        self.row_ptr[1:] = np.cumsum(np.bincount(s2, minlength=n)).astype(np.uint64)
        self.col = np.ascontiguousarray(d2.astype(np.uint32))
        self.m = int(self.col.size // 2)
        self.eu = a.astype(np.uint32)  # edge id = index in (u < v) lexicographic order
        self.ev = b.astype(np.uint32)

    @classmethod
    def of(cls, g):
        return cls(g.n, g.row_ptr, g.col)


def _clean(g) -> CleanGraph:
    return g if isinstance(g, CleanGraph) else CleanGraph.of(g)


# ------------------------------------------------------------------ keys
def key(v: int) -> int:
    """z(v) = splitmix64(v) | 1, in pure Python (independent of the C copy)."""
    x = (v + 0x9E3779B97F4A7C15) & MASK64
    x = ((x ^ (x >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    x = ((x ^ (x >> 27)) * 0x94D049BB133111EB) & MASK64
    x ^= x >> 31
    return x | 1


def key_c(v: int) -> int:
    return int(_load().oc_key(v))


def checksum_of(cliques) -> int:
    """Sum over the given cliques of the product of keys, mod 2^64."""
    s = 0
    for q in cliques:
        p = 1
        for v in q:
            p = (p * key(int(v))) & MASK64
        s = (s + p) & MASK64
    return s


# ------------------------------------------------------------------ counting
def count(g, k: int, shortcut: bool = True, checksum: bool = True, threads: int | None = None,
          tops=None):
    """Exact k-clique count (Python int) and checksum; optional bounded sample of top vertices.

    Returns dict(count, checksum, nodes, degeneracy).
    """
    cg = _clean(g)
    lib = _load()
    lo, hi, cs, nodes, wr = (np.zeros(1, np.uint64) for _ in range(5))
    dg = np.zeros(1, np.uint32)
    t = np.ascontiguousarray(tops, dtype=np.uint32) if tops is not None else None
    rc = lib.oc_count(cg.n, _p(cg.row_ptr, C.c_uint64), _p(cg.col, C.c_uint32), int(k), int(shortcut),
                      int(checksum), int(threads or threads_default()),
                      _p(t, C.c_uint32) if t is not None else None, 0 if t is None else t.size,
                      _p(lo, C.c_uint64), _p(hi, C.c_uint64), _p(cs, C.c_uint64), _p(nodes, C.c_uint64),
                      _p(dg, C.c_uint32), None, 0, _p(wr, C.c_uint64))
    if rc == 1:
        raise OverflowError("k-clique count exceeds 2^128")
    if rc:
        raise ValueError(f"oracle rejected k={k}")
    return {"count": int(lo[0]) | (int(hi[0]) << 64), "checksum": int(cs[0]), "nodes": int(nodes[0]),
            "degeneracy": int(dg[0])}


def list_cliques(g, k: int, cap: int | None = None) -> np.ndarray:
    """All k-cliques as rows of ascending vertex ids (plain recursion, no shortcut)."""
    cg = _clean(g)
    lib = _load()
    if cap is None:
        cap = count(cg, k, shortcut=True, checksum=False)["count"]
    out = np.zeros((max(cap, 1), k), dtype=np.uint32)
    lo, hi, cs, nodes, wr = (np.zeros(1, np.uint64) for _ in range(5))
    dg = np.zeros(1, np.uint32)
    rc = lib.oc_count(cg.n, _p(cg.row_ptr, C.c_uint64), _p(cg.col, C.c_uint32), int(k), 0, 1, 1, None, 0,
                      _p(lo, C.c_uint64), _p(hi, C.c_uint64), _p(cs, C.c_uint64), _p(nodes, C.c_uint64),
                      _p(dg, C.c_uint32), _p(out, C.c_uint32), cap, _p(wr, C.c_uint64))
    if rc:
        raise ValueError("oracle listing failed")
    return out[: min(int(wr[0]), cap)]


def brute_force(g, k: int):
    """Every k-subset checked pair by pair (tiny graphs only). Returns (count, checksum, cliques)."""
    cg = _clean(g)
    adj = [set() for _ in range(cg.n)]
    for a, b in zip(cg.eu.tolist(), cg.ev.tolist()):
        adj[a].add(b)
        adj[b].add(a)
    found = [q for q in itertools.combinations(range(cg.n), k)
             if all(y in adj[x] for x, y in itertools.combinations(q, 2))]
    return len(found), checksum_of(found), found


# ------------------------------------------------------------------ sparse complements
def sparse_complement_count(g, k: int):
    """Exact k-clique count and checksum of a graph whose complement has maximum degree
    at most 2 -- a 3-plex in the paper's terms (Sec. 5: every vertex misses at most t = 3
    vertices counting itself), e.g. K_n minus a matching (a 2-plex) or minus disjoint
    paths and cycles.  Used where enumeration cannot finish (the 250-vertex 2-plex blocks
    of the SBM workload at k up to 10).

    The k-cliques of G are the independent k-sets of its complement H.  H is a disjoint
    union of isolated vertices, paths and cycles; its weighted independence polynomial
    I(H; x) = sum over independent S of prod_{v in S} (z_v x) is the product of those of
    its components, and the k-clique count and checksum are the x^k coefficients of
    I(H; x) with z = 1 and with z = the keys.  A path's polynomial follows from the
    recurrence I(P_{v1..vm}) = I(P_{v2..vm}) + z_{v1} x I(P_{v3..vm}) (v1 out / v1 in);
    a cycle's is I(P_{v2..vm}) + z_{v1} x I(P_{v3..v(m-1)}).  Exact Python integers;
    the checksum is reduced mod 2^64 at the end.  Raises ValueError if the complement
    has a vertex of degree > 2.
    """
    cg = _clean(g)
    n = cg.n
    deg = np.diff(cg.row_ptr.astype(np.int64))
    active = np.nonzero(deg > 0)[0]
    # vertices without edges belong to no clique of size >= 2; the graph is taken on the
    # vertices that have edges (ids kept), as a subgraph of the SBM is
    vs = active.tolist()
    idx = {v: i for i, v in enumerate(vs)}
    nv = len(vs)
    nbr = [set() for _ in range(nv)]
    for a, b in zip(cg.eu.tolist(), cg.ev.tolist()):
        nbr[idx[a]].add(idx[b])
        nbr[idx[b]].add(idx[a])
    miss = []
    for i in range(nv):
        m = [j for j in range(nv) if j != i and j not in nbr[i]]
        if len(m) > 2:
            raise ValueError("the complement has a vertex of degree > 2")
        miss.append(m)
    z = [key(v) for v in vs]

    def mul(a, b):
        out = [0] * (k + 1)
        for i, x in enumerate(a):
            if x:
                for j, y in enumerate(b[: k + 1 - i]):
                    out[i + j] += x * y
        return out

    def path_poly(seq, w):
        # I(P) over the vertex sequence seq, truncated at x^k
        if not seq:
            return [1] + [0] * k
        prev2 = [1] + [0] * k                      # I of the empty suffix
        prev1 = [1] + [0] * k
        prev1[1] = w[seq[-1]]                      # I of the last vertex alone
        if k < 1:
            prev1 = prev1[:1]
        for v in reversed(seq[:-1]):
            cur = [prev1[j] + (w[v] * prev2[j - 1] if j >= 1 else 0) for j in range(k + 1)]
            prev2, prev1 = prev1, cur
        return prev1

    def component_polys(w):
        seen = [False] * nv
        total = [1] + [0] * k
        for start in range(nv):
            if seen[start] or len(miss[start]) == 2:
                continue
            seq, prev, cur = [], -1, start          # a path from an end (or an isolated vertex)
            while cur != -1:
                seen[cur] = True
                seq.append(cur)
                nxt = [x for x in miss[cur] if x != prev]
                prev, cur = cur, (nxt[0] if nxt else -1)
            total = mul(total, path_poly(seq, w))
        for start in range(nv):
            if seen[start]:
                continue
            seq, prev, cur = [], -1, start          # a cycle
            while not seen[cur]:
                seen[cur] = True
                seq.append(cur)
                nxt = [x for x in miss[cur] if x != prev]
                prev, cur = cur, nxt[0]
            v1 = seq[0]
            out_v1 = path_poly(seq[1:], w)
            in_v1 = path_poly(seq[2:-1], w)
            poly = [out_v1[j] + (w[v1] * in_v1[j - 1] if j >= 1 else 0) for j in range(k + 1)]
            total = mul(total, poly)
        return total

    cnt = component_polys([1] * nv)[k]
    cs = component_polys(z)[k] & MASK64
    return {"count": cnt, "checksum": cs}


# ------------------------------------------------------------------ edges
def truss_peel(g):
    """Level-synchronous truss peel: (level[m], round[m], rounds) per edge id."""
    cg = _clean(g)
    lib = _load()
    lvl = np.zeros(max(cg.m, 1), np.uint32)
    rnd = np.zeros(max(cg.m, 1), np.uint32)
    r = lib.oc_truss_peel(cg.n, _p(cg.row_ptr, C.c_uint64), _p(cg.col, C.c_uint32), cg.m,
                          _p(lvl, C.c_uint32), _p(rnd, C.c_uint32))
    return lvl[: cg.m], rnd[: cg.m], int(r)


def truss_sequential(g) -> np.ndarray:
    """Textbook one-edge-at-a-time truss peel: level[m] = trussness - 2."""
    cg = _clean(g)
    lib = _load()
    lvl = np.zeros(max(cg.m, 1), np.uint32)
    lib.oc_truss_sequential(cg.n, _p(cg.row_ptr, C.c_uint64), _p(cg.col, C.c_uint32), cg.m,
                            _p(lvl, C.c_uint32))
    return lvl[: cg.m]


def vset_sizes(g, rounds) -> np.ndarray:
    cg = _clean(g)
    lib = _load()
    r = np.ascontiguousarray(rounds, dtype=np.uint32)
    out = np.zeros(max(cg.m, 1), np.uint32)
    lib.oc_vset_sizes(cg.n, _p(cg.row_ptr, C.c_uint64), _p(cg.col, C.c_uint32), cg.m,
                      _p(r, C.c_uint32), _p(out, C.c_uint32))
    return out[: cg.m]


def edge_counts(g, k: int, rounds, edges, shortcut: bool = True, threads: int | None = None):
    """For each chosen edge id e: count and checksum of the k-cliques whose first edge
    in the (round, id) order is e -- the (k-2)-cliques of the sub-branch g_e of Eq. 2."""
    cg = _clean(g)
    lib = _load()
    r = np.ascontiguousarray(rounds, dtype=np.uint32)
    e = np.ascontiguousarray(edges, dtype=np.uint32)
    lo, hi, cs = (np.zeros(max(e.size, 1), np.uint64) for _ in range(3))
    rc = lib.oc_edge_counts(cg.n, _p(cg.row_ptr, C.c_uint64), _p(cg.col, C.c_uint32), cg.m,
                            _p(r, C.c_uint32), int(k), _p(e, C.c_uint32), e.size, int(shortcut),
                            int(threads or threads_default()), _p(lo, C.c_uint64), _p(hi, C.c_uint64),
                            _p(cs, C.c_uint64))
    if rc:
        raise OverflowError("per-edge count exceeds 2^128")
    counts = [int(a) | (int(b) << 64) for a, b in zip(lo[: e.size], hi[: e.size])]
    return counts, [int(x) for x in cs[: e.size]]
