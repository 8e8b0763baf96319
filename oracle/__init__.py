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
and a second truss-peel algorithm for the levels).
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
