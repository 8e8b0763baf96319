"""Pins for the CPU oracle against facts fixed by the paper and by mathematics.

Each test targets a plausible mistake in the oracle (a dropped clique, a doubled
clique, a wrong key, a wrong truss level, a non-partitioning sub-branch):
brute force over all k-subsets, closed forms for complete and complete
multipartite graphs, trace(A^3)/6 for triangles, the 2-plex count of Sec. 5.1,
the Appendix B example, complete bipartite graphs (tau = 0, Sec. 4.2
"Discussion on tau"), disjoint unions, relabelings, a brute-force trussness on
tiny graphs, and the partition of all cliques into edge sub-branches (Eq. 2).
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from synth import graphs as G

GOLD = os.path.join(os.path.dirname(__file__), "golden")
M64 = (1 << 64) - 1


def esym(vals, k):
    """Elementary symmetric polynomial e_k of Python ints (exact, big ints)."""
    e = [1] + [0] * k
    for x in vals:
        for j in range(k, 0, -1):
            e[j] += e[j - 1] * x
    return e[k]


def test_key_published_splitmix64_value():
    # SplitMix64 seeded with 0: first output is 0xE220A8397B1DCDAF (Vigna's splitmix64.c)
    assert O.key(0) == 0xE220A8397B1DCDAF
    for v in [0, 1, 2, 12345, 2**32 - 1, 999_999]:
        assert O.key(v) == O.key_c(v)
        assert O.key(v) & 1


@pytest.mark.parametrize("n,p,seed", [(10, 0.5, 1), (14, 0.6, 2), (16, 0.8, 3), (20, 0.3, 4), (18, 0.9, 5)])
def test_brute_force(n, p, seed):
    g = G.gnp(n, p, seed=seed)
    for k in range(3, 9):
        bf_count, bf_sum, bf_list = O.brute_force(g, k)
        for shortcut in (False, True):
            r = O.count(g, k, shortcut=shortcut)
            assert r["count"] == bf_count
            assert r["checksum"] == bf_sum
        got = sorted(map(tuple, O.list_cliques(g, k).tolist()))
        assert got == sorted(bf_list)


@pytest.mark.parametrize("n", [5, 17, 40, 70])
def test_complete_graph(n):
    g = G.complete(n)
    z = [O.key(v) for v in range(n)]
    for k in [3, 4, 5, 7]:
        if k > n:
            continue
        want = esym(z, k) & M64
        r = O.count(g, k, shortcut=False, threads=4) if n <= 40 or k <= 4 else None
        if r is not None:
            assert r["count"] == math.comb(n, k)
            assert r["checksum"] == want
        r2 = O.count(g, k, shortcut=True)
        assert r2["count"] == math.comb(n, k)
        assert r2["checksum"] == want


@pytest.mark.parametrize("parts", [[3, 3, 3], [1, 2, 3, 4, 5], [6, 6, 6, 6], [2] * 9])
def test_turan(parts):
    g = G.complete_multipartite(parts)
    lab = np.repeat(np.arange(len(parts)), parts)
    Z = [sum(O.key(v) for v in np.nonzero(lab == i)[0].tolist()) for i in range(len(parts))]
    for k in range(3, len(parts) + 2):
        want_c = esym(parts, k)
        want_s = esym(Z, k) & M64
        for shortcut in (False, True):
            r = O.count(g, k, shortcut=shortcut)
            assert r["count"] == want_c
            assert r["checksum"] == want_s


@pytest.mark.parametrize("n,p,seed", [(60, 0.3, 7), (120, 0.15, 8), (200, 0.08, 9)])
def test_triangles_trace(n, p, seed):
    g = G.gnp(n, p, seed=seed)
    A = np.zeros((n, n), dtype=object)
    u, v = g.edges()
    for a, b in zip(u.tolist(), v.tolist()):
        A[a, b] = A[b, a] = 1
    A3 = A.dot(A).dot(A)
    assert sum(A3[i, i] for i in range(n)) % 6 == 0
    want_c = sum(A3[i, i] for i in range(n)) // 6
    z = np.array([O.key(i) for i in range(n)], dtype=object)
    DA = A * z[:, None]          # D A with D = diag(z)
    T = DA.dot(DA).dot(DA)
    tr = sum(T[i, i] for i in range(n))
    assert tr % 6 == 0
    r = O.count(g, 3)
    assert r["count"] == want_c
    assert r["checksum"] == (tr // 6) & M64


def _two_plex_closed(f, p, l, zf, zpairs):
    cnt = sum(math.comb(f, l - j) * math.comb(p, j) * 2**j for j in range(0, l + 1))
    poly = [1]
    factors = [[1, z] for z in zf] + [[1, za + zb] for za, zb in zpairs]
    for fac in factors:
        nxt = [0] * (len(poly) + 1)
        for i, c in enumerate(poly):
            nxt[i] += c * fac[0]
            nxt[i + 1] += c * fac[1]
        poly = nxt
    return cnt, (poly[l] if l < len(poly) else 0) & M64


def test_fig3_two_plex_counts():
    fx = json.load(open(os.path.join(GOLD, "fig3_two_plex.json")))
    g = G.two_plex(fx["f"], fx["pairs"])
    for l, want in fx["counts_by_l_hand_counted"].items():
        l = int(l)
        if l >= 3:
            assert O.count(g, l, shortcut=False)["count"] == want
        cnt, _ = _two_plex_closed(fx["f"], fx["pairs"], l, [0] * fx["f"], [(0, 0)] * fx["pairs"])
        assert cnt == want


@pytest.mark.parametrize("f,p", [(0, 5), (3, 4), (10, 6), (20, 15)])
def test_two_plex_closed_form(f, p):
    g = G.two_plex(f, p)
    zf = [O.key(v) for v in range(f)]
    zpairs = [(O.key(f + i), O.key(f + p + i)) for i in range(p)]
    for l in range(3, min(f + p, 9) + 1):
        want_c, want_s = _two_plex_closed(f, p, l, zf, zpairs)
        r = O.count(g, l, shortcut=False, threads=4)
        assert r["count"] == want_c
        assert r["checksum"] == want_s


def test_appendix_b():
    fx = json.load(open(os.path.join(GOLD, "appendix_b.json")))
    e = np.array(fx["edges"]) - 1
    g = G.from_edges(4, e[:, 0], e[:, 1])
    r = O.count(g, fx["k"])
    assert r["count"] == fx["count"]
    got = sorted(map(tuple, (O.list_cliques(g, 3) + 1).tolist()))
    assert got == sorted(map(tuple, fx["cliques"]))
    # the paper's truss-based order is a valid truss order: every edge's support in the
    # suffix graph is minimal among the remaining edges when it is taken out
    order = [tuple(sorted((a - 1, b - 1))) for a, b in fx["truss_order_in_paper"]]
    remaining = set(order)
    for e0 in order:
        def sup(ed):
            a, b = ed
            return sum(1 for w in range(4) if tuple(sorted((a, w))) in remaining and tuple(sorted((b, w))) in remaining)
        assert sup(e0) == min(sup(x) for x in remaining)
        remaining.remove(e0)
    lvl, rnd, _ = O.truss_peel(g)
    assert (lvl == 1).all()


@pytest.mark.parametrize("p", [2, 5, 9])
def test_complete_bipartite_tau_zero(p):
    g = G.complete_bipartite(p, p)
    for k in (3, 4):
        assert O.count(g, k)["count"] == 0
    lvl, rnd, _ = O.truss_peel(g)
    assert lvl.max() == 0
    assert (O.truss_sequential(g) == 0).all()


def test_disjoint_union_additive():
    gs = [G.gnp(30, 0.5, seed=s) for s in range(3)] + [G.complete(9), G.two_plex(4, 3)]
    u = G.disjoint_union(gs)
    for k in (3, 4, 5, 6):
        parts = []
        off = 0
        for g in gs:
            # shift ids so keys match the union's ids
            uu, vv = g.edges()
            parts.append(O.count(G.from_edges(off + g.n, uu + off, vv + off), k))
            off += g.n
        whole = O.count(u, k)
        assert whole["count"] == sum(p["count"] for p in parts)
        assert whole["checksum"] == sum(p["checksum"] for p in parts) & M64


def test_relabel():
    g = G.gnp(40, 0.4, seed=11)
    perm = G.random_perm(40, 5, 6)
    h = G.relabel(g, perm)
    for k in (3, 4, 5):
        cl = O.list_cliques(g, k)
        want = O.checksum_of([[perm[v] for v in q] for q in cl.tolist()])
        r = O.count(h, k)
        assert r["count"] == len(cl)
        assert r["checksum"] == want


def _trussness_brute(n, edges):
    """Level (trussness - 2) by definition: the largest s such that the edge lies in a
    subgraph where every edge has >= s triangles inside that subgraph."""
    m = len(edges)
    best = [0] * m
    for mask in range(1, 1 << m):
        sub = [edges[i] for i in range(m) if mask >> i & 1]
        S = set(sub)
        sups = []
        for a, b in sub:
            sups.append(sum(1 for w in range(n) if (min(a, w), max(a, w)) in S and (min(b, w), max(b, w)) in S))
        s = min(sups)
        for i in range(m):
            if mask >> i & 1 and best[i] < s:
                best[i] = s
    return best


@pytest.mark.parametrize("n,p,seed", [(6, 0.8, 1), (7, 0.6, 2), (6, 0.9, 3)])
def test_truss_levels_brute_force(n, p, seed):
    g = G.gnp(n, p, seed=seed)
    u, v = g.edges()
    edges = list(zip(u.tolist(), v.tolist()))
    if len(edges) > 15:
        edges = edges[:15]
        g = G.from_edges(n, [a for a, _ in edges], [b for _, b in edges])
    want = _trussness_brute(n, edges)
    lvl, _, _ = O.truss_peel(g)
    assert lvl.tolist() == want
    assert O.truss_sequential(g).tolist() == want


@pytest.mark.parametrize("maker", [
    lambda: G.gnp(300, 0.1, seed=1),
    lambda: G.gnp(150, 0.4, seed=2),
    lambda: G.complete(25),
    lambda: G.two_plex(10, 8),
    lambda: G.chung_lu(n=3000, w_max=300.0, i0=30.0, planted=5, planted_min=10, planted_max=20, seed=3),
    lambda: G.sbm_2plex(blocks=6, block_size=40, p_out=0.01, two_plex_blocks=2, seed=4)[0],
])
def test_truss_peel_properties(maker):
    g = maker()
    lvl, rnd, nr = O.truss_peel(g)
    assert (O.truss_sequential(g) == lvl).all()
    sizes = O.vset_sizes(g, rnd)
    assert int(sizes.sum()) == O.count(g, 3)["count"]
    assert (sizes <= lvl).all()
    tau = int(lvl.max()) if lvl.size else 0
    assert int(sizes.max()) == tau
    # rounds are monotone in level
    order = np.lexsort((np.arange(lvl.size), rnd))
    assert (np.diff(lvl[order].astype(np.int64)) >= 0).all()


def test_complete_graph_tau():
    for n in (4, 10, 30):
        lvl, _, _ = O.truss_peel(G.complete(n))
        assert (lvl == n - 2).all()


@pytest.mark.parametrize("maker,ks", [
    (lambda: G.gnp(80, 0.35, seed=5), (3, 4, 5, 6)),
    (lambda: G.two_plex(8, 6), (3, 5, 7)),
    (lambda: G.t_plex(30, 3, seed=2), (4, 6, 8)),
    (lambda: G.chung_lu(n=2000, w_max=200.0, i0=25.0, planted=4, planted_min=8, planted_max=14, seed=6), (4, 5, 7)),
])
def test_edge_subbranches_partition_cliques(maker, ks):
    """Eq. 2: the sub-branches of all edges, in the (round, id) order, list every
    k-clique exactly once."""
    g = maker()
    _, rnd, _ = O.truss_peel(g)
    m = g.m
    for k in ks:
        cnt, cs = O.edge_counts(g, k, rnd, np.arange(m))
        whole = O.count(g, k)
        assert sum(cnt) == whole["count"]
        assert sum(cs) & M64 == whole["checksum"]


def test_overflow_guard():
    with pytest.raises(OverflowError):
        O.count(G.complete(300), 64)


def test_sample_of_tops_is_additive():
    g = G.gnp(200, 0.2, seed=12)
    full = O.count(g, 4)
    a = O.count(g, 4, tops=np.arange(0, 100))
    b = O.count(g, 4, tops=np.arange(100, 200))
    assert a["count"] + b["count"] == full["count"]
    assert (a["checksum"] + b["checksum"]) & M64 == full["checksum"]


def _complement_of(n, missing):
    """K_n minus the given pairs."""
    miss = {(min(a, b), max(a, b)) for a, b in missing}
    a, b = np.triu_indices(n, 1)
    keep = np.array([(int(x), int(y)) not in miss for x, y in zip(a, b)], dtype=bool)
    return G.from_edges(n, a[keep], b[keep])


@pytest.mark.parametrize("maker,ks", [
    (lambda: G.two_plex(5, 4), (3, 4, 5, 6)),
    (lambda: G.two_plex(0, 6), (3, 6, 7)),
    (lambda: G.t_plex(30, 3, seed=2), (3, 4, 5, 6)),
    (lambda: G.t_plex(14, 3, seed=7), (3, 4, 5, 6, 7)),
    (lambda: G.complete_multipartite([3] * 8), (3, 4, 5, 8, 9)),           # complement: triangles
    (lambda: _complement_of(12, [(i, (i + 1) % 12) for i in range(12)]), (3, 4, 5, 6, 7)),  # C_12
    (lambda: _complement_of(11, [(i, i + 1) for i in range(10)]), (3, 4, 5, 6)),           # P_11
    (lambda: _complement_of(13, [(0, 1), (1, 2), (2, 0), (3, 4), (4, 5), (5, 6), (6, 3), (7, 8)]), (3, 5, 7)),
    (lambda: G.complete(9), (3, 5, 9)),
])
def test_sparse_complement_closed_form(maker, ks):
    """Cliques of G = independent sets of its complement; for a complement of paths and
    cycles the product of their independence polynomials matches enumeration."""
    g = maker()
    for k in ks:
        a = O.sparse_complement_count(g, k)
        b = O.count(g, k, shortcut=False)
        assert (a["count"], a["checksum"]) == (b["count"], b["checksum"]), k
        if g.n <= 14:
            bf_c, bf_s, _ = O.brute_force(g, k)
            assert (a["count"], a["checksum"]) == (bf_c, bf_s)


def test_sparse_complement_rejects_denser_complement():
    g = _complement_of(8, [(0, 1), (0, 2), (0, 3)])
    with pytest.raises(ValueError):
        O.sparse_complement_count(g, 3)


def test_block_decomposition_of_sbm():
    """Every clique lies in one block or holds an inter-block edge: with the inter-block
    edges first in the edge order, their sub-branches (Eq. 2) hold exactly the latter,
    and the blocks plus that term give the whole."""
    g, info = G.sbm_2plex(blocks=6, block_size=40, p_in=0.8, p_out=0.08, two_plex_blocks=2, seed=3)
    blk = info["block_of"]
    cg = O.CleanGraph.of(g)
    cross = blk[cg.eu] != blk[cg.ev]
    rounds = np.where(cross, 0, 1).astype(np.uint32)
    u, v = g.edges()
    for k in (3, 4, 5):
        cnt, cs = O.edge_counts(cg, k, rounds, np.nonzero(cross)[0])
        parts = [O.count(G.from_edges(g.n, u[(blk[u] == b) & (blk[v] == b)], v[(blk[u] == b) & (blk[v] == b)]), k)
                 for b in range(6)]
        whole = O.count(g, k)
        assert sum(cnt) > 0 or k > 3
        assert whole["count"] == sum(p["count"] for p in parts) + sum(cnt)
        assert whole["checksum"] == (sum(p["checksum"] for p in parts) + sum(cs)) & M64
    for b in info["two_plex_blocks"]:
        keep = (blk[u] == b) & (blk[v] == b)
        sub = G.from_edges(g.n, u[keep], v[keep])
        for k in (4, 6):
            a = O.sparse_complement_count(sub, k)
            r = O.count(sub, k)
            assert (a["count"], a["checksum"]) == (r["count"], r["checksum"])
