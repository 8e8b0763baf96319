"""GPU parity for the wide bitset classes: sub-branches of 257..512 vertices (16 words)
and 513..1024 vertices (32 words), through the C ABI, exact integer equality.

Expected values come from the CPU oracle where it finishes in seconds (complete graphs
through its clique shortcut, G(n, 0.9) at small k) and otherwise from closed forms of
the mathematics: the k-cliques of K_{f+2p} minus a perfect matching on 2p vertices
(a 2-plex, Sec. 5.1) are sum_j C(f, k-j) C(p, j) 2^j with checksum the x^k coefficient
of prod_f (1 + z_f x) prod_pairs (1 + (z_a + z_b) x); those of a complete multipartite
graph are e_k(part sizes) with checksum e_k(per-part key sums).
"""
import math

import numpy as np
import pytest

import oracle as O
from synth import graphs as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
M64 = (1 << 64) - 1


def K():
    from paper_2311_13798_gb300 import kclique
    return kclique


def prep(g):
    rp = torch.from_numpy(g.row_ptr.astype(np.int32)).cuda()
    col = torch.from_numpy(g.col.astype(np.int32)).cuda()
    return K().kclique_prepare(rp, col, g.n)


def esym(vals, k):
    e = [1] + [0] * k
    for x in vals:
        for j in range(k, 0, -1):
            e[j] += e[j - 1] * x
    return e[k]


def width_of(h):
    return int(K().kclique_edge_data(h)["vset_size"].max())


@pytest.fixture(scope="module")
def cache():
    return {}


def get(cache, name, make):
    if name not in cache:
        g = make()
        cache[name] = (g, prep(g))
    return cache[name]


@pytest.mark.parametrize("n,lo,hi", [(400, 257, 512), (700, 513, 1024)])
def test_complete_graphs(cache, n, lo, hi):
    g, h = get(cache, f"k{n}", lambda: G.complete(n))
    assert lo <= width_of(h) <= hi
    for k in (3, 4, 5, 6, 8):
        want = O.count(g, k)
        assert want["count"] == math.comb(n, k)
        got = K().kclique_count(h, k, flags=K().KC_CHECKSUM)
        assert (got["count"], got["checksum"]) == (want["count"], want["checksum"]), (n, k)
        assert K().kclique_count(h, k)["count"] == want["count"]
        if k <= 5:  # no early termination: extraction, leaves and the l = 3 routine
            got = K().kclique_count(h, k, flags=K().KC_CHECKSUM | K().KC_NO_ET)
            assert (got["count"], got["checksum"]) == (want["count"], want["checksum"]), (n, k)
        if k >= 7:  # the heavy-branch split path
            got = K().kclique_count(h, k, split_min=3, flags=K().KC_CHECKSUM)
            assert (got["count"], got["checksum"]) == (want["count"], want["checksum"]), (n, k)


@pytest.mark.parametrize("n,kmax,lo,hi", [(420, 5, 257, 512), (800, 4, 513, 1024)])
def test_dense_random(cache, n, kmax, lo, hi):
    g, h = get(cache, f"gnp{n}", lambda: G.gnp(n, 0.9, seed=21))
    assert lo <= width_of(h) <= hi
    for k in range(3, kmax + 1):
        want = O.count(g, k)
        got = K().kclique_count(h, k, flags=K().KC_CHECKSUM)
        assert (got["count"], got["checksum"]) == (want["count"], want["checksum"]), (n, k)
        assert K().kclique_count(h, k)["count"] == want["count"]


def test_two_plex_600(cache):
    f, p = 100, 250
    g, h = get(cache, "two_plex600", lambda: G.two_plex(f, p))
    assert 513 <= width_of(h) <= 1024
    z = [O.key(v) for v in range(f + 2 * p)]
    for k in (4, 5, 7, 9):
        cnt = sum(math.comb(f, k - j) * math.comb(p, j) * 2**j for j in range(0, k + 1))
        poly = [1] + [0] * k
        for c in [z[v] for v in range(f)] + [z[f + i] + z[f + p + i] for i in range(p)]:
            for j in range(k, 0, -1):
                poly[j] += poly[j - 1] * c
        got = K().kclique_count(h, k, flags=K().KC_CHECKSUM)
        assert (got["count"], got["checksum"]) == (cnt, poly[k] & M64), k
        if k >= 5:  # k = 4 counts the edges of each sub-branch: no frame to close
            assert got["et_hits"] > 0


def test_cocktail_party_600_with_t3(cache):
    """K_{3,3,...,3} (200 parts): every vertex misses two others, so every sub-branch is a
    3-plex whose inverse graph is a union of triangles; t = 3 closes them at the top."""
    parts = [3] * 200
    g, h = get(cache, "cocktail600", lambda: G.complete_multipartite(parts))
    assert 513 <= width_of(h) <= 1024
    Z = [sum(O.key(3 * i + j) for j in range(3)) for i in range(200)]
    for k in (4, 5, 7, 9):
        got = K().kclique_count(h, k, t_max=3, flags=K().KC_CHECKSUM)
        assert (got["count"], got["checksum"]) == (esym(parts, k), esym(Z, k) & M64), k
        if k >= 7:
            assert got["et_hits"] > 0
