"""Dense l = 4 frames counted whole through their complement (even k), at every bitset
width, against exact values.

G is the complement of m disjoint copies of a small graph F (vertex ids shuffled), so a
k-clique of G is an independent k-set of those copies: the count is the x^k coefficient
of I_F(x)^m and the checksum (sum over cliques of the product of the vertices' keys,
mod 2^64) the x^k coefficient of the product over copies of I_F(x; z) = sum over
independent sets S of F of prod_{v in S} z_v x^|S|.  F holds a K4 and a 4-cycle, a
triangle with a pendant edge and a vertex of degree 5, so every subgraph type of the
inclusion-exclusion (edges, paths, stars, triangles, 4-cycles, paws, diamonds, K4) is
present in the complements of the frames, and no frame is a t-plex for t <= 3, so no
early termination closes them first.  The closed form is pinned to the oracle on small
cases (CPU test below).
"""
import itertools

import numpy as np
import pytest

import oracle as O
from synth import graphs as G

M64 = (1 << 64) - 1
F_N = 8
F_EDGES = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3),  # K4
           (3, 4), (4, 5), (5, 6), (6, 3),                  # 4-cycle through 3
           (2, 4), (6, 7)]                                  # triangle 2-3-4, pendant 6-7


def complement_of_copies(m: int, seed: int):
    """G and the vertex ids of every copy of F (copy i's vertex j is blocks[i][j])."""
    n = m * F_N
    perm = G.random_perm(n, seed, 5)
    blocks = [[int(perm[i * F_N + j]) for j in range(F_N)] for i in range(m)]
    h = set()
    for b in blocks:
        for a, c in F_EDGES:
            x, y = b[a], b[c]
            h.add((min(x, y), max(x, y)))
    u, v = [], []
    for x in range(n):
        for y in range(x + 1, n):
            if (x, y) not in h:
                u.append(x)
                v.append(y)
    return G.from_edges(n, np.array(u), np.array(v)), blocks


def _independent_sets():
    adj = {(a, c) for a, c in F_EDGES} | {(c, a) for a, c in F_EDGES}
    for r in range(F_N + 1):
        for s in itertools.combinations(range(F_N), r):
            if all((a, c) not in adj for a, c in itertools.combinations(s, 2)):
                yield s


def expected(blocks, k: int):
    """(count, checksum) of the k-cliques of the complement of the copies."""
    ind = list(_independent_sets())
    cnt = [1] + [0] * k
    cs = [1] + [0] * k
    for b in blocks:
        pc = [0] * (k + 1)
        pz = [0] * (k + 1)
        for s in ind:
            if len(s) <= k:
                pc[len(s)] += 1
                w = 1
                for j in s:
                    w = w * O.key(b[j]) & M64
                pz[len(s)] = (pz[len(s)] + w) & M64
        cnt = [sum(cnt[i] * pc[j - i] for i in range(j + 1)) for j in range(k + 1)]
        cs = [sum(cs[i] * pz[j - i] for i in range(j + 1)) & M64 for j in range(k + 1)]
    return cnt[k], cs[k]


def test_closed_form_matches_the_oracle():
    for m, seed in ((2, 1), (3, 2)):
        g, blocks = complement_of_copies(m, seed)
        for k in (3, 4, 5, 6, 7, 8):
            want = O.count(g, k, shortcut=False)
            assert expected(blocks, k) == (want["count"], want["checksum"]), (m, k)


@pytest.fixture(scope="module")
def kc():
    pytest.importorskip("torch")
    from paper_2311_13798_gb300 import kclique
    return kclique


# copies m -> largest sub-branch ~ 8m - 2 vertices: 1, 2, 4, 8, 16 and 32 bitset words
@pytest.mark.gpu
@pytest.mark.parametrize("m,ks,lo,hi", [(3, (6, 8, 9), 1, 32), (7, (6, 8), 33, 64), (14, (6, 8), 65, 128),
                                        (28, (6,), 129, 256), (40, (6,), 257, 512), (70, (6,), 513, 1024)])
def test_dense_frames_at_every_width(kc, m, ks, lo, hi):
    import torch
    g, blocks = complement_of_copies(m, seed=m)
    rp = torch.from_numpy(g.row_ptr.astype(np.int32)).cuda()
    col = torch.from_numpy(g.col.astype(np.int32)).cuda()
    h = kc.kclique_prepare(rp, col, g.n)
    assert lo <= int(kc.kclique_edge_data(h)["vset_size"].max()) <= hi
    for k in ks:
        want = expected(blocks, k)
        for t_max in (0, 2, 3):
            got = kc.kclique_count(h, k, t_max=t_max, flags=kc.KC_CHECKSUM)
            assert (got["count"], got["checksum"]) == want, (m, k, t_max)
            assert got["status"] == kc.KC_OK
        assert kc.kclique_count(h, k)["count"] == want[0], (m, k)
        got = kc.kclique_count(h, k, flags=kc.KC_CHECKSUM | kc.KC_NO_ET)
        assert (got["count"], got["checksum"]) == want, (m, k)
