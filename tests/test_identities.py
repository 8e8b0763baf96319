"""The counting identities the branch kernels use for dense l = 3 and l = 4 frames, restated in plain
Python and checked against brute force on random small graphs (CPU).

A 4-set of a frame C is a clique iff it spans no edge of the complement H, so by
inclusion-exclusion over the edge sets F of H on at most four vertices,
    #K4 = sum_F (-1)^|F| C(c - |V(F)|, 4 - |V(F)|),
and, weighting each 4-set by the product of its vertices' keys (the checksum),
    sum over K4 of z_a z_b z_c z_d = sum_F (-1)^|F| z(V(F)) e_{4-|V(F)|}(keys of C - V(F)).
The kernels evaluate both grouped by the subgraph types of H (edges, paths, stars,
triangles, disjoint edge pairs, 4-cycles, paws, diamonds, 4-cliques), element by element
and without division (mod 2^64 for the keys).  These tests restate that grouping.
"""
import itertools
import random
from math import comb as _comb

M64 = (1 << 64) - 1


def comb(n, k):
    return _comb(n, k) if n >= 0 else 0


def random_graph(rng, c, p):
    adj = [[False] * c for _ in range(c)]
    for a in range(c):
        for b in range(a + 1, c):
            if rng.random() < p:
                adj[a][b] = adj[b][a] = True
    return adj


def brute(c, adj, z=None):
    total = 0
    for q in itertools.combinations(range(c), 4):
        if all(adj[a][b] for a, b in itertools.combinations(q, 2)):
            total += 1 if z is None else z[q[0]] * z[q[1]] * z[q[2]] * z[q[3]]
    return total if z is None else total & M64


def k4_count(c, adj):
    """The count as the kernels fold it: every element of H visited once."""
    H = [[a != b and not adj[a][b] for b in range(c)] for a in range(c)]
    d = [sum(H[x]) for x in range(c)]
    M = sum(d) // 2
    total = comb(c, 4) - M * comb(c - 2, 2) + M * (M - 1) // 2
    for x in range(c):
        total += comb(d[x], 2) * (c - 4) - comb(d[x], 3)           # two-edge paths, stars
        for a in range(x + 1, c):
            if not H[x][a]:
                continue
            cm = [b for b in range(c) if H[x][b] and H[a][b]]
            total -= (d[x] - 1) * (d[a] - 1) + comb(len(cm), 2)    # three-edge paths, diamonds
            above = [b for b in cm if b > a]
            for b in above:
                total += d[x] + d[a] + d[b] - c                     # triangles, paws
                total += sum(1 for b2 in above if b2 > b and H[b][b2])   # 4-cliques of H
        for y in range(x + 1, c):                                   # 4-cycles at their least vertex
            cn = [b for b in range(x + 1, c) if b != y and H[x][b] and H[y][b]]
            total += comb(len(cn), 2)
    return total


def esym(vals, j):
    e = [1] + [0] * j
    for v in vals:
        for t in range(j, 0, -1):
            e[t] = (e[t] + e[t - 1] * v) & M64
    return e


def k4_weighted(c, adj, z):
    """The key-weighted sum as the kernels form it (mod 2^64, no division)."""
    H = [[a != b and not adj[a][b] for b in range(c)] for a in range(c)]
    N = [[b for b in range(c) if H[a][b]] for a in range(c)]
    e = esym(z, 4)
    Z, e2, e4 = e[1], e[2], e[4]
    S1 = [sum(z[b] for b in N[x]) & M64 for x in range(c)]
    total = e4
    ew1 = ew2 = 0  # e1, e2 of the H-edge weights z_x z_a
    for x in range(c):
        en = esym([z[b] for b in N[x]], 3)
        q2 = sum(z[b] ** 2 for b in N[x])
        q3 = sum(z[b] ** 3 for b in N[x])
        zx = z[x]
        total += zx * ((Z - zx) * en[2] - (S1[x] * q2 - q3)) - zx * en[3] - zx * zx * en[2]
        qx = 0
        for a in N[x]:
            cm = [b for b in N[x] if H[a][b]]
            zc_gt = sum(z[b] for b in cm if b > a)
            qx += z[a] * zc_gt
            if a < x:
                continue
            wt = zx * z[a]
            ew2 += ew1 * wt
            ew1 += wt
            e2r = e2 - (zx + z[a]) * (Z - zx - z[a]) - wt                 # e2 of C - {x, a}
            total -= wt * e2r + Z * wt * zc_gt                            # single edges, triangles
            total -= wt * ((S1[x] - z[a]) * (S1[a] - zx) - sum(z[b] ** 2 for b in cm))   # P4
            total -= wt * esym([z[b] for b in cm], 2)[2]                  # diamonds
            above = [b for b in cm if b > a]
            for b in above:
                total += wt * z[b] * sum(z[b2] for b2 in above if b2 > b and H[b][b2])   # 4-cliques of H
        total += zx * qx * (S1[x] - zx)                                   # triangle and paw terms
        for y in range(x + 1, c):                                         # 4-cycles
            cn = [b for b in range(x + 1, c) if b != y and H[x][b] and H[y][b]]
            total += zx * z[y] * esym([z[b] for b in cn], 2)[2]
    total += ew2                                                          # disjoint H-edge pairs
    return total & M64


def test_k4_identities_match_brute_force():
    rng = random.Random(20240501)
    for trial in range(250):
        c = rng.randint(0, 13)
        adj = random_graph(rng, c, rng.random())
        assert k4_count(c, adj) == brute(c, adj), trial
        z = [rng.getrandbits(64) | 1 for _ in range(c)]
        assert k4_weighted(c, adj, z) == brute(c, adj, z), trial


def test_k4_identities_on_dense_frames():
    # the regime the kernels use them in: complements sparser than a third of the pairs
    rng = random.Random(7)
    for trial in range(40):
        c = rng.randint(8, 16)
        adj = random_graph(rng, c, 0.8 + 0.2 * rng.random())
        z = [rng.getrandbits(64) | 1 for _ in range(c)]
        assert k4_count(c, adj) == brute(c, adj), trial
        assert k4_weighted(c, adj, z) == brute(c, adj, z), trial


def brute3(c, adj, z=None):
    total = 0
    for q in itertools.combinations(range(c), 3):
        if all(adj[a][b] for a, b in itertools.combinations(q, 2)):
            total += 1 if z is None else z[q[0]] * z[q[1]] * z[q[2]]
    return total if z is None else total & M64


def k3_identities(c, adj, z):
    """The l = 3 frame count and its key-weighted form through the complement H:
    #K3 = C(c,3) - |H|(c-2) + sum_x C(dbar_x, 2) - T(H), and
    e3(z) - sum_{ab in H} z_a z_b (Z - z_a - z_b) + sum_x z_x e2(keys of x's H-neighbours) - T_z(H)."""
    H = [[a != b and not adj[a][b] for b in range(c)] for a in range(c)]
    d = [sum(H[x]) for x in range(c)]
    M = sum(d) // 2
    tri_h = [(a, b, w) for a, b, w in itertools.combinations(range(c), 3) if H[a][b] and H[a][w] and H[b][w]]
    count = comb(c, 3) - M * (c - 2) + sum(comb(x, 2) for x in d) - len(tri_h)
    e = esym(z, 3)
    Z, e3 = e[1], e[3]
    w = e3
    for a, b in itertools.combinations(range(c), 2):
        if H[a][b]:
            w -= z[a] * z[b] * (Z - z[a] - z[b])
    for x in range(c):
        w += z[x] * esym([z[y] for y in range(c) if H[x][y]], 2)[2]
    for a, b, t in tri_h:
        w -= z[a] * z[b] * z[t]
    return count, w & M64


def test_k3_identities_match_brute_force():
    rng = random.Random(99)
    for trial in range(250):
        c = rng.randint(0, 14)
        adj = random_graph(rng, c, rng.random())
        z = [rng.getrandbits(64) | 1 for _ in range(c)]
        assert k3_identities(c, adj, z) == (brute3(c, adj), brute3(c, adj, z)), trial
