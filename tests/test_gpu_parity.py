"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, bit-exact.

Counts, checksums, listings, truss levels and rounds, VSet sizes and per-edge
sub-branch counts are integers, so every comparison is exact equality.  Graphs
span several bitset words and ragged tails (sub-branches of 1..300 vertices),
and the degenerate cases of the method: empty graphs, triangle-free graphs
(tau = 0), k > tau + 2, complete graphs (ET on the whole sub-branch), exact
2-plexes, t-plexes, duplicate / self-loop / one-directional input.
"""
import math

import numpy as np
import pytest

import oracle as O
from synth import graphs as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

M64 = (1 << 64) - 1


def kc():
    from paper_2311_13798_gb300 import kclique
    return kclique


def dev_csr(g):
    rp = torch.from_numpy(g.row_ptr.astype(np.int32)).cuda()
    col = torch.from_numpy(g.col.astype(np.int32)).cuda()
    return rp, col


def prep(g):
    rp, col = dev_csr(g)
    return kc().kclique_prepare(rp, col, g.n)


GRAPHS = {
    "gnp60": lambda: G.gnp(60, 0.3, seed=1),
    "gnp120_dense": lambda: G.gnp(120, 0.6, seed=2),
    "gnp400": lambda: G.gnp(400, 0.08, seed=3),
    "k40": lambda: G.complete(40),
    "k70": lambda: G.complete(70),
    "turan": lambda: G.complete_multipartite([7, 8, 9, 10, 11, 6]),
    "two_plex": lambda: G.two_plex(9, 12),
    "t3plex": lambda: G.t_plex(45, 3, seed=4),
    "appendix_b": lambda: G.appendix_b(),
    "kpp": lambda: G.complete_bipartite(12, 12),
    "chung_lu": lambda: G.chung_lu(n=4000, w_max=400.0, i0=40.0, planted=6, planted_min=12, planted_max=30, seed=5),
    "sbm": lambda: G.sbm_2plex(blocks=8, block_size=60, p_in=0.85, p_out=0.01, two_plex_blocks=3, seed=6)[0],
    "wide": lambda: G.gnp(300, 0.75, seed=7),   # sub-branches of ~170 vertices (6 words)
    "t3plex_big": lambda: G.t_plex(90, 3, seed=11),   # inverse graph: paths and cycles
    "t4plex": lambda: G.t_plex(64, 4, seed=12),
}


# largest k the oracle finishes in seconds on each graph
KMAX = {"wide": 5, "gnp400": 6, "t3plex_big": 6, "t4plex": 7}


@pytest.fixture(scope="module")
def cache():
    return {}


def get(cache, name):
    if name not in cache:
        g = GRAPHS[name]()
        cache[name] = (g, O.CleanGraph.of(g), prep(g))
    return cache[name]


@pytest.mark.parametrize("name", list(GRAPHS))
def test_prepare_matches_oracle(cache, name):
    g, cg, h = get(cache, name)
    info = kc().kclique_info(h)
    assert info["n"] == g.n and info["m"] == g.m
    ed = kc().kclique_edge_data(h)
    assert (ed["eu"] == cg.eu).all() and (ed["ev"] == cg.ev).all()
    lvl, rnd, nr = O.truss_peel(cg)
    assert (ed["level"] == lvl).all()
    assert (ed["round"] == rnd).all()
    assert info["rounds"] == nr
    vs = O.vset_sizes(cg, rnd)
    assert (ed["vset_size"] == vs).all()
    assert info["triangles"] == int(vs.sum()) == O.count(cg, 3)["count"]
    assert info["tau"] == (int(lvl.max()) if lvl.size else 0)


@pytest.mark.parametrize("name", list(GRAPHS))
def test_count_and_checksum(cache, name):
    g, cg, h = get(cache, name)
    tau = kc().kclique_info(h)["tau"]
    for k in range(3, KMAX.get(name, 9) + 1):
        want = O.count(cg, k)
        got = kc().kclique_count(h, k, flags=kc().KC_CHECKSUM)
        assert got["count"] == want["count"], (name, k)
        assert got["checksum"] == want["checksum"], (name, k)
        # count-only mode takes other kernel paths (l = 3 frames counted directly)
        assert kc().kclique_count(h, k)["count"] == want["count"], (name, k)
        if k > tau + 2:
            assert got["count"] == 0


@pytest.mark.parametrize("name", ["gnp120_dense", "k40", "two_plex", "t3plex", "chung_lu", "sbm", "wide"])
@pytest.mark.parametrize("flags", [0x1, 0x2, 0x8, 0x1 | 0x2 | 0x8])
def test_ablation_flags_do_not_change_results(cache, name, flags):
    g, cg, h = get(cache, name)
    K = kc()
    for k in range(4, min(KMAX.get(name, 7), 7) + 1):
        want = O.count(cg, k)
        got = K.kclique_count(h, k, flags=flags | K.KC_CHECKSUM)
        assert (got["count"], got["checksum"]) == (want["count"], want["checksum"]), (name, k, flags)
        assert K.kclique_count(h, k, flags=flags)["count"] == want["count"], (name, k, flags)


@pytest.mark.parametrize("t_max", [1, 2, 3, 0])
def test_early_termination_thresholds(cache, t_max):
    """t_max 1..3 and 0 (the paper's rule: t = 2 if k <= tau/2, else 3) give the oracle's
    results; t = 3 closes 3-plex frames through the inverse graph's paths and cycles."""
    for name in ("k70", "two_plex", "t3plex", "t3plex_big", "t4plex", "sbm", "gnp120_dense"):
        g, cg, h = get(cache, name)
        for k in (4, 5, 6, 7):
            if k > KMAX.get(name, 9):
                continue
            want = O.count(cg, k)
            got = kc().kclique_count(h, k, t_max=t_max, flags=kc().KC_CHECKSUM)
            assert (got["count"], got["checksum"]) == (want["count"], want["checksum"]), (name, k, t_max)
            assert kc().kclique_count(h, k, t_max=t_max)["count"] == want["count"], (name, k, t_max)
            for split_min in (3, 0xFFFFFFFF):
                r = kc().kclique_count(h, k, t_max=t_max, split_min=split_min, flags=kc().KC_CHECKSUM)
                assert (r["count"], r["checksum"]) == (want["count"], want["checksum"]), (name, k, t_max)


def test_early_termination_fires_on_cliques_and_plexes(cache):
    for name in ("k70", "two_plex"):
        g, cg, h = get(cache, name)
        got = kc().kclique_count(h, 6)
        assert got["et_hits"] > 0
    # a 3-plex: every sub-branch is a 3-plex, closed at its top frame with t = 3 only
    # (at k = 5 the top frame already has l = 3, which the l = 3 routine counts exactly
    # whatever t is, so the difference shows from k = 6 on, as more frames closed early)
    g, cg, h = get(cache, "t3plex_big")
    for k in (5, 6):
        t2 = kc().kclique_count(h, k, t_max=2)
        t3 = kc().kclique_count(h, k, t_max=3)
        assert t3["count"] == t2["count"] == O.count(cg, k)["count"]
        if k >= 6:
            assert t3["et_hits"] > t2["et_hits"]


@pytest.mark.parametrize("name", ["gnp60", "gnp120_dense", "k40", "turan", "two_plex", "t3plex", "appendix_b",
                                  "chung_lu", "sbm"])
def test_list_matches_oracle(cache, name):
    g, cg, h = get(cache, name)
    for k in (3, 4, 5, 6):
        want = O.count(cg, k)
        cap = max(want["count"], 1)
        if cap > 3_000_000:
            continue
        out = torch.full((cap, k), -1, dtype=torch.int32, device="cuda")
        got = kc().kclique_list(h, k, out)
        assert not got["truncated"]
        assert got["count"] == want["count"] and got["written"] == want["count"]
        assert got["checksum"] == want["checksum"]
        rows = out[: got["written"]].cpu().numpy().astype(np.int64)
        if rows.size:
            assert (np.diff(rows, axis=1) > 0).all()
        ref = O.list_cliques(cg, k).astype(np.int64)
        assert sorted(map(tuple, rows.tolist())) == sorted(map(tuple, ref.tolist()))


def test_list_truncation_keeps_full_count(cache):
    g, cg, h = get(cache, "gnp120_dense")
    k = 5
    want = O.count(cg, k)
    cap = want["count"] // 3
    out = torch.zeros((cap, k), dtype=torch.int32, device="cuda")
    got = kc().kclique_list(h, k, out)
    assert got["truncated"] and got["written"] == cap
    assert got["count"] == want["count"] and got["checksum"] == want["checksum"]
    rows = set(map(tuple, out.cpu().numpy().astype(np.int64).tolist()))
    ref = set(map(tuple, O.list_cliques(cg, k).astype(np.int64).tolist()))
    assert len(rows) == cap and rows <= ref


def test_rows_only_listing(cache):
    """KC_ROWS_ONLY: a full buffer ends the pass with KC_TRUNCATED and no totals; a buffer
    that holds every clique gives the exact totals as a normal listing does."""
    K = kc()
    g, cg, h = get(cache, "gnp120_dense")
    k = 5
    want = O.count(cg, k)
    ref = set(map(tuple, O.list_cliques(cg, k).astype(np.int64).tolist()))
    cap = want["count"] // 5
    out = torch.zeros((cap, k), dtype=torch.int32, device="cuda")
    got = K.kclique_list(h, k, out, flags=K.KC_ROWS_ONLY)
    assert got["truncated"] and got["written"] == cap and got["count"] == 0 and got["checksum"] == 0
    rows = set(map(tuple, out.cpu().numpy().astype(np.int64).tolist()))
    assert len(rows) == cap and rows <= ref
    out = torch.zeros((want["count"] + 7, k), dtype=torch.int32, device="cuda")
    got = K.kclique_list(h, k, out, flags=K.KC_ROWS_ONLY)
    assert not got["truncated"] and (got["count"], got["checksum"]) == (want["count"], want["checksum"])
    assert set(map(tuple, out[: got["written"]].cpu().numpy().astype(np.int64).tolist())) == ref


def test_concurrent_listings_from_host_threads(cache):
    """Listings and counts issued at once from several host threads, each on its own
    stream (the server's list workers), give the same results as alone."""
    import concurrent.futures as cf
    K = kc()
    names = ["gnp120_dense", "chung_lu", "sbm", "two_plex"]
    want = {}
    for name in names:
        g, cg, h = get(cache, name)
        for k in (4, 5, 6):
            want[(name, k)] = O.count(cg, k)

    def job(name, k, cap):
        torch.cuda.set_device(0)
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            h = get(cache, name)[2]
            out = torch.empty((cap, k), dtype=torch.int32, device="cuda")
            r = K.kclique_list(h, k, out, stream=st)
            c = K.kclique_count(h, k, stream=st, flags=K.KC_CHECKSUM)
        return name, k, r, c

    jobs = [(n, k, cap) for n in names for k in (4, 5, 6) for cap in (1, 1000)]
    with cf.ThreadPoolExecutor(6) as ex:
        for name, k, r, c in ex.map(lambda j: job(*j), jobs * 2):
            w = want[(name, k)]
            assert (r["count"], r["checksum"]) == (w["count"], w["checksum"]), (name, k)
            assert (c["count"], c["checksum"]) == (w["count"], w["checksum"]), (name, k)


def test_per_edge_counts(cache):
    for name in ("chung_lu", "sbm", "gnp120_dense"):
        g, cg, h = get(cache, name)
        _, rnd, _ = O.truss_peel(cg)
        m = g.m
        for k in (4, 6, 7):
            ec = torch.zeros(m, dtype=torch.int64, device="cuda")
            es = torch.zeros(m, dtype=torch.int64, device="cuda")
            got = kc().kclique_count(h, k, edge_count=ec, edge_checksum=es, flags=kc().KC_CHECKSUM)
            ec2 = torch.zeros(m, dtype=torch.int64, device="cuda")
            kc().kclique_count(h, k, edge_count=ec2)
            assert torch.equal(ec, ec2)
            rng = np.random.default_rng(k)
            sample = np.unique(np.concatenate([rng.choice(m, size=min(m, 150), replace=False),
                                               np.argsort(-O.vset_sizes(cg, rnd))[:20]]))
            cnt, cs = O.edge_counts(cg, k, rnd, sample)
            gc = ec.cpu().numpy().view(np.uint64)
            gs = es.cpu().numpy().view(np.uint64)
            assert [int(x) for x in gc[sample]] == cnt
            assert [int(x) for x in gs[sample]] == cs
            assert int(gc.astype(object).sum()) == got["count"]


def test_host_input_and_dirty_csr():
    """Host arrays, duplicates, self-loops and one-directional edges are cleaned."""
    g = G.gnp(150, 0.3, seed=9)
    u, v = g.edges()
    rng = np.random.default_rng(0)
    # keep each edge in one random direction, add duplicates and self loops
    flip = rng.random(u.size) < 0.5
    a = np.where(flip, v, u)
    b = np.where(flip, u, v)
    dup = rng.choice(u.size, 200)
    a = np.concatenate([a, a[dup], np.arange(20)])
    b = np.concatenate([b, b[dup], np.arange(20)])
    order = np.argsort(a, kind="stable")
    a, b = a[order], b[order]
    rp = np.zeros(g.n + 1, dtype=np.uint32)
    rp[1:] = np.cumsum(np.bincount(a, minlength=g.n))
    K = kc()
    h = K.kclique_prepare(rp, b.astype(np.uint32), g.n)
    assert K.kclique_info(h)["m"] == g.m
    for k in (3, 4, 5):
        want = O.count(g, k)
        got = K.kclique_count(h, k, flags=K.KC_CHECKSUM)
        assert (got["count"], got["checksum"]) == (want["count"], want["checksum"])


def test_empty_and_invalid():
    K = kc()
    h = K.kclique_prepare(np.zeros(6, np.uint32), np.zeros(0, np.uint32), 5)
    assert K.kclique_info(h)["m"] == 0
    assert K.kclique_count(h, 3)["count"] == 0
    with pytest.raises(K.KCliqueError):
        K.kclique_count(h, 2)
    with pytest.raises(K.KCliqueError):
        K.kclique_count(h, 33)
    with pytest.raises(K.KCliqueError):  # column id out of range
        K.kclique_prepare(np.array([0, 1], np.uint32), np.array([5], np.uint32), 1)
    with pytest.raises(K.KCliqueError):  # row_ptr not monotone
        K.kclique_prepare(np.array([0, 2, 1], np.uint32), np.array([1, 0], np.uint32), 2)


def test_relabel_invariance():
    g = G.gnp(200, 0.25, seed=10)
    perm = G.random_perm(200, 1, 2)
    h1, h2 = prep(g), prep(G.relabel(g, perm))
    for k in (4, 5, 6):
        a = kc().kclique_count(h1, k)["count"]
        b = kc().kclique_count(h2, k)["count"]
        assert a == b == O.count(g, k)["count"]


def test_batch_matches_single(cache):
    names = ["gnp60", "k40", "two_plex", "chung_lu", "sbm", "kpp", "appendix_b"]
    hs, ks, want = [], [], []
    for i, name in enumerate(names * 2):
        g, cg, h = get(cache, name)
        k = 3 + (i % 6)
        hs.append(h)
        ks.append(k)
        want.append(O.count(cg, k))
    K = kc()
    res = K.kclique_count_batch(hs, ks, flags=K.KC_CHECKSUM)
    for r, w in zip(res, want):
        assert (r["count"], r["checksum"]) == (w["count"], w["checksum"])


def test_overflow_is_reported():
    # K_300: C(300, 30) ~ 1.7e41 > 2^128 closed forms saturate -> KC_ERR_OVERFLOW
    K = kc()
    h = prep(G.complete(300))
    with pytest.raises(K.KCliqueError) as ei:
        K.kclique_count(h, 32)
    assert ei.value.status == K.KC_ERR_OVERFLOW


def test_large_counts_exceed_64_bits():
    """K_200 at k = 20: C(200, 20) = 1.6e27 > 2^64, exact in 128 bits."""
    import math
    K = kc()
    h = prep(G.complete(200))
    got = K.kclique_count(h, 20, flags=K.KC_CHECKSUM)
    assert got["count"] == math.comb(200, 20)
    assert got["checksum"] == O.count(G.complete(200), 20)["checksum"]


@pytest.mark.parametrize("name", ["gnp120_dense", "k70", "two_plex", "t3plex", "chung_lu", "sbm", "turan"])
def test_split_sub_branches_match(cache, name):
    """Heavy sub-branches split into per-vertex work items (forced with a tiny
    split_min) give the same counts, checksums and per-edge counts as unsplit runs."""
    g, cg, h = get(cache, name)
    K = kc()
    _, rnd, _ = O.truss_peel(cg)
    for k in (7, 8, 9):
        want = O.count(cg, k)
        for split_min in (3, 16, 0xFFFFFFFF):
            got = K.kclique_count(h, k, split_min=split_min, flags=K.KC_CHECKSUM)
            assert (got["count"], got["checksum"]) == (want["count"], want["checksum"]), (name, k, split_min)
            assert K.kclique_count(h, k, split_min=split_min)["count"] == want["count"]
        ec = torch.zeros(g.m, dtype=torch.int64, device="cuda")
        K.kclique_count(h, k, split_min=3, edge_count=ec)
        sample = np.argsort(-O.vset_sizes(cg, rnd))[:25]
        cnt, _ = O.edge_counts(cg, k, rnd, sample)
        assert [int(x) for x in ec.cpu().numpy().view(np.uint64)[sample]] == cnt


def test_ticket_shards_add_up(cache):
    """Disjoint shards of the ticket order (one per GPU of a multi-GPU run) sum to the whole."""
    K = kc()
    for name in ("chung_lu", "sbm", "gnp120_dense"):
        g, cg, h = get(cache, name)
        m = g.m
        for k in (4, 5, 7):
            whole = K.kclique_count(h, k, flags=K.KC_CHECKSUM)
            cuts = [0, 3, 40, m // 3, m]
            parts = [K.kclique_count(h, k, ticket_begin=a, ticket_end=b, flags=K.KC_CHECKSUM)
                     for a, b in zip(cuts[:-1], cuts[1:]) if b > a]
            assert sum(p["count"] for p in parts) == whole["count"]
            assert sum(p["checksum"] for p in parts) % (1 << 64) == whole["checksum"]


def test_size_range_shards_add_up(cache):
    """The multi-GPU split: ticket ranges cut between |VSet| sizes (the same edge sets on
    every replica of a prepared graph) count the whole graph between them."""
    from paper_2311_13798_gb300 import shard
    K = kc()
    for name in ("chung_lu", "sbm", "gnp400"):
        g, cg, h = get(cache, name)
        vs = K.kclique_edge_data(h)["vset_size"]
        for k in (4, 5, 7):
            want = O.count(cg, k)
            for n in (2, 3, 8):
                parts = [K.kclique_count(h, k, ticket_begin=b, ticket_end=e, flags=K.KC_CHECKSUM)
                         for b, e in shard.partition_by_size(vs, k, n) if e > b]
                limbs = [0] * 6  # no shard has work when k > tau + 2
                for p in parts:
                    limbs = [a + b for a, b in zip(limbs, shard.to_limbs(p["count"], p["checksum"]))]
                assert shard.from_limbs(limbs) == (want["count"], want["checksum"]), (name, k, n)


@pytest.mark.parametrize("name", ["gnp60", "gnp120_dense", "k40", "turan", "two_plex", "t3plex", "chung_lu", "sbm",
                                  "appendix_b", "kpp", "wide"])
def test_colour_based_ordering_matches_oracle(cache, name):
    """EBBkC-C's top level (the colour-based edge order, Sec. 4.3) reaches the same
    k-cliques as the truss-based order: counts, checksums and listings equal the oracle's."""
    g, cg, h = get(cache, name)
    K = kc()
    rp, col = dev_csr(g)
    hc = K.kclique_prepare(rp, col, g.n, ordering=K.KC_ORDER_COLOUR)
    for k in range(3, min(KMAX.get(name, 7), 7) + 1):
        want = O.count(cg, k)
        got = K.kclique_count(hc, k, flags=K.KC_CHECKSUM)
        assert (got["count"], got["checksum"]) == (want["count"], want["checksum"]), (name, k)
        for split_min in (3, 0xFFFFFFFF):
            r = K.kclique_count(hc, k, split_min=split_min, flags=K.KC_CHECKSUM)
            assert (r["count"], r["checksum"]) == (want["count"], want["checksum"]), (name, k, split_min)
    k = 4
    want = O.count(cg, k)
    if 0 < want["count"] <= 200_000:
        out = torch.full((want["count"], k), -1, dtype=torch.int32, device="cuda")
        got = K.kclique_list(hc, k, out)
        rows = sorted(map(tuple, out.cpu().numpy().astype(np.int64).tolist()))
        assert rows == sorted(map(tuple, O.list_cliques(cg, k).astype(np.int64).tolist()))


@pytest.mark.parametrize("name", ["gnp60", "gnp120_dense", "k40", "turan", "two_plex", "t3plex", "chung_lu", "sbm",
                                  "appendix_b", "kpp", "wide"])
def test_truss_order_at_every_level_matches_oracle(cache, name):
    """EBBkC-T (Alg. 3): every level of the branching in the global truss-based edge
    order, a child's graph being V(g) & VSet(e) with the edges of g after e.  A different
    partition of the cliques than EBBkC-H's; the same counts and checksums."""
    g, cg, h = get(cache, name)
    K = kc()
    for k in range(3, min(KMAX.get(name, 6), 6) + 1):
        want = O.count(cg, k)
        got = K.kclique_count(h, k, flags=K.KC_CHECKSUM | K.KC_TRUSS_INNER)
        assert (got["count"], got["checksum"]) == (want["count"], want["checksum"]), (name, k)
        assert K.kclique_count(h, k, flags=K.KC_TRUSS_INNER)["count"] == want["count"], (name, k)


def test_truss_order_at_every_level_wide_and_invalid():
    """K300: sub-branches of up to 298 vertices (16 bitset words); C(300, k) cliques with
    checksum e_k of the keys.  Listing and per-edge outputs are refused with this flag."""
    K = kc()
    h = prep(G.complete(300))
    keys = [O.key(v) for v in range(300)]
    for k in (3, 4):
        e = [1] + [0] * k
        for x in keys:
            for j in range(k, 0, -1):
                e[j] = (e[j] + e[j - 1] * x) & M64
        got = K.kclique_count(h, k, flags=K.KC_CHECKSUM | K.KC_TRUSS_INNER)
        assert (got["count"], got["checksum"]) == (math.comb(300, k), e[k]), k
    out = torch.empty((16, 4), dtype=torch.int32, device="cuda")
    with pytest.raises(K.KCliqueError):
        K.kclique_list(h, 4, out, flags=K.KC_TRUSS_INNER)
    per_edge = torch.empty(int(K.kclique_info(h)["m"]), dtype=torch.int64, device="cuda")
    with pytest.raises(K.KCliqueError):
        K.kclique_count(h, 4, flags=K.KC_TRUSS_INNER, edge_count=per_edge)


def test_batch_plan_replays_match_oracle(cache):
    """A batch captured once as a CUDA graph (kclique_batch_plan_*) and replayed: every
    replay gives the oracle's counts and checksums, also with split sub-branches (the
    item kernel inside the graph) and with a query that has no k-clique (k > tau + 2)."""
    K = kc()
    hs, ks, wants, choices = [], [], [], []
    for name in ("gnp60", "k40", "two_plex", "chung_lu", "sbm", "wide", "kpp"):
        g, cg, h = get(cache, name)
        for k in (4, 5, 7):
            if k > KMAX.get(name, 9):
                continue
            want = O.count(cg, k)
            hs.append(h)
            ks.append(k)
            wants.append((want["count"], want["checksum"]))
            choices.append({"split_min": 3} if k >= 7 else {})
    plan = K.kclique_batch_plan_create(hs, ks, choices=choices, flags=K.KC_CHECKSUM)
    try:
        for _ in range(3):
            got = plan.run()
            assert [(r["count"], r["checksum"]) for r in got] == wants
    finally:
        plan.release()
    once = K.kclique_count_batch(hs, ks, choices=choices, flags=K.KC_CHECKSUM)
    assert [(r["count"], r["checksum"]) for r in once] == wants
