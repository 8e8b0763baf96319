"""Write stored expected values for the full-size workloads into tests/golden/configs.json.

Calls only ``oracle`` (and the seeded generators in ``synth``); nothing here comes
from the GPU path.  Each entry records the graph fingerprint (so a test can tell a
generator mismatch from a parity failure), the oracle's count and checksum, the
wall time and the thread count.  Entries are merged into the file one at a time,
so a long run can be stopped and resumed.

    python oracle/make_golden.py c1            # seconds
    python oracle/make_golden.py c2 5 7 9      # minutes to hours
    python oracle/make_golden.py c2edges 9     # per-edge sub-branch values at k = 9
    python oracle/make_golden.py c3blocks 6 7  # per-block values for the SBM workload
    python oracle/make_golden.py c3plex        # closed forms of its 2-plex blocks, k = 6..10
    python oracle/make_golden.py c3cross       # its cliques with an inter-block edge, k = 6..10
    python oracle/make_golden.py c3dense 6     # every dense block at k (resumable; hours)

The SBM workload (50,000 vertices, 200 blocks of 250) is pinned as a decomposition:
every k-clique either lies inside one block or holds an inter-block edge, so
    count(G) = sum over blocks of count(block) + count(cliques with an inter-block edge),
and the same for the checksum (mod 2^64), block graphs keeping the original ids.
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
from synth import graphs as G  # noqa: E402

PATH = os.path.join(ROOT, "tests", "golden", "configs.json")
VSET_CAP = 100


def _load():
    if os.path.exists(PATH):
        return json.load(open(PATH))
    return {"note": "written by oracle/make_golden.py from the CPU oracle only; counts are decimal strings"}


def _store(key, val):
    d = _load()
    d[key] = val
    tmp = PATH + ".tmp"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, PATH)
    print(key, val, flush=True)


def _graph_entry(name, g):
    cg = O.CleanGraph.of(g)
    t = time.time()
    lvl, rnd, nr = O.truss_peel(cg)
    tp = time.time() - t
    tri = O.count(cg, 3)
    _store(f"{name}/graph", {"fingerprint": g.fingerprint(), "n": g.n, "m": g.m,
                             "tau": int(lvl.max()) if lvl.size else 0, "rounds": nr,
                             "triangles": str(tri["count"]), "triangle_checksum": str(tri["checksum"]),
                             "degeneracy": tri["degeneracy"], "peel_s": round(tp, 2)})
    return cg


def _count_entry(name, cg, k, threads):
    t = time.time()
    r = O.count(cg, k, shortcut=True, checksum=True, threads=threads)
    _store(f"{name}/k{k}", {"count": str(r["count"]), "checksum": str(r["checksum"]),
                            "wall_s": round(time.time() - t, 2), "threads": threads})


def main(argv):
    what = argv[0]
    ks = [int(x) for x in argv[1:]]
    threads = int(os.environ.get("ORACLE_THREADS", O.threads_default()))
    if what == "c1":
        g = G.config1()
        cg = _graph_entry("c1", g)
        for k in ks or [3, 4]:
            _count_entry("c1", cg, k, threads)
    elif what == "c2":
        g = G.chung_lu()
        cg = _graph_entry("c2", g)
        for k in ks or [5, 7, 9]:
            _count_entry("c2", cg, k, threads)
    elif what == "c2edges":
        # per-edge sub-branch counts (Eq. 2) for a deterministic sample of edges: the 8
        # largest VSets of at most VSET_CAP vertices (ties by edge id) and 40 random edges
        # with k-2 <= |VSet| <= VSET_CAP.  The cap keeps the oracle to minutes: at k = 9 one
        # sub-branch of 100 vertices in this graph's core already takes ~20 s on one core
        # and the work grows steeply with |VSet| (the largest is 246)
        g = G.chung_lu()
        cg = O.CleanGraph.of(g)
        lvl, rnd, _ = O.truss_peel(cg)
        vs = O.vset_sizes(cg, rnd).astype(np.int64)
        for k in ks or [9]:
            capped = np.where(vs <= VSET_CAP, vs, -1)
            order = np.lexsort((np.arange(vs.size), -capped))
            heavy = order[:8]
            rng = np.random.default_rng(k)
            cand = np.nonzero((vs >= k - 2) & (vs <= VSET_CAP))[0]
            rand = np.sort(rng.choice(cand, size=min(40, cand.size), replace=False))
            edges = np.unique(np.concatenate([heavy, rand]))
            t = time.time()
            cnt, cs = O.edge_counts(cg, k, rnd, edges, threads=threads)
            _store(f"c2/edges_k{k}", {"edges": edges.tolist(), "vset": vs[edges].tolist(),
                                      "count": [str(c) for c in cnt], "checksum": [str(c) for c in cs],
                                      "wall_s": round(time.time() - t, 2), "threads": threads})
    elif what == "c3blocks":
        g, info = G.sbm_2plex()
        _store("c3/graph", {"fingerprint": g.fingerprint(), "n": g.n, "m": g.m,
                            "two_plex_blocks": info["two_plex_blocks"]})
        blk = info["block_of"]
        u, v = g.edges()
        for b in [0, 1] + info["two_plex_blocks"][:2]:
            keep = (blk[u] == b) & (blk[v] == b)
            sub = G.from_edges(g.n, u[keep], v[keep])
            cg = O.CleanGraph.of(sub)
            for k in ks or [6, 7]:
                _count_entry(f"c3/block{b}", cg, k, threads)
    elif what in ("c3plex", "c3cross", "c3dense"):
        g, info = G.sbm_2plex()
        _store("c3/graph", {"fingerprint": g.fingerprint(), "n": g.n, "m": g.m,
                            "two_plex_blocks": info["two_plex_blocks"]})
        blk = info["block_of"]
        u, v = g.edges()
        if what == "c3plex":
            # each 2-plex block: K_250 minus a matching, closed form (pinned against
            # enumeration in tests/test_oracle_pins.py)
            out = {}
            t = time.time()
            for b in info["two_plex_blocks"]:
                keep = (blk[u] == b) & (blk[v] == b)
                sub = G.from_edges(g.n, u[keep], v[keep])
                out[str(b)] = {str(k): [str(r["count"]), str(r["checksum"])]
                               for k in (ks or range(6, 11))
                               for r in [O.sparse_complement_count(sub, k)]}
            _store("c3/plex_blocks", {"blocks": out, "wall_s": round(time.time() - t, 2)})
        elif what == "c3cross":
            # cliques with at least one inter-block edge: put every inter-block edge first
            # in the edge order (round 0, the rest round 1); the sub-branches of Eq. 2 then
            # list each such clique exactly once, at its first inter-block edge
            cg = O.CleanGraph.of(g)
            cross = blk[cg.eu] != blk[cg.ev]
            rounds = np.where(cross, 0, 1).astype(np.uint32)
            edges = np.nonzero(cross)[0]
            for k in ks or range(6, 11):
                t = time.time()
                cnt, cs = O.edge_counts(cg, k, rounds, edges, threads=threads)
                _store(f"c3/cross_k{k}", {"count": str(sum(cnt)), "checksum": str(sum(cs) & ((1 << 64) - 1)),
                                          "cross_edges": int(edges.size), "wall_s": round(time.time() - t, 2),
                                          "threads": threads})
        else:
            dense = [b for b in range(200) if b not in set(info["two_plex_blocks"])]
            have = _load()
            for k in ks or [6]:
                for b in dense:
                    key = f"c3/dense{b}/k{k}"
                    if key in have:
                        continue
                    keep = (blk[u] == b) & (blk[v] == b)
                    sub = G.from_edges(g.n, u[keep], v[keep])
                    _count_entry(f"c3/dense{b}", O.CleanGraph.of(sub), k, threads)
    else:
        raise SystemExit(__doc__)


if __name__ == "__main__":
    main(sys.argv[1:])
