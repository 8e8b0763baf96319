"""Host logic of the query server (continuous batching, HBM admission, LRU eviction),
exercised on CPU with a stand-in backend whose answers come from the oracle."""
import threading
import time

import numpy as np

import oracle as O
from paper_2311_13798_gb300.serve import KCliqueServer, Request
from synth import graphs as G


class FakeBackend:
    """Answers with the oracle; each batch call sleeps so that requests pile up."""

    def __init__(self, delay=0.02):
        self.delay = delay
        self.calls = []
        self.released = []
        self.lock = threading.Lock()

    def prepare(self, rp, col, n):
        time.sleep(self.delay)
        return {"g": O.CleanGraph(n, np.asarray(rp), np.asarray(col)), "bytes": 1000 + 8 * len(col)}

    def resident_bytes(self, h):
        return h["bytes"]

    def estimate_bytes(self, rp, col, n):
        return 1000 + 8 * len(col)

    def count_batch(self, hs, ks):
        with self.lock:
            self.calls.append(len(hs))
        time.sleep(self.delay)
        return [dict(O.count(h["g"], k)) for h, k in zip(hs, ks)]

    def list(self, h, k, cap, rows_only=False):
        rows = O.list_cliques(h["g"], k)
        r = O.count(h["g"], k)
        trunc = len(rows) > cap
        if rows_only and len(rows) >= cap:  # the library stops at a full buffer, totals unknown
            return {"count": 0, "checksum": 0, "written": cap, "truncated": True}, rows[:cap]
        return {"count": r["count"], "checksum": r["checksum"], "written": min(cap, len(rows)),
                "truncated": trunc}, rows[:cap]

    def release(self, h):
        self.released.append(h)


def _csr(g):
    return (g.row_ptr, g.col, g.n)


def test_results_alone_and_in_the_mix_are_identical():
    be = FakeBackend()
    srv = KCliqueServer(be, hbm_budget_bytes=1 << 30)
    graphs = {f"g{i}": G.gnp(40 + 5 * i, 0.3, seed=i) for i in range(4)}
    for name, g in graphs.items():
        srv.register(name, *_csr(g))
    reqs = []
    for i in range(60):
        name = f"g{i % 4}"
        kind = "list" if i % 7 == 0 else "count"
        reqs.append(srv.submit(Request(kind, name, k=3 + i % 3, cap=10**6)))
    res = [f.result(timeout=60) for f in reqs]
    srv.close()
    for i, r in enumerate(res):
        g = graphs[f"g{i % 4}"]
        alone = O.count(g, 3 + i % 3)
        assert r.status == "ok"
        assert (r.count, r.checksum) == (alone["count"], alone["checksum"])
    st = srv.stats()
    assert st["queries"] == 60 and st["p50_s"] is not None and st["p99_s"] >= st["p50_s"]
    # continuous batching: queries that waited behind a running batch went together
    assert max(be.calls) > 1 and sum(be.calls) == sum(1 for i in range(60) if i % 7)


def test_upload_admission_and_lru_eviction():
    be = FakeBackend(delay=0.0)
    small = G.gnp(30, 0.3, seed=1)
    per = be.estimate_bytes(small.row_ptr, small.col, small.n)
    srv = KCliqueServer(be, hbm_budget_bytes=int(2.5 * per))
    srv.register("base", *_csr(small), pin=True)
    f1 = srv.submit(Request("upload", "u1", csr=_csr(small)))
    assert f1.result(timeout=30).status == "ok"
    f2 = srv.submit(Request("upload", "u2", csr=_csr(small)))   # evicts u1 (LRU, not pinned)
    assert f2.result(timeout=30).status == "ok"
    assert "u1" not in srv.graphs and "base" in srv.graphs and "u2" in srv.graphs
    big = G.gnp(200, 0.5, seed=2)
    f3 = srv.submit(Request("upload", "big", csr=_csr(big)))    # cannot fit even after eviction
    assert f3.result(timeout=30).status.startswith("rejected")
    assert srv.submit(Request("count", "nope", k=3)).result(timeout=5).status == "unknown graph"
    r = srv.submit(Request("count", "u2", k=3)).result(timeout=30)
    assert r.count == O.count(small, 3)["count"]
    srv.close()
    assert srv.stats()["rejected"] == 1


def test_truncated_listings_get_their_totals_from_the_count_batch():
    be = FakeBackend()
    srv = KCliqueServer(be, hbm_budget_bytes=1 << 30)
    g = G.gnp(60, 0.4, seed=5)
    srv.register("g", *_csr(g))
    futs = [srv.submit(Request("list", "g", k=k, cap=cap)) for k in (3, 4) for cap in (1, 7, 10**6)]
    futs += [srv.submit(Request("count", "g", k=3))]
    res = [f.result(timeout=60) for f in futs]
    srv.close()
    i = 0
    for k in (3, 4):
        want = O.count(g, k)
        n = len(O.list_cliques(g, k))
        for cap in (1, 7, 10**6):
            r = res[i]
            i += 1
            assert r.status == "ok" and (r.count, r.checksum) == (want["count"], want["checksum"])
            assert r.written == min(cap, n) and len(r.rows) == r.written
    assert res[-1].count == O.count(g, 3)["count"]
    # 4 truncated listings (caps 1 and 7) went through the count batches, plus the count
    assert sum(be.calls) == 5
