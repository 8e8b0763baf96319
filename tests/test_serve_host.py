"""Host logic of the query server (continuous batching, HBM admission, LRU eviction,
listing totals), exercised on CPU: the library's server threads (kc_server_*) drive a
stand-in backend whose answers come from the oracle, through the C callbacks."""
import threading
import time

import numpy as np
import pytest

import oracle as O
from synth import graphs as G


def _server(*a, **kw):
    try:
        from paper_2311_13798_gb300.serve import KCliqueServer
        return KCliqueServer(*a, **kw)
    except RuntimeError as e:  # the library is not built here
        pytest.skip(str(e))


def _req(*a, **kw):
    from paper_2311_13798_gb300.serve import Request
    return Request(*a, **kw)


class FakeBackend:
    """Answers with the oracle; each batch call sleeps so that requests pile up."""

    def __init__(self, delay=0.02):
        self.delay = delay
        self.calls = []
        self.released = []
        self.lock = threading.Lock()

    @staticmethod
    def estimate(rp, col, n):
        # the server's admission estimate for an upload of this size
        return 4 * (n + 1) + 12 * len(col) + 28 * (len(col) // 2) + 16 * len(col)

    def prepare(self, rp, col, n):
        time.sleep(self.delay)
        return {"g": O.CleanGraph(n, np.asarray(rp), np.asarray(col)), "n": n}, self.estimate(rp, col, n)

    def count_batch(self, hs, ks):
        with self.lock:
            self.calls.append(len(hs))
        time.sleep(self.delay)
        return [dict(O.count(h["g"], k)) for h, k in zip(hs, ks)]

    def list(self, h, k, cap):
        rows = O.list_cliques(h["g"], k)
        if len(rows) >= cap:  # the library stops at a full buffer, totals unknown
            return {"count": 0, "checksum": 0, "truncated": True}, rows[:cap]
        r = O.count(h["g"], k)
        return {"count": r["count"], "checksum": r["checksum"], "truncated": False}, rows

    def release(self, h):
        with self.lock:
            self.released.append(h["n"])


def _csr(g):
    return (g.row_ptr, g.col, g.n)


def test_results_alone_and_in_the_mix_are_identical():
    be = FakeBackend()
    srv = _server(be, hbm_budget_bytes=1 << 30)
    graphs = {f"g{i}": G.gnp(40 + 5 * i, 0.3, seed=i) for i in range(4)}
    for name, g in graphs.items():
        srv.register(name, *_csr(g))
    reqs = []
    for i in range(60):
        name = f"g{i % 4}"
        kind = "list" if i % 7 == 0 else "count"
        reqs.append(srv.submit(_req(kind, name, k=3 + i % 3, cap=10**6)))
    res = [f.result(timeout=60) for f in reqs]
    srv.close()
    for i, r in enumerate(res):
        g = graphs[f"g{i % 4}"]
        alone = O.count(g, 3 + i % 3)
        assert r.status == "ok"
        assert (r.count, r.checksum) == (alone["count"], alone["checksum"])
        if i % 7 == 0:
            want = sorted(map(tuple, O.list_cliques(g, 3 + i % 3).tolist()))
            assert sorted(map(tuple, np.asarray(r.rows).tolist())) == want
    st = srv.stats()
    assert st["queries"] == 60 and st["p50_s"] is not None and st["p99_s"] >= st["p50_s"]
    # continuous batching: queries that waited behind a running batch went together
    assert max(be.calls) > 1 and sum(be.calls) == sum(1 for i in range(60) if i % 7)
    assert st["batches"] == len(be.calls)


def test_upload_admission_and_lru_eviction():
    be = FakeBackend(delay=0.0)
    small = G.gnp(30, 0.3, seed=1)
    per = be.estimate(*_csr(small))
    srv = _server(be, hbm_budget_bytes=int(2.5 * per))
    srv.register("base", *_csr(small), pin=True)
    f1 = srv.submit(_req("upload", "u1", csr=_csr(small)))
    assert f1.result(timeout=30).status == "ok"
    f2 = srv.submit(_req("upload", "u2", csr=_csr(small)))   # evicts u1 (LRU, not pinned)
    assert f2.result(timeout=30).status == "ok"
    assert len(be.released) == 1 and srv.counters()["evictions"] == 1 and srv.counters()["graphs"] == 2
    big = G.gnp(200, 0.5, seed=2)
    f3 = srv.submit(_req("upload", "big", csr=_csr(big)))    # cannot fit even after eviction
    assert f3.result(timeout=30).status.startswith("rejected")
    assert len(be.released) == 1                             # nothing released for it
    assert srv.submit(_req("count", "nope", k=3)).result(timeout=5).status == "unknown graph"
    r = srv.submit(_req("count", "u2", k=3)).result(timeout=30)
    assert r.count == O.count(small, 3)["count"]
    # a query on an upload still being prepared waits for it
    g3 = G.gnp(25, 0.4, seed=3)
    be.delay = 0.2
    fu = srv.submit(_req("upload", "u3", csr=_csr(g3)))
    fq = srv.submit(_req("count", "u3", k=3))
    assert fq.result(timeout=30).count == O.count(g3, 3)["count"] and fu.result(timeout=30).status == "ok"
    srv.close()
    assert srv.stats()["rejected"] == 1


def test_truncated_listings_get_their_totals_from_the_count_batch():
    be = FakeBackend()
    srv = _server(be, hbm_budget_bytes=1 << 30)
    g = G.gnp(60, 0.4, seed=5)
    srv.register("g", *_csr(g))
    futs = [srv.submit(_req("list", "g", k=k, cap=cap)) for k in (3, 4) for cap in (1, 7, 10**6)]
    futs += [srv.submit(_req("count", "g", k=3))]
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


def test_invalid_requests():
    from paper_2311_13798_gb300 import kclique as K
    be = FakeBackend(delay=0.0)
    srv = _server(be)
    srv.register("g", *_csr(G.gnp(20, 0.3, seed=1)))
    with pytest.raises(K.KCliqueError):
        srv.submit(_req("count", "g", k=2))
    srv.close()


class RecordingBackend(FakeBackend):
    """FakeBackend that logs when prepares and count batches start and end."""

    def __init__(self, prepare_delay):
        super().__init__(delay=0.0)
        self.prepare_delay = prepare_delay
        self.log = []

    def prepare(self, rp, col, n):
        self.log.append(("prepare_start", time.perf_counter()))
        time.sleep(self.prepare_delay)
        out = super().prepare(rp, col, n)
        self.log.append(("prepare_end", time.perf_counter()))
        return out

    def count_batch(self, hs, ks):
        self.log.append(("batch_start", time.perf_counter()))
        return super().count_batch(hs, ks)

    def when(self, what):
        return [t for w, t in self.log if w == what]


@pytest.mark.parametrize("yield_ms,expect", [(0, "after"), (0xFFFFFFFF, "during"), (50, "during")])
def test_count_batches_wait_for_uploads_in_flight(yield_ms, expect):
    """Short work first: a count batch waits while an upload is being prepared, at most
    yield_ms (0 = the default, 1000 ms; KC_SERVER_NO_YIELD = it never waits)."""
    be = RecordingBackend(prepare_delay=0.4)
    srv = _server(be, hbm_budget_bytes=1 << 30, yield_ms=yield_ms)
    base = G.gnp(30, 0.3, seed=1)
    srv.register("base", *_csr(base))
    be.log.clear()  # registration prepares too
    up = G.gnp(25, 0.4, seed=2)
    fu = srv.submit(_req("upload", "u", csr=_csr(up)))
    time.sleep(0.05)  # the upload is being prepared
    fc = srv.submit(_req("count", "base", k=3))
    assert fc.result(timeout=30).count == O.count(base, 3)["count"]
    assert fu.result(timeout=30).status == "ok"
    srv.close()
    (p_end,), (b_start,) = be.when("prepare_end"), be.when("batch_start")
    if expect == "after":
        assert b_start >= p_end
    else:
        assert b_start < p_end
