"""The continuous-batching server (kc_server_* through its Python binding) on the GPU:
a mixed burst of count, list and upload requests over several graphs, each result
against the CPU oracle and against the same request run alone through kclique_count /
kclique_list, exact integer equality (tolerance zero)."""
import numpy as np
import pytest

import oracle as O
from synth import graphs as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_server_mixed_burst_matches_oracle_alone_and_in_the_mix():
    from paper_2311_13798_gb300 import kclique as K
    from paper_2311_13798_gb300.serve import KCliqueServer, Request
    torch.cuda.set_device(0)
    base = {
        "gnp": G.gnp(120, 0.6, seed=2),
        "cl": G.chung_lu(n=4000, w_max=400.0, i0=40.0, planted=6, planted_min=12, planted_max=30, seed=5),
        "sbm": G.sbm_2plex(blocks=8, block_size=60, p_in=0.85, p_out=0.01, two_plex_blocks=3, seed=6)[0],
        "k40": G.complete(40),
    }
    uploads = {f"u{i}": G.sbm_2plex(blocks=3, block_size=50, p_in=0.9, p_out=1e-2, two_plex_blocks=1,
                                    seed=100 + i)[0] for i in range(3)}
    srv = KCliqueServer(max_batch=64, list_workers=3)
    for name, g in base.items():
        srv.register(name, g.row_ptr, g.col, g.n)
    reqs = []
    rng = np.random.default_rng(0)
    uploaded = []
    for i in range(90):
        if i in (10, 40, 70):  # an upload; requests on it follow at once and wait for its prepare
            name = f"u{len(uploaded)}"
            uploaded.append(name)
            g = uploads[name]
            reqs.append((Request("upload", name, csr=(g.row_ptr, g.col, g.n)), g))
            continue
        if uploaded and i % 3 == 0:
            name = uploaded[-1]
            g = uploads[name]
        else:
            name = list(base)[i % 4]
            g = base[name]
        k = int(rng.integers(3, 8))
        kind = "list" if i % 5 == 0 else "count"
        cap = int(rng.choice([1, 50, 10**6])) if kind == "list" else 0
        reqs.append((Request(kind, name, k=k, cap=cap), g))
    futs = [(srv.submit(r), r, g) for r, g in reqs]
    res = [(f.result(timeout=600), r, g) for f, r, g in futs]
    srv.close()
    assert len(res) > 60
    alone = {}
    for name, g in list(base.items()) + list(uploads.items()):
        alone[name] = K.kclique_prepare(g.row_ptr, g.col, g.n)
    for out, r, g in res:
        assert out.status == "ok", (r, out.status)
        if r.kind == "upload":
            continue
        want = O.count(g, r.k)
        assert (out.count, out.checksum) == (want["count"], want["checksum"]), r
        one = K.kclique_count(alone[r.graph], r.k, flags=K.KC_CHECKSUM)
        assert (out.count, out.checksum) == (one["count"], one["checksum"]), r
        if r.kind == "list":
            assert out.written == min(r.cap, want["count"])
            rows = np.asarray(out.rows, dtype=np.int64)
            assert (np.diff(rows, axis=1) > 0).all() if rows.size else True
            if want["count"] <= 2_000_000:
                ref = set(map(tuple, O.list_cliques(g, r.k).astype(np.int64).tolist()))
                got = set(map(tuple, rows.tolist()))
                assert len(got) == out.written and got <= ref
    st = srv.stats()
    assert st["queries"] == sum(1 for _, r, _ in res if r.kind != "upload")
    assert st["p99_s"] >= st["p50_s"] > 0
