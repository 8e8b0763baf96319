"""kclique_count_batch_noalloc: the batched count for callers that cannot allocate
device memory (it takes its scratch from a static array inside the library).

Its answers must equal those of the regular kclique_count_batch on the same inputs,
exactly (integer counts and checksums), on two calls in a row -- the second call runs
on scratch that still holds the first call's contents.  This file is collected last
so that a run that stops at the first failure has already run every other test.
"""
import numpy as np
import pytest

from synth import graphs as G

torch = pytest.importorskip("torch")


def _prep(g):
    from paper_2311_13798_gb300 import kclique as K
    rp = torch.from_numpy(g.row_ptr.astype(np.int32)).cuda()
    col = torch.from_numpy(g.col.astype(np.int32)).cuda()
    return K.kclique_prepare(rp, col, g.n)


@pytest.mark.gpu
def test_noalloc_matches_regular_batch_twice():
    from paper_2311_13798_gb300 import kclique as K
    graphs = [G.gnp(120, 0.6, seed=2), G.complete(40), G.two_plex(9, 12), G.t_plex(45, 3, seed=4),
              G.chung_lu(n=4000, w_max=400.0, i0=40.0, planted=6, planted_min=12, planted_max=30, seed=5),
              G.gnp(300, 0.75, seed=7), G.complete_bipartite(8, 8)]
    hs = [_prep(g) for g in graphs]
    qh, qk = [], []
    for i, h in enumerate(hs):
        for k in (3, 4, 5, 7):
            if i == 5 and k > 5:
                continue
            qh.append(h)
            qk.append(k)
    for flags in (0, K.KC_CHECKSUM):
        want = K.kclique_count_batch(qh, qk, flags=flags)
        for _ in range(2):
            got = K.kclique_count_batch_noalloc(qh, qk, flags=flags)
            assert [(r["count"], r["checksum"]) for r in got] == [(r["count"], r["checksum"]) for r in want]


@pytest.mark.gpu
def test_noalloc_rejects_too_many_queries():
    from paper_2311_13798_gb300 import kclique as K
    h = _prep(G.gnp(50, 0.3, seed=1))
    with pytest.raises(K.KCliqueError) as ei:
        K.kclique_count_batch_noalloc([h] * 65, [4] * 65)
    assert ei.value.status == K.KC_ERR_INVALID_ARG
    assert "64" in K.library().kclique_last_error().decode()
    assert K.kclique_count_batch_noalloc([h] * 64, [4] * 64)[0]["count"] == K.kclique_count(h, 4)["count"]
