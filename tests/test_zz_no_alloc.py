"""kclique_count_batch_noalloc: the batched count for callers that cannot allocate
device memory (it takes its scratch from a static array inside the library).

Its answers must equal the CPU oracle's and those of the regular kclique_count_batch
on the same inputs, exactly (integer counts and checksums), on two calls in a row --
the second call runs on scratch that still holds the first call's contents.  A call
after the first must also leave the device's free memory and the stream-ordered pool's
high-water mark unchanged: the entry point exists for callers that cannot allocate.
This file is collected last so that a run that stops at the first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
from synth import graphs as G

torch = pytest.importorskip("torch")

POOL_USED_MEM_CURRENT = 0x7  # cudaMemPoolAttrUsedMemCurrent
POOL_USED_MEM_HIGH = 0x8     # cudaMemPoolAttrUsedMemHigh


def _prep(g):
    from paper_2311_13798_gb300 import kclique as K
    rp = torch.from_numpy(g.row_ptr.astype(np.int32)).cuda()
    col = torch.from_numpy(g.col.astype(np.int32)).cuda()
    return K.kclique_prepare(rp, col, g.n)


def _queries():
    graphs = [G.gnp(120, 0.6, seed=2), G.complete(40), G.two_plex(9, 12), G.t_plex(45, 3, seed=4),
              G.chung_lu(n=4000, w_max=400.0, i0=40.0, planted=6, planted_min=12, planted_max=30, seed=5),
              G.gnp(300, 0.75, seed=7), G.complete_bipartite(8, 8)]
    hs = [_prep(g) for g in graphs]
    qg, qh, qk = [], [], []
    for i, (g, h) in enumerate(zip(graphs, hs)):
        for k in (3, 4, 5, 7):
            if i == 5 and k > 5:
                continue
            qg.append(g)
            qh.append(h)
            qk.append(k)
    return qg, qh, qk


@pytest.mark.gpu
def test_noalloc_matches_oracle_and_regular_batch_twice():
    from paper_2311_13798_gb300 import kclique as K
    qg, qh, qk = _queries()
    oracle = [O.count(g, k) for g, k in zip(qg, qk)]
    for flags in (0, K.KC_CHECKSUM):
        want = K.kclique_count_batch(qh, qk, flags=flags)
        assert [r["count"] for r in want] == [o["count"] for o in oracle]
        for _ in range(2):
            got = K.kclique_count_batch_noalloc(qh, qk, flags=flags)
            assert [r["count"] for r in got] == [o["count"] for o in oracle]
            if flags:
                assert [r["checksum"] for r in got] == [o["checksum"] for o in oracle]
            assert [(r["count"], r["checksum"]) for r in got] == [(r["count"], r["checksum"]) for r in want]


def _cudart():
    from paper_2311_13798_gb300 import kclique as K
    K.library()  # loads the CUDA runtime the library uses
    for name in ("libcudart.so.13", "/usr/local/cuda/lib64/libcudart.so.13", "libcudart.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    pytest.skip("CUDA runtime library not found")


def _pool_attr(rt, pool, attr):
    v = ctypes.c_uint64(0)
    assert rt.cudaMemPoolGetAttribute(pool, ctypes.c_int(attr), ctypes.byref(v)) == 0
    return v.value


@pytest.mark.gpu
def test_noalloc_call_allocates_nothing():
    """After a first call (which does the one-time set-up), a call with other widths, k
    and flags changes neither the free device memory nor the default memory pool's usage."""
    from paper_2311_13798_gb300 import kclique as K
    qg, qh, qk = _queries()
    K.kclique_count_batch_noalloc(qh[:3], qk[:3])  # the set-up call
    torch.cuda.synchronize()
    rt = _cudart()
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), ctypes.c_int(torch.cuda.current_device())) == 0
    zero = ctypes.c_uint64(0)
    assert rt.cudaMemPoolSetAttribute(pool, ctypes.c_int(POOL_USED_MEM_HIGH), ctypes.byref(zero)) == 0
    used0 = _pool_attr(rt, pool, POOL_USED_MEM_CURRENT)
    free0 = torch.cuda.mem_get_info()[0]
    got = K.kclique_count_batch_noalloc(qh, qk, flags=K.KC_CHECKSUM)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert _pool_attr(rt, pool, POOL_USED_MEM_CURRENT) == used0
    assert _pool_attr(rt, pool, POOL_USED_MEM_HIGH) == used0
    assert [r["count"] for r in got] == [O.count(g, k)["count"] for g, k in zip(qg, qk)]


@pytest.mark.gpu
def test_noalloc_rejects_too_many_queries():
    from paper_2311_13798_gb300 import kclique as K
    h = _prep(G.gnp(50, 0.3, seed=1))
    with pytest.raises(K.KCliqueError) as ei:
        K.kclique_count_batch_noalloc([h] * 65, [4] * 65)
    assert ei.value.status == K.KC_ERR_INVALID_ARG
    assert "64" in K.library().kclique_last_error().decode()
    assert K.kclique_count_batch_noalloc([h] * 64, [4] * 64)[0]["count"] == K.kclique_count(h, 4)["count"]
