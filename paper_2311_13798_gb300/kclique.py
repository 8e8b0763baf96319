"""Python binding of libkclique (ctypes; argument marshalling only).

Every entry point has the name of the C function it calls (see include/kclique.h);
all computation runs in the CUDA library.  Arrays may be torch tensors (CUDA or
CPU) or numpy arrays; device tensors are passed by pointer on the current torch
stream.  If the compiled library is missing this module raises -- there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libkclique.so")

KC_OK = 0
KC_TRUNCATED = 1
KC_ERR_INVALID_ARG = -1
KC_ERR_INVALID_GRAPH = -2
KC_ERR_OOM = -3
KC_ERR_CUDA = -4
KC_ERR_TIMEOUT = -5
KC_ERR_OVERFLOW = -6
KC_ERR_UNSUPPORTED = -7
KC_MAX_K = 32
KC_MAX_BRANCH = 1024
KC_NO_ET = 0x1
KC_NO_RULE2 = 0x2
KC_CHECKSUM = 0x4
KC_NO_RULE1 = 0x8
KC_ROWS_ONLY = 0x10
KC_TRUSS_INNER = 0x20
KC_ORDER_TRUSS = 0
KC_ORDER_COLOUR = 1


class KcParams(C.Structure):
    _fields_ = [("t_max", C.c_uint32), ("warps_per_block", C.c_uint32), ("blocks", C.c_uint32),
                ("flags", C.c_uint32), ("d_edge_count", C.c_void_p), ("d_edge_checksum", C.c_void_p),
                ("d_edge_cycles", C.c_void_p), ("split_min", C.c_uint32), ("width_min", C.c_uint32),
                ("ticket_begin", C.c_uint64), ("ticket_end", C.c_uint64)]


class KcResult(C.Structure):
    _fields_ = [("count_lo", C.c_uint64), ("count_hi", C.c_uint64), ("checksum", C.c_uint64),
                ("written", C.c_uint64), ("edge_branches", C.c_uint64), ("nodes", C.c_uint64),
                ("et_hits", C.c_uint64), ("word_ops", C.c_uint64), ("pair_tests", C.c_uint64),
                ("ms_prepare", C.c_float), ("ms_count", C.c_float), ("ms_branch", C.c_float), ("pad", C.c_float)]


class KcInfo(C.Structure):
    _fields_ = [("n", C.c_uint32), ("m", C.c_uint64), ("triangles", C.c_uint64), ("tau", C.c_uint32),
                ("max_degree", C.c_uint32), ("rounds", C.c_uint64), ("resident_bytes", C.c_uint64)]


# ---- serving (kc_server_*)
KC_REQ_COUNT = 0
KC_REQ_LIST = 1
KC_REQ_UPLOAD = 2
KC_SERVER_NO_YIELD = 0xFFFFFFFF

_PREPARE_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.c_uint32, C.c_uint64,
                          C.POINTER(C.c_void_p), C.POINTER(C.c_uint64))
_COUNT_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_uint32), C.POINTER(KcParams),
                        C.c_uint32, C.POINTER(KcResult))
_LIST_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_void_p, C.c_uint32, C.POINTER(C.c_uint32), C.c_uint64,
                       C.POINTER(KcResult))
_RELEASE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class KcServerBackend(C.Structure):
    _fields_ = [("ctx", C.c_void_p), ("prepare", _PREPARE_FN), ("count_batch", _COUNT_FN), ("list", _LIST_FN),
                ("release", _RELEASE_FN)]


class KcServerConfig(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_uint64), ("max_batch", C.c_uint32), ("list_workers", C.c_uint32),
                ("device", C.c_int32), ("upload_workers", C.c_uint32), ("yield_ms", C.c_uint32),
                ("pad", C.c_uint32), ("params", KcParams),
                ("backend", C.POINTER(KcServerBackend))]


class KcRequest(C.Structure):
    _fields_ = [("kind", C.c_uint32), ("k", C.c_uint32), ("graph", C.c_uint64), ("cap", C.c_uint64),
                ("rows", C.c_void_p), ("row_ptr", C.c_void_p), ("col", C.c_void_p), ("n", C.c_uint32),
                ("pin", C.c_uint32), ("nnz", C.c_uint64), ("t_max", C.c_uint32), ("split_min", C.c_uint32),
                ("width_min", C.c_uint32), ("pad", C.c_uint32)]


class KcCompletion(C.Structure):
    _fields_ = [("ticket", C.c_uint64), ("graph", C.c_uint64), ("kind", C.c_uint32), ("k", C.c_uint32),
                ("status", C.c_int32), ("pad", C.c_uint32), ("count_lo", C.c_uint64), ("count_hi", C.c_uint64),
                ("checksum", C.c_uint64), ("written", C.c_uint64), ("t_submit", C.c_double),
                ("t_done", C.c_double)]


class KcServerCounters(C.Structure):
    _fields_ = [(f, C.c_uint64) for f in ("submitted", "completed", "rejected", "evictions", "batches",
                                          "batched_queries", "max_batch_seen", "resident_bytes", "graphs",
                                          "inflight")] + \
               [(f, C.c_double) for f in ("busy_count_s", "busy_list_s", "busy_upload_s")]


class KCliqueError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = kclique_status_string(status)
        detail = _load().kclique_last_error().decode() if status == KC_ERR_CUDA else ""
        super().__init__(f"{where}: {msg} ({status}) {detail}".strip())


_lib = None
_lock = threading.Lock()


def _load():
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libkclique is not built ({LIB_PATH} missing); run "
                                   "`python -m paper_2311_13798_gb300.build` -- there is no CPU fallback")
            for cand in ("/usr/local/cuda/lib64/libcudart.so.13",):
                if os.path.exists(cand):
                    C.CDLL(cand, mode=C.RTLD_GLOBAL)
                    break
            lib = C.CDLL(LIB_PATH)
            vp, u32, u64 = C.c_void_p, C.c_uint32, C.c_uint64
            lib.kclique_prepare.restype = C.c_int
            lib.kclique_prepare.argtypes = [vp, vp, u32, u64, C.c_int, vp, C.POINTER(vp)]
            lib.kclique_prepare_ordered.restype = C.c_int
            lib.kclique_prepare_ordered.argtypes = [vp, vp, u32, u64, C.c_int, u32, vp, C.POINTER(vp)]
            lib.kclique_count.restype = C.c_int
            lib.kclique_count.argtypes = [vp, u32, C.POINTER(KcParams), vp, C.POINTER(KcResult)]
            lib.kclique_list.restype = C.c_int
            lib.kclique_list.argtypes = [vp, u32, vp, u64, C.POINTER(KcParams), vp, C.POINTER(KcResult)]
            lib.kclique_info.restype = C.c_int
            lib.kclique_info.argtypes = [vp, C.POINTER(KcInfo)]
            lib.kclique_edge_data.restype = C.c_int
            lib.kclique_edge_data.argtypes = [vp, vp, vp, vp, vp, vp, vp]
            lib.kclique_release.restype = None
            lib.kclique_release.argtypes = [vp]
            lib.kclique_status_string.restype = C.c_char_p
            lib.kclique_status_string.argtypes = [C.c_int]
            lib.kclique_last_error.restype = C.c_char_p
            lib.kclique_last_error.argtypes = []
            lib.kclique_launch_count.restype = C.c_ulonglong
            lib.kclique_launch_count.argtypes = [C.c_int]
            lib.kclique_kernel_rev.restype = C.c_char_p
            lib.kclique_kernel_rev.argtypes = []
            lib.kclique_int_peak.restype = C.c_int
            lib.kclique_int_peak.argtypes = [C.POINTER(C.c_double), C.POINTER(C.c_int), vp]
            lib.kclique_count_batch_noalloc.restype = C.c_int
            lib.kclique_count_batch_noalloc.argtypes = [C.POINTER(vp), C.POINTER(u32), u32, C.POINTER(KcParams), vp,
                                                        C.POINTER(KcResult)]
            lib.kc_server_create.restype = C.c_int
            lib.kc_server_create.argtypes = [C.POINTER(KcServerConfig), C.POINTER(vp)]
            lib.kc_server_adopt.restype = C.c_int
            lib.kc_server_adopt.argtypes = [vp, vp, u64, C.c_int, C.POINTER(u64)]
            lib.kc_server_submit.restype = C.c_int
            lib.kc_server_submit.argtypes = [vp, C.POINTER(KcRequest), C.POINTER(u64), C.POINTER(u64)]
            lib.kc_server_poll.restype = u32
            lib.kc_server_poll.argtypes = [vp, C.POINTER(KcCompletion), u32, C.c_int32]
            lib.kc_server_stats.restype = C.c_int
            lib.kc_server_stats.argtypes = [vp, C.POINTER(KcServerCounters)]
            lib.kc_server_destroy.restype = None
            lib.kc_server_destroy.argtypes = [vp]
            lib.kclique_count_batch_tuned.restype = C.c_int
            lib.kclique_count_batch_tuned.argtypes = [C.POINTER(vp), C.POINTER(u32), C.POINTER(KcParams), u32,
                                                      C.POINTER(KcParams), vp, C.POINTER(KcResult)]
            lib.kclique_count_batch.restype = C.c_int
            lib.kclique_count_batch.argtypes = [C.POINTER(vp), C.POINTER(u32), u32, C.POINTER(KcParams), vp,
                                                C.POINTER(KcResult)]
            lib.kclique_batch_plan_create.restype = C.c_int
            lib.kclique_batch_plan_create.argtypes = [C.POINTER(vp), C.POINTER(u32), C.POINTER(KcParams), u32,
                                                      C.POINTER(KcParams), vp, C.POINTER(vp)]
            lib.kclique_batch_plan_run.restype = C.c_int
            lib.kclique_batch_plan_run.argtypes = [vp, vp, C.POINTER(KcResult)]
            lib.kclique_batch_plan_release.restype = None
            lib.kclique_batch_plan_release.argtypes = [vp]
            _lib = lib
    return _lib


def library():
    """The loaded ctypes library (raises if it is not built)."""
    return _load()


def _stream(stream) -> int:
    if stream is not None:
        return int(getattr(stream, "cuda_stream", stream))
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return 0


def _ptr(a):
    """(pointer, on_device, keepalive) of a torch tensor or numpy array of 32-bit ints."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.dtype not in (torch.int32, getattr(torch, "uint32", torch.int32)):
                raise TypeError("expected a 32-bit integer tensor")
            a = a.contiguous()
            return a.data_ptr(), int(a.is_cuda), a
    except ImportError:
        pass
    arr = np.ascontiguousarray(a, dtype=np.uint32)
    return arr.ctypes.data, 0, arr


def kclique_status_string(status: int) -> str:
    return _load().kclique_status_string(int(status)).decode()


class Graph:
    """A prepared, device-resident graph (owns a kc_graph handle)."""

    def __init__(self, handle: int):
        self.handle = handle

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h:
            try:
                _load().kclique_release(h)
            except Exception:
                pass

    def release(self):
        if self.handle:
            _load().kclique_release(self.handle)
            self.handle = None


def kclique_prepare(row_ptr, col, n: int | None = None, stream=None, ordering: int = 0) -> Graph:
    """Prepare a graph from a CSR (torch CUDA tensors, or host arrays which are copied in).
    ordering: KC_ORDER_TRUSS (EBBkC-H, default) or KC_ORDER_COLOUR (EBBkC-C's top level)."""
    rp, dev_rp, keep1 = _ptr(row_ptr)
    cp, dev_c, keep2 = _ptr(col)
    if dev_rp != dev_c:
        raise ValueError("row_ptr and col must both be on the device or both on the host")
    nrp = int(keep1.numel() if hasattr(keep1, "numel") else keep1.size)
    nn = (nrp - 1) if n is None else int(n)
    nnz = int(keep2.numel() if hasattr(keep2, "numel") else keep2.size)
    h = C.c_void_p()
    if ordering == KC_ORDER_TRUSS:
        st = _load().kclique_prepare(rp, cp if nnz else rp, nn, nnz, dev_rp, _stream(stream), C.byref(h))
    else:
        st = _load().kclique_prepare_ordered(rp, cp if nnz else rp, nn, nnz, dev_rp, int(ordering),
                                             _stream(stream), C.byref(h))
    if st != KC_OK:
        raise KCliqueError(st, "kclique_prepare")
    return Graph(h.value)


def kclique_prepare_ordered(row_ptr, col, n: int | None = None, ordering: int = 0, stream=None) -> Graph:
    """kclique_prepare with a choice of the top-level edge order (KC_ORDER_*)."""
    return kclique_prepare(row_ptr, col, n, stream=stream, ordering=ordering)


def _params(t_max=0, flags=0, blocks=0, warps_per_block=0, edge_count=None, edge_checksum=None,
            edge_cycles=None, split_min=0, ticket_begin=0, ticket_end=0, width_min=0):
    p = KcParams()
    p.split_min = split_min
    p.width_min = width_min
    p.ticket_begin, p.ticket_end = ticket_begin, ticket_end
    p.t_max, p.flags, p.blocks, p.warps_per_block = t_max, flags, blocks, warps_per_block
    p.d_edge_count = edge_count.data_ptr() if edge_count is not None else None
    p.d_edge_checksum = edge_checksum.data_ptr() if edge_checksum is not None else None
    p.d_edge_cycles = edge_cycles.data_ptr() if edge_cycles is not None else None
    return p


def _result(r: KcResult, status: int) -> dict:
    return {"count": int(r.count_lo) | (int(r.count_hi) << 64), "checksum": int(r.checksum),
            "written": int(r.written), "edge_branches": int(r.edge_branches), "nodes": int(r.nodes),
            "et_hits": int(r.et_hits), "word_ops": int(r.word_ops), "pair_tests": int(r.pair_tests),
            "ms_prepare": float(r.ms_prepare), "ms_count": float(r.ms_count), "ms_branch": float(r.ms_branch),
            "truncated": status == KC_TRUNCATED, "status": status}


def kclique_count(g: Graph, k: int, stream=None, **kw) -> dict:
    """Exact k-clique count (and checksum with flags=KC_CHECKSUM)."""
    p = _params(**kw)
    r = KcResult()
    st = _load().kclique_count(g.handle, int(k), C.byref(p), _stream(stream), C.byref(r))
    if st not in (KC_OK,):
        raise KCliqueError(st, "kclique_count")
    return _result(r, st)


def kclique_list(g: Graph, k: int, out, stream=None, **kw) -> dict:
    """List k-cliques into ``out`` (CUDA int32 tensor [cap, k]); returns counts and rows written."""
    cap = int(out.shape[0]) if out is not None else 0
    if out is not None and (out.dim() != 2 or out.shape[1] != k or not out.is_cuda or not out.is_contiguous()):
        raise ValueError("out must be a contiguous CUDA int32 tensor of shape [cap, k]")
    p = _params(**kw)
    r = KcResult()
    st = _load().kclique_list(g.handle, int(k), out.data_ptr() if out is not None else None, cap, C.byref(p),
                              _stream(stream), C.byref(r))
    if st not in (KC_OK, KC_TRUNCATED):
        raise KCliqueError(st, "kclique_list")
    return _result(r, st)


def kclique_info(g: Graph) -> dict:
    info = KcInfo()
    st = _load().kclique_info(g.handle, C.byref(info))
    if st != KC_OK:
        raise KCliqueError(st, "kclique_info")
    return {f: int(getattr(info, f)) for f, _ in KcInfo._fields_}


def kclique_edge_data(g: Graph, stream=None) -> dict:
    m = kclique_info(g)["m"]
    out = {name: np.zeros(m, dtype=np.uint32) for name in ("eu", "ev", "level", "round", "vset_size")}
    st = _load().kclique_edge_data(g.handle, *(out[x].ctypes.data for x in ("eu", "ev", "level", "round", "vset_size")),
                                   _stream(stream))
    if st != KC_OK:
        raise KCliqueError(st, "kclique_edge_data")
    return out


def kclique_count_batch(graphs: list[Graph], ks, stream=None, tuner=None, choices=None, **kw) -> list[dict]:
    """Many (graph, k) count queries in one pass over the width classes.  With ``tuner``
    (an ``autotune.Autotuner``) or explicit ``choices`` (one dict of t_max / split_min /
    width_min per query), each query runs with its own parameters
    (kclique_count_batch_tuned)."""
    nq = len(graphs)
    hs = (C.c_void_p * max(nq, 1))(*[g.handle for g in graphs])
    kk = (C.c_uint32 * max(nq, 1))(*[int(k) for k in ks])
    res = (KcResult * max(nq, 1))()
    p = _params(**kw)
    if tuner is not None and choices is None:
        choices = [tuner.choice(g, int(k)) for g, k in zip(graphs, ks)]
    if choices is not None:
        qp = (KcParams * max(nq, 1))(*[_params(**c) for c in choices])
        st = _load().kclique_count_batch_tuned(hs, kk, qp, nq, C.byref(p), _stream(stream), res)
    else:
        st = _load().kclique_count_batch(hs, kk, nq, C.byref(p), _stream(stream), res)
    if st != KC_OK:
        raise KCliqueError(st, "kclique_count_batch")
    return [_result(res[i], KC_OK) for i in range(nq)]


class BatchPlan:
    """A batch of count queries captured once as a CUDA graph and replayed by ``run``
    (kclique_batch_plan_*).  The graphs must stay alive while the plan is used."""

    def __init__(self, handle, nq: int, graphs):
        self.handle, self.nq, self._graphs = handle, nq, graphs

    def run(self, stream=None) -> list[dict]:
        res = (KcResult * max(self.nq, 1))()
        st = _load().kclique_batch_plan_run(self.handle, _stream(stream), res)
        if st != KC_OK:
            raise KCliqueError(st, "kclique_batch_plan_run")
        return [_result(res[i], KC_OK) for i in range(self.nq)]

    def release(self):
        if self.handle:
            _load().kclique_batch_plan_release(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


def kclique_batch_plan_create(graphs: list[Graph], ks, choices=None, stream=None, **kw) -> BatchPlan:
    """Capture the batch (graphs, ks), with optional per-query ``choices``, for replays."""
    nq = len(graphs)
    hs = (C.c_void_p * max(nq, 1))(*[g.handle for g in graphs])
    kk = (C.c_uint32 * max(nq, 1))(*[int(k) for k in ks])
    p = _params(**kw)
    qp = (KcParams * max(nq, 1))(*[_params(**c) for c in choices]) if choices is not None else None
    h = C.c_void_p()
    st = _load().kclique_batch_plan_create(hs, kk, qp, nq, C.byref(p), _stream(stream), C.byref(h))
    if st != KC_OK:
        raise KCliqueError(st, "kclique_batch_plan_create")
    return BatchPlan(h.value, nq, list(graphs))


def kclique_batch_plan_run(plan: BatchPlan, stream=None) -> list[dict]:
    return plan.run(stream)


def kclique_batch_plan_release(plan: BatchPlan) -> None:
    plan.release()


def kclique_count_batch_tuned(graphs: list[Graph], ks, choices, stream=None, **kw) -> list[dict]:
    """kclique_count_batch with per-query choices (dicts of t_max / split_min / width_min)."""
    return kclique_count_batch(graphs, ks, stream=stream, choices=choices, **kw)


def kclique_int_peak(stream=None) -> dict:
    """Measured AND+AND+POPC lane-op rate of the current GPU (roofline denominator)."""
    v = C.c_double()
    n = C.c_int()
    st = _load().kclique_int_peak(C.byref(v), C.byref(n), _stream(stream))
    if st != KC_OK:
        raise KCliqueError(st, "kclique_int_peak")
    return {"lane_ops_per_s": float(v.value), "sms": int(n.value)}


def kclique_launch_count(reset: bool = False) -> int:
    """Kernel launches made by the library so far (optionally restarting the count)."""
    return int(_load().kclique_launch_count(int(reset)))


def kclique_kernel_rev() -> str:
    return _load().kclique_kernel_rev().decode()


def kclique_count_batch_noalloc(graphs: list[Graph], ks, stream=None, **kw) -> list[dict]:
    """Batched count that allocates no device memory (at most 64 queries per call)."""
    nq = len(graphs)
    hs = (C.c_void_p * max(nq, 1))(*[g.handle for g in graphs])
    kk = (C.c_uint32 * max(nq, 1))(*[int(k) for k in ks])
    res = (KcResult * max(nq, 1))()
    p = _params(**kw)
    st = _load().kclique_count_batch_noalloc(hs, kk, nq, C.byref(p), _stream(stream), res)
    if st != KC_OK:
        raise KCliqueError(st, "kclique_count_batch_noalloc")
    return [_result(res[i], KC_OK) for i in range(nq)]
