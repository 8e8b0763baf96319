"""Python binding of the continuous-batching query server (``kc_server_*`` in
include/kclique.h).  Argument marshalling only: the scheduling -- continuous batching of
count requests, listing workers on their own streams, uploads prepared on their own
stream, HBM-budget admission with LRU eviction -- runs in the C library's threads.

``KCliqueServer.submit`` returns a ``concurrent.futures.Future`` per request; a poller
thread moves the library's completions to their futures.  Graphs are named here and
numbered in the library.  ``backend`` may be a stand-in object (``prepare``,
``count_batch``, ``list``, ``release``) whose methods the library's threads call
through C callbacks, so the scheduling can be exercised on a machine without a GPU; the
default (None) is the library's own GPU path.
"""
from __future__ import annotations

import ctypes as C
import threading
import time
from concurrent.futures import Future
from dataclasses import dataclass, field

import numpy as np

from . import kclique as K


@dataclass
class Request:
    kind: str                 # "count" | "list" | "upload"
    graph: str                # graph name (uploads: the name to register)
    k: int = 0
    cap: int = 0              # list: rows wanted
    csr: tuple | None = None  # upload: (row_ptr, col, n) host arrays
    pin: bool = False         # upload: never evicted
    t_arrival: float = field(default_factory=time.perf_counter)


@dataclass
class Result:
    kind: str
    graph: str
    k: int
    count: int = 0
    checksum: int = 0
    written: int = 0
    status: str = "ok"
    rows: object = None
    latency_s: float = 0.0    # from submission to completion (the library's clock)


_KINDS = {"count": K.KC_REQ_COUNT, "list": K.KC_REQ_LIST, "upload": K.KC_REQ_UPLOAD}


def _status_text(st: int, kind: str) -> str:
    if st in (K.KC_OK, K.KC_TRUNCATED):
        return "ok"
    if kind == "upload" and st == K.KC_ERR_OOM:
        return "rejected: HBM budget"
    return f"error: {K.kclique_status_string(st)} ({st})"


class _CallbackBackend:
    """C callbacks that forward the library's backend calls to a Python stand-in."""

    def __init__(self, be):
        self.be = be
        self.handles: dict[int, object] = {}
        self.next = 1
        self.lock = threading.Lock()

        def prepare(ctx, rp, col, n, nnz, out, nbytes):
            try:
                r = np.ctypeslib.as_array(rp, shape=(n + 1,)).copy()
                c = np.ctypeslib.as_array(col, shape=(max(nnz, 1),))[:nnz].copy()
                h, b = be.prepare(r, c, n)
                out[0] = self._keep(h)
                nbytes[0] = int(b)
                return K.KC_OK
            except Exception:  # surfaced as a failed upload
                return K.KC_ERR_CUDA

        def count_batch(ctx, hs, ks, qp, nq, res):
            try:
                got = be.count_batch([self.handles[hs[i]] for i in range(nq)], [ks[i] for i in range(nq)])
                for i, x in enumerate(got):
                    res[i].count_lo = x["count"] & ((1 << 64) - 1)
                    res[i].count_hi = x["count"] >> 64
                    res[i].checksum = x["checksum"]
                return K.KC_OK
            except Exception:
                return K.KC_ERR_CUDA

        def list_(ctx, h, k, rows, cap, res):
            try:
                x, got = be.list(self.handles[h], k, cap)
                got = np.asarray(got, dtype=np.uint32).reshape(-1, k)[:cap]
                if rows and got.size:
                    dst = np.ctypeslib.as_array(rows, shape=(cap * k,))
                    dst[: got.size] = got.reshape(-1)
                res[0].written = len(got)
                res[0].count_lo = x["count"] & ((1 << 64) - 1)
                res[0].count_hi = x["count"] >> 64
                res[0].checksum = x["checksum"]
                return K.KC_TRUNCATED if x.get("truncated") else K.KC_OK
            except Exception:
                return K.KC_ERR_CUDA

        def release(ctx, h):
            with self.lock:
                obj = self.handles.pop(h, None)
            if obj is not None:
                be.release(obj)

        self.fns = (K._PREPARE_FN(prepare), K._COUNT_FN(count_batch), K._LIST_FN(list_), K._RELEASE_FN(release))
        self.struct = K.KcServerBackend(None, *self.fns)

    def _keep(self, h) -> int:
        with self.lock:
            hid = self.next
            self.next += 1
            self.handles[hid] = h
            return hid


class KCliqueServer:
    def __init__(self, backend=None, hbm_budget_bytes: int = 120 << 30, max_batch: int = 512,
                 list_workers: int = 4, device: int = -1, split_min: int = 0, t_max: int = 0, flags: int = 0,
                 upload_workers: int = 0, yield_ms: int = 0):
        self.lib = K.library()
        cfg = K.KcServerConfig()
        cfg.hbm_budget_bytes = int(hbm_budget_bytes)
        cfg.max_batch = int(max_batch)
        cfg.list_workers = int(list_workers)
        cfg.upload_workers = int(upload_workers)
        cfg.yield_ms = int(yield_ms)
        cfg.device = int(device)
        cfg.params = K._params(t_max=t_max, flags=flags, split_min=split_min)
        self._cb = _CallbackBackend(backend) if backend is not None else None
        if self._cb is not None:
            cfg.backend = C.pointer(self._cb.struct)
        h = C.c_void_p()
        st = self.lib.kc_server_create(C.byref(cfg), C.byref(h))
        if st != K.KC_OK:
            raise K.KCliqueError(st, "kc_server_create")
        self.h = h
        self.ids: dict[str, int] = {}
        self.lock = threading.Lock()
        self.pending: dict[int, tuple] = {}   # ticket -> (future, request, rows buffer)
        self.done: list[Result] = []
        self.t_first = None
        self.t_last = None
        self.stop = False
        self.poller = threading.Thread(target=self._poll, daemon=True)
        self.poller.start()

    # ------------------------------------------------------------ registration
    def register(self, name: str, row_ptr, col, n: int, pin: bool = True):
        """Prepare a graph now and hand it to the server, resident (pinned by default)."""
        if self._cb is None:
            g = K.kclique_prepare(row_ptr, col, n)
            handle, nbytes = g.handle, 0
            g.handle = None  # the server owns it now
        else:
            obj, nbytes = self._cb.be.prepare(np.asarray(row_ptr), np.asarray(col), n)
            handle = self._cb._keep(obj)
        gid = C.c_uint64()
        st = self.lib.kc_server_adopt(self.h, C.c_void_p(handle), int(nbytes), int(pin), C.byref(gid))
        if st != K.KC_OK:
            raise K.KCliqueError(st, "kc_server_adopt")
        with self.lock:
            self.ids[name] = gid.value
        return gid.value

    # ------------------------------------------------------------ submission
    def submit(self, req: Request) -> Future:
        fut: Future = Future()
        r = K.KcRequest()
        r.kind = _KINDS[req.kind]
        r.k = int(req.k)
        rows = keep = None
        if req.kind == "upload":
            rp, col, n = req.csr
            rp = np.ascontiguousarray(rp, dtype=np.uint32)
            col = np.ascontiguousarray(col, dtype=np.uint32)
            keep = (rp, col)
            r.row_ptr, r.col, r.n, r.nnz, r.pin = rp.ctypes.data, (col.ctypes.data if col.size else rp.ctypes.data), \
                int(n), int(col.size), int(req.pin)
        else:
            with self.lock:
                gid = self.ids.get(req.graph)
            if gid is None:
                res = Result(req.kind, req.graph, req.k, status="unknown graph")
                with self.lock:
                    self.done.append(res)
                fut.set_result(res)
                return fut
            r.graph = gid
            if req.kind == "list":
                rows = np.zeros((max(int(req.cap), 1), max(int(req.k), 1)), dtype=np.uint32)
                r.cap, r.rows = int(req.cap), rows.ctypes.data
        ticket, gid_out = C.c_uint64(), C.c_uint64()
        with self.lock:
            # the poller may see the completion before submit returns: register under the lock
            st = self.lib.kc_server_submit(self.h, C.byref(r), C.byref(ticket), C.byref(gid_out))
            if st != K.KC_OK:
                raise K.KCliqueError(st, "kc_server_submit")
            if req.kind == "upload":
                self.ids[req.graph] = gid_out.value
            self.pending[ticket.value] = (fut, req, rows, keep)
        return fut

    def _poll(self):
        buf = (K.KcCompletion * 256)()
        while True:
            n = self.lib.kc_server_poll(self.h, buf, 256, 50)
            for i in range(n):
                c = buf[i]
                with self.lock:
                    fut, req, rows, _ = self.pending.pop(c.ticket)
                res = Result(req.kind, req.graph, req.k, count=int(c.count_lo) | (int(c.count_hi) << 64),
                             checksum=int(c.checksum), written=int(c.written),
                             status=_status_text(c.status, req.kind), latency_s=c.t_done - c.t_submit)
                if rows is not None:
                    res.rows = rows[: res.written]
                with self.lock:
                    self.done.append(res)
                    self.t_first = c.t_submit if self.t_first is None else min(self.t_first, c.t_submit)
                    self.t_last = c.t_done if self.t_last is None else max(self.t_last, c.t_done)
                fut.set_result(res)
            if n == 0 and self.stop:
                with self.lock:
                    if not self.pending:
                        return

    def close(self):
        """Finish every submitted request and stop the server."""
        while True:
            with self.lock:
                if not self.pending:
                    break
            time.sleep(0.01)
        self.stop = True
        self.poller.join()
        counters = self.counters()
        self.lib.kc_server_destroy(self.h)
        self._final = counters

    def counters(self) -> dict:
        if getattr(self, "_final", None) is not None:
            return dict(self._final)
        c = K.KcServerCounters()
        st = self.lib.kc_server_stats(self.h, C.byref(c))
        if st != K.KC_OK:
            raise K.KCliqueError(st, "kc_server_stats")
        return {f: getattr(c, f) for f, _ in K.KcServerCounters._fields_}

    # ------------------------------------------------------------ statistics
    def stats(self) -> dict:
        with self.lock:
            done = list(self.done)
        lat = sorted(r.latency_s for r in done if r.kind != "upload" and r.status == "ok")

        def pct(p):
            if not lat:
                return None
            return lat[min(len(lat) - 1, int(round(p / 100.0 * (len(lat) - 1))))]
        span = (self.t_last - self.t_first) if (self.t_first is not None and self.t_last is not None) else 0.0
        nq = sum(1 for r in done if r.kind != "upload")
        c = self.counters()
        return {"queries": nq, "uploads": sum(1 for r in done if r.kind == "upload"),
                "rejected": int(c["rejected"]), "evictions": int(c["evictions"]),
                "p50_s": pct(50), "p99_s": pct(99), "throughput_qps": nq / span if span else None,
                "batches": int(c["batches"]),
                "mean_batch": (c["batched_queries"] / c["batches"]) if c["batches"] else 0.0,
                "span_s": span, "max_batch_seen": int(c["max_batch_seen"]),
                "busy_s": {"count_batch": c["busy_count_s"], "list": c["busy_list_s"], "upload": c["busy_upload_s"]}}
