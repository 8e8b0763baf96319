"""Continuous-batching query server over libkclique (count / list / upload requests).

Requests arrive at any time through ``submit``.  Two worker threads drive the GPU:

* the query worker takes every count request that arrived while the previous batch
  was running and runs them as ONE ``kclique_count_batch`` launch per width class
  (continuous batching: the batch is whatever is waiting, up to ``max_batch``); list
  requests go to a small pool of list workers, each on its own CUDA stream, which write
  the rows only (``KC_ROWS_ONLY``: the pass ends when the buffer is full); when a listing
  was truncated its exact totals (count, checksum) are computed by a count entry that
  joins the next batch, so a list query costs a short row pass plus a batched count;
* the upload worker prepares newly uploaded graphs (``kclique_prepare``) on its own
  CUDA stream, so uploads overlap with counting on the device.

Prepared graphs stay resident on the device across queries.  Uploads are admitted
against an HBM budget: resident bytes (``kclique_info``'s ``resident_bytes`` plus a
prepare-time estimate for graphs being built) may not exceed it; least-recently-used
uploaded graphs that no query is waiting on are released to make room, graphs
registered with ``pin=True`` are never evicted, and an upload that still does not fit
is rejected.  There is no result cache: every query runs.

The arithmetic is the library's; this module only schedules.  A backend object
(``CudaBackend`` by default) performs the calls, so the scheduling logic can be tested
with a stand-in backend on a machine without a GPU.
"""
from __future__ import annotations

import collections
import queue
import threading
import time
from concurrent.futures import Future, ThreadPoolExecutor
from dataclasses import dataclass, field


@dataclass
class Request:
    kind: str                 # "count" | "list" | "upload" ("totals": internal, see _run_list)
    graph: str                # graph name (uploads: the name to register)
    k: int = 0
    cap: int = 0              # list: rows wanted
    csr: tuple | None = None  # upload: (row_ptr, col, n) host arrays
    parent: object = None     # totals: (list request, its rows result)
    t_arrival: float = field(default_factory=time.perf_counter)
    future: Future = field(default_factory=Future)


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
    latency_s: float = 0.0


class CudaBackend:
    """libkclique calls on CUDA streams of their own: counts, uploads, and one stream
    per list-worker thread."""

    def __init__(self, device: int = 0, split_min: int = 0):
        import torch

        from . import kclique as K
        self.K = K
        self.torch = torch
        torch.cuda.set_device(device)
        self.device = device
        # |VSet| from which the batches split k >= 7 sub-branches (0: the library's default, 64)
        self.split_min = int(split_min)
        self.qstream = torch.cuda.Stream()
        self.ustream = torch.cuda.Stream()
        self.tls = threading.local()

    def prepare(self, row_ptr, col, n):
        with self.torch.cuda.stream(self.ustream):
            return self.K.kclique_prepare(row_ptr, col, n, stream=self.ustream)

    def resident_bytes(self, h) -> int:
        return self.K.kclique_info(h)["resident_bytes"]

    def estimate_bytes(self, row_ptr, col, n) -> int:
        nnz = len(col)
        # resident arrays (CSR, per-slot ids and rounds, per-edge arrays, VSet) with a
        # triangle allowance of 4 per edge; prepare also holds temporaries briefly
        return int(4 * (n + 1) + 12 * nnz + 28 * (nnz // 2) + 16 * nnz)

    def count_batch(self, handles, ks):
        with self.torch.cuda.stream(self.qstream):
            return self.K.kclique_count_batch(handles, ks, stream=self.qstream, flags=self.K.KC_CHECKSUM,
                                              split_min=self.split_min)

    def list(self, h, k, cap, rows_only=False):
        st = getattr(self.tls, "stream", None)
        if st is None:
            self.torch.cuda.set_device(self.device)
            st = self.tls.stream = self.torch.cuda.Stream()
        with self.torch.cuda.stream(st):
            out = self.torch.empty((max(cap, 1), k), dtype=self.torch.int32, device="cuda")
            r = self.K.kclique_list(h, k, out, stream=st, flags=self.K.KC_ROWS_ONLY if rows_only else 0)
            return r, out[: r["written"]].cpu().numpy()

    def release(self, h):
        h.release()


class KCliqueServer:
    def __init__(self, backend=None, hbm_budget_bytes: int = 120 << 30, max_batch: int = 512,
                 list_workers: int = 4):
        self.backend = backend or CudaBackend()
        self.budget = int(hbm_budget_bytes)
        self.max_batch = max_batch
        self.graphs: dict[str, object] = {}
        self.bytes: dict[str, int] = {}
        self.pinned: set[str] = set()
        self.lru: collections.OrderedDict[str, None] = collections.OrderedDict()
        self.waiting: collections.Counter = collections.Counter()  # queries not yet run, per graph
        self.reserved = 0
        self.lock = threading.Lock()
        self.cv = threading.Condition(self.lock)
        self.qq: collections.deque[Request] = collections.deque()
        self.uq: queue.Queue = queue.Queue()
        self.done: list[Result] = []
        self.batches: list[int] = []
        self.rejected = 0
        self.lists_inflight = 0
        self.busy = {"count_batch": 0.0, "list": 0.0, "upload": 0.0}  # seconds inside backend calls
        self.stop = False
        self.t_first = None
        self.t_last = None
        self.list_pool = ThreadPoolExecutor(max_workers=max(1, list_workers))
        self.qt = threading.Thread(target=self._query_worker, daemon=True)
        self.ut = threading.Thread(target=self._upload_worker, daemon=True)
        self.qt.start()
        self.ut.start()

    # ------------------------------------------------------------ registration
    def register(self, name: str, row_ptr, col, n: int, pin: bool = True):
        """Prepare a graph synchronously and keep it resident (pinned by default)."""
        h = self.backend.prepare(row_ptr, col, n)
        with self.lock:
            self.graphs[name] = h
            self.bytes[name] = self.backend.resident_bytes(h)
            if pin:
                self.pinned.add(name)
            self.lru[name] = None
        return h

    def resident(self) -> int:
        with self.lock:
            return sum(self.bytes.values()) + self.reserved

    # ------------------------------------------------------------ submission
    def submit(self, req: Request) -> Future:
        if self.t_first is None:
            self.t_first = req.t_arrival
        if req.kind == "upload":
            self.uq.put(req)
            return req.future
        with self.cv:
            known = req.graph in self.graphs
            if known:
                self.waiting[req.graph] += 1
                self.qq.append(req)
                self.cv.notify()
        if not known:
            self._finish(req, Result(req.kind, req.graph, req.k, status="unknown graph"))
        return req.future

    def close(self, timeout: float = 600.0):
        with self.cv:
            self.stop = True
            self.cv.notify_all()
        self.uq.put(None)
        self.qt.join(timeout)
        self.ut.join(timeout)
        self.list_pool.shutdown(wait=True)

    # ------------------------------------------------------------ workers
    def _finish(self, req: Request, res: Result):
        t = time.perf_counter()
        res.latency_s = t - req.t_arrival
        with self.lock:
            self.t_last = t
            self.done.append(res)
        req.future.set_result(res)

    def _evict_for(self, need: int) -> bool:
        """Release LRU uploaded graphs nobody waits on until `need` bytes fit (lock held).
        Nothing is released when even releasing every such graph would not make room."""
        evictable = [g for g in self.lru if g not in self.pinned and self.waiting[g] == 0]
        if sum(self.bytes.values()) + self.reserved + need - sum(self.bytes[g] for g in evictable) > self.budget:
            return False
        while sum(self.bytes.values()) + self.reserved + need > self.budget:
            victim = next((g for g in self.lru if g not in self.pinned and self.waiting[g] == 0), None)
            if victim is None:
                return False
            h = self.graphs.pop(victim)
            self.bytes.pop(victim)
            self.lru.pop(victim)
            self.backend.release(h)
        return True

    def _upload_worker(self):
        while True:
            req = self.uq.get()
            if req is None:
                return
            rp, col, n = req.csr
            need = self.backend.estimate_bytes(rp, col, n)
            with self.lock:
                ok = self._evict_for(need)
                if ok:
                    self.reserved += need
            if not ok:
                self.rejected += 1
                self._finish(req, Result("upload", req.graph, 0, status="rejected: HBM budget"))
                continue
            t0 = time.perf_counter()
            try:
                h = self.backend.prepare(rp, col, n)
                status = "ok"
            except Exception as e:  # surfaced to the client, the server keeps running
                h, status = None, f"error: {e}"
            with self.cv:
                self.busy["upload"] += time.perf_counter() - t0
                self.reserved -= need
                if h is not None:
                    old = self.graphs.get(req.graph)
                    if old is not None and self.waiting[req.graph] == 0:
                        self.backend.release(old)
                    self.graphs[req.graph] = h
                    self.bytes[req.graph] = self.backend.resident_bytes(h)
                    self.lru[req.graph] = None
                    self.lru.move_to_end(req.graph)
            self._finish(req, Result("upload", req.graph, 0, status=status))

    def _query_worker(self):
        while True:
            with self.cv:
                while not self.qq and not (self.stop and self.lists_inflight == 0):
                    self.cv.wait()
                if not self.qq:  # stopping, and no listing can still add a totals entry
                    return
                batch, lists = [], []
                while self.qq and len(batch) < self.max_batch:
                    r = self.qq.popleft()
                    (lists if r.kind == "list" else batch).append(r)  # count and totals batch
                handles = {r.graph: self.graphs[r.graph] for r in batch + lists}
                for g in handles:
                    self.lru.move_to_end(g)
                self.lists_inflight += len(lists)
            for r in lists:
                self.list_pool.submit(self._run_list, r, handles[r.graph])
            if batch:
                self.batches.append(len(batch))
                t0 = time.perf_counter()
                try:
                    res = self.backend.count_batch([handles[r.graph] for r in batch], [r.k for r in batch])
                    outs = [Result("count", r.graph, r.k, count=x["count"], checksum=x["checksum"])
                            for r, x in zip(batch, res)]
                except Exception as e:
                    outs = [Result("count", r.graph, r.k, status=f"error: {e}") for r in batch]
                self.busy["count_batch"] += time.perf_counter() - t0
                for r, o in zip(batch, outs):
                    if r.kind == "totals":  # completes a truncated listing
                        req, lo = r.parent
                        lo.count, lo.checksum = o.count, o.checksum
                        if o.status != "ok":
                            lo.status = o.status
                        self._finish(req, lo)
                    else:
                        self._finish(r, o)
            with self.cv:
                for r in batch:
                    self.waiting[r.graph] -= 1

    def _run_list(self, r: Request, h):
        t0 = time.perf_counter()
        try:
            x, rows = self.backend.list(h, r.k, r.cap, rows_only=True)
            o = Result("list", r.graph, r.k, count=x["count"], checksum=x["checksum"],
                       written=x["written"], rows=rows)
            truncated = bool(x.get("truncated"))
        except Exception as e:
            o = Result("list", r.graph, r.k, status=f"error: {e}")
            truncated = False
        with self.cv:
            self.busy["list"] += time.perf_counter() - t0
            if truncated:  # the totals join the next count batch; the graph stays held
                self.waiting[r.graph] += 1
                self.qq.append(Request("totals", r.graph, k=r.k, t_arrival=r.t_arrival, parent=(r, o)))
                self.cv.notify()
            self.waiting[r.graph] -= 1
            self.lists_inflight -= 1
            self.cv.notify_all()
        if not truncated:
            self._finish(r, o)

    # ------------------------------------------------------------ statistics
    def stats(self) -> dict:
        lat = sorted(r.latency_s for r in self.done if r.kind != "upload" and r.status == "ok")

        def pct(p):
            if not lat:
                return None
            return lat[min(len(lat) - 1, int(round(p / 100.0 * (len(lat) - 1))))]
        span = (self.t_last - self.t_first) if (self.t_first is not None and self.t_last is not None) else 0.0
        nq = sum(1 for r in self.done if r.kind != "upload")
        return {"queries": nq, "uploads": sum(1 for r in self.done if r.kind == "upload"),
                "rejected": self.rejected, "p50_s": pct(50), "p99_s": pct(99),
                "throughput_qps": nq / span if span else None, "batches": len(self.batches),
                "mean_batch": (sum(self.batches) / len(self.batches)) if self.batches else 0.0,
                "span_s": span, "busy_s": dict(self.busy), "max_batch_seen": max(self.batches, default=0)}
