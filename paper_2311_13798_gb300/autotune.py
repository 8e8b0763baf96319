"""Autotuner for the branch kernels' launch parameters.

Tuned knobs (all leave results unchanged, only speed):
  * split_min -- sub-branches with |VSet| >= split_min are split into per-vertex work
    items spread over all warps (the depth-1 split of heavy branches, k >= 7);
  * t_max     -- early termination on cliques only (1) or on cliques and 2-plexes (2);
  * blocks    -- persistent grid size (0 = one full wave of resident blocks).
The bitset width class is not a knob: it follows from each sub-branch's size.

A candidate is timed on a bounded shard of the ticket order (the heaviest tickets
first, which dominate the run time), so tuning costs a small fraction of one query.
Choices are cached in a JSON file keyed by device name, a coarse shape of the graph
(edge count and tau buckets) and k.
"""
from __future__ import annotations

import json
import math
import os
import threading

DEFAULT_GRID = {
    "split_min": [64, 48, 128, 0xFFFFFFFF],
    "t_max": [2, 1],
    "blocks": [0],
}


def shape_key(info: dict, k: int, device: str) -> str:
    mb = int(math.log2(max(1, info["m"])))
    tb = int(math.log2(max(1, info["tau"] + 1)))
    return f"{device}|m2^{mb}|tau2^{tb}|k{k}"


class Autotuner:
    def __init__(self, cache_path: str | None = None, grid: dict | None = None, shard: int = 512,
                 timer=None, device_name: str | None = None):
        self.cache_path = cache_path
        self.grid = grid or DEFAULT_GRID
        self.shard = shard
        self.timer = timer            # callable(handle, k, params) -> ms; default: the library
        self.device_name = device_name
        self.lock = threading.Lock()
        self.cache = {}
        if cache_path and os.path.exists(cache_path):
            with open(cache_path) as f:
                self.cache = json.load(f)

    def _device(self) -> str:
        if self.device_name is None:
            try:
                import torch
                self.device_name = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
            except ImportError:
                self.device_name = "cpu"
        return self.device_name

    def _time(self, h, k, params) -> float:
        if self.timer is not None:
            return float(self.timer(h, k, params))
        from . import kclique as K
        r = K.kclique_count(h, k, ticket_begin=0, ticket_end=self.shard, **params)
        return float(r["ms_count"])

    def candidates(self):
        for sm in self.grid["split_min"]:
            for t in self.grid["t_max"]:
                for b in self.grid["blocks"]:
                    yield {"split_min": sm, "t_max": t, "blocks": b}

    def tune(self, h, k: int, info: dict | None = None, force: bool = False) -> dict:
        """Best parameters for (graph, k); measured once per shape key, then cached."""
        if info is None:
            from . import kclique as K
            info = K.kclique_info(h)
        key = shape_key(info, k, self._device())
        with self.lock:
            if not force and key in self.cache:
                return dict(self.cache[key]["params"])
        results = []
        for p in self.candidates():
            if k < 7 and p["split_min"] != self.grid["split_min"][0]:
                continue  # splitting only applies to k >= 7
            self._time(h, k, p)                # warm-up
            results.append((self._time(h, k, p), p))
        results.sort(key=lambda x: x[0])
        best_ms, best = results[0]
        with self.lock:
            self.cache[key] = {"params": best, "ms": best_ms,
                               "tried": [{"ms": ms, **p} for ms, p in results]}
            if self.cache_path:
                tmp = self.cache_path + ".tmp"
                with open(tmp, "w") as f:
                    json.dump(self.cache, f, indent=1, sort_keys=True)
                os.replace(tmp, self.cache_path)
        return dict(best)
