"""Autotuner for the branch kernels' launch parameters.

Tuned knobs (every value gives the same counts and checksums, only the speed changes):
  * t_max      -- early termination on cliques (1), 2-plexes (2) or 3-plexes (3), or the
                  paper's rule (0: t = 2 if k <= tau/2, else 3);
  * split_min  -- sub-branches with |VSet| >= split_min are split across the warps of a
                  block, one work item per top-frame vertex (k >= 7; 0xFFFFFFFF = never);
  * width_min  -- the narrowest bitset width class used: a sub-branch that fits fewer
                  words runs in the kernels for width_min words;
  * warps_per_block -- warps that share one split sub-branch's frame (1..4).
Per-query knobs (t_max, split_min, width_min) go to kclique_count_batch_tuned and to the
server's requests; warps_per_block is a launch-wide knob of kclique_count.

A candidate is timed on a bounded shard of the ticket order (the heaviest tickets,
which dominate the run time), so tuning costs a small fraction of one query.  The
search is coordinate descent: one knob at a time, from the library defaults, keeping a
change only when it is faster by more than `margin`; a query whose shard runs in less
than `min_ms` is launch-bound and keeps the defaults.  Choices are cached per device,
coarse graph shape (edge count and tau, in powers of two) and k, in memory and, with
`cache_path`, in a JSON file.
"""
from __future__ import annotations

import json
import math
import os
import threading

DEFAULT_GRID = {
    "t_max": [0, 2, 3, 1],
    "split_min": [0, 32, 128, 0xFFFFFFFF],
    "width_min": [0, 2, 4],
    "warps_per_block": [0, 2],
}
PER_QUERY = ("t_max", "split_min", "width_min")


def shape_key(info: dict, k: int, device: str) -> str:
    mb = int(math.log2(max(1, info["m"])))
    tb = int(math.log2(max(1, info["tau"] + 1)))
    return f"{device}|m2^{mb}|tau2^{tb}|k{k}"


class Autotuner:
    def __init__(self, cache_path: str | None = None, grid: dict | None = None, shard: int = 512,
                 timer=None, device_name: str | None = None, margin: float = 0.03, reps: int = 2,
                 min_ms: float = 1.0):
        self.cache_path = cache_path
        self.grid = grid or DEFAULT_GRID
        self.shard = shard
        self.timer = timer            # callable(handle, k, params) -> ms; default: the library
        self.device_name = device_name
        self.margin = margin
        self.reps = reps
        self.min_ms = min_ms          # queries faster than this on the shard keep the defaults
        self.lock = threading.Lock()
        self.cache = {}
        self.infos = {}
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
        best = None
        for _ in range(self.reps):
            r = K.kclique_count(h, k, ticket_begin=0, ticket_end=self.shard, **params)
            best = r["ms_count"] if best is None else min(best, r["ms_count"])
        return float(best)

    def _info(self, h) -> dict:
        key = getattr(h, "handle", id(h))
        if key not in self.infos:
            from . import kclique as K
            self.infos[key] = K.kclique_info(h)
        return self.infos[key]

    def tune(self, h, k: int, info: dict | None = None, force: bool = False) -> dict:
        """Best parameters for (graph, k); measured once per shape key, then cached."""
        info = info if info is not None else self._info(h)
        key = shape_key(info, k, self._device())
        with self.lock:
            if not force and key in self.cache:
                return dict(self.cache[key]["params"])
        best = {name: vals[0] for name, vals in self.grid.items()}
        self._time(h, k, best)  # warm-up (module loading, first launches)
        best_ms = self._time(h, k, best)
        tried = [{"ms": best_ms, **best}]
        # a query this short is launch-bound: its timings cannot tell the knobs apart
        search = best_ms >= self.min_ms
        for name, vals in (self.grid.items() if search else ()):
            if name == "split_min" and k < 7:
                continue  # splitting applies to k >= 7 only
            for v in vals[1:]:
                cand = dict(best, **{name: v})
                ms = self._time(h, k, cand)
                tried.append({"ms": ms, **cand})
                if ms < best_ms * (1.0 - self.margin):
                    best, best_ms = cand, ms
        with self.lock:
            self.cache[key] = {"params": best, "ms": best_ms, "tried": tried}
            if self.cache_path:
                tmp = self.cache_path + ".tmp"
                with open(tmp, "w") as f:
                    json.dump(self.cache, f, indent=1, sort_keys=True)
                os.replace(tmp, self.cache_path)
        return dict(best)

    def choice(self, h, k: int, info: dict | None = None) -> dict:
        """The per-query part of the tuned parameters (t_max, split_min, width_min)."""
        p = self.tune(h, k, info)
        return {name: p[name] for name in PER_QUERY if name in p}
