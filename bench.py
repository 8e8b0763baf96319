#!/usr/bin/env python
"""Benchmark of the EBBkC hot path on the power-law workload (one JSON line on rank 0).

Workload: Chung-Lu power-law graph, n = 10^6, about 1.0e7 undirected edges, degree
exponent 2.1, max expected degree 10^4, 200 planted cliques of size 30-60, random
relabel (synth.graphs.chung_lu, seed = rank); k in {5, 7, 9}.

One step = the whole hot path over one graph resident in HBM:
  kclique_prepare (CSR clean-up, triangle incidence, truss peel, VSet),
  kclique_count for k = 5, 7, 9 and kclique_list for k = 5 into a 2^24-row buffer.
value = k-cliques counted per second (sum over the three counts / step time).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (the only reference: the paper ships no code) on
a bounded, deterministic sample of the same workload on this machine's host cores.
Multi-GPU (torchrun): every rank prepares the same graph and counts its share of the
top-level sub-branches (ticket ranges cut between |VSet| sizes, balanced by estimated
cost); one all-reduce of the exact counts ends the step; value = the graph's cliques /
max rank time ("strong": the total work is fixed).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# k = 9 on this graph holds ~1.4e17 cliques and one full pass takes minutes, so the timed
# step runs k = 5 and 7 and the line adds a k = 9 record of the heaviest sub-branches;
# --ks 5,7,9 puts all three in the timed step.
KS = (5, 7)
WORKLOAD = "chung_lu n=1e6 m=1.0e7 exp=2.1 wmax=1e4 +200 cliques(30-60)"
LIST_K = 5
LIST_CAP = 1 << 24
METRIC = "k-cliques/s (exact)"


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--ks", default=",".join(map(str, KS)))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-k9", action="store_true", help="skip the k = 9 record after the timed steps")
    ap.add_argument("--k9-tickets", type=int, default=2000,
                    help="k = 9 record: the heaviest this many sub-branches (tickets [0, n))")
    ap.add_argument("--workload", choices=["power_law", "batch", "serve", "probe", "ablation"], default="power_law",
                    help="power_law: the default bench line; batch / serve: the batching and serving "
                         "measurements (separate JSON lines); probe: one count on a Chung-Lu graph sized "
                         "by the --probe-* flags, the small case for profiler captures (not a bench value)")
    ap.add_argument("--batch-graphs", type=int, default=4096)
    ap.add_argument("--serve-yield-ms", type=int, default=0,
                    help="serve: how long a count batch waits for queued or running uploads and listings (0 = the server's default)")
    ap.add_argument("--serve-upload-workers", type=int, default=0, help="serve: uploads prepared at once (0 = default)")
    ap.add_argument("--serve-split-min", type=int, default=0,
                    help="serve: |VSet| from which the server's batches split k >= 7 sub-branches (0: library default)")
    ap.add_argument("--probe-n", type=int, default=1_000_000)
    ap.add_argument("--probe-wmax", type=float, default=3000.0)
    ap.add_argument("--probe-k", type=int, default=7)
    ap.add_argument("--probe-checksum", action="store_true")
    ap.add_argument("--probe-tickets", default="", help="b:e -- count only tickets [b, e) (a shard)")
    ap.add_argument("--probe-split-min", default="0",
                    help="comma list of |VSet| split thresholds to time in turn (0: the library default)")
    return ap.parse_args(argv)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------- aggregation (host)
def combine_counts(counts: list[int]) -> int:
    """Exact sum of per-rank 128-bit counts (Python ints)."""
    return sum(counts)


def allgather_ints(values: list[int], world: int):
    """Gather a list of non-negative Python ints (< 2^128) from every rank, as 4 x 32-bit limbs."""
    import torch
    import torch.distributed as dist
    limbs = []
    for v in values:
        limbs += [(v >> (32 * i)) & 0xFFFFFFFF for i in range(4)]
    t = torch.tensor(limbs, dtype=torch.int64)
    if dist.get_backend() == "nccl":
        t = t.cuda()
    out = [torch.zeros_like(t) for _ in range(world)]
    dist.all_gather(out, t)
    res = []
    for o in out:
        o = o.cpu().tolist()
        res.append([sum(o[4 * j + i] << (32 * i) for i in range(4)) for j in range(len(values))])
    return res


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.samples = []
        self.proc = None
        self.th = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        def reader():
            for line in self.proc.stdout:
                self.samples.append([x.strip() for x in line.split(",")])
        self.th = threading.Thread(target=reader, daemon=True)
        self.th.start()

    def stop(self) -> dict:
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.th:
            self.th.join(timeout=2)
        sm = [float(s[1]) for s in self.samples if len(s) > 2 and s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if len(s) > 2 and s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for i, nm in enumerate(names):
                if len(s) > 5 + i and s[5 + i].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


# ---------------------------------------------------------------- reference arm
# one vertex in SAMPLE_STRIDE[k] of the vertices sorted by degree (descending, ties by id):
# a systematic sample, so every degree stratum is represented (its counts scaled by the
# stride estimate the whole graph's within a few per cent)
SAMPLE_STRIDE = {5: 8, 7: 128, 9: 4096}


def cpu_oracle_rate(g, ks) -> dict:
    """The CPU oracle, as it stands, on the same deterministic sample of top vertices in
    both the bench leg and the reference arm: cliques counted per second of its run."""
    import numpy as np

    import oracle as O
    cg = O.CleanGraph.of(g)
    threads = O.threads_default()
    deg = np.diff(cg.row_ptr.astype(np.int64))
    order = np.lexsort((np.arange(g.n), -deg)).astype(np.uint32)
    cnt, spent, parts = 0, 0.0, []
    for k in ks:
        stride = SAMPLE_STRIDE.get(k, 4096)
        tops = np.ascontiguousarray(order[::stride])
        t0 = time.perf_counter()
        r = O.count(cg, k, shortcut=True, checksum=False, threads=threads, tops=tops)
        el = time.perf_counter() - t0
        cnt += r["count"]
        spent += el
        parts.append(f"k={k}: every {stride}th vertex by degree ({tops.size} top vertices), {el:.1f} s")
    return {"rate": cnt / spent if spent else 0.0, "cliques": cnt, "seconds": spent, "threads": threads,
            "sample": "the oracle's degeneracy-ordered vertex branching with the clique shortcut, count only, "
                      "rooted at a systematic sample of the vertices sorted by degree: " + "; ".join(parts)}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from synth import graphs as G
    g = G.chung_lu(seed=0)
    ks = [int(x) for x in args.ks.split(",")]
    # the oracle has no warm state; every step runs the same bounded sample
    tot_c, tot_s, r = 0, 0.0, None
    for _ in range(args.steps):
        r = cpu_oracle_rate(g, ks)
        tot_c += r["cliques"]
        tot_s += r["seconds"]
    val = tot_c / tot_s if tot_s else 0.0
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "k-cliques/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / max(args.steps, 1),
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOAD + f", k={','.join(map(str, ks))}", "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": val, "unit": "k-cliques/s", "cores": r["threads"], "kind": "oracle",
                             "sample": r["sample"]},
            "e2e": {"value": val, "unit": "k-cliques/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm
def run_batch(args):
    """Many small uneven graphs, each with its own k (config 4's shape): one batched call
    with the library defaults, one with the autotuner's per-query picks, against one
    kclique_count per graph; every result checked equal across the three."""
    import collections

    import numpy as np
    import torch

    from paper_2311_13798_gb300 import kclique as K
    from paper_2311_13798_gb300.autotune import Autotuner
    from synth import graphs as G
    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    specs = G.batch_specs(count=args.batch_graphs, seed=0)
    graphs = [G.batch_graph(sp) for sp in specs]
    gen_s = time.perf_counter() - t0
    handles = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for g in graphs:
        rp = torch.from_numpy(g.row_ptr.astype(np.int32)).cuda()
        col = torch.from_numpy(g.col.astype(np.int32)).cuda()
        handles.append(K.kclique_prepare(rp, col, g.n))
    torch.cuda.synchronize()
    prep_s = time.perf_counter() - t0
    ks = [sp["k"] for sp in specs]
    t0 = time.perf_counter()
    tuner = Autotuner(shard=256, reps=1)
    choices = [tuner.choice(h, k) for h, k in zip(handles, ks)]
    tune_s = time.perf_counter() - t0

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(args.steps):
            r = fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t) / args.steps, r

    batch_s, res_b = timed(lambda: K.kclique_count_batch(handles, ks, flags=K.KC_CHECKSUM))
    tuned_s, res_t = timed(lambda: K.kclique_count_batch(handles, ks, choices=choices, flags=K.KC_CHECKSUM))
    single_s, res_s = timed(lambda: [K.kclique_count(h, k, flags=K.KC_CHECKSUM) for h, k in zip(handles, ks)])
    # the tuned batch captured once as a CUDA graph and replayed
    t0 = time.perf_counter()
    plan = K.kclique_batch_plan_create(handles, ks, choices=choices, flags=K.KC_CHECKSUM)
    plan_create_s = time.perf_counter() - t0
    plan_s, res_p = timed(plan.run)
    plan.release()
    key = [(r["count"], r["checksum"]) for r in res_s]
    same = ([(r["count"], r["checksum"]) for r in res_b] == key == [(r["count"], r["checksum"]) for r in res_t] ==
            [(r["count"], r["checksum"]) for r in res_p])
    best_s = min(batch_s, tuned_s, plan_s)
    cliques = sum(r["count"] for r in res_b)
    picked = collections.Counter(json.dumps(c, sort_keys=True) for c in choices)
    line = {"metric": "batched k-clique queries/s", "workload": "batch", "value": len(ks) / best_s,
            "unit": "queries/s", "one_query_per_launch": len(ks) / single_s, "default_batch": len(ks) / batch_s,
            "tuned_batch": len(ks) / tuned_s, "graph_replay_batch": len(ks) / plan_s, "speedup": single_s / best_s,
            "speedup_tuned_vs_default": batch_s / tuned_s, "results_identical": same,
            "ms_graph_replay": plan_s * 1e3, "plan_create_s": plan_create_s,
            "k-cliques/s": cliques / best_s, "n_graphs": len(ks),
            "edges": int(sum(g.m for g in graphs)), "cliques": str(cliques),
            "ms_batch": batch_s * 1e3, "ms_tuned": tuned_s * 1e3, "ms_one_per_launch": single_s * 1e3,
            "tuned_choices": dict(picked.most_common(6)), "tune_s": tune_s, "shape_keys": len(tuner.cache),
            "prepare_s": prep_s, "generate_s": gen_s, "steps": args.steps, "warmup": args.warmup,
            "config": {"graphs": "G(n,p), n~U{64..4096}, avg degree U[8,64], 1-4 planted cliques U{8..24}, "
                                 "k~U{3..10}, seed 0", "checksum": True}}
    print(json.dumps(line), flush=True)


def serve_trace(n_arrivals: int, rate: float, seed: int = 0):
    """Poisson arrivals: 70% count/list queries (50/50) on 8 resident graphs with k ~ U{4..10},
    30% uploads of a small block graph (4 blocks x 250, one of them an exact 2-plex)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n_arrivals))
    kinds = rng.choice(["count", "list", "upload"], size=n_arrivals, p=[0.35, 0.35, 0.30])
    gids = rng.integers(0, 8, size=n_arrivals)
    ks = rng.integers(4, 11, size=n_arrivals)
    return [(float(t[i]), str(kinds[i]), int(gids[i]), int(ks[i]), i) for i in range(n_arrivals)]


def run_serve(args):
    """Continuous-batching server on a Poisson trace vs the same trace run FIFO with one
    query per launch; p50/p99 latency from arrival to completion."""
    import numpy as np
    import torch

    from paper_2311_13798_gb300 import kclique as K
    from paper_2311_13798_gb300.serve import KCliqueServer, Request
    from synth import graphs as G
    torch.cuda.set_device(0)
    base = [G.config1(seed=sd) for sd in range(4)] + \
           [G.chung_lu(n=100_000, w_max=2000.0, i0=40.0, planted=20, seed=sd) for sd in range(4)]
    n_arr = max(200, args.steps * 1000)
    trace = serve_trace(n_arr, 2000.0, seed=0)
    uploads = {}
    for (t, kind, gid, k, i) in trace:
        if kind == "upload":
            g, _ = G.sbm_2plex(blocks=4, block_size=250, p_in=0.9, p_out=1e-3, two_plex_blocks=1, seed=1000 + i)
            uploads[i] = g
    cap = 1024

    def replay_server():
        srv = KCliqueServer(hbm_budget_bytes=120 << 30, split_min=args.serve_split_min,
                            yield_ms=args.serve_yield_ms, upload_workers=args.serve_upload_workers)
        for j, g in enumerate(base):
            srv.register(f"g{j}", g.row_ptr, g.col, g.n)
        torch.cuda.synchronize()
        futs = []
        t0 = time.perf_counter()
        for (t, kind, gid, k, i) in trace:
            now = time.perf_counter() - t0
            if t > now:
                time.sleep(t - now)
            if kind == "upload":
                g = uploads[i]
                req = Request("upload", f"u{i}", csr=(g.row_ptr, g.col, g.n))
            else:
                req = Request(kind, f"g{gid}", k=k, cap=cap)
            futs.append(srv.submit(req))
        res = [f.result(timeout=3600) for f in futs]
        srv.close()
        st = srv.stats()
        return st, res

    def replay_fifo():
        hs = []
        for g in base:
            hs.append(K.kclique_prepare(g.row_ptr, g.col, g.n))
        lat, res, kept = [], [], []
        busy = {"count": 0.0, "list": 0.0, "upload": 0.0}
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for (t, kind, gid, k, i) in trace:
            now = time.perf_counter() - t0
            if t > now:
                time.sleep(t - now)
            tb = time.perf_counter()
            if kind == "upload":
                g = uploads[i]
                kept.append(K.kclique_prepare(g.row_ptr, g.col, g.n))  # resident, as in the server
                res.append(None)
            elif kind == "count":
                r = K.kclique_count(hs[gid], k, flags=K.KC_CHECKSUM)
                res.append((r["count"], r["checksum"]))
                lat.append(time.perf_counter() - t0 - t)
            else:
                o = torch.empty((cap, k), dtype=torch.int32, device="cuda")
                r = K.kclique_list(hs[gid], k, o)
                res.append((r["count"], r["checksum"]))
                lat.append(time.perf_counter() - t0 - t)
            busy[kind] += time.perf_counter() - tb
        span = time.perf_counter() - t0
        for h in kept:
            h.release()
        lat.sort()
        nq = len(lat)
        return {"p50_s": lat[nq // 2], "p99_s": lat[min(nq - 1, int(0.99 * (nq - 1)))], "throughput_qps": nq / span,
                "queries": nq, "busy_s": busy}, res

    st_srv, res_srv = replay_server()
    st_fifo, res_fifo = replay_fifo()
    same = all(a is None or r.kind == "upload" or (r.count, r.checksum) == a
               for r, a in zip(res_srv, res_fifo))
    errors = sorted({r.status for r in res_srv if r.status != "ok" and not r.status.startswith("rejected")})
    line = {"metric": "served k-clique queries/s (continuous batching)", "workload": "serve",
            "value": st_srv["throughput_qps"], "unit": "queries/s", "p50_s": st_srv["p50_s"],
            "p99_s": st_srv["p99_s"], "batches": st_srv["batches"], "mean_batch": st_srv["mean_batch"],
            "rejected": st_srv["rejected"], "span_s": st_srv["span_s"], "busy_s": st_srv["busy_s"],
            "max_batch_seen": st_srv["max_batch_seen"], "one_query_per_launch": st_fifo,
            "speedup": st_srv["throughput_qps"] / st_fifo["throughput_qps"], "results_identical": same,
            "errors": errors[:5],
            "config": {"arrivals": n_arr, "rate_qps": 2000, "split_min": args.serve_split_min,
                       "yield_ms": args.serve_yield_ms or "default", "upload_workers": args.serve_upload_workers or "default",
                       "resident": "4 x G(2000,0.01) seeds 0-3 + "
                       "4 x Chung-Lu n=1e5 wmax=2000 seeds 0-3", "k": "U{4..10}", "mix": "35% count, 35% list "
                       "(cap 1024 rows), 30% upload of 4x250 SBM with one 2-plex block", "hbm_budget_GB": 120}}
    print(json.dumps(line), flush=True)


def run_ablation(args):
    """The paper's ablations (Sec. 6.2): the edge order -- truss-based at the top and the
    colour order inside (EBBkC-H), the colour-based order at every level (EBBkC-C), the
    truss-based order at every level (EBBkC-T, Alg. 3) -- and pruning Rule (2) and early
    termination switched off.  On the power-law graph (n = 1e6) at k = 5 and 7, EBBkC-T at
    k = 5 only (without colours, rules or early termination its k = 7 run would take
    hours); on the same generator at n = 1e5 every order at k = 5 and 7.  Every
    variant's count must agree."""
    import numpy as np
    import torch

    from paper_2311_13798_gb300 import kclique as K
    from synth import graphs as G
    torch.cuda.set_device(0)
    rows = []
    counts = {}

    def timed(h, k, fl):
        r = K.kclique_count(h, k, flags=fl)
        if r["ms_branch"] < 2000.0:  # short: the second, warm run
            r = K.kclique_count(h, k, flags=fl)
        return r

    def ablate(gname, g, plan):
        rp = torch.from_numpy(g.row_ptr.astype(np.int32)).cuda()
        col = torch.from_numpy(g.col.astype(np.int32)).cuda()
        for name, order, variants in plan:
            h = K.kclique_prepare(rp, col, g.n, ordering=order)
            info = K.kclique_info(h)
            for fname, fl, ks in variants:
                for k in ks:
                    r = timed(h, k, fl)
                    counts.setdefault((gname, k), set()).add(r["count"])
                    rows.append({"graph": gname, "ordering": name, "variant": fname, "k": k,
                                 "ms_branch": r["ms_branch"], "ms_prepare": r["ms_prepare"], "nodes": r["nodes"],
                                 "et_hits": r["et_hits"], "edge_branches": r["edge_branches"],
                                 "max_vset": info["tau"], "count": str(r["count"])})
                    print(json.dumps(rows[-1]), flush=True)
            h.release()

    full = (("all on", 0), ("no Rule (2)", K.KC_NO_RULE2), ("no early termination", K.KC_NO_ET))
    tee = ("truss at every level (EBBkC-T)", K.KC_TRUSS_INNER)
    big = G.chung_lu()
    ablate("chung_lu n=1e6", big, (
        ("truss (EBBkC-H)", K.KC_ORDER_TRUSS, [(f, fl, (5, 7)) for f, fl in full]),
        ("colour (EBBkC-C)", K.KC_ORDER_COLOUR, [("all on", 0, (5, 7))])))
    small = G.chung_lu(n=100_000, w_max=2000.0, i0=40.0, planted=20, seed=1)
    ablate("chung_lu n=1e5", small, (
        ("truss (EBBkC-H)", K.KC_ORDER_TRUSS, [("all on", 0, (5, 7)), tee + ((5, 7),)]),
        ("colour (EBBkC-C)", K.KC_ORDER_COLOUR, [("all on", 0, (5, 7))])))
    ablate("chung_lu n=1e6", big, (("truss (EBBkC-H)", K.KC_ORDER_TRUSS, [tee + ((5,),)]),))
    print(json.dumps({"workload": "ablation", "counts_agree": all(len(v) == 1 for v in counts.values()),
                      "rows": len(rows)}), flush=True)


def run_probe(args):
    """Prepare a Chung-Lu graph (n = --probe-n, max expected degree --probe-wmax, seed 0) and
    run one count at k = --probe-k; prints the count, the branch time and the work counters."""
    import numpy as np
    import torch

    from paper_2311_13798_gb300 import kclique as K
    from synth import graphs as G
    torch.cuda.set_device(0)
    g = G.chung_lu(n=args.probe_n, w_max=args.probe_wmax)
    rp = torch.from_numpy(g.row_ptr.astype(np.int32)).cuda()
    col = torch.from_numpy(g.col.astype(np.int32)).cuda()
    h = K.kclique_prepare(rp, col, g.n)
    flags = K.KC_CHECKSUM if args.probe_checksum else 0
    tb, te = (int(x) for x in args.probe_tickets.split(":")) if args.probe_tickets else (0, 0)
    info = K.kclique_info(h)
    for sm in (int(x) for x in args.probe_split_min.split(",")):
        r = K.kclique_count(h, args.probe_k, flags=flags, ticket_begin=tb, ticket_end=te, split_min=sm)
        print(json.dumps({"workload": "probe", "n": g.n, "m": g.m, "w_max": args.probe_wmax, "tau": info["tau"],
                          "k": args.probe_k, "tickets": [tb, te], "split_min": sm, "count": str(r["count"]),
                          "checksum": str(r["checksum"]),
                          "ms_branch": r["ms_branch"], "word_ops": r["word_ops"], "nodes": r["nodes"],
                          "et_hits": r["et_hits"], "kernel_rev": K.kclique_kernel_rev()}), flush=True)


def stored_traffic(K, ks):
    """DRAM bytes (read + write) of one step's branch launches for the counts at ks, from
    the one-pass ncu capture summarised in profiles/ (scaled by nothing: it was taken on
    this workload); None unless the capture was taken with the kernels this library was
    built from."""
    path = os.path.join(ROOT, "profiles", "branch_traffic_power_law.json")
    if not os.path.exists(path):
        return None
    t = json.load(open(path))
    if t.get("kernel_rev") != K.kclique_kernel_rev():
        return None
    per_k = t.get("bytes_per_count", {})
    if not all(str(k) in per_k for k in ks):
        return None
    return sum(int(per_k[str(k)]) for k in ks)


def golden():
    path = os.path.join(ROOT, "tests", "golden", "configs.json")
    return json.load(open(path)) if os.path.exists(path) else {}


def main(argv=None):
    args = parse(argv)
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "batch":
        run_batch(args)
        return
    if args.workload == "serve":
        run_serve(args)
        return
    if args.workload == "probe":
        run_probe(args)
        return
    if args.workload == "ablation":
        run_ablation(args)
        return
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2311_13798_gb300 import kclique as K
    from paper_2311_13798_gb300 import shard
    from synth import graphs as G

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    ks = [int(x) for x in args.ks.split(",")]
    # every rank holds the same graph; the ranks split its top-level sub-branches
    g = G.chung_lu(seed=0)
    rp = torch.from_numpy(g.row_ptr.astype(np.int32)).cuda()
    col = torch.from_numpy(g.col.astype(np.int32)).cuda()
    out = torch.empty((LIST_CAP, LIST_K), dtype=torch.int32, device="cuda")
    out_h = torch.empty((LIST_CAP, LIST_K), dtype=torch.int32).pin_memory()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > 129 MB L2
    stream = torch.cuda.current_stream()
    h0 = K.kclique_prepare(rp, col, g.n)
    vs = K.kclique_edge_data(h0)["vset_size"]
    # this rank's ticket range per k: cut between |VSet| sizes, balanced by estimated cost
    shards = {k: shard.partition_by_size(vs, k, world)[rank] for k in set(ks) | {LIST_K, 9}}
    h0.release()

    def step(host=False, rp_h=None, col_h=None):
        h = K.kclique_prepare(rp_h, col_h, g.n) if host else K.kclique_prepare(rp, col, g.n)
        res = {k: K.kclique_count(h, k, ticket_begin=shards[k][0], ticket_end=shards[k][1]) for k in ks}
        lst = K.kclique_list(h, LIST_K, out, ticket_begin=shards[LIST_K][0], ticket_end=shards[LIST_K][1])
        if host:  # the listing's rows and the results go back to the host
            out_h[: lst["written"]].copy_(out[: lst["written"]], non_blocking=True)
        h.release()
        return res, lst

    def reduce_counts(res):
        if world == 1:
            return {k: r["count"] for k, r in res.items()}
        return {k: shard.allreduce_result(r["count"], 0)[0] for k, r in res.items()}

    for _ in range(args.warmup):
        res, lst = step()
    torch.cuda.synchronize()
    K.kclique_launch_count(reset=True)
    if world > 1:
        dist.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    torch.cuda.synchronize()
    times, cliques = [], 0
    phase = {"prepare": 0.0}
    branch_ms = {k: 0.0 for k in ks}
    word_ops = {k: 0 for k in ks}
    edge_branches = {k: 0 for k in ks}
    totals = {}
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res, lst = step()
        totals = reduce_counts(res)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        cliques += sum(totals.values())
        phase["prepare"] += lst["ms_prepare"]
        for k, r in res.items():
            branch_ms[k] += r["ms_branch"]
            word_ops[k] += r["word_ops"]
            edge_branches[k] += r["edge_branches"]
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    launches = K.kclique_launch_count()
    my_ms = sum(times)
    if world > 1:
        t = torch.tensor([my_ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_ms = float(t.item())
    else:
        tot_ms = my_ms
    value = cliques / (tot_ms / 1e3)

    e2e = None
    if not args.no_e2e:
        rp_h = torch.from_numpy(g.row_ptr.astype(np.int32)).pin_memory()
        col_h = torch.from_numpy(g.col.astype(np.int32)).pin_memory()
        step(True, rp_h, col_h)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        n_e2e, c_e2e, rows = max(1, min(args.steps, 2)), 0, 0
        for _ in range(n_e2e):
            res_e, lst_e = step(True, rp_h, col_h)
            c_e2e += sum(reduce_counts(res_e).values())
            rows = lst_e["written"]
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        if world > 1:
            t = torch.tensor([el], dtype=torch.float64, device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            el = float(t.item())
        e2e = {"value": c_e2e / el, "unit": "k-cliques/s",
               "h2d_bytes_per_step": int(4 * (g.n + 1) + 4 * g.col.size),
               # the listing's rows plus one result record per call
               "d2h_bytes_per_step": int(4 * LIST_K * rows + 72 * (len(ks) + 1))}

    # self-check against the oracle's stored values (outside the timed region): the
    # counts of the timed steps, and the checksums from one pass with KC_CHECKSUM
    gold = golden()
    verified = None
    if all(f"c2/k{k}" in gold for k in ks) and g.fingerprint() == gold.get("c2/graph", {}).get("fingerprint"):
        h = K.kclique_prepare(rp, col, g.n)
        sums = {}
        for k in ks:
            r = K.kclique_count(h, k, flags=K.KC_CHECKSUM, ticket_begin=shards[k][0], ticket_end=shards[k][1])
            c, cs = (r["count"], r["checksum"]) if world == 1 else shard.allreduce_result(r["count"], r["checksum"])
            sums[k] = (c, cs)
        h.release()
        verified = all(str(totals[k]) == gold[f"c2/k{k}"]["count"] and str(sums[k][0]) == gold[f"c2/k{k}"]["count"]
                       and str(sums[k][1]) == gold[f"c2/k{k}"]["checksum"] for k in ks)

    # k = 9 on the same graph: its heaviest sub-branches (a fixed ticket range) timed once
    # after the steps; the full pass takes minutes and is recorded with the profiles
    k9 = None
    if not args.no_k9 and 9 not in ks:
        h = K.kclique_prepare(rp, col, g.n)
        tb, te = 0, min(args.k9_tickets, shards[9][1])
        r = K.kclique_count(h, 9, ticket_begin=tb, ticket_end=te) if rank == 0 and te > tb else None
        h.release()
        if r is not None:
            k9 = {"tickets": [tb, te], "count": str(r["count"]), "ms_branch": r["ms_branch"],
                  "k-cliques/s": r["count"] / (r["ms_branch"] / 1e3) if r["ms_branch"] else None,
                  "edge_branches_per_s": r["edge_branches"] / (r["ms_branch"] / 1e3) if r["ms_branch"] else None}

    # roofline of the dominant kernels (the branch kernels of kclique_count): algorithmic
    # bitset lane-ops (3 per word of every candidate-set intersection, 2 per word of every
    # degree test, counted in-kernel) over their CUDA-event time, against the measured
    # AND+AND+POPC peak of this GPU
    # the dominant kernels are the branch launches of the count that takes longest (k = 7
    # on this workload: more than half the step); k = 5's time is mostly extraction
    peak = K.kclique_int_peak()["lane_ops_per_s"]
    kd = max(ks, key=lambda k: branch_ms[k])
    achieved = word_ops[kd] / (branch_ms[kd] / 1e3) if branch_ms[kd] else 0.0
    roof = {"bound": "alu", "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "G lane-ops/s",
            "frac": achieved / peak if peak else None, "traffic": stored_traffic(K, [kd]),
            "kernel": f"branch_kernel + branch_items_kernel of the k = {kd} count (all width classes), "
                      "measured live with CUDA events",
            "all_counts_frac": (sum(word_ops.values()) / (sum(branch_ms.values()) / 1e3) / peak
                                if sum(branch_ms.values()) and peak else None),
            "peak_kind": "measured AND+AND+POPC microbenchmark (kclique_int_peak) on this GPU"}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r = cpu_oracle_rate(g, ks)
        cpu = {"value": r["rate"], "unit": "k-cliques/s", "cores": r["threads"], "kind": "oracle",
               "sample": r["sample"]}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "k-cliques/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
                "scaling": "strong", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
                "config": {"workload": WORKLOAD + f", k={','.join(map(str, ks))} + list k={LIST_K} cap 2^24",
                           "graph": g.fingerprint(), "m": g.m,
                           "parallelism": f"{world} rank(s), one graph split by |VSet| ranges",
                           "l2": "flushed (256 MB write) before every step",
                           "ms_prepare": phase["prepare"] / args.steps,
                           "ms_count": {k: v / args.steps for k, v in branch_ms.items()},
                           "counts": {k: str(v) for k, v in totals.items()},
                           "verified": verified, "k9": k9},
                "clocks": clocks, "e2e": e2e, "roofline": roof, "cpu_baseline": cpu,
                "gpu_launches": launches,
                # top-level sub-branches (one per edge with |VSet| >= k-2) run per second of
                # branch-kernel time, per k (this rank's)
                "edge_branches_per_s": {k: (edge_branches[k] / (branch_ms[k] / 1e3) if branch_ms[k] else None)
                                        for k in ks}}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
