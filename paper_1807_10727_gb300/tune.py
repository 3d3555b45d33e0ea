"""Autotuner of the library's speed parameters, per graph-size class.

The parameters (lc_set_param: vertex blocks of the phase-0 edge buckets and
whether phase 0 groups its edges at all, the vertex window of the ungrouped
minimum, size and admission of the device-wide duplicate cache, the edge count from which phases plan their
deduplication late, segmented or bucket-partition deduplication) change the
speed of a run, never its result.  For each size
class, represented by one synthetic graph of the benchmark's recipes (or,
for the batch class, the benchmark's batch of 4096 graphs run as one), this
script times whole runs (CUDA events, after warm-up) and improves the
parameters by coordinate descent from the library's defaults: one parameter
at a time over its candidate values, keeping the best, two sweeps.  The
table it writes (tuned.json beside this file) maps each class, keyed by its
kind (single graph or batch) and by ceil(log2 n) and ceil(log2 m) of the
total sizes, to its parameters and to the measured times with the defaults
and with the tuned values.  LocalContraction applies the entry of the
nearest single-graph class, BatchLocalContraction that of the nearest batch
class (tuned=True, the default).

Run on the GPU that will run the library:
    python -m paper_1807_10727_gb300.tune [--classes rmat20,rmat26] [--out FILE] [--merge]
(--merge keeps the other classes' rows of an existing table.)
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE = os.path.join(HERE, "tuned.json")

# candidate values; the library's default comes first
CANDIDATES = {
    "bucket_window_bytes": [64 << 20, 32 << 20, 128 << 20],
    "relabel_cache_slots": [1 << 23, 1 << 22, 1 << 24, 1 << 21],
    "relabel_cache_admit": [3, 2, 4],
    "late_min_edges": [1 << 22, 1 << 20, 1 << 24],
    "seg_dedup": [1, 0],
    "bucket_blocks": [0, 1],  # phase-0 edge grouping: automatic, or off
    "window_bytes": [192 << 20, 2 << 30],  # ungrouped minimum: L2-sized windows, or one pass
}

# size classes: one workload each (synth.workload names; "batch<k>": synth.batch(k))
CLASSES = ["rmat18", "rmat20", "rmat22", "rmat24", "rmat26", "gridmix", "batch4096"]


def class_key(n: int, m: int) -> tuple[int, int]:
    return (max(0, math.ceil(math.log2(max(n, 1)))), max(0, math.ceil(math.log2(max(m, 1)))))


_table = None


def load_table(path: str = TABLE) -> list:
    global _table
    if _table is None:
        try:
            with open(path) as f:
                _table = json.load(f).get("classes", [])
        except (OSError, ValueError):
            _table = []
    return _table


def params_for(n: int, m: int, kind: str = "single", max_distance: float = 2.0) -> dict:
    """Tuned parameters of the class of this kind ("single" or "batch")
    nearest to (n, m) in (log2 n, log2 m), or {} when none is within
    max_distance."""
    kn, km = class_key(n, m)
    best, bd = None, None
    for c in load_table():
        if c.get("kind", "single") != kind:
            continue
        d = math.hypot(c["n_log2"] - kn, c["m_log2"] - km)
        if bd is None or d < bd:
            best, bd = c, d
    if best is None or bd > max_distance:
        return {}
    return dict(best["params"])


def _time_run(lc, g, src, dst, labels, params, steps, warmup):
    import torch
    ctx = lc.LocalContraction(g.n, src, dst, seed=g.seed, tuned=False)
    try:
        for k, v in params.items():
            ctx.set_param(k, int(v))
        for _ in range(warmup):
            ctx.run(labels)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            ctx.run(labels)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps
    finally:
        ctx.close()


def _time_batch(lc, b, src, dst, labels, params, steps, warmup):
    import torch
    ctx = lc.BatchLocalContraction(b.n, b.eoff, src, dst, b.seeds, tuned=False)
    try:
        for k, v in params.items():
            ctx.set_param(k, int(v))
        for _ in range(warmup):
            ctx.run(labels)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            ctx.run(labels)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps
    finally:
        ctx.close()


def tune_class(name: str, steps: int = 5, warmup: int = 2, sweeps: int = 2, log=print) -> dict:
    import torch

    from . import lc, synth
    dev = torch.device("cuda")
    if name.startswith("batch"):
        kind = "batch"
        g = synth.batch(k=int(name[len("batch"):] or 4096))
        n_tot, m_tot = int(g.n.astype(np.int64).sum()), int(g.eoff[-1])
        labels = torch.empty(max(n_tot, 1), dtype=torch.int32, device=dev)
        timer = _time_batch
    else:
        kind = "single"
        g = synth.workload(name)
        n_tot, m_tot = g.n, g.m
        labels = torch.empty(g.n, dtype=torch.int32, device=dev)
        timer = _time_run
    src = torch.from_numpy(g.src.view(np.int32)).to(dev)
    dst = torch.from_numpy(g.dst.view(np.int32)).to(dev)
    best = {k: v[0] for k, v in CANDIDATES.items()}
    default_ms = timer(lc, g, src, dst, labels, {}, steps, warmup)
    best_ms = timer(lc, g, src, dst, labels, best, steps, warmup)
    trials = 2
    for _ in range(sweeps):
        for name_p, values in CANDIDATES.items():
            for v in values:
                if v == best[name_p]:
                    continue
                trial = dict(best, **{name_p: v})
                ms = timer(lc, g, src, dst, labels, trial, steps, warmup)
                trials += 1
                if ms < best_ms * 0.99:  # keep a change only if it gains over 1%
                    best, best_ms = trial, ms
    kn, km = class_key(n_tot, m_tot)
    log("tune %s (n=%d, m=%d): default %.3f ms, tuned %.3f ms, %d trials, %s"
        % (name, n_tot, m_tot, default_ms, best_ms, trials, best))
    del src, dst, labels
    torch.cuda.empty_cache()
    return {"workload": name, "kind": kind, "n": n_tot, "m": m_tot, "n_log2": kn, "m_log2": km,
            "params": best, "default_ms": default_ms, "tuned_ms": best_ms, "trials": trials}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--classes", default=",".join(CLASSES))
    ap.add_argument("--out", default=TABLE)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--merge", action="store_true",
                    help="replace only the tuned classes' rows of an existing table")
    args = ap.parse_args(argv)
    import torch

    from . import lc
    lc.load()
    t0 = time.time()
    rows = []
    for name in args.classes.split(","):
        rows.append(tune_class(name.strip(), steps=args.steps,
                               log=lambda s: print("[tune] " + s, file=sys.stderr, flush=True)))
    if args.merge and os.path.exists(args.out):
        with open(args.out) as f:
            old = json.load(f).get("classes", [])
        names = {r["workload"] for r in rows}
        rows = [r for r in old if r.get("workload") not in names] + rows
    out = {"device": torch.cuda.get_device_name(0), "when": time.strftime("%Y-%m-%dT%H:%M:%SZ",
                                                                          time.gmtime()),
           "seconds": round(time.time() - t0, 1), "candidates": CANDIDATES, "classes": rows}
    with open(args.out, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
