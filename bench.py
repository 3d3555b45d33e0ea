"""Benchmark: input edges/s of the LocalContraction connected-components path
on one GB300 (R-MAT scale 26, 2^30 edges, permuted ids, rank seed 7).

One step = one lc_run over the whole phase loop (rank, closed-neighbourhood
minimum, pointer jumping, relabel / deduplicate / compact every phase, then
label composition) with the input already resident in HBM.  The input (8 GiB)
is far larger than the 129 MB L2, so no flush is needed between steps.  The
headline steps run with the library's per-launch event timing off; a second,
profiled pass of the same steps gives the per-kernel split.

Extra keys on the JSON line:
  roofline       the dominant step (one of parent, contract, relabel, dedup,
                 compact, labels; each the sum of its kernels): its
                 algorithmic bytes per run / its device time per run (CUDA
                 events, profiled pass), against the measured HBM copy peak.
  step_rooflines the same figures for every step, with the kernels each holds.
  path_roofline  all algorithmic bytes of a run / the headline step time.
  e2e            the same metric through lc_run_host (pinned host buffers;
                 host->device copy of the edges and device->host copy of the
                 labels inside the timed region).
  cpu_baseline   the CPU oracle (single thread) on a smaller graph of the same
                 recipe (R-MAT scale 22, edge factor 16), with the host's core
                 count and CPU model.
  configs        the ER (config 1) and grid-mix (config 3) workloads: GPU
                 edges/s, path fraction, and the oracle's edges/s on a sample.
  batched, serving  the batched (config 4) and serving (config 5) legs.

Algorithmic bytes (what the method itself must move; no sort-pass
multiplicity, no random-gather sector amplification), per phase i with n_i
vertices, m_i edges, m'_i non-loop relabelled edges and m_{i+1} distinct ones:
  parent   8 m_i (read edges) + 8 n_i (write minima)
  contract 4 n_i (read parents) + 8 n_i (one pointer pass, read + write)
  relabel  8 m_i (read edges) + 8 m'_i (write keys) + 4 n_i (read roots)
  dedup    16 m'_i (read + write keys)
  compact  8 m_{i+1} (write renamed edges) + 4 n_i (flags / scan)
  labels   8 n_i per phase + 8 n_0 (compose the maps down to level 0)

--impl reference times the CPU oracle (the reference arm is the oracle written
from the paper) on a bounded sample per step.  Multi-GPU (--gpus N under
torchrun): the single-graph path does not shard, so every rank runs its own
replica (weak scaling); value = all ranks' edges / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import platform
import subprocess
import sys
import time

import numpy as np

REPO = os.path.dirname(os.path.abspath(__file__))
if REPO not in sys.path:
    sys.path.insert(0, REPO)

METRIC = "input edges/sec to final labels (1 GB300), HBM roofline %"
UNIT = "edges/s"
CPU_SAMPLE = "rmat22"     # cpu_baseline: one oracle run, about 10 s
REF_SAMPLE = "rmat21"     # reference arm: one oracle run per step, a few seconds

# Kernels (lc_kernel_stats names) of each step of the path.  The phase-0 edge
# grouping serves the parent and relabel steps; it is counted in parent, the
# first step that reads the grouped edges.
STEP_KERNELS = {
    "parent": ["bucket_edges", "init_keys", "edge_min_soa", "edge_min_packed"],
    "contract": ["jump"],
    "relabel": ["relabel_soa", "relabel_packed", "relabel_split"],
    "dedup": ["filter_hll", "sort_hist", "hist_scan", "sort_pass", "bucket_bounds",
              "bucket_dedup", "unmix", "unique_rename", "seg_dedup"],
    "compact": ["scan_flags", "rename"],
    "labels": ["propagate", "identity"],
}

# DRAM bytes (ncu dram__bytes_read.sum + dram__bytes_write.sum) per
# algorithmic byte of a step, measured on R-MAT 23 with one-kernel captures
# of phase 0, keyed by the hash of the CUDA sources they were taken on: a
# changed kernel invalidates them (the line then reports traffic null).
TRAFFIC = {"sources": "5671513a3cdfe5d5", "workload": "rmat23",
           "per_alg_byte": {"parent": 3.833, "relabel": 0.875, "dedup": 1.000}}


def sources_hash() -> str:
    h = hashlib.sha256()
    d = os.path.join(REPO, "paper_1807_10727_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cuh")):
            with open(os.path.join(d, f), "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:16]


def peaks():
    path = os.path.join(REPO, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def step_bytes(n_i, m_i, mp_i):
    """Algorithmic bytes of one run per step (module docstring)."""
    out = {k: 0 for k in STEP_KERNELS}
    R = len(n_i)
    for i in range(R):
        n, m, mp = int(n_i[i]), int(m_i[i]), int(mp_i[i])
        m_next = int(m_i[i + 1]) if i + 1 < R else 0
        out["parent"] += 8 * m + 8 * n
        out["contract"] += 4 * n + 8 * n
        out["relabel"] += 8 * m + 8 * mp + 4 * n
        out["dedup"] += 16 * mp
        out["compact"] += 8 * m_next + 4 * n
        out["labels"] += 8 * n
    if R:
        out["labels"] += 8 * int(n_i[0])
    return out


def path_bytes(n_i, m_i, mp_i):
    return sum(step_bytes(n_i, m_i, mp_i).values())


def variant_path_bytes(variant, finish, n_i, m_i, mp_i):
    """path_bytes plus what a variant adds: the two-hop label reads every edge
    once more and writes and copies a second n-word key array per phase; the
    union-find finish phase reads its edges once for the unions."""
    total = path_bytes(n_i, m_i, mp_i)
    for n, m in zip(n_i, m_i):
        if finish and m <= finish:
            total += 8 * m + 8 * n
        elif variant == 1:
            total += 8 * m + 8 * n + 16 * n + 8 * n
    return total


def step_report(kstats, runs, n_i, m_i, mp_i, peak, peak_kind):
    """Per-step device time (sum of its kernels' event-timed launches) and
    algorithmic bandwidth; kstats: name -> (launches, ms) over `runs` runs."""
    sb = step_bytes(n_i, m_i, mp_i)
    steps = {}
    for step, names in STEP_KERNELS.items():
        ms = sum(kstats.get(k, (0, 0.0))[1] for k in names) / runs
        launches = sum(kstats.get(k, (0, 0.0))[0] for k in names) / runs
        ach = sb[step] / (ms / 1e3) / 1e9 if ms > 0 else None
        steps[step] = {"algorithmic_bytes": sb[step], "ms": ms, "launches": launches,
                       "achieved_gbs": ach, "frac": (ach / peak) if ach else None,
                       "kernels": {k: round(kstats[k][1] / runs, 4) for k in names
                                   if k in kstats and kstats[k][0]}}
    return steps


def roofline_of(steps, peak, peak_kind, workload):
    top = max(steps, key=lambda k: steps[k]["ms"])
    s = steps[top]
    traffic = None
    ratio = TRAFFIC["per_alg_byte"].get(top)
    if ratio and TRAFFIC["sources"] == sources_hash():
        traffic = ratio * s["algorithmic_bytes"]
    return {"bound": "hbm", "step": top, "kernels": sorted(s["kernels"]),
            "achieved": s["achieved_gbs"], "peak": peak, "unit": "GB/s", "frac": s["frac"],
            "peak_kind": peak_kind, "traffic": traffic,
            "traffic_note": ("DRAM bytes per run from one-kernel ncu captures on %s, scaled by "
                             "algorithmic bytes" % TRAFFIC["workload"]) if traffic else
                            "no capture of the current kernels",
            "algorithmic_bytes_per_run": s["algorithmic_bytes"], "ms_per_run": s["ms"],
            "launches_per_run": s["launches"]}


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = os.path.join("/tmp", "lc_clocks_%d.csv" % os.getpid())

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_id_for(device_index: int) -> str:
    import torch
    try:
        p = torch.cuda.get_device_properties(device_index)
        return "%08x:%02x:%02x.0" % (p.pci_domain_id, p.pci_bus_id, p.pci_device_id)
    except Exception:
        return str(device_index)


def host_info() -> dict:
    model = platform.processor() or platform.machine()
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model}


def oracle_rate(g, runs=1):
    """Edges/s of the oracle (single-threaded C++) over whole runs on g."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    for _ in range(runs):
        oracle.lc_run(g.n, g.src, g.dst, g.seed)
    dt = (time.perf_counter() - t0) / runs
    return g.m / dt, dt


def cpu_baseline():
    """The oracle on one smaller graph of the benchmark's recipe (R-MAT scale
    22 = 2^22 vertices, 2^26 edges, same quadrant probabilities, edge factor
    and permuted ids): the whole run, all phases, one thread."""
    from paper_1807_10727_gb300 import synth
    g = synth.workload(CPU_SAMPLE)
    rate, dt = oracle_rate(g)
    return dict({"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                 "sample": "whole oracle run on %s (n = %d, m = %d; the R-MAT 26 recipe at "
                           "scale 22), %.1f s" % (CPU_SAMPLE, g.n, g.m, dt)}, **host_info())


def time_steps(ctx, labels, stream, steps):
    import torch
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        ctx.run(labels)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def bench_config(name, dev, stream, steps, warmup, peak, lc, synth, oracle_sample):
    """GPU edges/s and path fraction of a named workload, plus the oracle's
    edges/s on `oracle_sample` (the workload itself or a smaller graph of its
    recipe)."""
    import torch
    g = synth.workload(name)
    src = torch.from_numpy(g.src.view(np.int32)).to(dev)
    dst = torch.from_numpy(g.dst.view(np.int32)).to(dev)
    labels = torch.empty(g.n, dtype=torch.int32, device=dev)
    ctx = lc.LocalContraction(g.n, src, dst, seed=g.seed, stream=stream)
    for _ in range(warmup):
        _, res = ctx.run(labels)
    mp, _ = lc.lc_last_stats(ctx.ctx)
    ms = time_steps(ctx, labels, stream, steps)
    ctx.close()
    del src, dst, labels
    torch.cuda.empty_cache()
    pb = path_bytes(res.n_i, res.m_i, mp)
    og = g if oracle_sample == name else synth.workload(oracle_sample)
    orate, odt = oracle_rate(og)
    out = {"n": g.n, "m": g.m, "rounds": res.rounds, "value": g.m / (ms / 1e3), "unit": UNIT,
           "ms_per_step": ms, "path_frac": pb / (ms / 1e3) / 1e9 / peak,
           "oracle_value": orate, "oracle_sample": "%s (n = %d, m = %d), %.2f s" % (
               oracle_sample, og.n, og.m, odt)}
    log("config %s: %.3f ms/step, %.3g edges/s, oracle %.3g edges/s" % (
        name, ms, out["value"], orate))
    return out


def bench_variants(ctx, labels, stream, steps, warmup, peak, lc):
    """The other phase variants and the union-find finish on the same graph
    and context as the headline: edges/s, phases and the path roofline."""
    out = {}
    # MergeToLarge parameters: alpha_0 = 4 ln n, squared every phase (the
    # recurrence of the O(log log n) argument, Section 5), capped at n
    a, alpha = 4 * math.log(ctx.n), []
    for _ in range(12):
        alpha.append(int(min(a, ctx.n)))
        a *= a
    cases = [("two_hop", lc.LC_VARIANT_TWO_HOP, 0, ()), ("tree", lc.LC_VARIANT_TREE, 0, ()),
             ("forest_finish_4M", lc.LC_VARIANT_FOREST, 1 << 22, ()),
             ("forest_finish_64M", lc.LC_VARIANT_FOREST, 1 << 26, ()),
             ("forest_merge_to_large", lc.LC_VARIANT_FOREST, 0, alpha),
             ("two_hop_merge_to_large", lc.LC_VARIANT_TWO_HOP, 0, alpha)]
    for name, variant, finish, merge in cases:
        lc.lc_configure(ctx.ctx, variant, finish)
        lc.lc_set_merge_to_large(ctx.ctx, merge)
        for _ in range(warmup):
            _, res = ctx.run(labels)
        mp, _ = lc.lc_last_stats(ctx.ctx)
        ms = time_steps(ctx, labels, stream, steps)
        ctx.profile(True)
        time_steps(ctx, labels, stream, 2)
        ks = ctx.kernel_stats()
        ctx.profile(False)
        pb = variant_path_bytes(variant, finish, res.n_i, res.m_i, mp)
        top = sorted(((v[1] / 2, k) for k, v in ks.items() if v[0]), reverse=True)[:4]
        out[name] = {"value": res.m_i[0] / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
                     "rounds": res.rounds, "sizes": [[int(a), int(b)] for a, b in
                                                     zip(res.n_i, res.m_i)],
                     "path_frac": pb / (ms / 1e3) / 1e9 / peak,
                     "gpu_launches_per_step": sum(v[0] for v in ks.values()) / 2,
                     "top_kernels_ms": {k: round(t, 3) for t, k in top}}
        if merge:
            out[name]["merge_alpha"] = list(merge[:res.rounds])
        log(f"variant {name}: {ms:.2f} ms/step, {res.rounds} phases")
    lc.lc_configure(ctx.ctx, lc.LC_VARIANT_FOREST, 0)
    lc.lc_set_merge_to_large(ctx.ctx, [])
    return out


def bench_batch(dev, stream, steps=9, k=4096, world=1, rank=0, barrier=None, reduce_max=None):
    """Config 4: 4096 independent graphs (n log-uniform in [2^6, 2^16]; half ER
    with average degree 4, half R-MAT with average degree 16), one batched
    context vs one lc_run per graph on the same GPU (contexts created up front
    in both cases; creation is not timed).  With several ranks each rank runs
    a size-balanced share of the graphs (no collective on the data path) and
    the batched rate is all graphs over the slowest rank's time; the
    one-run-per-graph comparison runs on a single rank only."""
    import torch

    from paper_1807_10727_gb300 import lc, shard, synth
    full = synth.batch(k=k)
    mine = shard.balance(shard.graph_work(full.n, np.diff(full.eoff)), world)[rank]
    n_, eoff_, src_, dst_, seeds_ = shard.sub_batch(full.n, full.eoff, full.src, full.dst,
                                                    full.seeds, mine)
    b = synth.Batch(n_, eoff_, src_, dst_, seeds_)
    k_mine = b.k
    src = torch.from_numpy(b.src.view(np.int32)).to(dev)
    dst = torch.from_numpy(b.dst.view(np.int32)).to(dev)
    total = int(b.n.astype(np.int64).sum())
    labels = torch.empty(max(total, 1), dtype=torch.int32, device=dev)
    # the tuned and the default context take turns, each run timed alone, so
    # that drift of the box between the two does not decide the comparison
    bls = {True: lc.BatchLocalContraction(b.n, b.eoff, src, dst, b.seeds, stream=stream,
                                          tuned=True)}
    params = dict(bls[True].params)
    if params:
        bls[False] = lc.BatchLocalContraction(b.n, b.eoff, src, dst, b.seeds, stream=stream,
                                              tuned=False)
    for bl in bls.values():
        for _ in range(2):
            bl.run(labels)
    samples = {t: [] for t in bls}
    rounds = None
    for _ in range(steps):
        for t, bl in bls.items():
            torch.cuda.synchronize(dev)
            if barrier:
                barrier()
            t0 = time.perf_counter()
            _, r, _, _ = bl.run(labels)
            torch.cuda.synchronize(dev)
            sec = time.perf_counter() - t0
            samples[t].append(reduce_max(sec) if reduce_max else sec)
            if t:
                rounds = r
    for bl in bls.values():
        bl.close()
    batched_s = float(np.median(samples[True]))
    default_s = float(np.median(samples[False])) if params else batched_s
    workload = "4096 graphs, n log-uniform [2^6, 2^16], ER deg 4 / R-MAT deg 16"
    if world > 1:
        return {"workload": workload, "graphs": k, "ranks": world, "graphs_this_rank": k_mine,
                "batched_graphs_per_s": k / batched_s, "batched_ms": batched_s * 1e3,
                "tuned_params": params, "default_params_ms": default_s * 1e3}
    # one context and one lc_run per graph
    voff = np.concatenate([[0], np.cumsum(b.n.astype(np.int64))])
    ctxs = []
    k = k_mine
    for g in range(k):
        lo, hi = int(b.eoff[g]), int(b.eoff[g + 1])
        ctxs.append(lc.LocalContraction(int(b.n[g]), src[lo:hi], dst[lo:hi], seed=int(b.seeds[g]),
                                        stream=stream))
    for g in range(min(k, 64)):
        ctxs[g].run(labels[voff[g]:voff[g + 1]])
    torch.cuda.synchronize(dev)
    lat = np.empty(k)
    t0 = time.perf_counter()
    for g in range(k):
        t1 = time.perf_counter()
        ctxs[g].run(labels[voff[g]:voff[g + 1]])
        lat[g] = time.perf_counter() - t1
    serial_s = time.perf_counter() - t0
    for c in ctxs:
        c.close()
    return {"workload": workload, "graphs": k, "vertices": total, "edges": int(b.eoff[-1]),
            "max_rounds": int(rounds.max()),
            "batched_graphs_per_s": k / batched_s, "batched_ms": batched_s * 1e3,
            "tuned_params": params, "default_params_ms": default_s * 1e3,
            "per_graph_graphs_per_s": k / serial_s, "per_graph_ms_total": serial_s * 1e3,
            "per_graph_latency_ms_p50": float(np.percentile(lat, 50) * 1e3),
            "per_graph_latency_ms_p99": float(np.percentile(lat, 99) * 1e3),
            "speedup": serial_s / batched_s}


SERVING_RATES = (100.0, 300.0, 1000.0, 3000.0, 10000.0, 20000.0)


def bench_serving(rates=SERVING_RATES, requests=1000, pool=200, slots=32, serial_max_s=20.0,
                  world=1, rank=0, barrier=None, gather=None):
    """Config 5: Poisson arrivals of CC requests (ER / R-MAT / permuted grid,
    n log-uniform in [2^10, 2^22], average degree 4-32) served by the
    continuous-batching loop vs the serial plain path (one request at a time,
    lc_run_host, in arrival order).  Latency = arrival to labels on the host.
    Each rate point replays `requests` arrivals drawn cyclically from a pool
    of `pool` generated graphs (host memory bounds the distinct graphs); the
    serial path is measured at every rate it can sustain, up to serial_max_s
    of arrivals.  With several ranks every rank sees the same arrival
    sequence, routes it with shard.Router (no collective on the data path)
    and serves its own requests on its own GPU; the latencies are gathered
    on rank 0 after each rate point."""
    import threading

    from paper_1807_10727_gb300 import lc, shard, synth
    reqs = synth.serving_stream(1000.0, pool)
    log("serving: %d distinct requests generated" % pool)
    edges = int(sum(r.graph.m for r in reqs))
    # unit-rate Poisson arrival offsets, shared by every rate point
    u = synth.uniforms(515, requests)
    base = np.cumsum(-np.log1p(-u))
    owner = shard.route_stream([reqs[k % pool].graph.m + reqs[k % pool].graph.n
                                for k in range(requests)], world)
    mine = [k for k in range(requests) if owner[k] == rank]

    def summarize(lat, t_first, t_last):
        lat = np.asarray(lat)
        return {"graphs_per_s": float(len(lat) / (t_last - t_first)),
                "latency_ms_p50": float(np.percentile(lat, 50) * 1e3),
                "latency_ms_p99": float(np.percentile(lat, 99) * 1e3), "requests": len(lat)}

    out = {"workload": "%d arrivals per rate over %d distinct requests (ER/R-MAT/grid, n in "
                       "[2^10, 2^22], degree 4-32, %d edges in the pool)" % (requests, pool, edges),
           "slots": slots, "ranks": world, "rates": [], "serial": []}
    srv = lc.Server(slots=slots)
    # warm-up: every distinct request once, so the timed arrivals find idle
    # contexts of every size in the server's pool (steady state)
    warm = [srv.submit(r.graph.n, r.graph.src, r.graph.dst, r.graph.seed) for r in reqs]
    for j in warm:
        srv.wait(j)
    for rate in rates:
        arr = base / rate
        ids = {}
        ready = threading.Semaphore(0)
        if barrier:
            barrier()
        t0 = time.time() + 0.05  # wall clock: the same arrival instants on every rank

        def producer():
            for k in mine:
                r = reqs[k % pool]
                d = t0 + arr[k] - time.time()
                if d > 0:
                    time.sleep(d)
                ids[k] = srv.submit(r.graph.n, r.graph.src, r.graph.dst, r.graph.seed)
                ready.release()

        th = threading.Thread(target=producer)
        th.start()
        lat, t_last = [], t0
        for k in mine:
            if not ready.acquire(timeout=300):
                raise RuntimeError("serving: request %d was not submitted within 300 s" % k)
            _, _, l = srv.wait(ids[k], timeout_s=300.0)
            lat.append(l)
            t_last = max(t_last, t0 + arr[k] + l)
        th.join()
        if gather is not None and world > 1:
            parts = gather((lat, t_last))
            if rank != 0:
                continue
            lat = [x for p in parts for x in p[0]]
            t_last = max(p[1] for p in parts)
        row = summarize(lat, t0, t_last)
        row["rate_req_s"] = rate
        row["saturated"] = bool(row["graphs_per_s"] < 0.9 * rate)
        out["rates"].append(row)
        log("serving: rate %g: %.0f graphs/s, p50 %.1f ms, p99 %.1f ms" % (
            rate, row["graphs_per_s"], row["latency_ms_p50"], row["latency_ms_p99"]))
    out["peak_active"] = srv.stats()["peak_active"]
    srv.close()
    if rank != 0:
        return None
    sat = [r["rate_req_s"] for r in out["rates"] if r["saturated"]]
    out["saturation_req_s"] = min(sat) if sat else None
    if world > 1:
        return out
    # serial plain path: every rate up to the first one it cannot sustain
    for rate in rates:
        n_req = int(min(requests, max(50, serial_max_s * rate)))
        arr = base[:n_req] / rate
        lat = []
        t0 = time.perf_counter() + 0.05
        for k in range(n_req):
            r = reqs[k % pool]
            d = t0 + arr[k] - time.perf_counter()
            if d > 0:
                time.sleep(d)
            c = lc.LocalContraction(r.graph.n, m=r.graph.m, seed=r.graph.seed)
            c.run_host(r.graph.src, r.graph.dst)
            c.close()
            lat.append(time.perf_counter() - (t0 + arr[k]))
        row = summarize(lat, t0, time.perf_counter())
        row["rate_req_s"] = rate
        row["saturated"] = bool(row["graphs_per_s"] < 0.9 * rate)
        out["serial"].append(row)
        log("serving serial: rate %g: %.0f graphs/s, p99 %.1f ms" % (
            rate, row["graphs_per_s"], row["latency_ms_p99"]))
        if row["saturated"]:
            break
    return out


def _plain(x):
    """JSON form of numpy scalars and arrays."""
    if isinstance(x, np.generic):
        return x.item()
    if isinstance(x, np.ndarray):
        return x.tolist()
    raise TypeError("not JSON serializable: %r" % type(x))


def log(msg):
    print("[bench] " + msg, file=sys.stderr, flush=True)


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args):
    """The oracle, as it stands, timed on the host cores: each step one whole
    oracle run on a smaller graph of the workload's recipe."""
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    from paper_1807_10727_gb300 import synth
    import oracle
    oracle.build()
    full = synth.workload(args.workload)
    sample = REF_SAMPLE if args.workload.startswith("rmat") else args.workload
    g = synth.workload(sample)
    for _ in range(args.warmup):
        oracle.lc_run(g.n, g.src, g.dst, g.seed)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.lc_run(g.n, g.src, g.dst, g.seed)
    dt = (time.perf_counter() - t0) / max(1, args.steps)
    value = g.m / dt
    desc = ("one whole oracle run per step on %s (n = %d, m = %d), a smaller graph of the %s "
            "recipe (n = %d, m = %d)" % (sample, g.n, g.m, args.workload, full.n, full.m))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32/u64",
        "data": "synthetic",
        "config": {"workload": args.workload, "n": full.n, "m": full.m, "sample": sample},
        "cpu_baseline": dict({"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                              "sample": desc}, **host_info()),
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rmat26")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched (config 4) leg")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving (config 5) leg")
    ap.add_argument("--no-configs", action="store_true", help="skip the config 1 and 3 rows")
    ap.add_argument("--param", action="append", default=[], metavar="NAME=VALUE",
                    help="lc_set_param tuning value for the headline context (repeatable)")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the two-hop / tree / union-find-finish leg")
    ap.add_argument("--no-profile", action="store_true",
                    help="skip the profiled pass (per-kernel split and step rooflines)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import torch.distributed as dist

    from paper_1807_10727_gb300 import lc, synth

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    def reduce_max(x):
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    lc.load()
    g = synth.workload(args.workload)
    src = torch.from_numpy(g.src.view(np.int32)).to(dev)
    dst = torch.from_numpy(g.dst.view(np.int32)).to(dev)
    labels = torch.empty(g.n, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    ctx = lc.LocalContraction(g.n, src, dst, seed=g.seed, stream=stream, tuned=not args.param)
    for kv in args.param:
        name, value = kv.split("=", 1)
        ctx.set_param(name, int(value))
    warmup = max(3, args.warmup)
    for _ in range(warmup):
        _, res = ctx.run(labels)
    mp, em = lc.lc_last_stats(ctx.ctx)
    kept, passes = lc.lc_last_dedup(ctx.ctx)

    # headline: library event timing off
    ctx.profile(False)
    clocks = ClockSampler(gpu_id_for(local))
    barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        ctx.run(labels)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    launches = sum(v[0] for v in ctx.kernel_stats().values())  # counted with timing off too
    ms_max = reduce_max(ms)
    log("timed steps done: %.2f ms/step" % ms)

    # profiled pass of the same steps: per-kernel event times
    peak, peak_kind = peaks()
    steps, roof, kernels, prof_ms = None, None, None, None
    if not args.no_profile:
        ctx.profile(True)
        prof_ms = time_steps(ctx, labels, stream, args.steps)
        kstats = ctx.kernel_stats()
        ctx.profile(False)
        steps = step_report(kstats, args.steps, res.n_i, res.m_i, mp, peak, peak_kind)
        roof = roofline_of(steps, peak, peak_kind, args.workload)
        kernels = {k: {"launches_per_step": v[0] / args.steps, "ms_per_step": v[1] / args.steps}
                   for k, v in kstats.items() if v[0]}
        log("roofline: step %s %.3f of peak; parent %.3f relabel %.3f dedup %.3f" % (
            roof["step"], roof["frac"] or 0, steps["parent"]["frac"] or 0,
            steps["relabel"]["frac"] or 0, steps["dedup"]["frac"] or 0))
    pb = path_bytes(res.n_i, res.m_i, mp)
    path_roof = {"bytes_per_step": pb, "achieved": pb / (ms / 1e3) / 1e9, "peak": peak,
                 "unit": "GB/s", "frac": pb / (ms / 1e3) / 1e9 / peak, "peak_kind": peak_kind}
    # the autotuner's parameters against the library's fixed defaults
    tuning = {"applied": dict(ctx.params), "tuned_ms_per_step": ms}
    if ctx.params and not args.param:
        dctx = lc.LocalContraction(g.n, src, dst, seed=g.seed, stream=stream, tuned=False)
        for _ in range(warmup):
            dctx.run(labels)
        tuning["default_ms_per_step"] = time_steps(dctx, labels, stream, args.steps)
        dctx.close()
        log("tuning: %.2f ms tuned vs %.2f ms defaults" % (ms, tuning["default_ms_per_step"]))

    variants = None
    if rank == 0 and not args.no_variants:
        variants = bench_variants(ctx, labels, stream, args.steps, warmup, peak, lc)

    # end to end through the public host-buffer entry point
    e2e = None
    del src, dst
    ctx.close()
    torch.cuda.empty_cache()
    if not args.no_e2e:
        h_src = torch.from_numpy(g.src.view(np.int32)).pin_memory().numpy().view(np.uint32)
        h_dst = torch.from_numpy(g.dst.view(np.int32)).pin_memory().numpy().view(np.uint32)
        h_lab = torch.empty(g.n, dtype=torch.int32).pin_memory().numpy().view(np.uint32)
        hctx = lc.LocalContraction(g.n, m=g.m, seed=g.seed, stream=stream)
        for kv in args.param:
            name, value = kv.split("=", 1)
            hctx.set_param(name, int(value))
        hctx.run_host(h_src, h_dst, h_lab)
        barrier()
        run_ms = []
        t0 = time.perf_counter()
        for _ in range(args.steps):
            t1 = time.perf_counter()
            hctx.run_host(h_src, h_dst, h_lab)
            run_ms.append((time.perf_counter() - t1) * 1e3)
        e2e_s = reduce_max((time.perf_counter() - t0) / args.steps)
        hctx.close()
        # the link alone: the same 8 B/edge host->device copy into a device buffer
        dbuf = torch.empty(2 * g.m, dtype=torch.int32, device=dev)
        hs, hd = torch.from_numpy(h_src.view(np.int32)), torch.from_numpy(h_dst.view(np.int32))
        torch.cuda.synchronize(dev)
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        dbuf[:g.m].copy_(hs, non_blocking=True)
        dbuf[g.m:].copy_(hd, non_blocking=True)
        c1.record(stream)
        torch.cuda.synchronize(dev)
        copy_ms = c0.elapsed_time(c1)
        del dbuf, hs, hd
        del h_src, h_dst, h_lab
        e2e = {"value": world * g.m / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": 8 * g.m, "d2h_bytes_per_step": 4 * g.n,
               "ms_per_step": e2e_s * 1e3, "median_ms": float(np.median(run_ms)),
               "runs_ms": [round(x, 2) for x in run_ms],
               "h2d_copy_ms": copy_ms,
               "h2d_gbs": 8 * g.m / (copy_ms / 1e3) / 1e9}
        log("e2e: %.2f ms/step" % (e2e_s * 1e3))
    del labels
    torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline()
        log("cpu baseline: %.3g edges/s" % cpu["value"])
    configs = None
    if rank == 0 and not args.no_configs:
        configs = {"er16": bench_config("er16", dev, stream, args.steps, warmup, peak, lc, synth,
                                        "er16"),
                   "gridmix": bench_config("gridmix", dev, stream, args.steps, warmup, peak, lc,
                                           synth, "gridmix_small")}
    batched = None
    if not args.no_batch:
        torch.cuda.empty_cache()
        batched = bench_batch(dev, stream, world=world, rank=rank, barrier=barrier,
                              reduce_max=reduce_max)
        log("batched: %.0f graphs/s, %.2f ms tuned vs %.2f ms defaults (one run per graph: %s "
            "graphs/s)" % (batched["batched_graphs_per_s"], batched["batched_ms"],
                           batched["default_params_ms"], batched.get("per_graph_graphs_per_s")))
    serving = None
    if not args.no_serving:
        torch.cuda.empty_cache()

        def gather(obj):
            if world == 1:
                return [obj]
            parts = [None] * world
            dist.all_gather_object(parts, obj)
            return parts

        serving = bench_serving(world=world, rank=rank, barrier=barrier, gather=gather)
        if rank == 0:
            log("serving: saturation %s req/s" % serving["saturation_req_s"])

    if rank == 0:
        line = {
            "metric": METRIC, "value": world * g.m / (ms_max / 1e3), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": warmup,
            "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32/u64", "data": "synthetic",
            "config": {"workload": args.workload, "n": g.n, "m": g.m, "rank_seed": g.seed,
                       "rounds": res.rounds, "parallelism": "replicas" if world > 1 else "single",
                       "params": args.param,
                       "l2": "inputs (8 B/edge) larger than L2; no flush"},
            "roofline": roof, "path_roofline": path_roof, "step_rooflines": steps, "tuning": tuning,
            "profiled_ms_per_step": prof_ms,
            "e2e": e2e, "cpu_baseline": cpu, "gpu_launches": launches, "configs": configs,
            "batched": batched, "serving": serving, "variants": variants,
            "clocks": clk, "kernels": kernels,
            "sizes": [[int(a), int(b), int(c), int(d), int(e)]
                      for a, b, c, d, e in zip(res.n_i, res.m_i, mp, em, kept)],
            "sizes_columns": ["n_i", "m_i", "m'_i", "relabel keys written", "keys deduplicated"],
        }
        print(json.dumps(line, default=_plain))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
