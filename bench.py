"""Benchmark: input edges/s of the LocalContraction connected-components path
on one GB300 (R-MAT scale 26, 2^30 edges, permuted ids, rank seed 7).

One step = one lc_run over the whole phase loop (rank, closed-neighbourhood
minimum, pointer jumping, relabel/sort/dedup/compact every phase, then label
composition) with the input already resident in HBM.  The input (8 GiB) is
far larger than the 129 MB L2, so no flush is needed between steps.

Extra keys on the JSON line:
  roofline      dominant kernel: algorithmic bytes / its CUDA-event-timed
                device time, against the measured HBM copy peak.
  path_roofline whole step: algorithmic bytes of all phases / step time.
  e2e           the same metric through lc_run_host (pinned host buffers,
                host->device copy of the edges and device->host copy of the
                labels inside the timed region).
  cpu_baseline  the CPU oracle (single thread) on a bounded prefix sample.

--impl reference times the CPU oracle on the same bounded sample per step
(the reference arm is the oracle written from the paper).
Multi-GPU (--gpus N under torchrun): the single-graph path does not shard, so
every rank runs its own replica (weak scaling); value = all ranks' edges /
the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

REPO = os.path.dirname(os.path.abspath(__file__))
if REPO not in sys.path:
    sys.path.insert(0, REPO)

METRIC = "input edges/sec to final labels (1 GB300), HBM roofline %"
# DRAM bytes / algorithmic bytes per launch of the phase-0 launches, from the
# committed full-size ncu capture (profiles/traffic_rmat26.md); valid while
# the kernels are unchanged and only for the R-MAT 26 workload.
TRAFFIC_RATIO = {"relabel_soa": 2.435, "relabel_split": 2.369, "edge_min_soa": 1.742,
                 "filter_hll": 1.342}
UNIT = "edges/s"
CPU_SAMPLE_EDGES = 1 << 24


def peaks():
    path = os.path.join(REPO, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# Algorithmic bytes of each kernel over one run, from the phase sizes (n_i
# vertices, m_i edges, mp_i non-loop keys after relabel, em_i keys the relabel
# wrote, m_{i+1} distinct edges): one read of every input a launch must
# consume and one write of every output it must produce.  Random-gather
# sector amplification is not algorithmic and is not counted; a phase-0
# minimum window pass or a relabel half-pass reads all edges, so each such
# launch counts that read.
def algorithmic_bytes(n_i, m_i, mp_i, em_i, kept_i, passes_i, window_passes, relabel_split):
    per = {}

    def add(k, b):
        per[k] = per.get(k, 0) + b

    R = len(n_i)
    for i in range(R):
        n, m, em = n_i[i], m_i[i], em_i[i]
        m_next = m_i[i + 1] if i + 1 < R else 0
        add("init_keys", 8 * n + (4 * n if i == 0 else 0))
        if i == 0:
            add("edge_min_soa", window_passes * 8 * m + 8 * n)
            if relabel_split:
                add("relabel_split", 8 * m + 8 * m + 4 * n)
                add("relabel_soa", 8 * m + 8 * em + 4 * n)
            else:
                add("relabel_soa", 8 * m + 8 * em + 4 * n)
        else:
            add("edge_min_packed", 8 * m + 8 * n)
            add("relabel_packed", 8 * m + 8 * em + 4 * n)
        add("jump", 8 * n + 4 * n + 4 * n)
        kept = kept_i[i]
        add("sort_pass", 16 * kept * passes_i[i])
        if kept != em or m >= LATE_PLAN_EDGES:
            # phases that size their buckets after the relabel: the filter
            # pass reads the written keys and writes the kept ones, the
            # histogram pass reads the kept keys
            add("filter_hll", 8 * em + 8 * kept)
            add("sort_hist", 8 * kept)
        add("bucket_dedup", 8 * kept + 8 * m_next + 2 * n)
        add("rename", 16 * m_next + 4 * n)
        add("scan_flags", n + 4 * n + 8 * (m_next and n))
        add("propagate", 4 * n + 4 * n + 4 * n)
    return per


LATE_PLAN_EDGES = 1 << 22  # phases of at least this many edges plan their dedup after relabel


def path_bytes(n_i, m_i, mp_i):
    """Whole-path algorithmic bytes: edges read by the minimum and relabel
    steps, keys written, one read+write of the keys for deduplication, the
    renamed edges written, and the per-vertex arrays of every phase."""
    total = 0
    R = len(n_i)
    for i in range(R):
        n, m, mp = n_i[i], m_i[i], mp_i[i]
        m_next = m_i[i + 1] if i + 1 < R else 0
        total += 8 * m + 8 * m + 8 * mp + 16 * mp + 8 * m_next
        total += n * (8 + 4 + 8 + 4 + 4)
    total += sum(8 * n for n in n_i) + 8 * (n_i[0] if n_i else 0)
    return total


def variant_path_bytes(variant, finish, n_i, m_i, mp_i):
    """path_bytes plus what a variant adds: the two-hop label reads every edge
    once more and writes and copies a second n-word key array per phase; the
    union-find finish phase reads its edges once for the unions."""
    total = path_bytes(n_i, m_i, mp_i)
    for i, (n, m) in enumerate(zip(n_i, m_i)):
        if finish and m <= finish:
            total += 8 * m + 8 * n
        elif variant == 1:
            total += 8 * m + 8 * n + 16 * n + 8 * n
    return total


def bench_variants(ctx, labels, stream, steps, warmup, peak, lc):
    """The other phase variants and the union-find finish on the same graph
    and context as the headline: edges/s, phases and the path roofline."""
    import torch
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
        ctx.profile(True)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            ctx.run(labels)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        ks = ctx.kernel_stats()
        ctx.profile(False)
        pb = variant_path_bytes(variant, finish, res.n_i, res.m_i, mp)
        top = sorted(((v[1] / steps, k) for k, v in ks.items() if v[0]), reverse=True)[:4]
        out[name] = {"value": res.m_i[0] / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
                     "rounds": res.rounds, "sizes": [[int(a), int(b)] for a, b in
                                                     zip(res.n_i, res.m_i)],
                     "path_frac": pb / (ms / 1e3) / 1e9 / peak,
                     "gpu_launches_per_step": sum(v[0] for v in ks.values()) / steps,
                     "top_kernels_ms": {k: round(t, 3) for t, k in top}}
        if merge:
            out[name]["merge_alpha"] = list(merge[:res.rounds])
        log(f"variant {name}: {ms:.2f} ms/step, {res.rounds} phases")
    lc.lc_configure(ctx.ctx, lc.LC_VARIANT_FOREST, 0)
    lc.lc_set_merge_to_large(ctx.ctx, [])
    return out


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


def cpu_baseline(g, sample_edges=CPU_SAMPLE_EDGES):
    """The oracle (single-threaded C++) on the first `sample_edges` edges of
    the same edge list, over all n vertices."""
    import oracle
    k = min(sample_edges, g.m)
    s, d = np.ascontiguousarray(g.src[:k]), np.ascontiguousarray(g.dst[:k])
    t0 = time.perf_counter()
    oracle.lc_run(g.n, s, d, g.seed)
    dt = time.perf_counter() - t0
    return {"value": k / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "first %d of %d edges of the same graph (all %d vertices), one oracle run, %.1f s"
                      % (k, g.m, g.n, dt)}


def bench_batch(dev, stream, steps=5, k=4096, world=1, rank=0, barrier=None, reduce_max=None):
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
    bl = lc.BatchLocalContraction(b.n, b.eoff, src, dst, b.seeds, stream=stream)
    for _ in range(2):
        bl.run(labels)
    torch.cuda.synchronize(dev)
    if barrier:
        barrier()
    t0 = time.perf_counter()
    for _ in range(steps):
        _, rounds, _, _ = bl.run(labels)
    torch.cuda.synchronize(dev)
    batched_s = (time.perf_counter() - t0) / steps
    if reduce_max:
        batched_s = reduce_max(batched_s)
    bl.close()
    if world > 1:
        return {"workload": "4096 graphs, n log-uniform [2^6, 2^16], ER deg 4 / R-MAT deg 16",
                "graphs": k, "ranks": world, "graphs_this_rank": k_mine,
                "batched_graphs_per_s": k / batched_s, "batched_ms": batched_s * 1e3}
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
    return {"workload": "4096 graphs, n log-uniform [2^6, 2^16], ER deg 4 / R-MAT deg 16",
            "graphs": k, "vertices": total, "edges": int(b.eoff[-1]),
            "max_rounds": int(rounds.max()),
            "batched_graphs_per_s": k / batched_s, "batched_ms": batched_s * 1e3,
            "per_graph_graphs_per_s": k / serial_s, "per_graph_ms_total": serial_s * 1e3,
            "per_graph_latency_ms_p50": float(np.percentile(lat, 50) * 1e3),
            "per_graph_latency_ms_p99": float(np.percentile(lat, 99) * 1e3),
            "speedup": serial_s / batched_s}


def bench_serving(rates=(300.0, 1000.0, 3000.0), count=160, slots=32):
    """Config 5: Poisson arrivals of CC requests (ER / R-MAT / permuted grid,
    n log-uniform in [2^10, 2^22], average degree 4-32), served by the
    continuous-batching loop vs the serial plain path (one request at a time,
    lc_run_host, in arrival order).  Latency = arrival to labels on the host.
    The same requests are replayed at every rate."""
    import threading

    from paper_1807_10727_gb300 import lc, synth
    reqs = synth.serving_stream(1000.0, count)
    log("serving: %d requests generated" % count)
    base = np.array([r.arrival_s for r in reqs])
    edges = int(sum(r.graph.m for r in reqs))

    def summarize(lat, t_first, t_last):
        lat = np.asarray(lat)
        return {"graphs_per_s": len(lat) / (t_last - t_first),
                "latency_ms_p50": float(np.percentile(lat, 50) * 1e3),
                "latency_ms_p99": float(np.percentile(lat, 99) * 1e3)}

    out = {"workload": "%d requests, ER/R-MAT/grid, n in [2^10, 2^22], degree 4-32, %d edges"
                       % (count, edges), "slots": slots, "rates": []}
    srv = lc.Server(slots=slots)
    warm = [srv.submit(r.graph.n, r.graph.src, r.graph.dst, r.graph.seed) for r in reqs[:8]]
    for j in warm:
        srv.wait(j)
    for rate in rates:
        arr = base * (1000.0 / rate)
        ids = [None] * count
        ready = threading.Semaphore(0)
        t0 = time.perf_counter() + 0.05

        def producer():
            for k, r in enumerate(reqs):
                d = t0 + arr[k] - time.perf_counter()
                if d > 0:
                    time.sleep(d)
                ids[k] = srv.submit(r.graph.n, r.graph.src, r.graph.dst, r.graph.seed)
                ready.release()

        th = threading.Thread(target=producer)
        th.start()
        lat, t_last = [], t0
        for k in range(count):
            if not ready.acquire(timeout=120):
                raise RuntimeError("serving: request %d was not submitted within 120 s" % k)
            _, _, l = srv.wait(ids[k], timeout_s=120.0)
            lat.append(l)
            t_last = max(t_last, t0 + arr[k] + l)
        th.join()
        row = summarize(lat, t0, t_last)
        row["rate_req_s"] = rate
        out["rates"].append(row)
        log("serving: rate %g done" % rate)
    out["peak_active"] = srv.stats()["peak_active"]
    srv.close()
    # serial plain path at the middle rate
    rate = rates[len(rates) // 2]
    arr = base * (1000.0 / rate)
    lat = []
    t0 = time.perf_counter() + 0.05
    for k, r in enumerate(reqs):
        d = t0 + arr[k] - time.perf_counter()
        if d > 0:
            time.sleep(d)
        c = lc.LocalContraction(r.graph.n, m=r.graph.m, seed=r.graph.seed)
        c.run_host(r.graph.src, r.graph.dst)
        c.close()
        lat.append(time.perf_counter() - (t0 + arr[k]))
    row = summarize(lat, t0, time.perf_counter())
    row["rate_req_s"] = rate
    out["serial"] = row
    return out


def log(msg):
    print("[bench] " + msg, file=sys.stderr, flush=True)


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args):
    """The oracle, as it stands, timed on the host cores on a bounded sample."""
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    from paper_1807_10727_gb300 import synth
    import oracle
    oracle.build()
    g = synth.workload(args.workload)
    k = min(CPU_SAMPLE_EDGES, g.m)
    s, d = np.ascontiguousarray(g.src[:k]), np.ascontiguousarray(g.dst[:k])
    for _ in range(args.warmup):
        oracle.lc_run(g.n, s, d, g.seed)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.lc_run(g.n, s, d, g.seed)
    dt = (time.perf_counter() - t0) / max(1, args.steps)
    value = k / dt
    sample = "first %d of %d edges of %s (all %d vertices) per step" % (k, g.m, args.workload, g.n)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32/u64",
        "data": "synthetic",
        "config": {"workload": args.workload, "n": g.n, "m": g.m, "sample_edges": k},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": sample},
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
    ap.add_argument("--param", action="append", default=[], metavar="NAME=VALUE",
                    help="lc_set_param tuning value for the headline context (repeatable)")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the two-hop / tree / union-find-finish leg")
    ap.add_argument("--no-profile", action="store_true",
                    help="skip the per-kernel event timing (roofline) of the timed steps")
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

    lc.load()
    g = synth.workload(args.workload)
    src = torch.from_numpy(g.src.view(np.int32)).to(dev)
    dst = torch.from_numpy(g.dst.view(np.int32)).to(dev)
    labels = torch.empty(g.n, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    ctx = lc.LocalContraction(g.n, src, dst, seed=g.seed, stream=stream)
    for kv in args.param:
        name, value = kv.split("=", 1)
        ctx.set_param(name, int(value))

    for _ in range(max(3, args.warmup)):
        _, res = ctx.run(labels)
    mp, em = lc.lc_last_stats(ctx.ctx)
    kept, passes = lc.lc_last_dedup(ctx.ctx)

    clocks = ClockSampler(gpu_id_for(local))
    ctx.profile(not args.no_profile)
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
    log("timed steps done")
    ms = e0.elapsed_time(e1) / args.steps
    kstats = ctx.kernel_stats()
    ctx.profile(False)
    launches = sum(v[0] for v in kstats.values())

    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())

    # dominant kernel and its roofline
    peak, peak_kind = peaks()
    wpass = max(1, -(-8 * g.n // (192 << 20)))
    split = g.n < (1 << 31) and 4 * g.n > (160 << 20)
    alg = algorithmic_bytes(res.n_i, res.m_i, mp, em, kept, passes, wpass, split)
    top = max(kstats.items(), key=lambda kv: kv[1][1])
    top_name, (top_launches, top_ms) = top
    roof = None
    if top_ms > 0:
        achieved = alg.get(top_name, 0) * args.steps / (top_ms / 1e3) / 1e9
        per_launch = alg.get(top_name, 0) * args.steps / max(1, top_launches)
        ratio = TRAFFIC_RATIO.get(top_name) if args.workload == "rmat26" and not args.param else None
        roof = {"bound": "hbm", "kernel": top_name, "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind,
                "traffic": ratio * per_launch if ratio else None,
                "algorithmic_bytes_per_launch": per_launch,
                "launches_per_step": top_launches / args.steps,
                "share_of_step": top_ms / args.steps / ms}
    pb = path_bytes(res.n_i, res.m_i, mp)
    path_roof = {"bytes_per_step": pb, "achieved": pb / (ms / 1e3) / 1e9, "peak": peak,
                 "unit": "GB/s", "frac": pb / (ms / 1e3) / 1e9 / peak}
    kernels = {k: {"launches_per_step": v[0] / args.steps, "ms_per_step": v[1] / args.steps}
               for k, v in kstats.items() if v[0]}

    variants = None
    if rank == 0 and not args.no_variants:
        variants = bench_variants(ctx, labels, stream, args.steps, max(3, args.warmup), peak, lc)

    # end to end through the public host-buffer entry point
    e2e = None
    if not args.no_e2e:
        del src, dst
        ctx.close()
        torch.cuda.empty_cache()
        h_src = torch.from_numpy(g.src.view(np.int32)).pin_memory().numpy().view(np.uint32)
        h_dst = torch.from_numpy(g.dst.view(np.int32)).pin_memory().numpy().view(np.uint32)
        h_lab = torch.empty(g.n, dtype=torch.int32).pin_memory().numpy().view(np.uint32)
        hctx = lc.LocalContraction(g.n, m=g.m, seed=g.seed, stream=stream)
        hctx.run_host(h_src, h_dst, h_lab)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            hctx.run_host(h_src, h_dst, h_lab)
        e2e_s = (time.perf_counter() - t0) / args.steps
        hctx.close()
        te = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(te, op=dist.ReduceOp.MAX)
        e2e = {"value": world * g.m / float(te.item()), "unit": UNIT,
               "h2d_bytes_per_step": 8 * g.m, "d2h_bytes_per_step": 4 * g.n,
               "ms_per_step": float(te.item()) * 1e3}
    else:
        ctx.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(g)
    batched = None
    if not args.no_batch:
        torch.cuda.empty_cache()

        def reduce_max(x):
            t = torch.tensor([x], dtype=torch.float64, device=dev)
            if world > 1:
                dist.all_reduce(t, op=dist.ReduceOp.MAX)
            return float(t.item())

        batched = bench_batch(dev, stream, world=world, rank=rank, barrier=barrier,
                              reduce_max=reduce_max)
        log("batched leg done")
    serving = None
    if rank == 0 and not args.no_serving:
        torch.cuda.empty_cache()
        serving = bench_serving()
        log("serving leg done")

    if rank == 0:
        line = {
            "metric": METRIC, "value": world * g.m / (ms_max / 1e3), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup),
            "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32/u64", "data": "synthetic",
            "config": {"workload": args.workload, "n": g.n, "m": g.m, "rank_seed": g.seed,
                       "rounds": res.rounds, "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs (8 B/edge) larger than L2; no flush"},
            "roofline": roof, "path_roofline": path_roof,
            "e2e": e2e, "cpu_baseline": cpu, "gpu_launches": launches, "batched": batched,
            "serving": serving, "variants": variants,
            "clocks": clk, "kernels": kernels,
            "sizes": [[int(a), int(b), int(c), int(d), int(e)]
                      for a, b, c, d, e in zip(res.n_i, res.m_i, mp, em, kept)],
            "sizes_columns": ["n_i", "m_i", "m'_i", "relabel keys written", "keys deduplicated"],
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
