"""Sharding of independent graphs across ranks (one GPU per rank).

A single graph's phase loop needs a cross-rank exchange every phase (a
min-reduce for the parents, pointer exchanges, an all-to-all shuffle of the
relabelled edges), so it runs as replicas, one per rank.  Batches of
independent graphs and serving streams shard without any data-path
collective: each rank takes a size-balanced share of the graphs and only the
per-rank results are gathered.  A batch is split up front (balance); a
serving stream is routed request by request (Router), by a rule every rank
evaluates identically on the same arrival sequence, so no rank has to tell
another which requests it took.
"""
from __future__ import annotations

import heapq

import numpy as np


def balance(work, world: int) -> list[list[int]]:
    """Greedy longest-processing-time packing: graphs (by decreasing work) go
    to the least-loaded rank.  Returns, per rank, the sorted graph indices."""
    if world < 1:
        raise ValueError("world must be >= 1")
    work = np.asarray(work, dtype=np.float64)
    heap = [(0.0, r) for r in range(world)]
    out: list[list[int]] = [[] for _ in range(world)]
    for g in np.argsort(-work, kind="stable"):
        load, r = heapq.heappop(heap)
        out[r].append(int(g))
        heapq.heappush(heap, (load + float(work[g]), r))
    return [sorted(x) for x in out]


def graph_work(n, m):
    """Work estimate of a graph for balancing: its edges plus vertices."""
    return np.asarray(m, dtype=np.float64) + np.asarray(n, dtype=np.float64)


def sub_batch(n, eoff, src, dst, seeds, idx):
    """The graphs `idx` of a packed batch, repacked (numpy host arrays)."""
    idx = list(idx)
    n = np.asarray(n)
    eoff = np.asarray(eoff, dtype=np.uint64)
    sn = n[idx].astype(np.uint32)
    sizes = np.array([int(eoff[g + 1] - eoff[g]) for g in idx], dtype=np.uint64)
    se = np.zeros(len(idx) + 1, dtype=np.uint64)
    np.cumsum(sizes, out=se[1:])
    ss = np.concatenate([src[int(eoff[g]):int(eoff[g + 1])] for g in idx]) if idx else \
        np.zeros(0, np.uint32)
    sd = np.concatenate([dst[int(eoff[g]):int(eoff[g + 1])] for g in idx]) if idx else \
        np.zeros(0, np.uint32)
    return sn, se, ss.astype(np.uint32), sd.astype(np.uint32), np.asarray(seeds)[idx]


class Router:
    """Online form of `balance` for a request stream: request k goes to the
    rank with the least work routed so far (ties to the lowest rank).  Every
    rank runs the same router over the same sequence of request sizes and
    serves only the requests routed to itself."""

    def __init__(self, world: int):
        if world < 1:
            raise ValueError("world must be >= 1")
        self.load = [0.0] * world

    def route(self, work: float) -> int:
        r = min(range(len(self.load)), key=lambda q: (self.load[q], q))
        self.load[r] += float(work)
        return r


def route_stream(works, world: int) -> list[int]:
    """Rank of every request of a stream (Router applied in arrival order)."""
    rt = Router(world)
    return [rt.route(w) for w in works]
