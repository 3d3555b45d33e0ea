"""lc_run_host end to end: the input copy overlapped with phase 0 (chunks of
"host_chunk_edges" edges; each chunk is grouped by vertex-block pair, or
only counted beyond the chunk limits, and gets its share of the
closed-neighbourhood minimum once it has arrived) and the copy-then-run path of the variants that do not overlap.
Labels, R and every per-phase (n_i, m_i) and m'_i bit-exact against the
oracle, from pinned and from pageable host arrays."""
from types import SimpleNamespace

import numpy as np
import pytest

import oracle
from paper_1807_10727_gb300 import lc, synth

pytestmark = pytest.mark.gpu

ORACLE_VARIANT = {lc.LC_VARIANT_FOREST: oracle.FOREST, lc.LC_VARIANT_TWO_HOP: oracle.TWO_HOP,
                  lc.LC_VARIANT_TREE: oracle.TREE}


def pinned(a: np.ndarray) -> np.ndarray:
    import torch
    return torch.from_numpy(a.view(np.int32)).pin_memory().numpy().view(np.uint32)


def check_host(g, params=(), variant=lc.LC_VARIANT_FOREST, finish=0, reps=2, pin=True):
    src, dst = (pinned(g.src), pinned(g.dst)) if pin else (g.src, g.dst)
    ctx = lc.LocalContraction(g.n, m=g.m, seed=g.seed, variant=variant, finish_edges=finish)
    try:
        for k, v in params:
            ctx.set_param(k, v)
        outs = [ctx.run_host(src, dst) for _ in range(reps)]
        mp = ctx.mprime()
    finally:
        ctx.close()
    ref = oracle.lc_run(g.n, g.src, g.dst, g.seed, variant=ORACLE_VARIANT[variant],
                        finish_edges=finish)
    for labels, res in outs:
        assert res.rounds == ref.rounds
        assert list(zip(res.n_i, res.m_i)) == ref.sizes()
        assert np.array_equal(labels, ref.labels)
    assert mp == [int(x) for x in ref.mp_i]


@pytest.mark.parametrize("chunk", [1000, 4099, 1 << 25])
@pytest.mark.parametrize("name", ["er16", "rmat14", "gridmix_small"])
def test_overlapped_chunks(lc_lib, cuda, name, chunk):
    """Chunks smaller and larger than the graph; ragged last chunks and
    chunks that start off a 16-byte boundary."""
    check_host(synth.workload(name), [("host_chunk_edges", chunk)])


@pytest.mark.parametrize("chunk", [1, 2, 3])
def test_overlapped_tiny_chunks(lc_lib, cuda, chunk):
    """Every edge or pair of edges its own chunk, on a small random graph."""
    rng = np.random.default_rng(11)
    n, m = 300, 700
    g = SimpleNamespace(n=n, m=m, seed=5, src=rng.integers(0, n, m, dtype=np.uint32),
                        dst=rng.integers(0, n, m, dtype=np.uint32))
    check_host(g, [("host_chunk_edges", chunk)])


@pytest.mark.parametrize("blocks", [2, 5])
def test_overlapped_chunks_grouped(lc_lib, cuda, blocks):
    """Phase 0 on grouped edges: the bucket counts are summed over the
    chunks before the edges are placed."""
    g = synth.workload("rmat18")
    check_host(g, [("bucket_blocks", blocks), ("host_chunk_edges", 300007)])


@pytest.mark.parametrize("blocks,chunk", [(3, 8192), (32, 220000), (4, (1 << 20) - 3)])
def test_overlapped_grouping_limits(lc_lib, cuda, blocks, chunk):
    """Each chunk is grouped on arrival while there are at most 256 chunks
    and 16384 (bucket, chunk) runs; beyond either limit (512 chunks; 1024
    buckets x 20 chunks) the chunks are only counted and grouped together
    afterwards.  The last case has 5 chunks, the last one of 12 edges."""
    g = synth.workload("rmat18")
    check_host(g, [("bucket_blocks", blocks), ("host_chunk_edges", chunk)])


def test_overlapped_pageable(lc_lib, cuda):
    g = synth.workload("rmat16")
    check_host(g, [("host_chunk_edges", 1 << 16), ("bucket_blocks", 3)], pin=False)


@pytest.mark.parametrize("variant,finish", [(lc.LC_VARIANT_TWO_HOP, 0),
                                            (lc.LC_VARIANT_TREE, 0),
                                            (lc.LC_VARIANT_FOREST, 1 << 40),
                                            (lc.LC_VARIANT_FOREST, 5000)])
def test_host_variants(lc_lib, cuda, variant, finish):
    """Two-hop overlaps like the forest; the tree variant (open minimum) and
    a union-find finish in phase 0 copy first, then run."""
    g = synth.workload("rmat14")
    check_host(g, [("host_chunk_edges", 5000), ("bucket_blocks", 3)], variant, finish)


def test_host_bad_vertex(lc_lib, cuda):
    """An id >= n in a late chunk is reported, and the context stays usable."""
    g = synth.workload("rmat14")
    src = g.src.copy()
    src[-3] = g.n + 5
    ctx = lc.LocalContraction(g.n, m=g.m, seed=g.seed)
    try:
        ctx.set_param("host_chunk_edges", 4096)
        with pytest.raises(lc.LCError) as ei:
            ctx.run_host(src, g.dst)
        assert ei.value.code == lc.LC_ERR_INVALID
        labels, res = ctx.run_host(g.src, g.dst)
    finally:
        ctx.close()
    ref = oracle.lc_run(g.n, g.src, g.dst, g.seed)
    assert res.rounds == ref.rounds and np.array_equal(labels, ref.labels)


def test_host_chunk_param_range(lc_lib, cuda):
    ctx = lc.LocalContraction(100, m=10, seed=1)
    try:
        with pytest.raises(lc.LCError):
            ctx.set_param("host_chunk_edges", 0)
        with pytest.raises(lc.LCError):
            ctx.set_param("host_chunk_edges", 1 << 32)
    finally:
        ctx.close()
