"""Phase 0 on edges grouped by vertex-block pair (the bucketed input that
large graphs use by default), forced on small graphs: labels, phase count,
every per-phase (n_i, m_i) and m'_i bit-exact against the oracle, for every
phase variant, ragged and unaligned inputs, bad ids and batches."""
import numpy as np
import pytest

import oracle
from paper_1807_10727_gb300 import lc, synth

from .test_gpu_parity import dev

pytestmark = pytest.mark.gpu


def run_bucketed(n, s, d, seed, cuda, blocks, **kw):
    ts, td = dev(s, cuda), dev(d, cuda)
    ctx = lc.LocalContraction(n, ts, td, seed=seed, **kw)
    try:
        ctx.set_param("bucket_blocks", blocks)
        labels, res = ctx.run()
        mp = ctx.mprime()
    finally:
        ctx.close()
    return labels.cpu().numpy().view(np.uint32), res, mp


def check(n, s, d, seed, cuda, blocks, variant=oracle.FOREST, finish=0, **kw):
    labels, res, mp = run_bucketed(n, s, d, seed, cuda, blocks, variant=variant,
                                   finish_edges=finish, **kw)
    ref = oracle.lc_run(n, s, d, seed, variant=variant, finish_edges=finish)
    assert res.rounds == ref.rounds
    assert list(zip(res.n_i, res.m_i)) == ref.sizes()
    assert mp == [int(x) for x in ref.mp_i]
    assert np.array_equal(labels, ref.labels)


@pytest.mark.parametrize("blocks", [2, 3, 16, 32])
@pytest.mark.parametrize("name", ["er16", "rmat18", "gridmix_small"])
def test_bucketed_workloads(lc_lib, cuda, name, blocks):
    g = synth.workload(name)
    check(g.n, g.src, g.dst, g.seed, cuda, blocks)


@pytest.mark.parametrize("dedup", [lc.LC_DEDUP_HASH, lc.LC_DEDUP_SORT])
def test_bucketed_dedup_modes(lc_lib, cuda, dedup):
    g = synth.workload("rmat14")
    check(g.n, g.src, g.dst, g.seed, cuda, 7, dedup=dedup)


@pytest.mark.parametrize("variant,finish", [(oracle.TWO_HOP, 0), (oracle.TREE, 0),
                                            (oracle.FOREST, 1 << 40), (oracle.FOREST, 5000)])
def test_bucketed_variants(lc_lib, cuda, variant, finish):
    g = synth.workload("rmat14")
    check(g.n, g.src, g.dst, g.seed, cuda, 5, variant=variant, finish=finish)


def test_bucketed_ragged_and_small(lc_lib, cuda):
    """Edge counts around the 2048-edge tile and the 4-edge vector loads,
    graphs smaller than the block count, one vertex."""
    rng = np.random.default_rng(11)
    for n, m in [(1, 3), (2, 1), (5, 7), (40, 2047), (300, 2048), (300, 2049), (40, 4095),
                 (300, 4096), (300, 4097), (1000, 8191), (70000, 12289), (70000, 4 * 4096 + 3)]:
        s = rng.integers(0, n, m, dtype=np.uint32)
        d = rng.integers(0, n, m, dtype=np.uint32)
        for blocks in (2, 32):
            check(n, s, d, int(rng.integers(0, 1 << 40)), cuda, blocks)


def test_bucketed_unaligned_inputs(lc_lib, cuda):
    """Input pointers one element off the 16-byte boundary take the scalar
    loads."""
    g = synth.workload("rmat14")
    ts, td = dev(np.concatenate([[0], g.src]), cuda), dev(np.concatenate([[0], g.dst]), cuda)
    ctx = lc.LocalContraction(g.n, ts[1:], td[1:], seed=g.seed)
    ctx.set_param("bucket_blocks", 9)
    labels, res = ctx.run()
    ctx.close()
    ref = oracle.lc_run(g.n, g.src, g.dst, g.seed)
    assert list(zip(res.n_i, res.m_i)) == ref.sizes()
    assert np.array_equal(labels.cpu().numpy().view(np.uint32), ref.labels)


def test_bucketed_bad_vertex_rejected(lc_lib, cuda):
    g = synth.workload("rmat14")
    s = g.src.copy()
    s[777] = g.n + 5
    ctx = lc.LocalContraction(g.n, dev(s, cuda), dev(g.dst, cuda), seed=g.seed)
    ctx.set_param("bucket_blocks", 4)
    with pytest.raises(lc.LCError) as ei:
        ctx.run()
    assert ei.value.code == lc.LC_ERR_INVALID
    ctx.close()


def test_bucketed_batch(lc_lib, cuda):
    b = synth.batch(k=48, hi_exp=12.0)
    src, dst = dev(b.src, cuda), dev(b.dst, cuda)
    bl = lc.BatchLocalContraction(b.n, b.eoff, src, dst, b.seeds)
    bl.set_param("bucket_blocks", 6)
    labels, rounds, n_i, m_i = bl.run()
    got = labels.cpu().numpy().view(np.uint32)
    bl.close()
    voff = np.concatenate([[0], np.cumsum(b.n.astype(np.int64))])
    for g in range(b.k):
        lo, hi = int(b.eoff[g]), int(b.eoff[g + 1])
        ref = oracle.lc_run(int(b.n[g]), b.src[lo:hi], b.dst[lo:hi], int(b.seeds[g]))
        R = int(rounds[g])
        assert R == ref.rounds
        assert list(zip(n_i[g, :R].tolist(), m_i[g, :R].tolist())) == ref.sizes()
        assert np.array_equal(got[voff[g]:voff[g + 1]], ref.labels)


def test_bucket_param_rejections(lc_lib, cuda):
    g = synth.workload("rmat14")
    ctx = lc.LocalContraction(g.n, dev(g.src, cuda), dev(g.dst, cuda), seed=g.seed)
    for name, bad in [("bucket_blocks", 33), ("bucket_window_bytes", 1000)]:
        with pytest.raises(lc.LCError):
            ctx.set_param(name, bad)
    ctx.close()


@pytest.mark.parametrize("variant", [oracle.FOREST, oracle.TWO_HOP, oracle.TREE])
def test_bucketed_self_loops(lc_lib, cuda, variant):
    """Phase 0 reads the raw input, self-loops included, through the grouped
    edges: a loop must not count as a neighbour in the open-neighbourhood
    minimum of TreeContraction (nor change anything elsewhere)."""
    rng = np.random.default_rng(21)
    for n, m, loops in [(2000, 6000, 0.3), (50000, 150000, 0.1), (300, 2000, 0.9)]:
        s = rng.integers(0, n, m, dtype=np.uint32)
        d = rng.integers(0, n, m, dtype=np.uint32)
        pick = rng.random(m) < loops
        d[pick] = s[pick]
        for blocks in (2, 7):
            check(n, s, d, int(rng.integers(0, 1 << 40)), cuda, blocks, variant=variant)
