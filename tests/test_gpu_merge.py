"""MergeToLarge (Section 5) on the GPU against the oracle: labels, phase
count, every per-phase (n_i, m_i) and m'_i bit-exact."""
import math

import numpy as np
import pytest

import oracle
from paper_1807_10727_gb300 import lc, synth

pytestmark = pytest.mark.gpu


def dev(a, cuda):
    import torch
    a = np.ascontiguousarray(np.asarray(a, dtype=np.uint32))
    return torch.from_numpy(a.view(np.int32)).to(cuda)


def assert_parity(n, s, d, seed, cuda, alpha, variant=lc.LC_VARIANT_FOREST, finish=0, **kw):
    ts, td = dev(s, cuda), dev(d, cuda)
    ctx = lc.LocalContraction(n, ts, td, seed=seed, variant=variant, finish_edges=finish,
                              merge_alpha=alpha, **kw)
    try:
        labels, res = ctx.run()
        mp = ctx.mprime()
    finally:
        ctx.close()
    ref = oracle.lc_run(n, s, d, seed, variant=variant, finish_edges=finish, merge_alpha=alpha)
    assert res.rounds == ref.rounds
    assert list(zip(res.n_i, res.m_i)) == ref.sizes()
    assert mp == [int(x) for x in ref.mp_i]
    assert np.array_equal(labels.cpu().numpy().view(np.uint32), ref.labels)
    return res, ref


def log_alpha(n, phases=8):
    """alpha_0 = 4 ln n, alpha_{i+1} = alpha_i^2 (the squaring of the
    O(log log n) argument), capped at n."""
    a, out = 4 * math.log(max(n, 2)), []
    for _ in range(phases):
        out.append(int(min(a, n)))
        a = a * a
    return out


@pytest.mark.parametrize("dedup", [lc.LC_DEDUP_HASH, lc.LC_DEDUP_SORT])
@pytest.mark.parametrize("variant", [lc.LC_VARIANT_FOREST, lc.LC_VARIANT_TWO_HOP,
                                     lc.LC_VARIANT_TREE])
@pytest.mark.parametrize("name", ["er16", "rmat14", "rmat18", "gridmix_small"])
def test_merge_workloads(lc_lib, cuda, name, variant, dedup):
    g = synth.workload(name)
    for alpha in (log_alpha(g.n), [4, 4, 4, 4], [2]):
        assert_parity(g.n, g.src, g.dst, g.seed, cuda, alpha, variant, dedup=dedup)


def test_merge_small_random_graphs(lc_lib, cuda):
    rng = np.random.default_rng(53)
    for t in range(150):
        n = int(rng.integers(1, 90))
        m = int(rng.integers(0, 4 * n))
        alpha = [int(rng.integers(0, 7)) for _ in range(int(rng.integers(1, 5)))]
        assert_parity(n, rng.integers(0, n, m), rng.integers(0, n, m), t, cuda, alpha,
                      int(rng.integers(0, 3)), finish=int(rng.integers(0, 2)) * int(rng.integers(1, 50)))


def test_merge_ragged_sizes(lc_lib, cuda):
    rng = np.random.default_rng(59)
    for n, m in [(4097, 4095), (5000, 8191), (70001, 123457), (2049, 20480)]:
        assert_parity(n, rng.integers(0, n, m), rng.integers(0, n, m), 9, cuda, [3, 9, 27])


def test_merge_giant_node(lc_lib, cuda):
    """A star (one node of ~all vertices after phase 0) and a dense random
    graph: large nodes with tens of thousands of members (the radix select
    over many candidates)."""
    k = 60000
    hub = np.zeros(k, dtype=np.uint32)
    leaves = np.arange(1, k + 1, dtype=np.uint32)
    rng = np.random.default_rng(61)
    extra_s = rng.integers(1, k + 1, 30000)
    extra_d = rng.integers(1, k + 1, 30000)
    s = np.concatenate([hub, extra_s])
    d = np.concatenate([leaves, extra_d])
    for alpha in ([1000], [30000], [59000], [2, 2]):
        assert_parity(k + 1, s, d, 3, cuda, alpha)
    n = 20000
    s, d = rng.integers(0, n, 40 * n), rng.integers(0, n, 40 * n)
    assert_parity(n, s, d, 4, cuda, [int(4 * math.log(n))], lc.LC_VARIANT_TWO_HOP)


def test_merge_degenerate_parameters(lc_lib, cuda):
    g = synth.workload("rmat14")
    plain = oracle.lc_run(g.n, g.src, g.dst, g.seed)
    for alpha in ([1] * 10, [g.n + 1] * 10, [0] * 10):
        res, _ = assert_parity(g.n, g.src, g.dst, g.seed, cuda, alpha)
        assert list(zip(res.n_i, res.m_i)) == plain.sizes()


def test_merge_random_graph_phases(lc_lib, cuda):
    """G(n, alpha/n) with alpha = 8 ln n: the two-hop label with MergeToLarge
    (parameter alpha/4) leaves at most n/alpha vertices after one phase
    (Lemma lem:random)."""
    n = 1 << 14
    a = 8 * math.log(n)
    m = int(round(a / n * n * (n - 1) / 2))
    rng = np.random.default_rng(67)
    s, d = rng.integers(0, n, m), rng.integers(0, n, m)
    res, _ = assert_parity(n, s, d, 5, cuda, [int(a / 4)] * 4, lc.LC_VARIANT_TWO_HOP)
    assert res.rounds == 1 or res.n_i[1] <= n / a


def test_merge_rejections(lc_lib, cuda):
    b = synth.batch(k=4, lo_exp=3, hi_exp=5)
    bl = lc.BatchLocalContraction(b.n, b.eoff, dev(b.src, cuda), dev(b.dst, cuda), b.seeds)
    with pytest.raises(lc.LCError) as ei:
        lc.lc_set_merge_to_large(bl.ctx, [4])
    assert ei.value.code == lc.LC_ERR_INVALID
    lc.lc_set_merge_to_large(bl.ctx, [])
    bl.close()
    # switching the step on and off on one context
    g = synth.workload("rmat14")
    ctx = lc.LocalContraction(g.n, dev(g.src, cuda), dev(g.dst, cuda), seed=g.seed)
    for alpha in ([8, 64], [], [3]):
        lc.lc_set_merge_to_large(ctx.ctx, alpha)
        labels, res = ctx.run()
        ref = oracle.lc_run(g.n, g.src, g.dst, g.seed, merge_alpha=alpha)
        assert res.rounds == ref.rounds and list(zip(res.n_i, res.m_i)) == ref.sizes()
        assert np.array_equal(labels.cpu().numpy().view(np.uint32), ref.labels)
    ctx.close()


@pytest.mark.slow
def test_merge_er_few_phases(lc_lib, cuda):
    """ER G(n, alpha/n), alpha = 4 ln n, n = 2^20 (~2.9e7 edges): with
    MergeToLarge (alpha_0 = alpha, squared every phase) the run is bit-exact
    with the oracle and needs no more phases than without it (Section 5's
    O(log log n) bound; log2 log2 n ~ 4.3 here)."""
    n = 1 << 20
    a = 4 * math.log(n)
    m = int(round(a / n * n * (n - 1) / 2))
    rng = np.random.default_rng(71)
    s = rng.integers(0, n, m).astype(np.uint32)
    d = rng.integers(0, n, m).astype(np.uint32)
    res, ref = assert_parity(n, s, d, 11, cuda, log_alpha(n), lc.LC_VARIANT_TWO_HOP)
    plain = oracle.lc_run(n, s, d, 11, variant=oracle.TWO_HOP)
    assert res.rounds <= plain.rounds and res.rounds <= 5
