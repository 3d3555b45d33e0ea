"""The other phase variants on the GPU against the oracle: the published
two-hop LocalContraction label, TreeContraction, and the union-find finish of
small graphs (Section 3 and Section 6, Empirical study).  Labels, phase count, every per-phase
(n_i, m_i) and m'_i bit-exact, single graphs and batches."""
import numpy as np
import pytest

import oracle
from paper_1807_10727_gb300 import lc, synth

pytestmark = pytest.mark.gpu

VARIANTS = [lc.LC_VARIANT_TWO_HOP, lc.LC_VARIANT_TREE]
ORACLE_VARIANT = {lc.LC_VARIANT_FOREST: oracle.FOREST, lc.LC_VARIANT_TWO_HOP: oracle.TWO_HOP,
                  lc.LC_VARIANT_TREE: oracle.TREE}


def dev(a, cuda):
    import torch
    a = np.ascontiguousarray(np.asarray(a, dtype=np.uint32))
    return torch.from_numpy(a.view(np.int32)).to(cuda)


def assert_parity(n, s, d, seed, cuda, variant, finish=0, **kw):
    ts, td = dev(s, cuda), dev(d, cuda)
    ctx = lc.LocalContraction(n, ts, td, seed=seed, variant=variant, finish_edges=finish, **kw)
    try:
        labels, res = ctx.run()
        mp = ctx.mprime()
    finally:
        ctx.close()
    ref = oracle.lc_run(n, s, d, seed, variant=ORACLE_VARIANT[variant], finish_edges=finish)
    assert res.rounds == ref.rounds
    assert list(zip(res.n_i, res.m_i)) == ref.sizes()
    assert mp == [int(x) for x in ref.mp_i]
    assert np.array_equal(labels.cpu().numpy().view(np.uint32), ref.labels)
    return res


@pytest.mark.parametrize("dedup", [lc.LC_DEDUP_HASH, lc.LC_DEDUP_SORT])
@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("name", ["er16", "rmat14", "rmat18", "gridmix_small"])
def test_variant_workloads(lc_lib, cuda, name, variant, dedup):
    g = synth.workload(name)
    assert_parity(g.n, g.src, g.dst, g.seed, cuda, variant, dedup=dedup)


@pytest.mark.parametrize("variant", VARIANTS)
def test_variant_small_random_graphs(lc_lib, cuda, variant):
    rng = np.random.default_rng(29)
    for t in range(100):
        n = int(rng.integers(1, 60))
        m = int(rng.integers(0, 3 * n))
        assert_parity(n, rng.integers(0, n, m), rng.integers(0, n, m), t, cuda, variant)


@pytest.mark.parametrize("variant", VARIANTS)
def test_variant_ragged_sizes(lc_lib, cuda, variant):
    rng = np.random.default_rng(31)
    for n, m in [(4097, 4095), (5000, 8191), (70001, 123457), (3, 100003), (2049, 2048)]:
        assert_parity(n, rng.integers(0, n, m), rng.integers(0, n, m), 9, cuda, variant)


@pytest.mark.parametrize("variant", VARIANTS)
def test_variant_degenerate_graphs(lc_lib, cuda, variant):
    # no edges, a lone loop, loops and duplicates only
    ts, td = dev([], cuda), dev([], cuda)
    ctx = lc.LocalContraction(7, ts, td, seed=1, variant=variant)
    labels, res = ctx.run()
    ctx.close()
    assert res.rounds == 0 and labels.cpu().tolist() == list(range(7))
    assert_parity(1, [0], [0], 1, cuda, variant)
    assert_parity(6, [2, 2, 5, 5], [2, 2, 5, 5], 3, cuda, variant)
    assert_parity(6, [1] * 500 + [4], [3] * 500 + [4], 3, cuda, variant)


@pytest.mark.parametrize("variant", VARIANTS)
def test_variant_path_star_clique(lc_lib, cuda, variant):
    n = 50000
    perm = np.random.default_rng(2).permutation(n).astype(np.uint32)
    s = np.arange(n - 1)
    assert_parity(n, perm[s], perm[s + 1], 5, cuda, variant)
    k = 20000
    hub = np.zeros(k, dtype=np.uint32)
    leaves = np.arange(1, k + 1, dtype=np.uint32)
    assert_parity(k + 1, hub, leaves, 1, cuda, variant)
    assert_parity(k + 1, leaves, hub, 2, cuda, variant)
    iu = np.triu_indices(200, 1)
    assert_parity(200, iu[0], iu[1], 4, cuda, variant)


@pytest.mark.parametrize("variant", [lc.LC_VARIANT_FOREST] + VARIANTS)
@pytest.mark.parametrize("finish", [1, 5000, 200000, 1 << 40])
def test_union_find_finish(lc_lib, cuda, variant, finish):
    """Thresholds that trigger in a late phase, a middle phase and phase 0."""
    g = synth.workload("rmat14")
    res = assert_parity(g.n, g.src, g.dst, g.seed, cuda, variant, finish=finish)
    if finish >= g.m:
        assert res.rounds == 1


def test_union_find_finish_random(lc_lib, cuda):
    rng = np.random.default_rng(37)
    for t in range(60):
        n = int(rng.integers(1, 80))
        m = int(rng.integers(0, 3 * n))
        fin = int(rng.integers(1, 3 * n + 2))
        assert_parity(n, rng.integers(0, n, m), rng.integers(0, n, m), t, cuda,
                      int(rng.integers(0, 3)), finish=fin)


def test_finish_path_long_chain(lc_lib, cuda):
    """A long path finished once few edges are left; ids reversed so that
    union-find hooks go against the id order."""
    n = 30000
    s = np.arange(n - 1, dtype=np.uint32)[::-1].copy()
    assert_parity(n, s + 1, s, 3, cuda, lc.LC_VARIANT_FOREST, finish=3000)
    assert_parity(n, s + 1, s, 3, cuda, lc.LC_VARIANT_FOREST, finish=n)


@pytest.mark.parametrize("variant", VARIANTS)
def test_variant_batch(lc_lib, cuda, variant):
    b = synth.batch(k=64, lo_exp=3, hi_exp=10)
    ts, td = dev(b.src, cuda), dev(b.dst, cuda)
    bl = lc.BatchLocalContraction(b.n, b.eoff, ts, td, b.seeds, variant=variant)
    labels, rounds, n_i, m_i = bl.run()
    bl.close()
    labels = labels.cpu().numpy().view(np.uint32)
    voff = np.zeros(len(b.n) + 1, dtype=np.int64)
    np.cumsum(np.asarray(b.n, dtype=np.int64), out=voff[1:])
    for g in range(len(b.n)):
        s, d = b.src[b.eoff[g]:b.eoff[g + 1]], b.dst[b.eoff[g]:b.eoff[g + 1]]
        ref = oracle.lc_run(int(b.n[g]), s, d, int(b.seeds[g]), variant=ORACLE_VARIANT[variant])
        R = int(rounds[g])
        assert R == ref.rounds, g
        assert list(zip(n_i[g, :R].tolist(), m_i[g, :R].tolist())) == ref.sizes(), g
        assert np.array_equal(labels[voff[g]:voff[g + 1]], ref.labels), g


def test_configure_rejections(lc_lib, cuda):
    ts, td = dev([0, 1], cuda), dev([1, 2], cuda)
    ctx = lc.LocalContraction(3, ts, td, seed=1)
    with pytest.raises(lc.LCError) as ei:
        lc.lc_configure(ctx.ctx, 3, 0)
    assert ei.value.code == lc.LC_ERR_INVALID
    # switching variants on one context keeps giving the oracle's results
    for variant in (lc.LC_VARIANT_TWO_HOP, lc.LC_VARIANT_TREE, lc.LC_VARIANT_FOREST):
        lc.lc_configure(ctx.ctx, variant, 0)
        labels, res = ctx.run()
        ref = oracle.lc_run(3, [0, 1], [1, 2], 1, variant=ORACLE_VARIANT[variant])
        assert res.rounds == ref.rounds
        assert np.array_equal(labels.cpu().numpy().view(np.uint32), ref.labels)
    ctx.close()
    b = synth.batch(k=4, lo_exp=3, hi_exp=5)
    bl = lc.BatchLocalContraction(b.n, b.eoff, dev(b.src, cuda), dev(b.dst, cuda), b.seeds)
    with pytest.raises(lc.LCError) as ei:
        lc.lc_configure(bl.ctx, lc.LC_VARIANT_FOREST, 10)
    assert ei.value.code == lc.LC_ERR_INVALID
    bl.close()


def test_variant_bad_vertex_rejected(lc_lib, cuda):
    for variant in VARIANTS:
        for finish in (0, 100):
            ts, td = dev([0, 1, 9], cuda), dev([1, 2, 3], cuda)
            ctx = lc.LocalContraction(5, ts, td, seed=1, variant=variant, finish_edges=finish)
            with pytest.raises(lc.LCError) as ei:
                ctx.run()
            assert ei.value.code == lc.LC_ERR_INVALID
            ctx.close()
