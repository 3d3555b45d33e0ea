"""GPU path (through the C ABI of liblc.so) against the CPU oracle: labels,
phase count and every per-phase (n_i, m_i) bit-exact, plus the diagnostic m'_i.
"""
from types import SimpleNamespace

import numpy as np
import pytest

import oracle
from paper_1807_10727_gb300 import lc, synth

pytestmark = pytest.mark.gpu


def dev(a, cuda):
    import torch
    a = np.ascontiguousarray(np.asarray(a, dtype=np.uint32))
    return torch.from_numpy(a.view(np.int32)).to(cuda)


def gpu_run(n, s, d, seed, cuda, **kw):
    ts, td = dev(s, cuda), dev(d, cuda)
    ctx = lc.LocalContraction(n, ts, td, seed=seed, **kw)
    try:
        labels, res = ctx.run()
        mp = ctx.mprime()
    finally:
        ctx.close()
    return labels.cpu().numpy().view(np.uint32), res, mp


def assert_parity(n, s, d, seed, cuda, **kw):
    labels, res, mp = gpu_run(n, s, d, seed, cuda, **kw)
    ref = oracle.lc_run(n, s, d, seed)
    assert res.rounds == ref.rounds
    assert [(a, b) for a, b in zip(res.n_i, res.m_i)] == ref.sizes()
    assert mp == [int(x) for x in ref.mp_i]
    assert np.array_equal(labels, ref.labels)
    return res


def test_rank_probe_matches_oracle(lc_lib, cuda):
    for seed, i, v0, count in [(1, 0, 0, 1 << 20), (7, 3, 2**32 - 5000, 4999), (2**63 + 5, 40, 12345, 77)]:
        got = lc.rank_probe(seed, i, v0, count).cpu().numpy().view(np.uint32)
        assert np.array_equal(got, oracle.ranks(seed, i, v0, count))


@pytest.mark.parametrize("dedup", [lc.LC_DEDUP_HASH, lc.LC_DEDUP_SORT])
@pytest.mark.parametrize("name", ["er16", "rmat14", "rmat18", "gridmix_small"])
def test_workload_parity(lc_lib, cuda, name, dedup):
    g = synth.workload(name)
    assert_parity(g.n, g.src, g.dst, g.seed, cuda, dedup=dedup)


def test_er16_several_seeds(lc_lib, cuda):
    g = synth.workload("er16")
    for seed in (0, 2, 3, 2**40 + 1):
        assert_parity(g.n, g.src, g.dst, seed, cuda)


@pytest.mark.parametrize("dedup", [lc.LC_DEDUP_HASH, lc.LC_DEDUP_SORT])
def test_many_small_random_graphs(lc_lib, cuda, dedup):
    rng = np.random.default_rng(17)
    for t in range(120):
        n = int(rng.integers(1, 70))
        m = int(rng.integers(0, 3 * n))
        s = rng.integers(0, n, m)
        d = rng.integers(0, n, m)
        assert_parity(n, s, d, t, cuda, dedup=dedup)


@pytest.mark.parametrize("dedup", [lc.LC_DEDUP_HASH, lc.LC_DEDUP_SORT])
def test_ragged_sizes_across_tiles(lc_lib, cuda, dedup):
    """Sizes around the 4096-key tile, the 2048-key dedup bucket and the
    16-element vector widths."""
    rng = np.random.default_rng(23)
    for n, m in [(4097, 4095), (4096, 4097), (5000, 8191), (70001, 123457), (3, 100003),
                 (2049, 2048), (100, 2049)]:
        s = rng.integers(0, n, m)
        d = rng.integers(0, n, m)
        assert_parity(n, s, d, 9, cuda, dedup=dedup)


# ---------------------------------------------------------- edge cases

def test_no_edges(lc_lib, cuda):
    labels, res, _ = gpu_run(10, [], [], 1, cuda)
    assert res.rounds == 0 and list(labels) == list(range(10))


def test_single_vertex_with_loop(lc_lib, cuda):
    res = assert_parity(1, [0], [0], 1, cuda)
    assert res.rounds == 1


def test_loops_and_duplicates_only(lc_lib, cuda):
    assert_parity(6, [2, 2, 5, 5], [2, 2, 5, 5], 3, cuda)
    assert_parity(6, [1] * 1000 + [4], [3] * 1000 + [4], 3, cuda)


def test_star_hub(lc_lib, cuda):
    k = 20000
    s = np.zeros(k, dtype=np.uint32)
    d = np.arange(1, k + 1, dtype=np.uint32)
    for seed in (1, 2):
        assert_parity(k + 1, s, d, seed, cuda)
        assert_parity(k + 1, d, s, seed, cuda)


def test_long_path_many_phases(lc_lib, cuda):
    n = 100000
    s = np.arange(n - 1, dtype=np.uint32)
    perm = np.random.default_rng(1).permutation(n).astype(np.uint32)
    res = assert_parity(n, perm[s], perm[s + 1], 5, cuda)
    assert res.rounds > 5


def test_complete_graph(lc_lib, cuda):
    n = 300
    iu = np.triu_indices(n, 1)
    res = assert_parity(n, iu[0], iu[1], 4, cuda)
    assert res.rounds == 1


def test_unaligned_input_pointers(lc_lib, cuda):
    """Caller buffers that are offset views (not 16-byte aligned)."""
    g = synth.workload("rmat14")
    ts, td = dev(np.concatenate([[0], g.src]), cuda), dev(np.concatenate([[0, 0], g.dst]), cuda)
    ctx = lc.LocalContraction(g.n, ts[1:], td[2:], seed=g.seed)
    labels, res = ctx.run()
    ctx.close()
    ref = oracle.lc_run(g.n, g.src, g.dst, g.seed)
    assert res.rounds == ref.rounds
    assert np.array_equal(labels.cpu().numpy().view(np.uint32), ref.labels)


def test_vertex_id_out_of_range_is_rejected(lc_lib, cuda):
    ts, td = dev([0, 1, 7], cuda), dev([1, 2, 3], cuda)
    ctx = lc.LocalContraction(5, ts, td, seed=1)
    with pytest.raises(lc.LCError) as ei:
        ctx.run()
    assert ei.value.code == lc.LC_ERR_INVALID
    ctx.close()


def test_context_reuse_is_repeatable(lc_lib, cuda):
    g = synth.workload("rmat16")
    ts, td = dev(g.src, cuda), dev(g.dst, cuda)
    ctx = lc.LocalContraction(g.n, ts, td, seed=g.seed)
    a, ra = ctx.run()
    b, rb = ctx.run()
    ctx.close()
    assert (a == b).all().item() and ra == rb


def test_run_host_matches_oracle(lc_lib, cuda):
    g = synth.workload("gridmix_small")
    ctx = lc.LocalContraction(g.n, m=g.m, seed=g.seed)
    labels, res = ctx.run_host(g.src, g.dst)
    labels2, res2 = ctx.run_host(g.src, g.dst)
    ctx.close()
    ref = oracle.lc_run(g.n, g.src, g.dst, g.seed)
    assert res.rounds == ref.rounds and [(a, b) for a, b in zip(res.n_i, res.m_i)] == ref.sizes()
    assert np.array_equal(labels, ref.labels) and np.array_equal(labels2, ref.labels)


def test_output_cap_too_small(lc_lib, cuda):
    g = synth.workload("rmat14")
    ts, td = dev(g.src, cuda), dev(g.dst, cuda)
    ctx = lc.LocalContraction(g.n, ts, td, seed=g.seed)
    import torch
    labels = torch.empty(g.n, dtype=torch.int32, device=cuda)
    with pytest.raises(lc.LCError) as ei:
        lc.lc_run(ctx.ctx, labels.data_ptr(), cap=1)
    assert ei.value.code == lc.LC_ERR_INVALID
    ctx.close()


@pytest.mark.parametrize("dedup", [lc.LC_DEDUP_HASH, lc.LC_DEDUP_SORT])
def test_relabel_cache_sizes(lc_lib, cuda, dedup):
    """The device-wide relabel cache (phases of >= 2^22 edges) at sizes from
    heavy collisions to none: results never change, and it only drops keys.
    The library defaults (not the tuned table, whose rmat18 entry plans
    phases of fewer than 2^24 edges early, without the cache) keep phase 0's
    2^22 edges on the cached path."""
    g = synth.workload("rmat18")
    ref = oracle.lc_run(g.n, g.src, g.dst, g.seed)
    ts, td = dev(g.src, cuda), dev(g.dst, cuda)
    emitted = {}
    for slots in (0, 1024, 1 << 16, 1 << 20, 1 << 24):
        ctx = lc.LocalContraction(g.n, ts, td, seed=g.seed, dedup=dedup, tuned=False)
        ctx.set_param("relabel_cache_slots", slots)
        labels, res = ctx.run()
        mp, em = lc.lc_last_stats(ctx.ctx)
        kept, passes = lc.lc_last_dedup(ctx.ctx)
        ctx.close()
        assert len(kept) == len(passes) == res.rounds
        assert all(k <= e <= p for k, e, p in zip(kept, em, mp))
        if slots == 0:
            assert kept == em  # nothing drops keys after the relabel
        if dedup == lc.LC_DEDUP_SORT:
            assert not any(passes)
        assert res.rounds == ref.rounds
        assert list(zip(res.n_i, res.m_i)) == ref.sizes()
        assert mp == [int(x) for x in ref.mp_i]
        assert np.array_equal(labels.cpu().numpy().view(np.uint32), ref.labels)
        emitted[slots] = kept[0]
    assert emitted[1 << 20] <= emitted[0]
    for bad in (3, 512, 1 << 27):
        ctx = lc.LocalContraction(g.n, ts, td, seed=g.seed)
        with pytest.raises(lc.LCError):
            ctx.set_param("relabel_cache_slots", bad)
        ctx.close()


@pytest.mark.parametrize("name", ["er16", "rmat18", "gridmix_small"])
def test_multi_part_relabel(lc_lib, cuda, name):
    """Phase 0 relabels in parts when the root array is larger than the part
    size: two parts and three parts (with a middle pass), forced here on
    small graphs."""
    g = synth.workload(name)
    ref = oracle.lc_run(g.n, g.src, g.dst, g.seed)
    ts, td = dev(g.src, cuda), dev(g.dst, cuda)
    for part_bytes in (4 * g.n - 1, (4 * g.n) // 3):
        ctx = lc.LocalContraction(g.n, ts, td, seed=g.seed)
        ctx.set_param("relabel_window_bytes", part_bytes)
        labels, res = ctx.run()
        mp = ctx.mprime()
        ctx.close()
        assert res.rounds == ref.rounds
        assert list(zip(res.n_i, res.m_i)) == ref.sizes()
        assert mp == [int(x) for x in ref.mp_i]
        assert np.array_equal(labels.cpu().numpy().view(np.uint32), ref.labels)


def test_round_cap_and_wait_timeout(lc_lib, cuda):
    """Failure paths that fault nothing: a phase cap below what the graph
    needs gives LC_ERR_NO_CONVERGENCE, and a partition pass whose tile 0 never
    publishes makes the look-back waits behind it run out (short limit) and
    gives LC_ERR_TIMEOUT.  After each, the same context gives the oracle's
    result again."""
    n = 20000
    perm = np.random.default_rng(3).permutation(n).astype(np.uint32)
    s = np.arange(n - 1)
    ps, pd = perm[s], perm[s + 1]
    ref = oracle.lc_run(n, ps, pd, 5)
    assert ref.rounds > 2
    ts, td = dev(ps, cuda), dev(pd, cuda)
    ctx = lc.LocalContraction(n, ts, td, seed=5)
    ctx.set_param("max_rounds", 2)
    with pytest.raises(lc.LCError) as ei:
        ctx.run()
    assert ei.value.code == lc.LC_ERR_NO_CONVERGENCE
    ctx.set_param("max_rounds", 0)
    labels, res = ctx.run()
    assert res.rounds == ref.rounds
    assert np.array_equal(labels.cpu().numpy().view(np.uint32), ref.labels)
    ctx.close()

    g = synth.workload("rmat14")  # 2^18 edges: phase 0 has a partition pass
    ref = oracle.lc_run(g.n, g.src, g.dst, g.seed)
    ctx = lc.LocalContraction(g.n, dev(g.src, cuda), dev(g.dst, cuda), seed=g.seed)
    ctx.set_param("spin_limit", 1 << 12)
    ctx.set_param("inject_lookback_stall", 1)
    with pytest.raises(lc.LCError) as ei:
        ctx.run()
    assert ei.value.code == lc.LC_ERR_TIMEOUT
    labels, res = ctx.run()  # the stall was one shot
    assert res.rounds == ref.rounds and list(zip(res.n_i, res.m_i)) == ref.sizes()
    assert np.array_equal(labels.cpu().numpy().view(np.uint32), ref.labels)
    ctx.close()


@pytest.mark.parametrize("name", ["gridmix_small", "er16", "path"])
def test_root_bitmap_jump(lc_lib, cuda, name):
    """The pointer chase with the root bitmap (forced on small phases; taken
    only by phases whose average degree is below 4) gives the oracle's
    result, also on a long path (deep parent chains)."""
    if name == "path":
        n = 100000
        perm = np.random.default_rng(4).permutation(n).astype(np.uint32)
        g = SimpleNamespace(n=n, src=perm[:-1].copy(), dst=perm[1:].copy(), seed=9)
    else:
        g = synth.workload(name)
    src, dst = dev(g.src, cuda), dev(g.dst, cuda)
    ctx = lc.LocalContraction(g.n, src, dst, seed=g.seed, tuned=False)
    try:
        ctx.set_param("jump_bits_min_vertices", 1)
        labels, res = ctx.run()
        labels2, res2 = ctx.run()
    finally:
        ctx.close()
    ref = oracle.lc_run(g.n, g.src, g.dst, g.seed)
    for lab, r in ((labels, res), (labels2, res2)):
        assert r.rounds == ref.rounds
        assert list(zip(r.n_i, r.m_i)) == ref.sizes()
        assert np.array_equal(lab.cpu().numpy().view(np.uint32), ref.labels)
