"""Deduplication paths of the large phases, forced on small graphs: the
segmented table slices, the bucket partition, the switch from slices to the
partition when the table is too small, and the full-sort fallback after an
overflow (driven by undersizing the distinct-key estimate).  Labels, phase
count, every per-phase (n_i, m_i) and m'_i bit-exact against the oracle."""
import numpy as np
import pytest

import oracle
from paper_1807_10727_gb300 import lc, synth

from .test_gpu_parity import dev

pytestmark = pytest.mark.gpu

WORKLOADS = ["er16", "rmat14", "rmat18", "gridmix_small"]


def run(g, cuda, params, variant=oracle.FOREST):
    ctx = lc.LocalContraction(g.n, dev(g.src, cuda), dev(g.dst, cuda), seed=g.seed,
                              variant=variant)
    try:
        for k, v in params.items():
            ctx.set_param(k, v)
        labels, res = ctx.run()
        mp, em = lc.lc_last_stats(ctx.ctx)
        kept, passes = lc.lc_last_dedup(ctx.ctx)
        fb = lc.lc_dedup_fallbacks(ctx.ctx)
    finally:
        ctx.close()
    assert all(k <= e <= p for k, e, p in zip(kept, em, mp))
    return labels.cpu().numpy().view(np.uint32), res, mp, fb


def check(g, cuda, params, variant=oracle.FOREST):
    labels, res, mp, fb = run(g, cuda, params, variant)
    ref = oracle.lc_run(g.n, g.src, g.dst, g.seed, variant=variant)
    assert res.rounds == ref.rounds
    assert list(zip(res.n_i, res.m_i)) == ref.sizes()
    assert mp == [int(x) for x in ref.mp_i]
    assert np.array_equal(labels, ref.labels)
    return fb


@pytest.mark.parametrize("seg", [1, 0])
@pytest.mark.parametrize("name", WORKLOADS)
def test_late_phases(lc_lib, cuda, name, seg):
    """Every phase of at least 4096 edges plans late, by slices or buckets."""
    g = synth.workload(name)
    assert check(g, cuda, {"late_min_edges": 4096, "seg_dedup": seg}) == 0


@pytest.mark.parametrize("variant", [oracle.TWO_HOP, oracle.TREE])
def test_late_phases_variants(lc_lib, cuda, variant):
    g = synth.workload("rmat14")
    check(g, cuda, {"late_min_edges": 2048}, variant)


@pytest.mark.parametrize("seg", [1, 0])
@pytest.mark.parametrize("name", ["rmat18", "gridmix_small"])
def test_overflow_falls_back_to_sort(lc_lib, cuda, name, seg):
    """An estimate 50 times too small overflows the slices (or the bucket
    sets); those phases are redone by the full sort with the same result."""
    g = synth.workload(name)
    fb = check(g, cuda, {"late_min_edges": 4096, "seg_dedup": seg, "target_permille": 20})
    assert fb > 0


@pytest.mark.parametrize("variant", [oracle.TWO_HOP, oracle.TREE])
def test_overflow_fallback_variants(lc_lib, cuda, variant):
    g = synth.workload("rmat18")
    fb = check(g, cuda, {"late_min_edges": 4096, "target_permille": 10}, variant)
    assert fb > 0


@pytest.mark.parametrize("name", ["rmat18", "gridmix_small"])
def test_table_groups_and_too_small(lc_lib, cuda, name):
    """A capped table takes the slices in several groups (one launch each);
    a table that cannot hold one slice per segment sends the kept keys,
    made contiguous again, to the bucket partition."""
    g = synth.workload(name)
    for cap in (1 << 16, 1 << 14):
        assert check(g, cuda, {"late_min_edges": 4096, "table_slots": cap}) == 0
    assert check(g, cuda, {"late_min_edges": 4096, "target_permille": 1000000,
                           "table_slots": 1 << 15}) == 0


def test_default_large_phase_parity(lc_lib, cuda):
    """R-MAT scale 20 (2^24 edges): phases 0 and 1 take the default
    segmented path without any forced parameter."""
    g = synth.workload("rmat20")
    assert check(g, cuda, {}) == 0


def test_dedup_param_rejections(lc_lib, cuda):
    g = synth.workload("rmat14")
    ctx = lc.LocalContraction(g.n, dev(g.src, cuda), dev(g.dst, cuda), seed=g.seed)
    for name, bad in [("seg_dedup", 2), ("target_permille", 0), ("late_min_edges", 100),
                      ("table_slots", 1000), ("table_slots", 1 << 13)]:
        with pytest.raises(lc.LCError):
            ctx.set_param(name, bad)
    ctx.close()
