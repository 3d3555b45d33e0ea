"""Allocation-failure paths, driven on the host by the library's one-shot
hook (lc_fail_alloc) rather than by exhausting the GPU: the failing call
returns LC_ERR_OOM, releases what it had allocated (free device memory is back
where it was), and the library keeps giving the oracle's results."""
import numpy as np
import pytest

import oracle
from paper_1807_10727_gb300 import lc, synth

from .test_gpu_parity import dev

pytestmark = pytest.mark.gpu


def free_bytes():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def parity(g, labels, res):
    ref = oracle.lc_run(g.n, g.src, g.dst, g.seed)
    assert res.rounds == ref.rounds and list(zip(res.n_i, res.m_i)) == ref.sizes()
    assert np.array_equal(labels.cpu().numpy().view(np.uint32), ref.labels)


def test_create_fails_at_every_allocation(lc_lib, cuda):
    """R-MAT scale 18 (2^22 edges): lc_create allocates the large-phase
    buffers too.  Failing each of its allocations in turn gives LC_ERR_OOM
    with nothing leaked, until the hook lands past the last one."""
    g = synth.workload("rmat18")
    ts, td = dev(g.src, cuda), dev(g.dst, cuda)
    warm = lc.LocalContraction(g.n, ts, td, seed=g.seed)  # loads the library's device code
    warm.run()
    warm.close()
    base = free_bytes()
    failed = 0
    for k in range(1, 64):
        lc.fail_alloc(k)
        try:
            ctx = lc.LocalContraction(g.n, ts, td, seed=g.seed)
        except lc.LCError as e:
            assert e.code == lc.LC_ERR_OOM
            failed += 1
            assert free_bytes() == base, k
            continue
        lc.fail_alloc(0)
        ctx.close()
        break
    lc.fail_alloc(0)
    assert failed >= 10  # every allocation of lc_create was reached
    assert free_bytes() == base
    ctx = lc.LocalContraction(g.n, ts, td, seed=g.seed)
    labels, res = ctx.run()
    ctx.close()
    parity(g, labels, res)


def test_configure_and_param_allocation_failures(lc_lib, cuda):
    """lc_configure(two-hop) and lc_set_param("late_min_edges") allocate;
    when that fails they return LC_ERR_OOM and the context runs as before."""
    g = synth.workload("rmat14")
    ctx = lc.LocalContraction(g.n, dev(g.src, cuda), dev(g.dst, cuda), seed=g.seed)
    lc.fail_alloc(1)
    with pytest.raises(lc.LCError) as ei:
        lc.lc_configure(ctx.ctx, lc.LC_VARIANT_TWO_HOP, 0)
    assert ei.value.code == lc.LC_ERR_OOM
    labels, res = ctx.run()
    parity(g, labels, res)
    for k in (1, 2, 3):
        lc.fail_alloc(k)
        with pytest.raises(lc.LCError) as ei:
            ctx.set_param("late_min_edges", 4096)
        assert ei.value.code == lc.LC_ERR_OOM
    lc.fail_alloc(0)
    labels, res = ctx.run()
    parity(g, labels, res)
    lc.lc_configure(ctx.ctx, lc.LC_VARIANT_TWO_HOP, 0)
    ctx.set_param("late_min_edges", 4096)
    labels, res = ctx.run()
    ref = oracle.lc_run(g.n, g.src, g.dst, g.seed, variant=oracle.TWO_HOP)
    assert list(zip(res.n_i, res.m_i)) == ref.sizes()
    assert np.array_equal(labels.cpu().numpy().view(np.uint32), ref.labels)
    ctx.close()


def test_arena_growth_failure_during_a_run(lc_lib, cuda):
    """A path with a MergeToLarge step after phase 0 needs more level storage
    than the first arena chunk (about 12 words per vertex against 8), so the
    run grows its arena; a failed growth ends that run with LC_ERR_OOM and
    the next run gives the right labels."""
    n = 200000
    perm = np.random.default_rng(4).permutation(n).astype(np.uint32)
    s, d = perm[:-1], perm[1:]
    ctx = lc.LocalContraction(n, dev(s, cuda), dev(d, cuda), seed=9, merge_alpha=[2])
    lc.fail_alloc(1)
    with pytest.raises(lc.LCError) as ei:
        ctx.run()
    assert ei.value.code == lc.LC_ERR_OOM
    lc.fail_alloc(0)
    labels, res = ctx.run()
    ctx.close()
    assert np.array_equal(labels.cpu().numpy().view(np.uint32), oracle.uf_labels(n, s, d))


def test_server_context_allocation_failure(lc_lib, cuda):
    """The server fails the job whose context cannot be created, then serves
    the next ones normally."""
    reqs = synth.serving_stream(1000.0, 6, lo_exp=8, hi_exp=12, seed=61)
    srv = lc.Server(slots=2)
    for k in (1, 2, 5):
        lc.fail_alloc(k)
        r = reqs[0].graph
        j = srv.submit(r.n, r.src, r.dst, r.seed)
        try:
            srv.wait(j)
        except lc.LCError as e:
            assert e.code == lc.LC_ERR_OOM
        lc.fail_alloc(0)
    ids = [srv.submit(r.graph.n, r.graph.src, r.graph.dst, r.graph.seed) for r in reqs]
    out = [srv.wait(j) for j in ids]
    srv.close()
    for r, (labels, rounds, _) in zip(reqs, out):
        ref = oracle.lc_run(r.graph.n, r.graph.src, r.graph.dst, r.graph.seed)
        assert rounds == ref.rounds and np.array_equal(labels, ref.labels)
