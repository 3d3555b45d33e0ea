"""Serving loop: every job's result in a mix of concurrently running jobs is
identical to the same job run alone (lc_run) and to the oracle."""
import threading
import time

import numpy as np
import pytest

import oracle
from paper_1807_10727_gb300 import lc, synth

pytestmark = pytest.mark.gpu


def requests(count, seed=505, lo=6, hi=13):
    return synth.serving_stream(1000.0, count, lo_exp=lo, hi_exp=hi, seed=seed)


def solo(g, cuda):
    import torch
    s = torch.from_numpy(g.src.view(np.int32)).to(cuda)
    d = torch.from_numpy(g.dst.view(np.int32)).to(cuda)
    c = lc.LocalContraction(g.n, s, d, seed=g.seed)
    labels, res = c.run()
    c.close()
    return labels.cpu().numpy().view(np.uint32), res.rounds


def test_mix_equals_alone(lc_lib, cuda):
    reqs = requests(48)
    srv = lc.Server(slots=8)
    ids = [srv.submit(r.graph.n, r.graph.src, r.graph.dst, r.graph.seed) for r in reqs]
    out = [srv.wait(j) for j in ids]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(reqs) and st["peak_active"] > 1
    for r, (labels, rounds, lat) in zip(reqs, out):
        ref_l, ref_r = solo(r.graph, cuda)
        assert rounds == ref_r
        assert np.array_equal(labels, ref_l)
        assert lat > 0


def test_arrivals_while_running_and_small_budget(lc_lib, cuda):
    """Jobs submitted from another thread while earlier ones run, with a
    budget that admits only a few at a time: all finish, all correct."""
    reqs = requests(24, seed=77, lo=8, hi=14)
    budget = 4 * max(1, max(r.graph.m for r in reqs)) * 40 + (64 << 20)
    srv = lc.Server(budget_bytes=budget, slots=16)
    ids = []

    def producer():
        for r in reqs:
            ids.append(srv.submit(r.graph.n, r.graph.src, r.graph.dst, r.graph.seed))
            time.sleep(0.002)

    t = threading.Thread(target=producer)
    t.start()
    t.join()
    out = [srv.wait(j) for j in ids]
    srv.close()
    for r, (labels, rounds, _) in zip(reqs, out):
        ref = oracle.lc_run(r.graph.n, r.graph.src, r.graph.dst, r.graph.seed)
        assert rounds == ref.rounds
        assert np.array_equal(labels, ref.labels)


def test_job_larger_than_budget_is_rejected(lc_lib, cuda):
    srv = lc.Server(budget_bytes=1 << 20, slots=2)
    g = synth.workload("er16")
    with pytest.raises(lc.LCError) as ei:
        srv.submit(g.n, g.src, g.dst, 1)
    assert ei.value.code == lc.LC_ERR_OOM
    srv.close()


def test_empty_and_invalid_jobs(lc_lib, cuda):
    srv = lc.Server(slots=4)
    e = np.zeros(0, np.uint32)
    j0 = srv.submit(5, e, e, 1)
    j1 = srv.submit(3, np.array([0, 1], np.uint32), np.array([1, 7], np.uint32), 1)  # id 7 >= 3
    j2 = srv.submit(4, np.array([0, 2], np.uint32), np.array([1, 3], np.uint32), 1)
    labels, rounds, _ = srv.wait(j0)
    assert rounds == 0 and list(labels) == list(range(5))
    with pytest.raises(lc.LCError) as ei:
        srv.wait(j1)
    assert ei.value.code == lc.LC_ERR_INVALID
    labels, rounds, _ = srv.wait(j2)
    assert list(labels) == [0, 0, 2, 2]
    srv.close()


def test_many_jobs_fresh_contexts_under_load(lc_lib, cuda):
    """Many concurrent jobs whose contexts are created while other jobs run
    (the case where context initialisation must be ordered on the job's own
    stream): all results equal the oracle's."""
    reqs = requests(200, seed=31, lo=6, hi=15)
    srv = lc.Server(slots=32)
    ids = [srv.submit(r.graph.n, r.graph.src, r.graph.dst, r.graph.seed) for r in reqs]
    out = [srv.wait(j) for j in ids]
    srv.close()
    for r, (labels, rounds, _) in zip(reqs, out):
        ref = oracle.lc_run(r.graph.n, r.graph.src, r.graph.dst, r.graph.seed)
        assert rounds == ref.rounds
        assert np.array_equal(labels, ref.labels)


def test_context_on_nonblocking_stream(lc_lib, cuda):
    """A context created on a non-blocking stream and run right away."""
    import torch
    g = synth.workload("rmat14")
    s = torch.cuda.Stream(device=cuda)  # non-blocking w.r.t. the legacy stream
    with torch.cuda.stream(s):
        src = torch.from_numpy(g.src.view(np.int32)).to(cuda)
        dst = torch.from_numpy(g.dst.view(np.int32)).to(cuda)
        s.synchronize()
        ref = oracle.lc_run(g.n, g.src, g.dst, g.seed)
        for _ in range(5):
            c = lc.LocalContraction(g.n, src, dst, seed=g.seed, stream=s)
            labels, res = c.run()
            c.close()
            assert res.rounds == ref.rounds
            assert np.array_equal(labels.cpu().numpy().view(np.uint32), ref.labels)


def test_config_sized_mix_sizes_match_oracle(lc_lib, cuda):
    """Jobs of the serving workload's largest sizes (n up to 2^20, up to 2^23
    edges: their large phases take the filter, distinct-count estimate and
    segmented deduplication inside the server) mixed with small ones; every
    job's labels, phase count and per-phase (n_i, m_i) equal the oracle's."""
    big = []
    s, d = synth.rmat(20, 1 << 23, 909, 910)
    big.append(synth.Graph(1 << 20, s, d, "rmat20", seed=11))
    s, d = synth.er(1 << 20, 1 << 22, 911)
    big.append(synth.Graph(1 << 20, s, d, "er20", seed=12))
    s, d = synth.grid(1024, 1024)
    synth.permute_ids(s, 1 << 20, 913)
    synth.permute_ids(d, 1 << 20, 913)
    big.append(synth.Graph(1 << 20, s, d, "grid1024", seed=13))
    small = [r.graph for r in requests(12, seed=71, lo=8, hi=14)]
    jobs = big + small
    srv = lc.Server(slots=8)
    ids = [srv.submit(g.n, g.src, g.dst, g.seed) for g in jobs]
    out = [srv.result(j) for j in ids]
    srv.close()
    for g, (labels, res, lat) in zip(jobs, out):
        ref = oracle.lc_run(g.n, g.src, g.dst, g.seed)
        assert res.rounds == ref.rounds, g.name
        assert list(zip(res.n_i, res.m_i)) == ref.sizes(), g.name
        assert np.array_equal(labels, ref.labels), g.name


def test_cancel_queued_and_running_jobs(lc_lib, cuda):
    """One slot: a cancelled queued job ends LC_ERR_CANCELLED at once; a
    running one stops at a phase boundary (or completes if it was already
    copying its labels out); the other jobs and later ones are unaffected."""
    g = synth.workload("rmat18")
    small = [r.graph for r in requests(4, seed=83, lo=8, hi=12)]
    srv = lc.Server(slots=1)
    a = srv.submit(g.n, g.src, g.dst, g.seed)
    b = srv.submit(small[0].n, small[0].src, small[0].dst, small[0].seed)
    c = srv.submit(small[1].n, small[1].src, small[1].dst, small[1].seed)
    assert srv.cancel(c)
    srv.cancel(a)
    with pytest.raises(lc.LCError) as ei:
        srv.wait(c)
    assert ei.value.code == lc.LC_ERR_CANCELLED
    try:
        labels, rounds, _ = srv.wait(a)
        ref = oracle.lc_run(g.n, g.src, g.dst, g.seed)
        assert rounds == ref.rounds and np.array_equal(labels, ref.labels)
    except lc.LCError as e:
        assert e.code == lc.LC_ERR_CANCELLED
    assert not srv.cancel(12345)
    for gg, j in [(small[0], b)] + [(x, srv.submit(x.n, x.src, x.dst, x.seed)) for x in small[2:]]:
        labels, rounds, _ = srv.wait(j)
        ref = oracle.lc_run(gg.n, gg.src, gg.dst, gg.seed)
        assert rounds == ref.rounds and np.array_equal(labels, ref.labels)
    srv.close()
