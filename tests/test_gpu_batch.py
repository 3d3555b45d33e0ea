"""Batched runs: every graph of a batch must get exactly what its own lc_run
gives (labels, phase count, per-phase sizes), and what the oracle gives."""
import os

import numpy as np
import pytest

import oracle
from paper_1807_10727_gb300 import lc, synth

pytestmark = pytest.mark.gpu


def to_dev(a, cuda):
    import torch
    a = np.ascontiguousarray(np.asarray(a, dtype=np.uint32))
    return torch.from_numpy(a.view(np.int32)).to(cuda)


def check_batch(n, eoff, src, dst, seeds, cuda, cap=256):
    k = len(n)
    ts, td = to_dev(src, cuda), to_dev(dst, cuda)
    b = lc.BatchLocalContraction(n, eoff, ts, td, seeds)
    labels, rounds, n_i, m_i = b.run(cap=cap)
    b.close()
    labels = labels.cpu().numpy().view(np.uint32)
    voff = np.zeros(k + 1, dtype=np.int64)
    np.cumsum(np.asarray(n, dtype=np.int64), out=voff[1:])
    for g in range(k):
        s, d = src[eoff[g]:eoff[g + 1]], dst[eoff[g]:eoff[g + 1]]
        ref = oracle.lc_run(int(n[g]), s, d, int(seeds[g]))
        assert rounds[g] == ref.rounds, g
        R = int(rounds[g])
        assert list(zip(n_i[g, :R].tolist(), m_i[g, :R].tolist())) == ref.sizes(), g
        assert np.array_equal(labels[voff[g]:voff[g + 1]], ref.labels), g


def test_batch_recipe_small(lc_lib, cuda):
    b = synth.batch(k=96, lo_exp=3, hi_exp=11)
    check_batch(b.n, b.eoff, b.src, b.dst, b.seeds, cuda)


def test_batch_matches_solo_lc_run(lc_lib, cuda):
    """Bit-identical to separate lc_run calls (not only to the oracle)."""
    import torch
    b = synth.batch(k=40, lo_exp=6, hi_exp=12, seed=9)
    ts, td = to_dev(b.src, cuda), to_dev(b.dst, cuda)
    bl = lc.BatchLocalContraction(b.n, b.eoff, ts, td, b.seeds)
    labels, rounds, n_i, m_i = bl.run()
    bl.close()
    voff = np.concatenate([[0], np.cumsum(b.n.astype(np.int64))])
    for g in range(b.k):
        gr = b.graph(g)
        solo = lc.LocalContraction(gr.n, to_dev(gr.src, cuda), to_dev(gr.dst, cuda), seed=gr.seed)
        sl, sr = solo.run()
        solo.close()
        R = int(rounds[g])
        assert (R, n_i[g, :R].tolist(), m_i[g, :R].tolist()) == (sr.rounds, sr.n_i, sr.m_i)
        assert torch.equal(labels[voff[g]:voff[g + 1]], sl)


def test_batch_edge_cases(lc_lib, cuda):
    # graphs without edges, a loops-only graph, one-vertex graphs, an empty graph
    n = np.array([5, 1, 3, 0, 4, 2], dtype=np.uint32)
    edges = [[], [(0, 0)], [(0, 1), (1, 2)], [], [(3, 3), (3, 3)], [(1, 0), (0, 1), (1, 1)]]
    eoff = np.zeros(len(n) + 1, dtype=np.uint64)
    src, dst = [], []
    for g, es in enumerate(edges):
        src += [a for a, _ in es]
        dst += [b for _, b in es]
        eoff[g + 1] = eoff[g] + len(es)
    check_batch(n, eoff, np.array(src, np.uint32), np.array(dst, np.uint32),
                np.arange(len(n), dtype=np.uint64) + 3, cuda)


def test_batch_single_graph_equals_config1(lc_lib, cuda):
    g = synth.workload("er16")
    check_batch(np.array([g.n], np.uint32), np.array([0, g.m], np.uint64), g.src, g.dst,
                np.array([g.seed], np.uint64), cuda)


def test_batch_many_small_graphs(lc_lib, cuda):
    """More graphs than a block keeps per-graph edge counts for in shared
    memory (8192), with empty and edgeless graphs in between: the per-level
    graph ids, the chunked offset walks and the global edge counting."""
    rng = np.random.default_rng(77)
    k = 9000
    n = rng.integers(0, 40, size=k).astype(np.uint32)
    n[rng.random(k) < 0.1] = 0
    m = np.where(n > 0, rng.integers(0, 3 * n + 1), 0).astype(np.uint64)
    eoff = np.concatenate([[0], np.cumsum(m)]).astype(np.uint64)
    src = np.concatenate([rng.integers(0, max(int(x), 1), size=int(c)) for x, c in zip(n, m)])
    dst = np.concatenate([rng.integers(0, max(int(x), 1), size=int(c)) for x, c in zip(n, m)])
    check_batch(n, eoff, src.astype(np.uint32), dst.astype(np.uint32),
                np.arange(k, dtype=np.uint64) * 7 + 1, cuda)


def test_batch_local_id_out_of_range(lc_lib, cuda):
    n = np.array([3, 3], dtype=np.uint32)
    eoff = np.array([0, 1, 2], dtype=np.uint64)
    ts, td = to_dev([0, 1], cuda), to_dev([2, 3], cuda)  # graph 1 uses id 3 >= 3
    b = lc.BatchLocalContraction(n, eoff, ts, td, np.array([1, 2], np.uint64))
    with pytest.raises(lc.LCError) as ei:
        b.run()
    assert ei.value.code == lc.LC_ERR_INVALID
    b.close()


@pytest.mark.slow
def test_config4_batch_at_size(lc_lib, cuda):
    """The batched workload at its stated size: 4096 graphs, n log-uniform in
    [2^6, 2^16], half ER (degree 4) and half R-MAT (degree 16), about 3.9e7
    vertices and 1.9e8 edges in one context.  Phase 0 of the batch then
    takes the large-phase path (edge buckets, duplicate filter, distinct-key
    estimate, segmented deduplication).  Every graph's labels, phase count
    and per-phase (n_i, m_i) are compared with the oracle (run on the host's
    cores in parallel)."""
    from concurrent.futures import ThreadPoolExecutor
    b = synth.batch(k=4096)
    assert int(b.eoff[-1]) >= 1 << 22 and int(b.n.max()) <= 1 << 16
    ts, td = to_dev(b.src, cuda), to_dev(b.dst, cuda)
    bl = lc.BatchLocalContraction(b.n, b.eoff, ts, td, b.seeds)
    labels, rounds, n_i, m_i = bl.run(cap=64)
    bl.close()
    labels = labels.cpu().numpy().view(np.uint32)
    voff = np.concatenate([[0], np.cumsum(b.n.astype(np.int64))])

    def ref(g):
        gr = b.graph(g)
        return oracle.lc_run(gr.n, gr.src, gr.dst, gr.seed)

    refs = [ref(0)]  # loads the oracle library before the threads share it
    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        refs += list(ex.map(ref, range(1, b.k)))
    for g, r in enumerate(refs):
        R = int(rounds[g])
        assert R == r.rounds, g
        assert list(zip(n_i[g, :R].tolist(), m_i[g, :R].tolist())) == r.sizes(), g
        assert np.array_equal(labels[voff[g]:voff[g + 1]], r.labels), g
