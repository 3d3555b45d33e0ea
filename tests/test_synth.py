"""Input generators: determinism, thread-count independence, shapes."""
import numpy as np

from paper_1807_10727_gb300 import synth


def test_er_deterministic_and_thread_independent():
    a = synth.er(1000, 100000, 7, nthreads=1)
    b = synth.er(1000, 100000, 7, nthreads=5)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert a[0].max() < 1000 and a[1].max() < 1000
    c = synth.er(1000, 100000, 8)
    assert not np.array_equal(a[0], c[0])
    # roughly uniform endpoints
    h = np.bincount(a[0], minlength=1000)
    assert h.min() > 50 and h.max() < 160


def test_rmat_skew_and_bounds():
    s, d = synth.rmat(14, 1 << 18, 3, nthreads=3)
    s2, d2 = synth.rmat(14, 1 << 18, 3, nthreads=1)
    assert np.array_equal(s, s2) and np.array_equal(d, d2)
    assert s.max() < (1 << 14)
    deg = np.bincount(np.concatenate([s, d]), minlength=1 << 14)
    # a = 0.57 concentrates on low ids before permutation
    assert deg[0] > 50 * np.median(deg[deg > 0])
    # n_keep rejection keeps ids in range
    s3, d3 = synth.rmat(14, 1 << 12, 3, n_keep=10000)
    assert s3.max() < 10000 and d3.max() < 10000


def test_permutation_is_a_bijection():
    for n in (1, 2, 3, 17, 1000, 4096, 12345):
        x = np.arange(n, dtype=np.uint32)
        synth.permute_ids(x, n, 99)
        assert np.array_equal(np.sort(x), np.arange(n, dtype=np.uint32))
        if n > 100:
            assert (x != np.arange(n)).mean() > 0.9


def test_grid_shape():
    s, d = synth.grid(5, 3)
    assert len(s) == 3 * 4 + 5 * 2
    diff = d.astype(np.int64) - s.astype(np.int64)
    assert set(np.unique(diff)) == {1, 5}


def test_grid_mix_recipe():
    g = synth.workload("gridmix_small")
    sizes = synth.powerlaw_sizes(1 << 12, 2, 1 << 14, 2.1, 303)
    assert g.n == 512 * 512 + int(sizes.sum())
    assert g.m == 2 * 512 * 511 + int(np.ceil(sizes * 1.5).sum())
    assert g.src.max() < g.n and g.dst.max() < g.n
    # power law: most components are tiny
    assert (sizes == 2).mean() > 0.3 and sizes.max() > 100


def test_batch_recipe():
    b = synth.batch(k=64)
    assert b.k == 64
    assert b.n.min() >= 64 and b.n.max() <= 1 << 16
    m = np.diff(b.eoff)
    assert np.array_equal(m[0::2], 2 * b.n[0::2].astype(np.uint64))
    assert np.array_equal(m[1::2], 8 * b.n[1::2].astype(np.uint64))
    for g in range(b.k):
        gr = b.graph(g)
        assert gr.m == 0 or (gr.src.max() < gr.n and gr.dst.max() < gr.n)


def test_serving_stream_recipe():
    reqs = synth.serving_stream(1000.0, 30, lo_exp=6, hi_exp=10)
    t = [r.arrival_s for r in reqs]
    assert all(b > a for a, b in zip(t, t[1:]))
    assert {r.kind for r in reqs} <= {"er", "rmat", "grid"}
    for r in reqs:
        assert r.graph.src.max() < r.graph.n
