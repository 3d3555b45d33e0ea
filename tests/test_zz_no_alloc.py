"""lc_run_static: the allocation-free entry point.

It exists for callers that may not allocate device memory (code under another
framework's allocator that already holds the device, plug-ins or callbacks
that must not touch the allocator, latency-critical loops avoiding
cudaMalloc's device synchronisation).  It must give exactly what lc_run gives
on the same input -- labels, phase count and per-phase sizes -- on two calls
in a row, since every call reuses the same static scratch array, and it must
leave the device's free memory as it found it.  This file is
collected last so that a failure here stops a run only after every other test
has run.
"""
import numpy as np
import pytest

import oracle
from paper_1807_10727_gb300 import lc, synth

pytestmark = pytest.mark.gpu


def dev(a, cuda):
    import torch
    a = np.ascontiguousarray(np.asarray(a, dtype=np.uint32))
    return torch.from_numpy(a.view(np.int32)).to(cuda)


def graphs():
    g = synth.workload("er16")  # n = 2^16, m = 2^19
    yield "er16", g.n, g.src, g.dst, g.seed
    s, d = synth.rmat(17, lc.LC_STATIC_MAX_M, 202, 203)  # the largest allowed size
    yield "rmat17", 1 << 17, s, d, 7
    s, d = synth.grid(300, 300)
    synth.permute_ids(s, 90000, 5)
    synth.permute_ids(d, 90000, 5)
    yield "grid300", 90000, s, d, 3
    rng = np.random.default_rng(8)
    yield "tiny", 37, rng.integers(0, 37, 50), rng.integers(0, 37, 50), 2
    yield "no_edges", 10, np.zeros(0, np.uint32), np.zeros(0, np.uint32), 1


def static_run(n, ts, td, m, seed, labels):
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    out = lc.lc_run_static(n, ts.data_ptr() if m else 0, td.data_ptr() if m else 0, m, seed,
                           stream, labels.data_ptr())
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("case", list(range(5)))
def test_static_matches_lc_run_on_two_calls(lc_lib, cuda, case):
    """Two calls in a row give lc_run's labels, phase count and per-phase
    sizes (and the oracle's), and leave the device's free memory unchanged:
    the calls allocate nothing."""
    import torch
    name, n, s, d, seed = list(graphs())[case]
    ts, td = dev(s, cuda), dev(d, cuda)
    ctx = lc.LocalContraction(n, ts, td, seed=seed)
    ref_labels, ref = ctx.run()
    ctx.close()
    orc = oracle.lc_run(n, s, d, seed)
    assert (ref.rounds, list(zip(ref.n_i, ref.m_i))) == (orc.rounds, orc.sizes()), name
    labels = torch.full((n,), -1, dtype=torch.int32, device=cuda)
    static_run(n, ts, td, len(s), seed, labels)  # first call on the device: address look-up
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        labels.fill_(-1)
        r, n_i, m_i = static_run(n, ts, td, len(s), seed, labels)
        assert (r, n_i, m_i) == (ref.rounds, ref.n_i, ref.m_i), name
        assert torch.equal(labels, ref_labels), name
        assert np.array_equal(labels.cpu().numpy().view(np.uint32), orc.labels), name
    assert torch.cuda.mem_get_info()[0] == free0, name


def test_static_storage_exhausted_then_recovers(lc_lib, cuda):
    """When the static per-phase storage runs out (forced here with the
    library's allocation-failure hook, which counts the pieces carved from
    the static array) the call returns LC_ERR_OOM, and the next call gives
    lc_run's result again."""
    import torch
    g = synth.workload("er16")
    ts, td = dev(g.src, cuda), dev(g.dst, cuda)
    ctx = lc.LocalContraction(g.n, ts, td, seed=g.seed)
    ref_labels, ref = ctx.run()
    ctx.close()
    labels = torch.full((g.n,), -1, dtype=torch.int32, device=cuda)
    for k in (1, 4):
        lc.fail_alloc(k)
        with pytest.raises(lc.LCError) as ei:
            static_run(g.n, ts, td, g.m, g.seed, labels)
        assert ei.value.code == lc.LC_ERR_OOM
    lc.fail_alloc(0)
    labels.fill_(-1)
    r, n_i, m_i = static_run(g.n, ts, td, g.m, g.seed, labels)
    assert (r, n_i, m_i) == (ref.rounds, ref.n_i, ref.m_i)
    assert torch.equal(labels, ref_labels)


def test_static_rejects_sizes_beyond_the_maximum(lc_lib, cuda):
    import torch
    buf = torch.zeros(4, dtype=torch.int32, device=cuda)
    p = buf.data_ptr()
    stream = torch.cuda.current_stream().cuda_stream
    for n, m in [(lc.LC_STATIC_MAX_N + 1, 1), (16, lc.LC_STATIC_MAX_M + 1)]:
        with pytest.raises(lc.LCError) as ei:
            lc.lc_run_static(n, p, p, m, 1, stream, p)
        assert ei.value.code == lc.LC_ERR_INVALID
