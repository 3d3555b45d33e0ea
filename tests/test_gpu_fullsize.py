"""Full-size parity in the benchmark's launch configuration (one context, the
default hashed dedup): R-MAT scale 26 (2^30 edges) and the 8192^2 grid +
2^20 power-law components mix.  Labels are compared element by element with
the oracle's union-find labels, and the phase count and every per-phase
(n_i, m_i) with the oracle's full run."""
import numpy as np
import pytest

import oracle
from paper_1807_10727_gb300 import lc, synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def run_full(name, cuda, variant=lc.LC_VARIANT_FOREST, finish=0):
    import torch
    g = synth.workload(name)
    src = torch.from_numpy(g.src.view(np.int32)).to(cuda)
    dst = torch.from_numpy(g.dst.view(np.int32)).to(cuda)
    ctx = lc.LocalContraction(g.n, src, dst, seed=g.seed, variant=variant, finish_edges=finish)
    labels, res = ctx.run()
    mp = ctx.mprime()
    ctx.close()
    got = labels.cpu().numpy().view(np.uint32)
    del src, dst, labels
    torch.cuda.empty_cache()
    return g, got, res, mp


@pytest.mark.parametrize("name", ["gridmix", "rmat26"])
def test_fullsize_parity(lc_lib, cuda, name):
    g, got, res, mp = run_full(name, cuda)
    uf = oracle.uf_labels(g.n, g.src, g.dst)
    assert np.array_equal(got, uf)
    ref = oracle.lc_run(g.n, g.src, g.dst, g.seed)
    assert res.rounds == ref.rounds
    assert list(zip(res.n_i, res.m_i)) == ref.sizes()
    assert mp == [int(x) for x in ref.mp_i]


@pytest.mark.parametrize("variant,finish", [(lc.LC_VARIANT_TWO_HOP, 0), (lc.LC_VARIANT_TREE, 0),
                                            (lc.LC_VARIANT_FOREST, 1 << 22)])
def test_fullsize_variants_gridmix(lc_lib, cuda, variant, finish):
    """The other variants and the finish on the 8192^2 grid + power-law mix
    (2^26 + ~1.2e7 vertices, ~1.5e8 edges)."""
    g, got, res, mp = run_full("gridmix", cuda, variant, finish)
    assert np.array_equal(got, oracle.uf_labels(g.n, g.src, g.dst))
    ref = oracle.lc_run(g.n, g.src, g.dst, g.seed, variant=variant, finish_edges=finish)
    assert res.rounds == ref.rounds
    assert list(zip(res.n_i, res.m_i)) == ref.sizes()
    assert mp == [int(x) for x in ref.mp_i]
