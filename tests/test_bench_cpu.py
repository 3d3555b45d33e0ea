"""bench.py's host-side parts, without a GPU: the reference arm (the oracle on
a bounded sample) prints one well-formed JSON line, and the algorithmic-byte
accounting behaves on hand-made phase sizes."""
import json
import os
import subprocess
import sys

REPO = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, REPO)

import bench  # noqa: E402


def test_reference_arm_prints_one_json_line():
    out = subprocess.run([sys.executable, os.path.join(REPO, "bench.py"), "--impl", "reference",
                          "--workload", "er16", "--steps", "1", "--warmup", "1"],
                         capture_output=True, text=True, timeout=600, check=True, cwd=REPO)
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_algorithmic_bytes_accounting():
    n_i, m_i = [1000, 100, 10], [8000, 500, 20]
    mp_i, em_i, kept_i, passes_i = [7000, 400, 15], [6000, 380, 15], [6000, 380, 15], [1, 0, 0]
    per = bench.algorithmic_bytes(n_i, m_i, mp_i, em_i, kept_i, passes_i, 1, False)
    # phase 0 reads its 8-byte edges in the minimum and the relabel
    assert per["edge_min_soa"] == 8 * 8000 + 8 * 1000
    assert per["relabel_soa"] == 8 * 8000 + 8 * 6000 + 4 * 1000
    # one partition pass over the kept keys of phase 0 only
    assert per["sort_pass"] == 16 * 6000
    assert "filter_hll" not in per  # no phase reaches the late-planning size
    assert all(v >= 0 for v in per.values())
    total = bench.path_bytes(n_i, m_i, mp_i)
    assert total > per["relabel_soa"]
    assert bench.variant_path_bytes(1, 0, n_i, m_i, mp_i) > total  # two-hop adds an edge pass
