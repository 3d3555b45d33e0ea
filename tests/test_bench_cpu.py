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
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["nproc"] >= 1 and cb["cpu_model"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_step_bytes_accounting():
    """Each step counts its edges once per phase, whatever the launch
    structure; the steps add up to the path total."""
    n_i, m_i, mp_i = [1000, 100, 10], [8000, 500, 20], [7000, 400, 15]
    sb = bench.step_bytes(n_i, m_i, mp_i)
    assert sb["parent"] == sum(8 * m + 8 * n for n, m in zip(n_i, m_i))
    assert sb["relabel"] == sum(8 * m + 8 * p + 4 * n for n, m, p in zip(n_i, m_i, mp_i))
    assert sb["dedup"] == 16 * sum(mp_i)
    assert sb["compact"] == 8 * (500 + 20) + 4 * sum(n_i)
    assert sb["labels"] == 8 * sum(n_i) + 8 * 1000
    total = bench.path_bytes(n_i, m_i, mp_i)
    assert total == sum(sb.values())
    # the survey's per-phase figure: 16 m + 24 m' + 8 m_next + 28 n, plus the labels
    assert total == sum(16 * m + 24 * p + 28 * n for n, m, p in zip(n_i, m_i, mp_i)) + \
        8 * (500 + 20) + 8 * sum(n_i) + 8 * 1000
    assert bench.variant_path_bytes(1, 0, n_i, m_i, mp_i) > total  # two-hop adds an edge pass


def test_step_report_and_roofline():
    """The dominant step's fraction is recomputable from the reported bytes
    and times."""
    n_i, m_i, mp_i = [1000, 100], [8000, 500], [7000, 400]
    kstats = {"edge_min_packed": (4, 2.0), "bucket_edges": (6, 1.0), "relabel_packed": (4, 6.0),
              "sort_pass": (2, 1.0), "jump": (4, 0.4)}
    steps = bench.step_report(kstats, 2, n_i, m_i, mp_i, 1000.0, "measured")
    assert abs(steps["parent"]["ms"] - 1.5) < 1e-12
    roof = bench.roofline_of(steps, 1000.0, "measured", "x")
    assert roof["step"] == "relabel"
    ach = steps["relabel"]["algorithmic_bytes"] / (3.0 / 1e3) / 1e9
    assert abs(roof["achieved"] - ach) < 1e-9 and abs(roof["frac"] - ach / 1000.0) < 1e-12
    # DRAM traffic: the captured ratio for this step times its algorithmic
    # bytes, only while the CUDA sources are the ones the captures were taken on
    ratio = bench.TRAFFIC["per_alg_byte"].get("relabel")
    if ratio and bench.TRAFFIC["sources"] == bench.sources_hash():
        assert abs(roof["traffic"] - ratio * steps["relabel"]["algorithmic_bytes"]) < 1e-6
    else:
        assert roof["traffic"] is None
    for names in bench.STEP_KERNELS.values():
        assert len(names) == len(set(names))


def test_tuned_table_lookup(tmp_path, monkeypatch):
    """The binding applies the entry of the nearest size class of the same
    kind in (log2 n, log2 m), and nothing when no class is near."""
    from paper_1807_10727_gb300 import tune
    table = {"classes": [
        {"n_log2": 20, "m_log2": 24, "params": {"relabel_cache_admit": 2}},
        {"n_log2": 26, "m_log2": 30, "kind": "single", "params": {"bucket_window_bytes": 32 << 20}},
        {"n_log2": 26, "m_log2": 28, "kind": "batch", "params": {"seg_dedup": 0}}]}
    path = tmp_path / "tuned.json"
    path.write_text(json.dumps(table))
    monkeypatch.setattr(tune, "_table", None)
    tune.load_table(str(path))
    assert tune.params_for(1 << 26, 1 << 30) == {"bucket_window_bytes": 32 << 20}
    assert tune.params_for((1 << 20) + 5, 3 << 22) == {"relabel_cache_admit": 2}
    assert tune.params_for(1 << 10, 1 << 12) == {}
    # batches take batch classes only, single graphs single-graph classes only
    assert tune.params_for(1 << 26, 1 << 28, "batch") == {"seg_dedup": 0}
    assert tune.params_for(1 << 26, 1 << 30, "batch") == {"seg_dedup": 0}
    assert tune.params_for(1 << 20, 1 << 24, "batch") == {}
    assert tune.params_for(1 << 26, 1 << 28) == {"bucket_window_bytes": 32 << 20}
    assert tune.class_key(1, 0) == (0, 0)
    monkeypatch.setattr(tune, "_table", None)
