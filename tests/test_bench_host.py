"""Host-side pieces of bench.py that need no GPU: where clock samples go, the
algorithmic bytes of a step, and the scaling of the measured DRAM traffic."""
import os

import pytest


@pytest.fixture(scope="module")
def bench():
    import bench as b
    return b


def test_clock_samples_follow_the_environment(bench, tmp_path, monkeypatch):
    monkeypatch.setenv("EO_CLOCKS_DIR", str(tmp_path))
    assert bench.clocks_path("clocks_rank0.csv") == os.path.join(str(tmp_path), "clocks_rank0.csv")
    # a variable that names no folder falls back to the temporary directory
    monkeypatch.setenv("EO_CLOCKS_DIR", str(tmp_path / "missing"))
    p = bench.clocks_path("clocks_rank0.csv")
    assert os.path.dirname(p) != str(tmp_path / "missing") and p.endswith("clocks_rank0.csv")
    monkeypatch.delenv("EO_CLOCKS_DIR")
    assert os.path.isdir(os.path.dirname(bench.clocks_path("x.csv")))


def test_step_bytes_count_what_the_method_must_move(bench):
    n, kv, k = 4_000_000, 64, 16
    one = 8 * n * (kv + k) + 8 * n * (kv + 2 * k) + 16 * n * k  # V^T Y, Y - V C, one CholQR update
    assert bench.step_bytes(n, kv, k, False) == one
    assert bench.step_bytes(n, kv, k, True) == one + 8 * n * k + 16 * n * k  # Q^T Q and the second update
    assert bench.step_bytes(n, kv, k, True) == 8_192_000_000


def test_gram_traffic_scales_reads_with_rows(bench):
    t1 = bench.gram_traffic(1_000_000, 64, 16)
    t4 = bench.gram_traffic(4_000_000, 64, 16)
    reads = (t4 - t1) / 3
    assert reads == pytest.approx(640e6, rel=1e-3)  # 1e6 rows x 80 columns x 8 B, no re-reads
    assert t1 - reads == pytest.approx(t4 - 4 * reads)  # the partials do not grow with n
    assert 0 < t1 - reads < 8e6
    assert bench.gram_traffic(1_000_000, 32, 16) is None


def test_reference_arm_prints_one_json_line(tmp_path):
    """`bench.py --impl reference` runs the oracle's CPU arithmetic (no GPU)
    and prints the base contract's line with the reference keys."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--n", "20000",
                          "--cpu-rows", "20000", "--steps", "2", "--warmup", "1"], capture_output=True, text=True,
                         timeout=600, cwd=str(tmp_path))
    assert out.returncode == 0, out.stderr
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    r = json.loads(lines[0])
    assert r["impl"] == "reference" and r["unit"] == "GB/s" and r["value"] > 0
    assert r["cpu_baseline"]["kind"] == "oracle" and r["cpu_baseline"]["cores"] >= 1
    assert r["e2e"]["h2d_bytes_per_step"] == 0 and r["e2e"]["value"] == r["value"]


def test_cpu_baseline_reports_dd_fp64_and_one_core(bench):
    import numpy as np
    import synth
    v = synth.orthonormal_basis(3000, 8, 1)
    y = synth.conditioned(3000, 4, 1e10, 2)
    r = bench.cpu_baseline(v, y, 0)
    assert r["kind"] == "oracle" and r["value"] > 0 and r["cores"] >= 1
    assert r["orth_err"] is not None and r["orth_err"] <= 1e-14  # the DD step is accurate at kappa = 1e10
    assert r["fp64_cholqr2"]["value"] > 0 and r["one_core_dd"]["rows"] == 3000


def test_other_configs_summarises_each_workload(bench, monkeypatch):
    """The default line's summary of the other workloads, from canned lines
    (no GPU): every field is taken from its workload's own line, serving at
    0.8x is offered 0.8x the capacity that run measured, and a workload that
    fails or lacks a field is reported without stopping the others."""
    import json
    import subprocess

    lines = {
        "sweep": {"config": {"workload": "sweep"}, "results": [
            {"k": 16, "mode": "dd", "xtx_gbs": 1200.04, "xty_gbs": 1300.06}]},
        "batched": {"config": {"workload": "batched"}, "ms_per_step": 150.0, "blocks_per_s": 3400.0, "value": 700.0,
                    "p50_ms": 150.0, "p99_ms": 151.0, "orth_err_max": 1e-16, "roofline": {"frac": 0.1},
                    "comparators": {"fp64_graph_ms": 330.0}, "clocks": {"sm_mhz": 2070.0}},
        "serve": {"config": {"workload": "serve"}, "value": 500.0, "gbs": 900.0, "p50_ms": 9.0, "p99_ms": 40.0,
                  "queue_p50_ms": 0.01, "queue_p99_ms": 10.0, "orth_err_max": 1e-18, "cross_err_max": 1e-18},
        "iterated": {"config": {"workload": "iterated"}},  # no results: a summary error
        "update": {"config": {"workload": "update"}, "results": {"16": {"p50_ms": 0.9054, "gbs": 1130.04}}},
    }
    seen = []

    class Done:
        def __init__(self, out, rc=0):
            self.stdout, self.stderr, self.returncode = out, "", rc

    def fake_run(cmd, **kw):
        args = cmd[2:]
        seen.append(args)
        w = args[args.index("--workload") + 1]
        return Done("noise\n" + json.dumps(lines[w]) + "\n")

    monkeypatch.setattr(subprocess, "run", fake_run)
    out = bench.other_configs()
    assert out["sweep"]["results"] == {"16": {"dd": [1200.0, 1300.1]}}
    assert out["batched"]["blocks_per_s"] == 3400.0 and out["batched"]["hbm_frac"] == 0.1
    assert out["serve_offered_2000"]["requests_per_s"] == 500.0
    assert ["--workload", "serve", "--rate", "400.0", "--requests", "1500"] in seen
    assert out["serve_at_0.8_capacity"]["offered_per_s"] == 400.0
    assert "error" in out["iterated"]
    assert out["update"]["p50_ms_and_gbs_per_k"] == {"16": [0.905, 1130.0]}

    monkeypatch.setattr(subprocess, "run", lambda cmd, **kw: Done("", rc=1))
    out = bench.other_configs()
    assert all("error" in v for v in out.values()) and "serve_at_0.8_capacity" not in out
