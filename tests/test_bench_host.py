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
