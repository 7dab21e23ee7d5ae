"""Host-only parts of bench.py: the statistics of the schedules config and the
planner config's JSON line (the planner runs on the CPU)."""
import json

import numpy as np
import pytest

import bench


def test_r2_loglog_exact_power_law():
    x = np.array([1.0, 2.0, 5.0, 10.0, 40.0])
    assert bench._r2_loglog(x, 3.0 * x ** 1.7) == pytest.approx(1.0)
    assert bench._r2_loglog([1, 2], [3, 4]) is None  # fewer than 3 points
    assert bench._r2_loglog([1, 1, 1], [1, 2, 3]) is None  # no spread


def test_r2_loglog_matches_least_squares():
    rng = np.random.default_rng(3)
    x = np.exp(rng.normal(size=30))
    y = np.exp(0.5 * np.log(x) + rng.normal(scale=0.5, size=30))
    lx, ly = np.log(x), np.log(y)
    a, b = np.polyfit(lx, ly, 1)
    resid = ly - (a * lx + b)
    r2 = 1 - (resid ** 2).sum() / ((ly - ly.mean()) ** 2).sum()
    assert bench._r2_loglog(x, y) == pytest.approx(r2)


def test_spearman():
    assert bench._spearman([1, 2, 3, 4], [10, 20, 30, 40]) == pytest.approx(1.0)
    assert bench._spearman([1, 2, 3, 4], [9, 7, 5, 1]) == pytest.approx(-1.0)
    assert bench._spearman([1, 2], [2, 1]) is None


def test_planner_config_line(capsys):
    pytest.importorskip("paper_1911_12877_gb300")
    assert bench.main(["--config", "planner", "--steps", "1", "--warmup", "3"]) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "config", "gpu_launches"):
        assert key in line
    assert line["gpu_launches"] == 0 and line["unit"] == "ms" and line["value"] > 0
    assert line["max_pattern_schedules"] >= 1


def test_committed_profile_matches_kernel_source():
    """The committed ncu summary of the dominant kernel was taken on the current
    source of that kernel, so the bench can report its DRAM traffic (a changed
    kernel must be profiled again, and its traffic reads null until then)."""
    d = bench.profiled(bench.PROFILE_K5)
    assert d is not None, "k_clique_warp changed since its ncu capture"
    assert d["dram_bytes_per_launch"] == d["dram_bytes_read"] + d["dram_bytes_write"]


def test_clique_roofline_arithmetic():
    """The fused count's roofline: achieved = the oracle's K4 + K5 bitset word
    operations / count time; peak = 16 popcounts per clock per SM x SMs x the
    sampled SM clock; traffic and DRAM fraction from the committed capture."""
    gold = json.load(open(bench.os.path.join(bench.GOLDEN, "clique_rmat20.json")))
    words = gold["k4"]["bitset_words"] + gold["k5"]["bitset_words"]
    prof = {"dram_bytes_per_launch": 470_000_000, "xu_pipe_pct": 40.0, "issue_active_pct": 70.0}
    r = bench.clique_roofline(words, 0.025, 4.97e12, {"sm_mhz": 2070.0}, 152, prof)
    peak = 16 * 152 * 2070e6 / 1e9
    assert r["bound"] == "alu" and r["unit"] == "Gword-op/s"
    assert r["peak"] == pytest.approx(peak, rel=1e-4)
    assert r["achieved"] == pytest.approx(words / 0.025 / 1e9, rel=1e-4)
    assert r["frac"] == pytest.approx(words / 0.025 / 1e9 / peak, abs=1e-4)
    assert r["traffic"] == 470_000_000
    assert r["dram_frac"] == pytest.approx(470e6 / 0.025 / 1e9 / bench.measured_peaks()[0], abs=1e-6)
    assert r["algorithmic_words"] == words
