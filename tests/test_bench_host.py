"""Host logic of bench.py (no GPU): the clock log parser that decides whether
a run saw throttling, and the error over the stored oracle entries."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_clock_summary_reports_median_and_active_reasons(tmp_path):
    clk = bench.ClockSampler(0)
    clk.path = str(tmp_path / "clocks.csv")
    rows = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 2040, 2070, 1350.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 1980, 2070, 1390.0, 0x8, Active, Not Active, Not Active, Not Active",
            "malformed line",
            "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    open(clk.path, "w").write("\n".join(rows) + "\n")
    clk.proc = object()                       # as if nvidia-smi had been started
    s = clk.summary()
    assert s["sm_mhz"] == 2040.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap"]
    clk.proc = None
    assert bench.ClockSampler(0).summary()["reasons"] == ["unsampled"]


def test_golden_error_over_the_stored_entries():
    d = np.loadtxt(os.path.join(ROOT, "tests", "golden", "cluster96_K_entries.txt"))
    mu, nu, ref = d[:, 0].astype(int), d[:, 1].astype(int), d[:, 2]
    K = np.zeros((992, 992))
    K[mu, nu] = ref
    assert bench.golden_err("cluster96", K) == 0.0
    K[mu[7], nu[7]] += 3e-9
    assert abs(bench.golden_err("cluster96", K) - 3e-9) < 1e-15
    assert bench.golden_err("cluster24", K) is None      # no stored entries for this workload
