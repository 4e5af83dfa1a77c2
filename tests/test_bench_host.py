"""CPU checks of bench.py's host logic that the GPU runs depend on: the
clock sampler's reading of nvidia-smi's CSV (median SM clock under load,
the throttle reasons that were active), and the work counts behind the
roofline figure."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


class _Done:
    def terminate(self):
        pass

    def wait(self):
        pass


def sampled(tmp_path, lines):
    path = tmp_path / "clocks.csv"
    path.write_text("\n".join(lines) + "\n")
    c = bench.ClockSampler()
    c.proc, c.path = _Done(), str(path)
    return c.stop()


def test_clock_sampler_reads_the_query_lines(tmp_path):
    # index, clocks.sm, clocks.max.sm, power.draw, reasons.active, hw_slowdown,
    # hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap (noheader, nounits)
    rows = [f"0, {mhz}, 2070, 900.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
            for mhz in (2070, 2070, 1980, 2070, 2055)]
    rows.insert(2, "0, 1995, 2070, 1390.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active")
    rows.append("not a sample line")
    r = sampled(tmp_path, rows)
    assert r["samples"] == 6 and r["sm_max_mhz"] == 2070.0
    assert r["sm_mhz"] == float(np.median([2070, 2070, 1995, 1980, 2070, 2055]))
    assert r["reasons"] == ["sw_power_cap"]  # "Not Active" is not active
    assert not os.path.exists(tmp_path / "clocks.csv")


def test_clock_sampler_reports_every_slowdown_it_saw(tmp_path):
    rows = ["0, 1500, 2070, 1200.0, 0x8, Active, Not Active, Not Active, Not Active",
            "0, 1400, 2070, 1200.0, 0x40, Not Active, Active, Active, Not Active"]
    r = sampled(tmp_path, rows)
    assert r["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_sampler_without_samples(tmp_path):
    assert sampled(tmp_path, ["garbage"]) is None
    c = bench.ClockSampler()  # never started (no nvidia-smi): no clocks to report
    assert c.stop() is None


def test_work_counts():
    # the per-step algorithmic count, 35 N s with s = 6 (N = 97 at hierarchies 30)
    assert bench.flops_per_step(97) == 35 * 97 * 6
    # projection points: l = 2 .. cut(x) per node, x = k (tau_0 - tau)
    n = bench.projection_points(np.array([0.0, 100.0, 200.0]), 200.0, np.array([1e-3, 1.0]), 400)
    cuts = bench.bessel_cut(np.outer([1e-3, 1.0], [200.0, 100.0, 0.0]), 400)
    assert n == float(np.maximum(cuts - 1, 0).sum())
    assert bench.whole_job_rate(64, 2, 4000.0) == 32.0
