"""Host arithmetic of the benchmark line, without a GPU: the whole-job value,
the roofline of the half-sweep kernel from its event timings, and the clock
summary parsed from nvidia-smi's CSV output."""
from __future__ import annotations

import os
import tempfile

import pytest

import bench


def test_job_value_is_slowest_rank_over_all_updates():
    # 2 ranks, 1e9 updates each, slowest rank 3 ms: 3e-3 s / 2e9 = 1.5 ps
    assert bench.job_value(3.0, 10 ** 9, 2) == pytest.approx(1.5)
    assert bench.rank_seed(7, 0) == 7 and bench.rank_seed(7, 3) != bench.rank_seed(7, 2)


def test_roofline_from_event_timing():
    from paper_2402_03920_gb300 import qisg
    w = bench.workload()
    steps = 4
    launches = 2 * bench.SWEEPS_PER_STEP * steps          # red and blue per sweep
    kern = {"sweep": {"timed": launches, "launched": launches, "ms": launches * 0.02}}   # 20 us each
    pk = {"sm_max_mhz": 2000.0}
    rl = bench.roofline(kern, w, qisg.QISG_LAYOUT_SAMPLES, 32, 100, pk, steps)
    ups = bench.updates_per_step(w) * steps / launches
    assert rl["updates_per_launch"] == pytest.approx(ups)
    assert rl["avg_launch_us"] == pytest.approx(20.0)
    assert rl["achieved"] == pytest.approx(bench.ALG_OPS["samples32"] * ups / 20e-6 / 1e12)
    assert rl["peak"] == pytest.approx(100 * bench.INT_LANES_PER_CLK_PER_SM * 2000e6 / 1e12)
    assert rl["frac"] == pytest.approx(rl["achieved"] / rl["peak"])
    assert rl["bound"] == "alu" and rl["unit"] == "Tops/s"
    assert "derived" in bench.alu_peak_source(100, pk, "measured")
    # the algorithmic cost per update: 40 word operations per word plus a
    # quarter Philox call (about 50 operations) per replica quad's word
    assert bench.ALG_OPS["samples32"] == pytest.approx(40 / 32 + 50 / 128)
    kern["sweep"]["timed"] = 0
    assert bench.roofline(kern, w, qisg.QISG_LAYOUT_SAMPLES, 32, 100, pk, steps) is None


class _Done:
    pass


def _summary(lines):
    cs = bench.ClockSampler(0)
    fd, cs.path = tempfile.mkstemp(suffix=".csv")
    with os.fdopen(fd, "w") as f:
        f.write("\n".join(lines) + "\n")
    cs.proc = _Done()          # as after a finished sampler process
    return cs.summary()


def test_clock_summary_median_max_and_reasons():
    ok = "0, {sm}, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, {pc}"
    rows = [ok.format(sm=sm, pc=pc) for sm, pc in ((2070, "Not Active"), (1950, "Active"), (2010, "Not Active"))]
    rows.append("0, [N/A], 2070, 900, 0x0, Not Active, Not Active, Not Active, Not Active")   # skipped
    rows.append("garbage")
    s = _summary(rows)
    assert s["sm_mhz"] == 2010 and s["sm_max_mhz"] == 2070 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    hot = _summary(["0, 1500, 2070, 1000, 0x8, Not Active, Active, Not Active, Not Active"])
    assert hot["reasons"] == ["hw_thermal_slowdown"]
    assert _summary([])["reasons"] == ["no samples"]


def test_reference_and_gpu_arms_share_the_workload_config():
    w = bench.workload()
    cfg = bench.base_config(w)
    assert cfg["workload"] == w.name
    assert bench.updates_per_step(w) == (w.n_samples * w.n_replicas * w.n_slots * w.L * w.L * w.L_tau
                                         * bench.SWEEPS_PER_STEP)
