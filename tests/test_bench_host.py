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


def test_roofline_from_plain_time_and_shares():
    """Per-kernel durations come from the plain step time split by each
    kind's share of the event-pair pass, so launches x duration fits in the
    timed step; red and blue are reported apart, the larger share first."""
    from paper_2402_03920_gb300 import qisg
    w = bench.workload()
    steps = 4
    per_kind = bench.SWEEPS_PER_STEP * steps                 # one red and one blue launch per sweep
    # event-pair pass: red 30 us, blue 50 us, PT 20 us per launch (shares 0.3, 0.5, 0.2)
    kern = {"red": {"timed": per_kind, "launched": per_kind, "ms": per_kind * 0.03},
            "blue": {"timed": per_kind, "launched": per_kind, "ms": per_kind * 0.05},
            "pt": {"timed": per_kind, "launched": per_kind, "ms": per_kind * 0.02}}
    pk = {"sm_max_mhz": 2000.0}
    ms_per_step = 0.4                                        # plain: 40 us per sweep
    rl, by = bench.form_roofline(kern, w, qisg.QISG_LAYOUT_SAMPLES, 32, 100, pk, steps, ms_per_step,
                                 ((1, 4), (0, 0)))
    assert rl is by["blue"] and rl["share"] == pytest.approx(0.5)
    assert by["red"]["avg_launch_us"] == pytest.approx(12.0) and rl["avg_launch_us"] == pytest.approx(20.0)
    for k in by.values():   # launches x duration within the plain step
        assert k["launches_per_step"] * k["avg_launch_us"] <= 1000 * ms_per_step + 1e-9
    ups = bench.updates_per_step(w) / bench.SWEEPS_PER_STEP / 2      # one colour's sites per launch
    assert rl["updates_per_launch"] == pytest.approx(ups)
    assert rl["algorithmic_bytes_per_launch"] == pytest.approx(0.25 * ups)
    assert rl["achieved"] == pytest.approx(bench.ALG_OPS["samples32"] * ups / 20e-6 / 1e12)
    assert rl["peak"] == pytest.approx(100 * bench.INT_LANES_PER_CLK_PER_SM * 2000e6 / 1e12)
    assert rl["frac"] == pytest.approx(rl["achieved"] / rl["peak"])
    assert rl["bound"] == "alu" and rl["unit"] == "Tops/s"
    assert rl["kernel"] == "samples_sweep4_kernel" and by["red"]["kernel"] == "samples_red_fused_kernel"
    assert "derived" in bench.alu_peak_source(100, pk, "measured")
    # the algorithmic cost per update: 40 word operations per word plus a
    # quarter Philox call (about 50 operations) per replica quad's word
    assert bench.ALG_OPS["samples32"] == pytest.approx(40 / 32 + 50 / 128)
    kern["red"]["launched"] = kern["blue"]["launched"] = 0
    assert bench.form_roofline(kern, w, qisg.QISG_LAYOUT_SAMPLES, 32, 100, pk, steps, ms_per_step,
                               ((1, 4), (0, 0)))[0] is None


def test_traffic_only_from_matching_kernel_sources(tmp_path, monkeypatch):
    """DRAM traffic from an ncu summary is taken only for the kernel sources
    it was captured on."""
    prof = tmp_path / "profiles"
    prof.mkdir()
    digest = bench.source_digest()
    (prof / "dram_traffic.md").write_text(
        "| kernel | workload | bytes per launch | source digest |\n|---|---|---|---|\n"
        f"| `k1` | wl | 1234.5 | {digest} |\n| `k2` | wl | 99 | 0000000000000000 |\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "source_digest", lambda: digest)
    assert bench.captured_traffic("k1", "wl") == pytest.approx(1234.5)
    assert bench.captured_traffic("k2", "wl") is None
    assert bench.captured_traffic("k1", "other") is None


class _Done:
    pass


def _summary(lines):
    cs = bench.ClockSampler(0)
    fd, cs.path = tempfile.mkstemp(suffix=".csv")
    with os.fdopen(fd, "w") as f:
        f.write("\n".join(lines) + "\n")
    cs.proc = _Done()          # as after a finished sampler process
    return cs.summary()


def test_kernel_names_follow_the_library_schedule_rule():
    """The red tile 0 (the default) means four threads per site while one
    thread per site would fill fewer than four waves of 2048 threads per SM:
    the 32-sample L = 16, L_tau = 256 word set (32768 red sites) takes the
    one-replica kernel on 152 SMs, a 1024-sample L = 24, L_tau = 512 batch
    (32 words x 147456 red sites) the replica-quad kernel."""
    from types import SimpleNamespace
    from paper_2402_03920_gb300 import qisg
    S = qisg.QISG_LAYOUT_SAMPLES
    small = SimpleNamespace(n_samples=32, n_replicas=4, L=16, L_tau=256)
    large = SimpleNamespace(n_samples=1024, n_replicas=4, L=24, L_tau=512)
    assert bench.kernel_names(S, 32, ((0, 0), (0, 0)), small, 152)["red"] == "samples_red_fused_kernel"
    assert bench.kernel_names(S, 32, ((0, 0), (0, 0)), large, 152)["red"] == "samples_red_fusedq_kernel<4>"
    assert bench.kernel_names(S, 32, ((2, 0), (0, 2)), large, 152) == {
        "red": "samples_red_fusedq_kernel<2>", "blue": "samples_sweep4_kernel<min 4 blocks>"}
    assert bench.kernel_names(S, 32, ((8, 4), (0, 1)), small, 152)["blue"] == "samples_half_sweep_kernel"
    assert bench.kernel_names(S, 64, ((0, 0), (0, 0)), small, 152)["red"] == "samples_red_fusedq_kernel<u64, 1>"
    assert bench.kernel_names(S, 64, ((0, 0), (0, 0)), large, 152)["red"] == "samples_red_fusedq_kernel<u64, 2>"
    assert bench.kernel_names(qisg.QISG_LAYOUT_LANES, 64, ((0, 0), (0, 0)), small, 152)["red"] == \
        "lanes_half_sweep_kernel"


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
