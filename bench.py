#!/usr/bin/env python
"""Benchmark of the MCQSG hot path (checkerboard Metropolis + PT for the 2D
+-J quantum Ising spin glass in Trotter-Suzuki form) on one GB300.

Workload: 32 disorder samples, L=16, L_tau=256, 4 replicas on a 16-slot PT
ladder (k in [0.2, 0.5], Gamma = 1), PT every sweep, measurements every 10
sweeps; synthetic +-J couplings from Philox.  One step = 10 sweeps (red
half sweep, blue half sweep with energy counting, PT pass) plus one
measurement, i.e. one pass over every step of the path.  The full workload
is 10^4 sweeps = 1000 steps.

Metric: ps per spin update (lower is better), for the batched form (one
launch per half sweep for all samples) next to the per-instance form (one
launch per sample per half sweep), both bit-exact with the oracle.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  Under torchrun every rank runs its own
samples (weak scaling, no collective on the data path); the time is the
maximum over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ps/spin-update, batched vs per-instance (bit-exact); % of INT/HBM roofline"
UNIT = "ps/spin-update"
SWEEPS_PER_STEP = 10
L2_BYTES = 129 * 1024 * 1024


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--forms", default="batched,per_instance")
    p.add_argument("--extras", default="uneven,large,paper,daemon,serving,transfer,tau,overlap",
                   help="other workloads measured beside the headline (empty: none)")
    p.add_argument("--serving-requests", type=int, default=100)
    p.add_argument("--tiles", default="",
                   help="pin the sweep schedule 'red_tile,blue_tile,red_variant,blue_variant'")
    p.add_argument("--autotune", action="store_true",
                   help="tune the sweep schedule on the live state (untimed) instead of the library's default")
    return p.parse_args()


TILES = None    # pinned sweep schedule (from --tiles)
AUTOTUNE = False   # tune the schedule on the live state (--autotune); else the library's default
TUNED = {}      # form -> schedule used


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload():
    from paper_2402_03920_gb300.workloads import PRODUCTION
    return PRODUCTION


def base_config(w) -> dict:
    """The workload's description, shared by both arms' JSON lines."""
    return {"workload": w.name, "L": w.L, "L_tau": w.L_tau, "n_samples": w.n_samples,
            "n_replicas": w.n_replicas, "n_slots": w.n_slots, "k": [w.k_lo, w.k_hi], "gamma": w.gamma,
            "measure_every": w.measure_every}


def updates_per_step(w):
    return w.n_samples * w.n_replicas * w.n_slots * w.L * w.L * w.L_tau * SWEEPS_PER_STEP


def rank_seed(base_seed: int, rank: int) -> int:
    """Weak scaling: every rank simulates its own disorder samples (a seed
    of its own), the same amount of work per rank."""
    return base_seed + 1000 * rank


def job_value(max_ms_over_ranks: float, updates_per_rank: int, world: int) -> float:
    """ps per spin update of the whole job: the slowest rank's time over the
    updates all ranks did."""
    return max_ms_over_ranks * 1e9 / (updates_per_rank * world)


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(rows), "reasons": reasons}


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------
OVERLAP = True   # programmatic dependent launch of the batched form's kernels (the library default)


def make_instance(qisg, w, form, seed):
    ladder = qisg.ladder_linear(w.k_lo, w.k_hi, w.n_slots, w.gamma)
    if form == "per_instance":
        cfg = qisg.Config(w.L, w.L_tau, ladder, w.n_replicas, w.n_samples, seed, word_bits=64,
                          measure_every=w.measure_every, layout=qisg.QISG_LAYOUT_LANES,
                          per_sample_launch=1)
    else:
        cfg = qisg.Config(w.L, w.L_tau, ladder, w.n_replicas, w.n_samples, seed, word_bits=0,
                          measure_every=w.measure_every, layout=batched_layout(qisg))
    inst = qisg.Instance(cfg)
    if form != "per_instance":
        inst.set_launch_overlap(OVERLAP)
    return inst


def batched_layout(qisg):
    return int(os.environ.get("QISG_BENCH_LAYOUT", qisg.QISG_LAYOUT_SAMPLES))


KINDS = (("red", 5), ("blue", 4), ("pt", 1), ("measure", 2), ("permute", 3))


def timed_steps(torch, inst, flush, steps):
    """Device time (ms) of `steps` steps, CUDA events on the library's stream
    (torch's current stream), L2 flushed before each step."""
    evs = []
    for _ in range(steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        inst.sweep(SWEEPS_PER_STEP)
        b.record()
        evs.append((a, b))
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in evs)


def read_profile(inst, names):
    out = {}
    for name, kind in KINDS:
        if name in names:
            ms, nt, nl = inst.profile_read(kind)
            out[name] = {"ms": ms, "timed": nt, "launched": nl,
                         "us_per_launch": 1000.0 * ms / nt if nt else None}
    return out


def time_form(torch, qisg, w, form, steps, warmup, seed):
    """The timed region: `steps` plain steps (no instrumentation).  Then a
    second pass of the same steps with CUDA event pairs around every launch,
    which gives each kernel kind's share of the device time (an event pair
    waits for the work before it, so that pass runs slower than the plain
    one and its absolute durations are not used)."""
    inst = make_instance(qisg, w, form, seed)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device="cuda")
    # the library's default schedule unless one is pinned (--tiles) or tuned
    # on the live state (--autotune, untimed); results do not depend on it.
    # Then realign to the graph cycle of measure_every sweeps
    if TILES is not None:
        inst.set_tiles(TILES[:2], TILES[2:])
    elif AUTOTUNE:
        inst.autotune(6)
    cyc = max(1, w.measure_every)
    inst.sweep((cyc - inst.sweep_count() % cyc) % cyc)
    TUNED[form] = inst.tiles()
    for _ in range(warmup):
        inst.sweep(SWEEPS_PER_STEP)
    inst.sync()
    torch.cuda.synchronize()
    launches0 = inst.launch_count()
    total_ms = timed_steps(torch, inst, flush, steps)
    launches = inst.launch_count() - launches0
    # the share pass runs the PT pass as a launch of its own, so each kernel
    # kind gets its own share (the timed steps run it in the blue pass's last
    # blocks)
    inst.set_pt_in_blue(False)
    inst.profile(True)
    pass_ms = timed_steps(torch, inst, flush, steps)
    kern = read_profile(inst, [k for k, _ in KINDS])
    inst.profile(False)
    inst.set_pt_in_blue(True)
    kern["pass_ms_per_step"] = pass_ms / steps
    layout, wb = inst.layout()
    inst.close()
    del flush
    return total_ms, launches, kern, layout, wb


def e2e_form(torch, qisg, w, form, steps, seed):
    """End to end through the public API with host buffers: couplings and the
    start state are uploaded from pinned host memory, every step reads the
    measurement sums back; wall clock around all of it."""
    from paper_2402_03920_gb300.workloads import random_spins
    n_sys = w.n_samples * w.n_replicas * w.n_slots
    J = torch.from_numpy(random_spins((w.n_samples, w.L * w.L, 2), seed)).pin_memory()
    S = torch.from_numpy(random_spins((w.n_samples, w.n_replicas, w.n_slots, w.L * w.L * w.L_tau),
                                      seed + 1)).pin_memory()
    wa = torch.from_numpy(np.tile(np.arange(w.n_slots, dtype=np.int32),
                                  (w.n_samples, w.n_replicas, 1))).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    inst = make_instance(qisg, w, form, seed)
    inst.set_couplings(J.numpy())
    inst.set_state(S.numpy(), wa.numpy(), 0)
    d2h = 0
    for _ in range(steps):
        inst.sweep(SWEEPS_PER_STEP)
        sA, sB, sq, sq2, nm = inst.measurements()
        d2h += sA.nbytes + sB.nbytes + sq.nbytes + sq2.nbytes
    A, B = inst.energies()
    d2h += A.nbytes + B.nbytes
    wall = time.perf_counter() - t0
    inst.close()
    h2d = J.numel() + S.numel() + 4 * wa.numel()
    ps = wall * 1e12 / (updates_per_step(w) * steps)
    return {"value": ps, "unit": UNIT, "h2d_bytes_per_step": h2d / steps,
            "d2h_bytes_per_step": d2h / steps, "n_sys": n_sys}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


# Algorithmic integer operations per spin update (32-bit operations), per
# packing: the shared-draw SAMPLES kernel spends about 40 word-wide logic
# operations per word plus a quarter Philox call per (replica-group, slot,
# site); the LANES kernel draws one Philox output per update.
ALG_OPS = {"samples32": 40 / 32 + 50 / (4 * 32), "samples64": 80 / 64 + 50 / (4 * 64),
           "lanes": 50 / 4 + 1.5}
INT_LANES_PER_CLK_PER_SM = 128


def kernel_shares(kern):
    """Each kernel kind's share of the device time of the event-pair pass."""
    tot = sum(kern[k]["ms"] for k, _ in KINDS if k in kern)
    return {k: (kern[k]["ms"] / tot if tot > 0 else 0.0) for k, _ in KINDS if k in kern}


def red_threads_per_site(w, wb, t_red, n_sm):
    """Threads per red site of the fused red pass: the library's rule (tile
    1 -> four, 2 -> two, 0 -> four while one thread per site would fill fewer
    than four waves of 2048 threads per SM, else one; 64-bit words at most
    two replicas per thread)."""
    if t_red == 0:
        site_threads = (-(-w.n_samples // wb)) * (-(-w.n_replicas // 4)) * w.L * w.L * (w.L_tau // 2)
        tps = 4 if site_threads < 4 * 2048 * max(1, n_sm) else 1
    else:
        tps = {1: 4, 2: 2}.get(t_red, 1)
    return 2 if (wb == 64 and tps == 1) else tps


def kernel_names(layout, wb, tiles, w, n_sm):
    """The CUDA kernels behind the red and blue kinds for this schedule."""
    from paper_2402_03920_gb300 import qisg
    if layout != qisg.QISG_LAYOUT_SAMPLES:
        return {"red": "lanes_half_sweep_kernel", "blue": "lanes_half_sweep_kernel"}
    (t_red, _t_blue), (_v_red, v_blue) = tiles
    tps = red_threads_per_site(w, wb, t_red, n_sm)
    if wb == 32:
        red = {4: "samples_red_fused_kernel", 2: "samples_red_fusedq_kernel<2>"}.get(tps, "samples_red_fusedq_kernel<4>")
        blue = {0: "samples_sweep4_kernel", 2: "samples_sweep4_kernel<min 4 blocks>"}.get(v_blue, "samples_half_sweep_kernel")
    else:
        red = "samples_red_fusedq_kernel<u64, 1>" if tps == 4 else "samples_red_fusedq_kernel<u64, 2>"
        blue = "samples_half_sweep_kernel"
    return {"red": red, "blue": blue}


KERNEL_SOURCES = ("samples.cu", "qisg_internal.cuh")   # where the SAMPLES sweep kernels are defined


def source_digest() -> str:
    """sha256 (16 hex) of the SAMPLES kernels' sources: DRAM traffic taken
    from an ncu capture is used only while the kernels are the ones
    captured."""
    import hashlib
    hsh = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2402_03920_gb300", "csrc")
    for name in KERNEL_SOURCES:
        with open(os.path.join(csrc, name), "rb") as f:
            hsh.update(f.read())
    return hsh.hexdigest()[:16]


def captured_traffic(kernel: str, workload_name: str):
    """DRAM bytes (read + write) per launch of `kernel` on `workload_name` from
    the ncu summary profiles/dram_traffic.md (rows: | kernel | workload |
    bytes per launch | source digest | ...), or None when absent or taken
    from other kernel sources."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.md")
    try:
        rows = open(path).read().splitlines()
    except OSError:
        return None
    digest = source_digest()
    for row in rows:
        cells = [c.strip().strip("`") for c in row.strip().strip("|").split("|")]
        if len(cells) >= 4 and cells[0] == kernel and cells[1] == workload_name and cells[3] == digest:
            try:
                return float(cells[2])
            except ValueError:
                return None
    return None


def roofline(kern, ups_per_step, key, n_sm, pk, steps, ms_per_step, names, wname):
    """ALU roofline of the red and the blue half-sweep kernels.  A kernel's
    average launch duration is the plain (timed) step time times its share
    of the event-pair pass, over its launches per step, so that launches x
    duration never exceeds the timed step; achieved = algorithmic integer
    operations per launch / that duration.  Returns (dominant, by kernel)."""
    shares = kernel_shares(kern)
    clk = pk.get("sm_max_mhz", 2070.0)
    peak = n_sm * INT_LANES_PER_CLK_PER_SM * clk * 1e6 / 1e12
    hbm_peak = pk.get("hbm_gbs", 6800.0)
    out = {}
    for kind in ("red", "blue"):
        k = kern.get(kind)
        if not k or not k["launched"]:
            continue
        per_step = k["launched"] / steps
        dur_ms = ms_per_step * shares[kind] / per_step
        ups_per_launch = ups_per_step / 2 / per_step   # a half sweep updates the sites of one colour
        ops = ALG_OPS[key] * ups_per_launch
        achieved = ops / (dur_ms * 1e-3) / 1e12
        alg_bytes = 0.25 * ups_per_launch   # one read and one write of each updated spin
        out[kind] = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                     "frac": achieved / peak, "traffic": captured_traffic(names[kind], wname),
                     "kernel": names[kind], "ops_per_update": ALG_OPS[key], "updates_per_launch": ups_per_launch,
                     "avg_launch_us": dur_ms * 1e3, "share": shares[kind], "launches_per_step": per_step,
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "hbm": {"achieved": alg_bytes / (dur_ms * 1e-3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                             "frac": alg_bytes / (dur_ms * 1e-3) / 1e9 / hbm_peak},
                     "timing": "plain step time x share of the event-pair pass / launches per step"}
    if not out:
        return None, {}
    dom = max(out, key=lambda k: out[k]["share"])
    return out[dom], out


def form_roofline(kern, w, layout, wb, n_sm, pk, steps, ms_per_step, tiles):
    from paper_2402_03920_gb300 import qisg
    key = f"samples{wb}" if layout == qisg.QISG_LAYOUT_SAMPLES else "lanes"
    return roofline(kern, updates_per_step(w), key, n_sm, pk, steps, ms_per_step,
                    kernel_names(layout, wb, tiles, w, n_sm), w.name)


def alu_peak_source(n_sm, pk, pk_kind) -> str:
    """How the ALU peak is made: unit counts times the maximum SM clock (the
    clock read from MEASURED_PEAKS.json, or the fallback figure)."""
    return (f"derived: {n_sm} SMs x {INT_LANES_PER_CLK_PER_SM} int32 lanes/clk x "
            f"{pk.get('sm_max_mhz', 2070.0):.0f} MHz (max SM clock, {pk_kind})")


def uneven_batch_entry(qisg, sweeps=100):
    """512 instances, L in {8,12,16,20,24}, L_tau in {64..1024}, 8..32 slots,
    Gamma in [0.8, 1.2], one persistent launch per chunk: ps per update,
    autotuned schedule against the fixed one."""
    import torch
    from paper_2402_03920_gb300.workloads import uneven_batch
    specs = uneven_batch(512, seed=2024, sweeps=sweeps)
    out = {}
    for mode in ("fixed", "autotuned"):
        with qisg.Batch(512, 0) as b:
            for sp in specs:
                b.admit(sp.L, sp.L_tau, qisg.ladder_linear(sp.k_lo, sp.k_hi, sp.n_slots, sp.gamma),
                        sp.n_replicas, sp.seed)
            if mode == "autotuned":
                rows, order = b.autotune(1)
                out["schedule"] = {"tile_rows": rows, "largest_first": bool(order)}
            else:
                b.set_schedule(4, 0)
            b.run(2)
            b.sync()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            b.run(sweeps)
            e1.record()
            b.sync()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
        ups = sum(sp.L * sp.L * sp.L_tau * sp.n_replicas * sp.n_slots for sp in specs) * sweeps
        out[mode] = {"value": ms * 1e9 / ups, "unit": UNIT, "ms": ms, "sweeps": sweeps}
    out["workload"] = "512 uneven instances (L 8..24, L_tau 64..1024, 8..32 slots), one persistent kernel"
    return out


def large_batched_entry(torch, qisg, sweeps=20, persistent_sweeps=2000):
    """1024 samples x 4 replicas x 32 slots, L=24, L_tau=512 (4.8 GB of
    spins, far larger than L2).  Three forms, all bit-exact with each other:
    the per-pass launches at 64-bit and at 32-bit words (graph replay, 20
    sweeps; kernel figures from plain time x each kernel's share of an
    event-pair pass), and the persistent form (one cooperative launch per 64
    sweeps: red | blue | PT with grid barriers, replayed from a graph,
    autotuned red tile and blue tau-walk depth) timed over the workload's full
    2000 sweeps."""
    from paper_2402_03920_gb300.workloads import BATCHED as w
    ladder = qisg.ladder_linear(w.k_lo, w.k_hi, w.n_slots, w.gamma)
    N = w.L * w.L * w.L_tau
    ups_per_sweep = w.n_samples * w.n_replicas * w.n_slots * N
    pk, _ = peaks()
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    alu_peak = n_sm * INT_LANES_PER_CLK_PER_SM * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    hbm_peak = pk.get("hbm_gbs", 6800.0)

    def timed(inst, n):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        inst.sweep(n)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    out = {"workload": w.name}
    for wb in (64, 32):
        cfg = qisg.Config(w.L, w.L_tau, ladder, w.n_replicas, w.n_samples, w.seed, word_bits=wb,
                          layout=qisg.QISG_LAYOUT_SAMPLES)
        with qisg.Instance(cfg) as inst:
            inst.sweep(2)
            inst.sync()
            ms = timed(inst, sweeps)                  # plain: the value
            inst.set_pt_in_blue(False)                # shares: PT as a launch of its own,
            inst.profile(True)
            timed(inst, sweeps)                       # event pairs on every launch
            kern = read_profile(inst, [k for k, _ in KINDS])
            inst.profile(False)
            inst.set_pt_in_blue(True)
            tiles = inst.tiles()
            layout, _ = inst.layout()
        rl, rl_all = roofline(kern, ups_per_sweep, f"samples{wb}", n_sm, pk, sweeps, ms / sweeps,
                              kernel_names(layout, wb, tiles, w, n_sm), w.name)
        out[f"per_pass_u{wb}"] = {"value": ms * 1e9 / (ups_per_sweep * sweeps), "unit": UNIT, "ms": ms,
                                  "sweeps": sweeps, "share": kernel_shares(kern), "roofline": rl,
                                  "roofline_by_kernel": rl_all}
    cfg = qisg.Config(w.L, w.L_tau, ladder, w.n_replicas, w.n_samples, w.seed, word_bits=32,
                      layout=qisg.QISG_LAYOUT_SAMPLES)
    with qisg.Instance(cfg) as inst:
        inst.set_persistent(True)
        if TILES is None:
            inst.autotune(2)
        inst.sweep((64 - inst.sweep_count() % 64) % 64)   # realign to the launch cycle
        inst.sync()
        tiles = inst.tiles()
        ms = timed(inst, persistent_sweeps)
        launches = persistent_sweeps // 64 + (1 if persistent_sweeps % 64 else 0)
    per_sweep_s = ms * 1e-3 / persistent_sweeps
    ops = (ALG_OPS["samples32"] * ups_per_sweep)
    alg_bytes = 0.25 * ups_per_sweep
    out["persistent_u32"] = {
        "value": ms * 1e9 / (ups_per_sweep * persistent_sweeps), "unit": UNIT, "ms": ms,
        "sweeps": persistent_sweeps, "launches": launches,
        "schedule": {"red_tile": tiles[0][0], "blue_tau_sites": tiles[0][1]},
        "roofline": {"bound": "alu", "kernel": "samples_persistent_kernel", "achieved": ops / per_sweep_s / 1e12,
                     "peak": alu_peak, "unit": "Tops/s", "frac": ops / per_sweep_s / 1e12 / alu_peak,
                     "ops_per_update": ALG_OPS["samples32"], "traffic": None,
                     "hbm": {"achieved": alg_bytes / per_sweep_s / 1e9, "peak": hbm_peak, "unit": "GB/s",
                             "frac": alg_bytes / per_sweep_s / 1e9 / hbm_peak, "bytes_per_update": 0.25},
                     "timing": "the whole persistent run (red, blue and PT of every sweep) over its sweeps"}}
    best = min(("per_pass_u64", "per_pass_u32", "persistent_u32"), key=lambda k: out[k]["value"])
    out["value"] = out[best]["value"]
    out["unit"] = UNIT
    out["best_form"] = best
    return out


def paper_shape_entry(torch, qisg, sweeps=10):
    """The lattice shapes of the paper's performance figures (Sec. 4: L=16,
    L_tau=8192 and L=24; 0.466 and 0.735 ps/spin-update on four A100s for one
    system and its k ladder) with equal couplings k_tau = k, run as the
    batched form: 32 samples x 4 replicas x 16 slots, k linear in [0.2, 0.5],
    PT every sweep.  L=24 is run at L_tau=2048 (the paper's production
    L_tau; the figure's L_tau is not given)."""
    out = {}
    n_slots = 16
    ks = np.linspace(0.2, 0.5, n_slots)
    ladder = np.stack([ks, ks], axis=1)   # equal coupling
    for L, Lt in ((16, 8192), (24, 2048)):
        cfg = qisg.Config(L, Lt, ladder, 4, 32, 1, word_bits=32, layout=qisg.QISG_LAYOUT_SAMPLES)
        with qisg.Instance(cfg) as inst:
            inst.autotune(1)
            inst.sweep(2)
            inst.sync()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            inst.sweep(sweeps)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            tiles = inst.tiles()
        ups = 32 * 4 * n_slots * L * L * Lt * sweeps
        out[f"L{L}_Ltau{Lt}"] = {"value": ms * 1e9 / ups, "unit": UNIT, "ms_per_sweep": ms / sweeps,
                                  "schedule": {"tiles": list(tiles[0]), "variants": list(tiles[1])}}
    out["workload"] = ("paper's lattice shapes, equal coupling k_tau = k, 32 samples x 4 replicas x 16 slots, "
                       "k in [0.2, 0.5], PT every sweep")
    out["paper_4xA100_ps"] = {"L16_Ltau8192": 0.466, "L24": 0.735}
    return out


def daemon_entry(torch, qisg, sweeps=10):
    """The paper's own update rule and packing (SITES: 32 tau-sites of one
    system per word, Ito-Kanada daemon bits from Philox + xoroshiro128++ +
    the inverse-cumulative bytes) at the lattice shapes of its performance
    figures, equal couplings: 16 samples x 4 replicas x 16 slots, k linear in
    [0.2, 0.5], PT every sweep.  L=24 at L_tau=2048 as above."""
    out = {}
    n_a, n_r, n_slots = 16, 4, 16
    ks = np.linspace(0.2, 0.5, n_slots)
    ladder = np.stack([ks, ks], axis=1)
    for L, Lt in ((16, 8192), (24, 2048)):
        cfg = qisg.Config(L, Lt, ladder, n_r, n_a, 1, layout=qisg.QISG_LAYOUT_SITES)
        with qisg.Instance(cfg) as inst:
            inst.sweep(3)
            inst.sync()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            inst.sweep(sweeps)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
        ups = n_a * n_r * n_slots * L * L * Lt * sweeps
        out[f"L{L}_Ltau{Lt}"] = {"value": ms * 1e9 / ups, "unit": UNIT, "ms_per_sweep": ms / sweeps}
    out["workload"] = ("SITES packing with the daemon-bit rule, equal coupling k_tau = k, 16 samples x 4 replicas "
                       "x 16 slots, k in [0.2, 0.5], PT every sweep")
    out["paper_4xA100_ps"] = {"L16_Ltau8192": 0.466, "L24": 0.735, "per_A100_L16": 1.864}
    return out


def serving_entry(qisg, n_requests, below_rate=5.0, below_requests=40):
    """Poisson stream of requests (L 8..24, L_tau 32..1024, 8..32 slots,
    100..5000 sweeps, Gamma in [0.8, 1.2]) through the continuous-batching
    server: p50/p99 latency and aggregate ps per update.  Two arrival rates:
    200/s, far above what one GPU serves (about 14/s for this distribution:
    latency is queueing), and 5/s, below it (the loop's own latency:
    admission, shared chunks, retirement)."""
    from paper_2402_03920_gb300.serving import Request, Server
    from paper_2402_03920_gb300.workloads import poisson_requests

    def run(n, rate):
        specs = poisson_requests(n, rate=rate, seed=7)
        reqs = [Request(rid=i, L=sp.L, L_tau=sp.L_tau, n_slots=sp.n_slots, gamma=sp.gamma, sweeps=sp.sweeps,
                        seed=sp.seed, arrival=sp.arrival) for i, sp in enumerate(specs)]
        srv = Server(capacity=512, mem_budget=16 << 30, chunk_sweeps=100)
        try:
            st = srv.serve(reqs, realtime=True)
        finally:
            srv.close()
        out = st.summary()
        out.update({"requests": n, "rate_per_s": rate, "arrival_seed": 7, "unit": UNIT, "value": out["ps_per_update"]})
        return out

    out = run(n_requests, 200.0)
    out["below_capacity"] = run(below_requests, below_rate)
    return out


FP64_NOMINAL_GFLOPS = 1250.0   # GB300 dense FP64 (nominal; MEASURED_PEAKS.json holds no FP64 figure)


def transfer_entry(torch, qisg, reps=50):
    """The exact-diagonalisation code's transfer-matrix product (Sec. 2.2) at
    the largest lattice one GPU holds, L = 5 (even sector, 2^24 doubles):
    time per product, against the FP64 roofline (on this part FP64 issue, not
    HBM, bounds it) with the HBM figure beside it.  Algorithmic work: the
    paper's formulas, 2 multiplies + 1 add per element and round for the
    L^2 - 1 rounds and the parity factor, 1 multiply for each of the two
    Boltzmann factors (77 flops per element at L = 5); bytes: one read of the
    input and one write of the output."""
    L, k = 5, 0.29
    rng = np.random.default_rng(5)
    J = np.where(rng.random((L * L, 2)) < 0.5, 1, -1).astype(np.int8)
    n = 1 << (L * L - 1)
    v = torch.randn(n, dtype=torch.float64, device="cuda")
    out = torch.empty_like(v)
    for _ in range(3):
        qisg.transfer_matvec(v.data_ptr(), out.data_ptr(), L, k, k, J, 1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        qisg.transfer_matvec(v.data_ptr(), out.data_ptr(), L, k, k, J, 1)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    pk, _ = peaks()
    flops = float(n) * (3 * (L * L - 1) + 3 + 2)
    alg = 16.0 * n
    hbm = pk.get("hbm_gbs", 6800.0)
    gflops = flops / (ms * 1e-3) / 1e9
    return {"workload": "EDQSG transfer-matrix product, L=5 even sector (2^24 doubles)", "ms_per_product": ms,
            "unit": "ms", "passes": 3,
            "roofline": {"bound": "fp64", "achieved": gflops, "peak": FP64_NOMINAL_GFLOPS, "unit": "GFLOP/s",
                         "frac": gflops / FP64_NOMINAL_GFLOPS, "flops_per_product": flops, "traffic": None,
                         "peak_source": "nominal GB300 dense FP64 (no measured FP64 peak on this pool)",
                         "hbm": {"achieved": alg / (ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                                 "frac": alg / (ms * 1e-3) / 1e9 / hbm, "algorithmic_bytes": alg}}}


def tau_entry(torch, qisg):
    """Imaginary-time observables (Appendix E.1) of the production workload's
    configurations (32 samples x 4 replicas x 16 slots, L=16, L_tau=256):
    time of one qisg_tau_observables call over all of them."""
    w = workload()
    ladder = qisg.ladder_linear(w.k_lo, w.k_hi, w.n_slots, w.gamma)
    cfg = qisg.Config(w.L, w.L_tau, ladder, w.n_replicas, w.n_samples, w.seed, layout=qisg.QISG_LAYOUT_SAMPLES)
    with qisg.Instance(cfg) as inst:
        inst.sweep(10)
        inst.tau_observables(0, 1)
        t0 = time.perf_counter()
        inst.tau_observables()
        wall = time.perf_counter() - t0
    pairs = w.n_samples * w.n_replicas * w.n_slots * w.L_tau * w.L_tau
    return {"workload": w.name, "s_per_call": wall, "configurations": w.n_samples * w.n_replicas * w.n_slots,
            "ns_per_tau_pair": wall * 1e9 / pairs}


def overlap_entry(torch, qisg, steps, warmup, seed):
    """The batched form with and without programmatic dependent launch of its
    kernels (same schedule, same trajectory): ps per update of each."""
    global OVERLAP
    w = workload()
    out = {}
    for on in (True, False):
        OVERLAP = on
        total_ms, _, _, _, _ = time_form(torch, qisg, w, "batched", steps, warmup, seed)
        out["on" if on else "off"] = total_ms * 1e9 / (updates_per_step(w) * steps)
    OVERLAP = True
    out["unit"] = UNIT
    return out


def cpu_baseline(w, budget_s=15.0):
    """The oracle as it stands on the host cores: nproc samples of the same
    workload, as many sweeps as fit in about budget_s seconds."""
    import oracle
    ncores = os.cpu_count() or 1
    ladder_k, ladder_kt = oracle.ladder_linear(w.k_lo, w.k_hi, w.n_slots, w.gamma)
    n_a = min(ncores, w.n_samples)
    st = oracle.new_state(w.L, w.L_tau, ladder_k, ladder_kt, w.n_replicas, w.seed, 0, n_a)
    t0 = time.perf_counter()
    oracle.run(st, 1, 1, w.measure_every, n_threads=ncores)
    one = time.perf_counter() - t0
    sweeps = max(1, int(budget_s / max(one, 1e-3)))
    t0 = time.perf_counter()
    oracle.run(st, sweeps, 1, w.measure_every, n_threads=ncores)
    wall = time.perf_counter() - t0
    ups = n_a * w.n_replicas * w.n_slots * w.L * w.L * w.L_tau * sweeps
    return {"value": wall * 1e12 / ups, "unit": UNIT, "cores": min(ncores, n_a), "kind": "oracle",
            "sample": f"{n_a} samples x {sweeps} sweeps of the workload ({wall:.1f} s)"}


def kernel_timing(kern, steps):
    return {"how": "second pass of the same steps with event pairs around every launch (pairs serialise "
                   "the graph; the PT pass has its own launch there, while the timed steps run it in the "
                   "blue pass's last blocks); only the shares of its device time are used",
            "share": kernel_shares(kern),
            "pair_us_per_launch": {k: kern[k]["us_per_launch"] for k, _ in KINDS},
            "launches_per_step": {k: kern[k]["launched"] / steps for k, _ in KINDS},
            "pair_pass_ms_per_step": kern["pass_ms_per_step"]}


def run_gpu(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2402_03920_gb300 import qisg
    qisg.load()
    w = workload()
    seed = rank_seed(w.seed, rank)
    forms = [f for f in args.forms.split(",") if f]
    results = {}
    clocks = None
    for form in forms:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        with ClockSampler(local) as cs:
            total_ms, launches, kern, layout, wb = time_form(torch, qisg, w, form, args.steps,
                                                             args.warmup, seed)
        if form == forms[0]:
            clocks = cs.summary()
        if world > 1:
            t = torch.tensor([total_ms], device="cuda", dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            total_ms = float(t.item())
        results[form] = (total_ms, launches, kern, layout, wb)
    if world > 1:
        dist.barrier()
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    ups_total = updates_per_step(w) * args.steps * world
    main = forms[0]
    total_ms, launches, kern, layout, wb = results[main]
    value = job_value(total_ms, updates_per_step(w) * args.steps, world)
    pk, pk_kind = peaks()
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None,
        "dtype": f"u{wb}",
        "data": "synthetic (+-J couplings and start spins from Philox)",
        "config": {**base_config(w), "sweeps_per_step": SWEEPS_PER_STEP, "form": main,
                   "arith": f"u{wb} words of bit-packed spins (1 bit/spin), u32 Philox draws, f64 PT",
                   "layout": "SAMPLES" if layout == qisg.QISG_LAYOUT_SAMPLES else "LANES",
                   "word_bits": wb,
                   "sweep_schedule": {"tiles": list(TUNED.get(main, ((0, 0), (0, 0)))[0]),
                                      "variants": list(TUNED.get(main, ((0, 0), (0, 0)))[1]),
                                      "how": "pinned" if TILES else ("autotuned (untimed)" if AUTOTUNE
                                                                      else "library default")},
                   "l2": "flushed between steps (2x L2 buffer written); lattice fits in L2 within a step"},
        "gpu_launches": launches,
        "clocks": clocks,
        "kernel_timing": kernel_timing(kern, args.steps),
    }
    rl, rl_all = form_roofline(kern, w, layout, wb, n_sm, pk, args.steps, total_ms / args.steps,
                               TUNED.get(main, ((0, 0), (0, 0))))
    if rl is not None:
        rl["peak_source"] = alu_peak_source(n_sm, pk, pk_kind)
    line["roofline"] = rl
    line["roofline_by_kernel"] = rl_all
    if not args.no_e2e:
        line["e2e"] = e2e_form(torch, qisg, w, main, args.steps, seed)
    extras = [x for x in args.extras.split(",") if x]
    if "uneven" in extras and world == 1:
        line["batched_uneven"] = uneven_batch_entry(qisg)
    if "large" in extras and world == 1:
        line["batched_large"] = large_batched_entry(torch, qisg)
    if "paper" in extras and world == 1:
        line["paper_shape"] = paper_shape_entry(torch, qisg)
    if "daemon" in extras and world == 1:
        line["paper_rule"] = daemon_entry(torch, qisg)
    if "serving" in extras and world == 1:
        line["serving"] = serving_entry(qisg, args.serving_requests)
    if "transfer" in extras and world == 1:
        line["transfer"] = transfer_entry(torch, qisg)
    if "tau" in extras and world == 1:
        line["tau_observables"] = tau_entry(torch, qisg)
    if "overlap" in extras and world == 1:
        line["launch_overlap"] = overlap_entry(torch, qisg, args.steps, args.warmup, seed)
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(w)
    # the other forms last, so that a tail of the line keeps them
    for form in forms[1:]:
        tm, ln, kn, lay, wbb = results[form]
        f_rl, _ = form_roofline(kn, w, lay, wbb, n_sm, pk, args.steps, tm / args.steps,
                                TUNED.get(form, ((0, 0), (0, 0))))
        line[form] = {"value": tm * 1e9 / ups_total, "unit": UNIT, "ms_per_step": tm / args.steps,
                      "gpu_launches": ln,
                      "layout": "SAMPLES" if lay == qisg.QISG_LAYOUT_SAMPLES else "LANES",
                      "roofline_frac": f_rl["frac"] if f_rl else None,
                      "vs_value": (tm * 1e9 / ups_total) / value}
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


# --------------------------------------------------------------------------
# reference arm: the oracle on the host cores
# --------------------------------------------------------------------------
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    w = workload()
    ncores = os.cpu_count() or 1
    k, kt = oracle.ladder_linear(w.k_lo, w.k_hi, w.n_slots, w.gamma)
    n_a = min(ncores, w.n_samples)
    st = oracle.new_state(w.L, w.L_tau, k, kt, w.n_replicas, w.seed, 0, n_a)
    for _ in range(args.warmup):
        oracle.run(st, 1, 1, w.measure_every, n_threads=ncores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.run(st, 1, 1, w.measure_every, n_threads=ncores)
    wall = time.perf_counter() - t0
    ups = n_a * w.n_replicas * w.n_slots * w.L * w.L * w.L_tau * args.steps
    value = wall * 1e12 / ups
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": wall * 1e3 / args.steps,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "i8",
            "data": "synthetic (+-J couplings and start spins from Philox)",
            "config": {**base_config(w), "arith": "one int8 spin per byte, u32 Philox draws, f64 PT",
                       "step": f"1 sweep of {n_a} samples (a bounded sample of the workload)"},
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": min(ncores, n_a), "kind": "oracle",
                             "sample": f"{n_a} samples x {args.steps} sweeps"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    global TILES, AUTOTUNE
    args = parse()
    AUTOTUNE = args.autotune
    if args.tiles:
        TILES = [int(v) for v in args.tiles.split(",")]
        if len(TILES) != 4:
            raise SystemExit("--tiles wants red_tile,blue_tile,red_variant,blue_variant")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
