"""Benchmark of the SPSTD hot path on GB300: grid-point-steps per second.

Default workload: the 3D anisotropic harmonic oscillator at scale -- 256^3 grid
on [-12, 12]^3, omegas (1.0, 1.3, 1.7), five seeded Gaussians, FP32 fields
with FP64 reductions, the six-stage SUZUKI6 integrator (11 half-stages per
step), 8 probes recorded every step.  One "step" is one full time step of
Eq. 17/18 (every half-stage: FFT second derivatives along x, y, z, the V term
and the axpy) plus the probe record.  The fields (3 x 64 MB) are larger than
the 129 MB L2, so no flush is needed between timed steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs an independent replica (weak scaling; the solves
share no data, so there is no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "aniso_ho_3d_256": dict(precision=32),
    "ho_3d_64_fp32": dict(precision=32),
    "ho_3d_64_fp64": dict(precision=64),
}


def make_problem(name, steps):
    from paper_1805_03155_gb300 import inputs
    if name == "aniso_ho_3d_256":
        return inputs.aniso_ho_3d(steps=steps)
    return inputs.ho_3d(steps=steps)


def max_over_ranks(x, dist, device="cuda"):
    """Largest value of x over all ranks (the job's time is its slowest rank)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(points_per_rank, steps, world, ms_max):
    """Whole-job grid-point-steps/s: every rank's points and steps over the
    slowest rank's time (weak scaling, independent replicas)."""
    return points_per_rank * steps * world / (ms_max * 1e-3)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def tf32_peak_tflops():
    """Dense TF32 tensor peak: the measured bf16 burst figure times the
    nominal TF32 / bf16 ratio (1.1 / 2.25); the nominal 1.1 PFLOP/s without a
    measurement."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        bf16 = json.load(open(p)).get("bf16_tflops")
        if bf16:
            return bf16 * 1.1 / 2.25
    return 1100.0


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the
# 256^3 FP32 kernels from one ncu capture (its summary is kept under profiles/),
# valid while the kernel sources hash to the recorded value.
MEASURED_TRAFFIC = {
    "source_hash": "8fedf3c09ac7918b",
    # per kernel kind and pass schedule; x pass: the separable-potential form
    # (V rebuilt from tables, no V field read); schedule 6: per-warp x tiles
    "aniso_ho_3d_256": {"x_pass": {6: 134.518528e6 + 6.964480e6},
                        "y_pass": {0: 134.246656e6 + 5.592576e6},
                        "z_pass": {0: 134.246912e6 + 5.464576e6}},
}
TRAFFIC_SOURCES = ["paper_1805_03155_gb300/csrc/pass_tmared.cuh", "paper_1805_03155_gb300/csrc/fft_line.cuh",
                   "paper_1805_03155_gb300/csrc/tma.cuh", "paper_1805_03155_gb300/csrc/pass_tma_launch.h"]


def traffic_source_hash():
    """First 16 hex digits of the SHA-256 of the sources of the recorded kernels."""
    import hashlib
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def measured_traffic(workload, kernel, schedule=0):
    """Recorded traffic of a kernel under a pass schedule; None where none was
    recorded or once the kernel sources have changed."""
    if traffic_source_hash() != MEASURED_TRAFFIC["source_hash"]:
        return None
    return MEASURED_TRAFFIC.get(workload, {}).get(kernel, {}).get(schedule)


KIND_AXIS = {"x_pass": 0, "y_pass": 1, "z_pass": 2, "xy_pass": 0}


def algorithmic_bytes(kind, n_total, es, v_separable=False):
    """Compulsory bytes of one launch: the x pass (and the fused x-y pass)
    reads src, V, dst and writes dst; a strided pass reads src, dst and writes
    dst.  With a separable potential the x pass rebuilds V from two tables of
    n_x and n_y n_z values, so its V field read drops out."""
    if kind == "x_pass" and v_separable:
        return 3 * es * n_total
    return (4 if kind in ("x_pass", "xy_pass") else 3) * es * n_total


L2_BYTES = 129 * 2 ** 20
SMS, FP32_LANES, FP64_NOMINAL_TFLOPS, SM_MAX_MHZ = 152, 128, 1.25, 2070.0


def algorithmic_flops(kind, n, n_total):
    """Nominal flops of one launch: 5 log2 N_d + 5 per grid point for each axis
    d it transforms (forward and inverse FFT of paired real lines, the k^2
    multiply and the axpy)."""
    axes = {"x_pass": (0,), "y_pass": (1,), "z_pass": (2,), "xy_pass": (0, 1)}[kind]
    return sum(5 * math.log2(n[a]) + 5 for a in axes) * n_total


def alu_peak_tflops(prec, sm_mhz):
    """Peak of the non-tensor pipes at the sampled SM clock: FP32 = 152 SMs x
    128 FMA lanes x 2 flops x clock; FP64 = the part's nominal 1.25 TFLOP/s
    scaled from its 2070 MHz maximum clock."""
    mhz = sm_mhz or SM_MAX_MHZ
    if prec == 32:
        return SMS * FP32_LANES * 2 * mhz * 1e6 / 1e12
    return FP64_NOMINAL_TFLOPS * mhz / SM_MAX_MHZ


def host_cpu():
    """The host's CPU model and core count (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    import platform
    return {"nproc": os.cpu_count(), "cpu": model, "arch": platform.machine()}


def cpu_baseline(problem, budget_s=20.0):
    """The FP64 oracle on the host: one half-stage (K apply + axpy) on the
    full grid, repeated while the budget lasts, scaled to grid-point-steps/s
    with the integrator's half-stages per step (an extrapolation from that
    sample, not a timed full step)."""
    import oracle

    g = oracle.make_grid(problem.dims, problem.n[: problem.dims], problem.lo[: problem.dims],
                         problem.hi[: problem.dims], problem.hbar, problem.mass)
    c, d = oracle.preset(problem.integrator)
    h = int(np.count_nonzero(c) + np.count_nonzero(d))
    reps, t0 = 0, time.perf_counter()
    R = problem.psiR.copy()
    while True:
        k = oracle.apply_K(problem.psiI, problem.V, g)
        R += c[0] * problem.dt * k
        reps += 1
        if time.perf_counter() - t0 > budget_s / 2 or reps >= 64:
            break
    t = (time.perf_counter() - t0) / reps
    return {"value": problem.n_total / (h * t), "unit": "grid-point-steps/s", "cores": 1, "kind": "oracle",
            "extrapolated": True, "host": host_cpu(),
            "sample": f"{reps} half-stage(s) (K apply + axpy) on the full {problem.n_total}-point grid, "
                      f"{t:.2f} s each, scaled by {h} half-stages per step; single thread, FP64"}


def _oracle_member_step_time(args):
    """Seconds per oracle step of one batch member (a worker of the spawn pool)."""
    import oracle
    from paper_1805_03155_gb300 import inputs  # noqa: F401  (the member arrives pickled)
    p, dt, steps = args
    g = oracle.make_grid(p.dims, p.n[: p.dims], p.lo[: p.dims], p.hi[: p.dims], p.hbar, p.mass)
    c, d = oracle.preset(p.integrator)
    t0 = time.perf_counter()
    oracle.run(p.psiR, p.psiI, p.V, g, c, d, dt, steps, p.probes)
    return (time.perf_counter() - t0) / steps


def batched_cpu_baseline(probs, dts, steps=2):
    """The FP64 oracle on the host for the mixed workload, one instance per
    core: one member of every shape stepped `steps` times in a spawn pool (all
    shapes at once, one process each), each shape's time per step weighted by
    its count in the mix, the total spread over the cores.  Sampled and
    extrapolated to 5000-step solves."""
    import multiprocessing as mp
    by_shape = {}
    for p, dt in zip(probs, dts):
        key = (p.dims, tuple(p.n))
        by_shape.setdefault(key, [p, dt, 0])[2] += 1
    items = list(by_shape.values())
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(min(cores, len(items))) as pool:
        per_step = pool.map(_oracle_member_step_time, [(p, dt, steps) for p, dt, _ in items])
    wall = time.perf_counter() - t0
    cpu_s_per_step = sum(t * cnt for t, (_, _, cnt) in zip(per_step, items))
    pts = sum(p.n_total * cnt for p, _, cnt in items)
    value = pts / (cpu_s_per_step / cores)
    count = sum(cnt for _, _, cnt in items)
    return {"value": value, "unit": "grid-point-steps/s", "cores": cores, "kind": "oracle", "extrapolated": True,
            "solves_per_s_5000_steps": count / (cpu_s_per_step / cores * 5000), "host": host_cpu(),
            "sample": f"one member of each of the {len(items)} shapes, {steps} oracle steps each, in a spawn pool "
                      f"({wall:.1f} s wall); per-step times weighted by the shape counts of the {count}-solve mix "
                      f"and divided over {cores} cores (one instance per core); FP64"}


def accuracy_vs_fp64(cases, local, stream, min_amp=1e-2, sep_bins=4.0, max_bin=0.5):
    """The accuracy gate of the batched and served forms.  Each case is
    (label, problem, dt, steps, probe capacity, FP32 peak energies, FP32
    probe series or None, FP32 state (psi_R, psi_I) or None).  The reference
    is a lone FP64 solve of the same problem, dt and step count on the
    device -- the FP64 path that the parity tests hold to 1e-10 of the FP64
    oracle.
    Energies: the dispersion-corrected peaks of the FP64 probe spectrum that
    are levels the window resolves -- at least min_amp of the largest peak, at
    least sep_bins Hann bins (2 pi hbar / (M dt), M samples) from every other
    peak and from zero, in a window whose bin is at most max_bin (the levels of
    these wells and oscillators lie about one energy unit apart) -- each
    against the nearest FP32 peak; None where the window resolves no level.
    State: relative L2 distance of the FP32 fields from the FP64 ones.
    Series: the largest deviation of the FP32 probe series, relative to the
    FP64 series' largest value (probes may sit where the state is small)."""
    from paper_1805_03155_gb300 import spstd
    out = {}
    kw = dict(max_peaks=16, thresh=1e-3, phase_correct=True)
    for label, p, dt, steps, cap, E32, z32, st32 in cases:
        ref = spstd.solver_for(p, precision=64, probe_capacity=cap, stream=stream, device=local, dt=dt)
        ref.spstd_step(steps)
        E64, A64 = ref.spstd_spectrum(-1, **kw)
        z64 = np.array([ref.spstd_probe(q) for q in range(len(p.probes))]) if z32 is not None else None
        st64 = ref.spstd_get_state() if st32 is not None else None
        ref.close()
        M = min(steps, cap)
        bin_e = 2 * np.pi * p.hbar / (M * dt)
        resolved = [e for e, a in zip(E64, A64)
                    if bin_e <= max_bin and a >= min_amp * A64.max() and e >= sep_bins * bin_e
                    and all(abs(e - f) >= sep_bins * bin_e for f in E64 if f != e)]
        err = (float(max(np.min(np.abs(np.asarray(E32) - e)) / abs(e) for e in resolved))
               if resolved and len(E32) else None)
        ser = float(np.max(np.abs(z32 - z64)) / np.max(np.abs(z64))) if z64 is not None else None
        sterr = None
        if st64 is not None:
            num = np.sum((st32[0] - st64[0]) ** 2 + (st32[1] - st64[1]) ** 2)
            sterr = float(np.sqrt(num / np.sum(st64[0] ** 2 + st64[1] ** 2)))
        out[label] = {"energy_rel_err": err, "resolved_peaks": len(resolved), "bin": float(bin_e),
                      "state_rel_l2": sterr, "series_rel_err": ser, "steps": int(steps)}
    return out


def accuracy_batch(probs, local, stream, steps=10000, precision=32):
    """One member of every shape of the mix, stepped `steps` times in a batch
    of their own (twice the workload's 5000, so that the window of most
    members resolves their levels), against lone FP64 solves
    (accuracy_vs_fp64)."""
    from paper_1805_03155_gb300 import spstd
    seen, sample = set(), []
    for p in probs:
        key = "%dd:%s" % (p.dims, "x".join(str(v) for v in p.n[: p.dims]))
        if key not in seen:
            seen.add(key)
            sample.append((key, p))
    solvers = [spstd.solver_for(p, precision=precision, probe_capacity=steps, stream=stream, device=local,
                                merge=False) for _, p in sample]
    b = spstd.Batch(len(solvers) + 1, device=local, stream=stream)
    for s in solvers:
        b.spstd_batch_add(s)
    b.spstd_batch_step(steps)
    b.spstd_batch_sync()
    b.close()
    kw = dict(max_peaks=16, thresh=1e-3, phase_correct=True)
    cases = []
    for (key, p), s in zip(sample, solvers):
        z = np.array([s.spstd_probe(q) for q in range(len(p.probes))])
        cases.append((key, p, s.spstd_get_dt(), steps, steps, s.spstd_spectrum(-1, **kw)[0], z,
                      s.spstd_get_state()))
    for s in solvers:
        s.close()
    return accuracy_vs_fp64(cases, local, stream)


def gate_summary(acc):
    e = [v["energy_rel_err"] for v in acc.values() if v["energy_rel_err"] is not None]
    z = [v["series_rel_err"] for v in acc.values() if v["series_rel_err"] is not None]
    st = [v["state_rel_l2"] for v in acc.values() if v["state_rel_l2"] is not None]
    return {"energy_rel_err_max": max(e) if e else None,
            "shapes_with_resolved_levels": len(e), "shapes": len(acc),
            "state_rel_l2_max": max(st) if st else None,
            "series_rel_err_max": max(z) if z else None}


def batched_vs_plain(count=512, steps=800, plain_steps=40, precision=32, local=0, plain=True, check=True,
                     general_v=True, schedules=None):
    """The mixed 512-solve workload (1D wells 128..8192, 2D oscillators
    64^2..512^2, 3D oscillators 32^3, 48^3, 64^3 and 96^3; FP32 fields, FP64
    reductions, FR4): every member stepped through one batch (graph-replayed
    chunks, 1D members resident) vs the same members stepped one after another
    with spstd_step on one stream (plain).  Device-resident inputs; CUDA-event
    time on the batch stream.  The batch is timed over `steps` steps (after a
    warm-up of as many, which captures its graph), the plain leg over
    `plain_steps` steps per member; solves/s is extrapolated to the 5000-step
    solves of the workload.  The members' potentials separate (harmonic wells),
    so every batched x pass rebuilds V from two tables; `general_v` times the
    batch again with potentials that do not.  Accuracy gate: one member of every
    shape, batched for 10000 steps, against lone FP64 solves (accuracy_batch)."""
    import torch
    from paper_1805_03155_gb300 import inputs, spstd

    probs = inputs.batch_mix(count, steps=steps)
    stream = torch.cuda.current_stream(local)
    cap = 2 * steps + 8
    # both legs run every half-stage of every step (batches do not fuse step
    # boundaries), so they do the same arithmetic
    solvers = [spstd.solver_for(p, precision=precision, probe_capacity=cap, stream=stream,
                                device=local, merge=False) for p in probs]
    pts = sum(p.n_total for p in probs)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    # plain: one member after another (warm-up captures each member's graph)
    plain_ms, plain_launches = float("nan"), 0
    if plain:
        for s in solvers:
            s.spstd_step(plain_steps)
        torch.cuda.synchronize()
        ev[0].record(stream)
        for s in solvers:
            s.spstd_step(plain_steps)
        ev[1].record(stream)
        torch.cuda.synchronize()
        plain_ms = ev[0].elapsed_time(ev[1])
        plain_launches = sum(s.spstd_launch_count(plain_steps) for s in solvers)
        # back to the initial states (and empty probe rings) for the batch
        for p, s in zip(probs, solvers):
            s.spstd_set_state(p.psiR, p.psiI)
        torch.cuda.synchronize()
    # batched
    b = spstd.Batch(count + 1, device=local, stream=stream)
    for s in solvers:
        b.spstd_batch_add(s)

    def timed_batch():
        ev[2].record(stream)
        b.spstd_batch_step(steps)
        ev[3].record(stream)
        torch.cuda.synchronize()
        return ev[2].elapsed_time(ev[3])

    default_ms = timed_batch()  # also the warm-up: captures the batch graph
    # autotuned schedules per member shape (timed on the members' scratch fields)
    t_tune = time.perf_counter()
    if schedules:
        # fixed schedules (profiler runs, whose serialised timings would mislead the tuner)
        for key, sched in schedules.items():
            dims, sizes = key.split(":")
            b.spstd_batch_set_schedule(precision, int(dims[0]), [int(v) for v in sizes.split("x")], sched)
    else:
        b.spstd_batch_tune(reps=3)
    tune_s = time.perf_counter() - t_tune
    shapes = sorted({(p.dims, tuple(p.n)) for p in probs if p.dims > 1})
    tuned = {"%dd:%s" % (d, "x".join(str(v) for v in n[:d])): b.spstd_batch_get_schedule(precision, d, n)[:d]
             for d, n in shapes}
    batch_ms = timed_batch()
    launches = b.spstd_batch_launch_count(steps)
    b.close()
    norms = []
    for s in solvers[:: max(1, count // 16)]:
        try:
            norms.append(s.spstd_energy_norm()[0])
        except spstd.SpstdError as e:
            norms.append(getattr(e, "norm", float("nan")))
    dts = [s.spstd_get_dt() for s in solvers]
    # the same mix with potentials that do not separate (V + 0.01 x y on the
    # 2D and 3D members; 1D members are unchanged): every x pass reads its
    # member's V field (16 B/pt) instead of rebuilding V from two tables
    gv = None
    if general_v:
        for p, s in zip(probs, solvers):
            if p.dims > 1:
                x, y = p.coords()[:2]
                V = p.V.reshape(-1, len(y), len(x)) + 0.01 * y[None, :, None] * x[None, None, :]
                s.spstd_set_potential(V.ravel())
                s.spstd_set_state(p.psiR, p.psiI)
        sep_left = sum(s.spstd_potential_separable() for p, s in zip(probs, solvers) if p.dims > 1)
        b = spstd.Batch(count + 1, device=local, stream=stream)
        for s in solvers:
            b.spstd_batch_add(s)
        gv_steps = max(1, steps // 4)
        b.spstd_batch_step(gv_steps)  # warm-up: captures the batch graph
        b.spstd_batch_tune(reps=3)
        ev[2].record(stream)
        b.spstd_batch_step(gv_steps)
        ev[3].record(stream)
        torch.cuda.synchronize()
        gv_ms = ev[2].elapsed_time(ev[3])
        b.close()
        gv = {"value": pts * gv_steps / (gv_ms * 1e-3), "ms": gv_ms, "steps_timed": gv_steps,
              "separable_members_left": int(sep_left),
              "what": "the same members with V + 0.01 x y on the 2D and 3D ones, so that no potential "
                      "separates and every batched x pass reads the V field"}
    for s in solvers:
        s.close()
    acc = accuracy_batch(probs, local, stream) if check else {}
    return {
        "workload": f"batch_mix_{count}",
        "members": count,
        "grid_points": pts,
        "shapes3d": sorted({p.n[0] for p in probs if p.dims == 3}),
        "steps": steps,
        "batched": {"value": pts * steps / (batch_ms * 1e-3), "ms": batch_ms, "steps_timed": steps,
                    "solves_per_s_5000_steps": count / (batch_ms * 1e-3 * 5000 / steps),
                    "extrapolated_from": f"{steps} steps of every member in {batch_ms:.0f} ms",
                    "gpu_launches": launches, "schedules": tuned, "tune_s": tune_s,
                    "default_schedule_ms": default_ms,
                    "default_schedule_value": pts * steps / (default_ms * 1e-3),
                    "v_separable": "x passes rebuild V from separable tables (all 2D/3D members)"},
        "batched_general_v": gv,
        "plain": {"value": pts * plain_steps / (plain_ms * 1e-3), "ms": plain_ms, "steps_timed": plain_steps,
                  "solves_per_s_5000_steps": count / (plain_ms * 1e-3 * 5000 / plain_steps),
                  "extrapolated_from": f"{plain_steps} steps of every member, one after another, in {plain_ms:.0f} ms",
                  "gpu_launches": plain_launches},
        "speedup": (plain_ms / plain_steps) / (batch_ms / steps),
        "unit": "grid-point-steps/s",
        "norm_drift_max": float(max(abs(n - 1.0) for n in norms)),
        **(gate_summary(acc) if acc else {}),
        "accuracy": acc,
        "accuracy_check": "one member per shape batched for 10000 steps vs a lone FP64 device solve of the same "
                          "member (the FP64 path matches the FP64 oracle to 1e-10 in the parity tests): the "
                          "dispersion-corrected probe-spectrum energies of the levels the window resolves (peaks "
                          ">= 1e-2 of the largest, >= 4 Hann bins from their neighbours, bin <= 0.5; None where "
                          "the window resolves no level: fine grids take small dt), the state's relative L2 "
                          "distance, and the probe series",
        "_dts": dts,
        "_probs": probs,
    }


def serving(rate=200.0, duration=1.0, steps=1000, chunk=500, precision=32, seed=9, local=0, hbm_cap=150e9,
            tune=True, check=True):
    """Poisson arrivals (rate/s for `duration` s) of solves drawn from the
    mixed workload plus 128^3 oscillators, each `steps` steps, served by
    continuous batching in `chunk`-step rounds under an HBM cap; p50/p99
    latency from arrival to retirement.  Compared with serving the same
    requests one at a time (plain: each solved alone, in arrival order)."""
    import torch
    from paper_1805_03155_gb300 import inputs, serve, spstd

    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=int(rate * duration * 3) + 8)
    t_arr = np.cumsum(gaps)
    t_arr = t_arr[t_arr < duration]
    n = len(t_arr)
    mix = inputs.batch_mix(max(n, 3), seed=seed, steps=steps)
    probs = []
    for i in range(n):
        if i % 10 == 9:
            p = inputs.gaussian_problem((128, 128, 128), (-8.0,) * 3, (8.0,) * 3, seed=seed * 7 + i,
                                        integrator="FR4", dt=0.0, steps=steps, n_probe=2)
        else:
            p = mix[i]
        probs.append(p)
    srv = serve.Server(hbm_cap_bytes=hbm_cap, max_slots=n + 1, chunk_steps=chunk, precision=precision,
                       device=local, spectrum=True, keep_series=check, keep_state=check, tune=tune)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for p, ta in zip(probs, t_arr):
        srv.submit(p, steps, arrival=t0 + ta)
    srv.run()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    lat = srv.latencies()
    pts = sum(p.n_total for p in probs) * steps
    chunks = srv.chunks
    diverged = sum(1 for r in srv.done if r.result.get("status") != "ok")
    # accuracy gate: the first finished request of every shape against a lone FP64 solve
    seen, cases = set(), []
    for r in sorted(srv.done, key=lambda r: r.rid):
        p = r.problem
        key = "%dd:%s" % (p.dims, "x".join(str(v) for v in p.n[: p.dims]))
        if key in seen or "E" not in r.result:
            continue
        seen.add(key)
        cases.append((key, p, r.result["dt"], r.steps, max(1, r.steps), r.result["E"], r.result.get("series"),
                      r.result.get("state")))
    srv.close()
    acc = accuracy_vs_fp64(cases, local, torch.cuda.current_stream(local)) if check else {}
    # plain: the same requests one at a time, each stepped alone
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    plain_lat = []
    for p, ta in zip(probs, t_arr):
        now = time.perf_counter() - t1
        if now < ta:
            time.sleep(ta - now)
        s = spstd.solver_for(p, precision=precision, probe_capacity=steps, device=local)
        s.spstd_step(steps)
        s.spstd_energy_norm()
        s.close()
        plain_lat.append(time.perf_counter() - t1 - ta)
    plain_wall = time.perf_counter() - t1
    plain_lat = np.array(plain_lat)
    return {
        "workload": f"serve_poisson_{int(rate)}_per_s",
        "requests": n, "steps_per_request": steps, "chunk_steps": chunk, "hbm_cap_bytes": hbm_cap,
        "batched": {"solves_per_s": n / wall, "grid_point_steps_per_s": pts / wall,
                    "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                    "wall_s": wall, "chunks": chunks},
        "plain": {"solves_per_s": n / plain_wall, "grid_point_steps_per_s": pts / plain_wall,
                  "p50_s": float(np.percentile(plain_lat, 50)), "p99_s": float(np.percentile(plain_lat, 99)),
                  "wall_s": plain_wall},
        "diverged_requests": diverged,
        **(gate_summary(acc) if acc else {}),
        "accuracy": acc,
        "accuracy_check": "the first finished request of every shape vs a lone FP64 device solve of the same "
                          "request: resolved level energies, state and probe series, as in batched_vs_plain (a "
                          "1000-step request resolves the levels of few shapes)",
        "latency_note": "wall clock from arrival to retirement, host-side admission included; the arrival rate "
                        "exceeds the service rate, so the latency is mostly queueing",
    }


def general_v_leg(steps, warmup, peak, local=0):
    """The same 256^3 workload with a potential that does not separate: the
    oscillator plus 0.01 x y.  Eq. 16's V term then needs the V field at every
    point, so the x pass reads it (16 B/pt) instead of rebuilding V from two
    tables.  Timed like the main line (one call of `steps` steps, CUDA events
    on the solver's stream)."""
    import dataclasses

    import torch
    from paper_1805_03155_gb300 import inputs, spstd

    p = inputs.aniso_ho_3d(steps=steps)
    x, y, _ = p.coords()
    nx, ny, nz = p.n
    V = (p.V.reshape(nz, ny, nx) + 0.01 * y[None, :, None] * x[None, None, :]).ravel()
    p = dataclasses.replace(p, V=V)
    stream = torch.cuda.Stream(device=local)
    s = spstd.solver_for(p, precision=32, probe_capacity=warmup + steps + 8, stream=stream, device=local)
    sep = s.spstd_potential_separable()
    s.spstd_tune(reps=10)  # as the main line: the tuner's pass schedules
    schedules = [s.spstd_get_schedule(a) for a in range(3)]
    s.spstd_step(warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.spstd_step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    prof = s.spstd_profile_steps(4)
    s.close()
    N = p.n_total
    xms = prof["x_pass"][0] / max(1, prof["x_pass"][1])
    hs = (steps * 10 + 1) / steps  # SUZUKI6 with fused step boundaries: 10 half-stages a step within a call
    half_ms = ms / steps / hs
    return {"workload": "aniso_ho_3d_256 with V + 0.01 x y (not separable)", "v_separable": sep,
            "schedules": schedules,
            "value": N * steps / (ms * 1e-3), "unit": "grid-point-steps/s", "ms_per_step": ms / steps,
            "steps": steps, "x_pass_ms": xms, "x_pass_frac": 16 * N / (xms * 1e-3) / 1e9 / peak,
            "half_stage_ms_in_graph": half_ms,
            "half_stage_frac": 16 * N / (half_ms * 1e-3) / 1e9 / peak,
            "what": "x pass fraction: its 16 B/pt (src, V, dst read, dst written) over its event-timed launch; "
                    "half-stage fraction: 16 B/pt over the in-graph step time per applied half-stage"}


def next_rows_leg(peak, sm_mhz, local=0):
    """The rows beyond the hot path, each timed once on a grid larger than L2
    where its bound is HBM (CUDA events around spstd_step on the solver's
    stream, after a warm-up call), with the roofline each is held to:
    * four-step long x lines (2D FP32, 65536 x 256, FR4): 16 B/pt per applied
      half-stage (the measurement unit) against the copy peak; the kernels
      move about 36 B/pt for the paired x lines plus 12 B/pt for y;
    * Dirichlet walls (3D FP32 128^3, DST on every axis, FR4): dense n x n
      line operators as tensor-core products (tcgen05 TF32, 3xTF32: 6n flops
      per point per axis) -- the passes' bytes (16 B/pt x with V, 12 B/pt y
      and z) against the copy peak, the flops against the TF32 peak (the
      measured bf16 peak x 1.1/2.25, the nominal ratio); and the same steps
      with the CUDA-core dense pass (schedule 4, 2n FP32 flops per point per
      axis) for comparison;
    * the RK4 comparison scheme (3D FP32 256^3): 8 H applications a step, the
      unit's 16 B/pt each;
    * eigenstate accumulation (3D FP32 256^3, FR4, 2 target energies): the
      extra time per step over plain unmerged steps, against the 72 B/pt the
      accumulator kernel moves (psi_R, psi_I read; two FP64 complex
      accumulators read and written)."""
    import torch
    from paper_1805_03155_gb300 import inputs, spstd

    stream = torch.cuda.Stream(device=local)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(s, steps):
        s.spstd_step(steps)  # warm-up (captures graphs)
        torch.cuda.synchronize()
        e0.record(stream)
        s.spstd_step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    out = {}
    h_applied = (10 * 6 + 1) / 10  # FR4 with fused step boundaries, 10 steps a call
    # long x lines
    p = inputs.gaussian_problem((65536, 256), (-64.0, -8.0), (64.0, 8.0), seed=21, dt=0.0, steps=10, n_probe=2)
    s = spstd.solver_for(p, precision=32, probe_capacity=64, stream=stream, device=local)
    ms = timed(s, 10)
    s.close()
    out["long_x_65536x256_fp32"] = {"ms_per_step": ms, "value": p.n_total / (ms * 1e-3), "bound": "hbm",
                                    "half_stage_frac": 16 * p.n_total / (ms / h_applied * 1e-3) / 1e9 / peak,
                                    "moved_frac": 48 * p.n_total / (ms / h_applied * 1e-3) / 1e9 / peak}
    # walls
    p = inputs.gaussian_problem((128, 128, 128), steps=10, seed=22, dt=0.0, n_probe=2, bc=(1, 1, 1))
    s = spstd.solver_for(p, precision=32, probe_capacity=64, stream=stream, device=local)
    ms = timed(s, 10)
    prof = s.spstd_profile_steps(2)
    pass_ms = sum(prof[k][0] for k in ("x_pass", "y_pass", "z_pass")) / max(1, sum(prof[k][1] for k in (
        "x_pass", "y_pass", "z_pass")))
    for a in range(3):
        s.spstd_set_schedule(a, 4)
    core_ms = timed(s, 10)
    s.close()
    tf32_peak = tf32_peak_tflops()
    row = {"ms_per_step": ms, "value": p.n_total / (ms * 1e-3), "bound": "hbm", "dense_pass_ms": pass_ms,
           "pass_frac": (40 / 3) * p.n_total / (pass_ms * 1e-3) / 1e9 / peak,
           "tensor_tflops": 6 * 128 * p.n_total / (pass_ms * 1e-3) / 1e12,
           "cuda_core_ms_per_step": core_ms,
           "cuda_core_alu_frac": (3 * 2 * 128 + 2) * p.n_total * h_applied / (core_ms * 1e-3) / 1e12 /
                                 alu_peak_tflops(32, sm_mhz)}
    row["tensor_frac"] = row["tensor_tflops"] / tf32_peak
    row["what"] = ("dense passes on the tensor cores (3 TF32 MMAs per product): pass_frac = their 13.3 B/pt "
                   "average over the event-timed pass, tensor_frac = 6n flops/pt over the TF32 peak "
                   f"({tf32_peak:.0f} TFLOP/s: measured bf16 x 1.1/2.25); the 25 MB grid stays in L2")
    out["walls_dirichlet_128^3_fp32"] = row
    # RK4
    p = inputs.gaussian_problem((256, 256, 256), (-12.0,) * 3, (12.0,) * 3, seed=23, integrator="RK4", dt=0.0,
                                steps=10, n_probe=2)
    s = spstd.solver_for(p, precision=32, probe_capacity=64, stream=stream, device=local, norm_drift_limit=0.0)
    ms = timed(s, 10)
    s.close()
    out["rk4_256^3_fp32"] = {"ms_per_step": ms, "value": p.n_total / (ms * 1e-3), "bound": "hbm",
                             "step_frac": 16 * 8 * p.n_total / (ms * 1e-3) / 1e9 / peak}
    # eigenstate accumulation
    p = inputs.gaussian_problem((256, 256, 256), (-12.0,) * 3, (12.0,) * 3, seed=24, dt=0.0, steps=10, n_probe=2)
    s = spstd.solver_for(p, precision=32, probe_capacity=64, stream=stream, device=local, merge=False,
                         max_eigenstates=2)
    plain = timed(s, 10)
    s.spstd_eigenstates_begin([1.5, 2.5], 1 << 20)
    acc = timed(s, 10)
    s.spstd_eigenstates_end()
    s.close()
    extra = max(acc - plain, 1e-9)
    out["eigen_accum_256^3_fp32_2_targets"] = {"ms_per_step": acc, "plain_ms_per_step": plain,
                                               "extra_ms_per_step": acc - plain, "bound": "hbm",
                                               "accum_frac": 72 * p.n_total / (extra * 1e-3) / 1e9 / peak}
    return out


def run_reference(args):
    """The oracle as it stands, on the host cores, same metric and workload.
    Each step is a bounded sample of one half-stage: the oracle's spectral
    second derivative along x, y and z over 256 full-length lines per axis
    (the per-line work of a full-grid K apply), plus the V term and the axpy,
    scaled to grid-point-steps/s by the half-stages per step."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    problem = make_problem(args.workload, 1)
    c, d = oracle.preset(problem.integrator)
    h = int(np.count_nonzero(c) + np.count_nonzero(d))
    n = problem.n[0]
    lines = 256 if n >= 16 else n * n
    side = int(round(np.sqrt(lines)))
    lo, hi = problem.lo[:3], problem.hi[:3]
    grids = []
    for ax in range(3):
        shape = [side, side, side]
        shape[ax] = problem.n[ax]
        grids.append((ax, oracle.make_grid(3, shape, lo, hi, problem.hbar, problem.mass)))
    S = side * side * n
    rng = np.random.default_rng(0)
    src = rng.standard_normal(S)
    V = rng.standard_normal(S)
    dst = np.zeros(S)

    def sample():
        acc = (V / problem.hbar) * src
        for ax, g in grids:
            acc += problem.hbar / (2 * problem.mass) * oracle.laplacian_axis(src, g, ax)
        dst[:] += c[0] * problem.dt * acc

    for _ in range(args.warmup):
        sample()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sample()
    t = time.perf_counter() - t0
    value = S * args.steps / (h * t)
    what = (f"each step: the oracle's x, y and z line transforms over {side * side} full-length lines per axis "
            f"({S} grid points, the per-point work of one half-stage) plus the V term and axpy, scaled by "
            f"{h} half-stages per step; single thread, FP64; the value is extrapolated from this sample to the "
            f"full {problem.n_total}-point grid")
    out = {"impl": "reference", "metric": "grid-point-steps/s", "value": value, "unit": "grid-point-steps/s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * t / args.steps,
           "ms_per_step_is": f"the measured time of one timed sample step ({S} points, one half-stage's work); a "
                             f"full {problem.n_total}-point step of {h} half-stages would take "
                             f"{1e3 * t * h * (problem.n_total / S) / args.steps:.0f} ms (extrapolated)",
           "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload, "grid": list(problem.n), "integrator": problem.integrator},
           "cpu_baseline": {"value": value, "unit": "grid-point-steps/s", "cores": 1, "kind": "oracle",
                            "extrapolated": True, "host": host_cpu(), "sample": what},
           "e2e": {"value": value, "unit": "grid-point-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="aniso_ho_3d_256", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-vs-plain and serving legs")
    ap.add_argument("--no-general-v", action="store_true", help="skip the leg with a potential that does not separate")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the default pass schedules (no autotuning launches; for profiler launch lists)")
    ap.add_argument("--schedules", default=None,
                    help="comma-separated pass schedule per axis to use instead of autotuning (for profiler runs, "
                         "whose timings would mislead the tuner), e.g. 6,0,0")
    ap.add_argument("--batch-schedules", default=None,
                    help='batch pass schedules per member shape instead of the batch autotuner (for profiler '
                         'runs), as JSON, e.g. {"3d:96x96x96": [6, 0, 0]}')
    ap.add_argument("--batch-steps", type=int, default=800,
                    help="timed steps of the batched leg (a short run for profiler launch lists)")
    ap.add_argument("--next-rows-only", action="store_true",
                    help="run only the rows beyond the hot path (long lines, walls, RK4, eigenstates) and print "
                         "their numbers (for profiler runs of their kernels)")
    ap.add_argument("--batch-only", action="store_true",
                    help="run only the batched leg of the 512-solve mix and print its numbers (for profiler "
                         "launch lists of the batched passes)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)
    if args.next_rows_only:
        import torch
        torch.cuda.set_device(0)
        from paper_1805_03155_gb300 import build
        if not os.path.exists(build.LIB):
            build.build()
        print(json.dumps({"next_rows_only": True, "next_rows": next_rows_leg(measured_peaks()[0], None)}))
        return 0
    if args.batch_only:
        import torch
        torch.cuda.set_device(0)
        r = batched_vs_plain(steps=args.batch_steps, plain=False, check=False, general_v=not args.no_general_v,
                             schedules=json.loads(args.batch_schedules) if args.batch_schedules else None)
        print(json.dumps({"batch_only": True, **{k: r[k] for k in ("workload", "members", "grid_points", "steps",
                                                                    "shapes3d", "batched", "batched_general_v",
                                                                    "unit")}}))
        return 0

    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1805_03155_gb300 import build, spstd
    if rank == 0 or not os.path.exists(build.LIB):
        build.build()
    if dist is not None:
        dist.barrier()

    wl = WORKLOADS[args.workload]
    prec = wl["precision"]
    es = 4 if prec == 32 else 8
    problem = make_problem(args.workload, args.steps)
    total_steps = args.warmup + args.steps + 8
    stream = torch.cuda.Stream(device=local)
    s = spstd.solver_for(problem, precision=prec, probe_capacity=total_steps, stream=stream, device=local)
    N = problem.n_total
    # autotune the pass schedules on this grid (outside the timed region)
    tune_ms = np.full((3, spstd.SCHEDULES), -1.0)
    if args.schedules:
        for a, v in enumerate(int(x) for x in args.schedules.split(",")):
            s.spstd_set_schedule(a, v)
    elif not args.no_tune:
        tune_ms = s.spstd_tune(reps=10)
    schedules = [s.spstd_get_schedule(a) for a in range(problem.dims)]
    xy_fused = s.spstd_get_xy_fusion()
    v_sep = s.spstd_potential_separable()

    # ---- timed region: K steps, device resident -------------------------------
    # the clock sampler starts first (nvidia-smi needs a moment), then the
    # warm-up steps (they also capture the step graph) run right before the
    # timed call, so that the GPU does not idle between them
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    s.spstd_step(args.warmup)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    ev0.record(stream)
    s.spstd_step(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    launches = s.spstd_launch_count(args.steps)
    ms = max_over_ranks(ms, dist)
    value = job_value(N, args.steps, ws, ms)

    # ---- per-kernel device times (event pair around each launch) ------------
    prof_steps = max(2, min(8, args.steps))
    prof = s.spstd_profile_steps(prof_steps)
    kinds = {k: v for k, v in prof.items() if v[1] > 0}
    dom = max(kinds, key=lambda k: kinds[k][0])
    dom_ms = kinds[dom][0] / kinds[dom][1]
    peak, peak_src = measured_peaks()
    abytes = algorithmic_bytes(dom, N, es, v_sep)
    achieved = abytes / (dom_ms * 1e-3) / 1e9
    step_bytes = sum(algorithmic_bytes(k, N, es, v_sep) * kinds[k][1] for k in ("x_pass", "y_pass", "z_pass", "xy_pass")
                     if k in kinds) / prof_steps
    half_stages = (kinds.get("x_pass", (0, 0))[1] + kinds.get("xy_pass", (0, 0))[1]) / prof_steps

    # ---- end to end through the C ABI with pinned host buffers --------------
    pin_r = torch.empty(N, dtype=torch.float64, pin_memory=True)
    pin_i = torch.empty(N, dtype=torch.float64, pin_memory=True)
    pin_r.numpy()[:] = problem.psiR
    pin_i.numpy()[:] = problem.psiI
    hr, hi_ = pin_r.numpy(), pin_i.numpy()
    out_r = torch.empty(N, dtype=torch.float64, pin_memory=True).numpy()
    out_i = torch.empty(N, dtype=torch.float64, pin_memory=True).numpy()
    probe_bytes = 16 * len(problem.probes)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.spstd_set_state(hr, hi_)
    chunk = 10
    done = 0
    while done < args.steps:
        n = min(chunk, args.steps - done)
        s.spstd_step(n)
        for q in range(len(problem.probes)):
            s.spstd_probe(q, cap=n)
        done += n
    s.spstd_get_state(out_r, out_i)
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    t_e2e = max_over_ranks(t_e2e, dist)
    nv, ev = s.spstd_energy_norm()
    cc, dd = s.spstd_get_coefficients()
    coeff_halfstages = int(np.count_nonzero(cc) + np.count_nonzero(dd))
    # half-stages the timed call applied per step (fused step boundaries: K (h - 1) + 1 in K steps)
    half_applied = ((args.steps * (coeff_halfstages - 1) + 1) / args.steps if half_stages < coeff_halfstages
                    else coeff_halfstages)

    # ---- the other rows of the path, each called as a user would ------------
    # a7: FP64 norm and energy (H applied to both fields, two fixed-order
    # reductions; synchronising).  a6: probe-series spectrum and peak fit of the
    # series recorded so far (2^16-point FP64 FFT for this workload).
    def host_ms(fn, reps):
        fn()
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t) * 1e3 / reps

    nfft = 1 << 16 if args.workload == "aniso_ho_3d_256" else 0
    rows = {
        "a5_probe_ms_per_step": kinds.get("probe", (0.0, 1))[0] / max(1, kinds.get("probe", (0.0, 1))[1]),
        "a6_nfft": nfft,
        "what": "a5 from the per-launch events; a6 and a7 by host clock around the synchronising C-ABI calls "
                "(spstd_spectrum over the sum of the probe series recorded so far, a6_samples of them; "
                "a6_spectrum_ms_50000_samples: the same call on a 50000-sample series, as the 50000-step "
                "workload records; spstd_energy_norm)",
    }
    try:
        rows["a6_spectrum_ms"] = host_ms(lambda: s.spstd_spectrum(-1, nfft=nfft), 3)
        rows["a6_samples"] = int(min(args.warmup + args.steps + 8, s.spstd_steps_taken()))
        rows["a7_energy_norm_ms"] = host_ms(s.spstd_energy_norm, 5)
    except spstd.SpstdError as e:
        rows["error"] = str(e)
    if args.workload == "aniso_ho_3d_256":
        # a6 at the workload's own series length: 50000 samples per probe and a
        # 2^16-point FFT (the cost depends on the series, not on the grid, so a
        # 1D solve -- one resident launch -- records it)
        from paper_1805_03155_gb300 import inputs
        w1 = inputs.well_1d(steps=50000)
        s1 = spstd.solver_for(w1, precision=32, probe_capacity=50000, stream=stream, device=local)
        s1.spstd_step(50000)
        rows["a6_spectrum_ms_50000_samples"] = host_ms(lambda: s1.spstd_spectrum(-1, nfft=1 << 16, max_peaks=32), 3)
        s1.close()
    s.close()

    if rank == 0:
        roofline = {
            "bound": "hbm",
            "kernel": dom,
            "achieved": achieved,
            "peak": peak,
            "unit": "GB/s",
            "frac": achieved / peak,
            "peak_source": f"{peak_src} hbm_gbs (burst copy)",
            "traffic": measured_traffic(args.workload, dom, schedules[KIND_AXIS[dom]] if dom in KIND_AXIS else 0),
            "algorithmic_bytes_per_launch": abytes,
            "avg_launch_ms": dom_ms,
            "step_algorithmic_bytes": step_bytes,
            # per half-stage: src, V, dst read and dst written (V from tables: 3 arrays)
            "step_floor_bytes": (3 if v_sep else 4) * es * N * coeff_halfstages,
            "step_floor_frac": ((3 if v_sep else 4) * es * N * coeff_halfstages) / (ms / args.steps * 1e-3) / 1e9
                               / peak,
            # the unit of the measurement definition: 16 B (FP32) per grid point per half-stage --
            # read src, V, dst and write dst -- whatever the kernels actually move
            "half_stage_ms_in_graph": ms / args.steps / half_applied,
            "half_stage_frac": 4 * es * N / (ms / args.steps / half_applied * 1e-3) / 1e9 / peak,
            "step_frac": 4 * es * N * coeff_halfstages / (ms / args.steps * 1e-3) / 1e9 / peak,
            "fractions_are": "of measured hbm_gbs; frac: the dominant kernel's own algorithmic bytes per launch; "
                             "half_stage_frac: 4 x (field bytes) per point over the in-graph time of one applied "
                             "half-stage; step_frac: the same over the step (h half-stages of the integrator)",
            "per_kernel_ms": {k: v[0] / v[1] for k, v in kinds.items()},
            "per_kernel_ms_are": "per launch, each launch timed alone by an event pair outside the captured "
                                 "graph (spstd_profile_steps); their per-step sum exceeds the in-graph step time",
            "per_kernel_share": {k: v[0] / sum(x[0] for x in kinds.values()) for k, v in kinds.items()},
        }
        if 3 * N * es <= L2_BYTES:
            # the three fields stay in L2 between passes: HBM does not bound the
            # kernels, the FFT arithmetic and shared-memory exchanges do
            aflops = algorithmic_flops(dom, problem.n, N)
            alu_peak = alu_peak_tflops(prec, clk.get("sm_mhz"))
            roofline.update({
                "bound": "alu",
                "achieved": aflops / (dom_ms * 1e-3) / 1e12,
                "peak": alu_peak,
                "unit": "TFLOP/s",
                "frac": aflops / (dom_ms * 1e-3) / 1e12 / alu_peak,
                "peak_source": ("derived: 152 SMs x 128 FP32 lanes x 2 flops x median SM clock" if prec == 32 else
                                "derived: nominal 1.25 TFLOP/s FP64 x median SM clock / 2070 MHz"),
                "traffic": None,
                "algorithmic_flops_per_launch": aflops,
                "hbm_frac_for_context": achieved / peak,
            })
        out = {
            "metric": "grid-point-steps/s",
            "value": value,
            "unit": "grid-point-steps/s",
            "n_gpus": ws,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": ms / args.steps,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32" if prec == 32 else "f64",
            "data": "synthetic",
            "config": {
                "workload": args.workload,
                "grid": list(problem.n),
                "box": [problem.lo[0], problem.hi[0]],
                "integrator": problem.integrator,
                "half_stages_per_step": coeff_halfstages,
                # the timed call of K steps applies K (h - 1) + 1 half-stages when step
                # boundaries are fused, K h otherwise
                "half_stages_applied_per_step": half_applied,
                "merged_step_boundaries": bool(half_stages < coeff_halfstages),
                "fields": "fp32" if prec == 32 else "fp64",
                "reductions": "fp64",
                "probes": len(problem.probes),
                "dt": problem.dt,
                "l2_policy": "inputs larger than L2 (psi_R, psi_I, V = 3 x %d MB), no flush" % (N * es >> 20)
                             if 3 * N * es > 129 * 2 ** 20 else "L2-resident grid: not flushed between steps",
                "parallelism": f"replicas{ws}",
                "schedules": schedules,
                "xy_fused": xy_fused,
                "v_separable": v_sep,
                "schedule_ms": [[round(float(t), 5) for t in row] for row in tune_ms[: problem.dims]],
            },
            "clocks": clk,
            "gpu_launches": int(launches),
            "roofline": roofline,
            "e2e": {
                "value": N * args.steps * ws / t_e2e,
                "unit": "grid-point-steps/s",
                "h2d_bytes_per_step": 2 * 8 * N / args.steps,
                "d2h_bytes_per_step": (2 * 8 * N + probe_bytes * args.steps) / args.steps,
                "what": "spstd_set_state from pinned FP64 host arrays, K steps in chunks of 10 with every "
                        "probe read back after each chunk, spstd_get_state to pinned FP64 host arrays",
            },
            "check": {"norm_after": nv, "energy_after": ev},
            "rows": rows,
        }
        if args.workload == "aniso_ho_3d_256" and not args.no_general_v:
            out["general_v"] = general_v_leg(args.steps, args.warmup, peak, local=local)
            out["next_rows"] = next_rows_leg(peak, clk.get("sm_mhz"), local=local)
        if not args.no_batch:
            bvp = batched_vs_plain(steps=args.batch_steps, local=local)
            probs, dts = bvp.pop("_probs"), bvp.pop("_dts")
            if not args.no_cpu_baseline:
                bvp["cpu_baseline"] = batched_cpu_baseline(probs, dts)
            out["batched_vs_plain"] = bvp
            out["serving"] = serving(local=local)
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(problem)
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
