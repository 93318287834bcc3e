"""Throughput of the lifted PDHG solver on one GB300 (or N replicas).

Workload (one "step"): the robust truncated-quadratic denoising problem,
512x512 pixels, rho = min(25 (u - f)^2, 0.1), lambda = 0.25, labels on [0,1]
with L = 20 (k = 19 intervals): 100 PDHG iterations (dual step + primal step
each), one FP64 energy / primal-dual gap evaluation and one unlift into a
device buffer -- one check interval of lift_solve.  Inputs are synthetic
(seeded Voronoi ramps + Gaussian noise + 10 % outliers).  The solver state
(160 MB) and the bytes streamed per iteration (403 MB) exceed the 129 MB L2.

Metric: pixel * k * iterations per second (whole job, all ranks).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank solves its own replica (weak scaling, no data
exchange); the timed region is bracketed by barriers and the max over ranks
is reported.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

H = W = 512
L = 20
K_INT = L - 1
ALPHA, NU, LAM = 25.0, 0.1, 0.25
# primal/dual step balance theta = k^2 (primal steps x theta, dual steps /
# theta): in FP64 oracle sweeps of the constant balance on this truncated-
# quadratic problem (40x40, 3000 iterations) the gap-minimising theta grows
# like k^2 (k = 4: 10-30, k = 9: about 100, k = 19: about 300)
THETA = float(K_INT * K_INT)
ITERS_PER_STEP = 100
SEED = 1512013831
METRIC = "lifted PDHG Gpix·label·iter/s"
UNIT = "Gpix*k*iter/s"
WORKLOAD = ("truncated-quadratic denoising 512x512, L=20 (k=19), alpha=25 nu=0.1 lambda=0.25, "
            "step balance theta=k^2; step = 100 PDHG iterations + FP64 gap check + unlift")
# Algorithmic DRAM bytes per pixel and launch (float32 records; halo re-reads,
# which hit L1/L2, are not counted):
#   dual step  : read xbar 8k + dual 16k + f 4 + q 4, write dual 16k + q 4 = 40k + 12
#   primal step: read primal 8k + dual 16k + q 4, write primal 8k + xbar 8k = 40k + 4
DUAL_BYTES_PER_PIX = 40 * K_INT + 12
PRIMAL_BYTES_PER_PIX = 40 * K_INT + 4
# DRAM bytes of one dual-step launch at this workload from an ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum), valid for the kernel sources
# whose SHA-256 (of the files below, in this order) is DUAL_TRAFFIC_SRC; with
# any other source the bench reports no traffic figure.
DUAL_TRAFFIC_NCU = 149552128          # 121 711 360 read + 27 840 768 written
DUAL_TRAFFIC_SRC = "d59f2f9f478ad6d2d0ecded1a4797ea20a187dd638984fbe79cdc19ebcc62b7b"
DUAL_KERNEL_FILES = ("pdhg_step.cu", "lift_device.cuh", "lift_bulk.cuh", "lift_params.h",
                     "lift_tile.cuh")


def dual_kernel_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for name in DUAL_KERNEL_FILES:
        with open(os.path.join(ROOT, "paper_1512_01383_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()
PEAK_FALLBACK_GBS = 6800.0


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            for key in ("hbm_gbs", "hbm_GBs", "hbm"):
                if key in d and isinstance(d[key], (int, float)):
                    return float(d[key]), "measured"
        except Exception:
            pass
    return PEAK_FALLBACK_GBS, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region.
    Entering waits (at most 5 s) for the first sample, so nvidia-smi's own
    start-up does not fall inside the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.ready = threading.Event()

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            self.ready.wait(timeout=5.0)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())
            self.ready.set()
        self.ready.set()

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(value: float, device) -> float:
    """The maximum of a per-rank scalar over all ranks (the job's wall time is
    the slowest rank's); the value itself when not distributed."""
    import torch
    import torch.distributed as tdist
    t = torch.tensor([value], device=device, dtype=torch.float64)
    if tdist.is_available() and tdist.is_initialized() and tdist.get_world_size() > 1:
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def make_input(rank: int = 0):
    from paper_1512_01383_gb300 import synth
    f, _ = synth.voronoi_ramps(H, W, SEED + rank)
    return synth.as_f32(f)


def cpu_sample(f: np.ndarray, side: int, iters: int):
    """Time the FP64 oracle on a side x side crop of the workload."""
    import oracle as O
    crop = np.ascontiguousarray(f[:side, :side]).astype(np.float64)
    P = O.Problem(O.TRUNC, side, side, L, 0.0, 1.0, lam=LAM, alpha=ALPHA, nu=NU, f=crop,
                  theta=THETA)
    X = O.State(P)
    t0 = time.perf_counter()
    O.pdhg(P, X, iters)
    O.energy(P, X)
    O.unlift(P, X.u)
    dt = time.perf_counter() - t0
    units = side * side * K_INT * iters
    return units / dt / 1e9, dt


def run_batch(G, torch, stream, dev, n=64, smin=128, smax=1024, iters=100, reps=3):
    """Serving-style batch: n truncated-quadratic instances, side ~ U{smin..smax},
    L ~ U{4,8,16,32}, theta = k^2 each: one graph launch per 100 iterations
    over all instances (schedule autotuned: the merged launch's tile width and
    which instances are big enough for the single-instance kernels) against a
    loop of single-handle solves of the same instances."""
    from paper_1512_01383_gb300 import synth
    inst = synth.batch_instances(n, synth.BASE_SEED + 2, smin, smax)
    fs = [torch.from_numpy(synth.as_f32(synth.voronoi_ramps(sd, sd, synth.BASE_SEED + 2 + 1000 * j)[0])).to(dev)
          for j, (sd, Lj) in enumerate(inst)]
    specs = [G.make_spec(G.LIFT_TRUNC_QUAD, sd, sd, Lj, 0.0, 1.0, LAM, ALPHA, NU, f=f,
                         check_every=iters, step_balance=float((Lj - 1) ** 2))
             for (sd, Lj), f in zip(inst, fs)]
    units = sum(sd * sd * (Lj - 1) for sd, Lj in inst) * iters
    # graph capture needs a stream other than the legacy default stream: run
    # the whole section (events included) on a stream of its own
    stream = torch.cuda.Stream(dev)
    torch.cuda.synchronize()
    b = G.lift_create_batch(specs, stream.cuda_stream)
    try:
        G.lift_batch_autotune(b, 3)
        threads, big_tiles, n_big = G.lift_batch_schedule(b)
        nfork = G.lift_batch_streams(b)
        G.lift_batch_iterate(b, iters)           # capture + warm-up
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            G.lift_batch_iterate(b, iters)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_batch = e0.elapsed_time(e1) / reps
    finally:
        G.lift_batch_destroy(b)
    # the same instances as a loop of single solves
    hs = [G.Solver(G.LIFT_TRUNC_QUAD, sd, sd, Lj, 0.0, 1.0, LAM, ALPHA, NU, f=f,
                   stream=stream.cuda_stream, step_balance=float((Lj - 1) ** 2))
          for (sd, Lj), f in zip(inst, fs)]
    for h in hs:
        h.iterate(2)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        for h in hs:
            h.iterate(iters)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_loop = e0.elapsed_time(e1) / reps
    for h in hs:
        h.close()
    return {"instances": n, "side_range": [smin, smax], "pixels": sum(sd * sd for sd, _ in inst),
            "pix_k": sum(sd * sd * (Lj - 1) for sd, Lj in inst), "iters_per_launch": iters,
            "schedule": {"merged_tile_threads": threads, "big_tiles": big_tiles,
                         "instances_on_single_kernels": n_big, "streams_of_big_instances": nfork},
            "value": units / (ms_batch * 1e-3) / 1e9, "unit": UNIT,
            "loop_of_single_solves": units / (ms_loop * 1e-3) / 1e9,
            "speedup_vs_loop": ms_loop / ms_batch,
            "ms_per_100_iters": ms_batch}


def time_iters(G, torch, solver, iters, stream):
    """Milliseconds for `iters` iterations of a solver on `stream` (events),
    after the same number untimed, which also builds the iteration graph."""
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    solver.iterate(iters)
    torch.cuda.synchronize()
    e0.record(stream)
    solver.iterate(iters)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def run_rof64(G, torch, stream, dev):
    """ROF denoising, 64x64 blobs + noise, L=2: 2000 iterations (latency-bound:
    reported in microseconds per iteration), and the time to relative gap 1e-5.
    lift_iterate runs this size inside one thread-block cluster with the state
    in shared memory; the per-half-step kernels (graph replay) are timed
    beside it."""
    from paper_1512_01383_gb300 import synth
    f = torch.from_numpy(synth.as_f32(synth.gaussian_blobs(64, 64, synth.BASE_SEED))).to(dev)
    out = {}
    for resident in (True, False):
        with G.Solver(G.LIFT_QUAD, 64, 64, 2, 0.0, 1.0, 0.2, 1.0, 0.0, f=f,
                      stream=stream.cuda_stream, check_every=100, resident=resident) as s:
            active = G.lift_set_resident(s.h, resident)
            ms = time_iters(G, torch, s, 2000, stream)
            s.reset()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc, n = s.solve(100000, 1e-5)
            dt = time.perf_counter() - t0
        r = {"us_per_iter": 1e3 * ms / 2000, "ms_2000_iters": ms,
             "time_to_gap_1e-5": {"converged": rc == G.LIFT_OK, "iters": n, "seconds": dt}}
        if resident:
            out.update(r)
            out["cluster_resident"] = active
        else:
            out["per_half_step_kernels"] = r
    return out


def run_stereo(G, torch, stream, dev, cap=60000, theta=0.1):
    """Stereo-style PL matching cost, 640x480, 65 integer disparities,
    lambda=0.05, L=8,16,32: throughput of 200 iterations per L, then a solve
    from zero with the balance theta = 0.1 (the best of 0.1, 1 and 10 in a
    sweep; the adaptive rule settles on worse balances here) to relative gap
    5e-2 and on to 1e-2, capped at `cap` iterations in all, with the mean
    |u~ - true disparity| at each stop.  On this piecewise-linear
    (polyhedral, nowhere strongly convex) cost the bounds of the last
    iterate oscillate and its gap stalls, in FP64 as in FP32, while bounds
    taken at the average of the iterates keep closing."""
    from paper_1512_01383_gb300 import synth
    cost, disp = synth.stereo_cost(480, 640, synth.BASE_SEED + 3, ndisp=65)
    cd = torch.from_numpy(synth.as_f32(cost)).to(dev)
    out = {}
    for Lx in (8, 16, 32):
        with G.Solver(G.LIFT_PL_SAMPLED, 480, 640, Lx, 0.0, 64.0, 0.05, cost=cd,
                      sample_min=0.0, sample_max=64.0, stream=stream.cuda_stream,
                      check_every=500, step_balance=theta) as s:
            ms = time_iters(G, torch, s, 200, stream)
            s.reset()
            r = {"value": 480 * 640 * (Lx - 1) * 200 / (ms * 1e-3) / 1e9, "unit": UNIT,
                 "ms_per_iter": ms / 200, "theta": theta}
            total, secs = 0, 0.0
            for tol in (5e-2, 1e-2):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                rc, n = s.solve(cap - total, tol)
                secs += time.perf_counter() - t0
                total += n
                r[f"time_to_gap_{tol:g}"] = {
                    "converged": rc == G.LIFT_OK, "iters": total, "seconds": secs,
                    "rel_gap": s.gap(), "cap_iters": cap,
                    "mean_abs_disparity_error": float(np.abs(s.unlift().astype(np.float64) - disp).mean())}
                if rc != G.LIFT_OK:
                    break
        out[f"L{Lx}"] = r
    return out


def run_stereo_averaged(G, torch, stream, dev, cap=60000, theta=0.1, every=10,
                        tols=(5e-2, 1e-2, 1e-3), levels=(8, 16, 32), restart=False):
    """The stereo solve of run_stereo with bounds also taken at the GPU's
    running average of the iterate: epochs ending at 1000, 2000, 4000, ...
    iterations (the last at `cap`); the iterate is added to the average every
    `every` iterations over the second half of each epoch (restart=False) or
    over the whole epoch (restart=True), and at the epoch's end P and D of the
    average and of the last iterate give two gaps.  With restart=True the
    iteration restarts from the average whenever its gap is the smaller.
    Reports the first epoch end at which the smaller gap is below each
    tolerance (iterations, seconds from the start, both gaps, restarts so
    far, the mean |u~ - true disparity| of the better point's image)."""
    from paper_1512_01383_gb300 import synth
    cost, disp = synth.stereo_cost(480, 640, synth.BASE_SEED + 3, ndisp=65)
    cd = torch.from_numpy(synth.as_f32(cost)).to(dev)
    out = {}
    for Lx in levels:
        with G.Solver(G.LIFT_PL_SAMPLED, 480, 640, Lx, 0.0, 64.0, 0.05, cost=cd,
                      sample_min=0.0, sample_max=64.0, stream=stream.cuda_stream,
                      check_every=every, step_balance=theta) as s:
            r = {"theta": theta, "average_every": every, "cap_iters": cap, "restart": restart}
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            n, end, ti, restarts = 0, 1000, 0, 0
            g = gl = float("nan")
            while ti < len(tols):
                end = min(end, cap)
                if not restart:
                    s.iterate(max(end // 2 - n, 0))
                    n = max(n, end // 2)
                s.average_reset()
                while n < end:
                    step = min(every, end - n)
                    s.iterate(step)
                    n += step
                    s.average_add()
                p, d, _ = s.energy_average()
                g = (p - d) / max(abs(p), abs(d), 1.0)
                gl = s.gap()
                secs = time.perf_counter() - t0
                while ti < len(tols) and min(g, gl) <= tols[ti]:
                    img = s.unlift_average() if g <= gl else s.unlift()
                    r[f"time_to_gap_{tols[ti]:g}"] = {
                        "converged": True, "iters": n, "seconds": secs, "rel_gap_average": g,
                        "rel_gap_last_iterate": gl, "restarts": restarts,
                        "mean_abs_disparity_error":
                            float(np.abs(img.astype(np.float64) - disp).mean())}
                    ti += 1
                if restart and g < gl:
                    s.average_restart()
                    restarts += 1
                if end >= cap:
                    break
                end *= 2
            for tol in tols[ti:]:
                r[f"time_to_gap_{tol:g}"] = {"converged": False, "iters": n, "seconds": secs,
                                             "rel_gap_average": g, "rel_gap_last_iterate": gl,
                                             "restarts": restarts}
        out[f"L{Lx}"] = r
    return out


def run_phase(G, torch, stream, dev):
    """Phase unwrapping (periodic quadratic pieces), 512x512 synthetic wrapped
    phase, labels on [0, 4 pi], L=8, lambda=0.2, alpha=1: throughput of 200
    iterations, then 20000 iterations from zero with the relative gap and the
    mean |u~ - true phase| of the result (with a weaker lambda the relaxation
    is not tight and the unlifted phase keeps 2 pi jumps)."""
    from paper_1512_01383_gb300 import synth
    w, true = synth.wrapped_phase(512, 512, synth.BASE_SEED + 5)
    fd = torch.from_numpy(synth.as_f32(w)).to(dev)
    L, n = 8, 20000
    with G.Solver(G.LIFT_PERIODIC_QUAD, 512, 512, L, 0.0, float(4 * np.pi), 0.2, 1.0,
                  float(2 * np.pi), f=fd, stream=stream.cuda_stream) as s:
        ms = time_iters(G, torch, s, 200, stream)
        s.reset()
        s.iterate(n)
        gap = s.gap()
        err = float(np.abs(s.unlift().astype(np.float64) - true).mean())
        # to gap 1e-3 within 60000 iterations: plain lift_solve against the
        # solve with restarts from the averaged iterate
        solves = {}
        for name in ("lift_solve", "lift_solve_averaged"):
            s.reset()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if name == "lift_solve":
                rc, it = s.solve(60000, 1e-3)
                g = s.gap()
            else:
                rc, it, g = s.solve_averaged(60000, 1e-3, first_epoch=1000, every=10)
            solves[name] = {"converged": rc == G.LIFT_OK, "iters": it,
                            "seconds": time.perf_counter() - t0, "rel_gap": g,
                            "mean_abs_error_vs_true_phase": float(
                                np.abs(s.unlift().astype(np.float64) - true).mean())}
    res = {"value": 512 * 512 * (L - 1) * 200 / (ms * 1e-3) / 1e9, "unit": UNIT,
           "ms_per_iter": ms / 200, f"rel_gap_after_{n}_iters": gap,
           f"mean_abs_error_vs_true_phase_after_{n}_iters": err,
           "time_to_gap_1e-3": solves}
    # the baseline lifting (squared circular distance sampled at the labels,
    # PL in between) with 8 and 32 labels, same iteration count
    for Lb in (8, 32):
        lab = torch.linspace(0.0, 4 * np.pi, Lb, dtype=torch.float64, device=dev)
        d = torch.remainder(lab[None, None, :] - fd.double()[:, :, None] + np.pi, 2 * np.pi) - np.pi
        cost = (0.5 * d * d).float().contiguous()
        with G.Solver(G.LIFT_PL_SAMPLED, 512, 512, Lb, 0.0, float(4 * np.pi), 0.2, cost=cost,
                      sample_min=0.0, sample_max=float(4 * np.pi), stream=stream.cuda_stream) as sb:
            sb.iterate(n)
            res[f"baseline_L{Lb}_mean_abs_error_after_{n}_iters"] = float(
                np.abs(sb.unlift().astype(np.float64) - true).mean())
            res[f"baseline_L{Lb}_rel_gap_after_{n}_iters"] = sb.gap()
    return res


def run_baseline_lifting(G, torch, stream, dev, f):
    """Proposed relaxation against the baseline lifting (Prop. 2: the PL kind
    with the cost sampled only at the labels, so rho_i** is the chord) on the
    512x512 truncated-quadratic workload, as in the comparison of Sec. 5.2:
    each solved to relative gap 1e-5 (cap 20000 iterations, adaptive balance),
    then the nonconvex energy E_nc of the unlifted result under the true
    truncated quadratic (the baseline's state is loaded into a truncated-
    quadratic handle, whose energy kernel evaluates it)."""
    fd = torch.from_numpy(f).to(dev)
    out = {}

    def solve(s):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, n = s.solve(20000, 1e-5)
        return {"converged": rc == G.LIFT_OK, "iters": n, "seconds": time.perf_counter() - t0,
                "rel_gap": s.gap()}

    for Lx, who in ((5, "both"), (10, "both"), (20, "both"), (64, "baseline")):
        with G.Solver(G.LIFT_TRUNC_QUAD, H, W, Lx, 0.0, 1.0, LAM, ALPHA, NU, f=fd,
                      check_every=100, stream=stream.cuda_stream, adaptive_balance=True) as sp:
            if who == "both":
                r = solve(sp)
                r["E_nc"] = sp.energy()[2]
                out[f"proposed_L{Lx}"] = r
            lab = torch.linspace(0.0, 1.0, Lx, dtype=torch.float64, device=dev)
            cost = torch.clamp(ALPHA * (lab[None, None, :] - fd.double()[:, :, None]) ** 2,
                               max=NU).float().contiguous()
            with G.Solver(G.LIFT_PL_SAMPLED, H, W, Lx, 0.0, 1.0, LAM, cost=cost,
                          sample_min=0.0, sample_max=1.0, check_every=100,
                          stream=stream.cuda_stream, adaptive_balance=True) as sb:
                r = solve(sb)
                st = torch.empty(G.lift_state_bytes(sb.h), dtype=torch.uint8, device=dev)
                G.lift_get_state(sb.h, st)
                G.lift_set_state(sp.h, st)
                r["E_nc"] = sp.energy()[2]
                out[f"baseline_L{Lx}"] = r
    return out


def run_volume(G, torch, stream, dev, D=128, L=8, iters=200):
    """Volume denoising (the d = 3 grid of Sec. 4): a 128^3 truncated-quadratic
    volume (3-D Voronoi ramps), L = 8, alpha=25 nu=0.1 lambda=0.25: throughput
    of 200 iterations, per-kernel bandwidth from the volume's algorithmic
    bytes (dual 48k+12, primal 44k+4 per voxel: the z component of p adds 4k
    read and 4k written in the dual step, 4k read in the primal step), and the
    solve to relative gap 1e-5 with the adaptive balance."""
    from paper_1512_01383_gb300 import synth
    f = torch.from_numpy(synth.as_f32(synth.voronoi_ramps_3d(D, D, D, synth.BASE_SEED + 7)[0])).to(dev)
    N, k = D * D * D, L - 1
    with G.Solver(G.LIFT_TRUNC_QUAD, D, D, L, 0.0, 1.0, LAM, ALPHA, NU, f=f, depth=D,
                  stream=stream.cuda_stream, check_every=100, adaptive_balance=True) as s:
        ms = time_iters(G, torch, s, iters, stream)
        nk = 50
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3 * nk)]
        torch.cuda.synchronize()
        for j in range(nk):
            ev[3 * j].record(stream)
            G.lift_dual_step(s.h)
            ev[3 * j + 1].record(stream)
            G.lift_primal_step(s.h)
            ev[3 * j + 2].record(stream)
        torch.cuda.synchronize()
        dual_ms = statistics.median(ev[3 * j].elapsed_time(ev[3 * j + 1]) for j in range(nk))
        primal_ms = statistics.median(ev[3 * j + 1].elapsed_time(ev[3 * j + 2]) for j in range(nk))
        s.reset()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, n = s.solve(20000, 1e-5)
        dt = time.perf_counter() - t0
        gap = s.gap()
    return {"value": N * k * iters / (ms * 1e-3) / 1e9, "unit": "Gvox*k*iter/s",
            "ms_per_iter": ms / iters,
            "state_mb": N * (36 * k + 4) / 1e6,
            "dual_step": {"launch_ms": dual_ms, "GB/s": (48 * k + 12) * N / (dual_ms * 1e-3) / 1e9},
            "primal_step": {"launch_ms": primal_ms,
                            "GB/s": (44 * k + 4) * N / (primal_ms * 1e-3) / 1e9},
            "time_to_gap_1e-5_adaptive": {"converged": rc == G.LIFT_OK, "iters": n,
                                          "seconds": dt, "rel_gap": gap}}


def run_differentiable(G, torch, stream, dev, iters=500, every=50, reps=3):
    """Unrolled solve for differentiation: 256x256 truncated quadratic, L=16,
    500 iterations, checkpoints every 50; forward (checkpointed) and the
    hand-written reverse pass (best of `reps` runs)."""
    from paper_1512_01383_gb300 import synth
    noisy, clean = synth.voronoi_ramps(256, 256, synth.BASE_SEED + 4)
    f = torch.from_numpy(synth.as_f32(noisy)).to(dev)
    cl = torch.from_numpy(clean.astype(np.float32)).to(dev)
    with G.Solver(G.LIFT_TRUNC_QUAD, 256, 256, 16, 0.0, 1.0, 0.25, 25.0, 0.1, f=f,
                  stream=stream.cuda_stream) as s:
        u = torch.empty((256, 256), device=dev)
        gf = torch.empty_like(u)
        res = []
        for _ in range(reps):
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            torch.cuda.synchronize()
            e0.record(stream)
            G.lift_unrolled_forward(s.h, iters, every)
            G.lift_unlift(s.h, u)
            e1.record(stream)
            gu = (2.0 * (u - cl)).contiguous()
            G.lift_unrolled_backward(s.h, gu, gf)
            e2.record(stream)
            torch.cuda.synchronize()
            res.append((e0.elapsed_time(e1), e1.elapsed_time(e2)))
    fwd, bwd = min(r[0] for r in res), min(r[1] for r in res)
    return {"forward_ms": fwd, "backward_ms": bwd, "backward_over_forward": bwd / fwd,
            "forward_value": 256 * 256 * 15 * iters / (fwd * 1e-3) / 1e9, "unit": UNIT}


def _host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_ready(_):
    import oracle  # noqa: F401  (loads the library before the timed map)
    return os.getpid()


def _oracle_crop(job):
    """One worker's share of the all-cores oracle leg: the unmodified FP64
    oracle on its own crop (in a spawned process; no CUDA)."""
    crop, iters = job
    import oracle as O
    side = crop.shape[0]
    P = O.Problem(O.TRUNC, side, side, L, 0.0, 1.0, lam=LAM, alpha=ALPHA, nu=NU, f=crop,
                  theta=THETA)
    X = O.State(P)
    t0 = time.perf_counter()
    O.pdhg(P, X, iters)
    O.energy(P, X)
    O.unlift(P, X.u)
    return side * side * K_INT * iters, time.perf_counter() - t0


def cpu_sample_all_cores(f: np.ndarray, side: int, iters: int, reps: int = 1,
                         workers: int | None = None):
    """The oracle as it stands on every host core: one single-threaded oracle
    per spawned worker process, each on its own side x side crop of the
    workload (distinct offsets), all at once.  Returns the worker count and,
    per repetition, (pixel*k*iter/s over the wall time of the whole map, wall
    seconds).  Spawned, not forked: the parent may hold a CUDA context."""
    import multiprocessing as mp
    n = workers or _host_cores()
    span_r, span_c = f.shape[0] - side, f.shape[1] - side
    jobs = []
    for j in range(n):
        r0, c0 = (j * 97) % (span_r + 1), (j * 61) % (span_c + 1)
        jobs.append((np.ascontiguousarray(f[r0:r0 + side, c0:c0 + side]).astype(np.float64), iters))
    out = []
    # bounded waits: a worker that cannot start is respawned by the pool
    # forever, so a map that does not finish raises instead of hanging
    with mp.get_context("spawn").Pool(n) as pool:
        pool.map_async(_oracle_ready, range(n), chunksize=1).get(timeout=300)
        for _ in range(reps):
            t0 = time.perf_counter()
            res = pool.map_async(_oracle_crop, jobs, chunksize=1).get(timeout=600)
            wall = time.perf_counter() - t0
            out.append((sum(u for u, _ in res) / wall / 1e9, wall))
    return n, out


# ---------------------------------------------------------------------------
# Error against the FP64 oracle, for every configuration: the FP32 GPU path
# and the oracle run the same problem (a crop or small instance of each
# configuration's inputs, same parameters and balance) for the same fixed
# number of iterations; the unlifted images and the three energies are
# compared.  Part of the CPU-baseline leg (the oracle runs in spawned workers).
# ---------------------------------------------------------------------------
def error_cases():
    """(name, problem description, iterations) per configuration."""
    from paper_1512_01383_gb300 import synth
    cases = []
    f = np.ascontiguousarray(make_input(0)[:192, :192])
    for Lx in (5, 10, 20):
        cases.append((f"truncated_512_L{Lx}", dict(kind=1, H=192, W=192, L=Lx, gmin=0.0, gmax=1.0,
                      lam=LAM, alpha=ALPHA, nu=NU, f=f, theta=float((Lx - 1) ** 2)), 100))
    fr = synth.as_f32(synth.gaussian_blobs(64, 64, synth.BASE_SEED))
    cases.append(("rof_64x64_L2", dict(kind=0, H=64, W=64, L=2, gmin=0.0, gmax=1.0, lam=0.2,
                                       alpha=1.0, nu=0.0, f=fr, theta=1.0), 2000))
    cost = synth.as_f32(synth.stereo_cost(480, 640, synth.BASE_SEED + 3, ndisp=65)[0][:96, :96])
    for Lx in (8, 16, 32):
        cases.append((f"stereo_640x480_L{Lx}", dict(kind=2, H=96, W=96, L=Lx, gmin=0.0, gmax=64.0,
                      lam=0.05, cost=cost, smin=0.0, smax=64.0, theta=1.0), 100))
    w = synth.as_f32(synth.wrapped_phase(512, 512, synth.BASE_SEED + 5)[0][:128, :128])
    cases.append(("phase_unwrapping_512_L8", dict(kind=3, H=128, W=128, L=8, gmin=0.0,
                  gmax=float(4 * np.pi), lam=0.2, alpha=1.0, nu=float(2 * np.pi), f=w,
                  theta=1.0), 100))
    fv = synth.as_f32(synth.voronoi_ramps_3d(128, 128, 128, synth.BASE_SEED + 7)[0][:24, :24, :24])
    cases.append(("volume_128cubed_L8", dict(kind=1, H=24, W=24, D=24, L=8, gmin=0.0, gmax=1.0,
                  lam=LAM, alpha=ALPHA, nu=NU, f=fv, theta=1.0), 50))
    fd = synth.as_f32(synth.voronoi_ramps(256, 256, synth.BASE_SEED + 4)[0][:96, :96])
    cases.append(("differentiable_256_L16", dict(kind=1, H=96, W=96, L=16, gmin=0.0, gmax=1.0,
                  lam=0.25, alpha=25.0, nu=0.1, f=fd, theta=1.0), 100))
    sd, Lb = synth.batch_instances(64, synth.BASE_SEED + 2, 128, 1024)[0]
    fb = synth.as_f32(synth.voronoi_ramps(sd, sd, synth.BASE_SEED + 2)[0][:128, :128])
    cases.append((f"batch_instance0_L{Lb}", dict(kind=1, H=128, W=128, L=Lb, gmin=0.0, gmax=1.0,
                  lam=LAM, alpha=ALPHA, nu=NU, f=fb, theta=float((Lb - 1) ** 2)), 100))
    lab = np.linspace(0.0, 1.0, 8)
    fl = np.ascontiguousarray(make_input(0)[:128, :128], dtype=np.float64)
    cl = synth.as_f32(np.minimum(ALPHA * (lab[None, None, :] - fl[:, :, None]) ** 2, NU))
    cases.append(("baseline_lifting_512_L8", dict(kind=2, H=128, W=128, L=8, gmin=0.0, gmax=1.0,
                  lam=LAM, cost=cl, smin=0.0, smax=1.0, theta=1.0), 100))
    return cases


def _oracle_case(job):
    """One configuration's oracle run (in a spawned worker): unlifted image
    and the three energies after `iters` iterations."""
    c, iters = job
    import oracle as O
    kinds = {0: O.QUAD, 1: O.TRUNC, 2: O.PL, 3: O.PERIODIC}
    P = O.Problem(kinds[c["kind"]], c["H"], c["W"], c["L"], c["gmin"], c["gmax"], lam=c["lam"],
                  alpha=c.get("alpha", 1.0), nu=c.get("nu", 0.0),
                  f=None if c.get("f") is None else c["f"].astype(np.float64),
                  cost=None if c.get("cost") is None else c["cost"].astype(np.float64),
                  smin=c.get("smin", 0.0), smax=c.get("smax", 1.0), theta=c["theta"],
                  D=c.get("D", 1))
    X = O.State(P)
    O.pdhg(P, X, iters)
    return O.unlift(P, X.u), O.energy(P, X)


def fp64_errors(G, torch, dev, pool):
    """Per configuration: max |u~_GPU - u~_oracle| / (label range) and the
    relative errors max(|.|, 1)-normalised of P, D and E_nc."""
    cases = error_cases()
    pending = pool.map_async(_oracle_case, [(c, it) for _, c, it in cases], chunksize=1)
    gpu = []
    for name, c, iters in cases:
        kw = dict(f=None if c.get("f") is None else torch.from_numpy(c["f"]).to(dev),
                  cost=None if c.get("cost") is None else torch.from_numpy(c["cost"]).to(dev),
                  sample_min=c.get("smin", 0.0), sample_max=c.get("smax", 1.0),
                  step_balance=c["theta"], depth=c.get("D", 1))
        with G.Solver(c["kind"], c["H"], c["W"], c["L"], c["gmin"], c["gmax"], c["lam"],
                      c.get("alpha", 1.0), c.get("nu", 0.0), **kw) as s:
            s.iterate(iters)
            gpu.append((s.unlift().reshape(-1).astype(np.float64), s.energy()))
    out = {}
    for (name, c, iters), (ug, eg), (uo, eo) in zip(cases, gpu, pending.get(timeout=900)):
        rng = c["gmax"] - c["gmin"]
        rel = [abs(a - b) / max(abs(b), 1.0) for a, b in zip(eg, eo)]
        shape = "x".join(str(v) for v in ([c["D"]] if c.get("D", 1) > 1 else []) + [c["H"], c["W"]])
        out[name] = {"u_maxabs_over_label_range": float(np.abs(ug - uo).max() / rng),
                     "P_rel": rel[0], "D_rel": rel[1], "E_nc_rel": rel[2],
                     "instance": f"{shape} of the configuration's inputs, L={c['L']}, "
                                 f"{iters} iterations"}
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    f = make_input(0)
    side, iters = 64, 20
    n, reps = cpu_sample_all_cores(f, side, iters, args.warmup + args.steps)
    timed = reps[args.warmup:]
    units = n * side * side * K_INT * iters
    value = units * len(timed) / sum(w for _, w in timed) / 1e9
    sample = (f"{n} single-threaded oracles at once (one per host core), each on its own "
              f"{side}x{side} crop of the workload, L={L}, {iters} PDHG iterations + energy + "
              f"unlift per step")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * units / (value * 1e9), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "H": H, "W": W, "L": L, "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": n, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_bands(args, G, torch, dist, rank, world, dev, barrier):
    """One (512 world) x 512 image split into bands of 512 rows, one per rank
    (the spatial decomposition of the grid of Sec. 4): per iteration the
    first own row's primal records go to the rank above and the last own
    row's dual records to the rank below (NCCL point to point), and at each
    check the three FP64 energy sums are all-reduced.  Weak scaling: the
    pixels per rank stay 512 x 512."""
    from paper_1512_01383_gb300.bands import DistributedBand, HandleBand
    Hg = H * world
    # the whole image's data: rank r's band is the replica input of rank r
    fg = np.concatenate([make_input(r) for r in range(world)], axis=0)
    fd = torch.from_numpy(fg).to(dev)
    stream = torch.cuda.current_stream(dev)
    spec = G.make_spec(G.LIFT_TRUNC_QUAD, Hg, W, L, 0.0, 1.0, LAM, ALPHA, NU, f=fd,
                       check_every=ITERS_PER_STEP, step_balance=THETA)
    band = HandleBand(spec, rank * H, (rank + 1) * H, stream.cuda_stream)
    sched = DistributedBand(band, rank, world,
                            lambda n: torch.empty(n, dtype=torch.uint8, device=dev))
    uout = torch.empty((H, W), device=dev)
    energy_buf = []

    def step():
        sched.iterate(ITERS_PER_STEP)
        energy_buf.append(sched.energy(dev))      # FP64 all_reduce of the three sums
        band.unlift(uout)

    for _ in range(args.warmup):
        step()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), dev)
    units = H * W * K_INT * ITERS_PER_STEP * args.steps * world
    value = units / (ms * 1e-3) / 1e9
    if rank == 0:
        P, Dl, E = energy_buf[-1]
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD + f"; one {Hg}x{W} image in {world} bands of {H} rows",
                       "H": Hg, "W": W, "L": L, "k": K_INT, "iters_per_step": ITERS_PER_STEP,
                       "parallelism": f"bands{world}",
                       "l2": "inputs larger than L2 (160 MB state per rank)"},
            "gpu_launches": args.steps * (2 * ITERS_PER_STEP + 3),
            "clocks": clk.summary(),
            "final_energy": {"primal": P, "dual": Dl, "nonconvex": E},
        }))
    band.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ttg", action="store_true", help="skip the time-to-gap runs")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-solve section")
    ap.add_argument("--parallelism", choices=["replicas", "bands"], default="replicas",
                    help="replicas: every rank solves its own 512x512 problem; bands: the ranks "
                         "share one (512 N) x 512 image, a band of 512 rows each, halo rows "
                         "exchanged between neighbours before each half-step")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the ROF, stereo, differentiable, phase, baseline-lifting and volume "
                         "sections")
    ap.add_argument("--only", choices=["differentiable"],
                    help="run one section alone and print its JSON (differentiable: the "
                         "256x256, L=16 unrolled solve and its reverse pass)")
    ap.add_argument("--iters", type=int, default=500,
                    help="unrolled iterations of --only differentiable")
    args = ap.parse_args()
    if args.only == "differentiable":
        import torch
        from paper_1512_01383_gb300 import lift as G
        dev = torch.device("cuda", 0)
        stream = torch.cuda.current_stream(dev)
        print(json.dumps(run_differentiable(G, torch, stream, dev, iters=args.iters,
                                            reps=max(args.steps, 1))))
        return 0
    if args.impl == "reference":
        return run_reference(args)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")

    import torch
    from paper_1512_01383_gb300 import lift as G

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    if args.parallelism == "bands":
        return run_bands(args, G, torch, dist, rank, world, dev, barrier)
    f = make_input(rank)
    fd = torch.from_numpy(f).to(dev)
    stream = torch.cuda.current_stream(dev)
    solver = G.Solver(G.LIFT_TRUNC_QUAD, H, W, L, 0.0, 1.0, LAM, ALPHA, NU, f=fd,
                      check_every=ITERS_PER_STEP, stream=stream.cuda_stream, step_balance=THETA)
    uout = torch.empty((H, W), device=dev)
    energy_buf = []

    def step():
        solver.iterate(ITERS_PER_STEP)
        energy_buf.append(solver.energy())       # FP64 gap check (syncs 24 bytes)
        solver.unlift(uout)

    for _ in range(args.warmup):
        step()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), dev)
    units = H * W * K_INT * ITERS_PER_STEP * args.steps * world
    value = units / (ms * 1e-3) / 1e9

    # per-kernel durations with events on the launching stream
    nk = 200
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3 * nk)]
    barrier()
    for j in range(nk):
        ev[3 * j].record(stream)
        G.lift_dual_step(solver.h)
        ev[3 * j + 1].record(stream)
        G.lift_primal_step(solver.h)
        ev[3 * j + 2].record(stream)
    torch.cuda.synchronize()
    dual_ms = statistics.median(ev[3 * j].elapsed_time(ev[3 * j + 1]) for j in range(nk))
    primal_ms = statistics.median(ev[3 * j + 1].elapsed_time(ev[3 * j + 2]) for j in range(nk))
    peak, peak_kind = peaks()
    bands = G.lift_set_bands(solver.h, 0)
    iter_gbs = ((DUAL_BYTES_PER_PIX + PRIMAL_BYTES_PER_PIX) * H * W * ITERS_PER_STEP
                * args.steps / (ms * 1e-3) / 1e9)
    dual_gbs = DUAL_BYTES_PER_PIX * H * W / (dual_ms * 1e-3) / 1e9
    primal_gbs = PRIMAL_BYTES_PER_PIX * H * W / (primal_ms * 1e-3) / 1e9
    # the iterations alone (graph replays, no gap check or unlift): the
    # median of 5 replays of 10 check intervals, events on the same stream
    reps = []
    for _ in range(5):
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        solver.iterate(10 * ITERS_PER_STEP)
        a1.record(stream)
        torch.cuda.synchronize()
        reps.append(a0.elapsed_time(a1) / (10 * ITERS_PER_STEP))
    iter_only_ms = statistics.median(reps)
    iter_only_gbs = (DUAL_BYTES_PER_PIX + PRIMAL_BYTES_PER_PIX) * H * W / (iter_only_ms * 1e-3) / 1e9

    # end to end through the C ABI with host buffers: upload f from pinned
    # host memory, reset, iterate, gap check, unlift to host
    fh = torch.from_numpy(f).pin_memory()
    uh = torch.empty((H, W), dtype=torch.float32).pin_memory()

    def e2e_step():
        solver.set_data(fh)
        solver.reset()
        solver.iterate(ITERS_PER_STEP)
        solver.energy()
        solver.unlift(uh)

    for _ in range(3):
        e2e_step()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    barrier()
    e2e_value = units / max_over_ranks(time.perf_counter() - t0, dev) / 1e9

    # time to relative gap 1e-5 (outside the timed region, per L)
    ttg = {}
    if not args.no_ttg and rank == 0:
        for Lx in (5, 10, 20):
            with G.Solver(G.LIFT_TRUNC_QUAD, H, W, Lx, 0.0, 1.0, LAM, ALPHA, NU, f=fd,
                          check_every=100, stream=stream.cuda_stream,
                          step_balance=float((Lx - 1) ** 2)) as s2:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                rc, n = s2.solve(60000, 1e-5)
                dt = time.perf_counter() - t0
                ttg[f"L{Lx}"] = {"converged": rc == G.LIFT_OK, "iters": n, "seconds": dt,
                                 "rel_gap": s2.gap(), "theta": float((Lx - 1) ** 2)}
            # the same from theta = 1 with the adaptive balance
            with G.Solver(G.LIFT_TRUNC_QUAD, H, W, Lx, 0.0, 1.0, LAM, ALPHA, NU, f=fd,
                          check_every=100, stream=stream.cuda_stream, step_balance=1.0,
                          adaptive_balance=True) as s2:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                rc, n = s2.solve(60000, 1e-5)
                dt = time.perf_counter() - t0
                ttg[f"L{Lx}_adaptive"] = {"converged": rc == G.LIFT_OK, "iters": n, "seconds": dt,
                                          "rel_gap": s2.gap(),
                                          "final_theta": G.lift_get_balance(s2.h)}

    extra = {}
    if not args.no_extra and rank == 0:
        extra["rof_64x64_L2"] = run_rof64(G, torch, stream, dev)
        extra["stereo_640x480"] = run_stereo(G, torch, stream, dev)
        extra["stereo_640x480"]["averaged_bounds"] = run_stereo_averaged(G, torch, stream, dev)
        extra["stereo_640x480"]["restarted_from_average"] = run_stereo_averaged(
            G, torch, stream, dev, restart=True)
        extra["differentiable_256_L16"] = run_differentiable(G, torch, stream, dev)
        extra["phase_unwrapping_512_L8"] = run_phase(G, torch, stream, dev)
        extra["proposed_vs_baseline_lifting_512"] = run_baseline_lifting(G, torch, stream, dev, f)
        extra["volume_128cubed_L8"] = run_volume(G, torch, stream, dev)

    batch = None
    if not args.no_batch and rank == 0:
        batch = run_batch(G, torch, stream, dev)
        batch["small_instances"] = run_batch(G, torch, stream, dev, n=256, smin=32, smax=128)

    cpu = None
    errors = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(min(_host_cores(), len(error_cases()))) as pool:
            errors = fp64_errors(G, torch, dev, pool)
        side, iters = 192, 60
        v1, dt = cpu_sample(f, side, iters)
        n, [(vn, wall)] = cpu_sample_all_cores(f, side, iters)
        cpu = {"value": vn, "unit": UNIT, "cores": n, "kind": "oracle",
               "sample": f"{n} single-threaded oracles at once (one per host core), each on its "
                         f"own {side}x{side} crop, L={L}, {iters} iterations + energy + unlift "
                         f"({wall:.1f} s wall)",
               "single_core": {"value": v1, "sample": f"one {side}x{side} crop, same iterations "
                                                      f"({dt:.1f} s)"},
               "fp64_error": errors}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "H": H, "W": W, "L": L, "k": K_INT,
                       "iters_per_step": ITERS_PER_STEP, "parallelism": f"replicas{world}",
                       "l2": "inputs larger than L2 (160 MB state, 403 MB per iteration)"},
            "roofline": {"bound": "hbm", "kernel": "dual_strip_kernel (dual step)", "achieved": dual_gbs,
                         "peak": peak, "peak_source": peak_kind, "unit": "GB/s",
                         "frac": dual_gbs / peak,
                         "traffic": DUAL_TRAFFIC_NCU if dual_kernel_hash() == DUAL_TRAFFIC_SRC else None,
                         "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one "
                                           "dual_strip_kernel launch at this workload, for the "
                                           "kernel source hash DUAL_TRAFFIC_SRC",
                         "algorithmic_bytes_per_launch": DUAL_BYTES_PER_PIX * H * W,
                         "launch_ms": dual_ms,
                         "primal_step": {"achieved": primal_gbs, "frac": primal_gbs / peak,
                                         "launch_ms": primal_ms,
                                         "algorithmic_bytes_per_launch": PRIMAL_BYTES_PER_PIX * H * W},
                         # the whole timed step: both half-steps' algorithmic bytes
                         # of every iteration over the step time (which also holds
                         # the gap check and the unlift); the banded graph overlaps
                         # the dual steps of some bands with the primal steps of
                         # others, so this exceeds the isolated kernels' rates
                         "iteration": {"achieved": iter_gbs, "frac": iter_gbs / peak,
                                       "bands": bands,
                                       # graph replays of the iterations alone
                                       "iterations_only": {"achieved": iter_only_gbs,
                                                           "frac": iter_only_gbs / peak,
                                                           "us_per_iteration": iter_only_ms * 1e3},
                                       "algorithmic_bytes_per_iteration":
                                           (DUAL_BYTES_PER_PIX + PRIMAL_BYTES_PER_PIX) * H * W}},
            "cpu_baseline": cpu,
            # the FP32 GPU path against the FP64 oracle, per configuration
            # (measured in the CPU-baseline leg, which runs the oracle)
            "fp64_error": errors,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": H * W * 4,
                    "d2h_bytes_per_step": H * W * 4 + 24},
            # per iteration one dual and one primal launch per band, then the
            # energy, its finish and the unlift per step
            "gpu_launches": args.steps * (2 * bands * ITERS_PER_STEP + 3),
            "clocks": clk.summary(),
            "time_to_gap_1e-5": ttg or None,
            "batch": batch,
            "other_configs": extra or None,
            "final_energy": {"primal": energy_buf[-1][0], "dual": energy_buf[-1][1],
                             "nonconvex": energy_buf[-1][2]},
        }
        print(json.dumps(line))
    solver.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
