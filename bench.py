#!/usr/bin/env python
"""Benchmark: VIE solves/sec to an FP64 residual of 1e-6 on 128^3 random bodies.

One step = one body of the 128^3 evaluation set (random unions of ellipsoids /
cuboids, eps_r in [1.5, 6], h = lambda/128, a 1-lambda box) solved for 32 incident channels (16
Fibonacci directions x 2 polarisations) in one batched call: right-hand-side
build, mixed-precision GMRES (FP32 FFT matvec, FP64 Arnoldi / Givens, FP64
iterative refinement) down to the FP64 residual check.  The kernel spectrum of
the (shared) grid is built once before timing; each step swaps the body with
vie_set_eps_device.  Inputs (all bodies' eps grids) are resident in HBM when
the timed region starts; the working set (kernel spectrum + Krylov bases, GBs)
is far larger than L2, so no explicit flush is done.

Reported on one JSON line (rank 0):
  value        solved RHS per second, whole job (all ranks), device-resident inputs
  e2e          same through the host-buffer C ABI (eps upload, solve, far field
               at the two detector directions read back to the host)
  plain_fp64   plain FP64 GMRES on the first timed body, all 32 channels, next to
               the mixed solver's time on exactly that body (speedup_vs_plain)
  roofline     live CUDA-event timing of the dominant kernel (library timer) vs
               the measured HBM copy bandwidth
  cpu_baseline the FP64 oracle timed on this host on a bounded sample

Multi-GPU: replicas (each rank solves its own bodies, no collective on the
data path), weak scaling.  ``--impl reference`` runs one complete FP64 oracle
solve on this host instead (RHS 0 of the first timed body, minutes).

``--workload metasurface-paper`` prints a separate line for the PB metasurface
of Sec. III-B at the paper's scale (or a ``--box`` piece of it): one batched
solve of the L and R channels with ``--solver`` GMRES / BiCGStab / COCR and an
optional block-Jacobi preconditioner (``--precond cells|blocks7``), the
operator timings, and the far-field g_LR check of Eq. 31.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "VIE solves/sec to FP64 residual 1e-6 (128^3 random bodies, 32 RHS/body)"
UNIT = "solves/s"
N_AXIS = 128
H = 1.0 / 128.0
N_DIRS = 16  # x 2 polarisations = 32 RHS
SEED0 = 20000


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=4)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--bodies", type=int, default=8)
    p.add_argument("--restart", type=int, default=None,
                   help="GMRES restart length (default: 160 for the random-body workloads, the fastest measured "
                        "with the one-sweep Arnoldi; 64 for the metasurface)")
    p.add_argument("--inner-floor", type=float, default=0.7,
                   help="mixed mode: inner solves stop at inner_floor x tol x ||b|| at the latest")
    p.add_argument("--arnoldi", type=int, default=1, choices=[0, 1],
                   help="GMRES orthogonalisation: 0 classical Gram-Schmidt (two passes over the basis), "
                        "1 one-sweep Arnoldi (one pass, shifted recurrence)")
    p.add_argument("--reorth-eta", type=float, default=0.1,
                   help="GMRES re-orthogonalisation threshold (second Gram-Schmidt pass when ||w'||^2 < eta ||w||^2)")
    p.add_argument("--inner-tol", type=float, default=1e-6,
                   help="mixed mode: relative residual reduction asked of each FP32 inner solve")
    p.add_argument("--no-plain", action="store_true")
    p.add_argument("--no-bicgstab", action="store_true",
                   help="skip the comparison solve with BiCGStab (the paper's solver) on the first timed body")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--max-iter", type=int, default=20000)
    p.add_argument("--apply-only", type=int, default=0,
                   help="profiling aid: one warm-up and one FP32 operator application with this many RHS on the "
                        "first bench body, then exit (no JSON line)")
    p.add_argument("--apply-fp64", action="store_true",
                   help="with --apply-only: apply the FP64 operator instead of the FP32 one")
    p.add_argument("--apply-f32x2", action="store_true",
                   help="with --apply-only: apply the double-float operator (the residual operator of the solves)")
    p.add_argument("--workload", default="bodies128", choices=["bodies128", "metasurface-paper", "bodies-uneven", "learned", "net"],
                   help="metasurface-paper: one solve of the paper-scale PB metasurface (its own JSON line); "
                        "bodies-uneven: the random-body set of uneven grids (32^3..96^3) in multi-body batches; "
                        "learned: train the initial-guess network on solver-generated solves, then the bench "
                        "bodies with and without it")
    p.add_argument("--n-bodies", type=int, default=64, help="bodies-uneven: bodies (seeds 0..n-1)")
    p.add_argument("--train-bodies", type=int, default=250,
                   help="learned: training bodies (64^3, 16 RHS each; 250 bodies = 4000 solves)")
    p.add_argument("--epochs", type=int, default=8, help="learned: training epochs")
    p.add_argument("--channels", type=int, nargs=4, default=(20, 40, 80, 128),
                   help="learned: U-Net widths per level (20 40 80 128: 1.9 M parameters)")
    p.add_argument("--batch", type=int, default=8, help="bodies-uneven: bodies per multi-body batch")
    p.add_argument("--box", type=float, nargs=3, default=(40.0, 12.0, 2.0),
                   help="metasurface-paper: box in wavelengths (paper x, y, z)")
    p.add_argument("--solver", default="gmres", choices=["gmres", "bicgstab", "cocr"],
                   help="inner Krylov solver (the FP64 refinement around it is the same)")
    p.add_argument("--precond", default="none", choices=["none", "cells", "blocks7"],
                   help="metasurface-paper: block-Jacobi preconditioner over the fin unit cells or over 7 x 7 "
                        "lateral blocks (FGMRES)")
    p.add_argument("--inner", type=int, default=8, help="metasurface-paper: inner COCR steps per block solve")
    p.add_argument("--profile-solve", type=int, default=0,
                   help="profiling aid: a 12-iteration solve with this many RHS on the first bench body, then exit")
    args = p.parse_args()
    if args.restart is None:
        args.restart = 160 if args.workload in ("bodies128", "bodies-uneven", "learned") else 64
    return args


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def body_seeds(rank, bodies):
    return [SEED0 + rank * bodies + i for i in range(bodies)]


def aggregate_over_ranks(ms, solved, device):
    """Whole-job figures of a replicated run: the slowest rank's time (ms) and
    the units solved by all ranks (no collective on the data path; this is the
    only exchange)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    n = torch.tensor([float(solved)], device=device, dtype=torch.float64)
    dist.all_reduce(n)
    return float(t.item()), int(n.item())


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"),
                               f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- #
# oracle timing (CPU baseline and the reference arm)
# --------------------------------------------------------------------------- #
def _oracle_setup(seed):
    from oracle import vie as ovie
    from paper_2508_16471_gb300 import inputs
    wl = inputs.random_body_workload(seed, n_axis=N_AXIS, h=H, n_dirs=N_DIRS)
    g = wl.grid
    chi = ovie.contrast(wl.eps)
    t0 = time.perf_counter()
    op = ovie.FFTOperator(g.n, g.h, wl.k0, chi, workers=-1)
    t_setup = time.perf_counter() - t0
    c = wl.channels[0]
    b = ovie.rhs(chi, ovie.incident_field(g.n, g.h, wl.k0, c.khat, c.pol))
    return ovie, op, b, t_setup


def oracle_full_solve(seed, restart):
    """One complete FP64 oracle solve (GMRES(restart) to 1e-6) of RHS 0 of the
    bench body ``seed`` on this host: the measured wall time and iteration
    count, nothing extrapolated."""
    ovie, op, b, t_setup = _oracle_setup(seed)
    t0 = time.perf_counter()
    _, info = ovie.gmres(op, b, tol=1e-6, restart=restart, maxiter=100000)
    t = time.perf_counter() - t0
    return dict(seconds=t, iters=int(info["iters"]), relres=float(info["relres"]),
                converged=bool(info["converged"]), setup_s=t_setup, cores=os.cpu_count())


def oracle_sample(iters, restart, n_iter=6, seed=SEED0):
    """Bounded sample of the FP64 oracle at the bench workload: operator setup
    once, ``n_iter`` GMRES iterations on RHS 0 of body ``seed`` (time t per
    iteration at Krylov dimensions 1..n_iter), plus the time g of one
    Gram-Schmidt projection (an inner product and an update over one basis
    vector, the work GMRES adds per basis vector).  A solve of ``iters``
    iterations with restart ``restart`` then costs
        iters * t + g * (sum over its iterations of the Krylov dimension - the sample's mean),
    which is returned as solves/s with the details."""
    import numpy as np
    ovie, op, b, t_setup = _oracle_setup(seed)
    t0 = time.perf_counter()
    ovie.gmres(op, b, tol=1e-6, restart=restart, maxiter=n_iter)
    t_it = (time.perf_counter() - t0) / n_iter
    v = b.reshape(-1) / np.linalg.norm(b)
    w = v.copy()
    reps = 5
    t0 = time.perf_counter()
    for _ in range(reps):
        hcoef = np.vdot(v, w)
        w = w - hcoef * v
    g = (time.perf_counter() - t0) / reps
    dims = [(i % restart) + 1 for i in range(iters)]
    sample_mean = (n_iter + 1) / 2.0
    per_solve = iters * t_it + g * (sum(dims) - iters * sample_mean)
    return 1.0 / per_solve, dict(setup_s=t_setup, s_per_iter=t_it, s_per_projection=g, iters_per_solve=iters,
                                 n_iter=n_iter, seconds_per_solve=per_solve, cores=os.cpu_count())


def run_reference(args):
    """The oracle arm: one complete FP64 oracle GMRES solve of RHS 0 of the
    first timed bench body (the body our arm times first), measured end to end
    on this host.  The oracle keeps no state between solves, so there is
    nothing to warm up; one solve takes minutes, so the arm runs exactly one
    and reports it (steps = 1)."""
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    seed = body_seeds(0, args.bodies)[args.warmup % args.bodies]
    r = oracle_full_solve(seed, args.restart)
    value = (1.0 / r["seconds"]) if r["converged"] else 0.0
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": 1, "warmup": 0, "ms_per_step": 1000.0 * r["seconds"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"random bodies {N_AXIS}^3, h=lambda/128 (1 lambda box), {2 * N_DIRS} RHS/body",
                       "solver": f"FP64 GMRES({args.restart}), modified Gram-Schmidt (oracle)",
                       "l2": "inputs larger than L2"},
            "cpu_baseline": {"kind": "oracle", "value": value, "unit": UNIT, "cores": r["cores"],
                             "sample": (f"one complete FP64 oracle solve (NumPy/SciPy FFT operator, GMRES("
                                        f"{args.restart}) to 1e-6) of RHS 0 of body seed {seed}: {r['iters']} "
                                        f"iterations, {r['seconds']:.1f} s, relres {r['relres']:.2e}; operator "
                                        f"setup {r['setup_s']:.1f} s not timed; requested --steps "
                                        f"{args.steps} --warmup {args.warmup} do not apply (one solve)")},
            "oracle_iters": r["iters"],
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- #
# our arm
# --------------------------------------------------------------------------- #
def sources_hash(files):
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel, alg_bytes_per_launch):
    """DRAM bytes per launch of `kernel`, from the committed ncu summary
    profiles/traffic_<kernel>.txt (DRAM traffic / algorithmic bytes measured
    on one launch, scaled to this run's launches), or None when that summary
    is missing or was taken on sources that have changed since."""
    path = os.path.join(ROOT, "profiles", f"traffic_{kernel}.txt")
    if not os.path.exists(path):
        return None
    kv = {}
    for line in open(path):
        if "=" in line and not line.startswith("#"):
            k, v = line.split("=", 1)
            kv[k.strip()] = v.strip()
    try:
        if kv.get("sources_sha256_16") != sources_hash(kv["sources"].split()):
            return None
        return float(kv["traffic_over_alg"]) * alg_bytes_per_launch
    except (KeyError, ValueError, OSError):
        return None


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2508_16471_gb300 import build as libbuild
    from paper_2508_16471_gb300 import inputs
    from paper_2508_16471_gb300 import vie as V
    if rank == 0:
        libbuild.build()
    if world > 1:
        torch.distributed.barrier()
    V.load()

    if args.apply_only:
        wl = inputs.random_body_workload(SEED0, n_axis=N_AXIS, h=H, n_dirs=N_DIRS)
        with V.Handle(wl.grid.n, wl.grid.h, wl.eps, wl.k0) as hd0:
            nb = hd0.info()["n_body"]
            dt, prec = ((torch.complex128, V.PREC_FP64) if args.apply_fp64 else
                        (torch.complex128, V.PREC_F32X2) if args.apply_f32x2 else (torch.complex64, V.PREC_MIXED))
            w = torch.randn(args.apply_only, 3, nb, dtype=dt, device="cuda")
            y = torch.empty_like(w)
            torch.cuda.synchronize()
            for _ in range(2):
                hd0.apply_device(w.data_ptr(), y.data_ptr(), args.apply_only, prec)
            torch.cuda.synchronize()
        return 0

    if args.profile_solve:
        wl = inputs.random_body_workload(SEED0, n_axis=N_AXIS, h=H, n_dirs=N_DIRS)
        chs0 = [(c.khat, c.pol) for c in wl.channels][:args.profile_solve]
        with V.Handle(wl.grid.n, wl.grid.h, wl.eps, wl.k0) as hd0:
            hd0.solve(chs0, tol=1e-6, restart=args.restart, max_iter=12, allow_noconv=True, arnoldi=args.arnoldi)
        return 0

    seeds = body_seeds(rank, args.bodies)
    wls = [inputs.random_body_workload(s, n_axis=N_AXIS, h=H, n_dirs=N_DIRS) for s in seeds]
    g = wls[0].grid
    chs = [(c.khat, c.pol) for c in wls[0].channels]
    R = len(chs)
    eps_dev = [torch.from_numpy(np.ascontiguousarray(w.eps)).cuda() for w in wls]
    eps_host = [torch.from_numpy(np.ascontiguousarray(w.eps)).pin_memory() for w in wls]
    torch.cuda.synchronize()  # the library runs on the handle's own stream
    hd = V.Handle(g.n, g.h, wls[0].eps, wls[0].k0)
    stream = torch.cuda.ExternalStream(hd.stream())
    solver = {"gmres": V.SOLVER_GMRES, "bicgstab": V.SOLVER_BICGSTAB, "cocr": V.SOLVER_COCR}[args.solver]
    opts = dict(tol=1e-6, restart=args.restart, precision=V.PREC_MIXED, max_iter=args.max_iter,
                inner_tol=args.inner_tol, reorth_eta=args.reorth_eta, inner_floor=args.inner_floor, solver=solver,
                arnoldi=args.arnoldi if solver == V.SOLVER_GMRES else 0)

    def step(i):
        hd.set_eps_device(eps_dev[i % len(eps_dev)].data_ptr())
        st = hd.solve(chs, allow_noconv=True, **opts)
        return st

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    V.timer_reset()
    V.timer_enable(True)
    launches0 = V.kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    t0 = time.perf_counter()
    solved, iters, outers, relmax, mv32 = 0, [], [], 0.0, 0
    first_iters = first_all_iters = None
    t_first = None
    for i in range(args.steps):
        ts = time.perf_counter()
        st = step(args.warmup + i)  # returns after the solve's final stream synchronisation
        if t_first is None:
            t_first = time.perf_counter() - ts
        if first_iters is None:
            first_iters = st["iters"].tolist()
            first_all_iters = st["iters"].tolist()
        solved += int(st["converged"])
        mv32 += int(st["matvecs32"])
        iters.extend(st["iters"].tolist())
        outers.append(st["outer_max"])
        relmax = max(relmax, float(st["relres_max"]))
    e1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ms = e0.elapsed_time(e1)
    V.timer_enable(False)
    launches = V.kernel_launches() - launches0
    timers = V.timer_read()
    clk = clocks.stop()
    t_max = ms
    tot_solved = solved
    if world > 1:
        t_max, tot_solved = aggregate_over_ranks(ms, solved, "cuda")
    value = tot_solved / (t_max / 1000.0)

    # ---- e2e through the host-buffer C ABI ---------------------------------
    e2e = None
    if not args.no_e2e:
        th = np.radians([60.0, 60.0])
        ph = np.radians([0.0, 180.0])
        dets = np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], -1)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        solved_e2e = 0
        for i in range(args.steps):
            hd.set_eps(eps_host[(args.warmup + i) % len(eps_host)].numpy())
            st = hd.solve(chs, allow_noconv=True, **opts)
            F = hd.farfield_dirs(dets)
            solved_e2e += int(st["converged"])
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        if world > 1:
            te, solved_e2e = aggregate_over_ranks(te, solved_e2e, "cuda")
        e2e = {"value": solved_e2e / te, "unit": UNIT, "h2d_bytes_per_step": int(8 * g.size + 72 * R),
               "d2h_bytes_per_step": int(F.nbytes + 12 * R)}

    # ---- plain FP64 GMRES on the first timed body, all its RHS ---------------
    # the same body and the same 32 channels that the first timed step solved in
    # mixed precision (t_first), so the two times divide the same work
    plain = None
    b0 = args.warmup % len(eps_dev)  # the body of the first timed step
    # the FP64 basis of 32 RHS takes 16 bytes per entry: GMRES(128) at most keeps it
    # (with the FP64 work arrays) well inside the device memory
    plain_restart = min(args.restart, 128)
    if not args.no_plain and rank == 0:
        hd.set_eps_device(eps_dev[b0].data_ptr())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = hd.solve(chs, allow_noconv=True, tol=1e-6, restart=plain_restart, precision=V.PREC_FP64,
                      max_iter=args.max_iter, arnoldi=args.arnoldi)
        torch.cuda.synchronize()
        tp = time.perf_counter() - t0
        plain = {"value": int(st["converged"]) / tp, "unit": UNIT, "rhs": R, "body_seed": seeds[b0],
                 "subset": f"body seed {seeds[b0]} (the first timed step), all {R} RHS",
                 "converged": int(st["converged"]), "seconds": tp,
                 "iters_mean": float(np.mean(st["iters"])), "iters_rhs0": int(st["iters"][0]),
                 "precision": "f64", "restart": plain_restart,
                 "mixed_seconds_same_set": t_first,
                 "mixed_iters_mean_same_set": float(np.mean(first_all_iters)) if first_all_iters else None,
                 "speedup_same_set": (tp / t_first) if t_first else None}

    # ---- the paper's solver (BiCGStab) on the same body, same refinement ------
    bicg = None
    if not args.no_bicgstab and rank == 0:
        hd.set_eps_device(eps_dev[b0].data_ptr())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = hd.solve(chs, allow_noconv=True, tol=1e-6, restart=args.restart, precision=V.PREC_MIXED,
                      max_iter=args.max_iter, inner_tol=args.inner_tol, solver=V.SOLVER_BICGSTAB)
        torch.cuda.synchronize()
        tb = time.perf_counter() - t0
        bicg = {"value": int(st["converged"]) / tb, "unit": UNIT, "rhs": R, "converged": int(st["converged"]),
                "seconds": tb, "steps_mean": float(np.mean(st["iters"])),
                "matvecs32_per_rhs": st["matvecs32"] / R, "body_seed": seeds[b0],
                "gmres_iters_mean_same_body": float(np.mean(first_all_iters)) if first_all_iters else None,
                "gmres_seconds_same_body": t_first}

    # ---- roofline of the dominant kernel -----------------------------------
    peaks = load_peaks()
    hbm = peaks["hbm_gbs"] if peaks else 6800.0
    # dominant HBM-bound kernel of the FP32 path (the FP64 residual operator is FP64-ALU bound)
    dom = max(((k, v) for k, v in timers.items() if k != "matvec_fp64"), key=lambda kv: kv[1][0])
    name, (kms, kn, kbytes) = dom
    achieved = kbytes / (kms / 1000.0) / 1e9 if kms > 0 else 0.0
    kernels = {k: {"ms": round(v[0], 3), "launches": v[1], "share": round(v[0] / max(1e-9, sum(x[0] for x in timers.values())), 4),
                   "alg_GBps": round(v[2] / (v[0] / 1000.0) / 1e9, 1) if v[0] > 0 else None}
               for k, v in timers.items() if v[1] > 0}
    tname = {"xfused": "xfused"}.get(name, name)
    traffic = profiled_traffic(tname, kbytes / max(1, kn))
    roof = {"bound": "hbm", "kernel": name, "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
            "frac": round(achieved / hbm, 4), "peak_source": "MEASURED_PEAKS.json hbm_gbs (burst copy)" if peaks
            else "fallback 6800 GB/s", "alg_bytes_per_launch": kbytes / max(1, kn),
            "traffic": traffic}

    # whole FP32 operator (five passes): algorithmic bytes and the 432 N bytes-per-RHS model
    passes = [k for k in ("zfwd", "yfwd", "xfused", "yinv", "zinv") if k in timers]
    pms = sum(timers[k][0] for k in passes)
    pbytes = sum(timers[k][2] for k in passes)
    matvec = None
    if pms > 0 and mv32 > 0:
        model = 432.0 * g.size * mv32
        matvec = {"rhs_applies": mv32, "ms": round(pms, 3), "us_per_rhs_apply": round(1000.0 * pms / mv32, 2),
                  "alg_GBps": round(pbytes / (pms / 1000.0) / 1e9, 1), "alg_frac": round(pbytes / (pms / 1000.0) / 1e9 / hbm, 4),
                  "model_432N_GBps": round(model / (pms / 1000.0) / 1e9, 1),
                  "model_432N_frac": round(model / (pms / 1000.0) / 1e9 / hbm, 4)}

    if rank != 0:
        return 0
    cpu = None
    if not args.no_cpu:
        # iterations of the oracle's FP64 GMRES on RHS 0 of the first timed body: plain FP64 GMRES on the
        # GPU runs the same algorithm on the same equations (same restart), so its count stands in for the
        # oracle's (the reference arm runs that solve in full and reports its own count)
        its = plain["iters_rhs0"] if plain else (int(round(float(np.mean(iters)))) if iters else 100)
        try:
            v, det = oracle_sample(its, args.restart, n_iter=6, seed=seeds[b0])
            cpu = {"value": v, "unit": UNIT, "cores": det["cores"], "kind": "oracle",
                   "sample": (f"FP64 oracle on body seed {seeds[b0]} ({N_AXIS}^3, RHS 0): operator setup "
                              f"{det['setup_s']:.1f}s, 6 GMRES iterations at {det['s_per_iter']:.2f} s each, "
                              f"one Gram-Schmidt projection {det['s_per_projection'] * 1e3:.1f} ms; modelled "
                              f"for a {its}-iteration GMRES({args.restart}) solve (the plain FP64 GPU solve's "
                              f"count for that RHS): {det['seconds_per_solve']:.0f} s per solve")}
        except Exception as ex:  # pragma: no cover
            cpu = {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                   "sample": f"failed: {ex}"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic (seeded random bodies)",
        "config": {"workload": f"random bodies {N_AXIS}^3, h=lambda/128 (1 lambda box), eps_r in [1.5,6], "
                               f"{R} RHS/body ({N_DIRS} Fibonacci directions x 2 pol), tol 1e-6",
                   "solver": (f"mixed FP32 matvec / FP64 Arnoldi GMRES({args.restart}), "
                              + ("one-sweep" if args.arnoldi else "classical Gram-Schmidt")
                              if args.solver == "gmres"
                              else f"mixed FP32 matvec {args.solver.upper()}") + " + FP64 refinement",
                   "bodies_per_rank": args.bodies, "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (no flush)"},
        "e2e": e2e, "gpu_launches": int(launches), "clocks": clk,
        "roofline": roof, "matvec_fp32": matvec, "cpu_baseline": cpu, "plain_fp64": plain, "bicgstab": bicg,
        "speedup_vs_plain": plain["speedup_same_set"] if plain else None,
        "solver_stats": {"solved": tot_solved, "rhs_total": args.steps * R * world,
                         "iters_mean": float(np.mean(iters)) if iters else None,
                         "iters_max": int(max(iters)) if iters else None, "outer_max": max(outers) if outers else None,
                         "relres_max": relmax, "wall_s": wall},
        "kernels": kernels,
    }
    print(json.dumps(line), flush=True)
    hd.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def circular_components(F, deg):
    """(E_L, E_R) = (E_theta +/- i E_phi)/sqrt2 (Eq. 30) of far fields F [R][D][3]
    (paper frame) at signed angles ``deg`` in the xz-plane (phi = 0 for
    theta >= 0, 180 deg below); returns [R][D][2]."""
    import numpy as np
    from paper_2508_16471_gb300 import inputs
    circ = np.zeros(F.shape[:2] + (2,), dtype=np.complex128)
    for i, th in enumerate(np.radians(np.asarray(deg, float))):
        _, et, ep = inputs.spherical_basis(abs(th), 0.0 if th >= 0 else math.pi)
        Et, Ep = F[:, i] @ et, F[:, i] @ ep
        circ[:, i, 0] = (Et + 1j * Ep) / math.sqrt(2.0)
        circ[:, i, 1] = (Et - 1j * Ep) / math.sqrt(2.0)
    return circ


def run_metasurface_paper(args):
    """The PB metasurface of Sec. III-B at the paper's scale: 40 x 12 x 2
    wavelengths at 62 cells per wavelength (2480 x 744 x 124 cells, 92 x 27
    silicon nanofins), normal incidence in L and R circular polarisation, one
    batched mixed-precision solve to an FP64 residual of 1e-6; then the far
    field in the xz-plane and the g_LR map of Eq. 31 (H / V by linearity).
    The grid is stored height-first (to_grid_frame); vectors are mapped both
    ways and the circular components are taken in the paper frame."""
    import numpy as np
    import torch
    from paper_2508_16471_gb300 import build as libbuild
    from paper_2508_16471_gb300 import inputs
    from paper_2508_16471_gb300 import vie as V
    torch.cuda.set_device(0)
    libbuild.build()
    V.load()
    log = lambda *a: print(*a, file=sys.stderr, flush=True)  # noqa: E731
    t0 = time.perf_counter()
    g, eps, info = inputs.metasurface_paper(box=tuple(args.box))
    t_gen = time.perf_counter() - t0
    solver = {"gmres": V.SOLVER_GMRES, "bicgstab": V.SOLVER_BICGSTAB, "cocr": V.SOLVER_COCR}[args.solver]
    chs_p = [(c.khat, c.pol) for c in inputs.channels_metasurface([0.0])]  # L, R along +z
    chs = [(inputs.to_grid_frame(k), inputs.to_grid_frame(p)) for k, p in chs_p]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hd = V.Handle(g.n, g.h, eps, 2.0 * math.pi)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    inf = hd.info()
    Nb = inf["n_body"]
    log(f"grid {g.n} P {inf['P']} body voxels {Nb} generate {t_gen:.1f}s setup {t_setup:.1f}s")
    stream = torch.cuda.ExternalStream(hd.stream())
    if args.apply_only:  # operator applications only (profiling)
        w = torch.randn(args.apply_only, 3, Nb, dtype=torch.complex64, device="cuda")
        y = torch.empty_like(w)
        torch.cuda.synchronize()
        for _ in range(2):
            hd.apply_device(w.data_ptr(), y.data_ptr(), args.apply_only, V.PREC_MIXED)
        torch.cuda.synchronize()
        hd.close()
        return 0

    def time_apply(prec, dt, reps):
        w = torch.randn(1, 3, Nb, dtype=dt, device="cuda")
        y = torch.empty_like(w)
        torch.cuda.synchronize()
        hd.apply_device(w.data_ptr(), y.data_ptr(), 1, prec)  # allocates the work arrays
        torch.cuda.synchronize()
        V.timer_reset()
        V.timer_enable(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            hd.apply_device(w.data_ptr(), y.data_ptr(), 1, prec)
        e1.record(stream)
        torch.cuda.synchronize()
        V.timer_enable(False)
        return e0.elapsed_time(e1) / reps, V.timer_read()

    t_pc = None
    if args.precond != "none":
        cuts = info["cell_cuts"] if args.precond == "cells" else \
            [[], inputs.even_cuts(g.n[1], 7), inputs.even_cuts(g.n[2], 7)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hd.set_block_precond(cuts, inner=args.inner)
        torch.cuda.synchronize()
        t_pc = time.perf_counter() - t0
        log(f"block preconditioner ({args.precond}) set up in {t_pc:.1f}s")
    ms32, tm32 = time_apply(V.PREC_MIXED, torch.complex64, 3)
    torch.cuda.empty_cache()
    ms_blk = None
    if t_pc is not None:
        w = torch.randn(3, Nb, dtype=torch.complex64, device="cuda")
        y = torch.empty_like(w)
        torch.cuda.synchronize()
        hd.block_apply_device(w.data_ptr(), y.data_ptr())
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            hd.block_apply_device(w.data_ptr(), y.data_ptr())
        e1.record(stream)
        torch.cuda.synchronize()
        ms_blk = e0.elapsed_time(e1) / 3.0
        del w, y
        log(f"block operator: {ms_blk:.1f} ms per vector")
    torch.cuda.empty_cache()
    log(f"operator: FP32 {ms32:.1f} ms per RHS")

    peaks = load_peaks()
    hbm = peaks["hbm_gbs"] if peaks else 6800.0
    passes = [k for k in ("zfwd", "yfwd", "xfused", "yinv", "zinv") if k in tm32]
    pbytes = sum(tm32[k][2] for k in passes) / 3.0
    op32 = {"ms": round(ms32, 2), "alg_GBps": round(pbytes / (ms32 / 1000.0) / 1e9, 1),
            "alg_frac": round(pbytes / (ms32 / 1000.0) / 1e9 / hbm, 4),
            "model_432N_GBps": round(432.0 * g.size / (ms32 / 1000.0) / 1e9, 1),
            "passes": {k: {"ms": round(tm32[k][0] / 3.0, 2),
                           "alg_GBps": round(tm32[k][2] / (tm32[k][0] / 1000.0) / 1e9, 1)} for k in passes}}

    clocks = ClockSampler(0)
    clocks.start()
    V.timer_reset()
    V.timer_enable(True)
    launches0 = V.kernel_launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    t0 = time.perf_counter()
    st = hd.solve(chs, tol=1e-6, restart=args.restart, precision=V.PREC_MIXED, max_iter=args.max_iter,
                  inner_tol=args.inner_tol, reorth_eta=args.reorth_eta, inner_floor=args.inner_floor,
                  solver=solver, precond=2 if args.precond != "none" else 0, allow_noconv=True)
    e1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    solve_s = e0.elapsed_time(e1) / 1000.0
    V.timer_enable(False)
    launches = V.kernel_launches() - launches0
    timers = V.timer_read()
    clk = clocks.stop()
    log(f"solve: {solve_s:.1f}s converged {st['converged']} iters {st['iters'].tolist()} "
        f"relres {st['relres'].tolist()}")
    # the FP64 operator is timed after the solve, so that the FP32 work arrays of the solve are sized first
    # (on large grids two RHS per fused-x launch fit only while the FP64 ones are not yet held)
    ms64, _ = time_apply(V.PREC_FP64, torch.complex128, 1)
    log(f"operator: FP64 {ms64:.1f} ms per RHS")

    dom = max(((k, v) for k, v in timers.items() if k != "matvec_fp64"), key=lambda kv: kv[1][0])
    name, (kms, kn, kbytes) = dom
    achieved = kbytes / (kms / 1000.0) / 1e9 if kms > 0 else 0.0
    roof = {"bound": "hbm", "kernel": name, "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
            "frac": round(achieved / hbm, 4), "alg_bytes_per_launch": kbytes / max(1, kn), "traffic": None}
    kernels = {k: {"ms": round(v[0], 1), "launches": v[1],
                   "share": round(v[0] / max(1e-9, sum(x[0] for x in timers.values())), 4)}
               for k, v in timers.items() if v[1] > 0}

    # far field in the xz-plane (signed angle: phi = 0 for theta > 0, 180 deg below)
    deg = np.arange(-30.0, 30.0 + 1e-9, 0.5)
    t = np.radians(deg)
    d_p = np.stack([np.sin(t), np.zeros_like(t), np.cos(t)], -1)
    F = inputs.to_grid_frame(hd.farfield_dirs(inputs.to_grid_frame(d_p), basis=V.BASIS_CART))  # [2][D][3]
    circ = circular_components(F, deg)
    s2 = math.sqrt(2.0)
    H = (circ[0] + circ[1]) / s2          # Eq. 28 inverted: H = (L + R)/sqrt2
    Vv = (circ[0] - circ[1]) / (1j * s2)  # V = (L - R)/(i sqrt2)
    Ea = np.stack([H[:, 1], Vv[:, 1]])    # detector a: R at r1
    Eb = np.stack([H[:, 0], Vv[:, 0]])    # detector b: L at r2
    g2, vis, _ = V.hom_map(Ea, Eb)
    i1 = int(np.argmin(np.abs(deg + 10.0)))
    i2 = int(np.argmin(np.abs(deg - 10.0)))
    row = g2[i1]
    peaks_deg = {f"{cin}_in_{cout}_out": float(deg[int(np.argmax(np.abs(circ[r, :, c]) ** 2))])
                 for r, cin in enumerate("LR") for c, cout in enumerate("LR")}
    line = {
        "metric": f"PB metasurface ({args.solver}): mixed-precision solve to FP64 residual 1e-6 "
                  f"({info['n_paper'][0]}x{info['n_paper'][1]}x{info['n_paper'][2]} cells, 2 RHS)",
        "value": solve_s, "unit": "s", "higher_is_better": False, "n_gpus": 1, "dtype": "f32+f64",
        "data": "synthetic (Sec. III-B design rule, Eq. 32)",
        "config": {"workload": f"PB metasurface {args.box[0]:g}x{args.box[1]:g}x{args.box[2]:g} lambda at 62 "
                               f"cells/lambda, {info['fins'][0]}x"
                               f"{info['fins'][1]} Si fins (eps_r {inputs.META_EPS_SI:.3f}), no substrate",
                   "grid": list(g.n), "padded": list(inf["P"]), "body_voxels": Nb, "unknowns": 3 * Nb,
                   "rhs": "normal incidence, L and R",
                   "solver": (f"GMRES({args.restart})" if args.solver == "gmres" else args.solver.upper()) +
                             " FP32 matvec + FP64 refinement", "max_iter": args.max_iter,
                   "precond": None if args.precond == "none" else
                   {"blocks": args.precond, "inner_cocr_steps": args.inner, "setup_s": t_pc}},
        "converged": int(st["converged"]), "iters": st["iters"].tolist(), "relres": st["relres"].tolist(),
        "outer_max": int(st["outer_max"]), "matvecs32": int(st["matvecs32"]), "matvecs64": int(st["matvecs64"]),
        "seconds_per_rhs": solve_s / 2.0, "wall_s": wall, "setup_s": t_setup, "generate_s": t_gen,
        "device_bytes": inf["device_bytes"],
        "operator_fp32": op32, "operator_fp64_ms": round(ms64, 1),
        "block_operator_ms": round(ms_blk, 2) if ms_blk is not None else None,
        "roofline": roof, "gpu_launches": int(launches), "clocks": clk, "kernels": kernels,
        "g_LR_at_m10_p10": float(g2[i1, i2]),
        "g_LR_row_theta1_m10": {"min": float(row.min()), "theta2_at_min": float(deg[int(np.argmin(row))]),
                                "max": float(row.max())},
        "deflection_peaks_deg": peaks_deg,
        "paper": {"hours": 24.0, "hours_unpreconditioned": 31.9,
                  "setup": "BiCGStab + 7x7 block preconditioner, 24 CPU threads, 54M unknowns"},
    }
    print(json.dumps(line), flush=True)
    hd.close()
    return 0


def run_bodies_uneven(args):
    """Random bodies of uneven grids (the generator's 32^3..96^3 draw, 1-lambda
    box: h = 1/n), 16 RHS each (8 Fibonacci directions x 2 polarisations),
    mixed-precision GMRES to an FP64 residual of 1e-6.  Bodies are sorted by
    size and solved in multi-body batches (vie_batch_*: the FP32 operator of
    all rows of a batch in one launch per pass and padded size); the same
    bodies are then solved one handle at a time for comparison.  Set-up (kernel
    spectra) is outside both timings."""
    import numpy as np
    import torch
    from paper_2508_16471_gb300 import build as libbuild
    from paper_2508_16471_gb300 import inputs
    from paper_2508_16471_gb300 import vie as V
    torch.cuda.set_device(0)
    libbuild.build()
    V.load()
    log = lambda *a: print(*a, file=sys.stderr, flush=True)  # noqa: E731
    bodies = []
    for s in range(args.n_bodies):
        g, eps = inputs.random_body(s)
        n = g.n[0]
        bodies.append(((n, n, n), 1.0 / n, eps))
    order = sorted(range(len(bodies)), key=lambda i: bodies[i][0][0])
    chs = [(c.khat, c.pol) for c in inputs.channels_fibonacci(8)]
    R = len(chs)
    opts = dict(tol=1e-6, restart=args.restart, max_iter=args.max_iter)
    # groups of up to --batch bodies in size order, closed early where the batch's Krylov basis
    # (rows x (m + 1) x 3 N_b of the largest body, complex64) would pass 100 GB
    nbody = [int(np.count_nonzero(bodies[i][2] > 1.0)) for i in range(len(bodies))]
    groups, cur = [], []
    for i in order:
        nmax = max([nbody[k] for k in cur] + [nbody[i]])
        if cur and (len(cur) >= args.batch or
                    (len(cur) + 1) * R * (args.restart + 1) * 3 * nmax * 8 > 100e9):
            groups.append(cur)
            cur = []
        cur.append(i)
    if cur:
        groups.append(cur)
    t_batch, solved, iters, launches = 0.0, 0, [], 0
    clocks = ClockSampler(0)
    clocks.start()
    for grp in groups:
        bt = V.Batch([bodies[i] for i in grp], 2.0 * math.pi)
        torch.cuda.synchronize()
        l0 = V.kernel_launches()
        t0 = time.perf_counter()
        st = bt.solve(chs, allow_noconv=True, **opts)
        torch.cuda.synchronize()
        t_batch += time.perf_counter() - t0
        launches += V.kernel_launches() - l0
        solved += int(st["converged"])
        iters.extend(st["iters"].reshape(-1).tolist())
        log(f"batch n={[bodies[i][0][0] for i in grp]} P={sorted({bt.info(k)['P'][0] for k in range(len(grp))})} "
            f"{time.perf_counter() - t0:.2f}s converged {st['converged']}/{R * len(grp)}")
        bt.close()
        torch.cuda.empty_cache()
    clk = clocks.stop()
    t_single, solved1 = 0.0, 0
    if not args.no_plain:
        for i in order:
            n, h, eps = bodies[i]
            with V.Handle(n, h, eps, 2.0 * math.pi) as hd:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                st = hd.solve(chs, allow_noconv=True, **opts)
                torch.cuda.synchronize()
                t_single += time.perf_counter() - t0
                solved1 += int(st["converged"])
    sizes = [bodies[i][0][0] for i in order]
    line = {"metric": "random bodies of uneven grids: solves/sec to FP64 residual 1e-6 in multi-body batches",
            "value": solved / t_batch, "unit": "solves/s", "higher_is_better": True, "n_gpus": 1,
            "dtype": "f32+f64", "data": "synthetic (seeded random bodies)",
            "config": {"workload": f"{len(bodies)} random bodies (seeds 0..{len(bodies) - 1}), n in "
                                   f"{min(sizes)}..{max(sizes)} (drawn 32..96), h = lambda/n, eps_r in [1.5, 6], "
                                   f"{R} RHS each", "batch": args.batch,
                       "batch_sizes": [len(gp) for gp in groups],
                       "solver": f"mixed FP32 matvec / FP64 Arnoldi GMRES({args.restart}) + double-float residual"},
            "bodies_per_s": len(bodies) * (solved / (R * len(bodies))) / t_batch, "seconds": t_batch,
            "solved": solved, "rhs_total": R * len(bodies), "iters_mean": float(np.mean(iters)),
            "gpu_launches": int(launches), "clocks": clk,
            "one_handle_per_body": {"seconds": t_single, "solved": solved1,
                                    "value": (solved1 / t_single) if t_single else None} if t_single else None,
            "speedup_vs_one_handle_per_body": (t_single / t_batch) if t_single else None}
    print(json.dumps(line), flush=True)
    return 0


def run_learned(args):
    """The learned initial guess at its configured scale: a 4-level 3-D U-Net
    (--channels, BF16 activations, FP32 accumulation) trained by the
    library's kernels on solver-generated solves of 64^3 random bodies (1-lambda
    box, seeds 10000+, 16 RHS each), then the 8 bench bodies (128^3, same box,
    32 RHS) solved with x0 = 0 and with the network's start (the network sees
    the same lambda/16 coarse voxels at both sizes: factor 4 at 64^3, 8 at
    128^3).  Solves/s of the learned solves include the network inference."""
    import numpy as np
    import torch
    from paper_2508_16471_gb300 import build as libbuild
    from paper_2508_16471_gb300 import inputs
    from paper_2508_16471_gb300 import learned
    from paper_2508_16471_gb300 import vie as V
    torch.cuda.set_device(0)
    libbuild.build()
    V.load()
    log = lambda *a: print(*a, file=sys.stderr, flush=True)  # noqa: E731
    n_tr, f_tr = 64, 4
    D = n_tr // f_tr
    t0 = time.perf_counter()
    X, T, M, it_tr = learned.generate(n_tr, 1.0 / n_tr, list(range(10000, 10000 + args.train_bodies)), 8, f_tr)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    log(f"training data: {X.shape[0]} solves in {t_gen:.1f}s")
    net = V.Net(tuple(args.channels), seed=0, bf16=True)
    t0 = time.perf_counter()
    hist = learned.train(net, X, T, M, D, epochs=args.epochs, batch=8, lr=2e-3, lr_decay=0.8)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    log(f"trained {net.num_params()} parameters, {args.epochs} epochs in {t_train:.1f}s, loss {hist[0]:.4f} -> "
        f"{hist[-1]:.4f}")
    del X, T, M
    torch.cuda.empty_cache()
    seeds = body_seeds(0, args.bodies)
    wls = [inputs.random_body_workload(s_, n_axis=N_AXIS, h=H, n_dirs=N_DIRS) for s_ in seeds]
    chs = [(c.khat, c.pol) for c in wls[0].channels]
    R = len(chs)
    g = wls[0].grid
    opts = dict(tol=1e-6, restart=args.restart, max_iter=args.max_iter)
    res = {"plain": [0.0, 0, []], "learned": [0.0, 0, []]}
    rejected = 0
    with V.Handle(g.n, g.h, wls[0].eps, wls[0].k0) as hd:
        hd.attach_net(net, N_AXIS // D)
        for i, wl in enumerate(wls):
            hd.set_eps(wl.eps)
            for mode in ("plain", "learned"):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                st = hd.solve(chs, allow_noconv=True, use_x0=2 if mode == "learned" else 0, **opts)
                torch.cuda.synchronize()
                r = res[mode]
                r[0] += time.perf_counter() - t0
                r[1] += int(st["converged"])
                r[2].extend(st["iters"].tolist())
            rejected += hd.guesses_rejected()
    out = {m: {"solves_per_s": v[1] / v[0], "seconds": v[0], "solved": v[1], "iters_mean": float(np.mean(v[2]))}
           for m, v in res.items()}
    line = {"metric": "VIE solves/sec to FP64 residual 1e-6 (128^3 random bodies, 32 RHS/body), learned start vs "
                      "zero start",
            "value": out["learned"]["solves_per_s"], "unit": "solves/s", "higher_is_better": True, "n_gpus": 1,
            "dtype": "f32+f64 (network bf16 storage, fp32 accumulate)", "data": "synthetic (seeded random bodies)",
            "config": {"workload": f"{len(wls)} bench bodies (seeds {seeds[0]}..{seeds[-1]}), 128^3, 1 lambda box, "
                                   f"{R} RHS", "train": f"{it_tr.size} solves of {args.train_bodies} 64^3 bodies "
                                   f"(seeds 10000+), {args.epochs} epochs, batch 8, Adam lr 2e-3 x 0.8/epoch",
                       "network": {"channels": list(args.channels), "params": net.num_params(),
                                   "coarse_grid": f"{D}^3 (lambda/16 voxels)"}},
            "learned": out["learned"], "plain": out["plain"], "guesses_rejected": rejected,
            "gain_iters": 1.0 - out["learned"]["iters_mean"] / out["plain"]["iters_mean"],
            "speedup": out["learned"]["solves_per_s"] / out["plain"]["solves_per_s"],
            "train_seconds": t_train, "generate_seconds": t_gen, "loss_first_last": [hist[0], hist[-1]]}
    print(json.dumps(line), flush=True)
    return 0


def run_net(args):
    """The learned part's network alone at its configured width (channels
    --channels, BF16 storage, 16^3 coarse grid, batch 8 as in training):
    forward and training step (forward, backward, Adam with a negligible
    learning rate so that the weights stay put) per call, with the 3x3x3
    convolutions on the tensor cores (tcgen05 implicit GEMM) and on the CUDA
    cores; TFLOP/s counts the convolution products only (2 x voxels x Cin x
    Cout x taps; three such products per training step)."""
    import numpy as np
    import torch
    from paper_2508_16471_gb300 import build as libbuild
    from paper_2508_16471_gb300 import vie as V
    libbuild.build()
    V.load()
    ch = tuple(args.channels)
    B, D = 8, 16
    rng = np.random.default_rng(0)
    x = torch.from_numpy(rng.standard_normal((B, 10, D, D, D)).astype(np.float32)).cuda()
    t = torch.from_numpy(rng.standard_normal((B, 6, D, D, D)).astype(np.float32)).cuda()
    m = torch.ones(B, D, D, D, device="cuda")
    y = torch.empty(B, 6, D, D, D, device="cuda")
    c0, c1, c2, c3 = ch
    layers = [(10, c0, 0), (c0, c0, 0), (c0, c1, 1), (c1, c1, 1), (c1, c2, 2), (c2, c2, 2), (c2, c3, 3), (c3, c3, 3),
              (c3 + c2, c2, 2), (c2, c2, 2), (c2 + c1, c1, 1), (c1, c1, 1), (c1 + c0, c0, 0), (c0, c0, 0)]
    fl = sum(2.0 * B * (D >> lv) ** 3 * ci * co * 27 for ci, co, lv in layers) + 2.0 * B * D ** 3 * c0 * 6
    res = {}
    for tc in (True, False):
        net = V.Net(ch, seed=1, bf16=True)
        net.set_tensor_cores(tc)
        torch.cuda.synchronize()
        for _ in range(args.warmup):
            net.forward(x.data_ptr(), y.data_ptr(), B, D)
            net.train_step(x.data_ptr(), t.data_ptr(), m.data_ptr(), B, D, 1e-12)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            net.forward(x.data_ptr(), y.data_ptr(), B, D)
        torch.cuda.synchronize()
        tf = (time.perf_counter() - t0) / args.steps
        t0 = time.perf_counter()
        for _ in range(args.steps):
            net.train_step(x.data_ptr(), t.data_ptr(), m.data_ptr(), B, D, 1e-12)
        torch.cuda.synchronize()
        tt = (time.perf_counter() - t0) / args.steps
        res["tensor_cores" if tc else "cuda_cores"] = {
            "forward_ms": 1e3 * tf, "train_step_ms": 1e3 * tt, "forward_conv_TFLOPs": fl / tf / 1e12,
            "train_conv_TFLOPs": 3 * fl / tt / 1e12}
        net.close()
    line = {"metric": "U-Net training steps/s (BF16 storage, FP32 accumulation)", "value": 1e3 / res["tensor_cores"]["train_step_ms"],
            "unit": "steps/s", "higher_is_better": True, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "dtype": "bf16", "data": "synthetic", "config": {"workload": f"U-Net {list(ch)}, batch {B}, {D}^3 grid",
                                                              "conv_flops_per_forward": fl},
            "tensor_cores": res["tensor_cores"], "cuda_cores": res["cuda_cores"],
            "speedup_train": res["cuda_cores"]["train_step_ms"] / res["tensor_cores"]["train_step_ms"]}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "metasurface-paper":
        return run_metasurface_paper(args)
    if args.workload == "bodies-uneven":
        return run_bodies_uneven(args)
    if args.workload == "learned":
        return run_learned(args)
    if args.workload == "net":
        return run_net(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
