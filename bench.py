#!/usr/bin/env python
"""Benchmark of the GB300 landmark-shooting library (libep.so).

One step = one complete feedback-control matching (Algorithm 1 of arXiv
1510.03816, gain M = h I on the momenta, p0 = 0, eps = 1e-6, at most 200
updates) of the N = 4096 planar Fourier-curve workload (Gaussian kernel
sigma = 0.1, RK4 with 100 steps, mixed precision: FP32 pair terms, per-particle
sums accumulated to FP64 accuracy, FP64 residual and momentum update), through
ep_match.

Reported (one JSON line on rank 0):
  value        pair interactions per second over the whole job (every (i, j)
               term the method evaluates: N^2 per RHS, 400 RHS per shoot, plus
               the default-gain and final-Hamiltonian evaluations), device-
               resident inputs, summed over ranks
  e2e          the same metric through ep_match with pinned host buffers
               (host<->device copies inside the timed region)
  roofline     the dominant kernel (the fused all-pairs RK4 stage) against the
               FP32 ALU peak derived from unit counts and the maximum clock
  cpu_baseline the FP64 CPU oracle on the host cores, on a bounded sample
  shoots_per_s, endpoint_err_vs_fp64, fp64_shoots_per_s: the shoot metric
               against the plain FP64 GPU shoot from the same momenta

--impl reference times the FP64 CPU oracle (the reference of this build) on
the same workload and metric, each step a bounded sample.

Multi-GPU (torchrun): every rank runs its own replica of the workload
(replicas only: the path has no data exchange), time = max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "pair interactions/s in EP RHS; shoots/s to 1e-6 endpoint err vs plain FP64"
UNIT = "pair interactions/s"
FP32_LANES_PER_SM = 128
FLOPS_PER_PAIR_2D_GAUSS = 19  # algorithmic flops of one (i, j) term of Eq. N-particle, exp counted as 1
FLOPS_PER_PAIR_2D_TENT = 20   # accepted tent pair: d, r^2, rsqrt, G, dq, p_i.p_j, weight, dp
FLOPS_PER_PAIR_3D_GAUSS = 28  # d (3), r^2 (5), G (2), dq (6), p_i.p_j (5), weight (1), dp (6)
FLOPS_PER_PAIR_3D_HVP = 65    # one (i, j) term of the Hessian-vector product of H (both blocks)
FLOPS_PER_PAIR_2D_TANGENT = 58  # FP64 tangent pair: d, dd (4), r^2, d.dd, p.p (12), dp.p + p.dp (8),
                                # phi, psi (6), dq block (10), dp block (18); exp not counted
FP64_LANES_PER_SM = 2  # FP64 FMA per clock per SM (one warp instruction per 64 cycles per SMSP)
# DRAM bytes (read + write) of one 400-stage launch of k_shoot_owner<512,8> (G=128) on the
# N = 4096 workload, from one ncu capture of that launch; reset to None when the kernel changes
OWNER_LAUNCH_DRAM_BYTES = 292352 + 49920
OWNER_TRAFFIC_KERNEL = "k_shoot_owner<512,8> (G=128)"
# L2 bytes (lts__t_bytes.sum) of one cell-list stage on the 512 x 512 jittered grid: scan
# 1.47 MB + scatter 28.0 MB + sweep 89.8 MB, from one ncu capture of a 1-step shoot
CELL_STAGE_L2_BYTES = 1466720 + 28011072 + 89718496
WORKLOAD = ("fourier_curve_warp: N=4096 2-D landmarks on a random Fourier curve -> sine warp; "
            "Gaussian sigma=0.1; RK4 100 steps on [0,1]; Algorithm 1 from p0=0, eps=1e-6 (max-norm), maxit=200; "
            "default gain h = 1/max_i sum_j G_ij")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--maxit", type=int, default=200)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true")
    ap.add_argument("--batched-maxit", type=int, default=10,
                    help="feedback iterations of the 512-problem batched row (200 = the stated configuration)")
    ap.add_argument("--profile", action="store_true",
                    help="only run warmup + steps shoots of the workload (for ncu captures); no JSON line")
    ap.add_argument("--profile-rk4-steps", type=int, default=0,
                    help="with --profile: RK4 steps per shoot (0 = the workload's 100), for short captures")
    ap.add_argument("--profile-row", default="", choices=["", "cell_list", "batched", "tangent", "match_fp64",
                                                           "velocity", "adjoint", "newton", "newton_mixed",
                                                           "rhs", "flow"],
                    help="run one small case of that secondary row (for ncu captures); no JSON line")
    return ap.parse_args()


def profile_row(name: str) -> None:
    """One small case of a secondary row, for a short ncu capture of its kernel:
    cell_list  the 512 x 512 jittered-grid tent shoot, 1 RK4 step (k_cell_sweep)
    batched    37 circle -> ellipse problems of n = 4096, alternating tent and Gaussian, 5 steps, 2 shoots
    tangent    the N = 1024 Fourier-curve tangent shoot, FP64, 5 steps (k_tangent_fp64)
    match_fp64 the N = 64 circle -> ellipse FP64 match, 5 updates (k_match_fp64)
    velocity   the same with the velocity update, 3 updates (factored G(X) inside k_match_fp64)
    adjoint    one gradient of the N = 16384 3-D star-surface workload (100 steps, checkpoints every 10)
    newton     the N = 64 circle -> ellipse Newton matching, FP64, 1 update (k_jac_fp64, k_lu_solve)
    newton_mixed  the same in mixed precision (k_jac_mixed)
    rhs        one mixed-precision RHS of the N = 4096 Fourier-curve workload (k_stage_mixed), twice
    flow       a 64 x 64 grid carried by the N = 4096 Fourier-curve shoot, 5 RK4 steps (k_flow_mixed)"""
    import torch
    from paper_1510_03816_gb300 import ep, workloads

    ep.load()
    dev = "cuda"
    if name in ("newton", "newton_mixed"):
        c = workloads.circle_to_ellipse()
        prec = ep.FP64 if name == "newton" else ep.MIXED
        prm = ep.params(dim=2, kernel=c.kernel, sigma=c.sigma, steps=c.steps, precision=prec, neigh=ep.ALLPAIRS)
        ep.match(torch.tensor(c.X, device=dev), torch.tensor(c.Y, device=dev), prm, h=1.0, eps=0.0, maxit=1,
                 rule=ep.RULE_NEWTON)
    elif name in ("rhs", "flow"):
        f = workloads.fourier_curve_warp(steps=5)
        X = torch.tensor(f.X, device=dev)
        p = 0.002 * (torch.tensor(f.Y, device=dev) - X)
        prm = ep.params(dim=2, kernel=f.kernel, sigma=f.sigma, steps=f.steps, precision=ep.MIXED, neigh=ep.ALLPAIRS)
        if name == "rhs":
            for _ in range(2):
                ep.rhs(X, p, prm)
        else:
            g = torch.linspace(0.0, 1.0, 64, device=dev, dtype=torch.float64)
            ep.flow(X, p, torch.cartesian_prod(g, g), prm)
    elif name == "adjoint":
        a3 = workloads.star_surface_3d()
        X3, Y3, p3 = (torch.tensor(v, device=dev) for v in (a3.X, a3.Y, a3.p0))
        prm3 = ep.params(dim=3, kernel=ep.GAUSS, sigma=a3.sigma, steps=a3.steps, precision=ep.MIXED)
        ep.adjoint(X3, p3, Y3, prm3, a3.lam, 10)
    elif name == "cell_list":
        g = workloads.jittered_grid()
        prm = ep.params(dim=2, kernel=ep.TENT, sigma=g.sigma, steps=1, precision=ep.MIXED, neigh=ep.CELLLIST)
        ep.shoot(torch.tensor(g.X, device=dev), torch.tensor(0.01 * (g.Y - g.X), device=dev), prm)
    elif name == "batched":
        probs = [workloads.circle_to_ellipse(n=4096, kernel=ep.TENT if b % 2 == 0 else ep.GAUSS,
                                             sigma=0.2 if b % 2 == 0 else 0.1, steps=5) for b in range(37)]
        prms = [ep.params(dim=2, kernel=p.kernel, sigma=p.sigma, steps=p.steps, precision=ep.MIXED) for p in probs]
        ep.match_batched([torch.tensor(p.X, device=dev) for p in probs], [torch.tensor(p.Y, device=dev) for p in probs],
                         prms, h=0.0, eps=1e-12, maxit=1)
    elif name == "tangent":
        f = workloads.fourier_curve_warp(n=1024, steps=5)
        X = torch.tensor(f.X, device=dev)
        v = torch.tensor(np.random.default_rng(3).normal(size=f.X.shape), device=dev)
        prm = ep.params(dim=2, kernel=f.kernel, sigma=f.sigma, steps=f.steps, precision=ep.FP64, neigh=ep.ALLPAIRS)
        ep.shoot_tangent(X, 0.002 * (torch.tensor(f.Y, device=dev) - X), torch.zeros_like(X), v, prm)
    else:
        c = workloads.circle_to_ellipse()
        prm = ep.params(dim=2, kernel=c.kernel, sigma=c.sigma, steps=c.steps, precision=ep.FP64, neigh=ep.ALLPAIRS)
        X, Y = torch.tensor(c.X, device=dev), torch.tensor(c.Y, device=dev)
        if name == "match_fp64":
            ep.match(X, Y, prm, h=0.0, eps=0.0, maxit=5)
        else:
            ep.match(X, Y, prm, h=0.5, eps=0.0, maxit=3, rule=ep.RULE_VELOCITY)
    torch.cuda.synchronize()


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist  # noqa: F811

        import torch

        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local, dist


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names[1:], f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def aggregate(ms: float, work: float, dist=None, device=None):
    """Whole-job numbers over the ranks: the slowest rank's time and the sum of the
    work (pair interactions) every rank did.  Returns (max_ms, total_work)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return ms, work
    import torch

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(work)], dtype=torch.float64, device=device)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), float(c.item())


def pairs_of(n: int, steps: int, shoots: int) -> int:
    # 4 RHS per RK4 step per shoot, + the default-gain RHS + the final-H RHS
    return n * n * (4 * steps * shoots + 2)


def run_gb300(args):
    import torch

    from paper_1510_03816_gb300 import build, ep, workloads

    world, rank, local, dist = dist_setup(args)
    build.build()
    ep.load()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    pr = workloads.fourier_curve_warp()
    n, S = pr.n, pr.steps
    X = torch.tensor(pr.X, device=dev)
    Y = torch.tensor(pr.Y, device=dev)
    prm = ep.params(dim=2, kernel=pr.kernel, sigma=pr.sigma, steps=S, precision=ep.MIXED, neigh=ep.ALLPAIRS)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > 129 MB L2

    def step():
        return ep.match(X, Y, prm, h=0.0, eps=pr.eps, maxit=args.maxit)

    if args.profile:
        p0 = 0.002 * (Y - X)
        pprm = prm
        if args.profile_rk4_steps > 0:
            pprm = ep.params(dim=2, kernel=pr.kernel, sigma=pr.sigma, steps=args.profile_rk4_steps,
                             precision=ep.MIXED, neigh=ep.ALLPAIRS)
        for _ in range(args.warmup + args.steps):
            ep.shoot(X, p0, pprm)
        torch.cuda.synchronize()
        return

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    clocks = ClockSampler(vis.split(",")[local] if vis else local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = ep.launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    shoots = 0
    last = None
    for k in range(args.steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        last = step()
        ev[k][1].record(stream)
        shoots += last.iters + 1
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = ep.launch_count() - l0
    ms = sum(a.elapsed_time(b) for a, b in ev)
    clk = clocks.stop()
    local_pairs = n * n * (4 * S * shoots + 2 * args.steps)
    t_max, total_pairs = aggregate(ms, local_pairs, dist, dev)
    value = total_pairs / (t_max / 1e3)

    # ---- dominant kernel: the persistent shoot (one cooperative launch per shoot,
    # 4 x 100 RK4 stages inside), its launches timed by the library with CUDA events
    # recorded on the launch stream around the cooperative launch
    p_fin = last.p0
    R = 5
    ep.shoot(X, p_fin, prm)
    torch.cuda.synchronize()
    ep.set_launch_timing(True)
    launch_times, kernel_name = [], ""
    for _ in range(R):
        q1m, _p1m = ep.shoot(X, p_fin, prm)
        t_ms, kernel_name = ep.last_launch()
        launch_times.append(t_ms)
    ep.set_launch_timing(False)
    launch_ms = float(np.mean(launch_times))
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_tflops = sm_count * FP32_LANES_PER_SM * 2 * 2070e6 / 1e12
    achieved = FLOPS_PER_PAIR_2D_GAUSS * n * n * 4 * S / (launch_ms / 1e3) / 1e12

    # ---- plain FP64 GPU shoot from the same momenta (the comparison point of the shoot metric)
    prm64 = ep.params(dim=2, kernel=pr.kernel, sigma=pr.sigma, steps=S, precision=ep.FP64, neigh=ep.ALLPAIRS)
    a.record(stream)
    q1d, _ = ep.shoot(X, p_fin, prm64)
    b.record(stream)
    torch.cuda.synchronize()
    fp64_ms = a.elapsed_time(b)
    err = float((q1m - q1d).abs().max().item())

    # ---- end to end through the public API with pinned host buffers
    Xh = torch.tensor(pr.X).pin_memory()
    Yh = torch.tensor(pr.Y).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    e2e_shoots = 0
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        r = ep.match(Xh, Yh, prm, h=0.0, eps=pr.eps, maxit=args.maxit)
        e2e_shoots += r.iters + 1
    e2e_s = time.perf_counter() - t0
    e2e_pairs = n * n * (4 * S * e2e_shoots + 2 * e2e_steps)
    h2d = 3 * n * 2 * 8  # X, Y, p0 (zeros) per step
    d2h = n * 2 * 8 + 16 * (e2e_shoots // e2e_steps) + 16  # p0, per-shoot residual, gain and H

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "rk4_steps": S, "precision": "FP32 pair terms; per-particle sums FP32 within warp blocks of at most 256 sources, accumulated across blocks in double-FP32 (TwoSum, FP64-level); FP64 step state, residual and update",
                   "loop": "Algorithm 1 as one CUDA graph per matching: a while-loop node over the persistent shoot and a one-CTA kernel for the FP64 residual, stop tests, update and next load (no host round trip per update)",
                   "shoots_per_step": shoots / args.steps, "l2": "256 MiB buffer written between steps (untimed)",
                   "parallelism": f"replicas x{world}"},
        "final": {"status": ep.STATUS_NAMES.get(last.status, last.status), "iters": last.iters,
                  "resid_inf": last.resid,
                  "note": "throughput metric: each step is the whole matching; with the default gain the momentum "
                          "rule stops at the iteration cap (maxit updates, maxit + 1 shoots) above eps"},
        "shoots_per_s": world * shoots / (t_max / 1e3),
        "endpoint_err_vs_fp64": err,
        "fp64_shoots_per_s": 1e3 / fp64_ms,
        "roofline": {"bound": "alu", "kernel": f"{kernel_name}: persistent all-pairs shoot, {4 * S} fused RK4 stages per launch",
                     "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s", "frac": achieved / peak_tflops,
                     "traffic": OWNER_LAUNCH_DRAM_BYTES if kernel_name == OWNER_TRAFFIC_KERNEL else None,
                     "traffic_basis": f"dram__bytes_read.sum + dram__bytes_write.sum of one 400-stage launch of "
                                      f"{OWNER_TRAFFIC_KERNEL} on this workload, from one ncu capture "
                                      "(292352 + 49920 B; the state is L2-resident)",
                     "launch_us": launch_ms * 1e3, "stage_us": launch_ms * 1e3 / (4 * S),
                     "peak_basis": f"{sm_count} SMs x 128 FP32 lanes x 2 flop x 2070 MHz (derived, not measured)",
                     "flops_per_pair": FLOPS_PER_PAIR_2D_GAUSS},
        "e2e": {"value": e2e_pairs / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if rank == 0 and not args.no_secondary:
        out["secondary"] = secondary(ep, workloads, dev, stream, peak_tflops, with_cpu=not args.no_cpu_baseline,
                                     batched_maxit=args.batched_maxit)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(pr, p_fin.cpu().numpy())
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


def dev_sm_count(torch) -> int:
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


def _events_ms(torch, stream, fn, reps):
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fn()
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(reps):
        r = fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps, r


def _l2_copy_gbs(torch) -> float:
    """Copy bandwidth of a 32 MiB -> 32 MiB copy that stays in the 129 MB L2 (read + write
    bytes per second, best of 5 x 50 copies): the L2 roofline's denominator."""
    a = torch.ones(8 * 1024 * 1024, dtype=torch.float32, device="cuda")
    b = torch.empty_like(a)
    for _ in range(10):
        b.copy_(a)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = 0.0
    for _ in range(5):
        e0.record()
        for _ in range(50):
            b.copy_(a)
        e1.record()
        torch.cuda.synchronize()
        best = max(best, 50 * 2 * a.numel() * 4 / (e0.elapsed_time(e1) * 1e-3) / 1e9)
    return best


def _alu_roofline(flops_per_s: float, peak_tflops: float, note: str) -> dict:
    a = flops_per_s / 1e12
    return {"bound": "alu", "achieved": a, "peak": peak_tflops, "unit": "TFLOP/s", "frac": a / peak_tflops,
            "note": note}


def _oracle_sample(fn, unit: str, sample: str) -> dict:
    """Time one bounded oracle call (FP64, all host threads); fn returns the work done
    in `unit`s (and may extrapolate, which `sample` then says)."""
    from oracle import oracle

    oracle.build()
    t0 = time.perf_counter()
    work = fn(oracle)
    dt = time.perf_counter() - t0
    return {"value": work / dt, "unit": unit, "cores": oracle.max_threads(), "kind": "oracle",
            "sample": f"{sample} ({dt:.2f} s)"}


def secondary(ep, workloads, dev, stream, peak_tflops, with_cpu: bool = True, batched_maxit: int = 10) -> dict:
    """The other rows of the path, each timed briefly after the main measurement,
    with its roofline and (with_cpu) a bounded sample of the FP64 oracle."""
    import torch

    out = {}
    l2_gbs = _l2_copy_gbs(torch)
    hbm = None
    try:
        hbm = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
    except Exception:
        hbm = 6800.0
    # cell list: 512 x 512 jittered grid, tent, 32 neighbours on average
    g = workloads.jittered_grid()
    Xg = torch.tensor(g.X, device=dev)
    pg = torch.tensor(0.01 * (g.Y - g.X), device=dev)
    prm = ep.params(dim=2, kernel=ep.TENT, sigma=g.sigma, steps=10, precision=ep.MIXED, neigh=ep.CELLLIST)
    cnt, _, acc_pairs = ep.cell_neighbors(Xg, prm)
    ms, _ = _events_ms(torch, stream, lambda: ep.shoot(Xg, pg, prm), 3)
    stage_us = ms * 1e3 / 40
    byts = 128 * g.n  # algorithmic bytes per particle per stage (state, accumulator, stage copy, keys)
    out["cell_list"] = {"workload": "jittered_grid 512x512, tent sigma=sqrt(32/(pi N)), RK4 10 steps",
                        "accepted_pairs_per_stage": acc_pairs, "stage_us": stage_us,
                        "pair_interactions_per_s": acc_pairs / (stage_us * 1e-6),
                        "roofline": {"bound": "hbm", "achieved": byts / (stage_us * 1e-6) / 1e9, "peak": hbm,
                                     "unit": "GB/s", "frac": byts / (stage_us * 1e-6) / 1e9 / hbm,
                                     "bytes_per_stage": byts, "note": "working set is L2-resident"},
                        "roofline_l2": {"bound": "l2", "achieved": byts / (stage_us * 1e-6) / 1e9, "peak": l2_gbs,
                                        "unit": "GB/s", "frac": byts / (stage_us * 1e-6) / 1e9 / l2_gbs,
                                        "traffic": CELL_STAGE_L2_BYTES,
                                        "traffic_frac": CELL_STAGE_L2_BYTES / (stage_us * 1e-6) / 1e9 / l2_gbs,
                                        "peak_basis": "L2-resident 32 MiB -> 32 MiB copy measured in this run "
                                                      "(read + write bytes, best of 5 x 50 copies)",
                                        "traffic_basis": "lts__t_bytes.sum of one stage's scan, scatter and sweep "
                                                         "(ncu, profiles/k_cell_sweep_jittered_grid_512.md)"},
                        "roofline_alu": _alu_roofline(acc_pairs * FLOPS_PER_PAIR_2D_TENT / (stage_us * 1e-6), peak_tflops,
                                                      f"{FLOPS_PER_PAIR_2D_TENT} flop per accepted pair")}
    # the cell-list matching at its stated configuration: Algorithm 1 on the jittered grid,
    # 100 RK4 steps, eps 1e-6, at most 200 updates, default gain
    prm_m = ep.params(dim=2, kernel=ep.TENT, sigma=g.sigma, steps=100, precision=ep.MIXED, neigh=ep.CELLLIST)
    Yg = torch.tensor(g.Y, device=dev)
    ep.match(Xg, Yg, prm_m, h=0.0, eps=1e-6, maxit=1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rm = ep.match(Xg, Yg, prm_m, h=0.0, eps=1e-6, maxit=200)
    torch.cuda.synchronize()
    dtm = time.perf_counter() - t0
    mshoots = rm.iters + 1
    out["cell_list_match"] = {"workload": "jittered_grid 512x512 (N=262144), tent sigma=sqrt(32/(pi N)), RK4 100 steps, "
                                          "Algorithm 1 from p0=0, eps 1e-6, maxit 200, default gain",
                              "seconds_per_match": dtm, "shoots": mshoots, "shoots_per_s": mshoots / dtm,
                              "pair_interactions_per_s": acc_pairs * 400 * mshoots / dtm,
                              "status": ep.STATUS_NAMES.get(rm.status, rm.status), "iters": rm.iters,
                              "resid_inf": rm.resid,
                              "roofline": {"bound": "latency", "note": "per stage as the cell_list row (its roofline); "
                                           "the host loop adds one residual read-back per update"}}
    if with_cpu:
        rows = np.random.default_rng(0).choice(g.n, 1024, replace=False)
        out["cell_list"]["cpu_baseline"] = _oracle_sample(
            lambda o: (o.rhs_rows(g.X, 0.01 * (g.Y - g.X), rows, ep.TENT, g.sigma), 1024 * g.n)[1],
            "pair interactions/s (all-pairs)",
            f"FP64 oracle RHS rows (brute force over all N={g.n} sources) for 1024 sampled particles")
    # adjoint: 16384 landmarks in 3-D, Gaussian, 100 steps, checkpoints every 10
    a3 = workloads.star_surface_3d()
    X3, Y3, p3 = (torch.tensor(v, device=dev) for v in (a3.X, a3.Y, a3.p0))
    prm3 = ep.params(dim=3, kernel=ep.GAUSS, sigma=a3.sigma, steps=a3.steps, precision=ep.MIXED)
    ms, _ = _events_ms(torch, stream, lambda: ep.adjoint(X3, p3, Y3, prm3, a3.lam, 10), 2)
    pairs = a3.n ** 2 * (4 * a3.steps * 2 + 2)  # forward + recompute RHS (+ G p0 and energy)
    hvp_pairs = a3.n ** 2 * 4 * a3.steps
    out["adjoint"] = {"workload": "star_surface_3d N=16384 3-D, Gaussian sigma=0.05, lambda=100, 100 steps, ckpt 10",
                      "ms_per_gradient": ms, "gradients_per_s": 1e3 / ms,
                      "rhs_pairs_per_gradient": pairs, "hvp_pairs_per_gradient": hvp_pairs,
                      "pair_interactions_per_s": (pairs + hvp_pairs) / (ms * 1e-3),
                      "roofline": _alu_roofline((pairs * FLOPS_PER_PAIR_3D_GAUSS + hvp_pairs * FLOPS_PER_PAIR_3D_HVP)
                                                / (ms * 1e-3), peak_tflops,
                                                f"{FLOPS_PER_PAIR_3D_GAUSS} flop per RHS pair, {FLOPS_PER_PAIR_3D_HVP} per HVP pair")}
    if with_cpu:
        small = workloads.star_surface_3d(n=512)
        k = (a3.n / small.n) ** 2 * (a3.steps / 10)
        out["adjoint"]["cpu_baseline"] = _oracle_sample(
            lambda o: (o.adjoint(small.X, small.p0, small.Y, ep.GAUSS, small.sigma, 10, small.lam), 1.0 / k)[1],
            "gradients/s (extrapolated)",
            f"FP64 oracle exact RK4 adjoint at N=512, 10 steps, scaled by (N ratio)^2 x (step ratio) = {k:.0f}")
    # batched: 512 curve problems, n log-uniform in [32, 8192]; maxit = batched_maxit (200 is the
    # stated configuration, ~60 s; the default run caps it at 10 for time)
    bp = workloads.batched_curves()
    Xs = [torch.tensor(p.X, device=dev) for p in bp]
    Ys = [torch.tensor(p.Y, device=dev) for p in bp]
    prms = [ep.params(dim=2, kernel=p.kernel, sigma=p.sigma, steps=p.steps, precision=ep.MIXED) for p in bp]
    ep.match_batched(Xs, Ys, prms, h=0.0, eps=1e-6, maxit=0)  # the launch-shape autotuner runs here, untimed
    torch.cuda.synchronize()
    ep.set_launch_timing(True)
    t0 = time.perf_counter()
    res = ep.match_batched(Xs, Ys, prms, h=0.0, eps=1e-6, maxit=batched_maxit)
    dt = time.perf_counter() - t0
    launch_ms, shape = ep.last_launch()
    ep.set_launch_timing(False)
    bpairs = sum(p.n ** 2 * (4 * p.steps * (r.iters + 1) + 2) for p, r in zip(bp, res))
    out["batched"] = {"workload": "512 curve problems, n log-uniform [32, 8192], tent 0.2 / Gaussian 0.1, 50 steps, "
                                  f"eps 1e-6, maxit {batched_maxit}" + (" (capped for time; --batched-maxit 200 is the "
                                                                         "stated configuration)" if batched_maxit < 200 else ""),
                      "seconds": dt, "matchings_per_s": len(bp) / dt, "pair_interactions_per_s": bpairs / dt,
                      "launch_ms": launch_ms, "launch_shape": shape,
                      "converged": sum(1 for r in res if r.status == ep.OK),
                      "not_converged": sum(1 for r in res if r.status == ep.ENOTCONVERGED),
                      "diverged": sum(1 for r in res if r.status == ep.EDIVERGED),
                      "shoots": sum(r.iters + 1 for r in res),
                      "roofline": _alu_roofline(bpairs * 19.5 / (launch_ms * 1e-3), peak_tflops,
                                                "19.5 flop per pair (Gaussian 19, tent 20, half the problems each), "
                                                "over the persistent launch's CUDA-event time")}
    if with_cpu:
        pick = sorted(range(len(bp)), key=lambda b: bp[b].n)[:8]
        spairs = sum(bp[b].n ** 2 * (4 * bp[b].steps * 3 + 2) for b in pick)

        def run(o):
            for b in pick:
                o.match(bp[b].X, bp[b].Y, bp[b].kernel, bp[b].sigma, bp[b].steps, h=0.0, eps=1e-6, maxit=2)
            return spairs

        out["batched"]["cpu_baseline"] = _oracle_sample(
            run, UNIT, "FP64 oracle Algorithm 1 (2 updates) on the 8 smallest problems of the batch")
    # flow: the N = 4096 Fourier-curve shoot (mixed, 100 steps) carrying a 128 x 128 grid (Eq. u)
    fc = workloads.fourier_curve_warp()
    Xf = torch.tensor(fc.X, device=dev)
    pf = torch.tensor(0.002 * (fc.Y - fc.X), device=dev)
    gx = np.linspace(0.05, 0.95, 128)
    grid = torch.tensor(np.stack(np.meshgrid(gx, gx), -1).reshape(-1, 2), device=dev)
    prmf = ep.params(dim=2, kernel=fc.kernel, sigma=fc.sigma, steps=fc.steps, precision=ep.MIXED, neigh=ep.ALLPAIRS)
    ms, _ = _events_ms(torch, stream, lambda: ep.flow(Xf, pf, grid, prmf), 3)
    m = grid.shape[0]
    tpairs = m * fc.n * 4 * fc.steps
    ppairs = fc.n * fc.n * 4 * fc.steps
    out["flow"] = {"workload": "fourier_curve_warp N=4096 shoot (Gaussian 0.1, 100 steps, mixed) carrying a 128x128 grid",
                   "ms_per_flow": ms, "points_per_s": m / (ms * 1e-3),
                   "target_pairs": tpairs, "particle_pairs": ppairs,
                   "pair_interactions_per_s": (tpairs + ppairs) / (ms * 1e-3),
                   "roofline": _alu_roofline((tpairs * 8 + ppairs * FLOPS_PER_PAIR_2D_GAUSS) / (ms * 1e-3), peak_tflops,
                                             "8 flop per target pair (Eq. u), 19 per particle pair; the particle "
                                             "shoot is recorded stage by stage")}
    if with_cpu:
        gs = grid.cpu().numpy()[::64]
        out["flow"]["cpu_baseline"] = _oracle_sample(
            lambda o: (o.flow(fc.X, 0.002 * (fc.Y - fc.X), gs, fc.kernel, fc.sigma, 2),
                       (gs.shape[0] * fc.n + fc.n * fc.n) * 8)[1],
            UNIT, f"FP64 oracle flow of {gs.shape[0]} grid points through 2 RK4 steps of the N=4096 shoot")
    # circle -> ellipse, 64 landmarks, tent, FP64 plain method, full Algorithm 1
    c = workloads.circle_to_ellipse()
    Xc, Yc = torch.tensor(c.X, device=dev), torch.tensor(c.Y, device=dev)
    for name, prec in (("fp64", ep.FP64), ("mixed", ep.MIXED)):
        prmc = ep.params(dim=2, kernel=c.kernel, sigma=c.sigma, steps=c.steps, precision=prec, neigh=ep.ALLPAIRS)
        t0 = time.perf_counter()
        r = ep.match(Xc, Yc, prmc, h=0.0, eps=c.eps, maxit=c.maxit)
        dt = time.perf_counter() - t0
        out[f"small_{name}"] = {"workload": "circle_to_ellipse N=64, tent sigma=0.25, 50 steps, eps 1e-6, maxit 200",
                                "seconds_per_match": dt, "iters": r.iters, "resid": r.resid,
                                "shoots_per_s": (r.iters + 1) / dt,
                                "roofline": {"bound": "latency", "note": "one launch: 201 dependent shoots of 200 dependent "
                                             "RHS (FP64: cooperative, 64 CTAs; mixed: one CTA); reported as shoots/s"}}
    # the inexact system (Sec. 6): circle -> ellipse, sigma_n^2 = 0.05, FP64, momentum-difference stop
    prmi = ep.params(dim=2, kernel=c.kernel, sigma=c.sigma, steps=c.steps, precision=ep.FP64, neigh=ep.ALLPAIRS,
                     inexact=0.05)
    t0 = time.perf_counter()
    r = ep.match(Xc, Yc, prmi, h=0.0, eps=c.eps, maxit=c.maxit)
    dt = time.perf_counter() - t0
    out["inexact_fp64"] = {"workload": "circle_to_ellipse N=64, tent sigma=0.25, sigma_n^2=0.05, 50 steps, FP64, "
                                       "stop on |p0^(k+1) - p0^(k)| < 1e-6",
                           "seconds_per_match": dt, "iters": r.iters, "status": r.status, "resid": r.resid,
                           "shoots_per_s": r.iters / dt,
                           "roofline": {"bound": "latency", "note": "one cooperative launch, FP64 pairs on 64 SMs"}}
    # the tangent-linear shoot (Sec. 5, D phi along one direction): N=1024 Fourier curve, FP64
    fcs = workloads.fourier_curve_warp(n=1024, steps=50)
    Xt = torch.tensor(fcs.X, device=dev)
    pt = torch.tensor(0.002 * (fcs.Y - fcs.X), device=dev)
    vt = torch.tensor(np.random.default_rng(3).normal(size=fcs.X.shape), device=dev)
    zt = torch.zeros_like(Xt)
    prmt = ep.params(dim=2, kernel=fcs.kernel, sigma=fcs.sigma, steps=fcs.steps, precision=ep.FP64,
                     neigh=ep.ALLPAIRS)
    ms, _ = _events_ms(torch, stream, lambda: ep.shoot_tangent(Xt, pt, zt, vt, prmt), 3)
    ep.set_launch_timing(True)
    ep.shoot_tangent(Xt, pt, zt, vt, prmt)
    lt_ms, lt_name = ep.last_launch()
    ep.set_launch_timing(False)
    tpairs = fcs.n ** 2 * 4 * fcs.steps
    fp64_peak = dev_sm_count(torch) * FP64_LANES_PER_SM * 2 * 2070e6 / 1e12
    out["tangent_fp64"] = {"workload": "fourier_curve_warp N=1024, Gaussian sigma=0.1, 50 steps, FP64: recorded "
                                       "primal shoot + tangent shoot along (0, v)",
                           "ms_per_call": ms, "tangent_kernel": lt_name, "tangent_launch_ms": lt_ms,
                           "pair_interactions_per_s": tpairs / (lt_ms * 1e-3),
                           "roofline": dict(_alu_roofline(tpairs * FLOPS_PER_PAIR_2D_TANGENT / (lt_ms * 1e-3),
                                                          fp64_peak,
                                                          f"FP64: {FLOPS_PER_PAIR_2D_TANGENT} flop per tangent pair "
                                                          f"(exp not counted) against {FP64_LANES_PER_SM} DFMA per "
                                                          "clock per SM at 2070 MHz"),
                                            unit="TFLOP/s (FP64)")}
    if with_cpu:
        sub = fcs.X[::4], 0.002 * (fcs.Y - fcs.X)[::4]
        k = (fcs.n / sub[0].shape[0]) ** 2 * (fcs.steps / 5)
        out["tangent_fp64"]["cpu_baseline"] = _oracle_sample(
            lambda o: (o.shoot_tangent(sub[0], sub[1], np.zeros_like(sub[0]), np.ones_like(sub[0]), fcs.kernel,
                                       fcs.sigma, 5), fcs.n ** 2 * 4 * fcs.steps / k)[1],
            UNIT, f"FP64 oracle tangent shoot (primal + tangent) at N={sub[0].shape[0]}, 5 steps; tangent pairs "
                  "counted as on the GPU")
    # the solved update rules on the N = 64 circle -> ellipse (tent sigma = 0.25, 50 steps, target noise),
    # where the momentum rule stays above 1e-6 after 200 iterations
    for name, rule, h in (("newton_fp64", ep.RULE_NEWTON, 1.0), ("velocity_fp64", ep.RULE_VELOCITY, 0.5)):
        prmc = ep.params(dim=2, kernel=c.kernel, sigma=c.sigma, steps=c.steps, precision=ep.FP64, neigh=ep.ALLPAIRS)
        ep.match(Xc, Yc, prmc, h=h, eps=c.eps, maxit=c.maxit, rule=rule)
        t0 = time.perf_counter()
        r = ep.match(Xc, Yc, prmc, h=h, eps=c.eps, maxit=c.maxit, rule=rule)
        dt = time.perf_counter() - t0
        note = (f"host GMRES; each of the {r.products} tangent shoots is one cooperative launch of 200 "
                "dependent FP64 stages on 64 particles" if rule == ep.RULE_NEWTON else
                f"one cooperative launch: 43 shoots of 200 dependent FP64 stages; G(X) factored once "
                f"(LU, one CTA), then {r.products} forward/back substitutions (one warp each)")
        out[name] = {"workload": f"circle_to_ellipse N=64, tent sigma=0.25, 50 steps, eps 1e-6, FP64, h={h}, "
                                 + ("Newton gain h (D phi)^-1" if rule == ep.RULE_NEWTON else "velocity update "
                                    "h G(X)^-1 r"),
                     "seconds_per_match": dt, "matchings_per_s": 1.0 / dt, "iters": r.iters, "status": r.status,
                     "resid": r.resid, "krylov_products": r.products,
                     "roofline": {"bound": "latency", "note": note}}
        if with_cpu:
            fn = "match_newton" if rule == ep.RULE_NEWTON else "match_velocity"

            def run_rule(o, fn=fn, h=h):
                getattr(o, fn)(c.X, c.Y, c.kernel, c.sigma, c.steps, h=h, eps=c.eps, maxit=c.maxit)
                return 1.0

            out[name]["cpu_baseline"] = _oracle_sample(
                run_rule, "matchings/s", f"FP64 oracle {fn} (dense Jacobian or Gram matrix, LU solve), whole match")
    # the Newton gain in mixed precision on the same workload: FP32 Jacobian (inexact Newton),
    # FP64 residual, solve and update
    prmm = ep.params(dim=2, kernel=c.kernel, sigma=c.sigma, steps=c.steps, precision=ep.MIXED, neigh=ep.ALLPAIRS)
    ep.match(Xc, Yc, prmm, h=1.0, eps=c.eps, maxit=c.maxit, rule=ep.RULE_NEWTON)
    t0 = time.perf_counter()
    r = ep.match(Xc, Yc, prmm, h=1.0, eps=c.eps, maxit=c.maxit, rule=ep.RULE_NEWTON)
    dt = time.perf_counter() - t0
    out["newton_mixed"] = {"workload": "circle_to_ellipse N=64, tent sigma=0.25, 50 steps, eps 1e-6, mixed precision, "
                                       "h=1.0, Newton gain with an FP32 Jacobian",
                           "seconds_per_match": dt, "matchings_per_s": 1.0 / dt, "iters": r.iters, "status": r.status,
                           "resid": r.resid, "krylov_products": r.products,
                           "roofline": {"bound": "latency", "note": f"{r.iters} updates, each a recorded mixed shoot, "
                                        "one launch of 128 FP32 tangent shoots (one per CTA), an FP64 LU on one CTA; "
                                        "the oracle's Newton time is the newton_fp64 row's"}}
    # the velocity update in mixed precision on the same workload: mixed shoots, G(X) factored once
    ep.match(Xc, Yc, prmm, h=0.5, eps=c.eps, maxit=c.maxit, rule=ep.RULE_VELOCITY)
    t0 = time.perf_counter()
    r = ep.match(Xc, Yc, prmm, h=0.5, eps=c.eps, maxit=c.maxit, rule=ep.RULE_VELOCITY)
    dt = time.perf_counter() - t0
    out["velocity_mixed"] = {"workload": "circle_to_ellipse N=64, tent sigma=0.25, 50 steps, eps 1e-6, mixed precision, "
                                         "h=0.5, velocity update h G(X)^-1 r",
                             "seconds_per_match": dt, "matchings_per_s": 1.0 / dt, "iters": r.iters, "status": r.status,
                             "resid": r.resid, "krylov_products": r.products,
                             "roofline": {"bound": "latency", "note": f"one launch on one CTA: {r.iters + 1} mixed shoots, FP64 "
                                          f"residuals and {r.iters} FP64 updates p0 += h G(X)^-1 r (G(X)^-1 formed "
                                          "once from its LU factors); the oracle's time is the velocity_fp64 row's"}}
    if with_cpu:
        def run_small(o):
            _, _, it, _, _ = o.match(c.X, c.Y, c.kernel, c.sigma, c.steps, h=0.0, eps=c.eps, maxit=c.maxit)
            return it + 1

        out["small_fp64"]["cpu_baseline"] = _oracle_sample(run_small, "shoots/s",
                                                           "FP64 oracle: the whole N=64 match (Algorithm 1)")
    return out


def cpu_baseline(pr, p0, budget_s: float = 15.0) -> dict:
    """The FP64 oracle (as it stands) on the host cores: an RK4 shoot of the same
    workload with as many steps as fit in about budget_s seconds."""
    from oracle import oracle

    oracle.build()
    cores = oracle.max_threads()
    t0 = time.perf_counter()
    oracle.rhs(pr.X, p0, pr.kernel, pr.sigma)
    t_rhs = time.perf_counter() - t0
    steps = max(1, int(budget_s / (4 * t_rhs)))
    t0 = time.perf_counter()
    oracle.shoot(pr.X, p0, pr.kernel, pr.sigma, steps)
    dt = time.perf_counter() - t0
    pairs = pr.n * pr.n * 4 * steps
    # one thread: a single RHS evaluation (N^2 pairs) of the same state
    oracle.set_threads(1)
    try:
        t0 = time.perf_counter()
        oracle.rhs(pr.X, p0, pr.kernel, pr.sigma)
        t1 = time.perf_counter() - t0
    finally:
        oracle.set_threads(cores)
    return {"value": pairs / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"FP64 oracle RK4 shoot of the N={pr.n} workload, {steps} steps ({4 * steps} RHS, "
                      f"{pairs:.3e} pair interactions) in {dt:.1f} s on {cores} threads",
            "single_thread": {"value": pr.n * pr.n / t1, "unit": UNIT, "cores": 1,
                              "sample": f"one FP64 oracle RHS of the N={pr.n} workload ({pr.n * pr.n:.3e} pair "
                                        f"interactions) in {t1:.2f} s on 1 thread"}}


def run_reference(args):
    """The FP64 CPU oracle as the reference arm: each step an RK4 shoot sample."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle

    from paper_1510_03816_gb300 import workloads

    oracle.build()
    pr = workloads.fourier_curve_warp()
    p0 = 0.002 * (pr.Y - pr.X)
    cores = oracle.max_threads()
    t0 = time.perf_counter()
    oracle.rhs(pr.X, p0, pr.kernel, pr.sigma)
    t_rhs = time.perf_counter() - t0
    steps_per_sample = max(1, int(2.0 / (4 * t_rhs)))
    for _ in range(args.warmup):
        oracle.shoot(pr.X, p0, pr.kernel, pr.sigma, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.shoot(pr.X, p0, pr.kernel, pr.sigma, steps_per_sample)
    dt = time.perf_counter() - t0
    pairs = pr.n * pr.n * 4 * steps_per_sample * args.steps
    value = pairs / dt
    sample = (f"per step: FP64 oracle RK4 shoot of the N={pr.n} workload with {steps_per_sample} RK4 steps "
              f"({4 * steps_per_sample} RHS) on {cores} threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": pr.n, "rk4_steps_per_sample": steps_per_sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    args = parse()
    if args.profile_row:
        profile_row(args.profile_row)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gb300(args)


if __name__ == "__main__":
    main()
