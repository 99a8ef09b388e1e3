#!/usr/bin/env python
"""Benchmark of the Stokes-Darcy Dirichlet-Neumann solve on one GB300.

Workload (one step): the unit sphere at h = 1/32 (N = 17070 quadrature points,
delta = 3h), mu = 1, U = e_z, BJS traction with gamma in {0.1, 1} and
kappa in {1, 1e-2, 1e-4} (six D-N solves, theta = 0.5 min(kappa, 1)),
interface GMRES to 1e-8 with local GMRES to 1e-9 (one Krylov cycle each).
Pair sums in FP32C (FP32 terms, compensated accumulation), Krylov and
interface arithmetic in FP64.  The plain FP64 comparison solves run to the
paper's 1e-9 / 1e-10.
The BJS slip is imposed implicitly in the Stokes step (one fused SL+DL pass
per matvec).

Metric: pair-interactions/s, i.e. ordered (target, source) pairs evaluated
by the pair kernels over the whole step divided by the step's device time.
Beside it: time-to-solution of each solve in FP32C and in plain FP64 (both
on the GPU) and the FP32C-vs-FP64 difference of every output.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
on a bounded sample of the same workload instead.
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

H = 1.0 / 32
KAPPAS = (1.0, 1e-2, 1e-4)
ALPHAS = (0.1, 1.0)
# FP32C runs to tolerances its arithmetic can reach (pair sums carry ~1e-7
# relative rounding); the plain FP64 comparison runs to the paper's 1e-9/1e-10.
TOL = {"fp32c": (1e-8, 1e-9), "fp64": (1e-9, 1e-10)}
METRIC = "pair-interactions/s (SL+DL matvec) & DDM time-to-solution at stated error, FP32c vs FP64"
UNIT = "pair-interactions/s"
# Nominal FP32 flops per pair of the Stokes double layer (FMA = 2, rsqrt,
# exp and erf counted as one each): far pairs (s4 = 1) and near pairs
# (rho < 5.5, smoothed kernel).
FLOPS_SDL_FAR = 33
FLOPS_SDL_NEAR = 50
RHO_FAR = 5.5
DRAM_BYTES_SSLDL = 1201152
L2_FLUSH_BYTES = 256 << 20


def workload_config():
    return {"workload": "unit sphere h=1/32 (N=17070), delta=3h, BJS traction, kappa in {1,1e-2,1e-4} x "
                        "alpha in {0.1,1}, D-N by interface GMRES; FP32C to 1e-8 (local GMRES 1e-9), "
                        "FP64 comparison to 1e-9 (local 1e-10)",
            "n_points": 17070, "solves_per_step": 6, "pair_sums": "FP32C (compensated)",
            "krylov": "FP64", "bjs": "implicit", "l2": "flushed before every timed step (inputs 1.4 MB < L2)"}


def ddm_prm(ssd, kappa, alpha, prec, maxit_outer=200):
    # one Krylov cycle per local solve (restart = maxit): in FP32C a restart
    # recomputes the true residual, which sits at the pair-sum rounding level
    tol_outer, tol_inner = TOL["fp32c" if prec == ssd.FP32C else "fp64"]
    inner = ssd.krylov(tol_inner, 256, 256, False, prec, deflate=True)
    return ssd.ddm_params(mu=1.0, kappa=kappa, gamma=alpha, uinf=(0.0, 0.0, 1.0), delta=3 * H,
                          theta=0.5 * min(kappa, 1.0), tol_outer=tol_outer, maxit_outer=maxit_outer,
                          outer_gmres=True, traction_mode=ssd.TRACTION_BJS, bjs_sign=1.0, inner=inner,
                          bjs_implicit=True)


class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, throttle reasons)."""

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            if len(r) >= 9:
                for k, nm in enumerate(names):
                    if r[5 + k].lower().startswith("active"):
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def near_fraction(xyz, delta, rng_seed=7, sample=1024):
    """Fraction of ordered pairs with r < RHO_FAR * delta (sampled targets)."""
    n = xyz.shape[1]
    idx = np.random.default_rng(rng_seed).choice(n, min(sample, n), replace=False)
    d2 = ((xyz[:, idx, None] - xyz[:, None, :]) ** 2).sum(0)
    return float((d2 < (RHO_FAR * delta) ** 2).mean())


def oracle_pair_rate(budget_s, xyz, nrm, w, delta):
    """FP64 oracle pair rate (pairs/s) on sampled target rows of the two
    double layers (the dominant operators), repeated for about budget_s."""
    import oracle
    pts = {"xyz": xyz, "nrm": nrm, "w": w}
    n = w.size
    rows = np.arange(0, n, 64)
    rng = np.random.default_rng(12345)
    u = rng.normal(size=(3, n))
    p = rng.normal(size=n)
    pairs, t0 = 0.0, time.perf_counter()
    calls = 0
    while True:
        oracle.stokes_dl(pts, delta, u, rows=rows)
        oracle.laplace_dl(pts, delta, p, rows=rows)
        pairs += 2.0 * rows.size * n
        calls += 1
        el = time.perf_counter() - t0
        if el >= budget_s:
            break
    return pairs / el, {"cores": oracle.num_threads(),
                        "sample": "%d x (Stokes DL + Laplace DL) on every 64th target row (%d rows x %d sources)"
                                  % (calls, rows.size, n)}


def oracle_single_thread_rate(budget_s, xyz, nrm, w, delta):
    """The same sampled oracle work on one OpenMP thread (thread count restored after)."""
    import oracle
    cores = oracle.num_threads()
    oracle.set_num_threads(1)
    try:
        rate, info = oracle_pair_rate(budget_s, xyz, nrm, w, delta)
    finally:
        oracle.set_num_threads(cores)
    return {"value": rate, "cores": info["cores"], "sample": info["sample"]}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    from oracle import quadrature as Q
    oracle.build()
    pts = Q.sphere_points(1.0, H)
    for _ in range(args.warmup):
        oracle_pair_rate(0.0, pts["xyz"], pts["nrm"], pts["w"], 3 * H)
    t0 = time.perf_counter()
    pairs = 0.0
    info = None
    for _ in range(args.steps):
        rate, info = oracle_pair_rate(0.0, pts["xyz"], pts["nrm"], pts["w"], 3 * H)
        pairs += 2.0 * len(range(0, pts["w"].size, 64)) * pts["w"].size
    el = time.perf_counter() - t0
    value = pairs / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": info["cores"], "kind": "oracle",
                             "sample": "per step: " + info["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def combine_ranks(ms, pairs, dist, device):
    """Whole-job figures: the slowest rank's time and the pairs of all ranks
    (identity without a process group)."""
    if dist is None:
        return ms, pairs
    import torch
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    pt = torch.tensor([pairs], device=device, dtype=torch.float64)
    dist.all_reduce(pt)
    return float(t.item()), float(pt.item())


def run_ours(args):
    import torch
    import paper_2110_10749_gb300 as ssd

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    ctx = ssd.Context(local)
    # inputs: quadrature points generated on the device (our kernel)
    q = ssd.quadrature_points(ctx, ssd.SPHERE, (1.0,), H)
    P = ssd.Points(q["xyz"], q["nrm"], q["w"]).prepare(ctx)
    n = P.n
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def one_step(prec):
        outs = []
        for kappa in KAPPAS:
            for alpha in ALPHAS:
                outs.append(ssd.ddm_solve(ctx, P, ddm_prm(ssd, kappa, alpha, prec), raise_on_notconv=False))
        return outs

    # plain FP64 reference solves on the GPU (untimed for the metric; timed per solve)
    fp64 = {}
    if not args.skip_fp64:
        for kappa in (KAPPAS if args.fp64_all else KAPPAS[:2]):
            for alpha in ALPHAS:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                r = ssd.ddm_solve(ctx, P, ddm_prm(ssd, kappa, alpha, ssd.FP64), raise_on_notconv=False)
                torch.cuda.synchronize()
                fp64[(kappa, alpha)] = (r, time.perf_counter() - t0)
    for _ in range(args.warmup):
        one_step(ssd.FP32C)
    # timed region
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ctx.reset_stats()
    ctx.set_timing(True)
    sampler = ClockSampler(local)
    sampler.start()
    l0 = ctx.launch_count()
    total_ms = 0.0
    per_solve = []
    last = None
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        outs = []
        for kappa in KAPPAS:
            for alpha in ALPHAS:
                s0 = torch.cuda.Event(enable_timing=True)
                s1 = torch.cuda.Event(enable_timing=True)
                s0.record(stream)
                outs.append(ssd.ddm_solve(ctx, P, ddm_prm(ssd, kappa, alpha, ssd.FP32C), raise_on_notconv=False))
                s1.record(stream)
                per_solve.append((s0, s1, kappa, alpha))
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        last = outs
    torch.cuda.synchronize()
    launches = ctx.launch_count() - l0
    clocks = sampler.stop()
    ctx.set_timing(False)
    stats = {k: ctx.kernel_stats(k, ssd.FP32C) for k in range(6)}
    pairs_total = sum(s["pairs"] for s in stats.values())
    total_ms, pairs_all = combine_ranks(total_ms, pairs_total, dist, dev)
    value = pairs_all / (total_ms / 1e3)

    # time-to-solution and FP32C-vs-FP64 errors per solve
    tts = {}
    for (s0, s1, kappa, alpha) in per_solve:
        tts.setdefault((kappa, alpha), []).append(s0.elapsed_time(s1))
    solves = []
    for k, (kappa, alpha) in enumerate([(a, b) for a in KAPPAS for b in ALPHAS]):
        r32 = last[k]
        row = {"kappa": kappa, "alpha": alpha, "status": r32["status"], "outer_its": r32["outer_its"],
               "outer_relres": r32["hist"][0] if r32["hist"] else None,
               "fp32c_ms": statistics.median(tts[(kappa, alpha)]), "drag_z": float(r32["drag"][2])}
        if (kappa, alpha) in fp64:
            r64, t64 = fp64[(kappa, alpha)]
            row["fp64_ms"] = 1e3 * t64
            row["fp64_outer_its"] = r64["outer_its"]
            row["fp64_status"] = r64["status"]
            for key in ("q", "p", "u", "f"):
                a, b = r32[key], r64[key]
                row["relerr_%s" % key] = float(torch.linalg.norm(a - b) / torch.linalg.norm(b))
            # velocity against the far-field speed (the surface velocity is ~kappa U)
            row["err_u_vs_U"] = float(torch.linalg.norm(r32["u"] - r64["u"]) / math.sqrt(n))
        solves.append(row)

    # dominant kernel: the fused/Stokes double layer (FP32C) -- roofline against FP32 peak
    dom_cls = max(stats, key=lambda c: stats[c]["ms"])
    dom = stats[dom_cls]
    names = ["laplace_SL", "laplace_DL", "stokes_SL", "stokes_DL", "stokes_SLDL", "laplace_SLDL"]
    xyz_h = q["xyz"].cpu().numpy()
    fnear = near_fraction(xyz_h, 3 * H)
    flops_pair = FLOPS_SDL_FAR * (1 - fnear) + FLOPS_SDL_NEAR * fnear
    if dom_cls == ssd.K_STOKES_SLDL:
        flops_pair += 15  # single-layer terms shared with the double layer pass
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    peak = sms * 128 * 2 * 2070e6 / 1e12
    achieved = dom["pairs"] * flops_pair / (dom["ms"] / 1e3) / 1e12 if dom["ms"] > 0 else 0.0
    # DRAM bytes (read + write) per launch of the fused Stokes kernel on this
    # workload, from one ncu capture (the sources stay in L2 between launches)
    traffic = DRAM_BYTES_SSLDL if dom_cls == ssd.K_STOKES_SLDL else None
    roofline = {"bound": "alu", "kernel": "pair32_kernel<%s> (FP32C, packed f32x2)" % names[dom_cls],
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                "flops_per_pair": flops_pair, "near_fraction": fnear,
                "launches": dom["launches"], "avg_launch_ms": dom["ms"] / max(dom["launches"], 1),
                "share_of_step": dom["ms"] / total_ms if total_ms > 0 else None,
                "peak_note": "FP32 FMA peak = %d SMs x 128 lanes x 2 flop x 2070 MHz (unit counts and max clock)"
                             % sms}

    # end to end through the C ABI with host buffers (pinned), copies inside
    xyz_p = q["xyz"].cpu().pin_memory()
    nrm_p = q["nrm"].cpu().pin_memory()
    w_p = q["w"].cpu().pin_memory()
    outs_h = [{"q": torch.empty(n, dtype=torch.float64).pin_memory(),
               "p": torch.empty(n, dtype=torch.float64).pin_memory(),
               "u": torch.empty((3, n), dtype=torch.float64).pin_memory(),
               "f": torch.empty((3, n), dtype=torch.float64).pin_memory()} for _ in range(6)]
    e2e_ms = 0.0
    e2e_steps = max(1, min(args.steps, 3))
    ctx.reset_stats()
    ctx.set_timing(True)
    for _ in range(e2e_steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        k = 0
        for kappa in KAPPAS:
            for alpha in ALPHAS:
                ssd.ddm_solve_host(ctx, xyz_p, nrm_p, w_p, ddm_prm(ssd, kappa, alpha, ssd.FP32C), out=outs_h[k],
                                   raise_on_notconv=False)
                k += 1
        torch.cuda.synchronize()
        e2e_ms += 1e3 * (time.perf_counter() - t0)
    ctx.set_timing(False)
    e2e_pairs = sum(ctx.kernel_stats(c, ssd.FP32C)["pairs"] for c in range(6))
    e2e_ms, e2e_pairs = combine_ranks(e2e_ms, e2e_pairs, dist, dev)
    e2e = {"value": e2e_pairs / (e2e_ms / 1e3), "unit": UNIT,
           "h2d_bytes_per_step": 6 * 7 * n * 8, "d2h_bytes_per_step": 6 * 8 * n * 8,
           "note": "ssd_ddm_solve_host per solve: host->device copy of the points, layout build, "
                   "solve, device->host copy of q, p, u, f"}

    cpu = None
    if rank == 0 and not args.skip_cpu:
        nrm_h, w_h = q["nrm"].cpu().numpy(), q["w"].cpu().numpy()
        rate, info = oracle_pair_rate(args.cpu_seconds, xyz_h, nrm_h, w_h, 3 * H)
        cpu = {"value": rate, "unit": UNIT, "cores": info["cores"], "kind": "oracle", "sample": info["sample"],
               "single_thread": oracle_single_thread_rate(0.25 * args.cpu_seconds, xyz_h, nrm_h, w_h, 3 * H)}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "precision": "FP32 pair terms with compensated accumulation; FP64 Krylov, interface and epilogue",
                "data": "synthetic", "config": workload_config(), "clocks": clocks, "gpu_launches": launches,
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "kernels": {names[c]: stats[c] for c in stats if stats[c]["launches"]},
                "solves": solves}
        print(json.dumps(line), flush=True)
    P.release()
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--skip-fp64", action="store_true", help="skip the plain FP64 GPU comparison solves")
    ap.add_argument("--fp64-all", action="store_true",
                    help="FP64 comparison for all six solves (kappa = 1e-4 takes minutes); default kappa >= 1e-2")
    ap.add_argument("--skip-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
