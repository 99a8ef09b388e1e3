"""Operator micro-benchmark: pair-interactions/s of each layer operator.

    python -m paper_2110_10749_gb300.opbench --surface sphere --h 1/32 \
        --ops stokes_DL,laplace_DL --prec fp32c --reps 20
    python -m paper_2110_10749_gb300.opbench --surface ellipsoid --h 1/128 --sweep --reps 3

With --sweep, times whole D-N sweeps (ssd_ddm_sweep) of the porous-body
problem with the lagged BJS slip (kappa = 1e-3, gamma = 1, theta = kappa/2,
U = e_z, local GMRES to 1e-9) from the state one sweep from zero reaches,
and prints the pair-interactions/s of each kernel class over those sweeps.

Builds the quadrature points on the device, prepares the sorted layout and
times every requested operator application with CUDA events on the current
stream (L2 flushed before each application; the pair kernels alone, through
the library's own event timing).  Prints one JSON line per operator.
"""
from __future__ import annotations

import argparse
import json
import sys
from fractions import Fraction

OPS = ("laplace_SL", "laplace_DL", "stokes_SL", "stokes_DL", "stokes_SLDL", "laplace_SLDL")


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--surface", default="sphere", choices=["sphere", "ellipsoid"])
    ap.add_argument("--abc", default="1,0.7,0.5")
    ap.add_argument("--h", default="1/32")
    ap.add_argument("--ops", default=",".join(OPS))
    ap.add_argument("--prec", default="fp32c", choices=["fp32c", "fp64"])
    ap.add_argument("--reps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--peak", action="store_true", help="also measure the FP32 FMA rate (FFMA and FFMA2)")
    ap.add_argument("--sweep", action="store_true", help="time D-N sweeps instead of single operators")
    args = ap.parse_args(argv)

    import torch
    import paper_2110_10749_gb300 as ssd

    h = float(Fraction(args.h))
    ctx = ssd.Context(0)
    if args.surface == "sphere":
        q = ssd.quadrature_points(ctx, ssd.SPHERE, (1.0,), h)
    else:
        q = ssd.quadrature_points(ctx, ssd.ELLIPSOID, tuple(float(v) for v in args.abc.split(",")), h)
    P = ssd.Points(q["xyz"], q["nrm"], q["w"]).prepare(ctx)
    n = P.n
    prec = ssd.FP32C if args.prec == "fp32c" else ssd.FP64
    gen = torch.Generator(device="cuda").manual_seed(12345)
    g = torch.randn(n, dtype=torch.float64, device="cuda", generator=gen)
    v = torch.randn((3, n), dtype=torch.float64, device="cuda", generator=gen)
    v2 = torch.randn((3, n), dtype=torch.float64, device="cuda", generator=gen)
    delta = 3 * h
    call = {
        "laplace_SL": lambda: ssd.laplace_SL(ctx, P, delta, g, prec),
        "laplace_DL": lambda: ssd.laplace_DL(ctx, P, delta, g, prec),
        "stokes_SL": lambda: ssd.stokes_SL(ctx, P, delta, 1.0, v, prec),
        "stokes_DL": lambda: ssd.stokes_DL(ctx, P, delta, v, prec),
        "stokes_SLDL": lambda: ssd.stokes_SLDL(ctx, P, delta, 1.0, v2, v, 1.0, -1.0, prec),
        "laplace_SLDL": lambda: ssd.laplace_SLDL(ctx, P, delta, g, g, 1.0, -1.0, prec),
    }
    cls = dict(zip(OPS, range(6)))
    if args.sweep:
        inner = ssd.krylov(1e-9, 256, 256, False, prec, deflate=True)
        prm = ssd.ddm_params(mu=1.0, kappa=1e-3, gamma=1.0, uinf=(0.0, 0.0, 1.0), delta=delta, theta=5e-4,
                             tol_outer=1e-8, maxit_outer=64, outer_gmres=True, traction_mode=ssd.TRACTION_BJS,
                             inner=inner)
        zero = torch.zeros(n, dtype=torch.float64, device="cuda")
        first = ssd.ddm_sweep(ctx, P, prm, zero)
        q1, u1 = first["q"].clone(), first["u"].clone()
        for _ in range(args.warmup):
            ssd.ddm_sweep(ctx, P, prm, q1, u1)
        torch.cuda.synchronize()
        ctx.reset_stats()
        ctx.set_timing(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.reps):
            o = ssd.ddm_sweep(ctx, P, prm, q1, u1)
        e1.record()
        e1.synchronize()
        ctx.set_timing(False)
        step_ms = e0.elapsed_time(e1) / args.reps
        for name, k in cls.items():
            st = ctx.kernel_stats(k, prec)
            if st["launches"]:
                print(json.dumps({"sweep": True, "op": name, "n": n, "launches_per_sweep": st["launches"] / args.reps,
                                  "ms_per_sweep": st["ms"] / args.reps, "share_of_sweep": st["ms"] / args.reps / step_ms,
                                  "pairs_per_s": st["pairs"] / (st["ms"] / 1e3)}), flush=True)
        print(json.dumps({"sweep": True, "ms_per_sweep": step_ms, "local_steps": list(o["inner_its"])}), flush=True)
        P.release()
        ctx.close()
        return 0
    if args.peak:
        props = torch.cuda.get_device_properties(0)
        for packed in (0, 1):
            print(json.dumps({"fp32_fma_rate_tflops": ctx.fp32_fma_rate(bool(packed)),
                              "form": "FFMA2 (f32x2)" if packed else "FFMA", "sms": props.multi_processor_count}),
                  flush=True)
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")
    for name in args.ops.split(","):
        for _ in range(args.warmup):
            call[name]()
        torch.cuda.synchronize()
        ctx.reset_stats()
        ctx.set_timing(True)
        for _ in range(args.reps):
            flush.fill_(1.0)
            call[name]()
        torch.cuda.synchronize()
        ctx.set_timing(False)
        st = ctx.kernel_stats(cls[name], prec)
        ms = st["ms"] / max(st["launches"], 1)
        print(json.dumps({"op": name, "prec": args.prec, "n": n, "launches": st["launches"],
                          "ms_per_launch": ms, "pairs_per_s": st["pairs"] / (st["ms"] / 1e3)}), flush=True)
    P.release()
    ctx.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
