"""Batched workload: many star-shaped surfaces and ellipsoids in one launch.

    python -m paper_2110_10749_gb300.batchbench [--n-star 64] [--n-ellipsoid 8] [--reps 3]
        [--ddm-surfaces 8]

The surfaces follow the seeded recipe of ``workloads.batch_recipe`` (star
coefficients c_lm ~ N(0, 0.05^2), ellipsoids (1, 0.8, 0.6), h drawn from
{1/16, 1/24, 1/32, 1/48}, delta = 3h, four far fields each).  Points come
from the device quadrature.  Timed with CUDA events on the current stream:

  * one batched FP32C application of the fused Stokes SL+DL (the implicit-BJS
    matvec) and of the Laplace DL (the Darcy matvec) over every surface and
    right-hand side, as pair-interactions/s;
  * the batched D-N solve (implicit BJS, kappa = 1e-2, gamma = 0.1, interface
    GMRES to 1e-8, local GMRES to 1e-9, FP32C pair sums) of the first
    --ddm-surfaces surfaces with their four far fields, as time-to-solution.

Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import sys
import time


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n-star", type=int, default=64)
    ap.add_argument("--n-ellipsoid", type=int, default=8)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--ddm-surfaces", type=int, default=8)
    args = ap.parse_args(argv)

    import numpy as np
    import torch
    import paper_2110_10749_gb300 as ssd
    from paper_2110_10749_gb300 import workloads

    ctx = ssd.Context(0)
    recipe = workloads.batch_recipe(args.n_star, args.n_ellipsoid)
    uinf = np.array(workloads.FAR_FIELDS)
    t0 = time.time()
    pts = []
    for s in recipe:
        if s["kind"] == "star":
            q = ssd.quadrature_points(ctx, ssd.STAR, h=s["h"], clm=s["clm"])
        else:
            q = ssd.quadrature_points(ctx, ssd.ELLIPSOID, s["abc"], s["h"])
        pts.append(q)
    torch.cuda.synchronize()
    t_quad = time.time() - t0

    def make_batch(sel):
        ns = [int(pts[k]["w"].numel()) for k in sel]
        offs = np.concatenate([[0], np.cumsum(ns)])
        cat = lambda key: torch.cat([pts[k][key] for k in sel], dim=-1).contiguous()
        b = ssd.Batch(cat("xyz"), cat("nrm"), cat("w"), offs, [3 * recipe[k]["h"] for k in sel]).prepare(ctx)
        return b, ns

    allsel = list(range(len(recipe)))
    B, ns = make_batch(allsel)
    n_total = B.n
    pairs_per_rhs = float(sum(float(n) * n for n in ns))
    nrhs = uinf.shape[0]
    gen = torch.Generator(device="cuda").manual_seed(7)
    v = torch.randn((nrhs, 3, n_total), dtype=torch.float64, device="cuda", generator=gen)
    f = torch.randn((nrhs, 3, n_total), dtype=torch.float64, device="cuda", generator=gen)
    g = torch.randn((nrhs, 1, n_total), dtype=torch.float64, device="cuda", generator=gen)
    ops = {}
    for name, call in (("stokes_SLDL", lambda: ssd.batch_apply(ctx, B, ssd.OP_STOKES_SLDL, v, f, 1.0, 1.0, -1.0,
                                                              ssd.FP32C)),
                       ("laplace_DL", lambda: ssd.batch_apply(ctx, B, ssd.OP_LAPLACE_DL, g, None, 1.0, 1.0, 1.0,
                                                             ssd.FP32C))):
        call()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.reps):
            call()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.reps
        ops[name] = {"ms_per_launch": ms, "pairs_per_s": pairs_per_rhs * nrhs / (ms / 1e3)}
    B.release()

    # batched D-N on a subset (every right-hand side)
    sel = allsel[:args.ddm_surfaces]
    Bd, nsd = make_batch(sel)
    inner = ssd.krylov(1e-9, 256, 256, False, ssd.FP32C, deflate=True)
    prm = ssd.ddm_params(mu=1.0, kappa=1e-2, gamma=0.1, theta=5e-3, tol_outer=1e-8, maxit_outer=100,
                         outer_gmres=True, traction_mode=ssd.TRACTION_BJS, bjs_implicit=True, inner=inner)
    ssd.batch_ddm_solve(ctx, Bd, prm, uinf[:1], raise_on_notconv=False)      # warm-up
    torch.cuda.synchronize()
    ctx.reset_stats()
    ctx.set_timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    r = ssd.batch_ddm_solve(ctx, Bd, prm, uinf, raise_on_notconv=False)
    e1.record()
    torch.cuda.synchronize()
    ctx.set_timing(False)
    ms_ddm = e0.elapsed_time(e1)
    pairs_ddm = sum(ctx.kernel_stats(k, ssd.FP32C)["pairs"] for k in range(8))
    Bd.release()
    out = {
        "workload": "%d star surfaces + %d ellipsoids (1,0.8,0.6), h in {1/16,1/24,1/32,1/48}, delta = 3h, "
                    "%d far fields" % (args.n_star, args.n_ellipsoid, nrhs),
        "surfaces": len(recipe), "points_total": n_total, "points_min": min(ns), "points_max": max(ns),
        "pairs_per_application": pairs_per_rhs * nrhs, "quadrature_s": t_quad,
        "batched_ops_fp32c": ops,
        "ddm": {"surfaces": len(sel), "rhs": nrhs, "points": int(sum(nsd)), "kappa": 1e-2, "gamma": 0.1,
                "status": r["status"], "ms": ms_ddm, "outer_its_max": int(r["outer_its"].max()),
                "outer_its_mean": float(r["outer_its"].mean()), "relres_max": float(r["relres"].max()),
                "pairs_per_s": pairs_ddm / (ms_ddm / 1e3)},
    }
    print(json.dumps(out), flush=True)
    ctx.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
