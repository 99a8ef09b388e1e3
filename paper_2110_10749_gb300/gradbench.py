"""Differentiation workload: adjoint gradients of the D-N solve on the sphere.

    python -m paper_2110_10749_gb300.gradbench [--h 1/32] [--kappa 1e-2] [--gamma 1]
        [--fd-params log_kappa,gamma,c0,c2,c6] [--step 1e-4]

On the unit sphere written as a star surface (all c_lm = 0) at spacing h:
J = drag along the flow and J = first moment of the interface flux, each with
dJ/dlog(kappa), dJ/dgamma and dJ/dc_lm (25 coefficients) from one forward
and one adjoint solve (FP64 pair sums, implicit BJS, interface GMRES to
1e-12, local GMRES to 1e-13).  Central differences of FP64 forward solves
check the parameters named by --fd-params.  Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import sys
import time
from fractions import Fraction


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--h", default="1/32")
    ap.add_argument("--kappa", type=float, default=1e-2)
    ap.add_argument("--gamma", type=float, default=1.0)
    ap.add_argument("--fd-params", default="log_kappa,gamma,c0,c2,c6")
    ap.add_argument("--step", type=float, default=1e-4)
    ap.add_argument("--tol", type=float, default=1e-12)
    args = ap.parse_args(argv)

    import numpy as np
    import torch
    import paper_2110_10749_gb300 as ssd

    h = float(Fraction(args.h))
    ctx = ssd.Context(0)

    def prm_of(kappa, gamma):
        inner = ssd.krylov(0.1 * args.tol, 256, 256, False, ssd.FP64, True)
        return ssd.ddm_params(mu=1.0, kappa=kappa, gamma=gamma, uinf=(0.0, 0.0, 1.0), delta=3 * h, theta=1.0,
                              tol_outer=args.tol, maxit_outer=200, outer_gmres=True,
                              traction_mode=ssd.TRACTION_BJS, inner=inner, bjs_implicit=True)

    clm0 = np.zeros(25)

    def J_of(clm, kappa, gamma, func):
        q = ssd.quadrature_points(ctx, ssd.STAR, h=h, clm=clm)
        P = ssd.Points(q["xyz"], q["nrm"], q["w"]).prepare(ctx)
        r = ssd.ddm_solve(ctx, P, prm_of(kappa, gamma), raise_on_notconv=False)
        if func == ssd.FUNC_DRAG:
            val = float(r["drag"][2])
        else:
            val = float((q["w"] * r["q"] * q["xyz"][2]).sum())
        P.release()
        return val

    res = {}
    for fname, func in (("drag", ssd.FUNC_DRAG), ("flux", ssd.FUNC_FLUX)):
        torch.cuda.synchronize()
        t0 = time.time()
        J, g, dc, st = ssd.ddm_shape_gradient(ctx, clm0, h, prm_of(args.kappa, args.gamma), func)
        torch.cuda.synchronize()
        t_grad = time.time() - t0
        t0 = time.time()
        Jf = J_of(clm0, args.kappa, args.gamma, func)
        torch.cuda.synchronize()
        t_fwd = time.time() - t0
        adj = {"log_kappa": g[0], "gamma": g[1]}
        for k in range(25):
            adj["c%d" % k] = dc[k]
        fd = {}
        e = args.step
        for name in [s for s in args.fd_params.split(",") if s]:
            if name == "log_kappa":
                jp = J_of(clm0, args.kappa * math.exp(e), args.gamma, func)
                jm = J_of(clm0, args.kappa * math.exp(-e), args.gamma, func)
            elif name == "gamma":
                jp = J_of(clm0, args.kappa, args.gamma + e, func)
                jm = J_of(clm0, args.kappa, args.gamma - e, func)
            else:
                k = int(name[1:])
                cp, cm = clm0.copy(), clm0.copy()
                cp[k] += e
                cm[k] -= e
                jp = J_of(cp, args.kappa, args.gamma, func)
                jm = J_of(cm, args.kappa, args.gamma, func)
            d = (jp - jm) / (2 * e)
            scale = max(abs(d), abs(J))
            fd[name] = {"fd": d, "adjoint": adj[name], "rel_err": abs(adj[name] - d) / scale}
        res[fname] = {"J": J, "J_forward_only": Jf, "status": st, "seconds_gradient": t_grad,
                      "seconds_forward": t_fwd, "grad": adj, "fd_check": fd,
                      "max_rel_err": max(v["rel_err"] for v in fd.values()) if fd else None}
    out = {"workload": "unit sphere as a star surface (c_lm = 0), h=%s, delta=3h, kappa=%g, gamma=%g, BJS implicit, "
                       "FP64, interface tol %g" % (args.h, args.kappa, args.gamma, args.tol),
           "fd_step": args.step, "results": res}
    print(json.dumps(out), flush=True)
    ctx.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
