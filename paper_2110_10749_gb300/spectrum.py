"""Eigenvalues of the discrete D-N iteration matrix (eq. A_mat, Fig. 5).

    python -m paper_2110_10749_gb300.spectrum --h 1/16 --kappas 1,1e-2,1e-4 --first 50

Assembles A~ on the device column by column (ssd_ddm_iteration_matrix: one
D-N sweep per column, porous-sphere problem with gamma = 0 on the unit
sphere, theta = kappa/2 as in Table 2's first column) and takes its
eigenvalues on the host (LAPACK through numpy).  Prints one JSON line per
kappa with the `first` eigenvalues in increasing order of their real part
(the lowest spherical-harmonic degrees first) and, for comparison, the
degree-one closed form (1 - theta) - theta R^2 / (3 kappa).
"""
from __future__ import annotations

import argparse
import json
import sys
import time
from fractions import Fraction

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--h", default="1/16")
    ap.add_argument("--kappas", default="1,1e-2,1e-4")
    ap.add_argument("--first", type=int, default=50)
    ap.add_argument("--prec", default="fp32c", choices=["fp32c", "fp64"])
    args = ap.parse_args(argv)

    import torch
    import paper_2110_10749_gb300 as ssd

    h = float(Fraction(args.h))
    ctx = ssd.Context(0)
    q = ssd.quadrature_points(ctx, ssd.SPHERE, (1.0,), h)
    P = ssd.Points(q["xyz"], q["nrm"], q["w"]).prepare(ctx)
    prec = ssd.FP32C if args.prec == "fp32c" else ssd.FP64
    for kappa in (float(k) for k in args.kappas.split(",")):
        theta = 0.5 * min(kappa, 1.0)
        inner = ssd.krylov(1e-9 if prec == ssd.FP32C else 1e-12, 256, 256, False, prec, False)
        prm = ssd.ddm_params(mu=1.0, kappa=kappa, gamma=0.0, uinf=(0.0, 0.0, 1.0), delta=3 * h, theta=theta,
                             tol_outer=1e-9, maxit_outer=100, outer_gmres=True, traction_mode=ssd.TRACTION_BJS,
                             inner=inner)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        A = ssd.ddm_iteration_matrix(ctx, P, prm).cpu().numpy()
        t_asm = time.perf_counter() - t0
        t0 = time.perf_counter()
        ev = np.linalg.eigvals(A)
        t_eig = time.perf_counter() - t0
        ev = ev[np.argsort(ev.real)]
        print(json.dumps({"kappa": kappa, "theta": theta, "n": P.n, "prec": args.prec,
                          "assembly_s": t_asm, "eig_s": t_eig, "max_imag": float(np.abs(ev.imag).max()),
                          "degree_one_closed_form": (1 - theta) - theta / (3 * kappa),
                          "first": [float(v) for v in ev.real[:args.first]]}), flush=True)
    P.release()
    ctx.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
