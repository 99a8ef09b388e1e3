"""BJS-slip D-N solves on the device with the slip lagged one sweep, as
Section 3 (step 2) and Section 6 (step (c)) print it: one sweep against the
oracle's, the kappa = 1e-4, gamma = 1 solve at h = 1/16 against the oracle's
stored solution (tests/golden/bjs_lagged_sphere_h16.txt), and the six
kappa x gamma solves of the h = 1/32 sphere in FP32C against the porous
sphere with slip (closed form in oracle/analytic.py)."""
import math

import numpy as np
import pytest

from conftest import read_golden
from oracle import analytic as A
from oracle import quadrature as Q
from oracle import solvers as S

pytestmark = pytest.mark.gpu


def T(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _prm(ssd, h, kappa, gamma, prec, tol_outer, tol_inner, maxit=600, uinf=(0.0, 0.0, 1.0), deflate=False,
         refine=0):
    inner = ssd.krylov(tol_inner, 256, 256, False, prec, deflate=deflate)
    return ssd.ddm_params(mu=1.0, kappa=kappa, gamma=gamma, uinf=uinf, delta=3 * h, theta=0.5 * min(kappa, 1.0),
                          tol_outer=tol_outer, maxit_outer=maxit, outer_gmres=True, traction_mode=ssd.TRACTION_BJS,
                          bjs_sign=1.0, inner=inner, bjs_implicit=False, refine=refine)


def test_one_sweep_matches_oracle(gpu_ctx):
    import paper_2110_10749_gb300 as ssd
    h, kappa, gamma = 1 / 8, 1e-2, 1.0
    p = Q.sphere_points(1.0, h)
    x, y, z = p["xyz"]
    rng = np.random.default_rng(5)
    q = np.cos(2 * x) * y + 0.3 * z + 0.01 * rng.normal(size=x.size)
    q -= (p["w"] @ q) / p["w"].sum()
    u_prev = np.stack([y * z, np.cos(x), x + 0.3 * z * z])
    uinf = (0.3, 0.0, 1.0)
    # the oracle's sweep, step by step (Section 6, steps (a)-(f))
    pd, _, _ = S.darcy_solve(p, 3 * h, 1.0, kappa, q, tol=1e-13)
    f = S.traction_bjs(p, pd, u_prev, kappa, gamma)
    u, _, _ = S.stokes_solve(p, 3 * h, 1.0, f, uinf, tol=1e-13)
    theta = 0.5 * kappa
    qn = (1 - theta) * q + theta * (u * p["nrm"]).sum(0)
    P = ssd.Points.from_numpy(p).prepare(gpu_ctx)
    ref = {"q": qn, "p": pd, "u": u, "f": f}
    for prec, tol, tol_in in ((ssd.FP64, 1e-10, 1e-13), (ssd.FP32C, 1e-5, 1e-9)):
        o = ssd.ddm_sweep(gpu_ctx, P, _prm(ssd, h, kappa, gamma, prec, 1e-8, tol_in, uinf=uinf), T(q), T(u_prev))
        assert o["status"] == ssd.SSD_OK and min(o["inner_its"]) > 0
        for k, v in ref.items():
            a = o[k].cpu().numpy()
            assert np.linalg.norm(a - v) / np.linalg.norm(v) < tol, (prec, k)
    # u_prev = NULL is the zero state; the Darcy solve with q = 0 takes no step
    o = ssd.ddm_sweep(gpu_ctx, P, _prm(ssd, h, kappa, gamma, ssd.FP64, 1e-8, 1e-13), T(np.zeros_like(q)))
    assert o["inner_its"][0] == 0 and np.abs(o["p"].cpu().numpy()).max() == 0.0
    P.release()


def _golden():
    rows = read_golden("bjs_lagged_sphere_h16.txt")
    drag = np.array([float(v) for v in rows[0][1:]])
    its = int(rows[1][1])
    data = np.array([[float(v) for v in r] for r in rows[2:]])
    return drag, its, data[:, 0].astype(int), data[:, 1:]


def test_lagged_kappa_1e4_matches_oracle_h16(gpu_ctx):
    # the hardest C2 case (gamma/sqrt(kappa) = 100) at h = 1/16: the device's
    # FP64 solve against the oracle's, FP32C against FP64, both against the
    # closed form at the discretization level
    import paper_2110_10749_gb300 as ssd
    h, kappa, gamma = 1 / 16, 1e-4, 1.0
    p = Q.sphere_points(1.0, h)
    P = ssd.Points.from_numpy(p).prepare(gpu_ctx)
    drag_o, its_o, idx, fo = _golden()
    r64 = ssd.ddm_solve(gpu_ctx, P, _prm(ssd, h, kappa, gamma, ssd.FP64, 1e-11, 1e-13))
    # FP32C against FP64 with the Stokes normal mode deflated in both: FP32
    # rounding along the near-null normal mode is otherwise amplified by the
    # inverse of its O(h^5) eigenvalue
    d64 = ssd.ddm_solve(gpu_ctx, P, _prm(ssd, h, kappa, gamma, ssd.FP64, 1e-10, 1e-11, deflate=True))
    r32 = ssd.ddm_solve(gpu_ctx, P, _prm(ssd, h, kappa, gamma, ssd.FP32C, 1e-9, 1e-10, deflate=True, refine=4))
    assert r64["status"] == 0 and r32["status"] == 0 and d64["status"] == 0
    assert abs(r64["outer_its"] - its_o) <= max(3, its_o // 20)
    assert np.abs(r64["drag"] - drag_o).max() < 1e-8 * abs(drag_o[2])
    dev = np.concatenate([r64["q"].cpu().numpy()[None, idx], r64["p"].cpu().numpy()[None, idx],
                          r64["u"].cpu().numpy()[:, idx]])
    # q = u.n is O(kappa U): compared against U; p and u against their size
    assert np.abs(dev[0] - fo[:, 0]).max() < 1e-9
    for k in range(1, 5):
        assert np.abs(dev[k] - fo[:, k]).max() < 1e-8 * np.abs(fo[:, k]).max(), k
    for k in ("p", "u", "f"):
        a, b = r32[k].cpu().numpy(), d64[k].cpu().numpy()
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-5, k
    # q = u.n is O(kappa U): compare it against U
    assert S.rms(r32["q"].cpu().numpy() - d64["q"].cpu().numpy()) < 1e-7
    # the refined FP32C solve ends on an FP64 residual below its tolerance
    assert r32["hist"][-1] <= 1e-9 and r32["hist"][-2] > r32["hist"][-1]
    assert abs(r32["drag"][2] - drag_o[2]) < 1e-6 * drag_o[2]
    d = A.bjs_drag(1.0, kappa, gamma, 1.0, 1.0)
    assert abs(r64["drag"][2] - d) < 1e-4 * d
    # the interface GMRES residual history: one estimate per step, ending below tol
    hist = r64["hist"]
    assert len(hist) == r64["outer_its"] and hist[-1] <= 1e-11 and hist[0] > hist[-1]
    P.release()


def test_six_c2_solves_converge_to_the_slip_sphere(gpu_ctx):
    # unit sphere h = 1/32 (N = 17070), kappa in {1, 1e-2, 1e-4} x gamma in
    # {0.1, 1}, FP32C pair sums with FP64-residual refinement, interface
    # GMRES to 1e-8; errors against the closed form at the discretisation
    # level of h = 1/32
    import paper_2110_10749_gb300 as ssd
    h = 1 / 32
    g = ssd.quadrature_points(gpu_ctx, ssd.SPHERE, (1.0,), h)
    P = ssd.Points(g["xyz"], g["nrm"], g["w"]).prepare(gpu_ctx)
    xyz = g["xyz"].cpu().numpy()
    for kappa in (1.0, 1e-2, 1e-4):
        for gamma in (0.1, 1.0):
            r = ssd.ddm_solve(gpu_ctx, P, _prm(ssd, h, kappa, gamma, ssd.FP32C, 1e-8, 1e-9, deflate=True, refine=4))
            assert r["status"] == 0, (kappa, gamma)
            d = A.bjs_drag(1.0, kappa, gamma, 1.0, 1.0)
            assert abs(r["drag"][2] - d) < 3e-6 * d, (kappa, gamma, r["drag"][2], d)
            q, pd, u, f = A.bjs_interface_fields(xyz, 1.0, kappa, gamma, 1.0, (0.0, 0.0, 1.0))
            assert S.rms(r["u"].cpu().numpy() - u) < 2e-4, (kappa, gamma)
            assert S.rms(r["p"].cpu().numpy() - pd) < 2e-4 * S.rms(pd), (kappa, gamma)
    P.release()
