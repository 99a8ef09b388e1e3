"""Geometric derivatives: the pair-kernel derivatives in the point data, the
D-N gradient in the point data, and derivatives in the 25 shape coefficients
of a star surface, against central finite differences of the oracle (and of
the device's own FP64 solves where the oracle would take minutes)."""
import math

import numpy as np
import pytest

import oracle
from oracle import quadrature as Q
from oracle import solvers as S
from paper_2110_10749_gb300.workloads import star_coefficients

pytestmark = pytest.mark.gpu

MU = 1.3


def T(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _B(name, p, d, a, b):
    """a . (K b) with K from the oracle's forward operators."""
    if name == "LSL":
        return float((a * oracle.laplace_sl(p, d, b)).sum())
    if name == "LDL":
        return float((a * oracle.laplace_dl(p, d, b)).sum())
    if name == "SSL":
        return float((a * oracle.stokes_sl(p, d, MU, b)).sum())
    return float((a * oracle.stokes_dl(p, d, b)).sum())


def _moved(p, e, dx, dn, dw):
    q = dict(p)
    q["xyz"] = p["xyz"] + e * dx
    q["nrm"] = p["nrm"] + e * dn
    q["w"] = p["w"] + e * dw
    return q


@pytest.mark.parametrize("name", ["LSL", "LDL", "SSL", "SDL"])
def test_pair_geometry_gradient_directional(gpu_ctx, name):
    import paper_2110_10749_gb300 as ssd
    h = 1 / 8
    p = Q.ellipsoid_points((1.0, 0.7, 0.5), h)
    n = p["w"].size
    d = 3 * h
    rng = np.random.default_rng(17)
    nc = 3 if name[0] == "S" else 1
    a = rng.normal(size=(nc, n)) if nc == 3 else rng.normal(size=n)
    b = rng.normal(size=(nc, n)) if nc == 3 else rng.normal(size=n)
    op = {"LSL": ssd.OP_LAPLACE_SL, "LDL": ssd.OP_LAPLACE_DL, "SSL": ssd.OP_STOKES_SL, "SDL": ssd.OP_STOKES_DL}[name]
    P = ssd.Points.from_numpy(p)
    gx, gn, gw = (t.cpu().numpy() for t in ssd.geometry_gradient(gpu_ctx, P, op, d, T(a), T(b), mu=MU))
    eps = 1e-5
    for kind in ("x", "n", "w", "all"):
        dx = rng.normal(size=(3, n)) if kind in ("x", "all") else np.zeros((3, n))
        dn = rng.normal(size=(3, n)) if kind in ("n", "all") else np.zeros((3, n))
        dw = rng.normal(size=n) * p["w"] if kind in ("w", "all") else np.zeros(n)
        fd = (_B(name, _moved(p, eps, dx, dn, dw), d, a, b) - _B(name, _moved(p, -eps, dx, dn, dw), d, a, b)) / (2 * eps)
        ad = float((gx * dx).sum() + (gn * dn).sum() + (gw * dw).sum())
        assert abs(ad - fd) <= 1e-6 * abs(fd), (name, kind, ad, fd)


def _prm(ssd, h, kappa, gamma, tol=1e-12):
    inner = ssd.krylov(0.1 * tol, 400, 100, False, ssd.FP64, True)
    return ssd.ddm_params(mu=1.0, kappa=kappa, gamma=gamma, uinf=(0.0, 0.0, 1.0), delta=3 * h, theta=1.0,
                          tol_outer=tol, maxit_outer=80, outer_gmres=True, traction_mode=ssd.TRACTION_BJS,
                          inner=inner, bjs_implicit=True)


def _oracle_J(p, h, kappa, gamma, func, tol=1e-12):
    r = S.ddm_solve(p, 3 * h, 1.0, kappa, gamma, [0.0, 0.0, 1.0], 1.0, tol=tol, maxit=80, outer="gmres",
                    traction="bjs", restart=100, inner_maxit=400, bjs_implicit=True, deflate=True)
    if func == 0:
        return float(r["drag"][2])
    return float((p["w"] * r["q"] * p["xyz"][2]).sum())


@pytest.mark.parametrize("func", [0, 1])
def test_ddm_geometry_gradient_against_oracle(gpu_ctx, func):
    """Directional derivative of J along a random change of all point data."""
    import paper_2110_10749_gb300 as ssd
    h = 1 / 8
    p = Q.star_points(star_coefficients(2), h)
    n = p["w"].size
    kappa, gamma = 0.1, 0.5
    P = ssd.Points.from_numpy(p).prepare(gpu_ctx)
    J, g, (gx, gn, gw), st = ssd.ddm_gradient_geometry(gpu_ctx, P, _prm(ssd, h, kappa, gamma), func)
    P.release()
    assert st == ssd.SSD_OK
    gx, gn, gw = gx.cpu().numpy(), gn.cpu().numpy(), gw.cpu().numpy()
    rng = np.random.default_rng(5)
    dx, dn, dw = rng.normal(size=(3, n)), rng.normal(size=(3, n)), rng.normal(size=n) * p["w"]
    eps = 1e-5
    fd = (_oracle_J(_moved(p, eps, dx, dn, dw), h, kappa, gamma, func)
          - _oracle_J(_moved(p, -eps, dx, dn, dw), h, kappa, gamma, func)) / (2 * eps)
    ad = float((gx * dx).sum() + (gn * dn).sum() + (gw * dw).sum())
    assert abs(ad - fd) <= 1e-6 * max(abs(fd), abs(J)), (ad, fd)


@pytest.mark.parametrize("seed,func,coefs", [(-1, 0, (0, 2, 6, 13, 20)), (5, 0, (1, 8, 24)), (5, 1, (2, 7))])
def test_shape_gradient_against_oracle(gpu_ctx, seed, func, coefs):
    """dJ/dc_k on a star surface (seed -1: the unit sphere, all c = 0)
    against central differences of the oracle's quadrature + D-N solve."""
    import paper_2110_10749_gb300 as ssd
    h = 1 / 8
    clm = np.zeros(25) if seed < 0 else star_coefficients(seed)
    kappa, gamma = 0.1, 0.5
    J, g, dc, st = ssd.ddm_shape_gradient(gpu_ctx, clm, h, _prm(ssd, h, kappa, gamma), func)
    assert st == ssd.SSD_OK
    assert abs(J - _oracle_J(Q.star_points(clm, h), h, kappa, gamma, func)) <= 1e-9 * abs(J)
    eps = 1e-4
    for k in coefs:
        cp, cm = clm.copy(), clm.copy()
        cp[k] += eps
        cm[k] -= eps
        fd = (_oracle_J(Q.star_points(cp, h), h, kappa, gamma, func)
              - _oracle_J(Q.star_points(cm, h), h, kappa, gamma, func)) / (2 * eps)
        assert abs(dc[k] - fd) <= 1e-6 * max(abs(fd), abs(J)), (k, dc[k], fd)


def test_shape_gradient_all_coefficients_device_fd(gpu_ctx):
    """All 25 coefficients on the unit sphere at h = 1/10 against central
    differences of device FP64 solves on the perturbed surfaces."""
    import paper_2110_10749_gb300 as ssd
    h = 1 / 10
    clm = np.zeros(25)
    kappa, gamma = 1e-2, 1.0
    prm = _prm(ssd, h, kappa, gamma)
    J, g, dc, st = ssd.ddm_shape_gradient(gpu_ctx, clm, h, prm, ssd.FUNC_DRAG)
    assert st == ssd.SSD_OK

    def Jd(c):
        q = ssd.quadrature_points(gpu_ctx, ssd.STAR, h=h, clm=c)
        P = ssd.Points(q["xyz"], q["nrm"], q["w"]).prepare(gpu_ctx)
        r = ssd.ddm_solve(gpu_ctx, P, prm)
        P.release()
        return float(r["drag"][2])

    eps = 1e-4
    scale = max(abs(J), np.abs(dc).max())
    for k in range(25):
        cp, cm = clm.copy(), clm.copy()
        cp[k] += eps
        cm[k] -= eps
        fd = (Jd(cp) - Jd(cm)) / (2 * eps)
        assert abs(dc[k] - fd) <= 1e-6 * scale, (k, dc[k], fd)


def test_shape_autograd(gpu_ctx):
    import torch
    import paper_2110_10749_gb300 as ssd
    h = 1 / 8
    clm = star_coefficients(5)
    prm = _prm(ssd, h, 0.1, 0.5)
    J, g, dc, _ = ssd.ddm_shape_gradient(gpu_ctx, clm, h, prm, ssd.FUNC_FLUX)
    c = torch.tensor(clm, dtype=torch.float64, requires_grad=True)
    lk = torch.tensor(math.log(0.1), dtype=torch.float64, requires_grad=True)
    gm = torch.tensor(0.5, dtype=torch.float64, requires_grad=True)
    out = ssd.ddm_shape_functional(gpu_ctx, c, h, prm, lk, gm, ssd.FUNC_FLUX)
    out.backward()
    assert abs(out.item() - J) <= 1e-12 * abs(J)
    assert np.allclose(c.grad.numpy(), dc, rtol=1e-12, atol=0)
    assert abs(lk.grad.item() - g[0]) <= 1e-12 * abs(g[0])


def test_config4_size_gradients_device_fd(gpu_ctx):
    """The differentiation workload at its own size: the unit sphere at
    h = 1/32 (N = 17070), drag and flux moment differentiated in log(kappa)
    and gamma, and the drag in two shape coefficients, by the adjoint,
    against central differences of device FP64 solves (the oracle would take
    minutes per solve at this size).  With the solves converged to 1e-12 and
    a step of 1e-4 the difference quotient is good to about 1e-8 (rounding
    1e-12 / 1e-4; truncation eps^2 / 6 times the third derivative), so one
    central difference per derivative suffices; each solve gives both
    functionals."""
    import paper_2110_10749_gb300 as ssd
    h = 1 / 32
    clm = np.zeros(25)
    kappa, gamma = 1e-2, 1.0
    prm = _prm(ssd, h, kappa, gamma)
    cache = {}

    def Jd(c, k, gm, func):
        key = (tuple(c), k, gm)
        if key not in cache:
            q = ssd.quadrature_points(gpu_ctx, ssd.STAR, h=h, clm=c)
            P = ssd.Points(q["xyz"], q["nrm"], q["w"]).prepare(gpu_ctx)
            r = ssd.ddm_solve(gpu_ctx, P, _prm(ssd, h, k, gm))
            cache[key] = (float(r["drag"][2]), float((q["w"] * r["q"] * q["xyz"][2]).sum()))
            P.release()
        return cache[key][0 if func == ssd.FUNC_DRAG else 1]

    def central(f, x0, eps=1e-4):
        return (f(x0 + eps) - f(x0 - eps)) / (2 * eps)

    for func in (ssd.FUNC_DRAG, ssd.FUNC_FLUX):
        J, g, dc, st = ssd.ddm_shape_gradient(gpu_ctx, clm, h, prm, func)
        assert st == ssd.SSD_OK
        assert abs(J - Jd(clm, kappa, gamma, func)) <= 1e-10 * abs(J)
        fk = central(lambda lk: Jd(clm, math.exp(lk), gamma, func), math.log(kappa))
        fg = central(lambda gm: Jd(clm, kappa, gm, func), gamma)
        assert abs(g[0] - fk) <= 1e-6 * abs(fk), (func, g[0], fk)
        assert abs(g[1] - fg) <= 1e-6 * abs(fg), (func, g[1], fg)
        if func == ssd.FUNC_FLUX:
            continue
        scale = np.abs(dc).max()
        for k in (0, 6):
            def fc(e, k=k):
                c = clm.copy()
                c[k] = e
                return Jd(c, kappa, gamma, func)
            fd = central(fc, 0.0)
            assert abs(dc[k] - fd) <= 1e-6 * scale, (func, k, dc[k], fd)
