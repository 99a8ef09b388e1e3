"""Transposed operators and the adjoint gradient of the D-N solve.

The transposes are checked against the plain definition (A^T y)_i =
(A e_i) . y with the columns A e_i taken from the oracle's forward operators,
and by the identity <A x, y> = <x, A^T y> with A x from the oracle.  The
adjoint gradients dJ/dlog(kappa) and dJ/dgamma are checked against central
finite differences of J computed by the oracle's D-N solve (the same
discretisation) and by the device's own FP64 forward solves.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import quadrature as Q
from oracle import solvers as S

pytestmark = pytest.mark.gpu

MU = 1.3
TOL = {0: 1e-12, 1: 1e-5}


def T(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _oracle_apply(name, p, d, x):
    if name == "LSL":
        return oracle.laplace_sl(p, d, x)
    if name == "LDL":
        return oracle.laplace_dl(p, d, x)
    if name == "SSL":
        return oracle.stokes_sl(p, d, MU, x)
    return oracle.stokes_dl(p, d, x)


def _op(ssd, name):
    return {"LSL": ssd.OP_LAPLACE_SL, "LDL": ssd.OP_LAPLACE_DL, "SSL": ssd.OP_STOKES_SL,
            "SDL": ssd.OP_STOKES_DL}[name]


@pytest.mark.parametrize("prepared", [False, True])
def test_transposes_match_oracle_columns(gpu_ctx, prepared):
    import paper_2110_10749_gb300 as ssd
    h = 1 / 8
    p = Q.ellipsoid_points((1.0, 0.7, 0.5), h)
    n = p["w"].size
    d = 3 * h
    rng = np.random.default_rng(7)
    idx = np.unique(np.concatenate([rng.choice(n, 20, replace=False), [0, n - 1]]))
    P = ssd.Points.from_numpy(p)
    if prepared:
        P.prepare(gpu_ctx)
    for name in ("LSL", "LDL", "SSL", "SDL"):
        nc = 3 if name[0] == "S" else 1
        y = rng.normal(size=(nc, n)) if nc == 3 else rng.normal(size=n)
        ref = np.zeros((nc, idx.size))
        for k, i in enumerate(idx):
            for c in range(nc):
                e = np.zeros((nc, n)) if nc == 3 else np.zeros(n)
                if nc == 3:
                    e[c, i] = 1.0
                else:
                    e[i] = 1.0
                ref[c, k] = float((_oracle_apply(name, p, d, e) * y).sum())
        for prec in (ssd.FP64, ssd.FP32C):
            out = ssd.apply_transpose(gpu_ctx, P, _op(ssd, name), d, T(y), mu=MU, prec=prec).cpu().numpy()
            got = out.reshape(nc, n)[:, idx]
            rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
            assert rel <= TOL[prec], (name, prec, rel)
    P.release()


def test_transpose_identity_against_oracle(gpu_ctx):
    import paper_2110_10749_gb300 as ssd
    h = 1 / 12
    p = Q.sphere_points(0.9, h, center=(0.1, -0.2, 0.05))
    n = p["w"].size
    assert n % 512 != 0
    d = 3 * h
    rng = np.random.default_rng(11)
    P = ssd.Points.from_numpy(p).prepare(gpu_ctx)
    for name in ("LSL", "LDL", "SSL", "SDL"):
        shape = (3, n) if name[0] == "S" else (n,)
        x, y = rng.normal(size=shape), rng.normal(size=shape)
        Ax = _oracle_apply(name, p, d, x)
        for prec in (ssd.FP64, ssd.FP32C):
            ATy = ssd.apply_transpose(gpu_ctx, P, _op(ssd, name), d, T(y), mu=MU, prec=prec).cpu().numpy()
            lhs, rhs = float((Ax * y).sum()), float((x * ATy).sum())
            scale = np.linalg.norm(Ax) * np.linalg.norm(y)
            assert abs(lhs - rhs) <= TOL[prec] * scale, (name, prec, lhs, rhs)
    P.release()


def _params(ssd, h, kappa, gamma, mode, tol=1e-11):
    inner = ssd.krylov(0.1 * tol, 400, 100, False, ssd.FP64, True)
    return ssd.ddm_params(mu=1.0, kappa=kappa, gamma=gamma, uinf=(0.0, 0.0, 1.0), delta=3 * h, theta=1.0,
                          tol_outer=tol, maxit_outer=80, outer_gmres=True, traction_mode=mode, radius=1.0,
                          inner=inner, bjs_implicit=True)


def _oracle_J(p, h, kappa, gamma, mode, func):
    traction = "bjs" if mode == 0 else "jt"
    r = S.ddm_solve(p, 3 * h, 1.0, kappa, gamma, [0.0, 0.0, 1.0], 1.0, tol=1e-11, maxit=80, outer="gmres",
                    traction=traction, R=1.0, restart=100, inner_maxit=400, bjs_implicit=True, deflate=True)
    if func == 0:
        return float(r["drag"][2])
    return float((p["w"] * r["q"] * p["xyz"][2]).sum())


def _richardson(J, x0, eps):
    """Central difference of J at x0 with Richardson's extrapolation from
    steps eps and eps/2: truncation O(eps^4) instead of O(eps^2)."""
    d1 = (J(x0 + eps) - J(x0 - eps)) / (2 * eps)
    d2 = (J(x0 + eps / 2) - J(x0 - eps / 2)) / eps
    return (4.0 * d2 - d1) / 3.0


@pytest.fixture(scope="module")
def sph8(gpu_ctx):
    import paper_2110_10749_gb300 as ssd
    p = Q.sphere_points(1.0, 1 / 8)
    P = ssd.Points.from_numpy(p).prepare(gpu_ctx)
    yield p, P
    P.release()


@pytest.mark.parametrize("mode,kappa,gamma,func", [
    (0, 0.1, 0.5, 0),     # implicit BJS, drag
    (0, 0.1, 0.5, 1),     # implicit BJS, flux moment
    (1, 1.0, 0.0, 0),     # porous-sphere benchmark traction, drag
])
def test_gradient_matches_oracle_finite_differences(gpu_ctx, sph8, mode, kappa, gamma, func):
    import paper_2110_10749_gb300 as ssd
    p, P = sph8
    h = 1 / 8
    J, g, st = ssd.ddm_gradient(gpu_ctx, P, _params(ssd, h, kappa, gamma, mode), func)
    assert st == ssd.SSD_OK
    J0 = _oracle_J(p, h, kappa, gamma, mode, func)
    assert abs(J - J0) <= 1e-8 * abs(J0)
    # the benchmark spec's 1e-6, relative to the finite difference itself
    eps = 2e-3
    fd_k = _richardson(lambda lk: _oracle_J(p, h, math.exp(lk), gamma, mode, func), math.log(kappa), eps)
    assert abs(g[0] - fd_k) <= 1e-6 * abs(fd_k), (g[0], fd_k)
    if mode == 0:
        fd_g = _richardson(lambda gm: _oracle_J(p, h, kappa, gm, mode, func), gamma, eps)
        assert abs(g[1] - fd_g) <= 1e-6 * abs(fd_g), (g[1], fd_g)
    else:
        assert g[1] == 0.0


def test_gradient_matches_device_finite_differences_small_kappa(gpu_ctx):
    """kappa = 1e-2 on the h = 1/16 sphere (several tiles, ragged tail)."""
    import paper_2110_10749_gb300 as ssd
    h = 1 / 16
    p = Q.sphere_points(1.0, h)
    P = ssd.Points.from_numpy(p).prepare(gpu_ctx)
    kappa, gamma = 1e-2, 1.0
    J, g, st = ssd.ddm_gradient(gpu_ctx, P, _params(ssd, h, kappa, gamma, 0), ssd.FUNC_DRAG)
    assert st == ssd.SSD_OK

    def Jd(k, gm):
        return float(ssd.ddm_solve(gpu_ctx, P, _params(ssd, h, k, gm, 0))["drag"][2])

    assert abs(Jd(kappa, gamma) - J) <= 1e-10 * abs(J)
    eps = 2e-3
    fd_k = _richardson(lambda lk: Jd(math.exp(lk), gamma), math.log(kappa), eps)
    fd_g = _richardson(lambda gm: Jd(kappa, gm), gamma, eps)
    assert abs(g[0] - fd_k) <= 1e-6 * abs(fd_k), (g[0], fd_k)
    assert abs(g[1] - fd_g) <= 1e-6 * abs(fd_g), (g[1], fd_g)
    P.release()


def test_autograd_function_and_argument_checks(gpu_ctx, sph8):
    import torch
    import paper_2110_10749_gb300 as ssd
    p, P = sph8
    h = 1 / 8
    prm = _params(ssd, h, 0.1, 0.5, 0)
    J, g, _ = ssd.ddm_gradient(gpu_ctx, P, prm, ssd.FUNC_DRAG)
    lk = torch.tensor(math.log(0.1), dtype=torch.float64, requires_grad=True)
    gm = torch.tensor(0.5, dtype=torch.float64, requires_grad=True)
    out = ssd.ddm_functional(gpu_ctx, P, prm, lk, gm, ssd.FUNC_DRAG)
    (2.0 * out).backward()
    assert abs(out.item() - J) <= 1e-12 * abs(J)
    assert abs(lk.grad.item() - 2 * g[0]) <= 1e-12 * abs(g[0]) + 1e-300
    assert abs(gm.grad.item() - 2 * g[1]) <= 1e-12 * abs(g[1]) + 1e-300
    bad = [
        _params(ssd, h, 0.1, 0.5, 0),
        _params(ssd, h, 0.1, 0.5, 0),
        _params(ssd, h, 0.1, 0.5, 0),
    ]
    bad[0].outer_gmres = 0
    bad[1].bjs_implicit = 0
    bad[2].inner.use_sa = 1
    for b in bad:
        with pytest.raises(ssd.SsdError) as ei:
            ssd.ddm_gradient(gpu_ctx, P, b, ssd.FUNC_DRAG)
        assert ei.value.status == ssd.SSD_EINVAL
    with pytest.raises(ssd.SsdError) as ei:
        ssd.ddm_gradient(gpu_ctx, P, prm, 7)
    assert ei.value.status == ssd.SSD_EINVAL
