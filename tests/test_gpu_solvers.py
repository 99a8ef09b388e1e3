"""Local solves and the Dirichlet-Neumann iteration on the device against the
oracle, the printed porous-sphere errors (Tables 1-2) and each other
(FP32C against FP64)."""
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


@pytest.fixture(scope="module")
def sph8(gpu_ctx):
    import paper_2110_10749_gb300 as ssd
    p = Q.sphere_points(1.0, 1 / 8)
    P = ssd.Points.from_numpy(p).prepare(gpu_ctx)
    yield p, P
    P.release()


def test_darcy_and_stokes_solves_match_oracle(gpu_ctx):
    import paper_2110_10749_gb300 as ssd
    h = 1 / 8
    p = Q.sphere_points(0.8, h)
    x, y, z = p["xyz"]
    n = p["nrm"]
    dP = np.exp(x) * (np.sin(y) * n[0] + np.cos(y) * n[1])
    q = -dP
    po, _, _ = S.darcy_solve(p, 3 * h, 1.0, 1.0, q, tol=1e-12)
    u, sig = A.stokeslet(p["xyz"], [0.2, 0.0, 0.0], [1.0, 0.0, 0.0], 1.0)
    f = np.einsum("ikn,kn->in", sig, n)
    uo, _, _ = S.stokes_solve(p, 3 * h, 1.0, f, [0.1, 0, 0], tol=1e-12)
    P = ssd.Points.from_numpy(p)
    for prepared in (False, True):
        if prepared:
            P.prepare(gpu_ctx)
        for prec, tol in ((ssd.FP64, 1e-9), (ssd.FP32C, 1e-5)):
            kr = ssd.krylov(1e-12 if prec == ssd.FP64 else 1e-9, 300, 50, False, prec)
            pg, its, rel = ssd.darcy_solve(gpu_ctx, P, 3 * h, 1.0, 1.0, T(q), kr)
            assert np.linalg.norm(pg.cpu().numpy() - po) / np.linalg.norm(po) < tol
            ug, its2, rel2 = ssd.stokes_solve(gpu_ctx, P, 3 * h, 1.0, T(f), (0.1, 0, 0), kr)
            # compare modulo the near-null mode n of I - D^S (see the oracle pins)
            e = ug.cpu().numpy() - uo
            e -= (e * n).sum() / (n * n).sum() * n
            assert np.linalg.norm(e) / np.linalg.norm(uo) < 10 * tol
    P.release()


def test_successive_approximation_variants(gpu_ctx, sph8):
    import paper_2110_10749_gb300 as ssd
    p, P = sph8
    h = 1 / 8
    pe = A.jt_pressure_darcy(p["xyz"], 1.0, 1.0, 1.0, [0, 0, 1.0])
    f = S.traction_joseph_tao(p, pe, 1.0, 1.0, 1.0, [0, 0, 1.0])
    uo, itso, _ = S.stokes_solve(p, 3 * h, 1.0, f, [0, 0, 1.0], tol=1e-11, use_sa=True)
    kr = ssd.krylov(1e-11, 500, 50, True, ssd.FP64)
    ug, its, rel = ssd.stokes_solve(gpu_ctx, P, 3 * h, 1.0, T(f), (0, 0, 1.0), kr)
    assert np.abs(ug.cpu().numpy() - uo).max() < 1e-9 and abs(its - itso) <= 1
    q = (uo * p["nrm"]).sum(0)
    po, itdo, _ = S.darcy_solve(p, 3 * h, 1.0, 1.0, q, tol=1e-11, use_sa=True)
    pg, itd, _ = ssd.darcy_solve(gpu_ctx, P, 3 * h, 1.0, 1.0, T(q), kr)
    assert np.abs(pg.cpu().numpy() - po).max() < 1e-9 and abs(itd - itdo) <= 1


def _bench_params(ssd, h, kappa, theta, outer_gmres, prec, tol=1e-9, deflate=False):
    inner = ssd.krylov(0.1 * tol if outer_gmres else tol, 300, 50, False, prec, deflate)
    return ssd.ddm_params(mu=1.0, kappa=kappa, gamma=0.0, uinf=(0, 0, 1.0), delta=3 * h, theta=theta,
                          tol_outer=tol, maxit_outer=60, outer_gmres=outer_gmres,
                          traction_mode=ssd.TRACTION_JOSEPH_TAO, radius=1.0, inner=inner)


@pytest.mark.parametrize("outer", ["sa", "gmres"])
def test_ddm_benchmark_matches_oracle(gpu_ctx, sph8, outer):
    import paper_2110_10749_gb300 as ssd
    p, P = sph8
    h, kappa, theta = 1 / 8, 1.0, 0.5
    ro = S.ddm_solve(p, 3 * h, 1.0, kappa, 0.0, [0, 0, 1.0], theta, tol=1e-9, maxit=60, outer=outer,
                     traction="jt")
    r64 = ssd.ddm_solve(gpu_ctx, P, _bench_params(ssd, h, kappa, theta, outer == "gmres", ssd.FP64))
    assert r64["outer_its"] == ro["outer_its"]
    assert np.abs(r64["p"].cpu().numpy() - ro["p"]).max() < 1e-8
    assert np.abs(r64["u"].cpu().numpy() - ro["u"]).max() < 1e-8
    assert np.allclose(r64["drag"], ro["drag"], atol=1e-8)
    # Relaxed sweeps in FP32C: the successive-difference residual levels off
    # at the pair-sum rounding (about 1e-7), so they run to 1e-6; the
    # interface GMRES reaches 1e-9 in its residual estimate.
    tol32 = 1e-9 if outer == "gmres" else 1e-6
    r32 = ssd.ddm_solve(gpu_ctx, P, _bench_params(ssd, h, kappa, theta, outer == "gmres", ssd.FP32C, tol32))
    for k in ("p", "u"):
        a, b = r32[k].cpu().numpy(), r64[k].cpu().numpy()
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-5


@pytest.mark.parametrize("row", [r for r in read_golden("porous_sphere_errors.txt") if r[1] == "16"],
                         ids=lambda r: "kappa%s" % r[0])
def test_ddm_printed_errors_h16(gpu_ctx, row):
    # Tables 1-2 at h = 1/16: FP64 and FP32C reproduce the printed errors
    import paper_2110_10749_gb300 as ssd
    kappa, inv_h, N, itD, itS, perr, uerr, _ = row
    kappa, h = float(kappa), 1.0 / int(inv_h)
    p = Q.sphere_points(1.0, h)
    P = ssd.Points.from_numpy(p).prepare(gpu_ctx)
    pe = A.jt_pressure_darcy(p["xyz"], 1.0, kappa, 1.0, [0, 0, 1.0])
    ue = A.jt_velocity_stokes(p["xyz"], 1.0, kappa, 1.0, [0, 0, 1.0])
    res = {}
    for prec in (ssd.FP64, ssd.FP32C):
        # the normal-mode deflation keeps FP32C rounding from being amplified
        # by the near-null vector of I - D^S; it does not change these errors
        prm = _bench_params(ssd, h, kappa, 0.75 * min(kappa, 1.0), True, prec, deflate=True)
        prm.maxit_outer = 100
        res[prec] = ssd.ddm_solve(gpu_ctx, P, prm)
    r = res[ssd.FP64]
    ep, eu = S.rms(r["p"].cpu().numpy() - pe), S.rms(r["u"].cpu().numpy() - ue)
    # kappa = 1e-4: the oracle itself lands within 10% of the printed p error
    rtol = 2e-3 if kappa >= 1e-2 else 0.12
    assert ep == pytest.approx(float(perr), rel=rtol)
    assert eu == pytest.approx(float(uerr), rel=max(rtol, 2e-3))
    D = A.jt_drag(1.0, kappa, 1.0, 1.0)
    assert abs(r["drag"][2] - D) / D < 1e-3
    # FP32C fields within 1e-5 of the FP64 ones, on their natural scales:
    # the pressure against its own norm, the velocity against the far-field
    # speed (at kappa = 1e-4 the surface velocity is only ~1e-4 U)
    n = p["w"].size
    a, b = res[ssd.FP32C]["p"].cpu().numpy(), r["p"].cpu().numpy()
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-5
    a, b = res[ssd.FP32C]["u"].cpu().numpy(), r["u"].cpu().numpy()
    assert np.linalg.norm(a - b) / max(np.linalg.norm(b), np.sqrt(n)) < 1e-5
    P.release()


def test_ddm_bjs_mode_matches_oracle(gpu_ctx, sph8):
    import paper_2110_10749_gb300 as ssd
    p, P = sph8
    h = 1 / 8
    for outer, kappa, gamma in (("sa", 1.0, 0.5), ("gmres", 1e-2, 1.0)):
        theta = 0.5 * min(kappa, 1.0)
        ro = S.ddm_solve(p, 3 * h, 1.0, kappa, gamma, [0.3, 0.0, 1.0], theta, tol=1e-10, maxit=80, outer=outer,
                         traction="bjs")
        inner = ssd.krylov(1e-11, 300, 50, False, ssd.FP64)
        prm = ssd.ddm_params(mu=1.0, kappa=kappa, gamma=gamma, uinf=(0.3, 0.0, 1.0), delta=3 * h, theta=theta,
                             tol_outer=1e-10, maxit_outer=80, outer_gmres=outer == "gmres",
                             traction_mode=ssd.TRACTION_BJS, bjs_sign=1.0, inner=inner)
        r = ssd.ddm_solve(gpu_ctx, P, prm)
        assert np.abs(r["u"].cpu().numpy() - ro["u"]).max() < 1e-7
        assert np.abs(r["q"].cpu().numpy() - ro["q"]).max() < 1e-7
        prm.inner.prec = ssd.FP32C
        if outer == "sa":
            prm.tol_outer = 1e-6
        r32 = ssd.ddm_solve(gpu_ctx, P, prm)
        a, b = r32["u"].cpu().numpy(), r["u"].cpu().numpy()
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-5


def test_host_buffer_entry_point(gpu_ctx, sph8):
    import paper_2110_10749_gb300 as ssd
    p, P = sph8
    prm = _bench_params(ssd, 1 / 8, 1.0, 0.75, True, ssd.FP32C)
    rd = ssd.ddm_solve(gpu_ctx, P, prm)
    rh = ssd.ddm_solve_host(gpu_ctx, p["xyz"], p["nrm"], p["w"], prm)
    assert np.array_equal(rh["u"], rd["u"].cpu().numpy())
    assert np.array_equal(rh["drag"], rd["drag"])


def test_iteration_limit_and_bad_parameters(gpu_ctx, sph8):
    import paper_2110_10749_gb300 as ssd
    p, P = sph8
    prm = _bench_params(ssd, 1 / 8, 1.0, 0.5, False, ssd.FP64)
    prm.maxit_outer = 2
    with pytest.raises(ssd.NotConverged):
        ssd.ddm_solve(gpu_ctx, P, prm)
    r = ssd.ddm_solve(gpu_ctx, P, prm, raise_on_notconv=False)
    assert r["status"] == ssd.SSD_ENOTCONV and r["outer_its"] == 2 and len(r["hist"]) == 2
    for field, bad in (("theta", 0.0), ("theta", 1.5), ("kappa", -1.0), ("mu", float("nan")),
                       ("tol_outer", 0.0), ("bjs_sign", 2.0)):
        prm = _bench_params(ssd, 1 / 8, 1.0, 0.5, False, ssd.FP64)
        prm.traction_mode = ssd.TRACTION_BJS
        setattr(prm, field, bad)
        with pytest.raises(ssd.SsdError) as e:
            ssd.ddm_solve(gpu_ctx, P, prm)
        assert e.value.status == ssd.SSD_EINVAL
    kr = ssd.krylov(1e-12, 1, 50, False, ssd.FP64)
    with pytest.raises(ssd.NotConverged):
        ssd.darcy_solve(gpu_ctx, P, 3 / 8, 1.0, 1.0, T(p["nrm"][2].copy()), kr)


def test_nonfinite_input_reports_numeric_error(gpu_ctx, sph8):
    import paper_2110_10749_gb300 as ssd
    p, P = sph8
    q = p["nrm"][2].copy()
    q[5] = np.nan
    with pytest.raises(ssd.SsdError) as e:
        ssd.darcy_solve(gpu_ctx, P, 3 / 8, 1.0, 1.0, T(q), ssd.krylov(1e-10, 50, 50, False, ssd.FP64))
    assert e.value.status == ssd.SSD_ENUMERIC


def test_deflated_stokes_solve(gpu_ctx):
    # Fig. 4 Stokeslet test solved with the normal-mode deflation: FP64
    # matches the oracle's deflated solve, FP32C stays within 1e-5 of FP64
    import paper_2110_10749_gb300 as ssd
    h = 1 / 16
    p = Q.sphere_points(0.8, h)
    u, sig = A.stokeslet(p["xyz"], [0.2, 0.0, 0.0], [1.0, 0.0, 0.0], 1.0)
    f = np.einsum("ikn,kn->in", sig, p["nrm"])
    uo, _, _ = S.stokes_solve(p, 3 * h, 1.0, f, [0, 0, 0], tol=1e-12, deflate=True)
    P = ssd.Points.from_numpy(p).prepare(gpu_ctx)
    u64, _, _ = ssd.stokes_solve(gpu_ctx, P, 3 * h, 1.0, T(f), (0, 0, 0), ssd.krylov(1e-12, 300, 50, False, ssd.FP64, True))
    u32, _, _ = ssd.stokes_solve(gpu_ctx, P, 3 * h, 1.0, T(f), (0, 0, 0), ssd.krylov(1e-10, 300, 50, False, ssd.FP32C, True))
    u64, u32 = u64.cpu().numpy(), u32.cpu().numpy()
    assert np.linalg.norm(u64 - uo) / np.linalg.norm(uo) < 1e-10
    assert np.linalg.norm(u32 - u64) / np.linalg.norm(u64) < 1e-5
    assert S.rms(u64 - u) < 1e-4
    P.release()


@pytest.mark.parametrize("kappa,gamma", [(1.0, 0.5), (1e-2, 1.0)])
def test_ddm_implicit_bjs_matches_oracle(gpu_ctx, sph8, kappa, gamma):
    import paper_2110_10749_gb300 as ssd
    p, P = sph8
    h = 1 / 8
    theta = 0.5 * min(kappa, 1.0)
    ro = S.ddm_solve(p, 3 * h, 1.0, kappa, gamma, [0.3, 0.0, 1.0], theta, tol=1e-10, maxit=80, outer="gmres",
                     traction="bjs", bjs_implicit=True, deflate=True, inner_tol=1e-11)
    res = {}
    for prec in (ssd.FP64, ssd.FP32C):
        inner = ssd.krylov(1e-11, 300, 50, False, prec, True)
        prm = ssd.ddm_params(mu=1.0, kappa=kappa, gamma=gamma, uinf=(0.3, 0.0, 1.0), delta=3 * h, theta=theta,
                             tol_outer=1e-10, maxit_outer=80, outer_gmres=True, traction_mode=ssd.TRACTION_BJS,
                             bjs_sign=1.0, inner=inner, bjs_implicit=True)
        res[prec] = ssd.ddm_solve(gpu_ctx, P, prm)
    r = res[ssd.FP64]
    assert r["outer_its"] == ro["outer_its"]
    for k in ("q", "p", "u", "f"):
        assert np.abs(r[k].cpu().numpy() - ro[k]).max() < 1e-8
        a, b = res[ssd.FP32C][k].cpu().numpy(), r[k].cpu().numpy()
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-5
    assert np.allclose(r["drag"], ro["drag"], atol=1e-8)
