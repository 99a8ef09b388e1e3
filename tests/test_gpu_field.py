"""Off-surface fields on the device (eqs. Greens and Stokes) against the
oracle's evaluation of the same boundary data, and against the Joseph-Tao
porous sphere in the bulk."""
import numpy as np
import pytest

from oracle import analytic as A
from oracle import field as F
from oracle import quadrature as Q

pytestmark = pytest.mark.gpu


def T(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _shell(r, m, seed):
    v = np.random.default_rng(seed).normal(size=(3, m))
    return r * v / np.linalg.norm(v, axis=0)


def _solve(ssd, ctx, P, h, kappa, prec):
    inner = ssd.krylov(1e-11 if prec == ssd.FP64 else 1e-9, 300, 100, False, prec, True)
    prm = ssd.ddm_params(mu=1.0, kappa=kappa, gamma=0.0, uinf=(0.0, 0.0, 1.0), delta=3 * h, theta=1.0,
                         tol_outer=1e-10 if prec == ssd.FP64 else 1e-8, maxit_outer=80, outer_gmres=True,
                         traction_mode=ssd.TRACTION_JOSEPH_TAO, radius=1.0, inner=inner)
    return ssd.ddm_solve(ctx, P, prm)


@pytest.mark.parametrize("kappa", [1.0, 1e-2])
def test_fields_match_oracle_and_porous_sphere(gpu_ctx, kappa):
    import paper_2110_10749_gb300 as ssd
    h = 1 / 8
    p = Q.sphere_points(1.0, h)
    P = ssd.Points.from_numpy(p).prepare(gpu_ctx)
    r = _solve(ssd, gpu_ctx, P, h, kappa, ssd.FP64)
    ti = np.concatenate([_shell(0.3, 150, 1), _shell(0.6, 150, 2), np.zeros((3, 1))], axis=1)   # 301: ragged
    to = np.concatenate([_shell(1.5, 150, 3), _shell(3.0, 150, 4)], axis=1)
    pg = ssd.darcy_pressure_field(gpu_ctx, P, 1.0, kappa, r["q"], r["p"], T(ti)).cpu().numpy()
    ug = ssd.stokes_velocity_field(gpu_ctx, P, 1.0, (0.0, 0.0, 1.0), r["f"], r["u"], T(to)).cpu().numpy()
    q, pd, f, u = (r[k].cpu().numpy() for k in ("q", "p", "f", "u"))
    po = F.darcy_pressure_field(p, q, pd, 1.0, kappa, ti)
    uo = F.stokes_velocity_field(p, f, u, 1.0, [0.0, 0.0, 1.0], to)
    assert np.abs(pg - po).max() <= 1e-12 * np.abs(po).max()
    assert np.abs(ug - uo).max() <= 1e-12 * np.abs(uo).max()
    # the Stokes pressure outside: against the oracle, and against the
    # porous sphere's mu U A1 cos(theta) / r^2 with A1 = -3R/(2 + kappa/R^2)
    sg = ssd.stokes_pressure_field(gpu_ctx, P, 1.0, r["f"], r["u"], T(to)).cpu().numpy()
    so = F.stokes_pressure_field(p, f, u, 1.0, to)
    assert np.abs(sg - so).max() <= 1e-12 * np.abs(so).max()
    sex = -3.0 / (2.0 + kappa) * to[2] / np.sqrt((to * to).sum(0)) ** 3
    assert np.abs(sg - sex).max() < 2e-2 * np.abs(sex).max()
    # the porous sphere in the bulk, to the discretisation error of h = 1/8
    assert np.abs(pg - A.jt_pressure_darcy(ti, 1.0, kappa, 1.0, [0.0, 0.0, 1.0])).max() < 1e-2
    assert np.abs(ug - A.jt_velocity_stokes(to, 1.0, kappa, 1.0, [0.0, 0.0, 1.0])).max() < 1e-2
    P.release()


def test_fp32c_solution_fields_at_h16(gpu_ctx):
    import paper_2110_10749_gb300 as ssd
    h = 1 / 16
    q = ssd.quadrature_points(gpu_ctx, ssd.SPHERE, (1.0,), h)
    P = ssd.Points(q["xyz"], q["nrm"], q["w"]).prepare(gpu_ctx)
    r = _solve(ssd, gpu_ctx, P, h, 1.0, ssd.FP32C)
    ti = _shell(0.5, 64, 5)
    to = _shell(2.0, 64, 6)
    pg = ssd.darcy_pressure_field(gpu_ctx, P, 1.0, 1.0, r["q"], r["p"], T(ti)).cpu().numpy()
    ug = ssd.stokes_velocity_field(gpu_ctx, P, 1.0, (0.0, 0.0, 1.0), r["f"], r["u"], T(to)).cpu().numpy()
    assert np.abs(pg - A.jt_pressure_darcy(ti, 1.0, 1.0, 1.0, [0.0, 0.0, 1.0])).max() < 2e-4
    assert np.abs(ug - A.jt_velocity_stokes(to, 1.0, 1.0, 1.0, [0.0, 0.0, 1.0])).max() < 2e-4
    # no field points is a no-op; missing boundary data is an error
    import torch
    empty = torch.empty((3, 0), dtype=torch.float64, device="cuda")
    assert ssd.darcy_pressure_field(gpu_ctx, P, 1.0, 1.0, r["q"], r["p"], empty).numel() == 0
    with pytest.raises(ssd.SsdError) as ei:
        ssd.darcy_pressure_field(gpu_ctx, P, 1.0, -1.0, r["q"], r["p"], T(ti))
    assert ei.value.status == ssd.SSD_EINVAL
    P.release()
