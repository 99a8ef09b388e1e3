"""Pins of the oracle's off-surface evaluation (eqs. Greens and Stokes):
exact fields reproduced from their own Cauchy data, and the Joseph-Tao
porous sphere (Section 7.3) reproduced in the bulk from the D-N solution,
with errors that fall at high order as h is refined."""
import math

import numpy as np
import pytest

from oracle import analytic as A
from oracle import field as F
from oracle import quadrature as Q
from oracle import solvers as S


def _shell(r, m, seed):
    v = np.random.default_rng(seed).normal(size=(3, m))
    return r * v / np.linalg.norm(v, axis=0)


def test_representations_reproduce_exact_fields():
    errs = []
    for h in (1 / 8, 1 / 12):
        p = Q.sphere_points(1.0, h)
        x, y, z = p["xyz"]
        n = p["nrm"]
        # harmonic pressure e^x sin y inside, from its values and normal derivative
        P = np.exp(x) * np.sin(y)
        dP = np.exp(x) * (np.sin(y) * n[0] + np.cos(y) * n[1])
        kappa, mu = 0.5, 1.3
        t = _shell(0.6, 30, 1)
        ed = np.abs(F.darcy_pressure_field(p, -(kappa / mu) * dP, P, mu, kappa, t)
                    - np.exp(t[0]) * np.sin(t[1])).max()
        # exterior Stokeslet (source inside the body), traction sigma . n
        u, sig = A.stokeslet(p["xyz"], [0.2, 0.0, 0.0], [1.0, 0.3, -0.2], mu)
        f = np.einsum("ikn,kn->in", sig, n)
        t = _shell(1.6, 30, 2)
        ue, _ = A.stokeslet(t, [0.2, 0.0, 0.0], [1.0, 0.3, -0.2], mu)
        es = np.abs(F.stokes_velocity_field(p, f, u, mu, [0.0, 0.0, 0.0], t) - ue).max() / np.abs(ue).max()
        errs.append((ed, es))
    assert errs[0][0] < 5e-3 and errs[0][1] < 1e-2, errs
    assert errs[1][0] < errs[0][0] / 8 and errs[1][1] < errs[0][1] / 8, errs


@pytest.mark.parametrize("kappa", [1.0, 1e-2])
def test_porous_sphere_bulk_fields(kappa):
    errs = []
    for h in (1 / 8, 1 / 12):
        p = Q.sphere_points(1.0, h)
        r = S.ddm_solve(p, 3 * h, 1.0, kappa, 0.0, [0.0, 0.0, 1.0], 1.0, tol=1e-11, maxit=80, outer="gmres",
                        traction="jt", R=1.0, restart=100)
        ti = np.concatenate([_shell(0.3, 20, 3), _shell(0.6, 20, 4)], axis=1)
        to = np.concatenate([_shell(1.5, 20, 5), _shell(3.0, 20, 6)], axis=1)
        ep = np.abs(F.darcy_pressure_field(p, r["q"], r["p"], 1.0, kappa, ti)
                    - A.jt_pressure_darcy(ti, 1.0, kappa, 1.0, [0.0, 0.0, 1.0])).max()
        eu = np.abs(F.stokes_velocity_field(p, r["f"], r["u"], 1.0, [0.0, 0.0, 1.0], to)
                    - A.jt_velocity_stokes(to, 1.0, kappa, 1.0, [0.0, 0.0, 1.0])).max()
        errs.append((ep, eu))
    assert errs[0][0] < 1e-2 and errs[0][1] < 1e-2, errs
    assert errs[1][0] < errs[0][0] / 6 and errs[1][1] < errs[0][1] / 6, errs


def test_stokes_pressure_representation():
    """The pressure counterpart of eq. Stokes reproduces two exact exterior
    pressures from their boundary data, with an error falling with h: the
    Stokeslet placed inside the body, and the porous sphere with slip
    (p_S = mu U A1 cos(theta) / r^2)."""
    errs = []
    for h in (1 / 8, 1 / 16):
        R, mu = 0.8, 1.3
        p = Q.sphere_points(R, h)
        x0, Fv = np.array([0.2, 0.0, 0.0]), np.array([1.0, 0.3, -0.5])
        u, sig = A.stokeslet(p["xyz"], x0, Fv, mu)
        f = np.einsum("ikn,kn->in", sig, p["nrm"])
        t = _shell(1.6, 30, 7)
        d = t - x0[:, None]
        pex = (Fv @ d) / (4.0 * math.pi * np.sqrt((d * d).sum(0)) ** 3)
        e1 = np.abs(F.stokes_pressure_field(p, f, u, mu, t) - pex).max() / np.abs(pex).max()
        ps = Q.sphere_points(1.0, h)
        kappa, gamma = 1e-2, 1.0
        _, _, us, fs = A.bjs_interface_fields(ps["xyz"], 1.0, kappa, gamma, 1.0, (0.0, 0.0, 1.0))
        x, _ = A.bjs_sphere_coefficients(1.0, kappa, gamma)
        t2 = _shell(1.5, 30, 8)
        pexs = x * t2[2] / np.sqrt((t2 * t2).sum(0)) ** 3
        e2 = np.abs(F.stokes_pressure_field(ps, fs, us, 1.0, t2) - pexs).max() / np.abs(pexs).max()
        errs.append((e1, e2))
    assert errs[0][0] < 2e-2 and errs[0][1] < 1e-2, errs
    assert errs[1][0] < errs[0][0] / 8 and errs[1][1] < errs[0][1] / 8, errs
