"""Off-surface evaluation of the Darcy pressure and the Stokes velocity from
their boundary data (eqs. Greens and Stokes, Section 5).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The representations hold for field points y off the surface, with the bare
kernels (no smoothing): the quadrature of Section 5.4 is accurate for points
a few grid spacings away from the surface (near-surface corrections are not
part of the paper).  n is the body's outward normal, so the Stokes domain's
normal is n_S = -n, and the Darcy flux q = u . n gives dp/dn = -(mu/kappa) q
(Darcy's law, Section 2).
"""
from __future__ import annotations

import math

import numpy as np


def _chunks(m, size=256):
    for a in range(0, m, size):
        yield a, min(m, a + size)


def darcy_pressure_field(pts, q, p, mu, kappa, targets):
    """p_D(y) = -int dp/dn G dS + int p dG/dn(x) dS, y inside (eq. Greens);
    G = -1/(4 pi r), dG/dn(x) = -(y - x) . n(x) / (4 pi r^3)."""
    x, n, w = pts["xyz"], pts["nrm"], pts["w"]
    y = np.asarray(targets, dtype=np.float64)
    dpdn = -(mu / kappa) * np.asarray(q)
    out = np.empty(y.shape[1])
    for a, b in _chunks(y.shape[1]):
        d = y[:, a:b, None] - x[:, None, :]            # [3][t][s]
        r = np.sqrt((d * d).sum(0))
        G = -1.0 / (4.0 * math.pi * r)
        dG = -(d * n[:, None, :]).sum(0) / (4.0 * math.pi * r ** 3)
        out[a:b] = (-(dpdn * w) * G + (p * w) * dG).sum(1)
    return out


def stokes_velocity_field(pts, f, u, mu, uinf, targets):
    """u_S(y) = U - 1/(8 pi mu) int S f dS + 1/(8 pi) int u . T . n_S dS,
    y outside (eq. Stokes), S_ij = delta_ij/r + yh_i yh_j/r^3,
    T_ijk = -6 yh_i yh_j yh_k / r^5, yh = y - x, n_S = -n."""
    x, n, w = pts["xyz"], pts["nrm"], pts["w"]
    y = np.asarray(targets, dtype=np.float64)
    out = np.empty((3, y.shape[1]))
    for a, b in _chunks(y.shape[1]):
        d = y[:, a:b, None] - x[:, None, :]            # [3][t][s]
        r = np.sqrt((d * d).sum(0))
        df = (d * f[:, None, :]).sum(0)
        single = (f[:, None, :] / r + d * df / r ** 3) * w
        du = (d * u[:, None, :]).sum(0)
        dn = (d * (-n)[:, None, :]).sum(0)
        double = -6.0 * d * du * dn / r ** 5 * w
        out[:, a:b] = (np.asarray(uinf, dtype=np.float64)[:, None]
                       - single.sum(2) / (8.0 * math.pi * mu) + double.sum(2) / (8.0 * math.pi))
    return out


def stokes_pressure_field(pts, f, u, mu, targets):
    """p_S(y) = -1/(8 pi) int P . f dS - mu/(8 pi) int u . Pi . n_S dS, y
    outside, with the pressures that go with the kernels of eq. Stokes: the
    Stokeslet's P_i = 2 yh_i / r^3 and the stresslet's
    Pi_ik = 4 (-delta_ik / r^3 + 3 yh_i yh_k / r^5), yh = y - x, n_S = -n;
    the far-field pressure is 0.  The paper prints the velocity
    representation only; this is its pressure counterpart."""
    x, n, w = pts["xyz"], pts["nrm"], pts["w"]
    y = np.asarray(targets, dtype=np.float64)
    out = np.empty(y.shape[1])
    nS = -n
    for a, b in _chunks(y.shape[1]):
        d = y[:, a:b, None] - x[:, None, :]            # [3][t][s]
        r = np.sqrt((d * d).sum(0))
        single = 2.0 * (d * f[:, None, :]).sum(0) / r ** 3 * w
        du = (d * u[:, None, :]).sum(0)
        dn = (d * nS[:, None, :]).sum(0)
        un = (u * nS).sum(0)
        double = 4.0 * (-un[None, :] / r ** 3 + 3.0 * du * dn / r ** 5) * w
        out[a:b] = -single.sum(1) / (8.0 * math.pi) - mu * double.sum(1) / (8.0 * math.pi)
    return out
