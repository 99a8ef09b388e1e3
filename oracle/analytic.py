"""Closed forms used to pin the oracle (Sections 4 and 7.3).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Joseph-Tao porous sphere: a sphere of radius R centred at the origin, Darcy
flow inside with permeability kappa, Stokes flow outside with far-field
velocity U along the unit vector e (the paper takes e = e_z).  The paper's
formulas are written in spherical coordinates about e; here cos(theta) =
(x . e)/|x| and the unit vector e_theta satisfies sin(theta) e_theta =
cos(theta) e_r - e.
"""
from __future__ import annotations

import math

import numpy as np


def _dir(uinf):
    uinf = np.asarray(uinf, dtype=np.float64)
    U = float(np.linalg.norm(uinf))
    return U, (uinf / U if U > 0 else np.array([0.0, 0.0, 1.0]))


def jt_pressure_darcy(xyz, R, kappa, mu, uinf):
    """p^D = -3 mu U r cos(theta) / (2 R^2 + kappa)  (Section 7.3)."""
    U, e = _dir(uinf)
    return -3.0 * mu * U * (e @ xyz) / (2.0 * R * R + kappa)


def jt_velocity_stokes(xyz, R, kappa, mu, uinf):
    """Exterior velocity u^S (Section 7.3) at points with |x| >= R, [3][N]."""
    U, e = _dir(uinf)
    r = np.sqrt((xyz * xyz).sum(0))
    ct = (e @ xyz) / r
    er = xyz / r
    c = 2.0 + kappa / (R * R)
    B = 1.0 + 2.0 * kappa / (R * R)
    ur = (-3.0 * R * U / (c * r) * (1.0 - R * R / (3.0 * r * r) * B) + U) * ct
    # u_theta e_theta = g(r) sin(theta) e_theta = g(r) (cos(theta) e_r - e)
    g = 3.0 * R * U / (c * 2.0 * r) * (1.0 + R * R / (3.0 * r * r) * B) - U
    return ur * er + g * (ct * er - e[:, None])


def jt_traction_exact_velocity_terms(xyz, R, kappa, mu, uinf):
    """Velocity-derivative part of the traction f = sigma . e_r on r = R.

    Returns (a, tang) with f = (-p_D + a) e_r + tang, where
    a = 2 mu du_r/dr and tang = f_theta e_theta (eqs. f_r, f_theta), both from
    the exact exterior velocity.  With c = 2 + kappa/R^2:
        2 mu du_r/dr |_R   = -12 mu U kappa cos(theta) / (R^3 c)
        f_theta |_R        = -(3 mu U / (R c)) (1 + 2 kappa / R^2) sin(theta).
    """
    U, e = _dir(uinf)
    r = np.sqrt((xyz * xyz).sum(0))
    ct = (e @ xyz) / r
    er = xyz / r
    c = 2.0 + kappa / (R * R)
    a = -12.0 * mu * U * kappa * ct / (R ** 3 * c)
    b = -(3.0 * mu * U / (R * c)) * (1.0 + 2.0 * kappa / (R * R))
    tang = b * (ct * er - e[:, None])
    return a, tang


def jt_drag(R, kappa, mu, U):
    """|D| = 6 pi mu R U / (1 + kappa / (2 R^2))  (eq. drag_value)."""
    return 6.0 * math.pi * mu * R * U / (1.0 + kappa / (2.0 * R * R))


def jt_flux_moment(R, kappa, U):
    """J = int q (e . x) dS with q = u_r^D on r = R: 4 pi kappa U R^3 / (2 R^2 + kappa)."""
    return 4.0 * math.pi * kappa * U * R ** 3 / (2.0 * R * R + kappa)


def spectrum(nmax, R, kappa, theta):
    """Eigenvalues A_n of the continuous D-N iteration on a sphere (eq. CA31)."""
    n = np.arange(1, nmax + 1, dtype=np.float64)
    return (1.0 - theta) - theta * (R * R / kappa) * (n + 1) / (n * (n + 2) * (2 * n - 1))


def stokeslet(xyz, x0, F, mu):
    """Velocity and stress of a point force F at x0: returns (u [3][N], sigma [3][3][N])."""
    r = xyz - np.asarray(x0, dtype=np.float64)[:, None]
    rr = np.sqrt((r * r).sum(0))
    F = np.asarray(F, dtype=np.float64)
    rF = F @ r
    u = (F[:, None] / rr + r * rF / rr ** 3) / (8.0 * math.pi * mu)
    sig = -(3.0 / (4.0 * math.pi)) * r[:, None, :] * r[None, :, :] * rF / rr ** 5
    return u, sig
