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


# ---------------------------------------------------------------------------
# Porous sphere in uniform flow with the Beavers-Joseph-Saffman slip
# (eqs. Vel_contin, BeaversJoseph, Press_contin; the D-N fixed point of
# Section 3 with the traction of eq. f).  Not printed in the paper: derived
# here.  Exterior Stokes flow about e (axisymmetric, degree one), stream
# function psi = (U/2) sin^2(theta) (r^2 + A1 r + A2 / r):
#     u_r     =  U cos(theta) (1 + A1/r + A2/r^3)
#     u_theta = -(U/2) sin(theta) (2 + A1/r - A2/r^3)
#     p_S     =  mu U A1 cos(theta) / r^2
# so that on r = R
#     sigma_rr    = -p_S + 2 mu du_r/dr = -mu U (3 A1/R^2 + 6 A2/R^4) cos(theta)
#     sigma_rtheta = -3 mu U A2 sin(theta) / R^4.
# Interior Darcy pressure p_D = P r cos(theta) (harmonic, zero mean on the
# sphere), u_D = -(kappa/mu) grad p_D.  With n = e_r (the body normal) the
# interface conditions read
#     u_r = u_D . e_r               ->  1 + x + y = -k (3x + 6y)
#     sigma_rr = -p_D               ->  P = mu U (3x + 6y) / R^2
#     sigma_rtheta = s c u_theta    ->  6 y = b (2 + x - y)
# with x = A1/R, y = A2/R^3, k = kappa/R^2, c = gamma/sqrt(kappa) (eq. f
# prints no mu) and b = s c R / mu; s = +1 is the sign of eq. BeaversJoseph
# (s = -1 the sign printed in eq. f).  Solving,
#     x = -(6 + 3b + 12 k b) / (6 + 2b + 18 k + 9 k b),   y = b (2 + x) / (6 + b),
# and the drag is the Stokeslet strength, D = -4 pi mu U R x (b -> infinity
# gives the no-slip sphere with normal-stress balance; b = 0 the shear-free
# one, x = -1/(1 + 3k)).
# ---------------------------------------------------------------------------

def bjs_sphere_coefficients(R, kappa, gamma, mu=1.0, sign=1.0):
    """(x, y) = (A1/R, A2/R^3) of the slip porous sphere (derivation above)."""
    k = kappa / (R * R)
    b = sign * gamma * R / (mu * math.sqrt(kappa))
    x = -(6.0 + 3.0 * b + 12.0 * k * b) / (6.0 + 2.0 * b + 18.0 * k + 9.0 * k * b)
    y = b * (2.0 + x) / (6.0 + b)
    return x, y


def bjs_drag(R, kappa, gamma, mu, U, sign=1.0):
    """Drag along e of the slip porous sphere: -4 pi mu U R x."""
    x, _ = bjs_sphere_coefficients(R, kappa, gamma, mu, sign)
    return -4.0 * math.pi * mu * U * R * x


def bjs_interface_fields(xyz, R, kappa, gamma, mu, uinf, sign=1.0):
    """Interface fields of the slip porous sphere at points on r = R.

    Returns (q, p_D, u_S [3][N], f_S [3][N]) with q = u . n, n = e_r, and
    f_S = sigma . n = -p_D n + s (gamma/sqrt(kappa)) (u - (u . n) n).
    """
    U, e = _dir(uinf)
    x, y = bjs_sphere_coefficients(R, kappa, gamma, mu, sign)
    r = np.sqrt((xyz * xyz).sum(0))
    ct = (e @ xyz) / r
    er = xyz / r
    ur = U * ct * (1.0 + x + y)
    g = -0.5 * U * (2.0 + x - y)                      # u_theta = g sin(theta)
    u = ur * er + g * (ct * er - e[:, None])          # sin(theta) e_theta = cos(theta) e_r - e
    P = mu * U * (3.0 * x + 6.0 * y) / (R * R)
    p = P * (e @ xyz)
    c = sign * gamma / math.sqrt(kappa)
    f = -p * er + c * (u - ur * er)
    return ur, p, u, f


def bjs_velocity_stokes(xyz, R, kappa, gamma, mu, uinf, sign=1.0):
    """Exterior velocity of the slip porous sphere at |x| >= R, [3][N]."""
    U, e = _dir(uinf)
    x, y = bjs_sphere_coefficients(R, kappa, gamma, mu, sign)
    A1, A2 = x * R, y * R ** 3
    r = np.sqrt((xyz * xyz).sum(0))
    ct = (e @ xyz) / r
    er = xyz / r
    ur = U * ct * (1.0 + A1 / r + A2 / r ** 3)
    g = -0.5 * U * (2.0 + A1 / r - A2 / r ** 3)
    return ur * er + g * (ct * er - e[:, None])
