"""Pins of the oracle's BJS-slip D-N solve against the porous sphere with slip.

The closed form (oracle/analytic.py, derived from eqs. Vel_contin,
BeaversJoseph and Press_contin) is first checked symbolically: the exterior
field solves the Stokes equations, and on r = R it satisfies mass
conservation with the interior Darcy flow, the normal-stress balance and the
slip condition.  The oracle's lagged (Section 3, step 2) and implicit D-N
solves are then compared with it; the opposite slip sign (s = -1, as printed
in eq. f) gives a different drag and field, so the pins tell the two readings
apart.
"""
import math

import numpy as np
import pytest

from oracle import analytic as A
from oracle import quadrature as Q
from oracle import solvers as S


def test_closed_form_satisfies_stokes_and_interface_conditions():
    sp = pytest.importorskip("sympy")
    r, th = sp.symbols("r theta", positive=True)
    R, kap, gam, mu, U = sp.Rational(13, 10), sp.Rational(3, 100), sp.Rational(7, 10), sp.Rational(3, 2), \
        sp.Rational(2, 1)
    for sign in (1, -1):
        x, y = A.bjs_sphere_coefficients(float(R), float(kap), float(gam), float(mu), sign)
        # exact rationals for the symbolic check: re-derive x, y from the same
        # linear system with sympy and compare with the floats
        X, Y = sp.symbols("X Y")
        b = sign * gam * R / (mu * sp.sqrt(kap))
        k = kap / R ** 2
        sol = sp.solve([1 + X + Y + k * (3 * X + 6 * Y), 6 * Y - b * (2 + X - Y)], [X, Y], dict=True)[0]
        assert abs(float(sol[X]) - x) < 1e-13 and abs(float(sol[Y]) - y) < 1e-13
        A1, A2 = sol[X] * R, sol[Y] * R ** 3
        psi = U / 2 * sp.sin(th) ** 2 * (r ** 2 + A1 * r + A2 / r)
        ur = sp.diff(psi, th) / (r ** 2 * sp.sin(th))
        ut = -sp.diff(psi, r) / (r * sp.sin(th))
        p = mu * U * A1 * sp.cos(th) / r ** 2
        # Stokes equations in spherical coordinates (axisymmetric, no swirl)
        lap = lambda f: sp.diff(r ** 2 * sp.diff(f, r), r) / r ** 2 + \
            sp.diff(sp.sin(th) * sp.diff(f, th), th) / (r ** 2 * sp.sin(th))
        mom_r = -sp.diff(p, r) + mu * (lap(ur) - 2 * ur / r ** 2 - 2 * sp.diff(ut * sp.sin(th), th)
                                       / (r ** 2 * sp.sin(th)))
        mom_t = -sp.diff(p, th) / r + mu * (lap(ut) + 2 * sp.diff(ur, th) / r ** 2 - ut / (r ** 2 * sp.sin(th) ** 2))
        div = sp.diff(r ** 2 * ur, r) / r ** 2 + sp.diff(sp.sin(th) * ut, th) / (r * sp.sin(th))
        for e in (mom_r, mom_t, div):
            assert sp.simplify(e) == 0
        # far field U e_z: u_r -> U cos, u_theta -> -U sin
        assert sp.limit(ur - U * sp.cos(th), r, sp.oo) == 0
        srr = -p + 2 * mu * sp.diff(ur, r)
        srt = mu * (sp.diff(ut, r) - ut / r + sp.diff(ur, th) / r)
        P = mu * U * (3 * sol[X] + 6 * sol[Y]) / R ** 2
        pD = P * r * sp.cos(th)
        uD_r = -(kap / mu) * sp.diff(pD, r)
        at = lambda e: sp.simplify(e.subs(r, R))
        assert at(ur - uD_r) == 0                                   # eq. Vel_contin
        assert at(srr + pD) == 0                                    # eq. Press_contin
        assert at(srt - sign * gam / sp.sqrt(kap) * ut) == 0        # eq. BeaversJoseph (coefficient as in eq. f)
        # drag = integral of f . e_z over the sphere = -4 pi mu U A1
        fz = srr * sp.cos(th) - srt * sp.sin(th)
        drag = sp.integrate(at(fz) * 2 * sp.pi * R ** 2 * sp.sin(th), (th, 0, sp.pi))
        assert abs(float(drag) - A.bjs_drag(float(R), float(kap), float(gam), float(mu), float(U), sign)) < 1e-12


def test_closed_form_limits():
    # shear-free (gamma = 0): x = -1/(1 + 3k); no-slip limit: x -> -(3 + 12k)/(2 + 9k)
    for kap in (1.0, 1e-2):
        x, y = A.bjs_sphere_coefficients(1.0, kap, 0.0)
        assert abs(x + 1.0 / (1.0 + 3.0 * kap)) < 1e-15 and y == 0.0
        x, _ = A.bjs_sphere_coefficients(1.0, kap, 1e12)
        assert abs(x + (3.0 + 12.0 * kap) / (2.0 + 9.0 * kap)) < 1e-9
    # kappa -> 0 with fixed gamma: the impermeable no-slip sphere, 6 pi mu R U
    assert abs(A.bjs_drag(1.0, 1e-14, 1.0, 1.0, 1.0) - 6.0 * math.pi) < 1e-5


def _errs(r, pts, kappa, gamma, sign=1.0):
    """Drag error relative to the drag; q and u errors relative to the
    far-field speed U = 1 (the interface velocity is O(kappa U) in the normal
    direction and small tangentially when the slip coefficient is large);
    p and f errors relative to their own size."""
    q, p, u, f = A.bjs_interface_fields(pts["xyz"], 1.0, kappa, gamma, 1.0, (0.0, 0.0, 1.0), sign)
    d = A.bjs_drag(1.0, kappa, gamma, 1.0, 1.0, sign)
    return ((r["drag"][2] - d) / d, S.rms(r["q"] - q), S.rms(r["p"] - p) / S.rms(p),
            S.rms(r["u"] - u), S.rms(r["f"] - f) / S.rms(f))


@pytest.mark.parametrize("kappa,gamma,hinv,bound", [(1.0, 0.5, 8, 5e-3), (1e-2, 1.0, 8, 1e-2),
                                                    (1e-4, 1.0, 6, 5e-2)])
def test_lagged_ddm_matches_slip_sphere(kappa, gamma, hinv, bound):
    h = 1.0 / hinv
    pts = Q.sphere_points(1.0, h)
    r = S.ddm_solve(pts, 3 * h, 1.0, kappa, gamma, (0.0, 0.0, 1.0), 0.5 * min(kappa, 1.0), tol=1e-9, maxit=400,
                    outer="gmres", traction="bjs", inner_tol=1e-11, restart=100)
    errs = _errs(r, pts, kappa, gamma)
    assert max(abs(e) for e in errs) < bound, errs
    # the other sign reading is far away: at least 100 times the error
    d_plus = A.bjs_drag(1.0, kappa, gamma, 1.0, 1.0, 1.0)
    d_minus = A.bjs_drag(1.0, kappa, gamma, 1.0, 1.0, -1.0)
    assert abs(r["drag"][2] - d_minus) > 100.0 * abs(r["drag"][2] - d_plus)


def test_slip_sphere_error_falls_with_h():
    errs = []
    for h in (1.0 / 8, 1.0 / 12):
        pts = Q.sphere_points(1.0, h)
        r = S.ddm_solve(pts, 3 * h, 1.0, 1.0, 0.5, (0.0, 0.0, 1.0), 0.5, tol=1e-10, maxit=100, outer="gmres",
                        traction="bjs", inner_tol=1e-12)
        errs.append(_errs(r, pts, 1.0, 0.5))
    for a, b in zip(errs[0], errs[1]):
        assert abs(b) < abs(a) / 4.0, errs     # O(h^5) for the delta = 3h method: (3/2)^5 = 7.6


def test_negative_sign_reading_matches_its_closed_form():
    # bjs_sign = -1 (eq. f as printed) solves a different problem: the s = -1 closed form
    h = 1.0 / 8
    pts = Q.sphere_points(1.0, h)
    r = S.ddm_solve(pts, 3 * h, 1.0, 1.0, 0.5, (0.0, 0.0, 1.0), 0.5, tol=1e-10, maxit=100, outer="gmres",
                    traction="bjs", inner_tol=1e-12, bjs_sign=-1.0)
    errs = _errs(r, pts, 1.0, 0.5, sign=-1.0)
    assert max(abs(e) for e in errs) < 5e-2, errs


def test_implicit_slip_matches_slip_sphere():
    h = 1.0 / 8
    pts = Q.sphere_points(1.0, h)
    r = S.ddm_solve(pts, 3 * h, 1.0, 1e-2, 1.0, (0.0, 0.0, 1.0), 0.005, tol=1e-10, maxit=100, outer="gmres",
                    traction="bjs", inner_tol=1e-12, bjs_implicit=True)
    errs = _errs(r, pts, 1e-2, 1.0)
    assert max(abs(e) for e in errs) < 2e-2, errs
