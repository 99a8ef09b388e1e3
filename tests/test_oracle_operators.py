"""Pins of the oracle's four layer operators (Sections 5.1-5.3).

Each identity below is a property of the continuous operators that the
smoothed, discretised ones reproduce exactly (subtraction identities) or at
high order in h (jump relations, spherical-harmonic eigenvalues, the Green
identities of the Fig. 4 tests).  Together they fix every sign, factor and
operand of the four kernels.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import analytic as A
from oracle import quadrature as Q


@pytest.fixture(scope="module")
def sph8():
    return Q.sphere_points(1.0, 1 / 8)


@pytest.fixture(scope="module")
def sph16():
    return Q.sphere_points(1.0, 1 / 16)


def test_subtraction_annihilates_constants_and_rigid_motion():
    p = Q.ellipsoid_points((1.0, 0.7, 0.5), 1 / 12)
    d = 3 / 12
    assert np.all(oracle.laplace_dl(p, d, np.full(p["w"].size, 2.5)) == 0.0)
    U = np.array([0.3, -0.2, 1.0])[:, None] * np.ones(p["w"].size)
    assert np.all(oracle.stokes_dl(p, d, U) == 0.0)
    rot = np.cross(np.array([0.3, -1.0, 0.5]), p["xyz"].T).T
    assert np.abs(oracle.stokes_dl(p, d, rot)).max() < 1e-14


def _sphere_eig_errors(p, h):
    d = 3 * h
    x, y, z = p["xyz"]
    return (np.abs(oracle.laplace_sl(p, d, z) + z / 3).max(),
            np.abs(oracle.laplace_sl(p, d, x * y) + x * y / 5).max(),
            np.abs(oracle.laplace_dl(p, d, z) + z / 3).max(),
            np.abs(oracle.laplace_dl(p, d, x * y) + 2 * x * y / 5).max())


def test_laplace_sphere_eigenvalues(sph8, sph16):
    # L Y_n = -Y_n/(2n+1), D^L Y_n = -n/(2n+1) Y_n on the unit sphere
    e8 = _sphere_eig_errors(sph8, 1 / 8)
    e16 = _sphere_eig_errors(sph16, 1 / 16)
    for a, b in zip(e8, e16):
        assert a < 2e-3 and b < 6e-5
        assert a / b > 20          # close to O(h^5)


def test_stokes_single_layer_sphere(sph16):
    # int_sphere S dS = (16 pi R/3) I, so M f = 2R/(3 mu) f for constant f
    R, mu, h = 0.8, 2.0, 1 / 16
    p = Q.sphere_points(R, h)
    f = np.array([0.3, -0.2, 1.0])[:, None] * np.ones(p["w"].size)
    Mf = oracle.stokes_sl(p, 3 * h, mu, f)
    assert np.abs(Mf - 2 * R / (3 * mu) * f).max() < 5e-5
    # a uniform normal load produces no velocity: int S n dS = 0
    Mn = oracle.stokes_sl(sph16, 3 * h, 1.0, sph16["nrm"])
    assert np.abs(Mn).max() < 5e-5


def test_single_layers_far_targets():
    # potential of a uniform shell at |y| > R: -R^2/|y|; Stokeslet far field
    p = Q.sphere_points(1.0, 1 / 32)
    ty = np.array([[5.0, 0.0], [0.0, 0.0], [0.0, 7.0]])
    v = oracle.laplace_sl(p, 3 / 32, np.ones(p["w"].size), targets=ty)
    assert v == pytest.approx([-1 / 5, -1 / 7], rel=1e-5)
    # uniform traction F/(4 pi R^2) on a sphere: exterior field of a rigid
    # translating sphere, u = (1/(8 pi mu)) [(1 + R^2/(3 r^2)) F/r + (1 - R^2/r^2) (r.F) r / r^3]
    F = np.array([0.0, 0.0, 1.0])
    f = F[:, None] * np.ones(p["w"].size) / (4 * math.pi)
    u = oracle.stokes_sl(p, 3 / 32, 1.0, f, targets=ty)
    for k in range(2):
        r = ty[:, k]
        rr = np.linalg.norm(r)
        ex = ((1 + 1 / (3 * rr ** 2)) * F / rr + (1 - 1 / rr ** 2) * (r @ F) * r / rr ** 3) / (8 * math.pi)
        assert u[:, k] == pytest.approx(ex, rel=1e-5, abs=1e-9)


def _darcy_identity(h):
    # interior harmonic p = e^x sin y on R = 0.8 (Fig. 4 test): D^L p = L dp/dn
    p = Q.sphere_points(0.8, h)
    x, y, z = p["xyz"]
    n = p["nrm"]
    P = np.exp(x) * np.sin(y)
    dP = np.exp(x) * (np.sin(y) * n[0] + np.cos(y) * n[1])
    res = oracle.laplace_dl(p, 3 * h, P) - oracle.laplace_sl(p, 3 * h, dP)
    return np.sqrt((res ** 2).mean())


def _stokes_identity(h):
    # exterior Stokeslet (1,0,0) at (0.2,0,0), R = 0.8 (Fig. 4 test):
    # u = -M f + D^S u with f = sigma . n
    p = Q.sphere_points(0.8, h)
    u, sig = A.stokeslet(p["xyz"], [0.2, 0.0, 0.0], [1.0, 0.0, 0.0], 1.0)
    f = np.einsum("ikn,kn->in", sig, p["nrm"])
    res = u - (-oracle.stokes_sl(p, 3 * h, 1.0, f) + oracle.stokes_dl(p, 3 * h, u))
    return np.sqrt((res ** 2).sum(0).mean())


def test_green_identities_fig4():
    d8, d16 = _darcy_identity(1 / 8), _darcy_identity(1 / 16)
    s8, s16 = _stokes_identity(1 / 8), _stokes_identity(1 / 16)
    assert d16 < 1e-4 and s16 < 5e-5
    assert d8 / d16 > 12 and s8 / s16 > 12
