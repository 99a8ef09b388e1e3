"""Pins of the oracle's star-shaped surfaces (r = 1 + sum c_lm Y_lm, l <= 4)
and of their quadrature sets (Section 5.4, eq. Quadrature, applied to the
level set phi = |x - c| - r(xi)).

The real harmonics are pinned against scipy's complex ones, orthonormality
and finite differences; the quadrature sets against the sphere generator
(the l = 0 case), finite-difference normals, and area and volume integrals
of the same surface taken by a tensor Gauss rule in (theta, phi)."""
import math

import numpy as np
import pytest
import scipy.special as sps

from oracle import quadrature as Q
from paper_2110_10749_gb300.workloads import star_coefficients


def real_sh(l, m, theta, phi):
    """Real orthonormal Y_lm from scipy's complex Y_l^m (Condon-Shortley phase)."""
    if m == 0:
        return sps.sph_harm_y(l, 0, theta, phi).real
    y = sps.sph_harm_y(l, abs(m), theta, phi)
    f = math.sqrt(2.0) * (-1.0) ** abs(m)
    return f * (y.real if m > 0 else y.imag)


def unit_vectors(n, seed):
    v = np.random.default_rng(seed).normal(size=(3, n))
    return v / np.linalg.norm(v, axis=0)


def test_real_harmonics_match_scipy():
    xi = unit_vectors(200, 1)
    theta = np.arccos(xi[2])
    phi = np.arctan2(xi[1], xi[0])
    p, _, _, _ = Q.star_polys(*xi)
    K = Q.star_constants()
    for l in range(5):
        for m in range(-l, l + 1):
            k = l * l + l + m
            assert np.abs(K[k] * p[k] - real_sh(l, m, theta, phi)).max() < 1e-13, (l, m)


def test_harmonics_orthonormal():
    # Gauss-Legendre in cos(theta) x trapezoid in phi integrates degree <= 8 exactly
    xg, wg = np.polynomial.legendre.leggauss(12)
    nphi = 24
    ph = 2 * np.pi * np.arange(nphi) / nphi
    CT, PH = np.meshgrid(xg, ph, indexing="ij")
    ST = np.sqrt(1 - CT ** 2)
    xi = (ST * np.cos(PH), ST * np.sin(PH), CT)
    W = np.outer(wg, np.full(nphi, 2 * np.pi / nphi))
    p, _, _, _ = Q.star_polys(*xi)
    Y = np.stack([Q.star_constants()[k] * p[k] for k in range(25)])
    G = np.einsum("kab,jab,ab->kj", Y, Y, W)
    assert np.abs(G - np.eye(25)).max() < 1e-13


def test_polynomial_gradients_by_finite_differences():
    X = np.random.default_rng(2).normal(size=(3, 50))
    e = 1e-6
    _, gx, gy, gz = Q.star_polys(*X)
    for d, g in enumerate((gx, gy, gz)):
        Xp, Xm = X.copy(), X.copy()
        Xp[d] += e
        Xm[d] -= e
        pp, _, _, _ = Q.star_polys(*Xp)
        pm, _, _, _ = Q.star_polys(*Xm)
        for k in range(25):
            fd = (pp[k] - pm[k]) / (2 * e)
            assert np.abs(np.asarray(g[k]) + 0 * X[0] - fd).max() < 1e-7 * (1 + np.abs(fd).max()), (d, k)
    a = star_coefficients(5) * Q.star_constants()
    P, G = Q.star_eval(a, X)
    for d in range(3):
        Xp, Xm = X.copy(), X.copy()
        Xp[d] += e
        Xm[d] -= e
        fd = (Q.star_eval(a, Xp)[0] - Q.star_eval(a, Xm)[0]) / (2 * e)
        assert np.abs(G[d] - fd).max() < 1e-7


@pytest.mark.parametrize("c00,h,center", [(0.0, 1 / 16, (0, 0, 0)), (0.3, 1 / 12, (0.05, -0.1, 0.2))])
def test_l0_star_is_sphere(c00, h, center):
    clm = np.zeros(25)
    clm[0] = c00
    R = 1.0 + c00 * Q.star_constants()[0]
    s = Q.star_points(clm, h, center=center)
    o = Q.sphere_points(R, h, center=center)
    assert np.array_equal(s["meta"], o["meta"])
    assert np.abs(s["xyz"] - o["xyz"]).max() <= 4e-16 * (1 + R)
    assert np.abs(s["nrm"] - o["nrm"]).max() <= 1e-15
    # acos in the partition of unity amplifies last-bit differences of the normals
    assert np.abs(s["w"] - o["w"]).max() <= 1e-14 * o["w"].max()


def _surface_integrals(clm, center=(0.0, 0.0, 0.0), n=96):
    """Area and volume of the star surface by Gauss-Legendre x trapezoid."""
    xg, wg = np.polynomial.legendre.leggauss(n)
    nphi = 2 * n
    ph = 2 * np.pi * np.arange(nphi) / nphi
    CT, PH = np.meshgrid(xg, ph, indexing="ij")
    ST = np.sqrt(1 - CT ** 2)
    xi = np.stack([ST * np.cos(PH), ST * np.sin(PH), CT])
    W = np.outer(wg, np.full(nphi, 2 * np.pi / nphi))
    a = clm * Q.star_constants()
    P, g = Q.star_eval(a, xi)
    r = 1.0 + P
    g = np.stack(g)
    gt = g - (g * xi).sum(0) * xi            # surface gradient of r on the unit sphere
    area = (r * np.sqrt(r * r + (gt * gt).sum(0)) * W).sum()
    vol = (r ** 3 * W).sum() / 3.0
    return area, vol


@pytest.mark.parametrize("seed", [0, 7])
def test_star_area_volume_and_closure(seed):
    clm = star_coefficients(seed)
    area, vol = _surface_integrals(clm)
    errs = []
    for h in (1 / 16, 1 / 32):
        q = Q.star_points(clm, h)
        A = q["w"].sum()
        V = (q["w"] * (q["xyz"] * q["nrm"]).sum(0)).sum() / 3.0
        # a closed surface: the weighted normals sum to zero
        C = np.abs((q["w"] * q["nrm"]).sum(1)).max()
        errs.append((abs(A / area - 1), abs(V / vol - 1), C))
    assert errs[1][0] < 1e-5 and errs[1][1] < 1e-5 and errs[1][2] < 1e-4, errs
    for k in range(3):
        assert errs[1][k] < errs[0][k] / 5, errs


def test_star_points_on_surface_and_normals():
    clm = star_coefficients(3)
    c = (0.02, -0.03, 0.01)
    q = Q.star_points(clm, 1 / 16, center=c)
    a = clm * Q.star_constants()
    X = q["xyz"]
    d = X - np.asarray(c)[:, None]
    rho = np.linalg.norm(d, axis=0)
    xi = d / rho
    P, _ = Q.star_eval(a, xi)
    assert np.abs(rho - (1.0 + P)).max() < 1e-14
    # normal from finite-difference tangents of x(xi) = c + r(xi) xi
    e = 1e-6
    t1 = np.cross(xi.T, np.array([0.3, 0.5, 0.8])).T
    t1 /= np.linalg.norm(t1, axis=0)
    t2 = np.cross(xi.T, t1.T).T

    def X_of(v):
        v = v / np.linalg.norm(v, axis=0)
        return np.asarray(c)[:, None] + (1.0 + Q.star_eval(a, v)[0]) * v
    T1 = (X_of(xi + e * t1) - X_of(xi - e * t1)) / (2 * e)
    T2 = (X_of(xi + e * t2) - X_of(xi - e * t2)) / (2 * e)
    N = np.cross(T1.T, T2.T).T
    N /= np.linalg.norm(N, axis=0)
    N *= np.sign((N * xi).sum(0))
    assert np.abs(N - q["nrm"]).max() < 1e-8
    assert np.all(np.abs(q["nrm"][q["meta"][0], np.arange(X.shape[1])]) >= Q.cos_threshold(70.0))


def test_star_roots_complete_on_dense_lines():
    """Every kept crossing is found: dense sampling of a subset of lines finds
    no further root with |n_i| >= cos(70 deg)."""
    clm = star_coefficients(11)
    h = 1 / 12
    q = Q.star_points(clm, h)
    a = clm * Q.star_constants()
    rb = Q.star_bound(clm)
    ct = Q.cos_threshold(70.0)
    rng = np.random.default_rng(4)
    found = {}
    for k in range(q["w"].size):
        key = tuple(int(v) for v in q["meta"][:3, k])
        found[key] = found.get(key, 0) + 1
    for i in range(3):
        a_, b_ = Q.OTHER[i]
        J = int(math.ceil(rb / h)) + 1
        for _ in range(40):
            ja, jb = rng.integers(-J, J + 1, size=2)
            t = np.linspace(-1.1 * rb, 1.1 * rb, 20001)
            X = np.zeros((3, t.size))
            X[i], X[a_], X[b_] = t, ja * h, jb * h
            F = Q.star_phi(a, (0, 0, 0), X)
            s = F > 0
            idx = np.nonzero(s[:-1] != s[1:])[0]
            kept = 0
            for j in idx:
                Xr = X[:, j:j + 1]
                n = Q.star_normal(a, (0, 0, 0), Xr)
                kept += int(abs(n[i, 0]) >= ct)
            assert found.get((i, int(ja), int(jb)), 0) == kept
