"""Pins of the oracle's discrete iteration matrix (eq. A_mat) and of the n = 1
multiplier used to read Fig. 5 / eq. CA31."""
import numpy as np

from oracle import analytic as A
from oracle import quadrature as Q
from oracle import solvers as S

KW = dict(traction="jt", R=1.0, outer="gmres", tol=1e-12, inner_tol=1e-13, restart=100)


def test_exterior_stokeslet_normal_response():
    """A point force at the centre of a sphere of radius R has a purely normal
    traction -P cos(theta) e_r on it and normal velocity R P cos(theta)/(3 mu):
    the n = 1 response of the exterior traction problem."""
    R, mu = 0.7, 1.3
    p = Q.sphere_points(R, 1 / 8)
    u, sig = A.stokeslet(p["xyz"], [0.0, 0.0, 0.0], [0.0, 0.0, 1.0], mu)
    n = p["nrm"]
    f = np.einsum("ikn,kn->in", sig, n)
    fn = (f * n).sum(0)
    ft = f - fn * n
    assert np.abs(ft).max() < 1e-13 * np.abs(f).max()
    ur = (u * n).sum(0)
    assert np.allclose(ur, R * (-fn) / (3.0 * mu), rtol=1e-12, atol=1e-15)


def test_ritz_values_reach_the_invariant_subspace():
    h = 1 / 4
    p = Q.sphere_points(1.0, h)
    r40 = S.ddm_solve(p, 3 * h, 1.0, 1.0, 0.0, [0.0, 0.0, 1.0], 0.5, arnoldi=40, **KW)
    rfull = S.ddm_solve(p, 3 * h, 1.0, 1.0, 0.0, [0.0, 0.0, 1.0], 0.5, arnoldi=p["w"].size, **KW)
    assert rfull["H"].shape[1] < p["w"].size          # Arnoldi stopped on an invariant subspace
    a = np.sort(r40["ritz"].real)[:8]
    b = np.sort(rfull["ritz"].real)[:8]
    assert np.abs(a - b).max() < 1e-8


def test_n1_mode_of_the_sphere():
    h = 1 / 8
    p = Q.sphere_points(1.0, h)
    for kappa, theta in ((1.0, 0.5), (1.0, 1.0)):
        r = S.ddm_solve(p, 3 * h, 1.0, kappa, 0.0, [0.0, 0.0, 1.0], theta, arnoldi=30, **KW)
        a = np.sort(r["ritz"].real)[:3]
        a1 = (1 - theta) - theta / (3 * kappa)
        assert np.abs(a - a1).max() < 5e-3, (a, a1)
        # the three n = 1 eigenvalues coincide (rotational symmetry of the point set)
        assert a.max() - a.min() < 1e-8
