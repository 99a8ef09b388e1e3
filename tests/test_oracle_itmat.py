"""Pins of the dense discrete iteration matrix (eq. A_mat, Section 6) of the
oracle: the dense operator matrices against the matrix-free operators, the
assembled matrix against one D-N sweep, and its spectrum against the n = 1
closed form of the porous sphere and the scaling in mu/kappa and theta that
eq. A_mat fixes."""
import numpy as np

import oracle
from oracle import quadrature as Q
from oracle import solvers as S


def test_operator_matrices_match_the_matrix_free_operators():
    h = 1 / 6
    p = Q.ellipsoid_points((1.0, 0.8, 0.6), h, center=(0.1, 0.0, -0.05))
    N = p["w"].size
    rng = np.random.default_rng(4)
    g, v = rng.normal(size=N), rng.normal(size=(3, N))
    d = 3 * h
    pairs = (("L", oracle.laplace_sl(p, d, g), g), ("DL", oracle.laplace_dl(p, d, g), g),
             ("M", oracle.stokes_sl(p, d, 1.7, v).ravel(), v.ravel()), ("DS", oracle.stokes_dl(p, d, v).ravel(),
                                                                        v.ravel()))
    for op, y, x in pairs:
        A = oracle.operator_matrix(p, d, op, mu=1.7)
        assert np.abs(A @ x - y).max() < 1e-13 * np.abs(y).max(), op
    # subtraction: the double layers annihilate constants and rigid motions
    DL = oracle.operator_matrix(p, d, "DL")
    assert np.abs(DL.sum(1)).max() < 1e-13
    DS = oracle.operator_matrix(p, d, "DS")
    for e in np.eye(3):
        assert np.abs(DS @ np.repeat(e, N)).max() < 1e-13


def _sweep_linear(p, h, kappa, theta, q):
    pd, _, _ = S.darcy_solve(p, 3 * h, 1.0, kappa, q, tol=1e-14, restart=200, maxit=2000)
    u, _, _ = S.stokes_solve(p, 3 * h, 1.0, -pd * p["nrm"], [0.0, 0.0, 0.0], tol=1e-14, restart=200, maxit=2000)
    return (1 - theta) * q + theta * (u * p["nrm"]).sum(0)


def test_matrix_is_the_linear_part_of_one_sweep():
    h = 1 / 6
    p = Q.sphere_points(1.0, h)
    kappa, theta = 0.3, 0.4
    A = S.iteration_matrix(p, 3 * h, 1.0, kappa, theta)
    q = np.random.default_rng(8).normal(size=p["w"].size)
    ref = _sweep_linear(p, h, kappa, theta, q)
    assert np.abs(A @ q - ref).max() < 1e-11 * np.abs(ref).max()


def test_spectrum_n1_mode_and_scaling():
    h = 1 / 8
    p = Q.sphere_points(1.0, h)
    ev = {}
    for kappa, theta in ((1.0, 0.5), (1e-2, 0.005)):
        ev[kappa] = np.linalg.eigvals(S.iteration_matrix(p, 3 * h, 1.0, kappa, theta))
        assert np.abs(ev[kappa].imag).max() < 1e-8
        lam = np.sort(ev[kappa].real)
        a1 = (1 - theta) - theta / (3 * kappa)
        # the three lowest eigenvalues are the degree-one modes: within the
        # discretization error of the closed form, and equal to each other
        assert np.abs(lam[:3] - a1).max() < 5e-3 * max(1.0, abs(a1))
        assert lam[2] - lam[0] < 1e-8
        # the rest lie between the degree-one modes and 1 - theta
        assert lam[3] > lam[2] and lam[-1] < (1 - theta) + 1e-8
    # A~ = (1 - theta) I - (theta / kappa) X with X independent of kappa and theta
    x1 = np.sort(((1 - 0.5) - ev[1.0].real) / (0.5 / 1.0))
    x2 = np.sort(((1 - 0.005) - ev[1e-2].real) / (0.005 / 1e-2))
    assert np.abs(x1 - x2).max() < 1e-9
