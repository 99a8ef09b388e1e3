"""The implicit-slip Stokes operator of the D-N sweep with the BJS traction
taken at the Stokes step's own velocity,
    A(c) = (I - D^S) + c M P + n (w . (u.n)) / sum(w),   P u = u - (u.n) n,
assembled column by column from the oracle's layer operators on the h = 1/6
unit sphere (N = 582, delta = 3h).  Without slip its spectrum lies in the
right half plane; as c = gamma/sqrt(kappa) grows, eigenvalues cross zero
(between c = 15 and 20 here) and at c = 100, the kappa = 1e-4, gamma = 1
case, dozens have negative real part.  This is the property that makes the
local GMRES of that case need long Krylov cycles."""
import numpy as np
import pytest

import oracle
from oracle import quadrature as Q


@pytest.fixture(scope="module")
def parts():
    oracle.build()
    h = 1.0 / 6
    p = Q.sphere_points(1.0, h)
    n = p["w"].size
    d = 3 * h

    def columns(f):
        out = np.zeros((3 * n, 3 * n))
        for k in range(3 * n):
            e = np.zeros(3 * n)
            e[k] = 1.0
            out[:, k] = f(e.reshape(3, n)).ravel()
        return out
    DS = columns(lambda u: oracle.stokes_dl(p, d, u))
    M = columns(lambda f: oracle.stokes_sl(p, d, 1.0, f))
    nv, w = p["nrm"], p["w"]
    Nm = np.zeros((3 * n, n))
    for c in range(3):
        Nm[c * n:(c + 1) * n, :] = np.diag(nv[c])
    P = np.eye(3 * n) - Nm @ Nm.T
    R1 = np.outer(nv.ravel(), Nm @ w) / w.sum()
    return np.eye(3 * n) - DS + R1, M @ P, (DS, M, P, Nm, nv, n)


def test_assembled_columns_apply_the_oracle_operator(parts):
    """The dense A(c) reproduces the matrix-free operator of the oracle's
    implicit-slip Stokes solve."""
    from oracle import solvers as S
    B0, MP, (DS, M, P, Nm, nv, n) = parts
    h = 1.0 / 6
    p = Q.sphere_points(1.0, h)
    rng = np.random.default_rng(4)
    u = rng.normal(size=(3, n))
    c = 7.0
    Pu = u - (u * nv).sum(0) * nv
    ref = u - oracle.stokes_dl(p, 3 * h, u) + c * oracle.stokes_sl(p, 3 * h, 1.0, Pu) + S.normal_flux_term(p, u)
    assert np.abs((B0 + c * MP) @ u.ravel() - ref.ravel()).max() < 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("c", [0.0, 10.0])
def test_small_slip_keeps_the_spectrum_in_the_right_half_plane(parts, c):
    B0, MP, _ = parts
    ev = np.linalg.eigvals(B0 + c * MP)
    assert ev.real.min() > 0.1


def test_large_slip_makes_the_operator_indefinite(parts):
    B0, MP, _ = parts
    ev = np.linalg.eigvals(B0 + 100.0 * MP)
    assert (ev.real < 0).sum() >= 20
    assert ev.real.min() < -1.0
    assert ev.real.max() > 30.0
