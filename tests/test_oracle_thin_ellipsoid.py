"""Pin of the oracle on the thin porous ellipsoid (1, 0.6, 0.4) (Section 7.4,
Table 3): with the BJS traction at gamma = 0 (f = -p_D n), U = e_z and
theta = kappa/2, the self-convergence errors between h = 1/16 and h = 1/32
at kappa = 1 reproduce the printed ||p_h - p_{h/2}|| and ||u_h - u_{h/2}||.
The points of the h set are points of the h/2 set: the same grid line
(indices doubled) and the same root."""
import numpy as np

from conftest import read_golden
from oracle import quadrature as Q
from oracle import solvers as S

ABC = (1.0, 0.6, 0.4)


def _solve(h, kappa):
    p = Q.ellipsoid_points(ABC, h)
    r = S.ddm_solve(p, 3 * h, 1.0, kappa, 0.0, [0.0, 0.0, 1.0], 0.5 * min(kappa, 1.0), tol=1e-9, maxit=60,
                    outer="gmres", traction="bjs", inner_tol=1e-10)
    return p, r


def coarse_in_fine(pc, pf):
    """Index in the h/2 set of every point of the h set (-1 if absent)."""
    key = {tuple(m): i for i, m in enumerate(pf["meta"].T)}
    return np.array([key.get((m[0], 2 * m[1], 2 * m[2], m[3]), -1) for m in pc["meta"].T])


def test_coarse_points_are_fine_points():
    pc, pf = Q.ellipsoid_points(ABC, 1 / 16), Q.ellipsoid_points(ABC, 1 / 32)
    idx = coarse_in_fine(pc, pf)
    assert (idx >= 0).all()
    assert np.array_equal(pc["xyz"], pf["xyz"][:, idx]) and np.array_equal(pc["nrm"], pf["nrm"][:, idx])


def test_self_convergence_errors_match_table3():
    rows = [r for r in read_golden("thin_ellipsoid_table3.txt") if float(r[0]) == 1.0 and r[1] == "16"]
    p_err, u_err = float(rows[0][7]), float(rows[0][8])
    pc, rc = _solve(1 / 16, 1.0)
    pf, rf = _solve(1 / 32, 1.0)
    assert pc["w"].size == int(rows[0][2]) and pf["w"].size == 6902
    idx = coarse_in_fine(pc, pf)
    ep = S.rms(rc["p"] - rf["p"][idx])
    eu = S.rms(rc["u"] - rf["u"][:, idx])
    assert abs(ep - p_err) < 2e-3 * p_err, ep
    assert abs(eu - u_err) < 2e-3 * u_err, eu
