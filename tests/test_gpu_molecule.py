"""The four-atom molecule (eq. Molecule, Table 4) on the device: quadrature
points bit-identical to the oracle's, and a D-N solve on the molecule against
the oracle's solve on the same points."""
import numpy as np
import pytest

from oracle import quadrature as Q
from oracle import solvers as S

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("h,center", [(1 / 16, (0.0, 0.0, 0.0)), (1 / 32, (0.05, -0.02, 0.1))])
def test_molecule_points_match_oracle(gpu_ctx, h, center):
    import paper_2110_10749_gb300 as ssd
    g = {k: v.cpu().numpy() for k, v in ssd.molecule_points(gpu_ctx, h, center=center).items()}
    cen = [tuple(np.add(c, center)) for c in Q.MOLECULE_CENTERS]
    o = Q.molecule_points(h, centers=cen)
    # both sides evaluate the Gaussians with the same stated exponential
    # (Cody-Waite reduction, Taylor polynomial): points, normals and labels
    # are bit-identical; the weights' bump uses the libraries' exp
    assert np.array_equal(g["meta"], o["meta"])
    assert np.array_equal(g["xyz"], o["xyz"])
    assert np.array_equal(g["nrm"], o["nrm"])
    assert np.abs(g["w"] - o["w"]).max() <= 1e-14 * o["w"].max()


def test_molecule_ddm_matches_oracle(gpu_ctx):
    import paper_2110_10749_gb300 as ssd
    h = 1 / 8
    q = ssd.molecule_points(gpu_ctx, h)
    pts = {k: q[k].cpu().numpy() for k in ("xyz", "nrm", "w")}
    P = ssd.Points(q["xyz"], q["nrm"], q["w"]).prepare(gpu_ctx)
    kappa, gamma = 1e-2, 0.5
    inner = ssd.krylov(1e-12, 300, 100, False, ssd.FP64, True)
    prm = ssd.ddm_params(mu=1.0, kappa=kappa, gamma=gamma, uinf=(0.0, 0.0, 1.0), delta=3 * h, theta=1.0,
                         tol_outer=1e-11, maxit_outer=80, outer_gmres=True, traction_mode=ssd.TRACTION_BJS,
                         inner=inner, bjs_implicit=True)
    r = ssd.ddm_solve(gpu_ctx, P, prm)
    o = S.ddm_solve(pts, 3 * h, 1.0, kappa, gamma, [0.0, 0.0, 1.0], 1.0, tol=1e-11, maxit=80, outer="gmres",
                    traction="bjs", restart=100, inner_maxit=400, bjs_implicit=True, deflate=True)
    for k in ("q", "p", "u", "f"):
        a, b = r[k].cpu().numpy(), o[k]
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-8, k
    assert np.allclose(r["drag"], o["drag"], rtol=1e-9, atol=1e-9 * np.abs(o["drag"]).max())
    P.release()
