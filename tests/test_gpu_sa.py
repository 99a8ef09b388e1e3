"""Relaxed D-N sweeps with warm-started successive approximations on the
device (the SA columns of Tables 1-2) against the oracle."""
import numpy as np
import pytest

from conftest import read_golden
from oracle import quadrature as Q
from oracle import solvers as S

pytestmark = pytest.mark.gpu


def _prm(ssd, h, kappa, theta, warm, use_sa=True):
    inner = ssd.krylov(1e-9, 1000, 50, use_sa, ssd.FP64, False, warm)
    return ssd.ddm_params(mu=1.0, kappa=kappa, gamma=0.0, uinf=(0.0, 0.0, 1.0), delta=3 * h, theta=theta,
                          tol_outer=1e-9, maxit_outer=100, outer_gmres=False,
                          traction_mode=ssd.TRACTION_JOSEPH_TAO, radius=1.0, inner=inner)


def test_warm_sa_matches_oracle_h8(gpu_ctx):
    import paper_2110_10749_gb300 as ssd
    h = 1 / 8
    p = Q.sphere_points(1.0, h)
    P = ssd.Points.from_numpy(p).prepare(gpu_ctx)
    r = ssd.ddm_solve(gpu_ctx, P, _prm(ssd, h, 1.0, 0.75, True))
    o = S.ddm_solve(p, 3 * h, 1.0, 1.0, 0.0, [0.0, 0.0, 1.0], 0.75, tol=1e-9, maxit=100, outer="sa",
                    traction="jt", R=1.0, use_sa=True, warm_inner=True)
    assert r["outer_its"] == o["outer_its"]
    for (dg, sg), (do, so) in zip(r["inner_its"], o["inner_its"]):
        assert abs(dg - do) <= 1 and abs(sg - so) <= 1
    for k in ("q", "p", "u"):
        a, b = r[k].cpu().numpy(), o[k]
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-8, k
    # a cold start converges to the same sweeps with more local iterations
    c = ssd.ddm_solve(gpu_ctx, P, _prm(ssd, h, 1.0, 0.75, False))
    assert c["outer_its"] == r["outer_its"]
    assert sum(s for _, s in c["inner_its"]) > sum(s for _, s in r["inner_its"])
    P.release()


@pytest.mark.parametrize("theta", [0.5, 0.75])
def test_sweep_counts_table1_h16(gpu_ctx, theta):
    import paper_2110_10749_gb300 as ssd
    row = [x for x in read_golden("sa_counts.txt") if x[0] == "1.0" and x[1] == "16" and float(x[2]) == theta][0]
    h = 1 / 16
    q = ssd.quadrature_points(gpu_ctx, ssd.SPHERE, (1.0,), h)
    P = ssd.Points(q["xyz"], q["nrm"], q["w"]).prepare(gpu_ctx)
    r = ssd.ddm_solve(gpu_ctx, P, _prm(ssd, h, 1.0, theta, True))
    # one more than printed: the first sweep's residual is 1 by definition
    assert r["outer_its"] == int(row[3]) + 1
    d = [a for a, _ in r["inner_its"]][1:r["outer_its"]]
    s = [b for _, b in r["inner_its"]][:r["outer_its"]]
    assert d[-1] <= 2 and s[-1] <= 2 and d[0] >= 20 and s[0] >= 20
    P.release()
