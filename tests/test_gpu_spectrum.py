"""Spectrum of the discrete D-N iteration matrix (eq. A_mat, Fig. 5) on the
device: Ritz values against the eigenvalues of the oracle's dense matrix
A~ assembled by its definition (eq. A_mat), against the eigenvalues of the
returned Hessenberg matrix, and the n = 1 mode of the porous sphere against
its closed form."""
import numpy as np
import pytest

from oracle import quadrature as Q
from oracle import solvers as S

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kappa,theta", [(1.0, 0.5), (1e-2, 0.005)])
def test_spectrum_matches_oracle(gpu_ctx, kappa, theta):
    import paper_2110_10749_gb300 as ssd
    h = 1 / 8
    p = Q.sphere_points(1.0, h)
    P = ssd.Points.from_numpy(p).prepare(gpu_ctx)
    inner = ssd.krylov(1e-13, 300, 100, False, ssd.FP64, False)
    prm = ssd.ddm_params(mu=1.0, kappa=kappa, gamma=0.0, uinf=(0.0, 0.0, 1.0), delta=3 * h, theta=theta,
                         tol_outer=1e-12, maxit_outer=80, outer_gmres=True, traction_mode=ssd.TRACTION_JOSEPH_TAO,
                         radius=1.0, inner=inner)
    ritz, H = ssd.ddm_spectrum(gpu_ctx, P, prm, 40)
    assert H.shape[1] == ritz.size
    ref = np.linalg.eigvals(H[:-1, :])
    assert np.abs(np.sort_complex(ritz) - np.sort_complex(ref)).max() < 1e-9
    ev = np.linalg.eigvals(S.iteration_matrix(p, 3 * h, 1.0, kappa, theta))
    # the extreme (well separated) eigenvalues: the n = 1 and n = 2 modes
    a = np.sort(ritz.real)[:8]
    b = np.sort(ev.real)[:8]
    assert np.abs(a - b).max() < 1e-7 * max(1.0, np.abs(b).max())
    # every Ritz value lies within the dense spectrum's range
    assert ritz.real.min() >= ev.real.min() - 1e-7 and ritz.real.max() <= ev.real.max() + 1e-7
    # n = 1: (1 - theta) - theta R^2 / (3 kappa), from the exterior Stokeslet
    a1 = (1 - theta) - theta / (3 * kappa)
    assert np.abs(a[:3] - a1).max() < 5e-3 * max(1.0, abs(a1))
    P.release()


@pytest.mark.parametrize("kappa,theta", [(1.0, 0.5), (1e-2, 0.005)])
def test_assembled_iteration_matrix_matches_oracle_definition(gpu_ctx, kappa, theta):
    """A~ assembled on the device column by column from sweeps (FP64, and
    FP32C) against the oracle's dense A~ of eq. A_mat, entry by entry, and
    their eigenvalues."""
    import paper_2110_10749_gb300 as ssd
    h = 1 / 8
    p = Q.sphere_points(1.0, h)
    P = ssd.Points.from_numpy(p).prepare(gpu_ctx)
    Ao = S.iteration_matrix(p, 3 * h, 1.0, kappa, theta)
    res = {}
    for prec, tol_in in ((ssd.FP64, 1e-13), (ssd.FP32C, 1e-9)):
        inner = ssd.krylov(tol_in, 300, 300, False, prec, False)
        prm = ssd.ddm_params(mu=1.0, kappa=kappa, gamma=0.0, uinf=(0.0, 0.0, 1.0), delta=3 * h, theta=theta,
                             tol_outer=1e-12, maxit_outer=80, outer_gmres=True, traction_mode=ssd.TRACTION_BJS,
                             inner=inner)
        res[prec] = ssd.ddm_iteration_matrix(gpu_ctx, P, prm).cpu().numpy()
    scale = np.abs(Ao - (1 - theta) * np.eye(Ao.shape[0])).max()
    assert np.abs(res[ssd.FP64] - Ao).max() < 1e-9 * scale
    # FP32C: the pair-sum rounding relative to the sweep's own size
    assert np.abs(res[ssd.FP32C] - Ao).max() < 1e-5 * np.abs(Ao).max()
    ev = np.sort(np.linalg.eigvals(res[ssd.FP64]).real)
    evo = np.sort(np.linalg.eigvals(Ao).real)
    assert np.abs(ev - evo).max() < 1e-8 * max(1.0, np.abs(evo).max())
    # a block of columns equals the same columns of the whole matrix
    blk = ssd.ddm_iteration_matrix(gpu_ctx, P, prm, col0=100, ncol=7).cpu().numpy()
    assert np.abs(blk - res[ssd.FP32C][:, 100:107]).max() < 1e-12 * np.abs(Ao).max()
    P.release()
