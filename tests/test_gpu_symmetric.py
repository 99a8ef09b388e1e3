"""The layer operators on the symmetric plans (far block pairs evaluated once
for both directions), FP32C and FP64: on the h = 1/48 sphere (N = 38310;
64% of the pairs in far block pairs at the FP32C smoothing radius, 61% at
the FP64 one) the whole application of each of the four operators against
the oracle element by element, and against the same operator with the plans
switched off (SSD_PAIR_SYM=0 when the context is created).  That the plan
ran is read from the library's launch counter: packing, near items, far
items and epilogue are four launches, the direct kernel's application three."""
import os

import numpy as np
import pytest

import oracle
from oracle import quadrature as Q

pytestmark = pytest.mark.gpu

H = 1 / 48
MU = 1.3


@pytest.fixture(scope="module")
def case():
    p = Q.sphere_points(1.0, H)
    n = p["w"].size
    d = 3 * H
    rng = np.random.default_rng(21)
    x, y, z = p["xyz"]
    g = np.exp(x) * np.sin(y) + 0.1 * rng.normal(size=n)
    v = np.stack([y * z, np.cos(x), x + 0.3 * z * z]) + 0.1 * rng.normal(size=(3, n))
    ref = {"LDL": oracle.laplace_dl(p, d, g), "SDL": oracle.stokes_dl(p, d, v),
           "LSL": oracle.laplace_sl(p, d, g), "SSL": oracle.stokes_sl(p, d, MU, v)}
    return p, d, g, v, ref


def _apply(ssd, ctx, P, d, tg, tv, prec):
    return {"LDL": ssd.laplace_DL(ctx, P, d, tg, prec), "SDL": ssd.stokes_DL(ctx, P, d, tv, prec),
            "LSL": ssd.laplace_SL(ctx, P, d, tg, prec), "SSL": ssd.stokes_SL(ctx, P, d, MU, tv, prec)}


@pytest.mark.parametrize("prec_name,tol_ref,tol_direct", [("FP32C", 1e-5, 1e-6), ("FP64", 1e-12, 1e-13)])
def test_symmetric_plan_matches_oracle_and_direct_kernel(gpu_ctx, case, prec_name, tol_ref, tol_direct):
    import torch
    import paper_2110_10749_gb300 as ssd
    p, d, g, v, ref = case
    n = p["w"].size
    prec = getattr(ssd, prec_name)
    tg, tv = torch.as_tensor(g, device="cuda"), torch.as_tensor(v, device="cuda")
    P = ssd.Points.from_numpy(p).prepare(gpu_ctx)
    out = {k: t.cpu().numpy() for k, t in _apply(ssd, gpu_ctx, P, d, tg, tv, prec).items()}
    for k, b in ref.items():
        a = out[k]
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < tol_ref, k
        assert np.abs(a - b).max() < tol_ref * np.abs(b).max(), k
    # the direct kernel (plan off) on the same points agrees to the rounding
    # of the precision
    old = os.environ.get("SSD_PAIR_SYM")
    os.environ["SSD_PAIR_SYM"] = "0"
    try:
        ctx2 = ssd.Context(0)
    finally:
        if old is None:
            del os.environ["SSD_PAIR_SYM"]
        else:
            os.environ["SSD_PAIR_SYM"] = old
    P2 = ssd.Points.from_numpy(p).prepare(ctx2)
    direct = {k: t.cpu().numpy() for k, t in _apply(ssd, ctx2, P2, d, tg, tv, prec).items()}
    for k, b in ref.items():
        assert np.linalg.norm(direct[k] - out[k]) / np.linalg.norm(b) < tol_direct, k
    # launches per application (plans and item orders are cached by now), and
    # the plan's two pair launches timed as one application of its class
    for c, (k, P_, n_launch) in enumerate(((gpu_ctx, P, 4), (ctx2, P2, 3))):
        l0 = k.launch_count()
        ssd.stokes_DL(k, P_, d, tv, prec)
        torch.cuda.synchronize()
        assert k.launch_count() - l0 == n_launch, (prec_name, c)
    gpu_ctx.reset_stats()
    gpu_ctx.set_timing(True)
    ssd.stokes_DL(gpu_ctx, P, d, tv, prec)
    torch.cuda.synchronize()
    gpu_ctx.set_timing(False)
    st = gpu_ctx.kernel_stats(ssd.K_STOKES_DL, prec)
    assert st["launches"] == 1 and st["pairs"] == float(n) * n
    P2.release()
    ctx2.close()
    P.release()
