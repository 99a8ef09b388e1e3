"""The FP32C layer operators on the symmetric plan (far block pairs evaluated
once for both directions): on the h = 1/48 sphere (N = 38310, 64% of the
pairs in far block pairs) the whole application of each of the four
operators against the oracle element by element, and against the same
operator with the plan switched off (SSD_PAIR_SYM=0 when the context is
created)."""
import os

import numpy as np
import pytest

import oracle
from oracle import quadrature as Q

pytestmark = pytest.mark.gpu


def test_symmetric_plan_matches_oracle_and_direct_kernel(gpu_ctx):
    import torch
    import paper_2110_10749_gb300 as ssd
    h = 1 / 48
    p = Q.sphere_points(1.0, h)
    n = p["w"].size
    d = 3 * h
    rng = np.random.default_rng(21)
    x, y, z = p["xyz"]
    g = np.exp(x) * np.sin(y) + 0.1 * rng.normal(size=n)
    v = np.stack([y * z, np.cos(x), x + 0.3 * z * z]) + 0.1 * rng.normal(size=(3, n))
    tg, tv = torch.as_tensor(g, device="cuda"), torch.as_tensor(v, device="cuda")
    P = ssd.Points.from_numpy(p).prepare(gpu_ctx)
    outL = ssd.laplace_DL(gpu_ctx, P, d, tg, ssd.FP32C).cpu().numpy()
    outS = ssd.stokes_DL(gpu_ctx, P, d, tv, ssd.FP32C).cpu().numpy()
    outl = ssd.laplace_SL(gpu_ctx, P, d, tg, ssd.FP32C).cpu().numpy()
    outs = ssd.stokes_SL(gpu_ctx, P, d, 1.3, tv, ssd.FP32C).cpu().numpy()
    refL = oracle.laplace_dl(p, d, g)
    refS = oracle.stokes_dl(p, d, v)
    refl = oracle.laplace_sl(p, d, g)
    refs = oracle.stokes_sl(p, d, 1.3, v)
    for a, b in ((outL, refL), (outS, refS), (outl, refl), (outs, refs)):
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-5
        assert np.abs(a - b).max() < 1e-5 * np.abs(b).max()
    # the direct kernel (plan off) on the same points agrees to FP32C rounding
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
    dL = ssd.laplace_DL(ctx2, P2, d, tg, ssd.FP32C).cpu().numpy()
    dS = ssd.stokes_DL(ctx2, P2, d, tv, ssd.FP32C).cpu().numpy()
    dl = ssd.laplace_SL(ctx2, P2, d, tg, ssd.FP32C).cpu().numpy()
    ds = ssd.stokes_SL(ctx2, P2, d, 1.3, tv, ssd.FP32C).cpu().numpy()
    for a, b, ref in ((dL, outL, refL), (dS, outS, refS), (dl, outl, refl), (ds, outs, refs)):
        assert np.linalg.norm(a - b) / np.linalg.norm(ref) < 1e-6
    # the plan's two launches are counted under the double-layer classes
    gpu_ctx.reset_stats()
    gpu_ctx.set_timing(True)
    ssd.stokes_DL(gpu_ctx, P, d, tv, ssd.FP32C)
    torch.cuda.synchronize()
    gpu_ctx.set_timing(False)
    st = gpu_ctx.kernel_stats(ssd.K_STOKES_DL, ssd.FP32C)
    assert st["launches"] == 1 and st["pairs"] == float(n) * n
    P2.release()
    ctx2.close()
    P.release()
