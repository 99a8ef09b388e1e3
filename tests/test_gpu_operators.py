"""The six pair-sum operators through the C ABI against the FP64 oracle.

Tolerances (relative 2-norm error against the oracle on the same inputs):
FP64 path 1e-12, FP32C path 1e-5; the element-wise error is also bounded
relative to the largest output entry.  Cases span several CTA target spans
and a ragged tail (N not a multiple of 256), the unsorted per-call layout
and the prepared (spatially sorted) one, a tiny point set, and the full
h = 1/32 sphere (N = 17070) in the launch configuration the benchmark uses;
the h = 1/128 ellipsoid (N = 138830) is compared on sampled targets.
"""
import numpy as np
import pytest

import oracle
from oracle import quadrature as Q

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}
OPS = ["LSL", "LDL", "SSL", "SDL", "SSLDL", "LSLDL"]
ALPHA, BETA, MU = 0.7, -1.1, 1.3


def oracle_ops(p, d, g, v, g2, v2):
    L = oracle.laplace_sl(p, d, g)
    M = oracle.stokes_sl(p, d, MU, v)
    return {"LSL": L, "LDL": oracle.laplace_dl(p, d, g), "SSL": M, "SDL": oracle.stokes_dl(p, d, v),
            "SSLDL": ALPHA * oracle.stokes_sl(p, d, MU, v2) + BETA * oracle.stokes_dl(p, d, v),
            "LSLDL": ALPHA * oracle.laplace_sl(p, d, g2) + BETA * oracle.laplace_dl(p, d, g)}


def device_ops(ctx, P, d, g, v, g2, v2, prec, which=OPS):
    import paper_2110_10749_gb300 as ssd
    fn = {"LSL": lambda: ssd.laplace_SL(ctx, P, d, g, prec), "LDL": lambda: ssd.laplace_DL(ctx, P, d, g, prec),
          "SSL": lambda: ssd.stokes_SL(ctx, P, d, MU, v, prec), "SDL": lambda: ssd.stokes_DL(ctx, P, d, v, prec),
          "SSLDL": lambda: ssd.stokes_SLDL(ctx, P, d, MU, v2, v, ALPHA, BETA, prec),
          "LSLDL": lambda: ssd.laplace_SLDL(ctx, P, d, g2, g, ALPHA, BETA, prec)}
    return {k: fn[k]().cpu().numpy() for k in which}


def densities(p, seed, smooth):
    n = p["w"].size
    rng = np.random.default_rng(seed)
    if smooth:
        x, y, z = p["xyz"]
        g = np.exp(x) * np.sin(y)
        v = np.stack([y * z, np.cos(x), x + 0.3 * z * z])
    else:
        g = rng.normal(size=n)
        v = rng.normal(size=(3, n))
    return g, v, rng.normal(size=n), rng.normal(size=(3, n))


def check(out, ref, prec):
    for k in ref:
        a, b = out[k], ref[k]
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        mx = np.abs(a - b).max() / np.abs(b).max()
        assert rel <= TOL[prec] and mx <= 10 * TOL[prec], (k, rel, mx)


SURFACES = [((1.0, 1.0, 1.0), 1 / 8), ((1.0, 0.6, 0.4), 1 / 16), ((1.0, 0.7, 0.5), 1 / 12)]


@pytest.mark.parametrize("abc,h", SURFACES)
@pytest.mark.parametrize("smooth", [False, True])
def test_operators_match_oracle(gpu_ctx, abc, h, smooth):
    import torch
    import paper_2110_10749_gb300 as ssd
    p = Q.ellipsoid_points(abc, h)
    d = 3 * h
    g, v, g2, v2 = densities(p, 11, smooth)
    ref = oracle_ops(p, d, g, v, g2, v2)
    P = ssd.Points.from_numpy(p)
    T = [torch.as_tensor(a, device="cuda") for a in (g, v, g2, v2)]
    for prepared in (False, True):
        if prepared:
            P.prepare(gpu_ctx)
        for prec in (ssd.FP64, ssd.FP32C):
            check(device_ops(gpu_ctx, P, d, *T, prec), ref, prec)
    P.release()


def test_tiny_point_set(gpu_ctx):
    # 7 points: one partial tile, most of the CTA span padding
    import torch
    import paper_2110_10749_gb300 as ssd
    full = Q.sphere_points(1.0, 1 / 4)
    idx = np.arange(0, full["w"].size, full["w"].size // 7)[:7]
    p = {k: np.ascontiguousarray(full[k][..., idx]) for k in ("xyz", "nrm", "w")}
    g, v, g2, v2 = densities(p, 3, False)
    ref = oracle_ops(p, 0.75, g, v, g2, v2)
    P = ssd.Points.from_numpy(p)
    T = [torch.as_tensor(a, device="cuda") for a in (g, v, g2, v2)]
    for prec in (ssd.FP64, ssd.FP32C):
        check(device_ops(gpu_ctx, P, 0.75, *T, prec), ref, prec)


def test_duplicate_points_take_the_limit(gpu_ctx):
    # two coincident points (r = 0 between different indices) use the
    # smoothed kernels' limits, as the oracle's series branch does
    import torch
    import paper_2110_10749_gb300 as ssd
    full = Q.sphere_points(1.0, 1 / 8)
    p = {k: np.ascontiguousarray(np.concatenate([full[k], full[k][..., :3]], axis=-1)) for k in ("xyz", "nrm", "w")}
    g, v, g2, v2 = densities(p, 4, False)
    ref = oracle_ops(p, 3 / 8, g, v, g2, v2)
    P = ssd.Points.from_numpy(p).prepare(gpu_ctx)
    T = [torch.as_tensor(a, device="cuda") for a in (g, v, g2, v2)]
    for prec in (ssd.FP64, ssd.FP32C):
        check(device_ops(gpu_ctx, P, 3 / 8, *T, prec), ref, prec)
    P.release()


def test_full_sphere_h32_bench_configuration(gpu_ctx):
    # the benchmark's workload size and launch configuration: prepared
    # (sorted) layout, FP32C, N = 17070; FP64 checked as well
    import torch
    import paper_2110_10749_gb300 as ssd
    p = Q.sphere_points(1.0, 1 / 32)
    d = 3 / 32
    g, v, g2, v2 = densities(p, 12345, False)
    ref = oracle_ops(p, d, g, v, g2, v2)
    P = ssd.Points.from_numpy(p).prepare(gpu_ctx)
    T = [torch.as_tensor(a, device="cuda") for a in (g, v, g2, v2)]
    check(device_ops(gpu_ctx, P, d, *T, ssd.FP32C), ref, 1)
    check(device_ops(gpu_ctx, P, d, *T, ssd.FP64, ["LDL", "SDL"]), {k: ref[k] for k in ("LDL", "SDL")}, 0)
    P.release()


def test_large_ellipsoid_sampled_rows(gpu_ctx):
    # h = 1/128 ellipsoid (1, 0.7, 0.5): N = 138830, 1.9e10 pairs per apply,
    # the launch configuration of the large workload (both precisions run
    # their symmetric plans there); the oracle evaluates 64 sampled targets of
    # each operator
    import torch
    import paper_2110_10749_gb300 as ssd
    p = Q.ellipsoid_points((1.0, 0.7, 0.5), 1 / 128)
    n = p["w"].size
    assert n == 138830
    d = 3 / 128
    g, v, _, _ = densities(p, 12345, True)
    rows = np.random.default_rng(9).choice(n, 64, replace=False)
    P = ssd.Points.from_numpy(p).prepare(gpu_ctx)
    tg, tv = torch.as_tensor(g, device="cuda"), torch.as_tensor(v, device="cuda")
    ref = {"LDL": oracle.laplace_dl(p, d, g, rows=rows), "SDL": oracle.stokes_dl(p, d, v, rows=rows),
           "LSL": oracle.laplace_sl(p, d, g, targets=p["xyz"][:, rows]),
           "SSL": oracle.stokes_sl(p, d, MU, v, targets=p["xyz"][:, rows])}
    for prec, tol in ((ssd.FP32C, 1e-5), (ssd.FP64, 1e-12)):
        out = {"LDL": ssd.laplace_DL(gpu_ctx, P, d, tg, prec), "SDL": ssd.stokes_DL(gpu_ctx, P, d, tv, prec),
               "LSL": ssd.laplace_SL(gpu_ctx, P, d, tg, prec), "SSL": ssd.stokes_SL(gpu_ctx, P, d, MU, tv, prec)}
        for k, b in ref.items():
            a = out[k].cpu().numpy()[..., rows]
            assert np.linalg.norm(a - b) / np.linalg.norm(b) < tol, (prec, k)
    P.release()


def test_invalid_arguments(gpu_ctx):
    import torch
    import paper_2110_10749_gb300 as ssd
    p = Q.sphere_points(1.0, 1 / 4)
    P = ssd.Points.from_numpy(p)
    g = torch.zeros(p["w"].size, dtype=torch.float64, device="cuda")
    for bad in (0.0, -1.0, float("nan"), float("inf")):
        with pytest.raises(ssd.SsdError) as e:
            ssd.laplace_SL(gpu_ctx, P, bad, g)
        assert e.value.status == ssd.SSD_EINVAL
    with pytest.raises(ssd.SsdError):
        ssd.stokes_SL(gpu_ctx, P, 0.5, -1.0, torch.zeros((3, p["w"].size), dtype=torch.float64, device="cuda"))
    with pytest.raises(ssd.SsdError):
        ssd.laplace_DL(gpu_ctx, P, 0.5, g, prec=7)


def test_sync_after_asynchronous_calls(gpu_ctx):
    # operator calls return once queued; ssd_sync waits for them on the
    # stream (or the device) and reports success when the kernels ran
    import torch
    import paper_2110_10749_gb300 as ssd
    p = Q.sphere_points(1.0, 1 / 8)
    P = ssd.Points.from_numpy(p)
    g = torch.ones(p["w"].size, dtype=torch.float64, device="cuda")
    out = ssd.laplace_DL(gpu_ctx, P, 3 / 8, g, ssd.FP32C)
    gpu_ctx.sync()
    gpu_ctx.sync(device_wide=True)
    # the double layer of a constant vanishes (subtracted form, eq. H_subtr)
    assert float(out.abs().max()) < 1e-12
