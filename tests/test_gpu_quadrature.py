"""Device quadrature points (Section 5.4) against the oracle: point set,
order, coordinates, normals and (axis, j1, j2, branch) bit for bit; weights
within 1e-14 of the largest weight (they pass through acos and exp, whose
library implementations differ in the last bits)."""
import numpy as np
import pytest

from conftest import read_golden
from oracle import quadrature as Q

pytestmark = pytest.mark.gpu

CASES = [
    ("sphere", (1.0, 1.0, 1.0), 1 / 8, (0.0, 0.0, 0.0)),
    ("sphere", (1.0, 1.0, 1.0), 1 / 32, (0.0, 0.0, 0.0)),
    ("sphere", (0.8, 0.8, 0.8), 1 / 24, (0.0, 0.0, 0.0)),
    ("sphere", (1.0, 1.0, 1.0), 1 / 20, (0.013, -0.2, 0.31)),
    ("ellipsoid", (1.0, 0.6, 0.4), 1 / 16, (0.0, 0.0, 0.0)),
    ("ellipsoid", (1.0, 0.7, 0.5), 1 / 96, (0.0, 0.0, 0.0)),
    ("ellipsoid", (1.0, 0.8, 0.6), 1 / 48, (0.1, 0.0, -0.05)),
]


def device_points(ctx, kind, abc, h, center):
    import paper_2110_10749_gb300 as ssd
    k = ssd.SPHERE if kind == "sphere" else ssd.ELLIPSOID
    g = ssd.quadrature_points(ctx, k, abc if kind == "ellipsoid" else abc[:1], h, 70.0, center)
    return {k2: v.cpu().numpy() for k2, v in g.items()}


@pytest.mark.parametrize("kind,abc,h,center", CASES)
def test_points_bit_identical(gpu_ctx, kind, abc, h, center):
    g = device_points(gpu_ctx, kind, abc, h, center)
    o = Q.ellipsoid_points(abc, h, 70.0, center)
    assert g["w"].size == o["w"].size
    assert np.array_equal(g["meta"], o["meta"])
    assert np.array_equal(g["xyz"], o["xyz"])
    assert np.array_equal(g["nrm"], o["nrm"])
    assert np.abs(g["w"] - o["w"]).max() <= 1e-14 * o["w"].max()


@pytest.mark.parametrize("row", read_golden("quadrature_counts.txt"), ids=lambda r: "%s-h1/%s" % (r[0], r[4]))
def test_counts_match_tables(gpu_ctx, row):
    import paper_2110_10749_gb300 as ssd
    surf, a, b, c, inv_h, N, _ = row
    g = ssd.quadrature_points(gpu_ctx, ssd.ELLIPSOID, (float(a), float(b), float(c)), 1.0 / int(inv_h))
    assert g["w"].numel() == int(N)


def test_size_query_and_capacity_error(gpu_ctx):
    import ctypes as C
    import torch
    import paper_2110_10749_gb300 as ssd
    surf = ssd.CSurface(ssd.SPHERE, (C.c_double * 3)(0, 0, 0), (C.c_double * 3)(1, 0, 0))
    n = C.c_int64()
    L = ssd.lib()
    assert L.ssd_quadrature_points(gpu_ctx.h, C.byref(surf), 1 / 8, 70.0, 0, C.byref(n), None, None, None,
                                   None, None) == ssd.SSD_OK
    assert n.value == 1062
    buf = torch.empty((3, 10), dtype=torch.float64, device="cuda")
    w = torch.empty(10, dtype=torch.float64, device="cuda")
    st = L.ssd_quadrature_points(gpu_ctx.h, C.byref(surf), 1 / 8, 70.0, 10, C.byref(n), buf.data_ptr(),
                                 buf.data_ptr(), w.data_ptr(), None, None)
    assert st == ssd.SSD_EINVAL and n.value == 1062
    assert L.ssd_quadrature_points(gpu_ctx.h, C.byref(surf), -1.0, 70.0, 0, C.byref(n), None, None, None,
                                   None, None) == ssd.SSD_EINVAL


STAR_CASES = [
    (0, 1 / 16, (0.0, 0.0, 0.0)),
    (3, 1 / 24, (0.02, -0.03, 0.01)),
    (11, 1 / 32, (0.0, 0.0, 0.0)),
    (-1, 1 / 20, (0.0, 0.1, 0.0)),      # -1: the unit sphere written as a star (all c = 0)
    (40, 1 / 48, (0.0, 0.0, 0.0)),
]


def _clm(seed):
    from paper_2110_10749_gb300.workloads import star_coefficients
    return np.zeros(25) if seed < 0 else star_coefficients(seed)


@pytest.mark.parametrize("seed,h,center", STAR_CASES)
def test_star_points_bit_identical(gpu_ctx, seed, h, center):
    import paper_2110_10749_gb300 as ssd
    clm = _clm(seed)
    g = ssd.quadrature_points(gpu_ctx, ssd.STAR, h=h, center=center, clm=clm)
    g = {k: v.cpu().numpy() for k, v in g.items()}
    o = Q.star_points(clm, h, 70.0, center)
    assert g["w"].size == o["w"].size
    assert np.array_equal(g["meta"], o["meta"])
    assert np.array_equal(g["xyz"], o["xyz"])
    assert np.array_equal(g["nrm"], o["nrm"])
    assert np.abs(g["w"] - o["w"]).max() <= 1e-14 * o["w"].max()


def test_star_rejects_large_coefficients(gpu_ctx):
    import paper_2110_10749_gb300 as ssd
    clm = np.zeros(25)
    clm[0] = 3.6      # |c_00| B_0 > 1
    with pytest.raises(ssd.SsdError) as ei:
        ssd.quadrature_points(gpu_ctx, ssd.STAR, h=1 / 8, clm=clm)
    assert ei.value.status == ssd.SSD_EINVAL


@pytest.mark.parametrize("seed", [5, -1])
def test_star_jacobian_against_oracle_differences(gpu_ctx, seed):
    """d(x, n, w)/dc_k against central differences of the oracle's point sets."""
    import paper_2110_10749_gb300 as ssd
    clm = _clm(seed)
    h = 1 / 16
    g = ssd.quadrature_points(gpu_ctx, ssd.STAR, h=h, clm=clm)
    n = g["w"].numel()
    J = {k: v.cpu().numpy() for k, v in ssd.quadrature_jacobian(gpu_ctx, clm, h, n).items()}
    eps = 1e-6
    for k in (0, 1, 5, 8, 12, 17, 20, 24):
        cp, cm = clm.copy(), clm.copy()
        cp[k] += eps
        cm[k] -= eps
        op, om = Q.star_points(cp, h), Q.star_points(cm, h)
        assert np.array_equal(op["meta"], om["meta"]) and op["w"].size == n
        for key, fk in (("xyz", "dxyz"), ("nrm", "dnrm"), ("w", "dw")):
            fd = (op[key] - om[key]) / (2 * eps)
            err = np.abs(J[fk][k] - fd).max()
            assert err <= 1e-6 * np.abs(fd).max() + 1e-9, (k, key, err, np.abs(fd).max())
