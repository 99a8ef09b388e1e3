"""Pins of the oracle's quadrature rule (Section 5.4, eq. Quadrature)."""
import math

import numpy as np
import pytest

from conftest import read_golden
from oracle import quadrature as Q


@pytest.mark.parametrize("row", read_golden("quadrature_counts.txt"), ids=lambda r: "%s-h1/%s" % (r[0], r[4]))
def test_counts_match_tables(row):
    surf, a, b, c, inv_h, N, _ = row
    pts = Q.ellipsoid_points((float(a), float(b), float(c)), 1.0 / int(inv_h))
    assert pts["w"].size == int(N)


def brute_force_count(abc, h, angle_deg=70.0):
    """Pure-Python count of grid-line intersections kept by the |n_i| test."""
    ct = math.cos(angle_deg * math.pi / 180.0)
    n = 0
    for i in range(3):
        a, b = [k for k in range(3) if k != i]
        J = int(math.ceil(max(abc) / h)) + 1
        for ja in range(-J, J + 1):
            for jb in range(-J, J + 1):
                s = 1.0 - (ja * h / abc[a]) ** 2 - (jb * h / abc[b]) ** 2
                if s <= 0:
                    continue
                for sg in (-1, 1):
                    x = [0.0, 0.0, 0.0]
                    x[a], x[b], x[i] = ja * h, jb * h, sg * abc[i] * math.sqrt(s)
                    g = [x[k] / abc[k] ** 2 for k in range(3)]
                    if abs(g[i]) / math.sqrt(sum(v * v for v in g)) >= ct:
                        n += 1
    return n


def test_brute_force_small_cases():
    for abc, h in [((1, 1, 1), 1 / 8), ((1, 0.6, 0.4), 1 / 8), ((1, 0.7, 0.5), 1 / 12)]:
        assert Q.ellipsoid_points(abc, h)["w"].size == brute_force_count(abc, h)


def test_sphere_area_superalgebraic():
    errs = []
    for h in (1 / 16, 1 / 32, 1 / 64):
        w = Q.sphere_points(1.0, h)["w"]
        errs.append(abs(w.sum() - 4 * math.pi) / (4 * math.pi))
    assert errs[0] < 5e-5 and errs[1] < 2e-6 and errs[2] < 1e-8
    assert errs[0] / errs[1] > 16 and errs[1] / errs[2] > 64


def test_ellipsoid_area_carlson():
    from scipy.special import elliprg
    a, b, c = 1.0, 0.6, 0.4
    exact = 4 * math.pi * a * b * c * elliprg(1 / a ** 2, 1 / b ** 2, 1 / c ** 2)
    errs = [abs(Q.ellipsoid_points((a, b, c), h)["w"].sum() - exact) / exact
            for h in (1 / 32, 1 / 64, 1 / 128)]
    # the thin ellipsoid converges more slowly than the sphere (cf. Table 3)
    assert errs[0] < 2e-4 and errs[1] < 2e-5 and errs[2] < 5e-7
    assert errs[0] / errs[1] > 8 and errs[1] / errs[2] > 16


def test_moments_on_sphere():
    p = Q.sphere_points(1.0, 1 / 32)
    x, y, z = p["xyz"]
    w = p["w"]
    assert (w * z * z).sum() == pytest.approx(4 * math.pi / 3, rel=1e-5)
    assert (w * x ** 4).sum() == pytest.approx(4 * math.pi / 5, rel=1e-5)
    assert abs((w * x * y * z).sum()) < 1e-12


def test_points_normals_meta_consistent():
    abc = (1.0, 0.7, 0.5)
    h = 1 / 24
    p = Q.ellipsoid_points(abc, h)
    x = p["xyz"]
    phi = (x[0] / abc[0]) ** 2 + (x[1] / abc[1]) ** 2 + (x[2] / abc[2]) ** 2 - 1
    assert np.abs(phi).max() < 1e-14
    assert np.abs((p["nrm"] ** 2).sum(0) - 1).max() < 1e-15
    g = x / np.array(abc)[:, None] ** 2
    assert np.abs(p["nrm"] - g / np.linalg.norm(g, axis=0)).max() < 1e-15
    ax, j1, j2, br = p["meta"]
    for i in range(3):
        a, b = Q.OTHER[i]
        m = ax == i
        assert np.array_equal(x[a][m], j1[m] * h) and np.array_equal(x[b][m], j2[m] * h)
        assert np.all(np.abs(p["nrm"][i][m]) >= Q.cos_threshold(70.0))
        # smaller root first on each line
        assert np.all((x[i][m] < 0) == (br[m] == 0))


def test_partition_of_unity():
    rng = np.random.default_rng(3)
    v = rng.normal(size=(3, 2000))
    v /= np.linalg.norm(v, axis=0)
    psi = Q.pou(v)
    assert np.abs(psi.sum(0) - 1).max() < 1e-15
    ct = Q.cos_threshold(70.0)
    assert np.all(psi[np.abs(v) <= ct] == 0.0)
    assert np.all(psi[np.abs(v) > ct + 1e-3] > 0.0)
