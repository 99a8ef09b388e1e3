"""Pins of the oracle's molecule surface (eq. Molecule, Section 5.4):
the one-atom case is a sphere, points lie on the level set with normals
along grad(phi), and the divergence-theorem volume of the quadrature set
matches a cell count of the level set's interior."""
import math

import numpy as np

from oracle import quadrature as Q


def test_one_atom_is_a_sphere():
    r, c = 0.5, 0.6
    R = r * math.sqrt(math.log(1.0 / c))
    s = Q.molecule_points(1 / 16, centers=[(0.0, 0.0, 0.0)], r=r, c=c)
    o = Q.sphere_points(R, 1 / 16)
    assert np.array_equal(s["meta"], o["meta"])
    assert np.abs(s["xyz"] - o["xyz"]).max() <= 1e-15
    assert np.abs(s["nrm"] - o["nrm"]).max() <= 1e-14
    assert np.abs(s["w"] - o["w"]).max() <= 1e-14 * o["w"].max()


def test_points_on_level_set_and_normals():
    m = Q.molecule_points(1 / 16)
    X = m["xyz"]
    cen, r, c = Q.MOLECULE_CENTERS, 0.5, 0.6
    assert np.abs(Q.molecule_phi(cen, r, c, X)).max() < 1e-14
    e = 1e-6
    G = np.zeros_like(X)
    for k in range(3):
        Xp, Xm = X.copy(), X.copy()
        Xp[k] += e
        Xm[k] -= e
        G[k] = (Q.molecule_phi(cen, r, c, Xp) - Q.molecule_phi(cen, r, c, Xm)) / (2 * e)
    G /= np.linalg.norm(G, axis=0)
    assert np.abs(G - m["nrm"]).max() < 1e-8
    ax = m["meta"][0]
    assert np.all(np.abs(m["nrm"][ax, np.arange(X.shape[1])]) >= Q.cos_threshold(70.0))


def test_volume_and_area_convergence():
    vol = {}
    area = {}
    for hinv in (16, 32, 48):
        m = Q.molecule_points(1 / hinv)
        vol[hinv] = (m["w"] * (m["xyz"] * m["nrm"]).sum(0)).sum() / 3.0
        area[hinv] = m["w"].sum()
    # interior cell count on a 1/128 grid (cell centres), slab by slab
    s = 1.0 / 128
    g = np.arange(-1.4, 1.4, s) + s / 2
    Y, Z = np.meshgrid(g, g, indexing="ij")
    inside = 0
    for x in g:
        inside += int((Q.molecule_phi(Q.MOLECULE_CENTERS, 0.5, 0.6, [np.full_like(Y, x), Y, Z]) < 0).sum())
    vcount = inside * s ** 3
    assert abs(vol[48] / vcount - 1) < 2e-4, (vol, vcount)
    assert abs(vol[32] - vol[48]) < abs(vol[16] - vol[32]) / 5
    assert abs(area[32] - area[48]) < abs(area[16] - area[32]) / 5


def test_gauss_exp_is_exp_to_two_ulps():
    """The molecule's stated exponential (Cody-Waite reduction, degree-13
    Taylor polynomial) against 40-digit exp, and its exact points."""
    mpmath = __import__("pytest").importorskip("mpmath")
    mpmath.mp.dps = 40
    rng = np.random.default_rng(3)
    xs = np.concatenate([-np.linspace(0.0, 60.0, 3001), -rng.uniform(0.0, 700.0, 2000), [-1e-300, -5e-17]])
    g = Q.gauss_exp(xs)
    worst = max(abs(float((mpmath.mpf(v) - mpmath.exp(x)) / mpmath.exp(x))) for x, v in zip(xs, g))
    assert worst < 2.0 * 2.0 ** -53
    assert Q.gauss_exp(np.array([0.0]))[0] == 1.0
    assert Q.gauss_exp(np.array([-800.0]))[0] == 0.0
