"""Pins of the oracle's smoothing factors s_1..s_4 (Section 5.3).

The closed forms are evaluated independently in 50-digit mpmath; the small-rho
limits come from sympy's series expansion of those closed forms.  A dropped
term, a wrong sign or a wrong power in either branch of the oracle (closed
form for rho >= 0.5, Taylor series below) fails one of these.
"""
import math

import numpy as np
import pytest

import oracle

mp = pytest.importorskip("mpmath")
sympy = pytest.importorskip("sympy")

# coefficient of rho^(2k+1) in the Gaussian part, written from Section 5.3
POLY = {
    1: (-1, 3, lambda r: r * (2 * r ** 2 - 5)),
    2: (+1, 3, lambda r: r * (2 * r ** 2 - 3)),
    3: (-1, 3, lambda r: r * (4 * r ** 4 - 14 * r ** 2 + 3)),
    4: (-1, 9, lambda r: r * (8 * r ** 6 - 36 * r ** 4 + 6 * r ** 2 + 9)),
}


def s_mp(i, r):
    mp.mp.dps = 50
    r = mp.mpf(r)
    sgn, den, P = POLY[i]
    return mp.erf(r) + sgn * 2 / (den * mp.sqrt(mp.pi)) * P(r) * mp.exp(-r * r)


RHOS = list(np.linspace(1e-3, 0.7, 200)) + list(np.linspace(0.7, 9.0, 200)) + [1e-6, 0.4999999, 0.5, 0.5000001]


@pytest.mark.parametrize("i", [1, 2, 3, 4])
def test_s_matches_mpmath(i):
    worst = 0.0
    for r in RHOS:
        ex = float(s_mp(i, r))
        worst = max(worst, abs(oracle.s(i, r) - ex) / abs(ex))
    assert worst < 3e-15


@pytest.mark.parametrize("i,p", [(1, 1), (2, 3), (3, 3), (4, 5)])
def test_small_rho_limit_from_sympy(i, p):
    r = sympy.symbols("r", positive=True)
    sgn, den, P = POLY[i]
    expr = sympy.erf(r) + sgn * 2 / (den * sympy.sqrt(sympy.pi)) * P(r) * sympy.exp(-r ** 2)
    ser = sympy.series(expr, r, 0, p + 3).removeO()
    lead = float(ser.coeff(r, p))
    nxt = float(ser.coeff(r, p + 2))
    # no lower power survives
    for k in range(p):
        assert abs(float(ser.coeff(r, k))) < 1e-30
    assert oracle.sigma(i, 0.0) == pytest.approx(lead, rel=1e-15)
    # second coefficient: finite difference of sigma in rho^2
    t = 1e-4
    assert (oracle.sigma(i, math.sqrt(t)) - oracle.sigma(i, 0.0)) / t == pytest.approx(nxt, rel=1e-3)


def test_printed_limits():
    # values quoted for the self terms: s_1/rho -> 16/(3 sqrt(pi)) etc.
    sp = math.sqrt(math.pi)
    assert oracle.sigma(1, 0.0) == pytest.approx(16 / (3 * sp), rel=1e-15)
    assert oracle.sigma(2, 0.0) == pytest.approx(8 / (3 * sp), rel=1e-15)
    assert oracle.sigma(3, 0.0) == pytest.approx(32 / (3 * sp), rel=1e-15)
    assert oracle.sigma(4, 0.0) == pytest.approx(128 / (15 * sp), rel=1e-15)


@pytest.mark.parametrize("i", [1, 2, 3, 4])
def test_branch_continuity_and_far_limit(i):
    below, above = oracle.sigma(i, 0.5 - 1e-15), oracle.sigma(i, 0.5)
    assert abs(below - above) / abs(above) < 2e-14
    assert oracle.s(i, 12.0) == 1.0
