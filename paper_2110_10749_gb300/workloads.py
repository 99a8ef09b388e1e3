"""Seeded synthetic workloads (inputs only; no arithmetic of the method).

Star-shaped surfaces r(xi) = 1 + sum_{l<=4} c_lm Y_lm(xi) with coefficients
c_lm ~ N(0, sigma^2) drawn from numpy's default_rng(seed), 25 coefficients in
the order k = l^2 + l + m.  The batched workload mixes such stars with
ellipsoids of axes (1, 0.8, 0.6), each with a grid spacing h drawn from
{1/16, 1/24, 1/32, 1/48} by the same generator, and four far-field flows per
surface.  Tests, the benchmark and the oracle's own checks all read their
inputs from here.
"""
from __future__ import annotations

import math

import numpy as np

STAR_NCOEF = 25
H_CHOICES = (1 / 16, 1 / 24, 1 / 32, 1 / 48)
FAR_FIELDS = ((1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0),
              (1.0 / math.sqrt(3.0),) * 3)


def star_coefficients(seed: int, sigma: float = 0.05) -> np.ndarray:
    """25 coefficients c_lm ~ N(0, sigma^2) from default_rng(seed)."""
    return np.random.default_rng(seed).normal(0.0, sigma, STAR_NCOEF)


def batch_recipe(n_star: int = 64, n_ellipsoid: int = 8, seed: int = 2024, h_choices=H_CHOICES):
    """Surfaces of the batched workload: list of dicts with kind ('star' or
    'ellipsoid'), clm or abc, and h.  Stars use seeds 0..n_star-1."""
    rng = np.random.default_rng(seed)
    out = []
    for s in range(n_star):
        out.append({"kind": "star", "clm": star_coefficients(s), "h": float(rng.choice(h_choices))})
    for _ in range(n_ellipsoid):
        out.append({"kind": "ellipsoid", "abc": (1.0, 0.8, 0.6), "h": float(rng.choice(h_choices))})
    return out
