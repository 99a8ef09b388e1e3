"""Quadrature points and weights on a closed surface (Section 5.4, eq. Quadrature).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

For each coordinate axis e_i, the lines of a grid of spacing h anchored at the
origin run along e_i through the points (j1 h, j2 h) of the other two
coordinates.  Every intersection x of such a line with the surface phi = 0 is
kept in the set R_i when |n(x) . e_i| >= cos(theta); it carries the weight
psi_i(n(x)) h^2 / |n(x) . e_i|.  The partition of unity is built from the bump
b(r) = exp(r^2 / (r^2 - 1)) (|r| < 1, else 0) as

    psi_i(n) = b(acos|n_i| / theta) / sum_j b(acos|n_j| / theta),

which vanishes when |n_i| <= cos(theta) as the paper requires.

Output order (shared by definition with the device generator): axis i = 0,1,2;
then the first remaining coordinate index j1 ascending; then j2 ascending; then
the root with the smaller coordinate first.  ``meta`` rows are
(axis, j1, j2, branch) with branch 0 for the smaller root and 1 for the larger.

The arithmetic of points and normals uses only +, -, *, / and sqrt, each
rounded once, in the order written here, so an implementation that follows
the same definition reproduces them bit for bit.
"""
from __future__ import annotations

import math

import numpy as np

OTHER = ((1, 2), (0, 2), (0, 1))


def cos_threshold(angle_deg: float) -> float:
    """cos(theta) for the partition angle, theta given in degrees."""
    return math.cos(angle_deg * (math.pi / 180.0))


def bump(r):
    """C-infinity bump b(r) = exp(r^2/(r^2-1)) for |r| < 1, else 0."""
    r = np.asarray(r, dtype=np.float64)
    out = np.zeros_like(r)
    m = np.abs(r) < 1.0
    r2 = r[m] * r[m]
    out[m] = np.exp(r2 / (r2 - 1.0))
    return out


def pou(nrm, angle_deg: float = 70.0):
    """psi_1, psi_2, psi_3 evaluated at unit normals nrm [3][N] -> [3][N]."""
    theta = angle_deg * (math.pi / 180.0)
    beta = np.stack([bump(np.arccos(np.abs(nrm[k])) / theta) for k in range(3)])
    return beta / ((beta[0] + beta[1]) + beta[2])


def ellipsoid_points(abc, h: float, angle_deg: float = 70.0, center=(0.0, 0.0, 0.0)):
    """Quadrature set of the ellipsoid sum_k ((x_k - c_k)/A_k)^2 = 1 (eq. Ellipsoid).

    The sphere of radius R (eq. Sphere) is the case abc = (R, R, R).
    Returns a dict with xyz [3][N], nrm [3][N], w [N], meta [4][N] (int32).
    """
    A = [float(a) for a in abc]
    c = [float(v) for v in center]
    h = float(h)
    ct = cos_threshold(angle_deg)
    xs, ns, ws, ms = [], [], [], []
    for i in range(3):
        a, b = OTHER[i]
        ja = np.arange(math.floor((c[a] - A[a]) / h) - 1, math.ceil((c[a] + A[a]) / h) + 2)
        jb = np.arange(math.floor((c[b] - A[b]) / h) - 1, math.ceil((c[b] + A[b]) / h) + 2)
        JA, JB = np.meshgrid(ja, jb, indexing="ij")
        JA, JB = JA.ravel(), JB.ravel()
        xa = JA.astype(np.float64) * h
        xb = JB.astype(np.float64) * h
        u = (xa - c[a]) / A[a]
        v = (xb - c[b]) / A[b]
        s = (1.0 - u * u) - v * v
        has = s > 0.0
        JA, JB, xa, xb, s = JA[has], JB[has], xa[has], xb[has], s[has]
        rt = np.sqrt(s)
        # two roots per line, smaller first
        ti = np.stack([c[i] - A[i] * rt, c[i] + A[i] * rt], axis=1).ravel()
        xa2 = np.repeat(xa, 2)
        xb2 = np.repeat(xb, 2)
        JA2 = np.repeat(JA, 2)
        JB2 = np.repeat(JB, 2)
        br = np.tile(np.array([0, 1]), JA.size)
        P = np.empty((3, ti.size))
        P[i], P[a], P[b] = ti, xa2, xb2
        # normal = grad(phi)/|grad(phi)|, grad(phi) proportional to (x_k - c_k)/A_k^2
        g = np.stack([(P[k] - c[k]) / (A[k] * A[k]) for k in range(3)])
        gn = np.sqrt((g[0] * g[0] + g[1] * g[1]) + g[2] * g[2])
        nrm = g / gn
        keep = np.abs(nrm[i]) >= ct
        P, nrm = P[:, keep], nrm[:, keep]
        psi = pou(nrm, angle_deg)[i]
        w = psi * (h * h) / np.abs(nrm[i])
        meta = np.stack([np.full(P.shape[1], i), JA2[keep], JB2[keep], br[keep]]).astype(np.int32)
        xs.append(P)
        ns.append(nrm)
        ws.append(w)
        ms.append(meta)
    return {
        "xyz": np.ascontiguousarray(np.concatenate(xs, axis=1)),
        "nrm": np.ascontiguousarray(np.concatenate(ns, axis=1)),
        "w": np.ascontiguousarray(np.concatenate(ws)),
        "meta": np.ascontiguousarray(np.concatenate(ms, axis=1)),
        "h": h,
    }


def sphere_points(R: float, h: float, angle_deg: float = 70.0, center=(0.0, 0.0, 0.0)):
    """Quadrature set of the sphere |x - c| = R (eq. Sphere)."""
    return ellipsoid_points((R, R, R), h, angle_deg, center)
