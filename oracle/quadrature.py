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


# ---------------------------------------------------------------- star surfaces
#
# Star-shaped surfaces |x - c| = r(xi), xi = (x - c)/|x - c|, with
#     r(xi) = 1 + sum_{l <= 4} sum_{m=-l..l} c_lm Y_lm(xi),
# real orthonormal spherical harmonics Y_lm written as Cartesian polynomials in
# the unit vector xi (no trigonometry).  Coefficient k = l^2 + l + m.  The
# level set is phi(x) = (|x - c| - 1) - P(xi), P = sum_k c_k Y_k, phi > 0
# outside; its gradient is grad phi = xi - (g - (xi . g) xi)/|x - c| with g the
# gradient of the polynomial P in R^3 (only its tangential part enters).
#
# Roots along a grid line are located by a fixed procedure, so that any
# implementation that follows it reproduces the points bit for bit: phi is
# sampled at t_k = t_lo + k dt (k = 0..K) on [c_i - 1.0625 Rb, c_i + 1.0625 Rb]
# with Rb = 1 + sum_k |c_k| B_l (B_l = sqrt((2l+1)/(4 pi)) bounds |Y_lm|),
# K = ceil(2.125 Rb / ds), ds = 1/64, dt = (t_hi - t_lo)/K; every k with
# (phi(t_k) > 0) != (phi(t_{k+1}) > 0) brackets one root, which bisection
# (mid = 0.5 (lo + hi), until mid equals an end point, at most 200 steps)
# narrows to two neighbouring doubles; the end point with the smaller |phi|
# is the root.  Two roots closer than one sample step are not resolved; for a
# kept root the next crossing of the line is farther than that on the
# surfaces used here (lines meet kept points at least 20 degrees from tangent).

STAR_NCOEF = 25


def star_constants():
    """Normalisation constants K_k of the 25 real orthonormal Y_lm (l <= 4)."""
    pi = math.pi
    s = math.sqrt
    return np.array([
        0.5 * s(1.0 / pi),
        s(3.0 / (4.0 * pi)), s(3.0 / (4.0 * pi)), s(3.0 / (4.0 * pi)),
        0.5 * s(15.0 / pi), 0.5 * s(15.0 / pi), 0.25 * s(5.0 / pi), 0.5 * s(15.0 / pi), 0.25 * s(15.0 / pi),
        0.25 * s(35.0 / (2.0 * pi)), 0.5 * s(105.0 / pi), 0.25 * s(21.0 / (2.0 * pi)), 0.25 * s(7.0 / pi),
        0.25 * s(21.0 / (2.0 * pi)), 0.25 * s(105.0 / pi), 0.25 * s(35.0 / (2.0 * pi)),
        0.75 * s(35.0 / pi), 0.75 * s(35.0 / (2.0 * pi)), 0.75 * s(5.0 / pi), 0.75 * s(5.0 / (2.0 * pi)),
        (3.0 / 16.0) * s(1.0 / pi), 0.75 * s(5.0 / (2.0 * pi)), 0.375 * s(5.0 / pi), 0.75 * s(35.0 / (2.0 * pi)),
        (3.0 / 16.0) * s(35.0 / pi),
    ])


def star_degree(k: int) -> int:
    return int(math.isqrt(k))


def star_polys(x, y, z):
    """The 25 polynomials p_k (Y_k = K_k p_k on the unit sphere) and their
    gradients in R^3: returns (p [25], gx [25], gy [25], gz [25]) lists of
    arrays (zeros as 0.0)."""
    x2, y2, z2 = x * x, y * y, z * z
    xy, yz, xz = x * y, y * z, x * z
    u = x2 - y2
    v3x = 3.0 * x2 - y2
    w3y = x2 - 3.0 * y2
    z5 = 5.0 * z2 - 1.0
    z53 = 5.0 * z2 - 3.0
    z7 = 7.0 * z2 - 1.0
    z73 = 7.0 * z2 - 3.0
    one = np.ones_like(x)
    zero = 0.0 * x
    p = [one, y, z, x,
         xy, yz, 3.0 * z2 - 1.0, xz, u,
         y * v3x, xy * z, y * z5, z * z53, x * z5, z * u, x * w3y,
         xy * u, yz * v3x, xy * z7, yz * z73, (35.0 * z2 - 30.0) * z2 + 3.0, xz * z73, u * z7, xz * w3y,
         x2 * w3y - y2 * v3x]
    gx = [zero, zero, zero, one,
          y, zero, zero, z, 2.0 * x,
          6.0 * xy, yz, zero, zero, z5, 2.0 * xz, 3.0 * u,
          y * v3x, 6.0 * xy * z, y * z7, zero, zero, z * z73, 2.0 * x * z7, 3.0 * z * u, 4.0 * x * w3y]
    gy = [zero, one, zero, zero,
          x, z, zero, zero, -2.0 * y,
          3.0 * u, xz, z5, zero, zero, -2.0 * yz, -6.0 * xy,
          x * w3y, 3.0 * z * u, x * z7, z * z73, zero, zero, -2.0 * y * z7, -6.0 * xy * z, -4.0 * y * v3x]
    gz = [zero, zero, one, zero,
          zero, y, 6.0 * z, x, zero,
          zero, xy, 10.0 * yz, 15.0 * z2 - 3.0, 10.0 * xz, u, zero,
          zero, y * v3x, 14.0 * xy * z, y * (21.0 * z2 - 3.0), z * (140.0 * z2 - 60.0), x * (21.0 * z2 - 3.0),
          14.0 * z * u, x * w3y, zero]
    return p, gx, gy, gz


# nonzero terms of each gradient component, in the order they are summed
_GX_TERMS = (3, 4, 7, 8, 9, 10, 13, 14, 15, 16, 17, 18, 21, 22, 23, 24)
_GY_TERMS = (1, 4, 5, 8, 9, 10, 11, 14, 15, 16, 17, 18, 19, 22, 23, 24)
_GZ_TERMS = (2, 5, 6, 7, 10, 11, 12, 13, 14, 17, 18, 19, 20, 21, 22, 23)


def star_eval(a, xi):
    """P(xi) = sum_k a_k p_k(xi) and its R^3 gradient, a_k = c_k K_k.

    Sums run over k ascending; the gradient sums skip the terms that vanish
    identically (their first term starts the sum)."""
    x, y, z = xi
    p, gx, gy, gz = star_polys(x, y, z)
    P = a[0] * p[0]
    for k in range(1, STAR_NCOEF):
        P = P + a[k] * p[k]

    def gsum(terms, comp):
        k0 = terms[0]
        s = a[k0] if k0 < 4 else a[k0] * comp[k0]
        for k in terms[1:]:
            s = s + a[k] * comp[k]
        return s
    return P, (gsum(_GX_TERMS, gx), gsum(_GY_TERMS, gy), gsum(_GZ_TERMS, gz))


def star_bound(clm) -> float:
    """Rb = 1 + sum_k |c_k| B_l, B_l = sqrt((2l+1)/(4 pi))."""
    rb = 1.0
    for k in range(STAR_NCOEF):
        rb = rb + abs(float(clm[k])) * math.sqrt((2.0 * star_degree(k) + 1.0) / (4.0 * math.pi))
    return rb


def star_phi(a, c, X):
    """phi(x) = (|x - c| - 1) - P(xi) at points X [3][...]."""
    d0, d1, d2 = X[0] - c[0], X[1] - c[1], X[2] - c[2]
    rho = np.sqrt((d0 * d0 + d1 * d1) + d2 * d2)
    with np.errstate(invalid="ignore", divide="ignore"):
        # at the centre itself phi is NaN, which counts as "not > 0" (inside)
        xi = (d0 / rho, d1 / rho, d2 / rho)
        P, _ = star_eval(a, xi)
        return (rho - 1.0) - P


def star_normal(a, c, X):
    """Unit normal grad(phi)/|grad(phi)| at points X [3][m]."""
    d = [X[k] - c[k] for k in range(3)]
    rho = np.sqrt((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2])
    xi = [d[k] / rho for k in range(3)]
    _, g = star_eval(a, xi)
    gxi = (g[0] * xi[0] + g[1] * xi[1]) + g[2] * xi[2]
    G = [xi[k] - (g[k] - gxi * xi[k]) / rho for k in range(3)]
    gn = np.sqrt((G[0] * G[0] + G[1] * G[1]) + G[2] * G[2])
    return np.stack([G[k] / gn for k in range(3)])


def star_points(clm, h: float, angle_deg: float = 70.0, center=(0.0, 0.0, 0.0)):
    """Quadrature set (eq. Quadrature) of the star surface r = 1 + sum c_lm Y_lm.

    Same output and order as ellipsoid_points; meta row 3 holds the root's
    ordinal along its line (0 for the smallest t)."""
    clm = np.asarray(clm, dtype=np.float64)
    assert clm.shape == (STAR_NCOEF,)
    K = star_constants()
    a = np.array([clm[k] * K[k] for k in range(STAR_NCOEF)])
    c = [float(v) for v in center]
    h = float(h)
    rb = star_bound(clm)
    assert rb < 2.0, "sum |c_k| B_l must stay below 1 (star-shaped, positive radius)"
    ct = cos_threshold(angle_deg)
    ds = 1.0 / 64.0
    nk = int(math.ceil(2.125 * rb / ds))
    xs, ns, ws, ms = [], [], [], []
    for i in range(3):
        a_, b_ = OTHER[i]
        ja = np.arange(math.floor((c[a_] - rb) / h) - 1, math.ceil((c[a_] + rb) / h) + 2)
        jb = np.arange(math.floor((c[b_] - rb) / h) - 1, math.ceil((c[b_] + rb) / h) + 2)
        JA, JB = np.meshgrid(ja, jb, indexing="ij")
        JA, JB = JA.ravel(), JB.ravel()
        xa = JA.astype(np.float64) * h
        xb = JB.astype(np.float64) * h
        da, db = xa - c[a_], xb - c[b_]
        near = da * da + db * db < rb * rb
        JA, JB, xa, xb = JA[near], JB[near], xa[near], xb[near]
        t_lo = c[i] - 1.0625 * rb
        t_hi = c[i] + 1.0625 * rb
        dt = (t_hi - t_lo) / nk
        T = t_lo + np.arange(nk + 1, dtype=np.float64) * dt          # [K+1]
        L = xa.size

        def phi_at(t, rows):
            X = [None, None, None]
            X[i] = t
            X[a_] = xa[rows]
            X[b_] = xb[rows]
            return star_phi(a, c, X)
        rows = np.repeat(np.arange(L), nk + 1)
        F = phi_at(np.tile(T, L), rows).reshape(L, nk + 1)
        pos = F > 0.0
        line, kk = np.nonzero(pos[:, :-1] != pos[:, 1:])             # row-major: line, then t
        lo, hi = T[kk].copy(), T[kk + 1].copy()
        flo, fhi = F[line, kk].copy(), F[line, kk + 1].copy()
        slo = flo > 0.0
        active = np.ones(lo.size, dtype=bool)
        for _ in range(200):
            if not active.any():
                break
            mid = 0.5 * (lo + hi)
            stop = (mid == lo) | (mid == hi)
            active &= ~stop
            idx = np.nonzero(active)[0]
            if idx.size == 0:
                break
            fm = phi_at(mid[idx], line[idx])
            same = (fm > 0.0) == slo[idx]
            lo[idx[same]] = mid[idx[same]]
            flo[idx[same]] = fm[same]
            hi[idx[~same]] = mid[idx[~same]]
            fhi[idx[~same]] = fm[~same]
        t = np.where(np.abs(flo) <= np.abs(fhi), lo, hi)
        # ordinal of each root along its line
        first = np.r_[True, line[1:] != line[:-1]]
        start = np.maximum.accumulate(np.where(first, np.arange(line.size), 0))
        ordinal = np.arange(line.size) - start
        P = np.empty((3, t.size))
        P[i], P[a_], P[b_] = t, xa[line], xb[line]
        nrm = star_normal(a, c, P) if t.size else np.zeros((3, 0))
        keep = np.abs(nrm[i]) >= ct
        P, nrm = P[:, keep], nrm[:, keep]
        psi = pou(nrm, angle_deg)[i]
        w = psi * (h * h) / np.abs(nrm[i])
        meta = np.stack([np.full(P.shape[1], i), JA[line][keep], JB[line][keep], ordinal[keep]]).astype(np.int32)
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


# ---------------------------------------------------------------- molecule
#
# The 'four-atom molecule' of Section 5.4 (eq. Molecule): sum_k exp(-|x - x_k|^2 / r^2) = c,
# written as phi(x) = c - sum_k exp(-|x - x_k|^2 / r^2) so that phi > 0 outside and the outward
# normal is grad(phi)/|grad(phi)|, grad(phi) = sum_k exp(-|x - x_k|^2/r^2) 2 (x - x_k) / r^2.
# Roots along the grid lines follow the same fixed sampling and bisection as the star surfaces,
# on [lo_i, hi_i] = [min_k x_k,i - D, max_k x_k,i + D] with D = 1.0625 r sqrt(log(n_atoms / c))
# (a point farther than r sqrt(log(n_atoms/c)) from every centre has phi > 0).

MOLECULE_CENTERS = (
    (math.sqrt(3.0) / 3.0, 0.0, -math.sqrt(6.0) / 12.0),
    (-math.sqrt(3.0) / 6.0, 0.5, -math.sqrt(6.0) / 12.0),
    (-math.sqrt(3.0) / 6.0, -0.5, -math.sqrt(6.0) / 12.0),
    (0.0, 0.0, math.sqrt(6.0) / 4.0),
)


# Taylor coefficients 1/j! of e^r, j = 0..13, each rounded to double
_EXP_TAYLOR = (1.0, 1.0, 0.5, 0.16666666666666666, 0.041666666666666664, 0.008333333333333333,
               0.001388888888888889, 0.0001984126984126984, 2.48015873015873e-05, 2.7557319223985893e-06,
               2.755731922398589e-07, 2.505210838544172e-08, 2.08767569878681e-09, 1.6059043836821613e-10)
_LN2_HEAD = 0.6931471803691238       # ln 2 to 32 significant bits: k * head is exact for |k| < 2^21
_LN2_TAIL = 1.9082149292705877e-10   # ln 2 - head, rounded
_INV_LN2 = 1.4426950408889634


def gauss_exp(x):
    """e^x (x <= 0) for the molecule's Gaussians by one stated method, so the
    point set does not depend on a math library's last bits: Cody and
    Waite's additive reduction x = k ln2 + r with k = floor(x/ln2 + 1/2) and
    ln2 split into a head and a tail, the degree-13 Taylor polynomial of e^r
    (|r| <= ln2/2, truncation below 5e-18) by Horner's rule, then 2^k.  Every
    operation is one rounded IEEE operation; zero below x = -700."""
    x = np.asarray(x, dtype=np.float64)
    k = np.floor(x * _INV_LN2 + 0.5)
    r = (x - k * _LN2_HEAD) - k * _LN2_TAIL
    p = np.full_like(x, _EXP_TAYLOR[13])
    for cj in _EXP_TAYLOR[12::-1]:
        p = p * r + cj
    out = np.ldexp(p, np.where(x < -700.0, 0, k).astype(np.int64))
    return np.where(x < -700.0, 0.0, out)


def molecule_phi(centers, r, c, X):
    s = 0.0 * X[0]
    for xk in centers:
        d2 = ((X[0] - xk[0]) ** 2 + (X[1] - xk[1]) ** 2) + (X[2] - xk[2]) ** 2
        s = s + gauss_exp(-d2 / (r * r))
    return c - s


def molecule_normal(centers, r, c, X):
    g = [0.0 * X[0], 0.0 * X[0], 0.0 * X[0]]
    for xk in centers:
        d = [X[k] - xk[k] for k in range(3)]
        e = gauss_exp(-((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]) / (r * r))
        for k in range(3):
            g[k] = g[k] + e * (2.0 * d[k] / (r * r))
    gn = np.sqrt((g[0] * g[0] + g[1] * g[1]) + g[2] * g[2])
    return np.stack([g[k] / gn for k in range(3)])


def molecule_points(h: float, angle_deg: float = 70.0, centers=MOLECULE_CENTERS, r: float = 0.5, c: float = 0.6):
    """Quadrature set (eq. Quadrature) of the molecule surface (eq. Molecule);
    same output and order as star_points."""
    centers = [tuple(float(v) for v in xk) for xk in centers]
    h = float(h)
    ct = cos_threshold(angle_deg)
    D = 1.0625 * r * math.sqrt(math.log(len(centers) / c))
    lo = [min(xk[k] for xk in centers) - D for k in range(3)]
    hi = [max(xk[k] for xk in centers) + D for k in range(3)]
    ds = 1.0 / 64.0
    xs, ns, ws, ms = [], [], [], []
    for i in range(3):
        a_, b_ = OTHER[i]
        nk = int(math.ceil((hi[i] - lo[i]) / ds))
        dt = (hi[i] - lo[i]) / nk
        ja = np.arange(math.floor(lo[a_] / h) - 1, math.ceil(hi[a_] / h) + 2)
        jb = np.arange(math.floor(lo[b_] / h) - 1, math.ceil(hi[b_] / h) + 2)
        JA, JB = np.meshgrid(ja, jb, indexing="ij")
        JA, JB = JA.ravel(), JB.ravel()
        xa = JA.astype(np.float64) * h
        xb = JB.astype(np.float64) * h
        near = np.zeros(xa.size, dtype=bool)
        for xk in centers:
            near |= (xa - xk[a_]) ** 2 + (xb - xk[b_]) ** 2 < D * D
        JA, JB, xa, xb = JA[near], JB[near], xa[near], xb[near]
        T = lo[i] + np.arange(nk + 1, dtype=np.float64) * dt
        L = xa.size

        def phi_at(t, rows):
            X = [None, None, None]
            X[i] = t
            X[a_] = xa[rows]
            X[b_] = xb[rows]
            return molecule_phi(centers, r, c, X)
        Fv = phi_at(np.tile(T, L), np.repeat(np.arange(L), nk + 1)).reshape(L, nk + 1)
        pos = Fv > 0.0
        line, kk = np.nonzero(pos[:, :-1] != pos[:, 1:])
        lo_t, hi_t = T[kk].copy(), T[kk + 1].copy()
        flo, fhi = Fv[line, kk].copy(), Fv[line, kk + 1].copy()
        slo = flo > 0.0
        active = np.ones(lo_t.size, dtype=bool)
        for _ in range(200):
            mid = 0.5 * (lo_t + hi_t)
            active &= ~((mid == lo_t) | (mid == hi_t))
            idx = np.nonzero(active)[0]
            if idx.size == 0:
                break
            fm = phi_at(mid[idx], line[idx])
            same = (fm > 0.0) == slo[idx]
            lo_t[idx[same]] = mid[idx[same]]
            flo[idx[same]] = fm[same]
            hi_t[idx[~same]] = mid[idx[~same]]
            fhi[idx[~same]] = fm[~same]
        t = np.where(np.abs(flo) <= np.abs(fhi), lo_t, hi_t)
        first = np.r_[True, line[1:] != line[:-1]]
        start = np.maximum.accumulate(np.where(first, np.arange(line.size), 0))
        ordinal = np.arange(line.size) - start
        P = np.empty((3, t.size))
        P[i], P[a_], P[b_] = t, xa[line], xb[line]
        nrm = molecule_normal(centers, r, c, P) if t.size else np.zeros((3, 0))
        keep = np.abs(nrm[i]) >= ct
        P, nrm = P[:, keep], nrm[:, keep]
        psi = pou(nrm, angle_deg)[i]
        w = psi * (h * h) / np.abs(nrm[i])
        meta = np.stack([np.full(P.shape[1], i), JA[line][keep], JB[line][keep], ordinal[keep]]).astype(np.int32)
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
