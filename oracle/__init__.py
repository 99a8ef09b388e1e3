"""FP64 CPU oracle for the regularized boundary-integral Stokes-Darcy solver.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference leg of ``bench.py`` may import anything here.
The product path (``paper_2110_10749_gb300``) never imports this package and
shares no code, header, table or constant with it.

Contents
--------
pairsum.c      smoothing factors s_1..s_4 and the four layer operators as
               plain double loops (Section 5.1-5.3), compiled with gcc.
quadrature.py  quadrature points and weights (Section 5.4, eq. Quadrature).
solvers.py     GMRES, successive approximations, Darcy and Stokes solves,
               the Dirichlet-Neumann iteration (Sections 3 and 6).
analytic.py    Joseph-Tao porous-sphere solution, drag, spectrum (Sections 4, 7.3);
               the porous sphere with Beavers-Joseph-Saffman slip (derived).
field.py       off-surface Darcy pressure and Stokes velocity (eqs. Greens, Stokes).

Parity status: every function is pinned by the ``-m "not gpu"`` tests
(closed forms, identities, printed table values); none is "parity unpinned".
The BJS mode of ``solvers.ddm_solve`` (no printed value exists) is pinned by
the porous sphere with slip, a closed form derived in ``analytic.py`` and
itself checked symbolically against the Stokes equations and the interface
conditions; the opposite slip sign gives a different drag and field.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pairsum.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile pairsum.c into ``oracle/_build/liboracle.so`` with gcc."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
           "-std=c11", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            d, i64, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_int
            P = ctypes.c_void_p
            L.ssdo_s_closed.argtypes = [i32, d]
            L.ssdo_s_closed.restype = d
            L.ssdo_sigma.argtypes = [i32, d]
            L.ssdo_sigma.restype = d
            L.ssdo_s.argtypes = [i32, d]
            L.ssdo_s.restype = d
            L.ssdo_laplace_sl.argtypes = [i64, P, i64, P, P, d, P, P]
            L.ssdo_laplace_dl.argtypes = [i64, P, P, P, d, P, i64, P, P]
            L.ssdo_stokes_sl.argtypes = [i64, P, i64, P, P, d, d, P, P]
            L.ssdo_stokes_dl.argtypes = [i64, P, P, P, d, P, i64, P, P]
            L.ssdo_operator_matrix.argtypes = [i32, i64, P, P, P, d, d, P]
            L.ssdo_operator_matrix.restype = None
            L.ssdo_num_threads.restype = i32
            L.ssdo_set_threads.argtypes = [i32]
            L.ssdo_set_threads.restype = None
            _lib = L
    return _lib


def _c(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.c_void_p)


def s(i: int, rho: float) -> float:
    """Smoothing factor s_i(rho), i = 1..4 (Section 5.3)."""
    return lib().ssdo_s(i, float(rho))


def s_closed(i: int, rho: float) -> float:
    """Closed form of s_i(rho) without the small-rho series branch."""
    return lib().ssdo_s_closed(i, float(rho))


def sigma(i: int, rho: float) -> float:
    """s_i(rho) / rho^p with p = 1, 3, 3, 5 for i = 1..4."""
    return lib().ssdo_sigma(i, float(rho))


def num_threads() -> int:
    return int(lib().ssdo_num_threads())


def set_num_threads(t: int) -> None:
    """Thread count of the oracle's OpenMP loops (for baseline timings)."""
    lib().ssdo_set_threads(int(t))


def laplace_sl(pts, delta, g, targets=None):
    """(L g)(y) = sum_x w g G^delta, G^delta = -s_1/(4 pi r)."""
    xyz, w = pts["xyz"], pts["w"]
    ty = xyz if targets is None else targets
    sx, psx = _c(xyz)
    ty, pty = _c(ty)
    w, pw = _c(w)
    g, pg = _c(g)
    nt, ns = ty.shape[1], sx.shape[1]
    out = np.empty(nt)
    lib().ssdo_laplace_sl(nt, pty, ns, psx, pw, float(delta), pg,
                          out.ctypes.data_as(ctypes.c_void_p))
    return out


def _rows(rows):
    if rows is None:
        return None, 0, None
    r = np.ascontiguousarray(rows, dtype=np.int64)
    return r, r.size, r.ctypes.data_as(ctypes.c_void_p)


def laplace_dl(pts, delta, p, rows=None):
    """(D^L p)(y) = sum_x w [p(x) - p(y)] dG^delta/dn_x  (eq. H_subtr).

    rows: optional target indices; the result then holds those targets only.
    """
    xyz, n_, w = _c(pts["xyz"]), _c(pts["nrm"]), _c(pts["w"])
    p = _c(p)
    n = xyz[0].shape[1]
    keep, nr, pr = _rows(rows)
    out = np.empty(nr if rows is not None else n)
    lib().ssdo_laplace_dl(n, xyz[1], n_[1], w[1], float(delta), p[1], nr, pr,
                          out.ctypes.data_as(ctypes.c_void_p))
    return out


def stokes_sl(pts, delta, mu, f, targets=None):
    """(M f)(y) = 1/(8 pi mu) sum_x w S^delta f; f is [3][n]."""
    xyz, w = pts["xyz"], pts["w"]
    ty = xyz if targets is None else targets
    sx, psx = _c(xyz)
    ty, pty = _c(ty)
    w, pw = _c(w)
    f, pf = _c(f)
    nt, ns = ty.shape[1], sx.shape[1]
    out = np.empty((3, nt))
    lib().ssdo_stokes_sl(nt, pty, ns, psx, pw, float(delta), float(mu), pf,
                         out.ctypes.data_as(ctypes.c_void_p))
    return out


def stokes_dl(pts, delta, u, rows=None):
    """(D^S u)(y) = -1/(8 pi) sum_x w [u(x)-u(y)].T^delta.n_x  (eq. K_subtr).

    rows: optional target indices; the result is then [3][len(rows)].
    """
    xyz, n_, w = _c(pts["xyz"]), _c(pts["nrm"]), _c(pts["w"])
    u = _c(u)
    n = xyz[0].shape[1]
    keep, nr, pr = _rows(rows)
    out = np.empty((3, nr if rows is not None else n))
    lib().ssdo_stokes_dl(n, xyz[1], n_[1], w[1], float(delta), u[1], nr, pr,
                         out.ctypes.data_as(ctypes.c_void_p))
    return out


def operator_matrix(pts, delta, op, mu=1.0):
    """Dense matrix of L, D^L, M or D^S (op = "L", "DL", "M", "DS"), acting on
    densities in the component-major order [3][n] -> 3n of the operators above."""
    code = {"L": 0, "DL": 1, "M": 2, "DS": 3}[op]
    xyz, n_, w = _c(pts["xyz"]), _c(pts["nrm"]), _c(pts["w"])
    n = xyz[0].shape[1]
    m = (3 if code >= 2 else 1) * n
    out = np.empty((m, m))
    lib().ssdo_operator_matrix(code, n, xyz[1], n_[1], w[1], float(delta), float(mu),
                               out.ctypes.data_as(ctypes.c_void_p))
    return out
