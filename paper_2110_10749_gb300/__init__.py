"""Python binding of libssd (C ABI in include/ssd.h).

Regularized boundary integrals and the Dirichlet-Neumann solve of the
coupled Stokes-Darcy problem (arXiv 2110.10749) on sm_103a.  This module only
marshals arguments: every step of the computation runs in the CUDA library.
PyTorch supplies device memory and the current stream.  Importing works
without a GPU; every call that computes needs the built library and a GPU and
raises if either is missing (there is no CPU fallback).  The one exception is
hessenberg_eigenvalues, the spectrum's host step, which is host code of the
library by design.

Functions keep the C names without the ``ssd_`` prefix.  Arrays are
structure-of-arrays float64 CUDA tensors: points and vector densities have
shape (3, n), scalars (n,).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libssd.so")

SSD_OK, SSD_EINVAL, SSD_ENOMEM, SSD_ECUDA, SSD_ENOTCONV, SSD_ENUMERIC = range(6)
FP64, FP32C = 0, 1
SPHERE, ELLIPSOID, STAR, MOLECULE = 0, 1, 2, 3
TRACTION_BJS, TRACTION_JOSEPH_TAO = 0, 1
K_LAPLACE_SL, K_LAPLACE_DL, K_STOKES_SL, K_STOKES_DL, K_STOKES_SLDL, K_LAPLACE_SLDL, K_LAPLACE_DL_T, K_STOKES_DL_T = range(8)

# Every entry point declared in include/ssd.h.
EXPORTS = [
    "ssd_ctx_create", "ssd_ctx_destroy", "ssd_status_string", "ssd_ctx_last_error",
    "ssd_ctx_set_timing", "ssd_ctx_kernel_stats", "ssd_ctx_reset_stats", "ssd_ctx_launch_count", "ssd_sync",
    "ssd_fp32_fma_rate",
    "ssd_quadrature_points", "ssd_quadrature_jacobian", "ssd_points_prepare", "ssd_points_release",
    "ssd_laplace_SL", "ssd_laplace_DL", "ssd_stokes_SL", "ssd_stokes_DL",
    "ssd_stokes_SLDL", "ssd_laplace_SLDL", "ssd_apply_rows", "ssd_points_order",
    "ssd_darcy_solve", "ssd_stokes_solve", "ssd_ddm_solve", "ssd_ddm_solve_host", "ssd_ddm_sweep",
    "ssd_batch_prepare", "ssd_batch_release", "ssd_batch_apply", "ssd_batch_ddm_solve",
    "ssd_stokes_DL_noalloc", "ssd_apply_transpose", "ssd_ddm_gradient",
    "ssd_ddm_gradient_geometry", "ssd_geometry_gradient", "ssd_shape_contract",
    "ssd_darcy_pressure_field", "ssd_stokes_velocity_field", "ssd_stokes_pressure_field", "ssd_ddm_spectrum",
    "ssd_ddm_iteration_matrix",
    "ssd_hessenberg_eigenvalues",
]
OP_LAPLACE_SL, OP_LAPLACE_DL, OP_STOKES_SL, OP_STOKES_DL, OP_STOKES_SLDL, OP_LAPLACE_SLDL = range(6)
FUNC_DRAG, FUNC_FLUX = 0, 1


class SsdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s (status %d)" % (msg, status))
        self.status = status


class NotConverged(SsdError):
    pass


class Layout(C.Structure):
    pass


class CPoints(C.Structure):
    _fields_ = [("n", C.c_int64), ("xyz", C.c_void_p), ("nrm", C.c_void_p), ("w", C.c_void_p),
                ("layout", C.POINTER(Layout))]


class CSurface(C.Structure):
    _fields_ = [("kind", C.c_int), ("center", C.c_double * 3), ("abc", C.c_double * 3),
                ("clm", C.POINTER(C.c_double))]


class CKrylov(C.Structure):
    _fields_ = [("tol", C.c_double), ("maxit", C.c_int), ("restart", C.c_int), ("use_sa", C.c_int),
                ("prec", C.c_int), ("deflate", C.c_int), ("warm", C.c_int)]


class CDdmParams(C.Structure):
    _fields_ = [("mu", C.c_double), ("kappa", C.c_double), ("gamma", C.c_double), ("uinf", C.c_double * 3),
                ("delta", C.c_double), ("theta", C.c_double), ("tol_outer", C.c_double),
                ("maxit_outer", C.c_int), ("outer_gmres", C.c_int), ("traction_mode", C.c_int),
                ("bjs_implicit", C.c_int), ("bjs_sign", C.c_double), ("radius", C.c_double), ("inner", CKrylov),
                ("refine", C.c_int)]


class BatchLayoutC(C.Structure):
    pass


class CBatch(C.Structure):
    _fields_ = [("nsurf", C.c_int32), ("offsets", C.POINTER(C.c_int64)), ("delta", C.POINTER(C.c_double)),
                ("xyz", C.c_void_p), ("nrm", C.c_void_p), ("w", C.c_void_p), ("layout", C.POINTER(BatchLayoutC))]


class CKernelStats(C.Structure):
    _fields_ = [("launches", C.c_int64), ("ms", C.c_double), ("pairs", C.c_double)]


_lib = None


def library_path() -> str:
    return LIB_PATH


def lib():
    """Load libssd.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libssd.so is not built (run __graft_entry__.build() or "
                           "python -m paper_2110_10749_gb300.build): %s" % LIB_PATH)
    L = C.CDLL(LIB_PATH)
    P, i, d, i64 = C.c_void_p, C.c_int, C.c_double, C.c_int64
    sig = {
        "ssd_ctx_create": [C.POINTER(P), i],
        "ssd_ctx_destroy": [P],
        "ssd_status_string": [i],
        "ssd_ctx_last_error": [P],
        "ssd_ctx_set_timing": [P, i],
        "ssd_ctx_kernel_stats": [P, i, i, C.POINTER(CKernelStats)],
        "ssd_ctx_reset_stats": [P],
        "ssd_ctx_launch_count": [P, C.POINTER(i64)],
        "ssd_sync": [P, P],
        "ssd_fp32_fma_rate": [P, i, C.POINTER(d)],
        "ssd_quadrature_points": [P, C.POINTER(CSurface), d, d, i64, C.POINTER(i64), P, P, P, P, P],
        "ssd_quadrature_jacobian": [P, C.POINTER(CSurface), d, d, i64, P, P, P, P],
        "ssd_points_prepare": [P, C.POINTER(CPoints), P],
        "ssd_points_release": [P, C.POINTER(CPoints)],
        "ssd_laplace_SL": [P, C.POINTER(CPoints), d, P, P, i, P],
        "ssd_laplace_DL": [P, C.POINTER(CPoints), d, P, P, i, P],
        "ssd_stokes_SL": [P, C.POINTER(CPoints), d, d, P, P, i, P],
        "ssd_stokes_DL": [P, C.POINTER(CPoints), d, P, P, i, P],
        "ssd_apply_rows": [P, C.POINTER(CPoints), i, d, d, P, i64, i64, P, i, P],
        "ssd_points_order": [P, C.POINTER(CPoints), P, P],
        "ssd_stokes_SLDL": [P, C.POINTER(CPoints), d, d, P, P, d, d, P, i, P],
        "ssd_laplace_SLDL": [P, C.POINTER(CPoints), d, P, P, d, d, P, i, P],
        "ssd_darcy_solve": [P, C.POINTER(CPoints), d, d, d, P, P, C.POINTER(CKrylov), C.POINTER(i),
                            C.POINTER(d), P],
        "ssd_stokes_solve": [P, C.POINTER(CPoints), d, d, P, C.POINTER(d), P, C.POINTER(CKrylov),
                             C.POINTER(i), C.POINTER(d), P],
        "ssd_ddm_solve": [P, C.POINTER(CPoints), C.POINTER(CDdmParams), P, P, P, P, C.POINTER(d),
                          C.POINTER(i), C.POINTER(i), C.POINTER(d), P],
        "ssd_ddm_solve_host": [P, i64, P, P, P, C.POINTER(CDdmParams), P, P, P, P, C.POINTER(d),
                               C.POINTER(i), C.POINTER(i), C.POINTER(d), P],
        "ssd_ddm_sweep": [P, C.POINTER(CPoints), C.POINTER(CDdmParams), P, P, P, P, P, P, C.POINTER(i), P],
        "ssd_stokes_DL_noalloc": [P, C.POINTER(CPoints), d, P, P, P],
        "ssd_apply_transpose": [P, C.POINTER(CPoints), i, d, d, P, P, i, P],
        "ssd_ddm_gradient": [P, C.POINTER(CPoints), C.POINTER(CDdmParams), i, C.POINTER(d), C.POINTER(d), P],
        "ssd_ddm_gradient_geometry": [P, C.POINTER(CPoints), C.POINTER(CDdmParams), i, C.POINTER(d),
                                      C.POINTER(d), P, P, P, P],
        "ssd_geometry_gradient": [P, C.POINTER(CPoints), i, d, d, d, P, P, P, P, P, P],
        "ssd_shape_contract": [P, i64, i, P, P, P, P, P, P, C.POINTER(d), P],
        "ssd_darcy_pressure_field": [P, C.POINTER(CPoints), d, d, P, P, i64, P, P, P],
        "ssd_ddm_spectrum": [P, C.POINTER(CPoints), C.POINTER(CDdmParams), i, C.POINTER(i), C.POINTER(d),
                             C.POINTER(d), C.POINTER(d), P],
        "ssd_stokes_velocity_field": [P, C.POINTER(CPoints), d, C.POINTER(d), P, P, i64, P, P, P],
        "ssd_stokes_pressure_field": [P, C.POINTER(CPoints), d, P, P, i64, P, P, P],
        "ssd_ddm_iteration_matrix": [P, C.POINTER(CPoints), C.POINTER(CDdmParams), i64, i64, P, P],
        "ssd_hessenberg_eigenvalues": [i, C.POINTER(d), i, C.POINTER(d), C.POINTER(d)],
        "ssd_batch_prepare": [P, C.POINTER(CBatch), P],
        "ssd_batch_release": [P, C.POINTER(CBatch)],
        "ssd_batch_apply": [P, C.POINTER(CBatch), i, i, d, d, d, P, P, P, i, P],
        "ssd_batch_ddm_solve": [P, C.POINTER(CBatch), C.POINTER(CDdmParams), i, C.POINTER(d), P, P, P, P,
                                C.POINTER(d), C.POINTER(i), C.POINTER(d), P],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = C.c_int
    L.ssd_status_string.restype = C.c_char_p
    L.ssd_ctx_last_error.restype = C.c_char_p
    _lib = L
    return L


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("a CUDA device is required; libssd has no CPU path")
    return torch


def _stream():
    torch = _torch()
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda or t.dtype != _torch().float64 or not t.is_contiguous():
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _check_arg(t, numel, device, what):
    """The C calls read or write exactly `numel` elements of each device
    array and cannot see a tensor's size: check it (and that the array sits
    on the points' device) before passing the pointer."""
    if t is None:
        return
    if t.numel() != numel:
        raise ValueError("%s: expected %d elements, got %d (shape %s)" % (what, numel, t.numel(), tuple(t.shape)))
    if device is not None and t.device != device:
        raise ValueError("%s: on %s, the points are on %s" % (what, t.device, device))


def _arg(t, numel, device, what):
    _check_arg(t, numel, device, what)
    return _ptr(t)


def _nc(op):
    """Components of an operator's densities (1 Laplace, 3 Stokes)."""
    return 1 if op in (OP_LAPLACE_SL, OP_LAPLACE_DL, OP_LAPLACE_SLDL) else 3


class Context:
    """Owns an ssd_ctx on one device."""

    def __init__(self, device: int = 0):
        _torch()
        h = C.c_void_p()
        st = lib().ssd_ctx_create(C.byref(h), int(device))
        if st != SSD_OK:
            raise SsdError(st, "ssd_ctx_create failed: %s" % lib().ssd_status_string(st).decode())
        self.h = h
        self.device = device

    def check(self, st, what):
        if st == SSD_OK:
            return
        msg = lib().ssd_ctx_last_error(self.h).decode()
        cls = NotConverged if st == SSD_ENOTCONV else SsdError
        raise cls(st, "%s: %s" % (what, msg))

    def close(self):
        if self.h:
            lib().ssd_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_timing(self, on=True):
        self.check(lib().ssd_ctx_set_timing(self.h, 1 if on else 0), "ssd_ctx_set_timing")

    def kernel_stats(self, kernel_class, prec):
        s = CKernelStats()
        self.check(lib().ssd_ctx_kernel_stats(self.h, kernel_class, prec, C.byref(s)), "ssd_ctx_kernel_stats")
        return {"launches": s.launches, "ms": s.ms, "pairs": s.pairs}

    def reset_stats(self):
        self.check(lib().ssd_ctx_reset_stats(self.h), "ssd_ctx_reset_stats")

    def fp32_fma_rate(self, packed=True):
        """Measured FP32 FMA rate of the device in TFLOP/s (FMA = 2 flops)."""
        v = C.c_double()
        self.check(lib().ssd_fp32_fma_rate(self.h, 1 if packed else 0, C.byref(v)), "ssd_fp32_fma_rate")
        return v.value

    def launch_count(self):
        v = C.c_int64()
        self.check(lib().ssd_ctx_launch_count(self.h, C.byref(v)), "ssd_ctx_launch_count")
        return v.value

    def sync(self, device_wide=False):
        """ssd_sync on torch's current stream (or the whole device): raises
        SsdError if a kernel of an asynchronous call failed."""
        self.check(lib().ssd_sync(self.h, None if device_wide else _stream()), "ssd_sync")


class Points:
    """A quadrature point set on the device: xyz, nrm (3, n) and w (n,)."""

    def __init__(self, xyz, nrm, w):
        torch = _torch()
        self.xyz = xyz.to(dtype=torch.float64).contiguous()
        self.nrm = nrm.to(dtype=torch.float64).contiguous()
        self.w = w.to(dtype=torch.float64).contiguous()
        self.n = int(self.w.numel())
        if self.xyz.shape != (3, self.n) or self.nrm.shape != (3, self.n):
            raise ValueError("xyz and nrm must have shape (3, n) with n = w.numel()")
        if self.xyz.device != self.w.device or self.nrm.device != self.w.device:
            raise ValueError("xyz, nrm and w must be on one device")
        self.c = CPoints(self.n, _ptr(self.xyz), _ptr(self.nrm), _ptr(self.w), None)
        self.ctx = None

    @classmethod
    def from_numpy(cls, pts, device="cuda"):
        torch = _torch()
        return cls(torch.as_tensor(pts["xyz"], device=device), torch.as_tensor(pts["nrm"], device=device),
                   torch.as_tensor(pts["w"], device=device))

    def prepare(self, ctx):
        ctx.check(lib().ssd_points_prepare(ctx.h, C.byref(self.c), _stream()), "ssd_points_prepare")
        self.ctx = ctx
        return self

    def release(self):
        if self.ctx is not None and self.c.layout:
            lib().ssd_points_release(self.ctx.h, C.byref(self.c))
        self.ctx = None


def surface(kind, abc=(1.0,), center=(0.0, 0.0, 0.0), clm=None):
    """ssd_surface for SPHERE (abc = (R,)), ELLIPSOID (abc = (a, b, c)) or STAR (clm[25])."""
    abc = list(abc) if kind != STAR else []
    cl = None
    if kind == STAR:
        cl = (C.c_double * 25)(*[float(v) for v in clm])
    s = CSurface(kind, (C.c_double * 3)(*center), (C.c_double * 3)(*(abc + [0.0] * (3 - len(abc)))),
                 C.cast(cl, C.POINTER(C.c_double)) if cl is not None else None)
    s._keep = cl
    return s


def quadrature_points(ctx, kind, abc=(1.0,), h=1 / 8, angle_deg=70.0, center=(0.0, 0.0, 0.0), clm=None):
    """Quadrature points (Section 5.4) of a sphere, ellipsoid or star surface: dict of CUDA tensors."""
    torch = _torch()
    surf = surface(kind, abc, center, clm)
    n = C.c_int64()
    L = lib()
    ctx.check(L.ssd_quadrature_points(ctx.h, C.byref(surf), float(h), float(angle_deg), 0, C.byref(n),
                                      None, None, None, None, _stream()), "ssd_quadrature_points")
    N = n.value
    dev = torch.device("cuda", ctx.device)
    xyz = torch.empty((3, N), dtype=torch.float64, device=dev)
    nrm = torch.empty((3, N), dtype=torch.float64, device=dev)
    w = torch.empty((N,), dtype=torch.float64, device=dev)
    meta = torch.empty((4, N), dtype=torch.int32, device=dev)
    ctx.check(L.ssd_quadrature_points(ctx.h, C.byref(surf), float(h), float(angle_deg), N, C.byref(n),
                                      _ptr(xyz), _ptr(nrm), _ptr(w), C.c_void_p(meta.data_ptr()), _stream()),
              "ssd_quadrature_points")
    return {"xyz": xyz, "nrm": nrm, "w": w, "meta": meta}


def molecule_points(ctx, h, r=0.5, c=0.6, angle_deg=70.0, center=(0.0, 0.0, 0.0)):
    """Quadrature points of the four-atom molecule (eq. Molecule)."""
    return quadrature_points(ctx, MOLECULE, (r, c), h, angle_deg, center)


def quadrature_jacobian(ctx, clm, h, n, angle_deg=70.0, center=(0.0, 0.0, 0.0)):
    """Derivatives of a STAR surface's points, normals and weights in its 25
    coefficients: dict dxyz (25, 3, n), dnrm (25, 3, n), dw (25, n)."""
    torch = _torch()
    surf = surface(STAR, (), center, clm)
    dev = torch.device("cuda", ctx.device)
    dx = torch.empty((25, 3, n), dtype=torch.float64, device=dev)
    dn = torch.empty((25, 3, n), dtype=torch.float64, device=dev)
    dw = torch.empty((25, n), dtype=torch.float64, device=dev)
    ctx.check(lib().ssd_quadrature_jacobian(ctx.h, C.byref(surf), float(h), float(angle_deg), int(n), _ptr(dx),
                                            _ptr(dn), _ptr(dw), _stream()), "ssd_quadrature_jacobian")
    return {"dxyz": dx, "dnrm": dn, "dw": dw}


def _out_like(t, out):
    return _torch().empty_like(t) if out is None else out


def laplace_SL(ctx, pts, delta, g, prec=FP64, out=None):
    out = _out_like(g, out)
    n, dv = pts.n, pts.xyz.device
    ctx.check(lib().ssd_laplace_SL(ctx.h, C.byref(pts.c), float(delta), _arg(g, n, dv, "g"), _arg(out, n, dv, "out"),
                                   prec, _stream()), "ssd_laplace_SL")
    return out


def laplace_DL(ctx, pts, delta, p, prec=FP64, out=None):
    out = _out_like(p, out)
    n, dv = pts.n, pts.xyz.device
    ctx.check(lib().ssd_laplace_DL(ctx.h, C.byref(pts.c), float(delta), _arg(p, n, dv, "p"), _arg(out, n, dv, "out"),
                                   prec, _stream()), "ssd_laplace_DL")
    return out


def stokes_SL(ctx, pts, delta, mu, f, prec=FP64, out=None):
    out = _out_like(f, out)
    n3, dv = 3 * pts.n, pts.xyz.device
    ctx.check(lib().ssd_stokes_SL(ctx.h, C.byref(pts.c), float(delta), float(mu), _arg(f, n3, dv, "f"),
                                  _arg(out, n3, dv, "out"), prec, _stream()), "ssd_stokes_SL")
    return out


def stokes_DL(ctx, pts, delta, u, prec=FP64, out=None):
    out = _out_like(u, out)
    n3, dv = 3 * pts.n, pts.xyz.device
    ctx.check(lib().ssd_stokes_DL(ctx.h, C.byref(pts.c), float(delta), _arg(u, n3, dv, "u"),
                                  _arg(out, n3, dv, "out"), prec, _stream()), "ssd_stokes_DL")
    return out


def apply_rows(ctx, pts, op, delta, dens, row_begin, row_end, mu=1.0, prec=FP64, out=None):
    """Rows [row_begin, row_end) of the spatial order of op (OP_LAPLACE_SL/DL,
    OP_STOKES_SL/DL) applied to dens; only those rows of `out` are written
    (a new zero-filled array when out is None)."""
    if out is None:
        out = _torch().zeros_like(dens)
    m, dv = _nc(op) * pts.n, pts.xyz.device
    ctx.check(lib().ssd_apply_rows(ctx.h, C.byref(pts.c), int(op), float(delta), float(mu), _arg(dens, m, dv, "dens"),
                                   int(row_begin), int(row_end), _arg(out, m, dv, "out"), int(prec), _stream()),
              "ssd_apply_rows")
    return out


def points_order(ctx, pts):
    """Spatial order of the point set: numpy int32 [n], caller index of each row."""
    order = np.empty(pts.n, dtype=np.int32)
    ctx.check(lib().ssd_points_order(ctx.h, C.byref(pts.c), order.ctypes.data_as(C.c_void_p), _stream()),
              "ssd_points_order")
    return order


def apply_transpose(ctx, pts, op, delta, dens, mu=1.0, prec=FP64, out=None):
    """out = A^T dens for op in OP_LAPLACE_SL/DL, OP_STOKES_SL/DL (adjoint operators)."""
    out = _out_like(dens, out)
    m, dv = _nc(op) * pts.n, pts.xyz.device
    ctx.check(lib().ssd_apply_transpose(ctx.h, C.byref(pts.c), int(op), float(delta), float(mu),
                                        _arg(dens, m, dv, "dens"), _arg(out, m, dv, "out"), int(prec), _stream()),
              "ssd_apply_transpose")
    return out


def stokes_DL_noalloc(ctx, pts, delta, u, out=None):
    """Stokes double layer in FP32C without device allocation (see include/ssd.h)."""
    out = _out_like(u, out)
    n3, dv = 3 * pts.n, pts.xyz.device
    ctx.check(lib().ssd_stokes_DL_noalloc(ctx.h, C.byref(pts.c), float(delta), _arg(u, n3, dv, "u"),
                                          _arg(out, n3, dv, "out"), _stream()), "ssd_stokes_DL_noalloc")
    return out


def stokes_SLDL(ctx, pts, delta, mu, f, u, alpha=1.0, beta=1.0, prec=FP64, out=None):
    out = _out_like(u, out)
    n3, dv = 3 * pts.n, pts.xyz.device
    ctx.check(lib().ssd_stokes_SLDL(ctx.h, C.byref(pts.c), float(delta), float(mu), _arg(f, n3, dv, "f"),
                                    _arg(u, n3, dv, "u"), float(alpha), float(beta), _arg(out, n3, dv, "out"), prec,
                                    _stream()), "ssd_stokes_SLDL")
    return out


def laplace_SLDL(ctx, pts, delta, g, p, alpha=1.0, beta=1.0, prec=FP64, out=None):
    out = _out_like(p, out)
    n, dv = pts.n, pts.xyz.device
    ctx.check(lib().ssd_laplace_SLDL(ctx.h, C.byref(pts.c), float(delta), _arg(g, n, dv, "g"), _arg(p, n, dv, "p"),
                                     float(alpha), float(beta), _arg(out, n, dv, "out"), prec, _stream()),
              "ssd_laplace_SLDL")
    return out


def krylov(tol=1e-9, maxit=200, restart=50, use_sa=False, prec=FP64, deflate=False, warm=False):
    return CKrylov(float(tol), int(maxit), int(restart), 1 if use_sa else 0, int(prec), 1 if deflate else 0,
                   1 if warm else 0)


def darcy_solve(ctx, pts, delta, mu, kappa, q, kr=None, out=None):
    kr = kr or krylov()
    out = _out_like(q, out)
    its, rel = C.c_int(), C.c_double()
    n, dv = pts.n, pts.xyz.device
    ctx.check(lib().ssd_darcy_solve(ctx.h, C.byref(pts.c), float(delta), float(mu), float(kappa),
                                    _arg(q, n, dv, "q"), _arg(out, n, dv, "out"), C.byref(kr), C.byref(its),
                                    C.byref(rel), _stream()),
              "ssd_darcy_solve")
    return out, its.value, rel.value


def stokes_solve(ctx, pts, delta, mu, f, uinf, kr=None, out=None):
    kr = kr or krylov()
    out = _out_like(f, out)
    its, rel = C.c_int(), C.c_double()
    ui = (C.c_double * 3)(*uinf)
    n3, dv = 3 * pts.n, pts.xyz.device
    ctx.check(lib().ssd_stokes_solve(ctx.h, C.byref(pts.c), float(delta), float(mu), _arg(f, n3, dv, "f"), ui,
                                     _arg(out, n3, dv, "out"), C.byref(kr), C.byref(its), C.byref(rel), _stream()),
              "ssd_stokes_solve")
    return out, its.value, rel.value


def ddm_params(mu=1.0, kappa=1.0, gamma=0.0, uinf=(0.0, 0.0, 1.0), delta=0.1, theta=0.5, tol_outer=1e-9,
               maxit_outer=100, outer_gmres=False, traction_mode=TRACTION_BJS, bjs_sign=1.0, radius=1.0,
               inner=None, bjs_implicit=False, refine=0):
    return CDdmParams(float(mu), float(kappa), float(gamma), (C.c_double * 3)(*uinf), float(delta), float(theta),
                      float(tol_outer), int(maxit_outer), 1 if outer_gmres else 0, int(traction_mode),
                      1 if bjs_implicit else 0, float(bjs_sign), float(radius), inner or krylov(), int(refine))


def _ddm_out(prm, n, dev):
    torch = _torch()
    return {"q": torch.empty((n,), dtype=torch.float64, device=dev),
            "p": torch.empty((n,), dtype=torch.float64, device=dev),
            "u": torch.empty((3, n), dtype=torch.float64, device=dev),
            "f": torch.empty((3, n), dtype=torch.float64, device=dev)}


def _history(hist, cap):
    """The entries of a residual history up to its -1 end mark."""
    out = []
    for k in range(max(cap, 1)):
        if hist[k] < 0.0:
            break
        out.append(hist[k])
    return out


def ddm_solve(ctx, pts, prm, raise_on_notconv=True):
    """Dirichlet-Neumann solve (Sections 3, 6).  Returns a dict of results."""
    o = _ddm_out(prm, pts.n, pts.xyz.device)
    drag = (C.c_double * 3)()
    oits = C.c_int()
    cap = 2 * (prm.maxit_outer + 2)
    inner = (C.c_int * cap)()
    hist = (C.c_double * max(prm.maxit_outer, 1))()
    st = lib().ssd_ddm_solve(ctx.h, C.byref(pts.c), C.byref(prm), _ptr(o["q"]), _ptr(o["p"]), _ptr(o["u"]),
                             _ptr(o["f"]), drag, C.byref(oits), inner, hist, _stream())
    if st != SSD_ENOTCONV or raise_on_notconv:
        ctx.check(st, "ssd_ddm_solve")
    o["drag"] = np.array(drag[:])
    o["outer_its"] = oits.value
    n_sweeps = oits.value + 2 if prm.outer_gmres else oits.value
    o["inner_its"] = [(inner[2 * k], inner[2 * k + 1]) for k in range(min(n_sweeps, cap // 2))]
    o["hist"] = _history(hist, prm.maxit_outer)
    o["status"] = st
    return o


def ddm_sweep(ctx, pts, prm, q, u_prev=None, out=None, raise_on_notconv=True):
    """One D-N sweep from (q, u_prev): dict with q (the relaxed update), p, u, f,
    inner_its (Darcy, Stokes) and status."""
    n, dv = pts.n, pts.xyz.device
    o = out or _ddm_out(prm, n, dv)
    its = (C.c_int * 2)()
    st = lib().ssd_ddm_sweep(ctx.h, C.byref(pts.c), C.byref(prm), _arg(q, n, dv, "q"),
                             _arg(u_prev, 3 * n, dv, "u_prev"), _arg(o["q"], n, dv, "q_out"),
                             _arg(o["p"], n, dv, "p"), _arg(o["u"], 3 * n, dv, "u"), _arg(o["f"], 3 * n, dv, "f"),
                             its, _stream())
    if st != SSD_ENOTCONV or raise_on_notconv:
        ctx.check(st, "ssd_ddm_sweep")
    o["inner_its"] = (its[0], its[1])
    o["status"] = st
    return o


def _host_ptr(a, shape, writable=False):
    """Pointer to a host float64 array of the given shape (numpy array or CPU
    tensor, pinned for the fastest copies).  Inputs of another dtype or
    layout are converted (the converted array is returned to keep it alive);
    outputs must already be contiguous float64 of that shape."""
    if hasattr(a, "data_ptr"):
        import torch
        if a.is_cuda or a.dtype != torch.float64 or not a.is_contiguous() or tuple(a.shape) != tuple(shape):
            raise ValueError("expected a contiguous float64 CPU tensor of shape %s" % (tuple(shape),))
        return C.c_void_p(a.data_ptr()), a
    if writable:
        if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous
                and a.flags.writeable and a.shape == tuple(shape)):
            raise ValueError("output must be a writable C-contiguous float64 array of shape %s" % (tuple(shape),))
    else:
        a = np.ascontiguousarray(a, dtype=np.float64)
        if a.shape != tuple(shape):
            raise ValueError("expected shape %s, got %s" % (tuple(shape), a.shape))
    return a.ctypes.data_as(C.c_void_p), a


def ddm_solve_host(ctx, xyz, nrm, w, prm, out=None, raise_on_notconv=True):
    """D-N solve with host (numpy or pinned CPU tensor) buffers; copies happen inside."""
    n = int(w.shape[0])
    out = out or {"q": np.empty(n), "p": np.empty(n), "u": np.empty((3, n)), "f": np.empty((3, n))}
    keep = [_host_ptr(xyz, (3, n)), _host_ptr(nrm, (3, n)), _host_ptr(w, (n,))]
    keep += [_host_ptr(out[k], sh, writable=True) for k, sh in (("q", (n,)), ("p", (n,)), ("u", (3, n)),
                                                                 ("f", (3, n)))]
    ptr = [k[0] for k in keep]
    drag = (C.c_double * 3)()
    oits = C.c_int()
    cap = 2 * (prm.maxit_outer + 2)
    inner = (C.c_int * cap)()
    hist = (C.c_double * max(prm.maxit_outer, 1))()
    st = lib().ssd_ddm_solve_host(ctx.h, n, ptr[0], ptr[1], ptr[2], C.byref(prm), ptr[3], ptr[4], ptr[5], ptr[6],
                                  drag, C.byref(oits), inner, hist, _stream())
    if st != SSD_ENOTCONV or raise_on_notconv:
        ctx.check(st, "ssd_ddm_solve_host")
    out["status"] = st
    out["drag"] = np.array(drag[:])
    out["outer_its"] = oits.value
    return out


def ddm_gradient(ctx, pts, prm, functional=FUNC_DRAG, raise_on_notconv=True):
    """J and (dJ/dlog(kappa), dJ/dgamma) of the D-N solve by the discrete adjoint.

    Returns (value, grad[2] as numpy, status)."""
    val = C.c_double()
    g = (C.c_double * 2)()
    st = lib().ssd_ddm_gradient(ctx.h, C.byref(pts.c), C.byref(prm), int(functional), C.byref(val), g, _stream())
    if st != SSD_ENOTCONV or raise_on_notconv:
        ctx.check(st, "ssd_ddm_gradient")
    return val.value, np.array(g[:]), st


def ddm_spectrum(ctx, pts, prm, m=50):
    """Ritz values of the discrete D-N iteration matrix (eq. A_mat) from m
    Arnoldi steps: (complex numpy array, Hessenberg (m+1, m) numpy array)."""
    mo = C.c_int()
    re = (C.c_double * m)()
    im = (C.c_double * m)()
    H = (C.c_double * ((m + 1) * m))()
    ctx.check(lib().ssd_ddm_spectrum(ctx.h, C.byref(pts.c), C.byref(prm), int(m), C.byref(mo), re, im, H,
                                     _stream()), "ssd_ddm_spectrum")
    k = mo.value
    ritz = np.array(re[:k]) + 1j * np.array(im[:k])
    Hm = np.array(H[:]).reshape(m, m + 1).T[:k + 1, :k]
    return ritz, Hm


def ddm_iteration_matrix(ctx, pts, prm, col0=0, ncol=None, out=None):
    """Columns col0 .. col0 + ncol - 1 of the discrete iteration matrix
    (eq. A_mat): CUDA tensor (n, ncol), column j = F(e_{col0+j}) - F(0)."""
    torch = _torch()
    n = pts.n
    ncol = n - col0 if ncol is None else int(ncol)
    if out is None:
        out = torch.empty((ncol, n), dtype=torch.float64, device=pts.xyz.device)
    ctx.check(lib().ssd_ddm_iteration_matrix(ctx.h, C.byref(pts.c), C.byref(prm), int(col0), ncol,
                                             _arg(out, n * ncol, pts.xyz.device, "out"), _stream()),
              "ssd_ddm_iteration_matrix")
    return out.T


def hessenberg_eigenvalues(H):
    """Eigenvalues (complex numpy array, in the library's deflation order) of
    the upper Hessenberg matrix H (n, n): the host QR step of ddm_spectrum,
    e.g. on a leading block of its H.  Host only; needs the built library but
    no GPU."""
    A = np.asfortranarray(np.asarray(H, dtype=np.float64))
    if A.ndim != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("expected a square matrix")
    n = A.shape[0]
    re = (C.c_double * max(n, 1))()
    im = (C.c_double * max(n, 1))()
    st = lib().ssd_hessenberg_eigenvalues(n, A.ctypes.data_as(C.POINTER(C.c_double)), n, re, im)
    if st != SSD_OK:
        raise SsdError(st, "ssd_hessenberg_eigenvalues: %s" % lib().ssd_status_string(st).decode())
    return np.array(re[:n]) + 1j * np.array(im[:n])


def darcy_pressure_field(ctx, pts, mu, kappa, q, p, targets, out=None):
    """Darcy pressure at field points inside the body (targets (3, nt) CUDA tensor)."""
    torch = _torch()
    nt = int(targets.shape[1])
    out = out if out is not None else torch.empty((nt,), dtype=torch.float64, device=targets.device)
    n, dv = pts.n, pts.xyz.device
    ctx.check(lib().ssd_darcy_pressure_field(ctx.h, C.byref(pts.c), float(mu), float(kappa), _arg(q, n, dv, "q"),
                                             _arg(p, n, dv, "p"), nt, _arg(targets, 3 * nt, dv, "targets"),
                                             _arg(out, nt, dv, "out"), _stream()), "ssd_darcy_pressure_field")
    return out


def stokes_velocity_field(ctx, pts, mu, uinf, f, u, targets, out=None):
    """Stokes velocity at field points outside the body (targets (3, nt) CUDA tensor)."""
    torch = _torch()
    nt = int(targets.shape[1])
    out = out if out is not None else torch.empty((3, nt), dtype=torch.float64, device=targets.device)
    ui = (C.c_double * 3)(*uinf)
    n3, dv = 3 * pts.n, pts.xyz.device
    ctx.check(lib().ssd_stokes_velocity_field(ctx.h, C.byref(pts.c), float(mu), ui, _arg(f, n3, dv, "f"),
                                              _arg(u, n3, dv, "u"), nt, _arg(targets, 3 * nt, dv, "targets"),
                                              _arg(out, 3 * nt, dv, "out"), _stream()), "ssd_stokes_velocity_field")
    return out


def stokes_pressure_field(ctx, pts, mu, f, u, targets, out=None):
    """Stokes pressure at field points outside the body (far-field pressure 0)."""
    torch = _torch()
    nt = int(targets.shape[1])
    out = out if out is not None else torch.empty((nt,), dtype=torch.float64, device=targets.device)
    n3, dv = 3 * pts.n, pts.xyz.device
    ctx.check(lib().ssd_stokes_pressure_field(ctx.h, C.byref(pts.c), float(mu), _arg(f, n3, dv, "f"),
                                              _arg(u, n3, dv, "u"), nt, _arg(targets, 3 * nt, dv, "targets"),
                                              _arg(out, nt, dv, "out"), _stream()), "ssd_stokes_pressure_field")
    return out


def geometry_gradient(ctx, pts, op, delta, a, b, mu=1.0, alpha=1.0, out=None):
    """Adds alpha d(a . K b)/d(x, n, w) to out = (gx, gn, gw) (allocated as zeros if None)."""
    torch = _torch()
    n = pts.n
    if out is None:
        dev = pts.xyz.device
        out = (torch.zeros((3, n), dtype=torch.float64, device=dev), torch.zeros((3, n), dtype=torch.float64,
               device=dev), torch.zeros((n,), dtype=torch.float64, device=dev))
    m, dv = _nc(op) * n, pts.xyz.device
    ctx.check(lib().ssd_geometry_gradient(ctx.h, C.byref(pts.c), int(op), float(delta), float(mu), float(alpha),
                                          _arg(a, m, dv, "a"), _arg(b, m, dv, "b"), _arg(out[0], 3 * n, dv, "gx"),
                                          _arg(out[1], 3 * n, dv, "gn"), _arg(out[2], n, dv, "gw"), _stream()),
              "ssd_geometry_gradient")
    return out


def ddm_gradient_geometry(ctx, pts, prm, functional=FUNC_DRAG, raise_on_notconv=True):
    """J, (dJ/dlog(kappa), dJ/dgamma) and dJ/d(x, n, w) per point."""
    torch = _torch()
    n = pts.n
    dev = pts.xyz.device
    gx = torch.empty((3, n), dtype=torch.float64, device=dev)
    gn = torch.empty((3, n), dtype=torch.float64, device=dev)
    gw = torch.empty((n,), dtype=torch.float64, device=dev)
    val = C.c_double()
    g = (C.c_double * 2)()
    st = lib().ssd_ddm_gradient_geometry(ctx.h, C.byref(pts.c), C.byref(prm), int(functional), C.byref(val), g,
                                         _ptr(gx), _ptr(gn), _ptr(gw), _stream())
    if st != SSD_ENOTCONV or raise_on_notconv:
        ctx.check(st, "ssd_ddm_gradient_geometry")
    return val.value, np.array(g[:]), (gx, gn, gw), st


def shape_contract(ctx, jac, geo):
    """dJ/dc_k from a quadrature Jacobian (dict) and geometry gradients (gx, gn, gw)."""
    ncoef, _, n = jac["dxyz"].shape
    out = (C.c_double * ncoef)()
    dv = jac["dxyz"].device
    ctx.check(lib().ssd_shape_contract(ctx.h, int(n), int(ncoef), _arg(jac["dxyz"], 3 * ncoef * n, dv, "dxyz"),
                                       _arg(jac["dnrm"], 3 * ncoef * n, dv, "dnrm"),
                                       _arg(jac["dw"], ncoef * n, dv, "dw"), _arg(geo[0], 3 * n, dv, "gx"),
                                       _arg(geo[1], 3 * n, dv, "gn"), _arg(geo[2], n, dv, "gw"), out, _stream()),
              "ssd_shape_contract")
    return np.array(out[:])


def ddm_shape_gradient(ctx, clm, h, prm, functional=FUNC_DRAG, angle_deg=70.0, center=(0.0, 0.0, 0.0)):
    """On the STAR surface with coefficients clm at spacing h (delta taken from
    prm): J, (dJ/dlog(kappa), dJ/dgamma) and dJ/dc_k for the 25 c_k."""
    q = quadrature_points(ctx, STAR, h=h, angle_deg=angle_deg, center=center, clm=clm)
    P = Points(q["xyz"], q["nrm"], q["w"]).prepare(ctx)
    try:
        J, g, geo, st = ddm_gradient_geometry(ctx, P, prm, functional)
        jac = quadrature_jacobian(ctx, clm, h, P.n, angle_deg, center)
        dc = shape_contract(ctx, jac, geo)
    finally:
        P.release()
    return J, g, dc, st


_DdmFunction = None
_ShapeFunction = None


def ddm_shape_functional(ctx, clm, h, prm, log_kappa, gamma, functional=FUNC_DRAG):
    """Differentiable J(log(kappa), gamma, c_lm) on a STAR surface (torch.autograd);
    clm is a (25,) float64 tensor."""
    global _ShapeFunction
    torch = _torch()
    if _ShapeFunction is None:
        class ShapeFunction(torch.autograd.Function):
            @staticmethod
            def forward(fctx, lk, gm, cl, c, h_, prm_, func):
                p2 = CDdmParams.from_buffer_copy(prm_)
                p2.kappa = float(np.exp(float(lk)))
                p2.gamma = float(gm)
                J, g, dc, _ = ddm_shape_gradient(c, cl.detach().cpu().numpy(), h_, p2, func)
                dev = lk.device
                fctx.save_for_backward(torch.tensor(g, dtype=torch.float64, device=dev),
                                       torch.tensor(dc, dtype=torch.float64, device=cl.device))
                return torch.tensor(J, dtype=torch.float64, device=dev)

            @staticmethod
            def backward(fctx, gout):
                g, dc = fctx.saved_tensors
                return gout * g[0], gout * g[1], gout * dc, None, None, None, None
        _ShapeFunction = ShapeFunction
    return _ShapeFunction.apply(log_kappa, gamma, clm, ctx, h, prm, functional)


def ddm_functional(ctx, pts, prm, log_kappa, gamma, functional=FUNC_DRAG):
    """Differentiable J(log(kappa), gamma) for torch.autograd.

    ``log_kappa`` and ``gamma`` are 0-d float64 tensors; the other parameters
    come from ``prm`` (left unchanged).  The backward pass uses the gradient
    that ssd_ddm_gradient computes together with J."""
    global _DdmFunction
    torch = _torch()
    if _DdmFunction is None:
        class DdmFunction(torch.autograd.Function):
            @staticmethod
            def forward(fctx, lk, gm, c, pts_, prm_, func):
                p2 = CDdmParams.from_buffer_copy(prm_)
                p2.kappa = float(np.exp(float(lk)))
                p2.gamma = float(gm)
                value, grad, _ = ddm_gradient(c, pts_, p2, func)
                fctx.save_for_backward(torch.tensor(grad, dtype=torch.float64, device=lk.device))
                return torch.tensor(value, dtype=torch.float64, device=lk.device)

            @staticmethod
            def backward(fctx, gout):
                (grad,) = fctx.saved_tensors
                return gout * grad[0], gout * grad[1], None, None, None, None
        _DdmFunction = DdmFunction
    return _DdmFunction.apply(log_kappa, gamma, ctx, pts, prm, functional)


class Batch:
    """Many surfaces in one launch: concatenated (3, n_total) point arrays with
    offsets[s] .. offsets[s+1] the points of surface s and one delta each."""

    def __init__(self, xyz, nrm, w, offsets, delta):
        torch = _torch()
        self.xyz = xyz.to(dtype=torch.float64).contiguous()
        self.nrm = nrm.to(dtype=torch.float64).contiguous()
        self.w = w.to(dtype=torch.float64).contiguous()
        self.offsets = (C.c_int64 * len(offsets))(*[int(v) for v in offsets])
        self.delta = (C.c_double * len(delta))(*[float(v) for v in delta])
        self.nsurf = len(delta)
        self.n = int(self.w.numel())
        if len(offsets) != self.nsurf + 1 or int(offsets[-1]) != self.n:
            raise ValueError("offsets must have nsurf + 1 entries ending at n_total")
        if self.xyz.shape != (3, self.n) or self.nrm.shape != (3, self.n):
            raise ValueError("xyz and nrm must have shape (3, n_total)")
        self.c = CBatch(self.nsurf, self.offsets, self.delta, _ptr(self.xyz), _ptr(self.nrm), _ptr(self.w), None)
        self.ctx = None

    @classmethod
    def from_numpy(cls, point_sets, deltas, device="cuda"):
        torch = _torch()
        offs = np.concatenate([[0], np.cumsum([p["w"].size for p in point_sets])])
        cat = lambda k: torch.as_tensor(np.ascontiguousarray(np.concatenate([p[k] for p in point_sets], axis=-1)),
                                        device=device)
        return cls(cat("xyz"), cat("nrm"), cat("w"), offs, deltas)

    def prepare(self, ctx):
        ctx.check(lib().ssd_batch_prepare(ctx.h, C.byref(self.c), _stream()), "ssd_batch_prepare")
        self.ctx = ctx
        return self

    def release(self):
        if self.ctx is not None and self.c.layout:
            lib().ssd_batch_release(self.ctx.h, C.byref(self.c))
        self.ctx = None


def batch_apply(ctx, batch, op, dens0, dens1=None, mu=1.0, alpha=1.0, beta=1.0, prec=FP64, out=None):
    """One launch of `op` for every surface and right-hand side; densities [nrhs][c][n_total]."""
    nrhs = int(dens0.shape[0])
    nc = _nc(op)
    if out is None:
        out = _torch().empty((nrhs, nc, batch.n), dtype=_torch().float64, device=dens0.device)
    m, dv = nrhs * nc * batch.n, batch.xyz.device
    ctx.check(lib().ssd_batch_apply(ctx.h, C.byref(batch.c), int(op), nrhs, float(mu), float(alpha), float(beta),
                                    _arg(dens0, m, dv, "dens0"), _arg(dens1, m, dv, "dens1"), _arg(out, m, dv, "out"),
                                    int(prec), _stream()), "ssd_batch_apply")
    return out


def batch_ddm_solve(ctx, batch, prm, uinf, raise_on_notconv=True):
    """D-N solves of every (surface, right-hand side); uinf is [nrhs][3]."""
    torch = _torch()
    uinf = np.asarray(uinf, dtype=np.float64).reshape(-1, 3)
    nrhs = uinf.shape[0]
    dev = batch.xyz.device
    o = {"q": torch.empty((nrhs, 1, batch.n), dtype=torch.float64, device=dev),
         "p": torch.empty((nrhs, 1, batch.n), dtype=torch.float64, device=dev),
         "u": torch.empty((nrhs, 3, batch.n), dtype=torch.float64, device=dev),
         "f": torch.empty((nrhs, 3, batch.n), dtype=torch.float64, device=dev)}
    drag = (C.c_double * (3 * nrhs * batch.nsurf))()
    its = (C.c_int * (nrhs * batch.nsurf))()
    rel = (C.c_double * (nrhs * batch.nsurf))()
    ui = (C.c_double * (3 * nrhs))(*uinf.ravel())
    st = lib().ssd_batch_ddm_solve(ctx.h, C.byref(batch.c), C.byref(prm), nrhs, ui, _ptr(o["q"]), _ptr(o["p"]),
                                   _ptr(o["u"]), _ptr(o["f"]), drag, its, rel, _stream())
    if st != SSD_ENOTCONV or raise_on_notconv:
        ctx.check(st, "ssd_batch_ddm_solve")
    o["drag"] = np.array(drag[:]).reshape(nrhs, batch.nsurf, 3)
    o["outer_its"] = np.array(its[:]).reshape(nrhs, batch.nsurf)
    o["relres"] = np.array(rel[:]).reshape(nrhs, batch.nsurf)
    o["status"] = st
    return o
