"""The Python binding's marshalling, run on the CPU against a recording
stand-in for the library: every wrapper passes the pointers of the arrays it
was given (or allocated) in the order the C declaration expects, with the
sizes the checks demand; wrong sizes are refused before any call."""
import ctypes

import numpy as np
import pytest
import torch


class Recorder:
    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        if not name.startswith("ssd_"):
            raise AttributeError(name)

        def fn(*args):
            self.calls.append((name, args))
            return 0
        return fn


@pytest.fixture
def fake(monkeypatch):
    import paper_2110_10749_gb300 as ssd
    rec = Recorder()
    monkeypatch.setattr(ssd, "lib", lambda: rec)
    monkeypatch.setattr(ssd, "_torch", lambda: torch)
    monkeypatch.setattr(ssd, "_stream", lambda: None)

    def ptr(t):
        if t is None:
            return None
        assert t.dtype == torch.float64 and t.is_contiguous()
        return ctypes.c_void_p(t.data_ptr())
    monkeypatch.setattr(ssd, "_ptr", ptr)

    class Ctx:
        h = None
        device = 0

        def check(self, st, what):
            assert st == 0, what
    pts = type("P", (), {})()
    n = 10
    pts.n = n
    pts.xyz = torch.zeros((3, n), dtype=torch.float64)
    pts.c = ssd.CPoints(n, None, None, None, None)
    return ssd, rec, Ctx(), pts


def _p(t):
    return t.data_ptr()


def test_operators_pass_their_arrays(fake):
    ssd, rec, ctx, pts = fake
    n = pts.n
    g = torch.randn(n, dtype=torch.float64)
    v = torch.randn((3, n), dtype=torch.float64)
    v2 = torch.randn((3, n), dtype=torch.float64)
    out = ssd.laplace_SL(ctx, pts, 0.1, g, ssd.FP32C)
    name, a = rec.calls[-1]
    assert name == "ssd_laplace_SL" and a[3].value == _p(g) and a[4].value == _p(out) and a[5] == ssd.FP32C
    out = ssd.stokes_SLDL(ctx, pts, 0.1, 2.0, v2, v, 0.5, -1.0, ssd.FP64)
    name, a = rec.calls[-1]
    assert name == "ssd_stokes_SLDL" and a[4].value == _p(v2) and a[5].value == _p(v)
    assert (a[6], a[7]) == (0.5, -1.0) and a[8].value == _p(out) and out.shape == (3, n)
    out = ssd.apply_rows(ctx, pts, ssd.OP_STOKES_DL, 0.1, v, 2, 7, mu=1.5, prec=ssd.FP32C)
    name, a = rec.calls[-1]
    assert name == "ssd_apply_rows" and a[2] == ssd.OP_STOKES_DL and a[4] == 1.5 and a[5].value == _p(v)
    assert (a[6], a[7]) == (2, 7) and a[8].value == _p(out) and a[9] == ssd.FP32C and out.shape == (3, n)
    with pytest.raises(ValueError):
        ssd.apply_rows(ctx, pts, ssd.OP_LAPLACE_DL, 0.1, v, 0, 3)
    order = ssd.points_order(ctx, pts)
    assert rec.calls[-1][0] == "ssd_points_order" and order.shape == (n,) and order.dtype == np.int32
    out = ssd.apply_transpose(ctx, pts, ssd.OP_LAPLACE_DL, 0.1, g)
    assert rec.calls[-1][0] == "ssd_apply_transpose" and out.shape == (n,)
    ssd.apply_transpose(ctx, pts, ssd.OP_STOKES_DL, 0.1, v)
    for call, arg in ((ssd.laplace_DL, v), (ssd.stokes_DL, g)):
        with pytest.raises(ValueError):
            call(ctx, pts, 0.1, arg)
    with pytest.raises(ValueError):
        ssd.apply_transpose(ctx, pts, ssd.OP_STOKES_SL, 0.1, g)
    with pytest.raises(ValueError):
        ssd.laplace_SL(ctx, pts, 0.1, g, out=torch.empty(n + 1, dtype=torch.float64))


def test_solves_fields_and_gradients_pass_their_arrays(fake):
    ssd, rec, ctx, pts = fake
    n = pts.n
    q = torch.randn(n, dtype=torch.float64)
    f = torch.randn((3, n), dtype=torch.float64)
    p, its, rel = ssd.darcy_solve(ctx, pts, 0.1, 1.0, 1.0, q)
    name, a = rec.calls[-1]
    assert name == "ssd_darcy_solve" and a[5].value == _p(q) and a[6].value == _p(p)
    u, _, _ = ssd.stokes_solve(ctx, pts, 0.1, 1.0, f, (0.0, 0.0, 1.0))
    name, a = rec.calls[-1]
    assert name == "ssd_stokes_solve" and a[4].value == _p(f) and list(a[5]) == [0.0, 0.0, 1.0]
    assert a[6].value == _p(u)
    prm = ssd.ddm_params(kappa=1e-2, gamma=1.0)
    o = ssd.ddm_sweep(ctx, pts, prm, q, f)
    name, a = rec.calls[-1]
    assert name == "ssd_ddm_sweep" and a[3].value == _p(q) and a[4].value == _p(f)
    assert a[5].value == _p(o["q"]) and a[6].value == _p(o["p"]) and a[7].value == _p(o["u"])
    assert a[8].value == _p(o["f"]) and o["u"].shape == (3, n)
    o = ssd.ddm_sweep(ctx, pts, prm, q)
    assert rec.calls[-1][1][4] is None
    with pytest.raises(ValueError):
        ssd.ddm_sweep(ctx, pts, prm, q, q)
    tg = torch.randn((3, 4), dtype=torch.float64)
    out = ssd.darcy_pressure_field(ctx, pts, 1.0, 0.5, q, q, tg)
    name, a = rec.calls[-1]
    assert name == "ssd_darcy_pressure_field" and a[6] == 4 and a[7].value == _p(tg) and out.shape == (4,)
    out = ssd.stokes_velocity_field(ctx, pts, 1.0, (0, 0, 1), f, f, tg)
    name, a = rec.calls[-1]
    assert name == "ssd_stokes_velocity_field" and a[6] == 4 and out.shape == (3, 4)
    with pytest.raises(ValueError):
        ssd.stokes_velocity_field(ctx, pts, 1.0, (0, 0, 1), q, f, tg)
    gx, gn, gw = ssd.geometry_gradient(ctx, pts, ssd.OP_STOKES_DL, 0.1, f, f)
    name, a = rec.calls[-1]
    assert name == "ssd_geometry_gradient" and a[8].value == _p(gx) and a[10].value == _p(gw)
    with pytest.raises(ValueError):
        ssd.geometry_gradient(ctx, pts, ssd.OP_LAPLACE_SL, 0.1, f, f)
    jac = {"dxyz": torch.zeros((25, 3, n), dtype=torch.float64), "dnrm": torch.zeros((25, 3, n), dtype=torch.float64),
           "dw": torch.zeros((25, n), dtype=torch.float64)}
    dc = ssd.shape_contract(ctx, jac, (gx, gn, gw))
    name, a = rec.calls[-1]
    assert name == "ssd_shape_contract" and a[1] == n and a[2] == 25 and dc.shape == (25,)


def test_batch_apply_passes_its_arrays(fake):
    ssd, rec, ctx, pts = fake
    b = type("B", (), {})()
    b.n = 12
    b.xyz = torch.zeros((3, b.n), dtype=torch.float64)
    b.c = ssd.CBatch(0, None, None, None, None, None, None)
    d0 = torch.randn((2, 3, b.n), dtype=torch.float64)
    d1 = torch.randn((2, 3, b.n), dtype=torch.float64)
    out = ssd.batch_apply(ctx, b, ssd.OP_STOKES_SLDL, d0, d1, alpha=0.5, beta=2.0)
    name, a = rec.calls[-1]
    assert name == "ssd_batch_apply" and a[3] == 2 and a[7].value == _p(d0) and a[8].value == _p(d1)
    assert out.shape == (2, 3, b.n) and a[9].value == _p(out)
    with pytest.raises(ValueError):
        ssd.batch_apply(ctx, b, ssd.OP_LAPLACE_DL, d0)


def test_host_solve_marshals_host_buffers(fake):
    ssd, rec, ctx, pts = fake
    n = 6
    xyz = np.random.default_rng(1).normal(size=(3, n))
    prm = ssd.ddm_params(maxit_outer=4)
    r = ssd.ddm_solve_host(ctx, xyz, xyz, np.ones(n), prm)
    name, a = rec.calls[-1]
    assert name == "ssd_ddm_solve_host" and a[1] == n
    assert a[6].value == r["q"].ctypes.data and a[9].value == r["f"].ctypes.data
    with pytest.raises(ValueError):
        ssd.ddm_solve_host(ctx, xyz[:, :n - 1], xyz, np.ones(n), prm)
