"""ssd_stokes_DL_noalloc: the Stokes double layer for callers that cannot
allocate device memory (their memory is reserved by another allocator, or
they must not trigger the synchronisation of cudaFree).  Called through the
C ABI, twice in a row with different densities, and compared with the
allocating entry point ssd_stokes_DL within the FP32C tolerance of the
other operator tests, and with the FP64 oracle directly, up to the largest
point set it accepts.  Kept in its own file, collected last."""
import ctypes as C

import numpy as np
import pytest

import oracle
from oracle import quadrature as Q

pytestmark = pytest.mark.gpu


def _call(lib, ctx, P, delta, u, out):
    import torch
    return lib.ssd_stokes_DL_noalloc(ctx.h, C.byref(P.c), float(delta), C.c_void_p(u.data_ptr()),
                                     C.c_void_p(out.data_ptr()), C.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("h", [1 / 16, 1 / 32])
def test_no_alloc_matches_allocating_entry_point(gpu_ctx, h):
    import torch
    import paper_2110_10749_gb300 as ssd
    lib = ssd.lib()
    p = Q.sphere_points(1.0, h)
    P = ssd.Points.from_numpy(p)
    rng = np.random.default_rng(31)
    for call in range(2):   # two calls in a row share the scratch array
        u = torch.as_tensor(rng.normal(size=(3, P.n)), device="cuda")
        out = torch.empty_like(u)
        assert _call(lib, gpu_ctx, P, 3 * h, u, out) == ssd.SSD_OK
        ref = ssd.stokes_DL(gpu_ctx, P, 3 * h, u, ssd.FP32C)
        torch.cuda.synchronize()
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-5, call


def test_no_alloc_rejects_sizes_beyond_its_limit(gpu_ctx):
    import torch
    import paper_2110_10749_gb300 as ssd
    p = Q.sphere_points(1.0, 1 / 64)          # 68166 points > 32768
    P = ssd.Points.from_numpy(p)
    u = torch.zeros((3, P.n), dtype=torch.float64, device="cuda")
    out = torch.empty_like(u)
    assert _call(ssd.lib(), gpu_ctx, P, 3 / 64, u, out) == ssd.SSD_EINVAL


@pytest.mark.parametrize("hinv", [16, 44])
def test_no_alloc_matches_oracle(gpu_ctx, hinv):
    # h = 1/44: 32310 points, padded to 32768, the largest set the call
    # accepts; its partial sums fill the 16 splits of the scratch array
    import torch
    import paper_2110_10749_gb300 as ssd
    h = 1.0 / hinv
    p = Q.sphere_points(1.0, h)
    P = ssd.Points.from_numpy(p)
    rng = np.random.default_rng(7)
    rows = np.arange(0, P.n, 37)
    for call in range(2):
        un = rng.normal(size=(3, P.n))
        u = torch.as_tensor(un, device="cuda")
        out = torch.empty_like(u)
        assert _call(ssd.lib(), gpu_ctx, P, 3 * h, u, out) == ssd.SSD_OK
        torch.cuda.synchronize()
        ref = oracle.stokes_dl(p, 3 * h, un, rows=rows)
        a = out.cpu().numpy()[:, rows]
        assert np.linalg.norm(a - ref) / np.linalg.norm(ref) < 1e-5, call
        assert np.abs(a - ref).max() < 1e-5 * np.abs(ref).max(), call
