"""The C ABI library loads and exports every entry point that include/ssd.h
declares; calls with invalid arguments fail cleanly before any GPU work.
No GPU is needed."""
import ctypes
import os
import re

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "ssd.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ssd_[A-Za-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2110_10749_gb300 import build
    build.build()
    import paper_2110_10749_gb300 as ssd
    return ssd.lib()


def test_header_and_binding_agree():
    import paper_2110_10749_gb300 as ssd
    assert declared_symbols() == sorted(ssd.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_null_context_is_rejected(lib):
    import paper_2110_10749_gb300 as ssd
    P = ctypes.c_void_p
    assert lib.ssd_laplace_SL(None, None, 1.0, None, None, 0, None) == ssd.SSD_EINVAL
    assert lib.ssd_stokes_DL(None, None, 1.0, None, None, 0, None) == ssd.SSD_EINVAL
    assert lib.ssd_ddm_solve(None, None, None, None, None, None, None, None, None, None, None, None) == ssd.SSD_EINVAL
    assert lib.ssd_ctx_set_timing(None, 1) == ssd.SSD_EINVAL
    assert lib.ssd_ctx_destroy(None) == ssd.SSD_OK
    assert lib.ssd_status_string(ssd.SSD_ENOTCONV) == b"iteration limit reached"


def test_context_creation_without_device_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = lib.ssd_ctx_create(ctypes.byref(h), 0)
    assert st != 0 and not h.value


def test_python_api_refuses_to_run_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2110_10749_gb300 as ssd
    with pytest.raises(RuntimeError):
        ssd.Context(0)


def test_host_buffer_marshalling():
    """ddm_solve_host's host buffers: inputs are converted to contiguous
    float64 (and kept alive), outputs must already be writable contiguous
    float64 of the right shape, CPU tensors are taken as they are."""
    import numpy as np
    import torch
    import paper_2110_10749_gb300 as ssd
    n = 5
    a = np.arange(3 * n, dtype=np.float32).reshape(n, 3).T      # non-contiguous float32 input
    p, keep = ssd._host_ptr(a, (3, n))
    assert keep.dtype == np.float64 and keep.flags.c_contiguous and np.array_equal(keep, a)
    assert p.value == keep.ctypes.data
    with pytest.raises(ValueError):
        ssd._host_ptr(np.zeros(n + 1), (n,))
    out = np.empty((3, n))
    p, keep = ssd._host_ptr(out, (3, n), writable=True)
    assert keep is out and p.value == out.ctypes.data
    for bad in (np.empty((3, n), dtype=np.float32), np.empty((n, 3)).T, np.empty(n)):
        with pytest.raises(ValueError):
            ssd._host_ptr(bad, (3, n), writable=True)
    t = torch.zeros((3, n), dtype=torch.float64)
    p, keep = ssd._host_ptr(t, (3, n), writable=True)
    assert keep is t and p.value == t.data_ptr()
    with pytest.raises(ValueError):
        ssd._host_ptr(torch.zeros((3, n), dtype=torch.float32), (3, n))


def test_device_array_size_and_device_checks():
    """The binding checks each device array's element count (the C calls
    cannot) and its device before passing a pointer."""
    import torch
    import paper_2110_10749_gb300 as ssd
    cpu = torch.device("cpu")
    ssd._check_arg(torch.zeros((3, 7)), 21, cpu, "u")
    ssd._check_arg(torch.zeros(21), 21, cpu, "u")          # any shape with the right count
    ssd._check_arg(None, 21, cpu, "optional")
    with pytest.raises(ValueError, match="expected 21 elements"):
        ssd._check_arg(torch.zeros((3, 6)), 21, cpu, "u")
    with pytest.raises(ValueError, match="points are on"):
        ssd._check_arg(torch.zeros(4), 4, torch.device("meta"), "g")
    assert ssd._nc(ssd.OP_LAPLACE_DL) == 1 and ssd._nc(ssd.OP_LAPLACE_SLDL) == 1
    assert ssd._nc(ssd.OP_STOKES_SL) == 3 and ssd._nc(ssd.OP_STOKES_SLDL) == 3


def test_status_strings_and_null_handles(lib):
    """Host-only entry points: every status code has its text, unknown codes
    a fallback; NULL handles are refused (or accepted where documented)."""
    import paper_2110_10749_gb300 as ssd
    texts = {ssd.SSD_OK: b"ok", ssd.SSD_EINVAL: b"invalid argument", ssd.SSD_ENOMEM: b"out of memory",
             ssd.SSD_ECUDA: b"CUDA error", ssd.SSD_ENOTCONV: b"iteration limit reached",
             ssd.SSD_ENUMERIC: b"non-finite value"}
    for st, text in texts.items():
        assert lib.ssd_status_string(st) == text
    assert lib.ssd_status_string(99) == b"unknown status"
    assert lib.ssd_status_string(-1) == b"unknown status"
    assert lib.ssd_ctx_last_error(None) == b""
    assert lib.ssd_ctx_create(None, 0) == ssd.SSD_EINVAL
    n = ctypes.c_int64()
    assert lib.ssd_ctx_launch_count(None, ctypes.byref(n)) == ssd.SSD_EINVAL
    assert lib.ssd_ctx_reset_stats(None) == ssd.SSD_EINVAL
    assert lib.ssd_points_release(None, None) == ssd.SSD_EINVAL
    assert lib.ssd_batch_release(None, None) == ssd.SSD_EINVAL
