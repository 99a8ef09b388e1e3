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
