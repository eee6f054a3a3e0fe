"""The C-ABI library on the host: it loads, exports every declared symbol, and
rejects bad arguments before touching CUDA (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_1905_02803_gb300 import build as lib_build
from paper_1905_02803_gb300 import p3dfft as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "p3dfft_gb300.h")


@pytest.fixture(scope="module")
def lib():
    lib_build.build()
    return P.load()


def _gpu_present():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(p3_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("p3_plan_create", "p3_plan_destroy", "p3_ftran_r2c", "p3_btran_c2r", "p3_plan_get_dims",
                 "p3_plan_workspace_bytes", "p3_plan_scale", "p3_status_string"):
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert set(declared_symbols()) == set(P.EXPORTS)


def test_version_and_status_strings(lib):
    assert P.p3_version() == 1
    assert P.p3_status_string(P.P3_OK) == "ok"
    assert P.p3_status_string(P.P3_ERR_WORKSPACE) == "workspace required"
    assert P.p3_status_string(99) == "unknown status"


FFT3 = (P.P3_FFT, P.P3_FFT, P.P3_FFT)


@pytest.mark.parametrize("args,expect", [
    ((0, 8, 8, P.P3_F32, FFT3, P.P3_LAYOUT_ZYX, 0), P.P3_ERR_INVALID),
    ((8, -1, 8, P.P3_F32, FFT3, P.P3_LAYOUT_ZYX, 0), P.P3_ERR_INVALID),
    ((8, 8, 8, 7, FFT3, P.P3_LAYOUT_ZYX, 0), P.P3_ERR_INVALID),
    ((8, 8, 8, P.P3_F32, FFT3, 5, 0), P.P3_ERR_INVALID),
    ((8, 8, 8, P.P3_F32, FFT3, P.P3_LAYOUT_ZYX, 32), P.P3_ERR_INVALID),
    ((8, 8, 8, P.P3_F32, FFT3, P.P3_LAYOUT_ZYX, P.P3_FLAG_PADDED_REAL), P.P3_ERR_UNSUPPORTED),
    ((8, 8, 8, P.P3_F32, (P.P3_FFT, P.P3_FFT, 9), P.P3_LAYOUT_ZYX, 0), P.P3_ERR_INVALID),
    ((8, 8, 1, P.P3_F64, (P.P3_FFT, P.P3_FFT, P.P3_CHEB), P.P3_LAYOUT_ZYX, 0), P.P3_ERR_INVALID),
    ((8, 8, 8, P.P3_F32, (P.P3_EMPTY, P.P3_FFT, P.P3_FFT), P.P3_LAYOUT_ZYX, 0), P.P3_ERR_UNSUPPORTED),
    ((8, 8, 8, P.P3_F32, (P.P3_FFT, P.P3_CHEB, P.P3_FFT), P.P3_LAYOUT_ZYX, 0), P.P3_ERR_UNSUPPORTED),
    ((8, 8, 8, P.P3_F32, (P.P3_FFT, P.P3_SINE, P.P3_FFT), P.P3_LAYOUT_ZYX, 0), P.P3_ERR_UNSUPPORTED),
    ((8, 8, 8, P.P3_F32, (P.P3_FFT, P.P3_FFT, 4), P.P3_LAYOUT_ZYX, 0), P.P3_ERR_INVALID),
    ((8, 8, 2047 + 2048, P.P3_F32, (P.P3_FFT, P.P3_FFT, P.P3_SINE), P.P3_LAYOUT_ZYX, 0), P.P3_ERR_UNSUPPORTED),
    ((8, 8192, 8, P.P3_F32, FFT3, P.P3_LAYOUT_ZYX, 0), P.P3_ERR_UNSUPPORTED),
    ((8, 8, 2053, P.P3_F32, FFT3, P.P3_LAYOUT_ZYX, 0), P.P3_ERR_UNSUPPORTED),   # prime > 2048
    ((2 * 4099, 8, 8, P.P3_F32, FFT3, P.P3_LAYOUT_ZYX, 0), P.P3_ERR_UNSUPPORTED),
    # extended third-dimension lengths 2(Nz - 1) / 2(Nz + 1) beyond int range
    ((8, 8, 2 ** 31 - 1, P.P3_F32, (P.P3_FFT, P.P3_FFT, P.P3_SINE), P.P3_LAYOUT_ZYX, 0), P.P3_ERR_UNSUPPORTED),
    ((8, 8, 2 ** 31 - 1, P.P3_F64, (P.P3_FFT, P.P3_FFT, P.P3_CHEB), P.P3_LAYOUT_XYZ, 0), P.P3_ERR_UNSUPPORTED),
    ((8, 8, 2 ** 30 + 1, P.P3_F64, (P.P3_FFT, P.P3_FFT, P.P3_CHEB), P.P3_LAYOUT_ZYX, 0), P.P3_ERR_UNSUPPORTED),
    ((8, 8, 2 ** 31 - 1, P.P3_F32, FFT3, P.P3_LAYOUT_ZYX, 0), P.P3_ERR_UNSUPPORTED),
    ((2 ** 31 - 1, 8, 8, P.P3_F32, FFT3, P.P3_LAYOUT_ZYX, 0), P.P3_ERR_UNSUPPORTED),
])
def test_plan_create_rejects_before_cuda(lib, args, expect):
    st, h = P.p3_plan_create(*args, check=False)
    assert st == expect and h is None


def test_plan_create_null_pointers(lib):
    tt = (ctypes.c_int * 3)(0, 0, 0)
    assert lib.p3_plan_create(None, 8, 8, 8, 0, tt, 0, 0) == P.P3_ERR_INVALID
    h = ctypes.c_void_p()
    assert lib.p3_plan_create(ctypes.byref(h), 8, 8, 8, 0, None, 0, 0) == P.P3_ERR_INVALID


@pytest.mark.skipif(_gpu_present(), reason="checks the no-device error path")
def test_plan_create_without_device_reports_cuda_error(lib):
    st, h = P.p3_plan_create(8, 8, 8, P.P3_F32, FFT3, P.P3_LAYOUT_ZYX, check=False)
    assert st == P.P3_ERR_CUDA and h is None


def test_null_plan_calls(lib):
    assert lib.p3_plan_destroy(None) == P.P3_OK
    assert lib.p3_ftran_r2c(None, None, None, None, None) == P.P3_ERR_INVALID
    assert lib.p3_btran_c2r(None, None, None, None, None) == P.P3_ERR_INVALID
    a = (ctypes.c_int * 3)()
    assert lib.p3_plan_get_dims(None, a, a) == P.P3_ERR_INVALID
    v = ctypes.c_size_t()
    assert lib.p3_plan_workspace_bytes(None, ctypes.byref(v)) == P.P3_ERR_INVALID
    d = ctypes.c_double()
    assert lib.p3_plan_scale(None, ctypes.byref(d)) == P.P3_ERR_INVALID
    assert lib.p3_plan_describe(None, ctypes.create_string_buffer(8), 8) == P.P3_ERR_INVALID
    n = ctypes.c_int()
    assert lib.p3_plan_launches(None, 0, ctypes.byref(n)) == P.P3_ERR_INVALID
    assert lib.p3_plan_set_stage_events(None, None, 0) == P.P3_ERR_INVALID
    assert P.p3_plan_set_z_hook(None, P.Z_HOOK(lambda *a: 0), check=False) == P.P3_ERR_INVALID
    assert P.p3_status_string(P.P3_ERR_HOOK) == "user Z hook failed"
    assert P.p3_plan_wait_status(None) == P.P3_ERR_INVALID
    f = ctypes.c_uint(7)
    assert lib.p3_plan_wait_flags(None, ctypes.byref(f)) == P.P3_ERR_INVALID
    assert P.p3_plan_set_wait_limits(None, 10, 0, check=False) == P.P3_ERR_INVALID
    assert P.p3_plan_set_fused_lag(None, 1, check=False) == P.P3_ERR_INVALID
    st, h = P.p3_batch_create(None, 2, check=False)
    assert st == P.P3_ERR_INVALID and h is None
    st, h = P.p3_batch_create([None], 2, check=False)
    assert st == P.P3_ERR_INVALID and h is None
    assert P.p3_batch_destroy(None) == P.P3_OK
    assert P.p3_batch_ftran_r2c(None, None, None, None, None, check=False) == P.P3_ERR_INVALID
    assert P.p3_batch_btran_c2r(None, None, None, None, None, check=False) == P.P3_ERR_INVALID
    assert P.p3_batch_wait_status(None) == P.P3_ERR_INVALID
    assert P.p3_batch_set_wait_limits(None, 10, 0, check=False) == P.P3_ERR_INVALID
    assert lib.p3_batch_launches(None, 0, ctypes.byref(n)) == P.P3_ERR_INVALID
    st, h = P.p3_batch_create(None, -1, check=False)
    assert st == P.P3_ERR_INVALID and h is None


def test_binding_raises_when_library_missing(tmp_path, monkeypatch):
    monkeypatch.setattr(P, "_lib", None)
    monkeypatch.setattr(P, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        P.load()
