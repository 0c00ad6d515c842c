"""The C ABI without a GPU: the library loads, exports every declared entry
point, generates and compiles (NVRTC, sm_103a) every spline, and rejects bad
descriptors with the documented status codes."""
import ctypes
import os
import re

import pytest

from paper_2102_08518_b300 import _abi
from paper_2102_08518_b300.api import table

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if not f.endswith(".h"):
            continue
        src = open(os.path.join(inc, f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(ls_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    L = _abi.lib()
    declared = _declared_functions()
    assert len(declared) >= 25
    for name in sorted(declared):
        assert hasattr(L, name), name
    # the Python binding covers the same names
    assert declared <= set(_abi.SIGNATURES)


def test_status_strings():
    L = _abi.lib()
    for code in range(9):
        assert L.ls_status_str(code)
    assert L.ls_abi_version() == 2


@pytest.mark.parametrize("name", ["tricubic", "bcc_linear", "bcc_quintic", "fcc6", "zp"])
@pytest.mark.parametrize("dtype", [_abi.LS_F32, _abi.LS_BF16, _abi.LS_F16])
def test_generated_kernels_compile_for_sm103a(name, dtype):
    h = _abi.DescHolder(table(name), f"{name}_t{dtype}")
    st = _abi.lib().ls_spline_precompile(ctypes.byref(h.desc), dtype, None)
    assert st == 0, _abi.lib().ls_last_error().decode()


def _desc(name="bcc_linear"):
    return _abi.DescHolder(table(name), "probe")


def _precompile(h):
    return _abi.lib().ls_spline_precompile(ctypes.byref(h.desc), _abi.LS_F32, None)


def test_rejects_bad_descriptors():
    L = _abi.lib()
    assert L.ls_spline_precompile(None, _abi.LS_F32, None) == 1        # INVALID_ARG
    h = _desc()
    h.desc.dim = 4
    assert _precompile(h) == 3                                         # UNSUPPORTED
    h = _desc()
    h.desc.scale = 3
    assert _precompile(h) == 3
    h = _desc()
    sig = (ctypes.c_int8 * 1)(5)                                       # sigma beyond n_ref
    h.desc.sigma = ctypes.cast(sig, ctypes.POINTER(ctypes.c_int8))
    assert _precompile(h) == 2                                         # BAD_TABLE
    h = _desc()
    off = (ctypes.c_int32 * 6)(0, 0, 0, 0, 0, 0)                       # duplicate coset
    h.desc.coset_offsets = ctypes.cast(off, _abi.c_i32p)
    assert _precompile(h) == 2
    h = _desc()
    h.desc.name = b"bad name!"
    assert _precompile(h) == 1
    h = _desc("fcc6")
    h.desc.n_planes = 0                                                 # K = 2 without planes
    assert _precompile(h) == 2
    h = _desc()
    h.desc.roe = _abi.LS_ROE_PARALLELEPIPED                             # scale 2 lattice
    assert _precompile(h) == 3
    assert L.ls_last_error()


def test_calls_with_null_handles_fail_cleanly():
    L = _abi.lib()
    assert L.ls_eval(None, None, 0, None, None) == 1
    assert L.ls_spline_destroy(None) == 0
    assert L.ls_volume_destroy(None) == 0
