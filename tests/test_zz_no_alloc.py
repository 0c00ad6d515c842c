"""The allocation-free Morton sort (ls_morton_sort_noalloc) through the C ABI.

Callers that cannot allocate device memory while they run use this entry point;
it must give exactly what the allocating ls_morton_sort gives, call after call,
although every call reuses the same static scratch array.  This file is
collected last so that a stopping run has executed every other test first.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2102_08518_b300 import _abi

pytestmark = pytest.mark.gpu

MAX_POINTS = 1 << 18


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _sort(fn_name, pts, origin, cell):
    n = pts.shape[0]
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    keys = torch.empty(n, dtype=torch.int32, device="cuda")
    o = (ctypes.c_float * 3)(*origin)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    L = _abi.lib()
    if fn_name == "ls_morton_sort_noalloc":
        st = L.ls_morton_sort_noalloc(_ptr(pts), n, o, cell, _ptr(perm), _ptr(keys), stream)
    else:
        st = L.ls_morton_sort(_ptr(pts), n, o, cell, _ptr(perm), _ptr(keys), ctypes.c_void_p(0), stream)
    return st, perm, keys


@pytest.mark.parametrize("sizes", [(MAX_POINTS, 70001), (1, 4097)])
def test_noalloc_sort_equals_allocating_sort_on_consecutive_calls(sizes):
    rng = np.random.default_rng(sum(sizes))
    for call, n in enumerate(sizes):
        pts_np = rng.uniform(-3.0, 260.0, (n, 3)).astype(np.float32)
        pts_np[: n // 4] = np.round(pts_np[: n // 4])          # repeated keys: order must be stable
        pts = torch.from_numpy(pts_np).cuda()
        st_a, perm_a, keys_a = _sort("ls_morton_sort", pts, (0.0, 0.0, 0.0), 2.0)
        st_b, perm_b, keys_b = _sort("ls_morton_sort_noalloc", pts, (0.0, 0.0, 0.0), 2.0)
        torch.cuda.synchronize()
        assert st_a == 0 and st_b == 0, _abi.lib().ls_last_error().decode()
        assert torch.equal(perm_a, perm_b), f"call {call}"
        assert torch.equal(keys_a, keys_b), f"call {call}"


def _sort_no_keys(fn_name, pts, origin, cell):
    """keys_out = NULL: the noalloc sort then keeps the keys in its static
    scratch, beside the sort's own workspace."""
    n = pts.shape[0]
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    o = (ctypes.c_float * 3)(*origin)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    L = _abi.lib()
    if fn_name == "ls_morton_sort_noalloc":
        st = L.ls_morton_sort_noalloc(_ptr(pts), n, o, cell, _ptr(perm), ctypes.c_void_p(0), stream)
    else:
        st = L.ls_morton_sort(_ptr(pts), n, o, cell, _ptr(perm), ctypes.c_void_p(0), ctypes.c_void_p(0), stream)
    return st, perm


def test_noalloc_sort_without_keys_output_on_consecutive_calls():
    rng = np.random.default_rng(5)
    for call, n in enumerate((MAX_POINTS, 9001)):
        pts_np = rng.uniform(-3.0, 260.0, (n, 3)).astype(np.float32)
        pts_np[: n // 3] = np.round(pts_np[: n // 3])
        pts = torch.from_numpy(pts_np).cuda()
        st_a, perm_a = _sort_no_keys("ls_morton_sort", pts, (0.0, 0.0, 0.0), 2.0)
        st_b, perm_b = _sort_no_keys("ls_morton_sort_noalloc", pts, (0.0, 0.0, 0.0), 2.0)
        torch.cuda.synchronize()
        assert st_a == 0 and st_b == 0, _abi.lib().ls_last_error().decode()
        assert torch.equal(perm_a, perm_b), f"call {call}"


@pytest.mark.parametrize("cell", [float("inf"), float("nan"), 0.0, -1.0])
def test_noalloc_sort_rejects_what_the_allocating_sort_rejects(cell):
    pts = torch.zeros(16, 3, device="cuda")
    st_a, _, _ = _sort("ls_morton_sort", pts, (0.0, 0.0, 0.0), cell)
    st_b, _, _ = _sort("ls_morton_sort_noalloc", pts, (0.0, 0.0, 0.0), cell)
    assert st_a == 1 and st_b == 1                       # LS_ERR_INVALID_ARG from both


def test_noalloc_sort_rejects_more_than_its_maximum():
    pts = torch.zeros(MAX_POINTS + 1, 3, device="cuda")
    st, _, _ = _sort("ls_morton_sort_noalloc", pts, (0.0, 0.0, 0.0), 1.0)
    assert st == 1                                       # LS_ERR_INVALID_ARG
    assert b"262144" in _abi.lib().ls_last_error()
