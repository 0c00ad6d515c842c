"""Failure detection without a GPU fault.

* A bounded device wait that runs out: the warp-specialized value kernel with
  its failure hook (wait_probe = 1: the producer warps never signal their
  slots, a flag that nothing sets) and a short wait limit.  Every consumer
  wait gives up, sets the spline's status word and returns; the kernel ends,
  ls_spline_status reports LS_ERR_TIMEOUT once (and clears the word), the
  outputs stay unwritten, and the next launches on the same device are clean.
  The kernel holds no tensor memory.
* Host-side allocation failures (ls_debug_fail_alloc): every device
  allocation a call makes is failed in turn; the call returns LS_ERR_OOM and
  the library holds no more device allocations than before it.
"""
import ctypes

import numpy as np
import pytest
import torch

import workloads
from paper_2102_08518_b300 import _abi
from paper_2102_08518_b300.api import Spline, Volume

from tests.test_gpu_eval import SMALL_EXT, TOL, oracle_eval

pytestmark = pytest.mark.gpu


def _case(name="bcc_quintic", n=5000):
    lat = workloads.SPLINE_LATTICE[name]
    ext = SMALL_EXT[name]
    coef = workloads.coef_uniform(lat, ext, seed=31)
    lo, hi = workloads.bounding_box(lat, ext)
    pts = workloads.points_uniform(n, lo, hi, seed=32)
    return ext, coef, pts


def test_bounded_wait_runs_out():
    ext, coef, pts = _case()
    c = torch.from_numpy(coef).cuda()
    p = torch.from_numpy(pts).cuda()
    probe = Spline("bcc_quintic", "f32", block=256, producers=2, wait_limit=64, wait_probe=1)
    vol = Volume(probe, ext, c)
    out = torch.full((len(pts),), 12345.0, device="cuda")
    vol.eval(p, out)
    torch.cuda.synchronize()                         # the kernel returned
    st = _abi.lib().ls_spline_status(probe.handle, None)
    assert st == _abi.LS_ERR_TIMEOUT
    assert _abi.lib().ls_spline_status(probe.handle, None) == 0       # reading it cleared the word
    assert bool(torch.all(out == 12345.0))          # consumers gave up before writing anything
    # the same device keeps working: the warp-specialized kernel with normal
    # waits, and the default kernel, both give the oracle's values
    want = oracle_eval("bcc_quintic", ext, coef, pts)
    cmax = float(np.abs(coef).max())
    for sp in (Spline("bcc_quintic", "f32", block=256, producers=2), Spline("bcc_quintic", "f32")):
        got = Volume(sp, ext, c).eval(p).cpu().numpy().astype(np.float64)
        sp.status()
        assert np.max(np.abs(got - want)) <= TOL * cmax


def test_wait_probe_needs_warp_specialized_kernel():
    with pytest.raises(RuntimeError, match="wait_probe"):
        Spline("bcc_quintic", "f32", wait_probe=1)


def _each_allocation_fails(call, max_allocs=12):
    """Fail the k-th device allocation of call() for k = 0, 1, ... until the
    call succeeds; each failing call must return LS_ERR_OOM and leave the
    library's live allocations as they were."""
    L = _abi.lib()
    failures = 0
    for k in range(max_allocs):
        before = L.ls_debug_live_allocs()
        L.ls_debug_fail_alloc(k)
        try:
            st = call()
        finally:
            L.ls_debug_fail_alloc(-1)
        torch.cuda.synchronize()
        if st == 0:
            return failures
        assert st == _abi.LS_ERR_OOM, (k, st, L.ls_last_error())
        assert L.ls_debug_live_allocs() == before, k
        failures += 1
    raise AssertionError("call never succeeded")


def test_allocation_failures_leak_nothing():
    L = _abi.lib()
    ext, coef, pts = _case(n=3000)
    sp = Spline("bcc_quintic", "f32")
    c = torch.from_numpy(coef).cuda()
    p = torch.from_numpy(pts).cuda()
    handles = []

    def spline_create():
        h = ctypes.c_void_p()
        st = L.ls_spline_create(ctypes.byref(sp._desc.desc), _abi.LS_F32, None, ctypes.byref(h))
        if st == 0:
            handles.append(("s", h))
        return st

    def volume_create():
        h = ctypes.c_void_p()
        e3 = (ctypes.c_int64 * 3)(*ext)
        st = L.ls_volume_create(sp.handle, e3, _abi.LS_LAYOUT_COSET_MAJOR, ctypes.byref(h))
        if st == 0:
            handles.append(("v", h))
        return st

    assert _each_allocation_fails(spline_create) >= 1
    assert _each_allocation_fails(volume_create) >= 1
    vol = Volume(sp, ext, c)
    host = torch.from_numpy(pts).pin_memory()
    hout = torch.empty(len(pts)).pin_memory()
    # staging of the host-buffer path; scratch of the deterministic adjoints
    # and of the Morton sort (none kept between calls)
    assert _each_allocation_fails(lambda: L.ls_eval_host(vol.handle, ctypes.c_void_p(host.data_ptr()), len(pts),
                                                          ctypes.c_void_p(hout.data_ptr()), None)) >= 1
    g = torch.ones(len(pts), device="cuda")
    dc = torch.zeros_like(c)
    for mode in (_abi.LS_ADJ_DETERMINISTIC_FIXED, _abi.LS_ADJ_DETERMINISTIC):
        assert _each_allocation_fails(lambda: L.ls_adjoint_coef(vol.handle, ctypes.c_void_p(p.data_ptr()),
                                                                ctypes.c_void_p(g.data_ptr()), len(pts),
                                                                ctypes.c_void_p(dc.data_ptr()), mode, None,
                                                                None)) >= 1
    perm = torch.empty(len(pts), dtype=torch.int32, device="cuda")
    origin = (ctypes.c_float * 3)(0.0, 0.0, 0.0)
    assert _each_allocation_fails(lambda: L.ls_morton_sort(ctypes.c_void_p(p.data_ptr()), len(pts), origin,
                                                           ctypes.c_float(1.0), ctypes.c_void_p(perm.data_ptr()),
                                                           None, None, None)) >= 1
    # results after the failures are the oracle's
    want = oracle_eval("bcc_quintic", ext, coef, pts)
    assert np.max(np.abs(hout.numpy() - want)) <= TOL * float(np.abs(coef).max())
    for kind, h in handles:
        (L.ls_volume_destroy if kind == "v" else L.ls_spline_destroy)(h)
