"""The algorithmic-traffic model of the benchmark's roofline (roofline.py).

Its stencil indices for the interleaved and bricked layouts must be the
coset-major indices moved by the layout maps (checked here against numpy
reshapes, independently of the library), and the distinct-sector counts must
follow from them.
"""
import numpy as np
import pytest

import workloads
from paper_2102_08518_b300.api import table
from paper_2102_08518_b300.roofline import distinct_sectors_per_point, stencil_indices

from tests.host_kernels import generated_source


def _maps(C, ext):
    """Element index of every coset-major element in the interleaved and bricked layouts."""
    P = int(np.prod(ext))
    cm = np.arange(C * P).reshape(C, *reversed(ext))            # (C, E2, E1, E0)
    il = np.empty(C * P, np.int64)
    il[np.ascontiguousarray(cm.reshape(C, -1).T).ravel()] = np.arange(C * P)
    e0, e1, e2 = ext
    bk_order = np.ascontiguousarray(cm.reshape(C, e2 // 2, 2, e1 // 2, 2, e0 // 2, 2)
                                    .transpose(1, 3, 5, 2, 4, 6, 0)).ravel()
    bk = np.empty(C * P, np.int64)
    bk[bk_order] = np.arange(C * P)
    return il, bk


@pytest.mark.parametrize("name", ["bcc_quintic", "fcc6", "tricubic"])
def test_layout_indices_follow_the_layout_maps(name):
    ext = (8, 6, 10)
    lat = workloads.SPLINE_LATTICE[name]
    C = len(workloads.LATTICES[lat][2])
    lo, hi = workloads.bounding_box(lat, ext)
    pts = workloads.points_uniform(300, lo - 1.0, hi + 1.0, seed=7)
    t = table(name)
    cm = stencil_indices(t, ext, pts, "coset")
    il_map, bk_map = _maps(C, ext)
    for layout, mp in (("interleaved", il_map), ("bricked", bk_map)):
        got = stencil_indices(t, ext, pts, layout)
        assert np.array_equal(got >= 0, cm >= 0)
        assert np.array_equal(got[cm >= 0], mp[cm[cm >= 0]])


def test_distinct_sectors_of_the_benchmark_layouts():
    """BCC quintic, 2 x 128^3: interleaving the cosets lowers the distinct
    32-byte sectors of a stencil; a single-coset spline is unchanged."""
    ext = (128, 128, 128)
    pts = workloads.points_uniform(4096, *workloads.inner_box("bcc_quintic", ext), seed=1)
    q = table("bcc_quintic")
    a = distinct_sectors_per_point(q, ext, pts, layout="coset")
    b = distinct_sectors_per_point(q, ext, pts, layout="interleaved")
    assert 16.5 < a < 18.0 and 12.0 < b < 13.5
    ptc = workloads.points_uniform(4096, *workloads.inner_box("tricubic", ext), seed=2)
    tc = table("tricubic")
    assert distinct_sectors_per_point(tc, ext, ptc, layout="coset") == \
        distinct_sectors_per_point(tc, ext, ptc, layout="interleaved")


def test_tensor_shape_matches_the_generated_kernel():
    """K and N of the transform product against the generated tensor-core
    kernel's shared-memory table (2 N K floats: TF32 hi and lo)."""
    import ctypes
    import os
    import re
    from paper_2102_08518_b300 import _abi, api
    from paper_2102_08518_b300.roofline import tensor_shape
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    for name in ("bcc_quintic", "fcc6", "bcc_linear"):
        K, N, nnz = tensor_shape(api.table(name))
        kn = api.kernel_name(name, "f32", tensor=1)
        h = _abi.DescHolder(api.table(name), kn)
        assert _abi.lib().ls_spline_precompile(ctypes.byref(h.desc), _abi.LS_F32,
                                               ctypes.byref(_abi.variant(tensor=1))) == 0
        src = generated_source(name, tensor=1)
        m = re.search(r"float ls_sB\[(\d+)\]", src)
        assert int(m.group(1)) == 2 * N * K, name
        assert K % 8 == 0 and N % 16 == 0 and nnz <= K * N


def test_tensor_shape_of_the_fp16_form():
    """The FP16 form pads K to 16: its table holds 2 N K FP16 values (hi, lo)."""
    import ctypes
    import os
    import re
    from paper_2102_08518_b300 import _abi, api
    from paper_2102_08518_b300.roofline import tensor_shape
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    for name in ("bcc_quintic", "fcc6"):
        K, N, nnz = tensor_shape(api.table(name), kstep=16)
        kn = api.kernel_name(name, "f32", tensor=1, tensor_kind=1)
        h = _abi.DescHolder(api.table(name), kn)
        assert _abi.lib().ls_spline_precompile(ctypes.byref(h.desc), _abi.LS_F32,
                                               ctypes.byref(_abi.variant(tensor=1, tensor_kind=1))) == 0
        src = generated_source(name, tensor=1, tensor_kind=1)
        m = re.search(r"unsigned short ls_tcB_\w+\[(\d+)\]", src)
        assert int(m.group(1)) == 2 * N * K and K % 16 == 0, name


def test_link_schedule_of_the_end_to_end_step():
    """The host-link bound of the bench's end-to-end step: both directions at
    the duplex rate while the smaller flow lasts, the rest alone; with one
    flow empty it is that flow at its own rate, and with equal flows both
    finish together at the duplex rate."""
    import bench
    GB = 1e9
    assert bench.link_schedule_ms(10 * GB, 0, 50.0, 60.0, 30.0) == pytest.approx(200.0)
    assert bench.link_schedule_ms(0, 6 * GB, 50.0, 60.0, 30.0) == pytest.approx(100.0)
    assert bench.link_schedule_ms(3 * GB, 3 * GB, 50.0, 60.0, 30.0) == pytest.approx(100.0)
    # the step: 402 MB in, 268 MB out at the measured 55.3 / 57.2 / 37.4 GB/s
    ms = bench.link_schedule_ms(402653184, 268435456, 55.3, 57.2, 37.4)
    assert ms == pytest.approx(268435456 / 37.4e6 + (402653184 - 268435456) / 55.3e6)
    assert 9.5 < ms < 9.7
