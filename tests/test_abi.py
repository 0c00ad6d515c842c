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

from tests.host_kernels import generated_source


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
    assert L.ls_abi_version() == 8


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


def test_new_entry_points_validate_their_arguments_without_a_device():
    """Argument checks that return before any CUDA call."""
    L = _abi.lib()
    e3 = (ctypes.c_int64 * 3)(8, 6, 4)
    buf_a, buf_b = ctypes.c_void_p(16), ctypes.c_void_p(32)            # never dereferenced: checks fail first
    CM, IL, BK = _abi.LS_LAYOUT_COSET_MAJOR, _abi.LS_LAYOUT_INTERLEAVED, _abi.LS_LAYOUT_BRICKED
    assert L.ls_relayout(buf_a, CM, buf_b, IL, 0, e3, 4, None) == 1            # no cosets
    assert L.ls_relayout(buf_a, CM, buf_b, IL, 9, e3, 4, None) == 1            # more than 8
    assert L.ls_relayout(buf_a, CM, buf_b, IL, 2, None, 4, None) == 1          # no extents
    assert L.ls_relayout(buf_a, CM, buf_b, IL, 2, e3, 3, None) == 1            # element size
    assert L.ls_relayout(buf_a, CM, buf_b, 7, 2, e3, 4, None) == 1             # layout
    assert L.ls_relayout(buf_a, CM, buf_a, IL, 2, e3, 4, None) == 1            # in place
    assert L.ls_relayout(None, CM, buf_b, IL, 2, e3, 4, None) == 1
    odd = (ctypes.c_int64 * 3)(7, 6, 4)                                         # 7 is odd: no whole bricks
    assert L.ls_relayout(buf_a, CM, buf_b, BK, 2, odd, 4, None) == 1
    assert b"brick" in L.ls_last_error()
    big = (ctypes.c_int64 * 3)(1 << 11, 1 << 11, 1 << 10)                     # 2^32 elements
    assert L.ls_relayout(buf_a, CM, buf_b, IL, 1, big, 4, None) == 3            # UNSUPPORTED
    assert L.ls_eval_hess(None, None, 0, None, None, None, None) == 1
    assert L.ls_volume_texture_sync(None, None) == 1
    assert L.ls_eval_linear_fetch(None, None, 0, None, None) == 1
    assert L.ls_spline_status(None, None) == 1
    assert L.ls_volume_layout(None) == -1
    assert L.ls_adjoint_coef(None, None, None, 0, None, 0, None, None) == 1


def test_variant_fields_reach_the_generated_code():
    """The layout, pipelining and warp-specialization variants change the
    generated kernels (and only the value kernel for the last two)."""
    import re
    from paper_2102_08518_b300 import api
    srcs = {}
    for tag, var in (("plain", {}), ("brick", {"brick": 1}), ("pipe", {"pipeline": 1}), ("ws", {"producers": 2}),
                     ("stage", {"stage": 1})):
        h = _abi.DescHolder(table("bcc_quintic"), api.kernel_name("bcc_quintic", "f32", **var))
        assert _abi.lib().ls_spline_precompile(ctypes.byref(h.desc), _abi.LS_F32,
                                               ctypes.byref(_abi.variant(**var))) == 0
        srcs[tag] = generated_source("bcc_quintic", **var)
    assert "BB0" in srcs["brick"] and "BB0" not in srcs["plain"]
    assert "P_c0" in srcs["pipe"] and "mbarrier.try_wait" in srcs["ws"]
    assert "cp.async.bulk.tensor.3d" in srcs["stage"] and "cp.async.bulk.tensor" not in srcs["plain"]
    def canon(src):
        # generated temporaries are numbered file-wide: renumber them in order of appearance
        names = {}
        return re.sub(r"\b(?:h|dA|hA|sh|w)\d+\b", lambda m: names.setdefault(m.group(0), f"t{len(names)}"), src)

    for tag in ("pipe", "ws", "stage"):                       # the other kernels are the plain ones
        suffix = {"pipe": "pp", "ws": "ws2", "stage": "st1"}[tag]
        for kern in ("ls_adjoint_atomic__", "ls_eval_hess__"):
            a = srcs["plain"][srcs["plain"].index(kern):].split("extern")[0]
            b = srcs[tag][srcs[tag].index(kern):].split("extern")[0]
            assert canon(a.replace("bcc_quintic_f32", "X")) == canon(b.replace(f"bcc_quintic_f32_{suffix}", "X"))


def test_stage_variant_is_validated_before_any_device_call():
    """The staged kernel is 3D, FP32, linear layouts, tile edge a multiple of 4
    with edge * cosets <= 256 (the TMA box) and at most 160 KiB of tile."""
    L = _abi.lib()
    for name, dt, var in (("fcc6", _abi.LS_F32, {"stage": 6}), ("fcc6", _abi.LS_BF16, {"stage": 1}),
                          ("bcc_quintic", _abi.LS_F32, {"stage": 1, "brick": 1}), ("zp", _abi.LS_F32, {"stage": 1}),
                          ("fcc6", _abi.LS_F32, {"stage": 80}), ("tricubic", _abi.LS_F32, {"stage": 36}),
                          ("bcc_quintic", _abi.LS_F32, {"stage": 1, "producers": 2})):
        h = _abi.DescHolder(table(name), "probe")
        out = ctypes.c_void_p()
        assert L.ls_spline_create(ctypes.byref(h.desc), dt, ctypes.byref(_abi.variant(**var)), ctypes.byref(out)) == 1
        assert b"stage" in L.ls_last_error() or b"3D" in L.ls_last_error() or b"FP32" in L.ls_last_error()


def test_tensor_variant_is_validated_before_any_device_call():
    """The tensor-core value kernel needs a non-separable table and excludes the
    other value-kernel variants."""
    L = _abi.lib()
    for name, var in (("tricubic", {"tensor": 1}), ("trilinear", {"tensor": 1}),
                      ("bcc_quintic", {"tensor": 1, "stage": 1}), ("fcc6", {"tensor": 1, "producers": 2}),
                      ("bcc_quintic", {"tensor": 1, "pts_per_thread": 4}), ("bcc_quintic", {"tensor_kind": 1}),
                      ("fcc6", {"tensor": 1, "tensor_kind": 2})):
        h = _abi.DescHolder(table(name), "probe")
        out = ctypes.c_void_p()
        assert L.ls_spline_create(ctypes.byref(h.desc), _abi.LS_F32, ctypes.byref(_abi.variant(**var)),
                                  ctypes.byref(out)) == 1
        assert b"tensor" in L.ls_last_error()
    # the FP16 form is for FP32 coefficients (BF16 / FP16 data are exact in TF32)
    h = _abi.DescHolder(table("fcc6"), "probe")
    out = ctypes.c_void_p()
    assert L.ls_spline_create(ctypes.byref(h.desc), _abi.LS_BF16, ctypes.byref(_abi.variant(tensor=1, tensor_kind=1)),
                              ctypes.byref(out)) == 1
    assert b"tensor_kind" in L.ls_last_error()


def test_tensor_variant_source():
    """The generated value kernel issues tcgen05 products from tensor memory and
    keeps the transform matrix as TF32 hi / lo pairs."""
    import re
    from paper_2102_08518_b300 import api
    var = {"tensor": 1}
    name = api.kernel_name("bcc_quintic", "f32", **var)
    h = _abi.DescHolder(table("bcc_quintic"), name)
    assert _abi.lib().ls_spline_precompile(ctypes.byref(h.desc), _abi.LS_F32, ctypes.byref(_abi.variant(**var))) == 0
    src = generated_source("bcc_quintic", **var)
    kern = src[src.index("ls_eval__"):]
    assert "tcgen05.mma.cta_group::1.kind::tf32" in kern and "tcgen05.alloc" in kern and "tcgen05.dealloc" in kern
    # the value and the value + gradient kernels: 3 products x K = 32 in steps of 8 each
    assert kern.count("tcgen05.mma.cta_group::1.kind::tf32") == 24
    # the table's hi / lo entries: every hi is a TF32 value (low 13 mantissa bits zero)
    import struct
    tab = src[src.index("ls_tcB_"):]
    vals = re.findall(r"(-?0x[0-9a-fA-F.p+-]+f|0\.0f)", tab[:tab.index("};")])
    half = len(vals) // 2
    for v in vals[:half]:
        f = float.fromhex(v[:-1]) if v != "0.0f" else 0.0
        bits = struct.unpack("<I", struct.pack("<f", f))[0]
        assert bits & 0x1FFF == 0


def _tensor_source(name, **var):
    import re
    from paper_2102_08518_b300 import api
    kn = api.kernel_name(name, "f32", **var)
    h = _abi.DescHolder(table(name), kn)
    assert _abi.lib().ls_spline_precompile(ctypes.byref(h.desc), _abi.LS_F32, ctypes.byref(_abi.variant(**var))) == 0
    return generated_source(name, **var)


def _table_entries(src):
    import re
    tab = src[src.index("ls_tcB_"):]
    m = re.match(r"ls_tcB_\w+\[(\d+)\] = \{", tab)
    body = tab[m.end():tab.index("};")]
    return int(m.group(1)), [v.strip() for v in body.replace("\n", " ").split(",") if v.strip()]


@pytest.mark.parametrize("name", ["bcc_quintic", "fcc6"])
def test_tensor_fp16_form_source(name):
    """The FP16 form: kind::f16 products in K steps of 16, and a transform
    table of FP16 hi / lo pairs that is the TF32 form's matrix scaled by one
    power of two (largest entry in [2^14, 2^15)), to 21 significant bits."""
    import numpy as np
    src32 = _tensor_source(name, tensor=1)
    src16 = _tensor_source(name, tensor=1, tensor_kind=1)
    kern = src16[src16.index("ls_eval__"):]
    assert "kind::tf32" not in kern
    n32, v32 = _table_entries(src32)
    n16, v16 = _table_entries(src16)
    f32 = np.array([float.fromhex(v[:-1]) if v != "0.0f" else 0.0 for v in v32])
    b16 = np.array([int(v) for v in v16], dtype=np.uint16).view(np.float16).astype(np.float64)
    # K (padded to 16 here, to 8 in the TF32 form) from the product count: 3 products x 2 kernels x K / 16
    kp = kern.count("tcgen05.mma.cta_group::1.kind::f16") // 6 * 16
    assert kp > 0 and (n16 // 2) % kp == 0
    N = n16 // 2 // kp
    kp32 = n32 // 2 // N
    assert kp32 * N * 2 == n32 and kp - 16 < kp32 <= kp
    m32 = np.zeros((N, kp))
    m16 = np.zeros((N, kp))
    for idx in range(N * kp32):
        g, r = divmod(idx, 8 * kp32)
        m32[g * 8 + (r % 32) // 4, (r // 32) * 4 + r % 4] += f32[idx] + f32[N * kp32 + idx]
    for idx in range(N * kp):
        g, r = divmod(idx, 8 * kp)
        m16[g * 8 + (r % 64) // 8, (r // 64) * 8 + r % 8] += b16[idx] + b16[N * kp + idx]
    scale = np.abs(m16).max() / np.abs(m32).max()
    assert 2.0 ** np.round(np.log2(scale)) == pytest.approx(scale, rel=1e-5)
    scale = 2.0 ** np.round(np.log2(scale))
    assert 2.0 ** 14 <= np.abs(m16).max() < 2.0 ** 15
    assert np.max(np.abs(m16 / scale - m32) / np.maximum(np.abs(m32), 1e-30)) < 2.0 ** -20
    assert np.array_equal(m16 == 0, m32 == 0)


def test_tensor_kernel_readback_and_union_zeroing_in_source():
    """Generated-source checks of two tensor-core kernel details.
    (1) Past 5 slots a large spline reads its 48 products back in 8-column
    pieces, each with its own wait; at 5 slots all at once, with one wait.
    (2) With two reference regions (FCC) the union sites outside the point's
    region are zeroed before staging, in both forms; a single-region spline
    has nothing to zero."""
    import re

    def eval_kernel(src, name):
        i = src.index("ls_eval__" + name + "(")
        return src[i:src.index("ls_eval_grad__", i)]

    from paper_2102_08518_b300 import api
    q6 = _tensor_source("bcc_quintic", tensor=6, tensor_kind=1)
    q5 = _tensor_source("bcc_quintic", tensor=1, tensor_kind=1)
    k6 = eval_kernel(q6, api.kernel_name("bcc_quintic", "f32", tensor=6, tensor_kind=1))
    k5 = eval_kernel(q5, api.kernel_name("bcc_quintic", "f32", tensor=1, tensor_kind=1))
    assert "__launch_bounds__(768, 1)" in q6 and "__launch_bounds__(640, 1)" in q5
    assert k6.count("tcgen05.ld.sync.aligned.32x32b.x8.b32") == 6 and k6.count("tcgen05.wait::ld") == 6
    assert k5.count("tcgen05.wait::ld") == 1
    assert len(re.findall(r"if \(tpsi != \d\) tc\d+ = 0\.0f;", k5)) == 0
    for kw in ({"tensor": 1}, {"tensor": 1, "tensor_kind": 1}):
        f = _tensor_source("fcc6", **kw)
        kf = eval_kernel(f, api.kernel_name("fcc6", "f32", **kw))
        assert len(re.findall(r"if \(tpsi != \d\) tc\d+ = 0\.0f;", kf)) > 0


def test_generate_source_sizes_and_truncates():
    """ls_spline_generate_source: a NULL buffer reports the length; a short
    buffer gets a NUL-terminated prefix; NULL len is rejected; the text is
    the same on every call and names the variant's kernels."""
    from paper_2102_08518_b300 import api
    L = _abi.lib()
    kn = api.kernel_name("bcc_linear", "f32", block=512)
    h = _abi.DescHolder(table("bcc_linear"), kn)
    var = _abi.variant(block=512)
    n = ctypes.c_size_t(0)
    assert L.ls_spline_generate_source(ctypes.byref(h.desc), _abi.LS_F32, ctypes.byref(var), None, 0,
                                       ctypes.byref(n)) == 0
    assert n.value > 1000
    full = generated_source("bcc_linear", block=512)
    assert len(full) == n.value and f"ls_eval__{kn}(" in full
    buf = ctypes.create_string_buffer(17)
    m = ctypes.c_size_t(0)
    assert L.ls_spline_generate_source(ctypes.byref(h.desc), _abi.LS_F32, ctypes.byref(var), buf, 17,
                                       ctypes.byref(m)) == 0
    assert m.value == n.value and buf.value.decode() == full[:16]
    assert L.ls_spline_generate_source(ctypes.byref(h.desc), _abi.LS_F32, ctypes.byref(var), None, 0, None) != 0
