"""Generated point functions compiled for the host (test helper only).

The generator emits one CUDA C++ point function per spline and variant
(ls_eval_pt__*, ls_eval_grad_pt__*, ls_eval_hess_pt__*).  Their arithmetic is
plain C++ (fmaf, rintf, selects, integer address arithmetic) around a few
device intrinsics, so with host stand-ins for those intrinsics the same text
compiles with g++ and runs on the CPU.  The tests use this to check the
generator's arithmetic and addressing (every layout, every variant that keeps
the point function) against the FP64 oracle without a GPU.  The GPU parity
tests still check the compiled kernels themselves.  Not part of the product.
"""
import ctypes
import hashlib
import os
import subprocess
import tempfile

import numpy as np

from paper_2102_08518_b300 import _abi, api

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BUILD = os.path.join(tempfile.gettempdir(), "ls_host_kernels")

SHIM = r"""
#include <math.h>
#include <cstring>
#include <cstddef>
#define __device__
#define __forceinline__ inline
#define __restrict__
static inline void ls_ld8(const float* p, float& r0, float& r1, float& r2, float& r3, float& r4, float& r5,
                          float& r6, float& r7) { r0 = p[0]; r1 = p[1]; r2 = p[2]; r3 = p[3]; r4 = p[4]; r5 = p[5];
                                                  r6 = p[6]; r7 = p[7]; }
template <class T> static inline T __ldg(const T* p) { return *p; }
static inline float __int_as_float(int v) { float f; std::memcpy(&f, &v, 4); return f; }
static inline float __uint_as_float(unsigned v) { float f; std::memcpy(&f, &v, 4); return f; }
static inline int __float_as_int(float v) { int i; std::memcpy(&i, &v, 4); return i; }
static inline unsigned __float_as_uint(float v) { unsigned i; std::memcpy(&i, &v, 4); return i; }
static inline int __float2int_rz(float v) { return v != v ? 0 : (int)v; }
static inline int __float2int_rn(float v) { return v != v ? 0 : (int)rintf(v); }
static inline float __ldcs(const float* p) { return *p; }
static inline void __stcs(float* p, float v) { *p = v; }
static inline float ls_ldk_f32(const float* p) { return *p; }
#define __constant__
struct float2 { float x, y; };
static inline float2 make_float2(float a, float b) { float2 r; r.x = a; r.y = b; return r; }
static inline float2 __ffma2_rn(float2 a, float2 b, float2 c) { return make_float2(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y)); }
static inline float2 __fmul2_rn(float2 a, float2 b) { return make_float2(a.x * b.x, a.y * b.y); }
static inline unsigned short ls_ldk_u16(const unsigned short* p) { return *p; }

"""


def generated_source(name: str, dtype: str = "f32", expansion: str = "sparse", **var) -> str:
    """Source of the kernels of spline `name` with variant `var`, as the
    generator emits it (ls_spline_generate_source: host only, no device)."""
    kn = api.kernel_name(name, dtype, expansion=expansion, **var)
    h = _abi.DescHolder(api.table(name), kn, expansion)
    L = _abi.lib()
    vr = _abi.variant(**var)
    n = ctypes.c_size_t(0)
    rc = L.ls_spline_generate_source(ctypes.byref(h.desc), api.DTYPES[dtype], ctypes.byref(vr), None, 0,
                                     ctypes.byref(n))
    assert rc == 0, L.ls_last_error()
    buf = ctypes.create_string_buffer(n.value + 1)
    rc = L.ls_spline_generate_source(ctypes.byref(h.desc), api.DTYPES[dtype], ctypes.byref(vr), buf, n.value + 1,
                                     ctypes.byref(n))
    assert rc == 0, L.ls_last_error()
    return buf.value.decode()


def _function(src: str, fname: str) -> str:
    i = src.index("static __device__ __forceinline__ void " + fname + "(")
    j = src.index("\n}\n", i)
    return src[i:j + 3]


class HostKernels:
    """The value, value + gradient and value + gradient + Hessian point
    functions of one generated spline variant, built for the host."""

    def __init__(self, name: str, dtype: str = "f32", expansion: str = "sparse", **var):
        src = generated_source(name, dtype, expansion, **var)
        tag = api.kernel_name(name, dtype, expansion=expansion, **var)
        lines = [ln for ln in src.splitlines() if ln.startswith(("typedef", "struct LsEvalArgs", "#define LS_CSWAP",
                                                                 "__constant__ float2 ls_K2_",
                                                                 "static __device__ __forceinline__ float ls_ld_pt",
                                                                 "static __device__ __forceinline__ void ls_st_out"))]
        loader = {"f32": "ls_ld_f32", "bf16": "ls_ld_bf16", "f16": "ls_ld_f16"}[dtype]
        ld = [ln for ln in src.splitlines() if ln.startswith("static __device__ __forceinline__ float " + loader + "(")]
        # kernels that load a thread's next point ahead (variant prefetch) take
        # the coordinates as arguments: the driver passes them
        D = api.table(name).spline.lattice.dim
        fn = {w: f"ls_{w}_pt__{tag}" + ("_x" if f"ls_{w}_pt__{tag}_x(" in src else "")
              for w in ("eval", "eval_grad", "eval_hess")}
        body = [_function(src, fn[w]) for w in ("eval", "eval_grad", "eval_hess")]

        def call(w):
            if fn[w].endswith("_x"):
                z = "pts[i * 3 + 2]" if D == 3 else "0.0f"
                return f"{fn[w]}(a, i, pts[i * {D}], pts[i * {D} + 1], {z})"
            return f"{fn[w]}(a, i)"
        drivers = "".join(
            f'extern "C" void host_{w}(const float* pts, long long n, float* out, float* grad, float* hess,'
            f' const void* coef, int e0, int e1, int e2, int cs, int cu) {{\n'
            f'  LsEvalArgs a; std::memset(&a, 0, sizeof a); a.pts = pts; a.out = out; a.grad = grad; a.hess = hess;'
            f' a.coef = coef; a.n = n; a.e0 = e0; a.e1 = e1; a.e2 = e2; a.cstride = cs; a.cunit = cu;\n'
            f'  for (long long i = 0; i < n; ++i) {call(w)};\n}}\n'
            for w in ("eval", "eval_grad", "eval_hess"))
        code = SHIM + "\n".join(lines + ld) + "\n" + "\n".join(body) + drivers
        if dtype == "f16":
            code = code.replace('asm("cvt.f32.f16 %0, %1;" : "=f"(f) : "h"(h));', "f = (float)(_Float16&)h;")
        os.makedirs(BUILD, exist_ok=True)
        key = hashlib.sha256(code.encode()).hexdigest()[:16]
        so = os.path.join(BUILD, f"{tag}_{key}.so")
        if not os.path.exists(so):
            cpp = so[:-3] + ".cpp"
            with open(cpp, "w") as f:
                f.write(code)
            tmp = so + f".tmp{os.getpid()}"
            subprocess.run(["g++", "-O1", "-ffp-contract=off", "-shared", "-fPIC", "-w", "-o", tmp, cpp], check=True)
            os.replace(tmp, so)
        self.lib = ctypes.CDLL(so)
        self.dim = api.table(name).spline.lattice.dim

    def _call(self, what, pts, coef, ext, layout, n_cosets, need_grad=False, need_hess=False):
        pts = np.ascontiguousarray(pts, dtype=np.float32)
        n = len(pts)
        D = self.dim
        out = np.zeros(n, np.float32)
        grad = np.zeros(n * D, np.float32) if need_grad else None
        nh = 6 if D == 3 else 3
        hess = np.zeros(n * nh, np.float32) if need_hess else None
        e = list(ext) + [1] * (3 - len(ext))
        P = int(np.prod(ext))
        copy = n_cosets * (e[0] + 2) * (e[1] + 2) * e[2]
        copy3 = n_cosets * (e[0] + 2) * (e[1] + 2) * (e[2] + 2)
        cs, cu = {"coset": (P, 1), "interleaved": (1, n_cosets), "bricked": (1, n_cosets),
                  "bricked_shifted": (copy, n_cosets), "bricked_shifted_xyz": (copy3, n_cosets)}[layout]
        coef = np.ascontiguousarray(coef)
        ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p) if a is not None else None
        fn = getattr(self.lib, "host_" + what)
        fn.argtypes = [ctypes.c_void_p, ctypes.c_longlong] + [ctypes.c_void_p] * 4 + [ctypes.c_int] * 5
        fn(ptr(pts), n, ptr(out), ptr(grad), ptr(hess), ptr(coef), e[0], e[1], e[2], cs, cu)
        return out, (grad.reshape(n, D) if need_grad else None), (hess.reshape(n, nh) if need_hess else None)

    def eval(self, pts, coef, ext, layout="coset", n_cosets=1):
        return self._call("eval", pts, coef, ext, layout, n_cosets)[0]

    def eval_grad(self, pts, coef, ext, layout="coset", n_cosets=1):
        f, g, _ = self._call("eval_grad", pts, coef, ext, layout, n_cosets, need_grad=True)
        return f, g

    def eval_hess(self, pts, coef, ext, layout="coset", n_cosets=1):
        return self._call("eval_hess", pts, coef, ext, layout, n_cosets, need_grad=True, need_hess=True)
