"""ctypes binding of the FP64 oracle library built from ``orc.c`` (test infrastructure)."""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field
from typing import Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "orc.c")
_LIB = os.path.join(_HERE, "liborc.so")

MAXDIR = 16
MAXCOSET = 8


class _CSpec(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int32),
        ("kind", ctypes.c_int32),
        ("ndir", ctypes.c_int32),
        ("pad0", ctypes.c_int32),
        ("dirs", ctypes.c_double * (MAXDIR * 3)),
        ("detL", ctypes.c_double),
        ("scale", ctypes.c_int32),
        ("ncoset", ctypes.c_int32),
        ("coset", ctypes.c_int32 * (MAXCOSET * 3)),
        ("ext", ctypes.c_int64 * 3),
    ]


@dataclass
class OrcSpec:
    """A spline on a lattice as the oracle sees it.

    dirs: columns of Xi (m x dim); kind 1 selects the closed-form tensor-product
    cubic B-spline instead of the box-spline recurrence.  Sites are stored as
    Cartesian cosets: site = scale*i + coset[j], one array of extent ``ext`` per
    coset, coset-major, axis 0 fastest.
    """
    dim: int
    dirs: Sequence[Sequence[float]]
    detL: float
    scale: int = 1
    cosets: Sequence[Sequence[int]] = ((0, 0, 0),)
    ext: Sequence[int] = (1, 1, 1)
    kind: int = 0
    name: str = ""

    def with_extent(self, ext) -> "OrcSpec":
        e = list(ext) + [1] * (3 - len(ext))
        return OrcSpec(self.dim, self.dirs, self.detL, self.scale, self.cosets, tuple(e),
                       self.kind, self.name)

    def n_coef(self) -> int:
        n = 1
        for i in range(self.dim):
            n *= int(self.ext[i])
        return n * len(self.cosets)

    def to_c(self) -> _CSpec:
        c = _CSpec()
        c.dim = self.dim
        c.kind = self.kind
        c.ndir = len(self.dirs)
        if c.ndir > MAXDIR or len(self.cosets) > MAXCOSET:
            raise ValueError("too many directions or cosets for the oracle")
        for j, d in enumerate(self.dirs):
            for i in range(self.dim):
                c.dirs[3 * j + i] = float(d[i])
        c.detL = float(self.detL)
        c.scale = int(self.scale)
        c.ncoset = len(self.cosets)
        for j, l in enumerate(self.cosets):
            for i in range(self.dim):
                c.coset[3 * j + i] = int(l[i])
        for i in range(3):
            c.ext[i] = int(self.ext[i]) if i < len(self.ext) else 1
        return c


def library_path() -> str:
    return _LIB


def build_library(force: bool = False) -> str:
    """Compile ``orc.c`` into ``liborc.so`` (gcc, -O2, OpenMP, no fast-math)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
           "-ffp-contract=off", "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def configure(lib):
    """Set the ctypes signatures on a loaded oracle library (also used on
    deliberately broken copies in the mutation tests)."""
    dp = ctypes.POINTER(ctypes.c_double)
    sp = ctypes.POINTER(_CSpec)
    i64p = ctypes.POINTER(ctypes.c_int64)
    lib.orc_box.restype = ctypes.c_double
    lib.orc_box.argtypes = [ctypes.c_int32, ctypes.c_int32, dp, dp]
    lib.orc_phi.restype = ctypes.c_int32
    lib.orc_phi.argtypes = [sp, dp, ctypes.c_int64, dp, dp]
    lib.orc_eval.restype = ctypes.c_int32
    lib.orc_eval.argtypes = [sp, dp, dp, ctypes.c_int64, dp, dp, ctypes.c_int32]
    lib.orc_adjoint.restype = ctypes.c_int32
    lib.orc_adjoint.argtypes = [sp, dp, dp, ctypes.c_int64, dp]
    lib.orc_design_triplets.restype = ctypes.c_int64
    lib.orc_design_triplets.argtypes = [sp, dp, ctypes.c_int64, i64p, i64p, dp, ctypes.c_int64]
    lib.orc_morton3.restype = ctypes.c_uint32
    lib.orc_morton3.argtypes = [ctypes.c_uint32] * 3
    lib.orc_phi_hess.restype = ctypes.c_int32
    lib.orc_phi_hess.argtypes = [sp, dp, ctypes.c_int64, dp]
    lib.orc_eval_hess.restype = ctypes.c_int32
    lib.orc_eval_hess.argtypes = [sp, dp, dp, ctypes.c_int64, dp, ctypes.c_int32]
    return lib


def _load():
    global _lib
    if _lib is None:
        build_library()
        _lib = configure(ctypes.CDLL(_LIB))
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def box(dirs, x) -> float:
    """M_Xi(x): the (uncentred, unnormalised) box spline with columns ``dirs``."""
    d = _f64(dirs)
    k = d.shape[1] if d.size else len(x)
    cols = np.zeros((MAXDIR, 3))
    cols[: d.shape[0], :k] = d
    xx = np.zeros(3)
    xx[:k] = np.asarray(x, dtype=np.float64)
    return float(_load().orc_box(k, d.shape[0], _dptr(cols), _dptr(xx)))


def phi(spec: OrcSpec, y) -> np.ndarray:
    """Centred basis function phi at points y (n x dim)."""
    y = _f64(y).reshape(-1, spec.dim)
    out = np.zeros(len(y))
    cs = spec.to_c()
    if _load().orc_phi(ctypes.byref(cs), _dptr(y), len(y), _dptr(out), None) != 0:
        raise RuntimeError("orc_phi failed")
    return out


def phi_grad(spec: OrcSpec, y):
    y = _f64(y).reshape(-1, spec.dim)
    out = np.zeros(len(y))
    g = np.zeros((len(y), spec.dim))
    cs = spec.to_c()
    if _load().orc_phi(ctypes.byref(cs), _dptr(y), len(y), _dptr(out), _dptr(g)) != 0:
        raise RuntimeError("orc_phi failed")
    return out, g


def _is_voronoi(spec) -> bool:
    return type(spec).__name__ == "VoronoiSpec"


def eval_sum(spec: OrcSpec, coef, pts, nthreads: int = 0) -> np.ndarray:
    """Naive convolution sum (Eq. 1) at points pts (n x dim) in FP64 (Voronoi
    splines: oracle.voronoi)."""
    if _is_voronoi(spec):
        from . import voronoi
        return voronoi.eval_sum(spec, coef, pts)
    c = _f64(coef).ravel()
    if c.size != spec.n_coef():
        raise ValueError(f"coef has {c.size} values, spec wants {spec.n_coef()}")
    p = _f64(pts).reshape(-1, spec.dim)
    out = np.zeros(len(p))
    cs = spec.to_c()
    if _load().orc_eval(ctypes.byref(cs), _dptr(c), _dptr(p), len(p), _dptr(out), None,
                        nthreads) != 0:
        raise RuntimeError("orc_eval failed")
    return out


def eval_sum_grad(spec: OrcSpec, coef, pts, nthreads: int = 0):
    """f and grad f (n x dim) of the naive convolution sum in FP64."""
    if _is_voronoi(spec):
        from . import voronoi
        return voronoi.eval_sum_grad(spec, coef, pts)
    c = _f64(coef).ravel()
    p = _f64(pts).reshape(-1, spec.dim)
    out = np.zeros(len(p))
    g = np.zeros((len(p), spec.dim))
    cs = spec.to_c()
    if _load().orc_eval(ctypes.byref(cs), _dptr(c), _dptr(p), len(p), _dptr(out), _dptr(g),
                        nthreads) != 0:
        raise RuntimeError("orc_eval failed")
    return out, g


def _hess_width(dim: int) -> int:
    return 6 if dim == 3 else 3


def phi_hess(spec: OrcSpec, y) -> np.ndarray:
    """Hessian of phi at points y: (n, 6) as xx yy zz xy xz yz in 3D, (n, 3) as xx yy xy in 2D."""
    y = _f64(y).reshape(-1, spec.dim)
    h = np.zeros((len(y), _hess_width(spec.dim)))
    cs = spec.to_c()
    if _load().orc_phi_hess(ctypes.byref(cs), _dptr(y), len(y), _dptr(h)) != 0:
        raise RuntimeError("orc_phi_hess failed")
    return h


def eval_sum_hess(spec: OrcSpec, coef, pts, nthreads: int = 0) -> np.ndarray:
    """Hessian of the naive convolution sum (same layout as phi_hess)."""
    c = _f64(coef).ravel()
    p = _f64(pts).reshape(-1, spec.dim)
    h = np.zeros((len(p), _hess_width(spec.dim)))
    cs = spec.to_c()
    if _load().orc_eval_hess(ctypes.byref(cs), _dptr(c), _dptr(p), len(p), _dptr(h), nthreads) != 0:
        raise RuntimeError("orc_eval_hess failed")
    return h


def adjoint(spec: OrcSpec, pts, g) -> np.ndarray:
    """dc_n = sum_p g_p phi(x_p - n), same layout as the coefficients."""
    if _is_voronoi(spec):
        from . import voronoi
        return voronoi.adjoint(spec, pts, g)
    p = _f64(pts).reshape(-1, spec.dim)
    gg = _f64(g).ravel()
    dc = np.zeros(spec.n_coef())
    cs = spec.to_c()
    if _load().orc_adjoint(ctypes.byref(cs), _dptr(p), _dptr(gg), len(p), _dptr(dc)) != 0:
        raise RuntimeError("orc_adjoint failed")
    return dc


def design_triplets(spec: OrcSpec, pts):
    """(rows, cols, vals) of A[p, n] = phi(x_p - n)."""
    p = _f64(pts).reshape(-1, spec.dim)
    cs = spec.to_c()
    cap = max(16, len(p) * 64)
    while True:
        rows = np.zeros(cap, dtype=np.int64)
        cols = np.zeros(cap, dtype=np.int64)
        vals = np.zeros(cap)
        n = _load().orc_design_triplets(
            ctypes.byref(cs), _dptr(p), len(p),
            rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
            cols.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dptr(vals), cap)
        if n < 0:
            raise RuntimeError("orc_design_triplets failed")
        if n <= cap:
            return rows[:n], cols[:n], vals[:n]
        cap = int(n)


def morton3(c0: int, c1: int, c2: int) -> int:
    return int(_load().orc_morton3(c0, c1, c2))
