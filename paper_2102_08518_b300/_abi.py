"""ctypes binding of libls.so: the C ABI of include/lattice_spline.h, same names.

Argument marshalling only; every step of the computation runs in the
library's kernels.  Loading fails loudly when the library is missing.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libls.so")

# ls_status
LS_OK = 0
STATUS_NAMES = {0: "LS_OK", 1: "LS_ERR_INVALID_ARG", 2: "LS_ERR_BAD_TABLE", 3: "LS_ERR_UNSUPPORTED",
                4: "LS_ERR_OOM", 5: "LS_ERR_CUDA", 6: "LS_ERR_COMPILE", 7: "LS_ERR_TIMEOUT",
                8: "LS_ERR_DEVICE"}
(LS_ERR_INVALID_ARG, LS_ERR_BAD_TABLE, LS_ERR_UNSUPPORTED, LS_ERR_OOM, LS_ERR_CUDA, LS_ERR_COMPILE, LS_ERR_TIMEOUT,
 LS_ERR_DEVICE) = range(1, 9)
# ls_dtype
LS_F32, LS_BF16, LS_F16, LS_F64 = 0, 1, 2, 3
# ls_roe / ls_fold
LS_ROE_PARALLELEPIPED, LS_ROE_VORONOI = 0, 1
LS_FOLD_NONE, LS_FOLD_SIGNED_PERM = 0, 1
# ls_layout
LS_LAYOUT_COSET_MAJOR, LS_LAYOUT_INTERLEAVED, LS_LAYOUT_BRICKED, LS_LAYOUT_BRICKED_SHIFTED = 0, 1, 2, 3
LS_LAYOUT_BRICKED_SHIFTED_XYZ = 4
# ls_adjoint_mode
LS_ADJ_ATOMIC, LS_ADJ_DETERMINISTIC, LS_ADJ_ATOMIC_WARP, LS_ADJ_DETERMINISTIC_FIXED = 0, 1, 2, 3
LS_ADJ_ATOMIC_TILED, LS_ADJ_DETERMINISTIC_FIXED_TILED = 4, 5

c_i32p = ctypes.POINTER(ctypes.c_int32)
c_i64p = ctypes.POINTER(ctypes.c_int64)
c_f64p = ctypes.POINTER(ctypes.c_double)
c_f32p = ctypes.POINTER(ctypes.c_float)
c_u32p = ctypes.POINTER(ctypes.c_uint32)


class RefRegionC(ctypes.Structure):
    _fields_ = [("n_sites", ctypes.c_int32), ("sites", c_i32p), ("n_monos", ctypes.c_int32),
                ("mono_exp", c_i32p), ("coef", c_f64p), ("center", ctypes.c_double * 3)]


class AxisFactorC(ctypes.Structure):
    _fields_ = [("n_sites", ctypes.c_int32), ("sites", c_i32p), ("degree", ctypes.c_int32),
                ("coef", c_f64p), ("center", ctypes.c_double)]


class SplineDescC(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("dim", ctypes.c_int32), ("roe", ctypes.c_int32),
                ("fold", ctypes.c_int32), ("scale", ctypes.c_int32), ("generator", ctypes.c_double * 9),
                ("n_cosets", ctypes.c_int32), ("coset_offsets", c_i32p), ("n_planes", ctypes.c_int32),
                ("planes", c_f64p), ("bsp_mod", ctypes.c_int32), ("sigma", ctypes.POINTER(ctypes.c_int8)),
                ("n_ref", ctypes.c_int32), ("ref", ctypes.POINTER(RefRegionC)),
                ("separable", ctypes.POINTER(AxisFactorC))]


class VariantC(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int32), ("pts_per_thread", ctypes.c_int32), ("branchy", ctypes.c_int32),
                ("min_blocks", ctypes.c_int32), ("group", ctypes.c_int32), ("depth", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("brick", ctypes.c_int32), ("pipeline", ctypes.c_int32),
                ("producers", ctypes.c_int32), ("stage", ctypes.c_int32), ("tensor", ctypes.c_int32),
                ("tensor_kind", ctypes.c_int32), ("plain_transform", ctypes.c_int32),
                ("wait_limit", ctypes.c_int32), ("wait_probe", ctypes.c_int32), ("prefetch", ctypes.c_int32),
                ("l2_keep", ctypes.c_int32), ("fma2", ctypes.c_int32)]


# name -> (restype, argtypes); every function declared in include/lattice_spline.h
SIGNATURES = {
    "ls_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "ls_last_error": (ctypes.c_char_p, []),
    "ls_abi_version": (ctypes.c_int32, []),
    "ls_debug_fail_alloc": (None, [ctypes.c_int32]),
    "ls_debug_live_allocs": (ctypes.c_int64, []),
    "ls_spline_create": (ctypes.c_int, [ctypes.POINTER(SplineDescC), ctypes.c_int, ctypes.POINTER(VariantC),
                                        ctypes.POINTER(ctypes.c_void_p)]),
    "ls_spline_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "ls_spline_precompile": (ctypes.c_int, [ctypes.POINTER(SplineDescC), ctypes.c_int, ctypes.POINTER(VariantC)]),
    "ls_spline_source": (ctypes.c_char_p, [ctypes.c_void_p]),
    "ls_spline_generate_source": (ctypes.c_int, [ctypes.POINTER(SplineDescC), ctypes.c_int, ctypes.POINTER(VariantC),
                                                 ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
    "ls_spline_status": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "ls_spline_info": (ctypes.c_int, [ctypes.c_void_p, c_i32p, c_i32p, c_i32p, c_i32p]),
    "ls_volume_create": (ctypes.c_int, [ctypes.c_void_p, c_i64p, ctypes.c_int32, ctypes.POINTER(ctypes.c_void_p)]),
    "ls_volume_wrap": (ctypes.c_int, [ctypes.c_void_p, c_i64p, ctypes.c_int32, ctypes.c_void_p,
                                      ctypes.POINTER(ctypes.c_void_p)]),
    "ls_volume_layout": (ctypes.c_int32, [ctypes.c_void_p]),
    "ls_relayout": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                   c_i64p, ctypes.c_int32, ctypes.c_void_p]),
    "ls_volume_upload": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int,
                                        ctypes.c_void_p]),
    "ls_volume_device_ptr": (ctypes.c_void_p, [ctypes.c_void_p]),
    "ls_volume_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "ls_eval": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]),
    "ls_eval_grad": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p]),
    "ls_eval_hess": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "ls_volume_texture_sync": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "ls_eval_linear_fetch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                            ctypes.c_void_p]),
    "ls_eval_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                    ctypes.c_void_p]),
    "ls_eval_host_multi": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p,
                                          ctypes.c_int64, ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p]),
    "ls_adjoint_coef": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                       ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    "ls_adjoint_scratch_bytes": (ctypes.c_size_t, [ctypes.c_void_p, ctypes.c_int64]),
    "ls_morton_sort": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_float,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "ls_morton_sort_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_float,
                                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "ls_morton_scratch_bytes": (ctypes.c_size_t, [ctypes.c_int64]),
    "ls_permute_rows": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                       ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    "ls_probe_gather": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p,
                                       ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p]),
    "ls_plan_create": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ctypes.c_void_p),
                                      ctypes.POINTER(ctypes.c_void_p), c_i64p, ctypes.POINTER(ctypes.c_void_p),
                                      ctypes.c_int32, ctypes.POINTER(ctypes.c_void_p)]),
    "ls_plan_info": (ctypes.c_int, [ctypes.c_void_p, c_i32p, c_i32p, c_i32p, c_i32p]),
    "ls_plan_launch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "ls_plan_status": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "ls_plan_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "ls_cg_fit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                 ctypes.c_double, ctypes.c_int32, ctypes.c_double, ctypes.c_int32, c_f64p, c_i32p,
                                 ctypes.c_void_p]),
    "ls_dot_f64": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                  ctypes.c_void_p]),
}

_lib = None


class LsError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


ABI_VERSION = 8          # ls_abi_version() of the library these struct layouts match


def lib():
    """The loaded libls.so (built on first use if absent)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            from . import build as _build
            _build.build()
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        if L.ls_abi_version() != ABI_VERSION:
            # the structs below would be read with another layout
            raise RuntimeError(f"{LIB_PATH} has ABI version {L.ls_abi_version()}, these bindings {ABI_VERSION}: "
                               "rebuild it (paper_2102_08518_b300.build.build())")
        _lib = L
    return _lib


def check(status: int, where: str):
    if status != LS_OK:
        raise LsError(status, where, lib().ls_last_error().decode(errors="replace"))


# ---------------------------------------------------------------------------
# descriptor marshalling
# ---------------------------------------------------------------------------

class DescHolder:
    """A ls_spline_desc plus the arrays it points to (kept alive together)."""

    def __init__(self, table, name: Optional[str] = None, expansion: str = "sparse"):
        spl = table.spline
        lat = spl.lattice
        s = lat.dim
        self._keep: List = []
        d = SplineDescC()
        self.name_b = (name or spl.name).encode()
        d.name = self.name_b
        d.dim = s
        d.roe = LS_ROE_VORONOI if spl.roe == "voronoi" else LS_ROE_PARALLELEPIPED
        d.fold = LS_FOLD_SIGNED_PERM if table.fold == "hyperoctahedral" else LS_FOLD_NONE
        d.scale = lat.scale
        for c in range(s):
            for r in range(s):
                d.generator[3 * c + r] = float(lat.generator[c][r])
        d.n_cosets = len(lat.cosets)
        d.coset_offsets = self._i32([v for l in lat.cosets for v in l])
        d.n_planes = len(table.planes)
        d.planes = self._f64([float(v) for p, dd in table.planes for v in list(p) + [dd]]) if table.planes else None
        d.bsp_mod = table.bsp_mod
        sig = (ctypes.c_int8 * len(table.sigma))(*table.sigma)
        self._keep.append(sig)
        d.sigma = ctypes.cast(sig, ctypes.POINTER(ctypes.c_int8))
        regions = table.regions
        if expansion == "centroid" and getattr(table, "regions_centroid", None):
            regions = table.regions_centroid
        regs = (RefRegionC * len(regions))()
        for k, r in enumerate(regions):
            rc = regs[k]
            rc.n_sites = len(r.sites)
            rc.sites = self._i32([v for site in r.sites for v in site])
            rc.n_monos = len(r.monomials)
            rc.mono_exp = self._i32([v for m in r.monomials for v in m])
            M = r.coef_matrix()
            rc.coef = self._f64([float(v) for row in M for v in row])
            for i in range(3):
                rc.center[i] = float(r.center[i]) if i < s else 0.0
        self._keep.append(regs)
        d.n_ref = len(regions)
        d.ref = ctypes.cast(regs, ctypes.POINTER(RefRegionC))
        if table.separable:
            axes = (AxisFactorC * s)()
            for i, a in enumerate(table.separable):
                axes[i].n_sites = len(a.sites)
                axes[i].sites = self._i32(a.sites)
                axes[i].degree = a.degree
                coef = []
                for w in a.weights:
                    coef += [float(w.c.get((p,), 0)) for p in range(a.degree + 1)]
                axes[i].coef = self._f64(coef)
                axes[i].center = float(a.center)
            self._keep.append(axes)
            d.separable = ctypes.cast(axes, ctypes.POINTER(AxisFactorC))
        else:
            d.separable = None
        self.desc = d

    def _i32(self, vals):
        arr = (ctypes.c_int32 * max(1, len(vals)))(*vals)
        self._keep.append(arr)
        return ctypes.cast(arr, c_i32p)

    def _f64(self, vals):
        arr = (ctypes.c_double * max(1, len(vals)))(*vals)
        self._keep.append(arr)
        return ctypes.cast(arr, c_f64p)


def variant(block=256, pts_per_thread=1, branchy=0, min_blocks=0, group=0, depth=0, blocks_per_sm=0,
            brick=0, pipeline=0, producers=0, stage=0, tensor=0, tensor_kind=0, plain_transform=0,
            wait_limit=0, wait_probe=0, prefetch=0, l2_keep=0, fma2=0) -> VariantC:
    return VariantC(block, pts_per_thread, branchy, min_blocks, group, depth, blocks_per_sm, brick, pipeline,
                    producers, stage, tensor, tensor_kind, plain_transform, wait_limit, wait_probe, prefetch,
                    l2_keep, fma2)
