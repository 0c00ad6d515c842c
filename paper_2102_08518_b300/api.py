"""Python API over the C ABI: splines, coefficient volumes, evaluation.

PyTorch provides device memory and streams; every computation runs in the
library's kernels (libls.so and the kernels it generates).  There is no CPU
fallback: without a CUDA device the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import pickle
from typing import Dict, Optional, Sequence, Tuple

import torch

from . import _abi
from .splines import BY_NAME
from .subregions import Table, build_table

_TABLE_CACHE: Dict[str, Table] = {}
_TABLE_VERSION = 4
_CACHE_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "kcache")

DTYPES = {"f32": _abi.LS_F32, "bf16": _abi.LS_BF16, "f16": _abi.LS_F16}
LAYOUTS = {"coset": _abi.LS_LAYOUT_COSET_MAJOR, "interleaved": _abi.LS_LAYOUT_INTERLEAVED,
           "bricked": _abi.LS_LAYOUT_BRICKED, "bricked_shifted": _abi.LS_LAYOUT_BRICKED_SHIFTED,
           "bricked_shifted_xyz": _abi.LS_LAYOUT_BRICKED_SHIFTED_XYZ}
# the kernels' variant.brick for each layout
LAYOUT_BRICK = {"coset": 0, "interleaved": 0, "bricked": 1, "bricked_shifted": 2, "bricked_shifted_xyz": 3}


def layout_elems(n_cosets: int, ext: Sequence[int], layout: str) -> int:
    """Elements a coefficient layout holds (the shifted bricked copies: four
    padded copies)."""
    e = tuple(int(v) for v in ext) + (1,) * (3 - len(ext))
    if layout == "bricked_shifted":
        return 4 * n_cosets * (e[0] + 2) * (e[1] + 2) * e[2]
    if layout == "bricked_shifted_xyz":
        return 8 * n_cosets * (e[0] + 2) * (e[1] + 2) * (e[2] + 2)
    return n_cosets * e[0] * e[1] * e[2]
TORCH_DTYPES = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}


def table(name: str) -> Table:
    """Sub-region table of a named spline (built once, cached on disk)."""
    if name in _TABLE_CACHE:
        return _TABLE_CACHE[name]
    path = os.path.join(_CACHE_DIR, f"table_{name}_v{_TABLE_VERSION}.pkl")
    t = None
    if os.path.exists(path):
        try:
            with open(path, "rb") as f:
                t = pickle.load(f)
        except Exception:
            t = None
    if t is None:
        t = build_table(BY_NAME[name])
        try:
            os.makedirs(_CACHE_DIR, exist_ok=True)
            tmp = path + f".tmp{os.getpid()}"
            with open(tmp, "wb") as f:
                pickle.dump(t, f)
            os.replace(tmp, path)
        except OSError:
            pass
    _TABLE_CACHE[name] = t
    return t


def _stream(stream: Optional[torch.cuda.Stream]):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t: Optional[torch.Tensor]):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def kernel_name(name: str, dtype: str, block: int = 256, branchy: int = 0, min_blocks: int = 0, group: int = 0,
                depth: int = 0, pts_per_thread: int = 1, blocks_per_sm: int = 0, expansion: str = "sparse",
                brick: int = 0, pipeline: int = 0, producers: int = 0, stage: int = 0, tensor: int = 0,
                tensor_kind: int = 0, plain_transform: int = 0, wait_limit: int = 0, wait_probe: int = 0,
                prefetch: int = 0, l2_keep: int = 0, fma2: int = 0) -> str:
    """The name tag of a generated kernel variant (blocks_per_sm only sizes the
    grid, so it shares the compiled kernel)."""
    return f"{name}_{dtype}" + (f"_b{block}" if block != 256 else "") + ("_br" if branchy else "") + \
        (f"_m{min_blocks}" if min_blocks else "") + (f"_g{group}d{depth}" if group and depth else "") + \
        (f"_t{pts_per_thread}" if pts_per_thread > 1 else "") + ("_ec" if expansion == "centroid" else "") + \
        (f"_bk{brick}" if brick >= 2 else "_bk" if brick else "") + ("_pp" if pipeline else "") + (f"_ws{producers}" if producers else "") + \
        (f"_st{stage}" if stage else "") + (("_tc" + (str(tensor) if tensor > 1 else "")) if tensor else "") + \
        ("h" if tensor and tensor_kind else "") + ("_pt" if plain_transform else "") + \
        (f"_wl{wait_limit}" if wait_limit else "") + ("_wp" if wait_probe else "") + ("_pf" if prefetch else "") + \
        ("_lk" if l2_keep else "") + ("_f2" if fma2 else "")


class Spline:
    """Generated, compiled and loaded kernels of one spline for one storage dtype."""

    def __init__(self, name: str, dtype: str = "f32", block: int = 256, branchy: int = 0,
                 min_blocks: int = 0, group: int = 0, depth: int = 0, pts_per_thread: int = 1,
                 blocks_per_sm: int = 0, expansion: str = "sparse", brick: int = 0, pipeline: int = 0,
                 producers: int = 0, stage: int = 0, tensor: int = 0, tensor_kind: int = 0,
                 plain_transform: int = 0, wait_limit: int = 0, wait_probe: int = 0, prefetch: int = 0,
                 l2_keep: int = 0, fma2: int = 0, kernel_name: Optional[str] = None):
        if not torch.cuda.is_available():
            raise RuntimeError("lattice spline kernels need a CUDA device")
        self.name = name
        self.dtype = dtype
        self.table = table(name)
        self.dim = self.table.spline.lattice.dim
        self.n_cosets = len(self.table.spline.lattice.cosets)
        self.scale = self.table.spline.lattice.scale
        kname = kernel_name or globals()["kernel_name"](name, dtype, block, branchy, min_blocks, group, depth,
                                                         pts_per_thread, blocks_per_sm, expansion, brick, pipeline,
                                                         producers, stage, tensor, tensor_kind,
                                                         plain_transform, wait_limit, wait_probe, prefetch,
                                                         l2_keep, fma2)
        self.variant = {"block": block, "branchy": branchy, "min_blocks": min_blocks, "group": group,
                        "depth": depth, "pts_per_thread": pts_per_thread, "blocks_per_sm": blocks_per_sm,
                        "expansion": expansion}
        if brick:
            self.variant["brick"] = brick
        if pipeline:
            self.variant["pipeline"] = 1
        if producers:
            self.variant["producers"] = producers
        if stage:
            self.variant["stage"] = stage
        if tensor:
            self.variant["tensor"] = tensor
        if tensor_kind:
            self.variant["tensor_kind"] = tensor_kind
        if plain_transform:
            self.variant["plain_transform"] = 1
        if wait_limit:
            self.variant["wait_limit"] = wait_limit
        if wait_probe:
            self.variant["wait_probe"] = wait_probe
        if prefetch:
            self.variant["prefetch"] = 1
        if l2_keep:
            self.variant["l2_keep"] = 1
        if fma2:
            self.variant["fma2"] = 1
        self.kernel_name = kname
        self._desc = _abi.DescHolder(self.table, kname, expansion)
        var = _abi.variant(block=block, pts_per_thread=pts_per_thread, branchy=branchy, min_blocks=min_blocks,
                           group=group, depth=depth, blocks_per_sm=blocks_per_sm, brick=brick, pipeline=pipeline,
                           producers=producers, stage=stage, tensor=tensor, tensor_kind=tensor_kind,
                           plain_transform=plain_transform, wait_limit=wait_limit, wait_probe=wait_probe,
                           prefetch=prefetch, l2_keep=l2_keep, fma2=fma2)
        h = ctypes.c_void_p()
        torch.cuda.init()
        _abi.check(_abi.lib().ls_spline_create(ctypes.byref(self._desc.desc), DTYPES[dtype], ctypes.byref(var),
                                               ctypes.byref(h)), "ls_spline_create")
        self.handle = h

    def info(self):
        n, fv, fg, regs = (ctypes.c_int32() for _ in range(4))
        _abi.check(_abi.lib().ls_spline_info(self.handle, ctypes.byref(n), ctypes.byref(fv), ctypes.byref(fg),
                                             ctypes.byref(regs)), "ls_spline_info")
        return {"n_sites": n.value, "fma_value": fv.value, "fma_grad": fg.value, "regs_eval": regs.value}

    def source(self) -> str:
        return _abi.lib().ls_spline_source(self.handle).decode()

    def status(self, stream=None):
        """Raise if a bounded wait in one of this spline's kernels gave up."""
        _abi.check(_abi.lib().ls_spline_status(self.handle, _stream(stream)), "ls_spline_status")

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            try:
                _abi.lib().ls_spline_destroy(h)
            except Exception:
                pass
            self.handle = None


class Volume:
    """Coefficients of a spline on n_cosets arrays of extent ext (axis 0 fastest).

    ``layout``: "coset" (one array after another: shape (n_cosets, ext[dim-1],
    ..., ext[0])), "interleaved" (the cosets' values of one grid index
    adjacent: shape (ext[dim-1], ..., ext[0], n_cosets)), "bricked" (bricks
    of 2 x 2 x 2 grid indices, cosets interleaved inside; needs a spline made
    with brick=1) or "bricked_shifted" (four bricked copies with shifted brick
    grids, each point reading the one that cuts its stencil into the fewest
    sectors; evaluation only; needs a spline made with brick=2); see
    ``relayout``.
    ``coef`` (device tensor of the spline's storage dtype in that layout) is
    wrapped without a copy; otherwise a zero volume is allocated by the library.
    """

    def __init__(self, spline: Spline, ext: Sequence[int], coef: Optional[torch.Tensor] = None,
                 layout: str = "coset"):
        self.spline = spline
        self.layout = layout
        lay = LAYOUTS[layout]
        self.ext = tuple(int(e) for e in ext) + (1,) * (3 - len(ext))
        e64 = (ctypes.c_int64 * 3)(*self.ext)
        h = ctypes.c_void_p()
        if coef is not None:
            want = layout_elems(spline.n_cosets, self.ext[:spline.dim], layout)
            if not coef.is_cuda or not coef.is_contiguous() or coef.numel() != want or \
                    coef.dtype != TORCH_DTYPES[spline.dtype]:
                raise ValueError("coef must be a contiguous CUDA tensor of the spline's dtype and volume size")
            self.coef = coef
            _abi.check(_abi.lib().ls_volume_wrap(spline.handle, e64, lay, _ptr(coef), ctypes.byref(h)),
                       "ls_volume_wrap")
        else:
            self.coef = None
            _abi.check(_abi.lib().ls_volume_create(spline.handle, e64, lay, ctypes.byref(h)), "ls_volume_create")
        self.handle = h

    @property
    def n_coef(self) -> int:
        n = self.spline.n_cosets
        for i in range(self.spline.dim):
            n *= self.ext[i]
        return n

    def upload(self, src: torch.Tensor, stream=None):
        """Copy coefficients given in coset-major order (host or device, any
        float dtype) into the volume, converting dtype and layout."""
        dt = {torch.float32: _abi.LS_F32, torch.float64: _abi.LS_F64, torch.bfloat16: _abi.LS_BF16,
              torch.float16: _abi.LS_F16}[src.dtype]
        src = src.contiguous()
        if src.numel() != self.n_coef:
            raise ValueError("upload size mismatch")
        _abi.check(_abi.lib().ls_volume_upload(self.handle, _ptr(src), int(src.is_cuda), dt, _stream(stream)),
                   "ls_volume_upload")
        if not src.is_cuda:
            torch.cuda.current_stream().synchronize()

    def eval(self, pts: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        pts = _check_pts(pts, self.spline.dim)
        n = pts.shape[0]
        if out is None:
            out = torch.empty(n, device=pts.device, dtype=torch.float32)
        _abi.check(_abi.lib().ls_eval(self.handle, _ptr(pts), n, _ptr(out), _stream(stream)), "ls_eval")
        return out

    def eval_grad(self, pts: torch.Tensor, want_value: bool = True, stream=None):
        pts = _check_pts(pts, self.spline.dim)
        n = pts.shape[0]
        val = torch.empty(n, device=pts.device, dtype=torch.float32) if want_value else None
        grad = torch.empty(n, self.spline.dim, device=pts.device, dtype=torch.float32)
        _abi.check(_abi.lib().ls_eval_grad(self.handle, _ptr(pts), n, _ptr(val), _ptr(grad), _stream(stream)),
                   "ls_eval_grad")
        return val, grad

    def eval_hess(self, pts: torch.Tensor, want_value: bool = True, want_grad: bool = True, stream=None):
        """(f, grad f, Hessian) with the Hessian as (n, 6) xx yy zz xy xz yz in 3D,
        (n, 3) xx yy xy in 2D; f and grad are None unless wanted."""
        pts = _check_pts(pts, self.spline.dim)
        n = pts.shape[0]
        dim = self.spline.dim
        val = torch.empty(n, device=pts.device, dtype=torch.float32) if want_value else None
        grad = torch.empty(n, dim, device=pts.device, dtype=torch.float32) if want_grad else None
        hess = torch.empty(n, 6 if dim == 3 else 3, device=pts.device, dtype=torch.float32)
        _abi.check(_abi.lib().ls_eval_hess(self.handle, _ptr(pts), n, _ptr(val), _ptr(grad), _ptr(hess),
                                           _stream(stream)), "ls_eval_hess")
        return val, grad, hess

    def texture_sync(self, stream=None):
        """Copy the coefficients into the volume's texture (for eval_linear_fetch)."""
        _abi.check(_abi.lib().ls_volume_texture_sync(self.handle, _stream(stream)), "ls_volume_texture_sync")

    def eval_linear_fetch(self, pts: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        """f(pts) by hardware-interpolated texture fetches (tensor-product splines;
        within 6/256 of max|c|, see ls_eval_linear_fetch)."""
        pts = _check_pts(pts, self.spline.dim)
        if out is None:
            out = torch.empty(pts.shape[0], device=pts.device, dtype=torch.float32)
        _abi.check(_abi.lib().ls_eval_linear_fetch(self.handle, _ptr(pts), pts.shape[0], _ptr(out), _stream(stream)),
                   "ls_eval_linear_fetch")
        return out

    def eval_host(self, pts_host, out_host, stream=None):
        """Host buffers in, host buffer out (copies inside the call)."""
        n = pts_host.shape[0]
        _abi.check(_abi.lib().ls_eval_host(self.handle, ctypes.c_void_p(pts_host.data_ptr()), n,
                                           ctypes.c_void_p(out_host.data_ptr()), _stream(stream)), "ls_eval_host")
        return out_host

    def adjoint(self, pts: torch.Tensor, gout: torch.Tensor, dcoef: Optional[torch.Tensor] = None,
                deterministic: bool = False, warp_aggregated: bool = False, tiled: bool = False,
                stream=None) -> torch.Tensor:
        """dcoef += A^T gout in the volume's layout: atomic (default), bitwise
        deterministic, or atomic with warp aggregation of equal sites; tiled:
        per-block shared-memory sums for spatially sorted points."""
        pts = _check_pts(pts, self.spline.dim)
        mode = _adjoint_mode(deterministic, warp_aggregated, tiled)
        gout = gout.contiguous().float()
        if dcoef is None:
            dcoef = torch.zeros(self.n_coef, device=pts.device, dtype=torch.float32)
        _abi.check(_abi.lib().ls_adjoint_coef(self.handle, _ptr(pts), _ptr(gout), pts.shape[0], _ptr(dcoef),
                                              mode, ctypes.c_void_p(0), _stream(stream)),
                   "ls_adjoint_coef")
        return dcoef

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            try:
                _abi.lib().ls_volume_destroy(h)
            except Exception:
                pass
            self.handle = None


def _adjoint_mode(deterministic, warp_aggregated: bool, tiled: bool = False) -> int:
    """deterministic: False, True / "binned" (fixed summation order) or "fixed"
    (fixed-point integer atomics); warp_aggregated: aggregated FP32 atomics;
    tiled: shared-memory tiles for spatially sorted points (FP32 atomics or,
    with deterministic="fixed", the fixed-point sums)."""
    if deterministic and warp_aggregated:
        raise ValueError("choose deterministic or warp_aggregated")
    if tiled:
        if warp_aggregated or deterministic not in (False, "fixed"):
            raise ValueError("tiled goes with the atomic or the fixed-point adjoint")
        return _abi.LS_ADJ_DETERMINISTIC_FIXED_TILED if deterministic == "fixed" else _abi.LS_ADJ_ATOMIC_TILED
    if deterministic == "fixed":
        return _abi.LS_ADJ_DETERMINISTIC_FIXED
    if deterministic:
        return _abi.LS_ADJ_DETERMINISTIC
    return _abi.LS_ADJ_ATOMIC_WARP if warp_aggregated else _abi.LS_ADJ_ATOMIC


def relayout(coef: torch.Tensor, n_cosets: int, ext: Sequence[int], to: str = "interleaved",
             src: str = "coset", stream=None) -> torch.Tensor:
    """A copy of n_cosets coefficient arrays of extent ext (axis 0 first) moved
    from layout ``src`` to layout ``to`` ("coset", "interleaved", "bricked",
    "bricked_shifted")."""
    coef = coef.contiguous()
    e = tuple(int(v) for v in ext) + (1,) * (3 - len(ext))
    if not coef.is_cuda or coef.numel() != layout_elems(n_cosets, e, src):
        raise ValueError("coef must be a CUDA tensor holding the source layout's elements")
    dst = torch.empty(layout_elems(n_cosets, e, to), dtype=coef.dtype, device=coef.device)
    _abi.check(_abi.lib().ls_relayout(_ptr(coef), LAYOUTS[src], _ptr(dst), LAYOUTS[to], int(n_cosets),
                                      (ctypes.c_int64 * 3)(*e), coef.element_size(), _stream(stream)),
               "ls_relayout")
    return dst


def _check_pts(pts: torch.Tensor, dim: int) -> torch.Tensor:
    if not pts.is_cuda or pts.dtype != torch.float32 or pts.dim() != 2 or pts.shape[1] != dim:
        raise ValueError(f"points must be a CUDA float32 tensor of shape (n, {dim})")
    return pts.contiguous()


# ---------------------------------------------------------------------------
# point ordering and device reductions
# ---------------------------------------------------------------------------

def morton_sort(pts: torch.Tensor, origin=(0.0, 0.0, 0.0), cell: float = 1.0, want_keys: bool = False,
                scratch: Optional[torch.Tensor] = None, stream=None):
    """perm (int32) ordering points by the Morton code of their cell; stable."""
    pts = _check_pts(pts, 3)
    n = pts.shape[0]
    perm = torch.empty(n, dtype=torch.int32, device=pts.device)
    keys = torch.empty(n, dtype=torch.int32, device=pts.device) if want_keys else None
    o = (ctypes.c_float * 3)(*[float(v) for v in origin])
    _abi.check(_abi.lib().ls_morton_sort(_ptr(pts), n, o, float(cell), _ptr(perm), _ptr(keys), _ptr(scratch),
                                         _stream(stream)), "ls_morton_sort")
    return (perm, keys) if want_keys else perm


def morton_scratch_bytes(n: int) -> int:
    return int(_abi.lib().ls_morton_scratch_bytes(n))


def permute_rows(src: torch.Tensor, perm: torch.Tensor, inverse: bool = False, stream=None) -> torch.Tensor:
    """dst[i] = src[perm[i]] (inverse: dst[perm[i]] = src[i]) for rows of src."""
    src = src.contiguous()
    n = src.shape[0]
    width = src.numel() // max(n, 1)
    dst = torch.empty_like(src)
    _abi.check(_abi.lib().ls_permute_rows(_ptr(src), _ptr(perm), n, width, int(inverse), _ptr(dst),
                                          _stream(stream)), "ls_permute_rows")
    return dst


def dot_f64(a: torch.Tensor, b: torch.Tensor, stream=None) -> torch.Tensor:
    """sum a*b accumulated in FP64 on the device (returns a 1-element float64 tensor)."""
    a = a.contiguous().float()
    b = b.contiguous().float()
    out = torch.empty(1, dtype=torch.float64, device=a.device)
    _abi.check(_abi.lib().ls_dot_f64(_ptr(a), _ptr(b), a.numel(), _ptr(out), _stream(stream)), "ls_dot_f64")
    return out


def probe_gather(table_t: torch.Tensor, loads: int, nthreads: int, blocks: int = 0, out=None, stream=None):
    if out is None:
        out = torch.empty(nthreads, device=table_t.device)
    _abi.check(_abi.lib().ls_probe_gather(_ptr(table_t), table_t.numel(), loads, _ptr(out), nthreads, blocks,
                                          _stream(stream)), "ls_probe_gather")
    return out


# ---------------------------------------------------------------------------
# least-squares fit and autograd
# ---------------------------------------------------------------------------

def cg_fit(volume: "Volume", pts: torch.Tensor, y: torch.Tensor, lam: float = 0.0, max_iter: int = 200,
           rel_tol: float = 1e-6, deterministic: bool = False, warp_aggregated: bool = False, tiled: bool = False,
           stream=None):
    """CGLS on min ||A c - y||^2 + lam ||c||^2; the volume's coefficients (FP32)
    hold the initial guess and receive the result.  Returns (iterations, history)."""
    import numpy as np
    pts = _check_pts(pts, volume.spline.dim)
    y = y.contiguous().float()
    hist = np.zeros(max_iter + 1)
    iters = ctypes.c_int32()
    _abi.check(_abi.lib().ls_cg_fit(volume.handle, _ptr(pts), _ptr(y), pts.shape[0], float(lam), int(max_iter),
                                    float(rel_tol), _adjoint_mode(deterministic, warp_aggregated, tiled),
                                    hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(iters),
                                    _stream(stream)), "ls_cg_fit")
    return iters.value, hist[: iters.value + 1]


class SplineEval(torch.autograd.Function):
    """f(pts) = sum_n coef_n phi(pts - n) with gradients for coef and pts.

    Forward runs the fused value + gradient kernel when pts needs a gradient;
    backward is the adjoint kernel for coef (atomic or deterministic) and
    gout * grad f for pts.
    """

    @staticmethod
    def forward(ctx, coef, pts, spline, ext, deterministic, layout="coset"):
        vol = Volume(spline, ext, coef.detach().contiguous(), layout=layout)
        if pts.requires_grad:
            val, grad = vol.eval_grad(pts.detach())
        else:
            val, grad = vol.eval(pts.detach()), None
        ctx.vol = vol
        ctx.deterministic = deterministic
        ctx.coef_shape = coef.shape
        ctx.save_for_backward(pts.detach(), grad if grad is not None else torch.empty(0, device=pts.device))
        return val

    @staticmethod
    def backward(ctx, gout):
        pts, grad = ctx.saved_tensors
        gcoef = gpts = None
        gout = gout.contiguous()
        if ctx.needs_input_grad[0]:
            gcoef = ctx.vol.adjoint(pts, gout, deterministic=ctx.deterministic).view(ctx.coef_shape)
        if ctx.needs_input_grad[1]:
            gpts = gout[:, None] * grad
        return gcoef, gpts, None, None, None, None


def spline_eval(spline: Spline, ext: Sequence[int], coef: torch.Tensor, pts: torch.Tensor,
                deterministic: bool = False, layout: str = "coset") -> torch.Tensor:
    """Differentiable f(pts); coef in ``layout``, and its gradient in the same layout."""
    return SplineEval.apply(coef, pts, spline, tuple(ext), deterministic, layout)


# ---------------------------------------------------------------------------
# batched persistent evaluation
# ---------------------------------------------------------------------------

class Plan:
    """One persistent launch over many volumes, each with its own point batch."""

    def __init__(self, volumes: Sequence["Volume"], pts: Sequence[torch.Tensor], outs: Sequence[torch.Tensor],
                 tile: int = 0):
        n = len(volumes)
        self.volumes = list(volumes)
        self.pts = [_check_pts(p, v.spline.dim) for p, v in zip(pts, volumes)]
        self.outs = list(outs)
        vh = (ctypes.c_void_p * n)(*[v.handle.value for v in volumes])
        ph = (ctypes.c_void_p * n)(*[p.data_ptr() for p in self.pts])
        nh = (ctypes.c_int64 * n)(*[p.shape[0] for p in self.pts])
        oh = (ctypes.c_void_p * n)(*[o.data_ptr() for o in self.outs])
        h = ctypes.c_void_p()
        _abi.check(_abi.lib().ls_plan_create(n, vh, ph, nh, oh, int(tile), ctypes.byref(h)), "ls_plan_create")
        self.handle = h

    def info(self):
        t, b, ni, g = (ctypes.c_int32() for _ in range(4))
        _abi.check(_abi.lib().ls_plan_info(self.handle, ctypes.byref(t), ctypes.byref(b), ctypes.byref(ni),
                                           ctypes.byref(g)), "ls_plan_info")
        return {"tile": t.value, "block": b.value, "n_items": ni.value, "grid": g.value}

    def launch(self, stream=None):
        _abi.check(_abi.lib().ls_plan_launch(self.handle, _stream(stream)), "ls_plan_launch")

    def status(self, stream=None):
        _abi.check(_abi.lib().ls_plan_status(self.handle, _stream(stream)), "ls_plan_status")

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            try:
                _abi.lib().ls_plan_destroy(h)
            except Exception:
                pass
            self.handle = None


# ---------------------------------------------------------------------------
# autotuning of the evaluation kernel variant
# ---------------------------------------------------------------------------

DEFAULT_CANDIDATES = (
    dict(block=256), dict(block=512), dict(block=256, min_blocks=2), dict(block=128, min_blocks=4),
    dict(block=256, group=8, depth=2), dict(block=256, group=8, depth=3), dict(block=256, group=4, depth=4),
    dict(block=512, group=8, depth=2), dict(block=512, group=16, depth=1), dict(block=256, group=16, depth=1),
)


# the variants that won or came close somewhere in the full sweep (block size
# and occupancy; limiting gathers in flight, 4 warps per SM, the software-
# pipelined and the warp-specialized kernels never won on B300)
TUNE_CANDIDATES_SMALL = tuple([dict(block=256, blocks_per_sm=b, expansion=x) for b in (0, 2, 3) for x in
                               ("sparse", "centroid")] +
                              [dict(block=512, expansion=x) for x in ("sparse", "centroid")] +
                              [dict(block=384, expansion=x) for x in ("sparse", "centroid")] +
                              [dict(block=128, blocks_per_sm=b) for b in (2, 4)] +
                              [dict(block=384, min_blocks=2), dict(block=256, min_blocks=3)] +
                              [dict(block=b, prefetch=1) for b in (256, 384, 512)] +
                              [dict(block=256, blocks_per_sm=2, prefetch=1)] +
                              [dict(block=b) for b in (640, 672)] +
                              [dict(block=b, group=16, depth=1) for b in (256, 384, 512)] +
                              [dict(block=512, group=8, depth=2), dict(block=512, group=4, depth=4)] +
                              [dict(block=b, l2_keep=1) for b in (384, 512, 672)] +
                              [dict(tensor=1, expansion=x) for x in ("sparse", "centroid")] +
                              [dict(tensor=1, tensor_kind=1, expansion=x) for x in ("sparse", "centroid")] +
                              [dict(tensor=4, tensor_kind=1)] +
                              [dict(tensor=6, tensor_kind=1, expansion=x) for x in ("sparse", "centroid")])


def autotune(name: str, dtype: str, ext: Sequence[int], coef: torch.Tensor, pts_sets: Sequence[torch.Tensor],
             candidates=DEFAULT_CANDIDATES, reps: int = 5, tag: str = "", layout: str = "coset") -> "Spline":
    """Generate the evaluation kernel in each candidate variant (block size,
    minimum blocks per SM, gather group size m and depth d), time it on the
    caller's volume (``coef`` in ``layout``) and point sets, and return the
    fastest Spline.  The choice is cached on disk per (spline, dtype, GPU, tag,
    layout)."""
    import json
    key = _tune_key(name, dtype, ext, pts_sets, tag, layout)
    path = os.path.join(_CACHE_DIR, "autotune.json")
    cache = {}
    try:
        with open(path) as f:
            cache = json.load(f)
    except (OSError, ValueError):
        cache = {}
    if key in cache:
        return Spline(name, dtype, **cache[key]["variant"])
    # results measured earlier on this GPU model, shipped with the package
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "autotune_b300.json")) as f:
            shipped = json.load(f)
        if key in shipped:
            return Spline(name, dtype, **shipped[key]["variant"])
    except (OSError, ValueError):
        pass
    best = None
    results = []
    separable = bool(table(name).separable)
    for cand in candidates:
        if cand.get("tensor") and separable:
            continue                      # tensor-product tables have no coefficient transform to offload
        if cand.get("tensor") and LAYOUT_BRICK[layout]:
            continue                      # on B300 the tensor-core kernels never won on bricks: linear layouts only
        if cand.get("tensor_kind") and dtype != "f32":
            continue                      # the FP16 form splits FP32 data; BF16 / FP16 data are exact in TF32
        sp = Spline(name, dtype, **cand, **({"brick": LAYOUT_BRICK[layout]} if LAYOUT_BRICK[layout] else {}))
        vol = Volume(sp, ext, coef, layout=layout)
        outs = [torch.empty(p.shape[0], device=p.device) for p in pts_sets]
        for p, o in zip(pts_sets, outs):
            vol.eval(p, o)
        torch.cuda.synchronize()
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record()
        for _ in range(reps):
            for p, o in zip(pts_sets, outs):
                vol.eval(p, o)
        e.record()
        torch.cuda.synchronize()
        ms = s.elapsed_time(e) / reps
        results.append({"variant": sp.variant, "ms": ms})
        if best is None or ms < best[0]:
            best = (ms, sp)
    cache[key] = {"variant": best[1].variant, "ms": best[0], "all": results}
    try:
        os.makedirs(_CACHE_DIR, exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, path)
    except OSError:
        pass
    return best[1]


def _tune_key(name, dtype, ext, pts_sets, tag, layout="coset"):
    # the generated kernel's FMA count identifies the table version the choice was made for
    fma = Spline(name, dtype).info()["fma_value"]
    gpu = torch.cuda.get_device_name()
    lay = "" if layout == "coset" else f"|{layout}"
    return f"{name}|{dtype}|fma{fma}|{gpu}|{tuple(ext)}|{tag}|{[int(p.shape[0]) for p in pts_sets]}{lay}"


def autotune_record(name: str, dtype: str, ext, pts_sets, tag: str = "", layout: str = "coset"):
    """The autotuning entry for this workload (the local cache first, then the
    results shipped with the package), if any: its variant and time in ms."""
    import json
    key = _tune_key(name, dtype, ext, pts_sets, tag, layout)
    for path in (os.path.join(_CACHE_DIR, "autotune.json"),
                 os.path.join(os.path.dirname(os.path.abspath(__file__)), "autotune_b300.json")):
        try:
            with open(path) as f:
                rec = json.load(f).get(key)
        except (OSError, ValueError):
            rec = None
        if rec is not None:
            return rec
    return None


def eval_host_multi(volumes: Sequence["Volume"], pts_host: torch.Tensor, outs_host: Sequence[torch.Tensor],
                    stream=None):
    """Host points in, one host output per volume (points cross to the device once)."""
    n = len(volumes)
    vh = (ctypes.c_void_p * n)(*[v.handle.value for v in volumes])
    oh = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs_host])
    _abi.check(_abi.lib().ls_eval_host_multi(n, vh, ctypes.c_void_p(pts_host.data_ptr()), pts_host.shape[0], oh,
                                             _stream(stream)), "ls_eval_host_multi")
    return outs_host
