"""Seeded synthetic inputs (coefficient volumes and query points).

Shared by the tests, the benchmark and both sides of every parity check.  Holds
no spline arithmetic: only random numbers, smooth test fields and point sets
with the shapes of the paper's workloads (random locations in synthetic
volumes, Sec. 5; sizes from the benchmark configurations).

Coefficient arrays are returned coset-major with axis 0 fastest, i.e. numpy
shape (n_cosets, E2, E1, E0), for sites scale*i + coset_offset.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Sequence, Tuple

import numpy as np

LATTICES = {
    # name: (dim, scale, cosets)
    "cc": (3, 1, ((0, 0, 0),)),
    "bcc": (3, 2, ((0, 0, 0), (1, 1, 1))),
    "fcc": (3, 2, ((0, 0, 0), (1, 1, 0), (1, 0, 1), (0, 1, 1))),
    "z2": (2, 1, ((0, 0),)),
}
SPLINE_LATTICE = {"tricubic": "cc", "trilinear": "cc", "triquadratic": "cc", "bcc_linear": "bcc",
                  "bcc_quintic": "bcc", "bcc_quartic": "bcc", "fcc6": "fcc", "zp": "z2", "voronoi2_bcc": "bcc",
                  "voronoi2_fcc": "fcc"}
# half-width of the support box along an axis: 1/2 sum_xi |xi_i| (input margins only)
SUPPORT_HALF = {"tricubic": 2.0, "trilinear": 1.0, "triquadratic": 1.5, "bcc_linear": 2.0, "bcc_quintic": 4.0,
                "bcc_quartic": 3.0, "fcc6": 2.0, "zp": 1.5, "voronoi2_bcc": 2.0, "voronoi2_fcc": 2.0}


def site_coords(lattice: str, ext: Sequence[int]) -> np.ndarray:
    """Coordinates of all stored sites, in coefficient order, shape (n, dim)."""
    dim, scale, cosets = LATTICES[lattice]
    e = list(ext) + [1] * (3 - len(ext))
    out = []
    for l in cosets:
        i2, i1, i0 = np.meshgrid(np.arange(e[2]), np.arange(e[1]), np.arange(e[0]), indexing="ij")
        pts = np.stack([scale * i0 + l[0], scale * i1 + l[1]] + ([scale * i2 + l[2]] if dim == 3 else []), -1)
        out.append(pts.reshape(-1, dim))
    return np.concatenate(out).astype(np.float64)


def coef_uniform(lattice: str, ext: Sequence[int], seed: int = 0) -> np.ndarray:
    """c ~ U[-1, 1] (FP32)."""
    dim, _, cosets = LATTICES[lattice]
    shape = (len(cosets),) + tuple(int(v) for v in reversed(list(ext)[:dim]))
    return np.random.default_rng(seed).uniform(-1.0, 1.0, shape).astype(np.float32)


def coef_smooth(lattice: str, ext: Sequence[int], seed: int = 0) -> np.ndarray:
    """c_n = sin(0.05 n_x) cos(0.07 n_y) + 0.1 N(0,1) at the site coordinates (FP32)."""
    dim, _, cosets = LATTICES[lattice]
    x = site_coords(lattice, ext)
    v = np.sin(0.05 * x[:, 0]) * np.cos(0.07 * x[:, 1]) + 0.1 * np.random.default_rng(seed).normal(size=len(x))
    shape = (len(cosets),) + tuple(int(v) for v in reversed(list(ext)[:dim]))
    return v.reshape(shape).astype(np.float32)


def bounding_box(lattice: str, ext: Sequence[int]) -> Tuple[np.ndarray, np.ndarray]:
    """[lo, hi] of the stored site coordinates."""
    dim, scale, cosets = LATTICES[lattice]
    lo = np.zeros(dim)
    hi = np.array([scale * (ext[i] - 1) + max(l[i] for l in cosets) for i in range(dim)], dtype=np.float64)
    return lo, hi


def inner_box(spline: str, ext: Sequence[int]):
    """The bounding box shrunk by the support half-width, so every stencil site is stored."""
    lo, hi = bounding_box(SPLINE_LATTICE[spline], ext)
    m = SUPPORT_HALF[spline]
    return lo + m, hi - m


def points_uniform(n: int, lo, hi, seed: int = 0) -> np.ndarray:
    """n points ~ U(box) as FP32, shape (n, dim)."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    return np.random.default_rng(seed).uniform(lo, hi, (n, len(lo))).astype(np.float32)


def points_rays(n_rays: int, steps: int, lo, hi, direction=(1.0, 0.37, 0.21), seed: int = 0) -> np.ndarray:
    """Ray-march order: n_rays parallel rays (origins on a square grid in the plane
    through the box centre orthogonal to `direction`, jittered by `seed`), each
    sampled at `steps` equally spaced points between its box entry and exit.
    Returned ray-major, shape (n_rays * steps, 3), FP32."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    d = np.asarray(direction, dtype=np.float64)
    d /= np.linalg.norm(d)
    u = np.cross(d, [0.0, 0.0, 1.0])
    u /= np.linalg.norm(u)
    w = np.cross(d, u)
    c = 0.5 * (lo + hi)
    g = int(round(np.sqrt(n_rays)))
    assert g * g == n_rays, "n_rays must be a square"
    half = 0.3 * float(np.min(hi - lo))
    s = np.linspace(-half, half, g)
    rng = np.random.default_rng(seed)
    jit = rng.uniform(-0.25, 0.25, (n_rays, 2)) * (2 * half / max(g - 1, 1))
    su, sw = np.meshgrid(s, s, indexing="ij")
    origins = c + (su.reshape(-1, 1) + jit[:, :1]) * u + (sw.reshape(-1, 1) + jit[:, 1:]) * w
    # entry/exit of each ray in the box (slab method)
    with np.errstate(divide="ignore"):
        t0 = (lo - origins) / d
        t1 = (hi - origins) / d
    tmin = np.max(np.minimum(t0, t1), axis=1)
    tmax = np.min(np.maximum(t0, t1), axis=1)
    eps = 1e-3
    t = tmin[:, None] + eps + (tmax - tmin - 2 * eps)[:, None] * (np.arange(steps)[None, :] / max(steps - 1, 1))
    pts = origins[:, None, :] + t[..., None] * d
    pts = np.clip(pts, lo, hi)
    return pts.reshape(-1, 3).astype(np.float32)


def gaussian_samples(n: int, lo, hi, noise: float = 0.01, width: float = 400.0, seed: int = 0):
    """Scattered samples of f(x) = exp(-|x - c|^2 / width) + noise N(0,1), c = box centre."""
    pts = points_uniform(n, lo, hi, seed)
    c = 0.5 * (np.asarray(lo) + np.asarray(hi))
    r2 = np.sum((pts.astype(np.float64) - c) ** 2, axis=1)
    y = np.exp(-r2 / width) + noise * np.random.default_rng(seed + 1).normal(size=n)
    return pts, y.astype(np.float32)


@dataclass
class BatchItem:
    spline: str
    edge: int
    ext: Tuple[int, int, int]
    n_points: int
    seed: int


def batch_recipe(n_vol: int = 64, seed: int = 0, edges=(32, 48, 64, 96, 128, 192, 256),
                 splines=("tricubic", "bcc_linear", "bcc_quintic", "fcc6"), log2_lo=10.0, log2_hi=22.0):
    """Volumes of the batched workload: edge length (bounding box) ~ U(edges),
    spline ~ U(splines), point count log-uniform in [2^log2_lo, 2^log2_hi].
    Non-Cartesian lattices store (edge/2)^3 sites per coset."""
    rng = np.random.default_rng(seed)
    out = []
    for v in range(n_vol):
        e = int(rng.choice(edges))
        sp = str(rng.choice(list(splines)))
        scale = LATTICES[SPLINE_LATTICE[sp]][1]
        ext = (e // scale,) * 3
        npts = int(round(2.0 ** rng.uniform(log2_lo, log2_hi)))
        out.append(BatchItem(sp, e, ext, npts, seed * 1000 + v))
    return out


def coef_uniform_torch(lattice: str, ext: Sequence[int], seed: int, dtype=None, device="cuda"):
    """c ~ U[-1, 1] drawn on the device with a seeded torch generator (large
    benchmark volumes); shape (n_cosets, E2, E1, E0)."""
    import torch
    dim, _, cosets = LATTICES[lattice]
    shape = (len(cosets),) + tuple(int(v) for v in reversed(list(ext)[:dim]))
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    c = torch.rand(shape, generator=g, device=device, dtype=torch.float32) * 2.0 - 1.0
    return c if dtype is None else c.to(dtype)


def points_uniform_torch(n: int, lo, hi, seed: int, device="cuda"):
    """n points ~ U(box) drawn on the device with a seeded torch generator."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    lo_t = torch.tensor(list(lo), dtype=torch.float32, device=device)
    hi_t = torch.tensor(list(hi), dtype=torch.float32, device=device)
    return lo_t + (hi_t - lo_t) * torch.rand((n, len(lo)), generator=g, device=device, dtype=torch.float32)
