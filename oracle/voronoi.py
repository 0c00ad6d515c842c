"""FP64 oracle for the second-order Voronoi splines (test infrastructure only).

The paper's Voronoi-spline study (Sec. 5, Voronoi splines) evaluates, on the
BCC and FCC lattices, the splines built from the indicator of the lattice's
Voronoi cell P: the order-2 one is the convolution of that indicator with
itself, normalised to a partition of unity,

    phi(x) = (chi_P * chi_P)(x) / vol(P) = vol(P n (P + x)) / vol(P),

(the translates of P tile space, so sum_n phi(x - n) = 1 and the integral of
phi is vol(P) = |det L|).  On the Cartesian lattice P is the unit cube and phi
is the tensor-product hat function.  This module computes phi by that
definition: P from its half-spaces {y : v.y <= |v|^2 / 2} over the short
lattice vectors v, the intersection with its translate by x as a half-space
intersection, and its volume as a convex hull (Qhull through scipy, FP64).
Eq. 1 then sums c_n phi(x - n) over every stored site within the support 2P.
Shares nothing with the product path; only tests/ use it.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass
from typing import Sequence, Tuple

import numpy as np
from scipy.spatial import ConvexHull, HalfspaceIntersection


@dataclass(frozen=True)
class VoronoiSpec:
    """A lattice given as Cartesian cosets of scale * Z^3 and its stored extent."""
    name: str
    scale: int
    cosets: Tuple[Tuple[int, int, int], ...]
    det: float
    ext: Tuple[int, int, int] = (1, 1, 1)

    def with_extent(self, ext: Sequence[int]) -> "VoronoiSpec":
        return VoronoiSpec(self.name, self.scale, self.cosets, self.det, tuple(int(e) for e in ext))

    def n_coef(self) -> int:
        return len(self.cosets) * int(np.prod(self.ext))

    def contains(self, n) -> bool:
        return any(all((n[i] - l[i]) % self.scale == 0 for i in range(3)) for l in self.cosets)


CC = VoronoiSpec("voronoi2_cc", 1, ((0, 0, 0),), 1.0)
BCC = VoronoiSpec("voronoi2_bcc", 2, ((0, 0, 0), (1, 1, 1)), 4.0)
FCC = VoronoiSpec("voronoi2_fcc", 2, ((0, 0, 0), (1, 1, 0), (1, 0, 1), (0, 1, 1)), 2.0)


def cell_halfspaces(spec: VoronoiSpec, radius2: int = 8) -> Tuple[np.ndarray, np.ndarray]:
    """Rows (v, |v|^2 / 2) for every lattice vector 0 < |v|^2 <= radius2: the
    Voronoi cell of the origin is {y : v.y <= |v|^2 / 2 for all of them}."""
    r = int(np.ceil(np.sqrt(radius2)))
    A, b = [], []
    for v in itertools.product(range(-r, r + 1), repeat=3):
        n2 = sum(x * x for x in v)
        if 0 < n2 <= radius2 and spec.contains(v):
            A.append(v)
            b.append(n2 / 2.0)
    return np.array(A, dtype=np.float64), np.array(b, dtype=np.float64)


def _overlap_volume(A: np.ndarray, b: np.ndarray, x: np.ndarray) -> float:
    """vol(P n (P + x)) for P = {A y <= b} (centrally symmetric)."""
    rhs = np.minimum(b, b + A @ x)
    mid = 0.5 * x                        # interior whenever x lies inside 2P
    slack = rhs - A @ mid
    if np.min(slack) <= 1e-12 * np.max(np.abs(b)):
        return 0.0
    hs = np.hstack([A, -rhs[:, None]])
    try:
        pts = HalfspaceIntersection(hs, mid).intersections
        return float(ConvexHull(pts).volume)
    except Exception:                     # a sliver too thin for Qhull: volume ~ 0
        return 0.0


def phi(spec: VoronoiSpec, y: np.ndarray) -> np.ndarray:
    """phi at points y (n, 3)."""
    A, b = cell_halfspaces(spec)
    vol = _overlap_volume(A, b, np.zeros(3))
    y = np.atleast_2d(np.asarray(y, dtype=np.float64))
    return np.array([_overlap_volume(A, b, v) / vol for v in y])


def _sites_near(spec: VoronoiSpec, x: np.ndarray, reach: float):
    lo = np.floor(x - reach).astype(int)
    hi = np.ceil(x + reach).astype(int)
    for n in itertools.product(*[range(lo[i], hi[i] + 1) for i in range(3)]):
        if not spec.contains(n):
            continue
        for j, l in enumerate(spec.cosets):
            if all((n[i] - l[i]) % spec.scale == 0 for i in range(3)):
                q = [(n[i] - l[i]) // spec.scale for i in range(3)]
                if all(0 <= q[i] < spec.ext[i] for i in range(3)):
                    yield n, j * int(np.prod(spec.ext)) + q[0] + spec.ext[0] * (q[1] + spec.ext[1] * q[2])
                break


def eval_sum(spec: VoronoiSpec, coef: np.ndarray, pts: np.ndarray) -> np.ndarray:
    """Eq. 1: f(x) = sum over stored sites n of c_n phi(x - n) (coset-major
    coefficients, axis 0 fastest; sites outside the arrays contribute 0)."""
    A, b = cell_halfspaces(spec)
    vol = _overlap_volume(A, b, np.zeros(3))
    verts = HalfspaceIntersection(np.hstack([A, -b[:, None]]), np.zeros(3)).intersections
    reach = 2.0 * float(np.max(np.abs(verts))) + 1e-9           # the support 2P lies in this box
    coef = np.asarray(coef, dtype=np.float64).ravel()
    out = np.zeros(len(pts))
    for i, x in enumerate(np.asarray(pts, dtype=np.float64)):
        s = 0.0
        for n, idx in _sites_near(spec, x, reach):
            w = _overlap_volume(A, b, x - np.asarray(n, dtype=np.float64))
            if w > 0.0:
                s += coef[idx] * w
        out[i] = s / vol
    return out


def eval_sum_grad(spec: VoronoiSpec, coef: np.ndarray, pts: np.ndarray, h: float = 1e-5):
    """f and grad f: the gradient by central differences of Eq. 1 (h = 1e-5;
    the pieces are cubic, so the difference error is O(h^2) inside a piece;
    points within h of a knot plane get a one-sided mixture)."""
    pts = np.asarray(pts, dtype=np.float64)
    f = eval_sum(spec, coef, pts)
    g = np.zeros((len(pts), 3))
    for i in range(3):
        e = np.zeros(3)
        e[i] = h
        g[:, i] = (eval_sum(spec, coef, pts + e) - eval_sum(spec, coef, pts - e)) / (2 * h)
    return f, g


def adjoint(spec: VoronoiSpec, pts: np.ndarray, g: np.ndarray) -> np.ndarray:
    """dc_n = sum_p g_p phi(x_p - n), coset-major like the coefficients."""
    A, b = cell_halfspaces(spec)
    vol = _overlap_volume(A, b, np.zeros(3))
    verts = HalfspaceIntersection(np.hstack([A, -b[:, None]]), np.zeros(3)).intersections
    reach = 2.0 * float(np.max(np.abs(verts))) + 1e-9
    dc = np.zeros(spec.n_coef())
    for x, gp in zip(np.asarray(pts, dtype=np.float64), np.asarray(g, dtype=np.float64).ravel()):
        for n, idx in _sites_near(spec, x, reach):
            dc[idx] += gp * _overlap_volume(A, b, x - np.asarray(n, dtype=np.float64)) / vol
    return dc
