"""Sub-region tables: the representation the code generator consumes.

Sec. 3 (Background) describes the input to code generation: a shift-invariant
region of evaluation (ROE), dissected into sub-regions, each holding one
polynomial in the coefficients of a fixed list of lattice sites, with symmetric
sub-regions related by rigid transforms to a few reference sub-regions (Fig. 1).
Part I of the paper produces it; that analysis is not part of this paper, so
this module derives it for the box splines used here:

1. ROE: the Voronoi cell of the lattice (or the parallelepiped L[0,1)^s), as in
   the region-of-evaluation block of Sec. 4.1.
2. Symmetry: when the lattice and the direction multiset are invariant under all
   signed permutations, every point of the ROE is mapped into the chamber
   y_0 >= y_1 >= ... >= y_{s-1} >= 0 by one of them; the sub-regions of the ROE
   are then images of the sub-regions of ROE n chamber (their transforms T, t
   of Algorithm 1 are the signed permutations, with t = 0).
3. Reference sub-regions: ROE n chamber is cut by the knot planes of the
   shifted basis functions that cross it; each cell carries one polynomial per
   site.  Cells with identical tables are merged.  The cutting planes become the
   BSP tests of Sec. 4.1 (bit i set iff p_i . y - d_i >= 0), the realised bit
   patterns map through the LUT sigma(q mod p) to reference sub-regions.
4. Per reference sub-region: the stencil (sites s_j with phi(y - s_j) not
   identically zero there) and the weight polynomials w_j(y) = phi(y - s_j),
   exact, re-expanded about a dyadic centre of the region for FP32 evaluation.

Tensor-product splines are additionally given as per-axis 1D tables so that the
generator can emit the separable form.
"""
from __future__ import annotations

import itertools
import random
from dataclasses import dataclass, field
from fractions import Fraction
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from .boxpieces import BoxPieces, NotGenericError, dot, knot_normals, knot_offsets, rank
from .exactpoly import Poly, monomials_upto

Vec = Tuple[int, ...]


# ---------------------------------------------------------------------------
# inputs
# ---------------------------------------------------------------------------

@dataclass(frozen=True)
class Lattice:
    """A lattice stored as Cartesian cosets of scale*Z^s: site = scale*i + coset[j]."""
    name: str
    dim: int
    scale: int
    cosets: Tuple[Vec, ...]
    generator: Tuple[Vec, ...]          # columns of L (lattice = L Z^s)

    def det(self) -> int:
        from .boxpieces import det
        return abs(int(det(self.generator)))

    def contains(self, n: Sequence[int]) -> bool:
        return any(all((n[i] - l[i]) % self.scale == 0 for i in range(self.dim))
                   for l in self.cosets)

    def coset_of(self, n: Sequence[int]) -> int:
        for j, l in enumerate(self.cosets):
            if all((n[i] - l[i]) % self.scale == 0 for i in range(self.dim)):
                return j
        raise ValueError(f"{n} is not a lattice site")

    def sites_in_box(self, lo: Sequence[int], hi: Sequence[int]):
        rng = [range(int(lo[i]), int(hi[i]) + 1) for i in range(self.dim)]
        return [n for n in itertools.product(*rng) if self.contains(n)]


@dataclass(frozen=True)
class Spline:
    name: str
    lattice: Lattice
    dirs: Tuple[Vec, ...]
    roe: str = "voronoi"                 # "voronoi" | "parallelepiped"
    kind: str = "box"                    # "box": box spline of dirs; "voronoi2": second-order Voronoi spline


# ---------------------------------------------------------------------------
# outputs
# ---------------------------------------------------------------------------

@dataclass
class RefRegion:
    """One reference sub-region: f(y) = sum_j c[k + R^T s_j] w_j(y_ref - center)."""
    sites: List[Vec]
    center: Tuple[Fraction, ...]
    weights: List[Poly]                  # w_j in local coordinates u = y_ref - center
    monomials: List[Tuple[int, ...]]

    def coef_matrix(self) -> List[List[Fraction]]:
        return [w.coeff_vector(self.monomials) for w in self.weights]


@dataclass
class Axis1D:
    """Per-axis factor of a tensor-product spline on the parallelepiped ROE."""
    sites: List[int]
    center: Fraction
    weights: List[Poly]                  # univariate, in u = y - center
    degree: int


@dataclass
class Table:
    spline: Spline
    fold: str                            # "hyperoctahedral" | "none"
    planes: List[Tuple[Tuple[Fraction, ...], Fraction]]   # BSP planes (p_i, d_i) in ROE n chamber
    bsp_mod: int                         # p
    sigma: List[int]                     # LUT of size p -> reference region (or -1: unused)
    regions: List[RefRegion]
    separable: Optional[List[Axis1D]] = None
    degree: int = 0
    support_halfwidth: Tuple[Fraction, ...] = ()
    # the same regions expanded about their dyadic centroids (an alternative the
    # autotuner may pick: more FMAs, different register/load schedule)
    regions_centroid: Optional[List[RefRegion]] = None

    def region_of(self, y_ref: Sequence[float]) -> int:
        q = 0
        for i, (p, d) in enumerate(self.planes):
            if sum(float(a) * b for a, b in zip(p, y_ref)) - float(d) >= 0:
                q |= 1 << i
        return self.sigma[q % self.bsp_mod]


# ---------------------------------------------------------------------------
# geometry helpers
# ---------------------------------------------------------------------------

def _half_sum(dirs) -> Tuple[Fraction, ...]:
    s = len(dirs[0])
    return tuple(Fraction(sum(d[i] for d in dirs), 2) for i in range(s))


def _voronoi_constraints(lat: Lattice):
    """a . y <= b with a = n, b = |n|^2 / 2 for lattice vectors near the origin."""
    r = lat.scale
    out = []
    for n in lat.sites_in_box([-r] * lat.dim, [r] * lat.dim):
        if any(n):
            out.append((tuple(Fraction(v) for v in n), Fraction(dot(n, n), 2)))
    return out


def _parallelepiped_constraints(lat: Lattice):
    from .boxpieces import solve
    s = lat.dim
    # rows of L^-1: y = L w, 0 <= w <= 1
    Linv_rows = []
    for i in range(s):
        e = [0] * s
        e[i] = 1
        # solve L^T r = e_i  -> r is row i of L^-1
        LT = [[lat.generator[j][k] for j in range(s)] for k in range(s)]   # columns of L^T
        Linv_rows.append(tuple(solve(LT, e)))
    out = []
    for r in Linv_rows:
        out.append((r, Fraction(1)))
        out.append((tuple(-v for v in r), Fraction(0)))
    return out


def _chamber_constraints(s: int):
    """y_0 >= y_1 >= ... >= y_{s-1} >= 0 as a . y <= 0."""
    out = []
    for i in range(s - 1):
        a = [Fraction(0)] * s
        a[i], a[i + 1] = Fraction(-1), Fraction(1)
        out.append((tuple(a), Fraction(0)))
    a = [Fraction(0)] * s
    a[s - 1] = Fraction(-1)
    out.append((tuple(a), Fraction(0)))
    return out


def _nonredundant(cons):
    """Drop half-spaces that never bind (float LP per constraint; bounded polytope)."""
    from scipy.optimize import linprog
    s = len(cons[0][0])
    A = np.array([[float(v) for v in a] for a, _ in cons])
    b = np.array([float(v) for _, v in cons])
    keep = []
    for i in range(len(cons)):
        others = [j for j in range(len(cons)) if j != i]
        A2 = np.vstack([A[others], A[i:i + 1]])
        b2 = np.concatenate([b[others], [b[i] + 1.0]])
        res = linprog(-A[i], A_ub=A2, b_ub=b2, bounds=[(None, None)] * s, method="highs")
        if res.status == 0 and -res.fun > b[i] + 1e-9:
            keep.append(cons[i])
        elif res.status != 0:
            keep.append(cons[i])
    return keep


def _vertices(cons):
    """Exact vertices of {y : a.y <= b for all (a, b)} (bounded polytope)."""
    from .boxpieces import solve
    cons = _nonredundant(cons)
    s = len(cons[0][0])
    verts = set()
    for idx in itertools.combinations(range(len(cons)), s):
        A = [cons[i][0] for i in idx]
        if rank(A) < s:
            continue
        cols = [[A[r][c] for r in range(s)] for c in range(s)]
        y = tuple(solve(cols, [cons[i][1] for i in idx]))
        if all(dot(a, y) <= b for a, b in cons):
            verts.add(y)
    return sorted(verts)


def _chebyshev(cons):
    """Centre and radius of the largest ball in {a.y <= b} (float LP)."""
    from scipy.optimize import linprog
    s = len(cons[0][0])
    A = np.array([[float(v) for v in a] + [float(np.linalg.norm([float(v) for v in a]))]
                  for a, _ in cons])
    b = np.array([float(b) for _, b in cons])
    c = np.zeros(s + 1)
    c[-1] = -1.0
    res = linprog(c, A_ub=A, b_ub=b, bounds=[(None, None)] * s + [(0, None)], method="highs")
    if not res.success:
        return None, 0.0
    return res.x[:s], res.x[-1]


def _symmetric_under_signed_perms(spl: Spline) -> bool:
    s = spl.lattice.dim
    canon = sorted(_canon_dir(d) for d in spl.dirs)
    for perm in itertools.permutations(range(s)):
        for sg in itertools.product((1, -1), repeat=s):
            img = sorted(_canon_dir(tuple(sg[i] * d[perm[i]] for i in range(s))) for d in spl.dirs)
            if img != canon:
                return False
            for l in spl.lattice.cosets:
                if not spl.lattice.contains(tuple(sg[i] * l[perm[i]] for i in range(s))):
                    return False
    return True


def _canon_dir(d):
    for v in d:
        if v != 0:
            return tuple(d) if v > 0 else tuple(-x for x in d)
    return tuple(d)


# ---------------------------------------------------------------------------
# the builder
# ---------------------------------------------------------------------------

class TableBuilder:
    def __init__(self, spline: Spline, seed: int = 12345):
        self.spl = spline
        self.s = spline.lattice.dim
        self.bp = BoxPieces()
        self.half = _half_sum(spline.dirs) if spline.dirs else (Fraction(0),) * self.s
        self.detL = spline.lattice.det()
        self.rng = random.Random(seed)
        self.hw = tuple(Fraction(sum(abs(d[i]) for d in spline.dirs), 2) for i in range(self.s))
        self.degree = len(spline.dirs) - self.s

    def _symmetric(self) -> bool:
        return _symmetric_under_signed_perms(self.spl)

    # weight polynomial w(y) = |det L| M(y - n + half) of site n near generic y*
    def weight(self, n: Vec, ystar) -> Poly:
        z = tuple(ystar[i] - n[i] + self.half[i] for i in range(self.s))
        if any(abs(z[i] - self.half[i]) >= self.hw[i] for i in range(self.s)):
            return Poly(self.s)
        p = self.bp.piece(self.spl.dirs, z)
        if p.is_zero():
            return p
        return p.shift([self.half[i] - n[i] for i in range(self.s)]).scale(self.detL)

    def _stencil_at(self, ystar):
        lo = [int(np.floor(float(ystar[i] - self.hw[i]))) - 1 for i in range(self.s)]
        hi = [int(np.ceil(float(ystar[i] + self.hw[i]))) + 1 for i in range(self.s)]
        out = {}
        for n in self.spl.lattice.sites_in_box(lo, hi):
            w = self.weight(n, ystar)
            if not w.is_zero():
                out[n] = w
        return out

    def _generic_point(self, cons):
        """A rational point strictly inside the polytope, generic for all knot planes."""
        ctr, rad = _chebyshev(cons)
        if ctr is None or rad < 1e-9:
            return None
        for _ in range(200):
            jit = [self.rng.uniform(-0.3, 0.3) * rad for _ in range(self.s)]
            y = tuple(Fraction(float(ctr[i] + jit[i])).limit_denominator(997 * 1009)
                      for i in range(self.s))
            if not all(dot(a, y) < b for a, b in cons):
                continue
            try:
                return y, self._stencil_at(y)
            except NotGenericError:
                continue
        raise RuntimeError("no generic interior point found")

    def _cutting_planes(self, cons):
        """Knot planes of the shifted basis functions that cross the polytope's interior."""
        verts = _vertices(cons)
        lat = self.spl.lattice
        planes = []
        for nu in knot_normals(self.spl.dirs):
            vals = [dot(nu, v) for v in verts]
            lo, hi = min(vals), max(vals)
            # plane of phi(. - n): nu.y = nu.n + (subset sum) - nu.half
            sub = knot_offsets(self.spl.dirs, nu)
            nh = dot(nu, self.half)
            r = int(np.ceil(float(max(abs(lo), abs(hi))))) + max(abs(x) for x in sub) + 2 * lat.scale
            shifts = set()
            for n in lat.sites_in_box([-r] * self.s, [r] * self.s):
                shifts.add(dot(nu, n))
            offs = sorted({Fraction(a + b) - nh for a in shifts for b in sub})
            for d in offs:
                if lo < d < hi:
                    planes.append((tuple(Fraction(v) for v in nu), d))
        return planes

    def build(self) -> Table:
        spl = self.spl
        s = self.s
        if spl.roe == "voronoi":
            base = _voronoi_constraints(spl.lattice)
        else:
            base = _parallelepiped_constraints(spl.lattice)
        fold = "none"
        cons = list(base)
        if spl.roe == "voronoi" and not self._axis_aligned():
            if not self._symmetric():
                raise NotImplementedError("Voronoi ROE without full signed-permutation symmetry")
            fold = "hyperoctahedral"
            cons += _chamber_constraints(s)
        planes = self._cutting_planes(cons)
        # cells of the arrangement: split by each plane in turn
        cells = [([], cons)]          # (sign vector so far, constraints)
        for (p, d) in planes:
            nxt = []
            for signs, cc in cells:
                below = cc + [(p, d)]                                   # p.y - d <= 0
                above = cc + [(tuple(-v for v in p), -d)]               # p.y - d >= 0
                for sg, c2 in ((0, below), (1, above)):
                    _, rad = _chebyshev(c2)
                    if rad > 1e-9:
                        nxt.append((signs + [sg], c2))
            cells = nxt
        # tables per cell; merge identical ones
        regions: List[Tuple[Dict, List]] = []      # (stencil dict, list of (q, cons))
        q_to_region: Dict[int, int] = {}
        for signs, cc in cells:
            found = self._generic_point(cc)
            if found is None:
                continue
            ystar, st = found
            q = sum(b << i for i, b in enumerate(signs))
            match = None
            for r, (st2, members) in enumerate(regions):
                if set(st2) == set(st) and all(st2[n] == st[n] for n in st):
                    match = r
                    break
            if match is None:
                regions.append((st, [(q, cc)]))
                match = len(regions) - 1
            else:
                regions[match][1].append((q, cc))
            q_to_region[q] = match
        # drop planes that separate nothing (all cells on both sides share a table)
        planes, q_to_region = _prune_planes(planes, q_to_region)
        # BSP compression: smallest p with collision-free q mod p
        p = 1
        while True:
            lut = {}
            ok = True
            for q, r in q_to_region.items():
                if lut.setdefault(q % p, r) != r:
                    ok = False
                    break
            if ok:
                break
            p += 1
        sigma = [-1] * p
        for q, r in q_to_region.items():
            sigma[q % p] = r
        # reference regions in local coordinates
        degree = self.degree
        mons = monomials_upto(s, degree)
        refs = []
        refs_c = []
        for st, members in regions:
            verts = []
            for _, cc in members:
                verts += _vertices(cc)
            sites = sorted(st, key=lambda n: (tuple(abs(v) for v in n), n))
            if spl.roe == "parallelepiped":
                # tensor-product splines are evaluated from their per-axis factors;
                # the full table (kept for checks) is expanded about the centroid
                vf = [[float(x) for x in v] for v in verts]
                cen = tuple(Fraction(round(sum(v[i] for v in vf) / len(vf) * 64), 64) for i in range(s))
            else:
                cen = _choose_center([st[n] for n in sites], verts, [cc for _, cc in members], degree, self.rng)
            weights = [st[n].shift(cen) for n in sites]
            refs.append(RefRegion(sites=sites, center=cen, weights=weights, monomials=mons))
            vf = [[float(x) for x in v] for v in verts]
            cc0 = tuple(Fraction(round(sum(v[i] for v in vf) / len(vf) * 64), 64) for i in range(s))
            refs_c.append(RefRegion(sites=sites, center=cc0, weights=[st[n].shift(cc0) for n in sites],
                                    monomials=mons))
        table = Table(spline=spl, fold=fold, planes=planes, bsp_mod=p, sigma=sigma,
                      regions=refs, degree=degree, support_halfwidth=self.hw, regions_centroid=refs_c)
        table.separable = self._separable()
        return table

    def _axis_aligned(self) -> bool:
        """Every direction is a unit coordinate vector on the Cartesian grid."""
        spl = self.spl
        if spl.lattice.scale != 1 or len(spl.lattice.cosets) != 1:
            return False
        return all(sum(1 for v in d if v != 0) == 1 and sum(abs(v) for v in d) == 1 for d in spl.dirs)

    def _separable(self) -> Optional[List[Axis1D]]:
        """Per-axis 1D tables when every direction is a coordinate axis: the
        region of evaluation is [0,1)^s (parallelepiped, centre 1/2) or the
        Voronoi cube [-1/2,1/2]^s (centre 0); the 1D factor must be a single
        polynomial piece there."""
        spl = self.spl
        s = self.s
        if not self._axis_aligned():
            return None
        cen = Fraction(1, 2) if spl.roe == "parallelepiped" else Fraction(0)
        axes = []
        for i in range(s):
            mult = 0
            for d in spl.dirs:
                nz = [k for k in range(s) if d[k] != 0]
                if len(nz) != 1 or abs(d[nz[0]]) != 1:
                    return None
                if nz[0] == i:
                    mult += 1
            if mult == 0:
                return None
            bp = BoxPieces()
            half = Fraction(mult, 2)
            # knots of the centred factor lie at z - half - n = integers: inside the
            # region only at its boundary when mult is even (parallelepiped) or odd (Voronoi)
            if (mult % 2 == 0) != (spl.roe == "parallelepiped"):
                return None
            ystar = cen + Fraction(1, 1009)
            sites, weights = [], []
            for n in range(-mult, mult + 1):
                z = (ystar - n + half,)
                if not (0 < z[0] < mult):
                    continue
                pc = bp.piece([(1,)] * mult, z)
                if pc.is_zero():
                    continue
                sites.append(n)
                weights.append(pc.shift([half - n]).shift([cen]))
            axes.append(Axis1D(sites=sites, center=cen, weights=weights, degree=mult - 1))
        return axes


def _dense(poly: Poly, deg: int, dim: int) -> np.ndarray:
    a = np.zeros((deg + 1,) * dim)
    for e, v in poly.c.items():
        a[e] = float(v)
    return a


def _shift_dense(a: np.ndarray, c) -> np.ndarray:
    """Coefficients of p(u + c) from those of p(u) (binomial matrix per axis)."""
    from math import comb
    deg = a.shape[0] - 1
    for ax, cv in enumerate(c):
        T = np.zeros((deg + 1, deg + 1))
        for i in range(deg + 1):
            for j in range(i, deg + 1):
                T[i, j] = comb(j, i) * cv ** (j - i)
        a = np.moveaxis(np.tensordot(T, np.moveaxis(a, ax, 0), axes=(1, 0)), 0, ax)
    return a


def _choose_center(weights, verts, cells, deg, rng):
    """Expansion point of a reference sub-region's polynomials for FP32
    evaluation.  The generated kernel spends one FMA per nonzero monomial
    coefficient, and the FP32 rounding error of the Horner forms grows with
    B(u) = sum_j sum_a |coef_ja| |u|^a over the region.  Among the points of the
    1/8 grid inside the region's bounding box, take the one with the fewest
    nonzero coefficients whose max B stays within 10 % of that of the dyadic
    centroid (1/64 grid); ties go to the smaller B."""
    dim = len(verts[0])
    vf = np.array([[float(x) for x in v] for v in verts])
    centroid = tuple(Fraction(round(float(vf[:, i].mean()) * 64), 64) for i in range(dim))
    # samples of the region (rejection in the bounding box against the cells' constraints)
    lo, hi = vf.min(0), vf.max(0)
    pts = []
    tries = 0
    while len(pts) < 4000 and tries < 200:
        tries += 1
        cand = lo + (hi - lo) * np.array([[rng.random() for _ in range(dim)] for _ in range(2000)])
        ok = np.zeros(len(cand), bool)
        for cc in cells:
            A = np.array([[float(x) for x in a] for a, _ in cc])
            b = np.array([float(x) for _, x in cc])
            ok |= np.all(cand @ A.T <= b + 1e-12, axis=1)
        pts.extend(cand[ok].tolist())
    if not pts:
        return centroid
    Y = np.array(pts[:4000])
    dense = [_dense(w, deg, dim) for w in weights]
    exps = np.array(list(np.ndindex(*(deg + 1,) * dim)))

    def score(c):
        cf = [float(x) for x in c]
        U = np.abs(Y - np.array(cf))
        powers = np.prod(U[:, None, :] ** exps[None, :, :], axis=2)          # (npts, nmono)
        nnz, absum = 0, np.zeros(len(exps))
        for a in dense:
            sh = _shift_dense(a, cf).reshape(-1)
            nz = np.abs(sh) > 1e-12
            nnz += int(nz.sum())
            absum += np.abs(sh) * nz
        return nnz, float((powers @ absum).max())

    base_nnz, base_b = score(centroid)
    best = (base_nnz, base_b, centroid)
    g0 = [int(np.floor(lo[i] * 8)) for i in range(dim)]
    g1 = [int(np.ceil(hi[i] * 8)) for i in range(dim)]
    for idx in itertools.product(*[range(g0[i], g1[i] + 1) for i in range(dim)]):
        c = tuple(Fraction(v, 8) for v in idx)
        nnz, b = score(c)
        if b <= 1.1 * base_b and (nnz, b) < best[:2]:
            best = (nnz, b, c)
    return best[2]


def _prune_planes(planes, q_to_region):
    """Remove BSP planes whose bit never changes the region."""
    keep = list(range(len(planes)))
    changed = True
    while changed:
        changed = False
        for bit_pos, pi in enumerate(list(keep)):
            b = keep.index(pi)
            useful = False
            for q, r in q_to_region.items():
                q2 = q ^ (1 << b)
                if q2 in q_to_region and q_to_region[q2] != r:
                    useful = True
                    break
            if not useful:
                # drop bit b: re-index q
                newmap = {}
                for q, r in q_to_region.items():
                    lowmask = (1 << b) - 1
                    nq = (q & lowmask) | ((q >> (b + 1)) << b)
                    newmap[nq] = r
                q_to_region = newmap
                keep.remove(pi)
                changed = True
                break
    return [planes[i] for i in keep], q_to_region


class VoronoiTableBuilder(TableBuilder):
    """The same construction for the second-order Voronoi spline of a lattice
    (Sec. 5, Voronoi splines): phi(x) = vol(P n (P + x)) / vol(P) for the
    Voronoi cell P, whose exact cubic pieces and knot planes come from
    voronoi.OverlapPieces instead of the box-spline recurrence."""

    def __init__(self, spline: Spline, seed: int = 12345):
        from .voronoi import OverlapPieces
        super().__init__(spline, seed)
        self.op = OverlapPieces(_nonredundant(_voronoi_constraints(spline.lattice)))
        self.half = (Fraction(0),) * self.s
        self.hw = self.op.support_halfwidth()
        self.degree = 3

    def _symmetric(self) -> bool:
        lat = self.spl.lattice
        s = self.s
        return all(lat.contains(tuple(sg[i] * l[perm[i]] for i in range(s)))
                   for perm in itertools.permutations(range(s)) for sg in itertools.product((1, -1), repeat=s)
                   for l in lat.cosets)

    def _axis_aligned(self) -> bool:
        return False

    def _separable(self):
        return None

    def weight(self, n: Vec, ystar) -> Poly:
        x = tuple(ystar[i] - n[i] for i in range(self.s))
        if any(abs(x[i]) >= self.hw[i] for i in range(self.s)):
            return Poly(self.s)
        p = self.op.piece(x)
        if p.is_zero():
            return p
        return p.shift([-Fraction(v) for v in n])

    def _cutting_planes(self, cons):
        verts = _vertices(cons)
        lat = self.spl.lattice
        lo_box = [min(v[i] for v in verts) - self.hw[i] for i in range(self.s)]
        hi_box = [max(v[i] for v in verts) + self.hw[i] for i in range(self.s)]
        sites = list(lat.sites_in_box([int(np.floor(float(x))) for x in lo_box],
                                      [int(np.ceil(float(x))) for x in hi_box]))
        planes = set()
        for nu, d in self.op.knot_planes():
            vals = [dot(nu, v) for v in verts]
            lo, hi = min(vals), max(vals)
            for n in sites:
                dd = d + dot(nu, n)
                if lo < dd < hi:
                    planes.add((tuple(Fraction(v) for v in nu), Fraction(dd)))
        return sorted(planes)


def build_table(spline: Spline, seed: int = 12345) -> Table:
    if spline.kind == "voronoi2":
        return VoronoiTableBuilder(spline, seed).build()
    return TableBuilder(spline, seed).build()
