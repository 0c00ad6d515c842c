"""Second-order Voronoi splines: exact polynomial pieces for the table builder.

The Voronoi splines of the paper's Voronoi study (Sec. 5) are built from the
indicator of the lattice's Voronoi cell P.  The second-order one is

    phi(x) = vol(P n (P + x)) / vol(P)

(the indicator convolved with itself, normalised to a partition of unity).
For x in an open cell of the arrangement of "knot" planes below, the
intersection Q(x) = P n (P + x) keeps one combinatorial type: the same
facets, and vertices that each solve the same three facet equations, whose
right-hand sides are affine in x.  Its volume, summed over fan triangles of
the faces as (1/6) det(v_0, v_j, v_j+1), is then one cubic polynomial in x.
This module finds that type at a generic rational point exactly and returns
the polynomial (exact rationals).

Knot planes in x: a facet of P and the parallel facet of P + x change roles
(a_i . x = 0); a vertex of one polytope crosses a facet plane of the other
(a_i . x = a_i . w - b_i or b_i - a_i . w for vertices w of P); an edge of P
crosses an edge of P + x (normal e x f through w - u for edges from w and u).
"""
from __future__ import annotations

import itertools
import math
from fractions import Fraction
from typing import Dict, List, Sequence, Tuple

from .boxpieces import NotGenericError, rank, solve
from .exactpoly import Poly

Vec = Tuple[Fraction, ...]


def _dot(a, b):
    return sum(x * y for x, y in zip(a, b))


def _cross(a, b):
    return (a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0])


def _primitive(v):
    """Integer multiple of v with coprime entries and a positive first nonzero entry."""
    den = 1
    for x in v:
        den = den * Fraction(x).denominator // math.gcd(den, Fraction(x).denominator)
    iv = [int(Fraction(x) * den) for x in v]
    g = 0
    for x in iv:
        g = math.gcd(g, abs(x))
    iv = [x // g for x in iv]
    for x in iv:
        if x:
            if x < 0:
                iv = [-y for y in iv]
            break
    return tuple(Fraction(x) for x in iv), Fraction(g, den)


class OverlapPieces:
    """Exact pieces of phi(x) = vol(P n (P + x)) / vol(P) for a Voronoi cell P
    given by its facets a . y <= b (centrally symmetric, rational)."""

    def __init__(self, facets: Sequence[Tuple[Sequence, Fraction]]):
        self.facets = [(tuple(Fraction(v) for v in a), Fraction(b)) for a, b in facets]
        self.verts, self.edges = self._skeleton()
        self.vol = self._volume_at((Fraction(0),) * 3)
        if self.vol <= 0:
            raise ValueError("the cell has no volume")
        self.memo: Dict[tuple, Poly] = {}

    # -- the cell's own vertices and edges -----------------------------------------
    def _skeleton(self):
        verts = {}
        for i, j, k in itertools.combinations(range(len(self.facets)), 3):
            A = [self.facets[t][0] for t in (i, j, k)]
            if rank(A) < 3:
                continue
            v = tuple(solve([[A[r][c] for r in range(3)] for c in range(3)], [self.facets[t][1] for t in (i, j, k)]))
            if all(_dot(a, v) <= b for a, b in self.facets):
                verts.setdefault(v, set()).update((i, j, k))
        vs = list(verts)
        tight = {v: {i for i, (a, b) in enumerate(self.facets) if _dot(a, v) == b} for v in vs}
        edges = []
        for u, w in itertools.combinations(vs, 2):
            common = tight[u] & tight[w]
            if len(common) >= 2 and rank([self.facets[i][0] for i in common]) == 2:
                edges.append((u, w))
        return vs, edges

    def support_halfwidth(self) -> Tuple[Fraction, ...]:
        """Half-widths of the box holding the support 2P."""
        return tuple(2 * max(abs(v[i]) for v in self.verts) for i in range(3))

    # -- knot planes in x -----------------------------------------------------------------
    def knot_planes(self) -> List[Tuple[Vec, Fraction]]:
        """Distinct planes nu . x = d (nu primitive integer) where phi's piece can change."""
        out = set()

        def add(nu, d):
            if not any(nu):
                return
            p, g = _primitive(nu)
            out.add((p, Fraction(d) / g))

        for a, b in self.facets:
            add(a, Fraction(0))
            for w in self.verts:
                add(a, _dot(a, w) - b)
                add(a, b - _dot(a, w))
        for (w1, w2), (u1, u2) in itertools.product(self.edges, repeat=2):
            e = tuple(x - y for x, y in zip(w2, w1))
            f = tuple(x - y for x, y in zip(u2, u1))
            nu = _cross(e, f)
            if any(nu):
                add(nu, _dot(nu, tuple(x - y for x, y in zip(w1, u1))))
        return sorted(out)

    # -- the piece at a generic point ----------------------------------------------------
    def _type_at(self, x: Vec):
        """Binding side of each facet pair, and the vertices of Q(x) with their tight facets."""
        side = []
        for a, b in self.facets:
            ax = _dot(a, x)
            if ax == 0:
                raise NotGenericError("parallel facets coincide")
            side.append(1 if ax < 0 else 0)           # 1: the facet of P + x binds
        rhs = [b + (side[i] * _dot(a, x)) for i, (a, b) in enumerate(self.facets)]
        verts = {}
        n = len(self.facets)
        for i, j, k in itertools.combinations(range(n), 3):
            A = [self.facets[t][0] for t in (i, j, k)]
            if rank(A) < 3:
                continue
            v = tuple(solve([[A[r][c] for r in range(3)] for c in range(3)], [rhs[t] for t in (i, j, k)]))
            if v in verts:
                continue
            ok = True
            tight = []
            for t, (a, b) in enumerate(self.facets):
                s = _dot(a, v) - rhs[t]
                if s > 0:
                    ok = False
                    break
                if s == 0:
                    tight.append(t)
            if ok:
                if len({side[t] for t in tight}) > 1 and len(tight) > 3:
                    raise NotGenericError("a vertex of one cell on a facet of the other")
                verts[v] = tight
        return side, rhs, verts

    def _volume_at(self, x: Vec) -> Fraction:
        """Exact vol(Q(x)) (used for the cell itself and in checks)."""
        try:
            side, rhs, verts = self._type_at(x)
        except NotGenericError:
            side, rhs, verts = [0] * len(self.facets), [b for _, b in self.facets], None
            verts = {}
            n = len(self.facets)
            for i, j, k in itertools.combinations(range(n), 3):
                A = [self.facets[t][0] for t in (i, j, k)]
                if rank(A) < 3:
                    continue
                v = tuple(solve([[A[r][c] for r in range(3)] for c in range(3)], [rhs[t] for t in (i, j, k)]))
                if all(_dot(a, v) <= rhs[t] for t, (a, b) in enumerate(self.facets)):
                    verts[v] = [t for t, (a, b) in enumerate(self.facets) if _dot(a, v) == rhs[t]]
        vol = Fraction(0)
        for f, (a, _) in enumerate(self.facets):
            ring = self._face_ring(a, [v for v, tight in verts.items() if f in tight])
            for j in range(1, len(ring) - 1):
                vol += _dot(ring[0], _cross(ring[j], ring[j + 1])) / 6
        return vol

    @staticmethod
    def _face_ring(normal, pts):
        """The face's vertices in counter-clockwise order seen from outside."""
        if len(pts) < 3:
            return []
        c = tuple(sum(p[i] for p in pts) / len(pts) for i in range(3))
        u = tuple(pts[0][i] - c[i] for i in range(3))
        w = _cross(normal, u)
        uf = [float(t) for t in u]
        wf = [float(t) for t in w]

        def ang(p):
            d = [float(p[i] - c[i]) for i in range(3)]
            return math.atan2(sum(d[i] * wf[i] for i in range(3)), sum(d[i] * uf[i] for i in range(3)))

        return sorted(pts, key=ang)

    def piece(self, x: Sequence) -> Poly:
        """phi as a polynomial in x (3 variables), valid on the open cell of the
        knot-plane arrangement that holds the generic point x; 0 outside 2P."""
        x = tuple(Fraction(v) for v in x)
        side, rhs, verts = self._type_at(x)
        if len(verts) < 4:
            return Poly(3)
        key = (tuple(side), tuple(sorted((v, tuple(t)) for v, t in verts.items())))
        hit = self.memo.get(key)
        if hit is not None:
            return hit
        # affine vertex positions: three independent tight facets, right-hand sides affine in x
        rhs_poly = [Poly.linear([side[i] * a[c] for c in range(3)], b) for i, (a, b) in enumerate(self.facets)]
        vpoly = {}
        for v, tight in verts.items():
            trip = next(t for t in itertools.combinations(tight, 3) if rank([self.facets[i][0] for i in t]) == 3)
            A = [self.facets[i][0] for i in trip]
            # v(x) = A^-1 rhs(x): the columns of A^-1 from unit right-hand sides
            inv_cols = [solve([[A[r][c] for r in range(3)] for c in range(3)], [1 if r == k else 0 for r in range(3)])
                        for k in range(3)]
            vpoly[v] = [sum((rhs_poly[trip[k]].scale(inv_cols[k][c]) for k in range(3)), Poly(3)) for c in range(3)]
        vol = Poly(3)
        for f, (a, _) in enumerate(self.facets):
            ring = self._face_ring(a, [v for v, tight in verts.items() if f in tight])
            for j in range(1, len(ring) - 1):
                p0, p1, p2 = vpoly[ring[0]], vpoly[ring[j]], vpoly[ring[j + 1]]
                cr = [p1[1] * p2[2] - p1[2] * p2[1], p1[2] * p2[0] - p1[0] * p2[2], p1[0] * p2[1] - p1[1] * p2[0]]
                vol = vol + (p0[0] * cr[0] + p0[1] * cr[1] + p0[2] * cr[2]).scale(Fraction(1, 6))
        out = vol.scale(1 / self.vol)
        self.memo[key] = out
        return out
