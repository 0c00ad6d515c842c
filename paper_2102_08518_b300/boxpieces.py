"""Exact polynomial pieces of box splines.

Sec. 3 takes as given that a spline is a piecewise polynomial whose pieces are
known ("each sub-region contains a polynomial").  For the box splines the paper
benchmarks, this module derives those pieces exactly, in rational arithmetic,
from the convolution structure of the box spline:

    M_Xi(x) = integral_0^1 M_{Xi \\ xi}(x - t xi) dt      (Xi \\ xi still spanning),
    M_B(x)  = 1[0 < B^-1 x < 1] / |det B|               (|B| = s).

Along the segment x - t xi, t in [0, 1], M_{Xi \\ xi} is one polynomial between
consecutive crossings of its knot planes; for x near a generic point z the
crossings t_k(x) are affine in x and keep their order, so the integral is a
polynomial in x.  Since it agrees with M_Xi on a neighbourhood of z, it is the
polynomial of M_Xi on z's cell.  Pieces are memoised per (direction multiset,
cell of its knot-plane arrangement).

Knot planes of M_Xi: nu . x = nu . (sum of a sub-multiset of Xi), for every
normal nu orthogonal to s-1 independent columns of Xi.
"""
from __future__ import annotations

import bisect
from fractions import Fraction
from functools import lru_cache
from math import gcd
from typing import Dict, List, Sequence, Tuple

from .exactpoly import Poly

Vec = Tuple[int, ...]


# interior points of a breakpoint interval tried in turn (the midpoint first)
_INTERIOR = (Fraction(1, 2), Fraction(3, 7), Fraction(5, 9), Fraction(7, 19), Fraction(13, 29), Fraction(31, 53))


class NotGenericError(ValueError):
    """The evaluation point (or a derived point) sits on a knot plane or makes
    two crossings coincide; the caller retries with another point."""


# ---------------------------------------------------------------------------
# exact small linear algebra
# ---------------------------------------------------------------------------

def det(cols: Sequence[Sequence]) -> Fraction:
    """Determinant of the square matrix with the given columns."""
    n = len(cols)
    a = [[Fraction(cols[j][i]) for j in range(n)] for i in range(n)]
    d = Fraction(1)
    for c in range(n):
        p = next((r for r in range(c, n) if a[r][c] != 0), None)
        if p is None:
            return Fraction(0)
        if p != c:
            a[c], a[p] = a[p], a[c]
            d = -d
        d *= a[c][c]
        for r in range(c + 1, n):
            f = a[r][c] / a[c][c]
            for j in range(c, n):
                a[r][j] -= f * a[c][j]
    return d


def solve(cols: Sequence[Sequence], b: Sequence) -> List[Fraction]:
    """x with sum_j x_j cols[j] = b (square, nonsingular)."""
    n = len(cols)
    a = [[Fraction(cols[j][i]) for j in range(n)] + [Fraction(b[i])] for i in range(n)]
    for c in range(n):
        p = next((r for r in range(c, n) if a[r][c] != 0), None)
        if p is None:
            raise ZeroDivisionError("singular")
        a[c], a[p] = a[p], a[c]
        for r in range(n):
            if r != c and a[r][c] != 0:
                f = a[r][c] / a[c][c]
                for j in range(c, n + 1):
                    a[r][j] -= f * a[c][j]
    return [a[i][n] / a[i][i] for i in range(n)]


def rank(vectors: Sequence[Sequence]) -> int:
    if not vectors:
        return 0
    rows = [[Fraction(v) for v in vec] for vec in vectors]
    n = len(rows[0])
    r = 0
    for c in range(n):
        p = next((i for i in range(r, len(rows)) if rows[i][c] != 0), None)
        if p is None:
            continue
        rows[r], rows[p] = rows[p], rows[r]
        for i in range(len(rows)):
            if i != r and rows[i][c] != 0:
                f = rows[i][c] / rows[r][c]
                rows[i] = [a - f * b for a, b in zip(rows[i], rows[r])]
        r += 1
    return r


def dot(a: Sequence, b: Sequence):
    return sum(x * y for x, y in zip(a, b))


def _primitive(v: Sequence[int]) -> Vec:
    g = 0
    for x in v:
        g = gcd(g, abs(int(x)))
    v = tuple(int(x) // g for x in v)
    for x in v:
        if x != 0:
            return v if x > 0 else tuple(-y for y in v)
    return v


# ---------------------------------------------------------------------------
# knot-plane arrangement of a direction multiset
# ---------------------------------------------------------------------------

@lru_cache(maxsize=None)
def knot_normals(dirs: Tuple[Vec, ...]) -> Tuple[Vec, ...]:
    """Primitive integer normals of the hyperplanes spanned by s-1 independent columns."""
    s = len(dirs[0])
    out = set()
    if s == 1:
        return ((1,),)
    uniq = sorted(set(dirs))
    if s == 2:
        for d in uniq:
            if any(d):
                out.add(_primitive((-d[1], d[0])))
    elif s == 3:
        for i in range(len(uniq)):
            for j in range(i + 1, len(uniq)):
                u, v = uniq[i], uniq[j]
                n = (u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0])
                if any(n):
                    out.add(_primitive(n))
    else:
        raise NotImplementedError("dimension > 3")
    return tuple(sorted(out))


@lru_cache(maxsize=None)
def knot_offsets(dirs: Tuple[Vec, ...], normal: Vec) -> Tuple[int, ...]:
    """Sorted values nu . (sum of a sub-multiset of dirs)."""
    sums = {0}
    for d in dirs:
        v = dot(normal, d)
        sums |= {s + v for s in sums}
    return tuple(sorted(sums))


def cell_key(dirs: Tuple[Vec, ...], z: Sequence[Fraction]):
    key = []
    for nu in knot_normals(dirs):
        d = dot(nu, z)
        offs = knot_offsets(dirs, nu)
        i = bisect.bisect_left(offs, d)
        if i < len(offs) and offs[i] == d:
            raise NotGenericError("point on a knot plane")
        key.append(i)
    return tuple(key)


# ---------------------------------------------------------------------------
# pieces
# ---------------------------------------------------------------------------

class BoxPieces:
    """Memoised exact pieces of M_Xi for the sub-multisets of one direction set."""

    def __init__(self):
        self.memo: Dict[tuple, Poly] = {}

    def piece(self, dirs: Sequence[Sequence[int]], z: Sequence) -> Poly:
        """Polynomial (in x, s variables) equal to M_dirs near the generic point z."""
        dd = tuple(sorted(tuple(int(v) for v in d) for d in dirs))
        zz = tuple(Fraction(v) for v in z)
        return self._piece(dd, zz)

    def _piece(self, dirs: Tuple[Vec, ...], z: Tuple[Fraction, ...]) -> Poly:
        s = len(z)
        if rank(dirs) < s:
            return Poly(s)
        key = (dirs, cell_key(dirs, z))
        hit = self.memo.get(key)
        if hit is not None:
            return hit
        if len(dirs) == s:
            w = solve(dirs, z)
            inside = all(0 < v < 1 for v in w)
            res = Poly.const(s, 1 / abs(det(dirs))) if inside else Poly(s)
            self.memo[key] = res
            return res
        # remove one copy of a direction whose removal keeps the set spanning
        xi, rest = None, None
        for j in range(len(dirs) - 1, -1, -1):
            cand = dirs[:j] + dirs[j + 1:]
            if rank(cand) == s:
                xi, rest = dirs[j], cand
                break
        # crossings of the segment z - t xi (t in (0,1)) with the knot planes of rest
        cuts = []
        for nu in knot_normals(rest):
            nx = dot(nu, xi)
            if nx == 0:
                continue
            nz = dot(nu, z)
            for o in knot_offsets(rest, nu):
                t = (nz - o) / nx
                if 0 < t < 1:
                    cuts.append((t, nu, o, nx))
                elif t == 0 or t == 1:
                    raise NotGenericError("segment end on a knot plane")
        cuts.sort(key=lambda c: c[0])
        for a, b in zip(cuts, cuts[1:]):
            if a[0] == b[0]:
                raise NotGenericError("coincident crossings")
        # affine breakpoints t_k(x) in x, as polynomials in s variables
        bps = [Poly.const(s, 0)]
        tvals = [Fraction(0)]
        for t, nu, o, nx in cuts:
            bps.append(Poly.linear([Fraction(c, 1) / nx for c in nu], Fraction(-o) / nx))
            tvals.append(t)
        bps.append(Poly.const(s, 1))
        tvals.append(Fraction(1))
        # x_i -> x_i - xi_i t in (x, t)
        shift_images = [Poly.linear([1 if j == i else 0 for j in range(s)] + [-xi[i]])
                        for i in range(s)]
        res = Poly(s)
        for k in range(len(bps) - 1):
            # the smaller set's piece is one polynomial on the whole open
            # interval; a point of it that lies on one of that set's own knot
            # planes (possible for structured direction sets) is replaced by
            # another point of the interval
            for frac in _INTERIOR:
                tm = tvals[k] + (tvals[k + 1] - tvals[k]) * frac
                zm = tuple(zi - tm * xii for zi, xii in zip(z, xi))
                try:
                    q = self._piece(rest, zm)
                    break
                except NotGenericError:
                    if frac is _INTERIOR[-1]:
                        raise
            if q.is_zero():
                continue
            anti = q.substitute(shift_images).integrate_last()          # A(x, t)
            xs = [Poly.var(s, i) for i in range(s)]
            hi = anti.substitute(xs + [bps[k + 1]])
            lo = anti.substitute(xs + [bps[k]])
            res = res + hi - lo
        self.memo[key] = res
        return res
