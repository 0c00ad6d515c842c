"""Exact multivariate polynomials with rational coefficients.

A polynomial is a dict mapping exponent tuples to ``Fraction`` coefficients.
Used by the sub-region table builder, which derives the per-region polynomials
of a spline exactly (the representation Sec. 3 assumes as input to code
generation).
"""
from __future__ import annotations

from fractions import Fraction
from itertools import product
from typing import Dict, Iterable, Sequence, Tuple

Exp = Tuple[int, ...]


class Poly:
    __slots__ = ("n", "c")

    def __init__(self, nvars: int, coeffs: Dict[Exp, Fraction] | None = None):
        self.n = nvars
        self.c: Dict[Exp, Fraction] = {}
        if coeffs:
            for e, v in coeffs.items():
                if v != 0:
                    self.c[e] = Fraction(v)

    # -- construction -----------------------------------------------------
    @staticmethod
    def const(nvars: int, v) -> "Poly":
        return Poly(nvars, {(0,) * nvars: Fraction(v)})

    @staticmethod
    def var(nvars: int, i: int) -> "Poly":
        e = [0] * nvars
        e[i] = 1
        return Poly(nvars, {tuple(e): Fraction(1)})

    @staticmethod
    def linear(coef: Sequence, const=0) -> "Poly":
        """sum_i coef[i] x_i + const."""
        n = len(coef)
        d: Dict[Exp, Fraction] = {}
        for i, a in enumerate(coef):
            if a != 0:
                e = [0] * n
                e[i] = 1
                d[tuple(e)] = Fraction(a)
        if const != 0:
            d[(0,) * n] = Fraction(const)
        return Poly(n, d)

    # -- arithmetic ---------------------------------------------------------
    def is_zero(self) -> bool:
        return not self.c

    def degree(self) -> int:
        return max((sum(e) for e in self.c), default=0)

    def __add__(self, o: "Poly") -> "Poly":
        r = dict(self.c)
        for e, v in o.c.items():
            r[e] = r.get(e, 0) + v
        return Poly(self.n, r)

    def __sub__(self, o: "Poly") -> "Poly":
        r = dict(self.c)
        for e, v in o.c.items():
            r[e] = r.get(e, 0) - v
        return Poly(self.n, r)

    def scale(self, a) -> "Poly":
        a = Fraction(a)
        if a == 0:
            return Poly(self.n)
        return Poly(self.n, {e: v * a for e, v in self.c.items()})

    def __mul__(self, o: "Poly") -> "Poly":
        r: Dict[Exp, Fraction] = {}
        for e1, v1 in self.c.items():
            for e2, v2 in o.c.items():
                e = tuple(a + b for a, b in zip(e1, e2))
                r[e] = r.get(e, 0) + v1 * v2
        return Poly(self.n, r)

    def __eq__(self, o) -> bool:
        return isinstance(o, Poly) and self.n == o.n and self.c == o.c

    def __hash__(self):
        return hash((self.n, frozenset(self.c.items())))

    def __call__(self, x: Sequence) -> Fraction:
        s = Fraction(0)
        for e, v in self.c.items():
            t = v
            for xi, k in zip(x, e):
                if k:
                    t *= Fraction(xi) ** k
            s += t
        return s

    def evalf(self, x: Sequence[float]) -> float:
        s = 0.0
        for e, v in self.c.items():
            t = float(v)
            for xi, k in zip(x, e):
                if k:
                    t *= xi ** k
            s += t
        return s

    # -- substitutions --------------------------------------------------------
    def substitute(self, images: Sequence["Poly"]) -> "Poly":
        """Replace variable i by images[i] (all images share one variable count)."""
        m = images[0].n
        powers = [[Poly.const(m, 1)] for _ in images]
        out = Poly(m)
        for e, v in self.c.items():
            term = Poly.const(m, v)
            for i, k in enumerate(e):
                while len(powers[i]) <= k:
                    powers[i].append(powers[i][-1] * images[i])
                if k:
                    term = term * powers[i][k]
            out = out + term
        return out

    def extend(self, nvars: int) -> "Poly":
        """Same polynomial in more variables (new ones appended, unused)."""
        return Poly(nvars, {e + (0,) * (nvars - self.n): v for e, v in self.c.items()})

    def integrate_last(self) -> "Poly":
        """Antiderivative with respect to the last variable."""
        r = {}
        for e, v in self.c.items():
            k = e[-1]
            r[e[:-1] + (k + 1,)] = v / (k + 1)
        return Poly(self.n, r)

    def diff(self, i: int) -> "Poly":
        r = {}
        for e, v in self.c.items():
            if e[i]:
                ee = list(e)
                ee[i] -= 1
                r[tuple(ee)] = r.get(tuple(ee), 0) + v * e[i]
        return Poly(self.n, r)

    def shift(self, c: Sequence) -> "Poly":
        """p(x + c) as a polynomial in x."""
        n = self.n
        return self.substitute([Poly.linear([1 if j == i else 0 for j in range(n)], c[i])
                                for i in range(n)])

    def coeff_vector(self, monomials: Iterable[Exp]):
        return [self.c.get(m, Fraction(0)) for m in monomials]


def monomials_upto(nvars: int, degree: int):
    """All exponent tuples of total degree <= degree, graded, then reverse-lex."""
    out = []
    for d in range(degree + 1):
        for e in product(range(d + 1), repeat=nvars):
            if sum(e) == d:
                out.append(e)
    out.sort(key=lambda e: (sum(e), tuple(-v for v in e)))
    return out
