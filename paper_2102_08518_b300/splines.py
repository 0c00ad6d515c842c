"""The lattices and box splines this library evaluates (Sec. 5.1, Fig. 1).

Lattices are unions of Cartesian cosets of scale*Z^s, stored one coefficient
array per coset (the per-coset memory lookup of Sec. 4.1):
  CC  = Z^3                                  scale 1, one coset
  BCC = 2Z^3 u (2Z^3 + (1,1,1))              scale 2, two cosets,  |det L| = 4
  FCC = {n in Z^3 : n_0 + n_1 + n_2 even}    scale 2, four cosets, |det L| = 2
  Z^2 (the ZP element of Fig. 1)             scale 1, one coset
"""
from .subregions import Lattice, Spline

CC = Lattice("cc", 3, 1, ((0, 0, 0),), ((1, 0, 0), (0, 1, 0), (0, 0, 1)))
BCC = Lattice("bcc", 3, 2, ((0, 0, 0), (1, 1, 1)), ((-1, 1, 1), (1, -1, 1), (1, 1, -1)))
FCC = Lattice("fcc", 3, 2, ((0, 0, 0), (1, 1, 0), (1, 0, 1), (0, 1, 1)),
              ((1, 1, 0), (1, 0, 1), (0, 1, 1)))
Z2 = Lattice("z2", 2, 1, ((0, 0),), ((1, 0), (0, 1)))

_E = ((1, 0, 0), (0, 1, 0), (0, 0, 1))
_BCC4 = ((1, 1, 1), (1, -1, -1), (-1, 1, -1), (-1, -1, 1))
_FCC6 = ((1, 1, 0), (1, -1, 0), (1, 0, 1), (1, 0, -1), (0, 1, 1), (0, 1, -1))

TRICUBIC = Spline("tricubic", CC, tuple(d for d in _E for _ in range(4)), "parallelepiped")
# the paper's Cartesian comparison splines (Sec. 5.1): order 2 (knots at the
# integers: region of evaluation [0,1)^3) and order 3 (knots at the half-integers:
# the Voronoi cell [-1/2,1/2]^3 around the nearest site)
TRILINEAR = Spline("trilinear", CC, tuple(d for d in _E for _ in range(2)), "parallelepiped")
TRIQUADRATIC = Spline("triquadratic", CC, tuple(d for d in _E for _ in range(3)), "voronoi")
BCC_LINEAR = Spline("bcc_linear", BCC, _BCC4, "voronoi")
BCC_QUINTIC = Spline("bcc_quintic", BCC, _BCC4 + _BCC4, "voronoi")
# the paper's other order-4 BCC spline (Sec. 5.1, "BCC quartic"): the four
# diagonals plus the three axes at their shortest lattice length 2 e_i; seven
# directions in 3D give degree 4, and no plane holds more than three of them,
# so it reproduces cubics (approximation order 4)
BCC_QUARTIC = Spline("bcc_quartic", BCC, _BCC4 + ((2, 0, 0), (0, 2, 0), (0, 0, 2)), "voronoi")
FCC6 = Spline("fcc6", FCC, _FCC6, "voronoi")
ZP = Spline("zp", Z2, ((1, 0), (0, 1), (1, 1), (-1, 1)), "voronoi")

# the second-order Voronoi splines of the paper's Voronoi study (Sec. 5): the
# Voronoi cell's indicator convolved with itself, normalised (on the Cartesian
# lattice this is the trilinear spline)
VORONOI2_BCC = Spline("voronoi2_bcc", BCC, (), "voronoi", "voronoi2")
VORONOI2_FCC = Spline("voronoi2_fcc", FCC, (), "voronoi", "voronoi2")

BY_NAME = {s.name: s for s in (TRICUBIC, TRILINEAR, TRIQUADRATIC, BCC_LINEAR, BCC_QUINTIC, BCC_QUARTIC, FCC6, ZP,
                               VORONOI2_BCC, VORONOI2_FCC)}
