"""The oracle's own definitions of the splines and lattices it evaluates.

Written independently of the product package.  Direction sets are those of the
box splines benchmarked in Sec. 5.1 (tensor-product cubic on the Cartesian
lattice, the linear rhombic-dodecahedron, the doubled "quintic" and the
seven-direction "quartic" box splines on BCC, the six-direction
truncated-octahedron box spline on FCC) and of the ZP element of Fig. 1.

Lattices are stored as unions of Cartesian cosets of scale*Z^s:
  CC  = Z^3                                   (scale 1, |det L| = 1)
  BCC = 2Z^3 u (2Z^3 + (1,1,1))               (scale 2, |det L| = 4)
  FCC = {n in Z^3 : n0+n1+n2 even}            (scale 2, |det L| = 2)
  Z^2 for the ZP element                      (scale 1, |det L| = 1)
"""
from .lib import OrcSpec
from . import voronoi as _voronoi

E1, E2, E3 = (1, 0, 0), (0, 1, 0), (0, 0, 1)

BCC_DIRS = ((1, 1, 1), (1, -1, -1), (-1, 1, -1), (-1, -1, 1))
FCC_DIRS = ((1, 1, 0), (1, -1, 0), (1, 0, 1), (1, 0, -1), (0, 1, 1), (0, 1, -1))
BCC_COSETS = ((0, 0, 0), (1, 1, 1))
FCC_COSETS = ((0, 0, 0), (1, 1, 0), (1, 0, 1), (0, 1, 1))


def tricubic(closed_form: bool = True) -> OrcSpec:
    """Tensor-product cubic B-spline on Z^3; kind 1 is the closed form, kind 0
    the same function through the box-spline recurrence (each axis four times)."""
    dirs = (E1,) * 4 + (E2,) * 4 + (E3,) * 4
    return OrcSpec(3, dirs, 1.0, 1, ((0, 0, 0),), (1, 1, 1), 1 if closed_form else 0,
                   "tricubic")


def trilinear() -> OrcSpec:
    """Tensor-product linear B-spline (the hat function) on Z^3: each axis twice."""
    return OrcSpec(3, (E1,) * 2 + (E2,) * 2 + (E3,) * 2, 1.0, 1, ((0, 0, 0),), (1, 1, 1), 0, "trilinear")


def triquadratic() -> OrcSpec:
    """Tensor-product quadratic B-spline on Z^3: each axis three times."""
    return OrcSpec(3, (E1,) * 3 + (E2,) * 3 + (E3,) * 3, 1.0, 1, ((0, 0, 0),), (1, 1, 1), 0, "triquadratic")


def bcc_linear() -> OrcSpec:
    return OrcSpec(3, BCC_DIRS, 4.0, 2, BCC_COSETS, (1, 1, 1), 0, "bcc_linear")


def bcc_quintic() -> OrcSpec:
    return OrcSpec(3, BCC_DIRS + BCC_DIRS, 4.0, 2, BCC_COSETS, (1, 1, 1), 0, "bcc_quintic")


def bcc_quartic() -> OrcSpec:
    """The seven-direction box spline on BCC: the four diagonal directions of
    the linear spline and the three axis directions at their shortest lattice
    length, 2 e_i (degree 7 - 3 = 4, approximation order 4)."""
    return OrcSpec(3, BCC_DIRS + ((2, 0, 0), (0, 2, 0), (0, 0, 2)), 4.0, 2, BCC_COSETS, (1, 1, 1), 0,
                   "bcc_quartic")


def fcc6() -> OrcSpec:
    return OrcSpec(3, FCC_DIRS, 2.0, 2, FCC_COSETS, (1, 1, 1), 0, "fcc6")


def voronoi2_bcc():
    """Second-order Voronoi spline on BCC (oracle.voronoi: cell overlap volume)."""
    return _voronoi.BCC


def voronoi2_fcc():
    """Second-order Voronoi spline on FCC (oracle.voronoi: cell overlap volume)."""
    return _voronoi.FCC


def zp2d() -> OrcSpec:
    """ZP element of Fig. 1: directions (1,0),(0,1),(1,1),(-1,1) on Z^2."""
    return OrcSpec(2, ((1, 0), (0, 1), (1, 1), (-1, 1)), 1.0, 1, ((0, 0),), (1, 1, 1), 0,
                   "zp2d")


ALL_3D = {"tricubic": tricubic, "trilinear": trilinear, "triquadratic": triquadratic,
          "bcc_linear": bcc_linear, "bcc_quintic": bcc_quintic, "bcc_quartic": bcc_quartic, "fcc6": fcc6}
# the Voronoi splines (their own oracle: oracle.voronoi)
VORONOI = {"voronoi2_bcc": voronoi2_bcc, "voronoi2_fcc": voronoi2_fcc}
