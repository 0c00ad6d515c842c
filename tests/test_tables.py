"""The sub-region tables (the generator's input) against the paper and the oracle."""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workloads
from oracle import specs as ospecs
from paper_2102_08518_b300 import splines
from paper_2102_08518_b300.api import table
from tests.table_eval import eval_separable, eval_table

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ORACLE_SPEC = {"tricubic": ospecs.tricubic, "trilinear": ospecs.trilinear, "triquadratic": ospecs.triquadratic,
               "bcc_linear": ospecs.bcc_linear, "bcc_quintic": ospecs.bcc_quintic, "bcc_quartic": ospecs.bcc_quartic,
               "voronoi2_bcc": ospecs.voronoi2_bcc, "voronoi2_fcc": ospecs.voronoi2_fcc, "fcc6": ospecs.fcc6,
               "zp": ospecs.zp2d}


def test_zp_table_reproduces_fig1():
    """Sub-region 1 of Fig. 1 contains the chamber x0 >= x1 >= 0 of the ZP table:
    same sites, same polynomials (exact rationals)."""
    with open(os.path.join(GOLDEN, "fig1_zp_subregion1.json")) as f:
        g = json.load(f)
    t = table("zp")
    assert t.fold == "hyperoctahedral" and len(t.regions) == 1
    reg = t.regions[0]
    got = {}
    for s, w in zip(reg.sites, reg.weights):
        wy = w.shift([-c for c in reg.center])          # back to y coordinates
        got[tuple(s)] = {e: v for e, v in wy.c.items()}
    want = {}
    for j, s in enumerate(g["sites"]):
        want[tuple(s)] = {tuple(m): Fraction(v) for m, v in zip(g["monomials"], g["weights"][f"c{j}"])
                          if Fraction(v) != 0}
    assert got == want


@pytest.mark.parametrize("name", ["tricubic", "trilinear", "triquadratic", "bcc_linear", "bcc_quintic", "bcc_quartic",
                                  "fcc6", "zp", "voronoi2_bcc", "voronoi2_fcc"])
def test_table_weights_partition_unity_exactly(name):
    t = table(name)
    for reg in t.regions:
        tot = reg.weights[0]
        for w in reg.weights[1:]:
            tot = tot + w
        assert tot.c == {(0,) * t.spline.lattice.dim: Fraction(1)}


def test_structural_facts_from_the_paper():
    # BCC linear needs 4 lookups (Sec. 5.1); the tricubic 64 (Sec. 5.1, order 4);
    # the FCC six-direction spline has two reference sub-regions (Sec. 3, Sec. 5.1);
    # most splines need one distinct polynomial (Sec. 3).
    assert [len(r.sites) for r in table("bcc_linear").regions] == [4]
    assert len(table("tricubic").regions[0].sites) == 64
    assert len(table("fcc6").regions) == 2
    assert len(table("bcc_quintic").regions) == 1 and len(table("bcc_linear").regions) == 1
    sep = table("tricubic").separable
    assert sep is not None and [len(a.sites) for a in sep] == [4, 4, 4]
    # the Cartesian comparison splines: trilinear 8 lookups (Sec. 5.1, order 2), triquadratic 27
    assert len(table("trilinear").regions[0].sites) == 8
    assert len(table("triquadratic").regions[0].sites) == 27
    # the seven-direction BCC spline: quartic pieces (degree |Xi| - 3)
    assert table("bcc_quartic").degree == 4
    # second-order Voronoi splines: cubic pieces, 8 sites per point (as the
    # trilinear spline); more than one reference sub-region on BCC, so the
    # branchy / predicated choice of the paper's Voronoi study applies
    for name in ("voronoi2_bcc", "voronoi2_fcc"):
        t = table(name)
        assert t.degree == 3 and all(len(r.sites) == 8 for r in t.regions)
    assert len(table("voronoi2_bcc").regions) > 1


@pytest.mark.parametrize("name", ["tricubic", "trilinear", "triquadratic", "bcc_linear", "bcc_quintic", "bcc_quartic",
                                  "fcc6", "zp", "voronoi2_bcc", "voronoi2_fcc"])
def test_table_matches_oracle_by_brute_force(name):
    """Algorithm 1 over the table in FP64 vs the oracle's naive sum, tiny grids,
    points everywhere (inside, near and beyond the edges)."""
    t = table(name)
    lat = workloads.SPLINE_LATTICE[name]
    dim = workloads.LATTICES[lat][0]
    ext = (6,) * dim if lat in ("cc", "z2") else (5,) * dim
    coef = workloads.coef_uniform(lat, ext, seed=3)
    lo, hi = workloads.bounding_box(lat, ext)
    pts = workloads.points_uniform(150, lo - 1.5, hi + 1.5, seed=4).astype(np.float64)
    spec = ORACLE_SPEC[name]().with_extent(ext)
    want = oracle.eval_sum(spec, coef.ravel(), pts)
    got = eval_table(t, coef, ext, pts)
    assert np.max(np.abs(got - want)) < 1e-12


def test_table_matches_oracle_on_symmetry_planes():
    """Points exactly on the folding mirrors and the FCC BSP plane."""
    for name in ("bcc_quintic", "bcc_quartic", "fcc6"):
        t = table(name)
        lat = workloads.SPLINE_LATTICE[name]
        ext = (6, 6, 6)
        coef = workloads.coef_uniform(lat, ext, seed=5)
        rng = np.random.default_rng(6)
        base = rng.uniform(4.0, 7.0, (40, 3))
        base[:10, 1] = base[:10, 0]                         # y0 = y1 relative to a site is not
        base[10:20] = np.round(base[10:20])                 # guaranteed; lattice-aligned points
        base[20:30, 2] = np.round(base[20:30, 2])
        base[30:, :] = np.round(base[30:, :] * 2) / 2
        spec = ORACLE_SPEC[name]().with_extent(ext)
        want = oracle.eval_sum(spec, coef.ravel(), base)
        got = eval_table(t, coef, ext, base)
        assert np.max(np.abs(got - want)) < 1e-11, name


@pytest.mark.parametrize("name,nsites", [("tricubic", 4), ("trilinear", 2), ("triquadratic", 3)])
def test_separable_factors_match_oracle(name, nsites):
    """The per-axis factors the kernels evaluate (region [0,1)^3 for even order,
    the Voronoi cube around the nearest site for the quadratic) against the naive sum."""
    t = table(name)
    assert t.separable is not None and [len(a.sites) for a in t.separable] == [nsites] * 3
    assert t.spline.roe == ("voronoi" if nsites == 3 else "parallelepiped")
    ext = (6, 6, 6)
    coef = workloads.coef_uniform("cc", ext, seed=13)
    pts = workloads.points_uniform(200, [-1.5] * 3, [6.5] * 3, seed=14).astype(np.float64)
    pts[:20] = np.round(pts[:20] * 2) / 2                      # on the knot planes
    spec = ORACLE_SPEC[name]().with_extent(ext)
    want = oracle.eval_sum(spec, coef.ravel(), pts)
    assert np.max(np.abs(eval_separable(t, coef, ext, pts) - want)) < 1e-12
