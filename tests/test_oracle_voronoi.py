"""Pins of the second-order Voronoi-spline oracle (oracle/voronoi.py).

phi(x) = vol(P n (P + x)) / vol(P) for the Voronoi cell P of the lattice
(Sec. 5, Voronoi splines).  What fixes it independently of its own code:
* on the Cartesian lattice the same code must give the textbook
  tensor-product hat function;
* the cells are the truncated octahedron (BCC) and the rhombic dodecahedron
  (FCC) with volume |det L|;
* phi interpolates (phi(n) = delta_n0: distinct Voronoi cells overlap in
  measure zero), is a partition of unity, reproduces linear but not quadratic
  polynomials (order 2), has the lattice's 48 signed-permutation symmetries,
  support 2P, and integral |det L|.
"""
import itertools

import numpy as np
import pytest
from scipy.spatial import HalfspaceIntersection

from oracle import voronoi as V

SPECS = {"bcc": V.BCC, "fcc": V.FCC}


def _perms():
    for p in itertools.permutations(range(3)):
        for s in itertools.product((1, -1), repeat=3):
            yield p, s


def test_cartesian_case_is_the_hat_function():
    rng = np.random.default_rng(1)
    y = rng.uniform(-1.3, 1.3, (300, 3))
    tent = np.prod(np.clip(1.0 - np.abs(y), 0.0, None), axis=1)
    assert np.max(np.abs(V.phi(V.CC, y) - tent)) < 1e-13


@pytest.mark.parametrize("name,nverts,det", [("bcc", 24, 4.0), ("fcc", 14, 2.0)])
def test_cells_are_the_textbook_polytopes(name, nverts, det):
    spec = SPECS[name]
    A, b = V.cell_halfspaces(spec)
    verts = HalfspaceIntersection(np.hstack([A, -b[:, None]]), np.zeros(3)).intersections
    uniq = np.unique(np.round(verts, 9), axis=0)
    assert len(uniq) == nverts
    if name == "bcc":          # truncated octahedron: the permutations of (0, +-1/2, +-1)
        want = {tuple(float(v) for v in p) for q in itertools.permutations((0.0, 0.5, 1.0))
                for p in itertools.product(*[(x, -x) if x else (0.0,) for x in q])}
    else:                      # rhombic dodecahedron: (+-1, 0, 0) and (+-1/2, +-1/2, +-1/2)
        want = {p for q in itertools.permutations((1.0, 0.0, 0.0)) for p in
                itertools.product(*[(x, -x) if x else (0.0,) for x in q])}
        want |= set(itertools.product((0.5, -0.5), repeat=3))
    assert {tuple(float(v) for v in r) for r in uniq} == want
    assert abs(V._overlap_volume(A, b, np.zeros(3)) - det) < 1e-12


@pytest.mark.parametrize("name", ["bcc", "fcc"])
def test_interpolates(name):
    spec = SPECS[name]
    sites = [n for n in itertools.product(range(-3, 4), repeat=3) if spec.contains(n)]
    v = V.phi(spec, np.array(sites, dtype=np.float64))
    want = np.array([1.0 if n == (0, 0, 0) else 0.0 for n in sites])
    assert np.max(np.abs(v - want)) < 1e-12


@pytest.mark.parametrize("name", ["bcc", "fcc"])
def test_partition_of_unity_and_linear_reproduction(name):
    spec = SPECS[name].with_extent((6, 6, 6))
    rng = np.random.default_rng(2)
    pts = rng.uniform(4.0, 7.0, (60, 3))
    assert np.max(np.abs(V.eval_sum(spec, np.ones(spec.n_coef()), pts) - 1.0)) < 1e-12
    sites = []
    for l in spec.cosets:
        for i2, i1, i0 in itertools.product(range(6), repeat=3):
            sites.append([spec.scale * i0 + l[0], spec.scale * i1 + l[1], spec.scale * i2 + l[2]])
    sites = np.array(sites, dtype=np.float64)
    a = rng.normal(size=3)
    v = V.eval_sum(spec, sites @ a + 0.25, pts)
    assert np.max(np.abs(v - (pts @ a + 0.25))) < 1e-11
    # order 2: a quadratic is not reproduced up to a constant
    q = V.eval_sum(spec, sites[:, 0] ** 2, pts) - pts[:, 0] ** 2
    assert np.ptp(q) > 1e-3


@pytest.mark.parametrize("name", ["bcc", "fcc"])
def test_symmetry_support_and_positivity(name):
    spec = SPECS[name]
    A, b = V.cell_halfspaces(spec)
    rng = np.random.default_rng(3)
    y = rng.uniform(-2.2, 2.2, (400, 3))
    base = V.phi(spec, y)
    for p, s in list(_perms())[::5]:
        img = np.stack([s[i] * y[:, p[i]] for i in range(3)], 1)
        assert np.max(np.abs(V.phi(spec, img) - base)) < 1e-12
    margin = np.min(2 * b[None, :] - y @ A.T, axis=1)          # inside 2P iff > 0
    assert np.all(base[margin > 1e-6] > 0.0)
    assert np.all(base[margin < -1e-6] == 0.0)
    assert (margin > 1e-6).sum() > 50 and (margin < -1e-6).sum() > 50


@pytest.mark.parametrize("name,det", [("bcc", 4.0), ("fcc", 2.0)])
def test_integral_equals_lattice_density(name, det):
    spec = SPECS[name]
    h = 0.25
    g = np.arange(-2.0 + h / 2, 2.0, h)
    Y = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3) + np.array([1e-3, 2e-3, 3e-3])
    total = V.phi(spec, Y).sum() * h ** 3
    assert abs(total - det) < 2e-2 * det
