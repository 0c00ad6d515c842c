"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: values the
paper prints (Fig. 1), textbook closed forms, invariants every basis function
here must satisfy (partition of unity, polynomial reproduction with the
closed-form moment defect, lattice symmetry, support, integral), brute force on
tiny inputs, and identities between the oracle's own entry points (finite
differences, the adjoint dot-product test).
"""
import itertools
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import specs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SIGNED_PERMS_3 = [
    (p, s) for p in itertools.permutations(range(3)) for s in itertools.product((1, -1), repeat=3)
]


def _apply(p, s, x):
    x = np.asarray(x)
    return np.stack([s[i] * x[..., p[i]] for i in range(len(p))], axis=-1)


# --------------------------------------------------------------------------
# textbook closed forms
# --------------------------------------------------------------------------

def _cardinal_bspline(n, x):
    """M_{1,...,1} (n ones) by the truncated-power formula
    sum_k (-1)^k C(n,k) (x-k)_+^{n-1} / (n-1)!."""
    def tp(u):                       # truncated power (u)_+^{n-1}, with (u)_+^0 = 1[u > 0]
        return (u ** (n - 1)) if u > 0 else 0.0
    return sum((-1) ** k * math.comb(n, k) * tp(x - k) for k in range(n + 1)) / math.factorial(n - 1)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_cardinal_bspline_closed_form(n):
    rng = np.random.default_rng(n)
    for x in rng.uniform(-0.5, n + 0.5, 40):
        got = oracle.box([[1.0]] * n, [x])
        assert abs(got - _cardinal_bspline(n, x)) < 1e-12


def test_centred_cubic_bspline_values():
    s = specs.tricubic(closed_form=False)
    # beta3(0) = 2/3, beta3(+-1) = 1/6, beta3(+-2) = 0  ->  phi(0) = 8/27 etc.
    pts = [[0, 0, 0], [1, 0, 0], [1, 1, 0], [1, -1, 1], [2, 0, 0], [0, 0.5, 0]]
    want = [8 / 27, 4 / 54, 2 / 108, 1 / 216, 0.0, (2 / 3) ** 2 * (2 / 3 - 0.25 + 0.0625)]
    got = oracle.phi(s, pts)
    assert np.max(np.abs(got - want)) < 1e-11


def _hat(t):
    """Centred linear B-spline (order 2)."""
    return np.maximum(0.0, 1.0 - np.abs(t))


def _beta2(t):
    """Centred quadratic B-spline (order 3): 3/4 - t^2 on |t| <= 1/2,
    (3/2 - |t|)^2 / 2 on 1/2 <= |t| <= 3/2, 0 beyond."""
    a = np.abs(t)
    return np.where(a <= 0.5, 0.75 - a * a, np.where(a <= 1.5, 0.5 * (1.5 - a) ** 2, 0.0))


@pytest.mark.parametrize("name,factor", [("trilinear", _hat), ("triquadratic", _beta2)])
def test_trilinear_and_triquadratic_are_products_of_textbook_bsplines(name, factor):
    """The recurrence with each axis repeated 2 or 3 times equals the product of
    the closed-form centred B-splines of order 2 or 3 (incl. beta2(0) = 3/4)."""
    rng = np.random.default_rng(2)
    y = rng.uniform(-1.8, 1.8, (400, 3))
    y[:5] = [[0, 0, 0], [0.5, 0, 0], [1, 1, 0], [-0.25, 0.75, 1.25], [1.5, 0, 0]]
    got = oracle.phi(specs.ALL_3D[name](), y)
    want = np.prod(factor(y), axis=1)
    assert np.max(np.abs(got - want)) < 1e-13


def test_tricubic_recurrence_matches_closed_form():
    rng = np.random.default_rng(1)
    y = rng.uniform(-2.2, 2.2, (300, 3))
    a = oracle.phi(specs.tricubic(closed_form=True), y)
    b = oracle.phi(specs.tricubic(closed_form=False), y)
    assert np.max(np.abs(a - b)) < 1e-13


# --------------------------------------------------------------------------
# the paper's worked example: Fig. 1
# --------------------------------------------------------------------------

def _fig1():
    with open(os.path.join(GOLDEN, "fig1_zp_subregion1.json")) as f:
        g = json.load(f)
    sites = np.array(g["sites"])
    mons = g["monomials"]
    W = np.array([[float(Fraction(v)) for v in g["weights"][f"c{j}"]] for j in range(7)])
    return sites, mons, W


def _fig1_poly(x, c):
    sites, mons, W = _fig1()
    m = np.array([x[0] ** a * x[1] ** b for a, b in mons])
    return float(c @ (W @ m))


def _zp_grid(c_sites, c_vals, ext=7, origin=3):
    """Coefficient array on a 7x7 grid with the given values at sites (relative
    to the grid point `origin`), random elsewhere."""
    rng = np.random.default_rng(7)
    coef = rng.uniform(-1, 1, (ext, ext))
    for (s0, s1), v in zip(c_sites, c_vals):
        coef[origin + s1, origin + s0] = v      # axis 0 fastest: coef[i1, i0]
    return coef


def test_fig1_zp_subregion1_polynomial():
    sites, _, _ = _fig1()
    spec = specs.zp2d().with_extent((7, 7))
    rng = np.random.default_rng(11)
    for trial in range(5):
        c = rng.uniform(-1, 1, 7)
        coef = _zp_grid(sites, c)
        pts = []
        while len(pts) < 60:
            x = rng.uniform(-0.5, 0.5, 2)
            if x[0] > abs(x[1]):
                pts.append(x)
        pts = np.array(pts)
        got = oracle.eval_sum(spec, coef.ravel(), pts + 3.0)
        want = np.array([_fig1_poly(x, c) for x in pts])
        assert np.max(np.abs(got - want)) < 1e-12


@pytest.mark.parametrize("turns", [1, 2, 3])
def test_fig1_zp_rotated_subregions(turns):
    """Sub-regions 2-4 of Fig. 1 reuse the sub-region 1 polynomial after a
    rotation: f(R x; c) = P1(x; c o R)."""
    sites, _, _ = _fig1()
    spec = specs.zp2d().with_extent((7, 7))
    ang = -turns * math.pi / 2     # clockwise
    R = np.array([[round(math.cos(ang)), -round(math.sin(ang))],
                  [round(math.sin(ang)), round(math.cos(ang))]])
    rng = np.random.default_rng(20 + turns)
    c = rng.uniform(-1, 1, 7)
    coef = _zp_grid([R @ s for s in sites], c)
    for _ in range(40):
        while True:
            x = rng.uniform(-0.5, 0.5, 2)
            if x[0] > abs(x[1]):
                break
        got = oracle.eval_sum(spec, coef.ravel(), (R @ x + 3.0)[None])[0]
        assert abs(got - _fig1_poly(x, c)) < 1e-12


# --------------------------------------------------------------------------
# invariants
# --------------------------------------------------------------------------

# The recurrence form of the tricubic is pinned to the closed form above; the
# invariants below run on the closed form (the recurrence costs ~1 s/point there).
ALL = dict(specs.ALL_3D)


def _interior_pts(rng, n, lo, hi, dim=3):
    return rng.uniform(lo, hi, (n, dim))


def _sites_and_grid(spec):
    """All stored site coordinates, in coefficient order."""
    out = []
    e = spec.ext
    for l in spec.cosets:
        for i2 in range(e[2]):
            for i1 in range(e[1]):
                for i0 in range(e[0]):
                    out.append([spec.scale * i0 + l[0], spec.scale * i1 + l[1],
                                spec.scale * i2 + l[2]])
    return np.array(out, dtype=np.float64)


def _small(spec):
    e = 10 if spec.scale == 1 else 7       # CC 10^3; BCC/FCC cosets 7^3 (box 0..13)
    return spec.with_extent((e, e, e))


@pytest.mark.parametrize("name", sorted(ALL))
def test_partition_of_unity(name):
    spec = _small(ALL[name]())
    rng = np.random.default_rng(3)
    pts = _interior_pts(rng, 150, 4.5, 6.5 if spec.scale == 1 else 8.5)
    v = oracle.eval_sum(spec, np.ones(spec.n_coef()), pts)
    assert np.max(np.abs(v - 1.0)) < 1e-12


def _moment_defect(dirs, H):
    """1/2 tr(H Xi Xi^T / 12): the second moment of the centred box spline."""
    X = np.asarray(dirs, dtype=np.float64).T
    return 0.5 * np.trace(H @ (X @ X.T) / 12.0)


@pytest.mark.parametrize("name", sorted(ALL))
def test_linear_reproduction(name):
    spec = _small(ALL[name]())
    sites = _sites_and_grid(spec)
    rng = np.random.default_rng(4)
    a = rng.normal(size=3)
    b = 0.3
    pts = _interior_pts(rng, 100, 4.5, 6.5 if spec.scale == 1 else 8.5)
    v = oracle.eval_sum(spec, sites @ a + b, pts)
    assert np.max(np.abs(v - (pts @ a + b))) < 1e-11


@pytest.mark.parametrize("name", ["tricubic", "triquadratic", "bcc_quintic", "bcc_quartic", "fcc6"])
def test_quadratic_reproduction_with_moment_defect(name):
    spec = _small(ALL[name]())
    sites = _sites_and_grid(spec)
    rng = np.random.default_rng(5)
    Q = rng.normal(size=(3, 3))
    Q = Q + Q.T
    g = rng.normal(size=3)
    vals = 0.5 * np.einsum("ni,ij,nj->n", sites, Q, sites) + sites @ g
    pts = _interior_pts(rng, 100, 4.5, 6.5 if spec.scale == 1 else 8.5)
    want = 0.5 * np.einsum("ni,ij,nj->n", pts, Q, pts) + pts @ g + _moment_defect(spec.dirs, Q)
    v = oracle.eval_sum(spec, vals, pts)
    assert np.max(np.abs(v - want)) < 1e-10


@pytest.mark.parametrize("name", ["tricubic", "bcc_quintic", "bcc_quartic"])
def test_cubic_reproduction_with_moment_defect(name):
    """Order-4 splines reproduce cubics up to the (linear) second-moment term;
    odd central moments vanish by symmetry."""
    spec = _small(ALL[name]())
    sites = _sites_and_grid(spec)
    rng = np.random.default_rng(6)
    pts = _interior_pts(rng, 60, 4.5, 6.5 if spec.scale == 1 else 8.5)

    def p(x):
        return x[..., 0] ** 2 * x[..., 1] - 0.5 * x[..., 2] ** 3 + x[..., 0] * x[..., 1] * x[..., 2]

    def hess(x):
        H = np.zeros((3, 3))
        H[0, 0] = 2 * x[1]
        H[0, 1] = H[1, 0] = 2 * x[0] + x[2]
        H[2, 2] = -3 * x[2]
        H[0, 2] = H[2, 0] = x[1]
        H[1, 2] = H[2, 1] = x[0]
        return H

    v = oracle.eval_sum(spec, p(sites), pts)
    want = np.array([p(x) + _moment_defect(spec.dirs, hess(x)) for x in pts])
    assert np.max(np.abs(v - want)) < 1e-9


@pytest.mark.parametrize("name", ["bcc_linear", "trilinear"])
def test_second_order_splines_do_not_reproduce_quadratics(name):
    """Sanity of the previous tests: a second-order spline must fail them."""
    spec = _small(specs.ALL_3D[name]())
    sites = _sites_and_grid(spec)
    rng = np.random.default_rng(5)
    pts = _interior_pts(rng, 50, 4.5, 6.5 if spec.scale == 1 else 8.5)
    v = oracle.eval_sum(spec, sites[:, 0] ** 2, pts)
    want = pts[:, 0] ** 2 + _moment_defect(spec.dirs, np.diag([2.0, 0, 0]))
    assert np.max(np.abs(v - want)) > 1e-3


@pytest.mark.parametrize("name", sorted(specs.ALL_3D))
def test_signed_permutation_symmetry(name):
    spec = specs.ALL_3D[name]()
    rng = np.random.default_rng(8)
    y = rng.uniform(-2.5, 2.5, (40, 3))
    base = oracle.phi(spec, y)
    for p, s in SIGNED_PERMS_3:
        assert np.max(np.abs(oracle.phi(spec, _apply(p, s, y)) - base)) < 1e-12


def test_zp_dihedral_symmetry():
    spec = specs.zp2d()
    rng = np.random.default_rng(9)
    y = rng.uniform(-1.6, 1.6, (80, 2))
    base = oracle.phi(spec, y)
    for p in itertools.permutations(range(2)):
        for s in itertools.product((1, -1), repeat=2):
            assert np.max(np.abs(oracle.phi(spec, _apply(p, s, y)) - base)) < 1e-12


@pytest.mark.parametrize("name", sorted(specs.ALL_3D))
def test_support_and_positivity(name):
    """phi > 0 inside the centred zonotope {|nu.y| < 1/2 sum|nu.xi|} and 0 outside."""
    spec = specs.ALL_3D[name]()
    X = np.asarray(spec.dirs, dtype=np.float64)
    normals = []
    for a, b in itertools.combinations(range(len(X)), 2):
        n = np.cross(X[a], X[b])
        if np.abs(n).sum() > 1e-9:
            normals.append(n)
    normals = np.array(normals)
    bound = 0.5 * np.abs(normals @ X.T).sum(axis=1)
    rng = np.random.default_rng(10)
    reach = float(np.max(bound / np.linalg.norm(normals, axis=1)))     # farthest facet of the zonotope
    L = min(4.5, 1.6 * reach)
    y = rng.uniform(-L, L, (3000, 3))
    margin = np.min(bound[None, :] - np.abs(y @ normals.T), axis=1) / np.linalg.norm(normals, axis=1).max()
    v = oracle.phi(spec, y)
    inside = margin > 1e-6
    outside = margin < -1e-6
    assert inside.sum() > 50 and outside.sum() > 50
    assert np.all(v[inside] > 0.0)
    assert np.all(v[outside] == 0.0)


@pytest.mark.parametrize("name,det", [("tricubic", 1.0), ("trilinear", 1.0), ("triquadratic", 1.0),
                                      ("bcc_linear", 4.0), ("bcc_quintic", 4.0), ("bcc_quartic", 4.0),
                                      ("fcc6", 2.0)])
def test_integral_equals_lattice_density(name, det):
    """integral phi = |det L| (midpoint rule on a fine grid)."""
    spec = specs.ALL_3D[name]()
    h = 1.0 / 8.0 if name not in ("bcc_quintic", "bcc_quartic") else 1.0 / 6.0
    R = {"bcc_quintic": 4.0, "bcc_quartic": 3.0}.get(name, 2.0)
    g = np.arange(-R + h / 2, R, h)
    Y = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    # shift by a generic offset so that no sample sits on a knot plane
    Y = Y + np.array([1e-3, 2e-3, 3e-3])
    total = oracle.phi(spec, Y).sum() * h ** 3
    assert abs(total - det) < 2e-3 * det


@pytest.mark.parametrize("name,degree", [("bcc_linear", 1), ("fcc6", 3), ("bcc_quartic", 4), ("bcc_quintic", 5)])
def test_piece_degree(name, degree):
    """Each polynomial piece has degree |Xi| - 3 (the "quartic" BCC spline: 4):
    along short segments inside one piece the (degree + 1)-th differences
    vanish and the degree-th do not.  Segments that cross a knot plane are rare
    and only fail the first half, so the test asks most segments (60 %) to pass."""
    spec = specs.ALL_3D[name]()
    rng = np.random.default_rng(40)
    h = 2e-2
    ok = 0
    n = 40
    for _ in range(n):
        y0 = rng.uniform(-1.0, 1.0, 3)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        v = oracle.phi(spec, y0[None, :] + h * np.arange(degree + 2)[:, None] * d[None, :])
        top = np.min(np.abs(np.diff(v, degree)))
        if abs(np.diff(v, degree + 1)[0]) <= 1e-3 * top and top >= 1e-12:
            ok += 1
    assert ok >= 0.6 * n, ok


def test_bcc_linear_interpolates():
    """The linear BCC box spline is interpolating: phi(n) = delta_{n,0} on BCC."""
    spec = specs.bcc_linear()
    sites = [n for n in itertools.product(range(-3, 4), repeat=3)
             if len({v % 2 for v in n}) == 1]
    v = oracle.phi(spec, sites)
    for n, val in zip(sites, v):
        assert abs(val - (1.0 if n == (0, 0, 0) else 0.0)) < 1e-10


@pytest.mark.parametrize("name", sorted(specs.ALL_3D))
def test_value_on_knot_planes_is_the_continuous_limit(name):
    spec = specs.ALL_3D[name]()
    rng = np.random.default_rng(12)
    base = rng.uniform(-1.5, 1.5, (30, 3))
    # put points on planes x_i = x_j, x_i = 0, x_0+x_1+x_2 = 1
    on = base.copy()
    on[:10, 1] = on[:10, 0]
    on[10:20, 2] = 0.0
    on[20:, 2] = 1.0 - on[20:, 0] - on[20:, 1]
    v = oracle.phi(spec, on)
    for d in (np.array([1.0, -2.0, 0.5]), np.array([-0.3, 1.0, 1.7])):
        e = 1e-9 * d / np.linalg.norm(d)
        avg = 0.5 * (oracle.phi(spec, on + e) + oracle.phi(spec, on - e))
        assert np.max(np.abs(v - avg)) < 1e-8


# --------------------------------------------------------------------------
# identities between the oracle's own entry points
# --------------------------------------------------------------------------

def test_site_enumeration_matches_brute_force():
    """orc_eval's support-box site enumeration vs a sum over ALL stored sites."""
    for name in sorted(specs.ALL_3D):
        spec = specs.ALL_3D[name]().with_extent((5, 5, 5) if specs.ALL_3D[name]().scale == 2 else (6, 6, 6))
        rng = np.random.default_rng(13)
        coef = rng.uniform(-1, 1, spec.n_coef())
        sites = _sites_and_grid(spec)
        hi = 5.0 if spec.scale == 1 else 8.0
        pts = rng.uniform(-1.0, hi + 1.0, (12, 3))     # includes points near and past the edges
        got = oracle.eval_sum(spec, coef, pts)
        for q, x in enumerate(pts):
            want = float(coef @ oracle.phi(spec, x[None, :] - sites))
            assert abs(got[q] - want) < 1e-12, name


@pytest.mark.parametrize("name", sorted(specs.ALL_3D))
def test_gradient_matches_central_differences(name):
    spec = _small(specs.ALL_3D[name]())
    rng = np.random.default_rng(14)
    coef = rng.uniform(-1, 1, spec.n_coef())
    pts = _interior_pts(rng, 40, 4.5, 6.5 if spec.scale == 1 else 8.5)
    f, g = oracle.eval_sum_grad(spec, coef, pts)
    h = 1e-6
    checked = 0
    for i in range(3):
        e = np.zeros(3)
        e[i] = h
        fp = oracle.eval_sum(spec, coef, pts + e)
        fm = oracle.eval_sum(spec, coef, pts - e)
        fwd, bwd = (fp - f) / h, (f - fm) / h
        smooth = np.abs(fwd - bwd) < 1e-3         # skip kinks of C0 splines
        cd = (fp - fm) / (2 * h)
        assert np.all(np.abs(cd[smooth] - g[smooth, i]) < 1e-6)
        checked += smooth.sum()
    assert checked > 100


@pytest.mark.parametrize("name", sorted(specs.ALL_3D))
def test_adjoint_dot_product(name):
    spec = _small(specs.ALL_3D[name]())
    rng = np.random.default_rng(15)
    coef = rng.uniform(-1, 1, spec.n_coef())
    pts = rng.uniform(0.0, 9.0 if spec.scale == 1 else 13.0, (80, 3))
    gout = rng.normal(size=80)
    lhs = gout @ oracle.eval_sum(spec, coef, pts)
    rhs = oracle.adjoint(spec, pts, gout) @ coef
    assert abs(lhs - rhs) < 1e-10 * max(1.0, abs(lhs))


def test_design_triplets_match_eval():
    spec = _small(specs.fcc6())
    rng = np.random.default_rng(16)
    coef = rng.uniform(-1, 1, spec.n_coef())
    pts = rng.uniform(0.0, 13.0, (50, 3))
    r, c, v = oracle.design_triplets(spec, pts)
    Ac = np.zeros(50)
    np.add.at(Ac, r, v * coef[c])
    assert np.max(np.abs(Ac - oracle.eval_sum(spec, coef, pts))) < 1e-12


def test_morton_definition():
    assert oracle.morton3(1, 0, 0) == 1
    assert oracle.morton3(0, 1, 0) == 2
    assert oracle.morton3(0, 0, 1) == 4
    assert oracle.morton3(3, 0, 0) == 0b1001
    assert oracle.morton3(1023, 1023, 1023) == (1 << 30) - 1
    rng = np.random.default_rng(17)
    for _ in range(200):
        a, b, c = (int(v) for v in rng.integers(0, 1024, 3))
        k = oracle.morton3(a, b, c)
        # de-interleave with plain integer arithmetic
        back = [sum(((k >> (3 * bit + i)) & 1) << bit for bit in range(10)) for i in range(3)]
        assert back == [a, b, c]


# --------------------------------------------------------------------------
# Hessian (second derivatives of the per-region polynomials, Sec. 3)
# --------------------------------------------------------------------------

_HIDX = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]


def _hmat(h):
    H = np.zeros(h.shape[:-1] + (3, 3))
    for k, (a, b) in enumerate(_HIDX):
        H[..., a, b] = h[..., k]
        H[..., b, a] = h[..., k]
    return H


def _d2_factors(name):
    """Closed-form second derivatives of the centred 1D B-splines (orders 2-4)."""
    def hat(t):
        return np.maximum(0.0, 1.0 - np.abs(t)), -np.sign(t) * (np.abs(t) < 1), np.zeros_like(t)

    def quad(t):
        a = np.abs(t)
        b = np.where(a <= 0.5, 0.75 - a * a, np.where(a <= 1.5, 0.5 * (1.5 - a) ** 2, 0.0))
        db = np.where(a <= 0.5, -2 * t, np.where(a <= 1.5, -np.sign(t) * (1.5 - a), 0.0))
        d2 = np.where(a <= 0.5, -2.0, np.where(a <= 1.5, 1.0, 0.0))
        return b, db, d2

    def cub(t):
        a = np.abs(t)
        b = np.where(a < 1, 2 / 3 - a * a + 0.5 * a ** 3, np.where(a < 2, (2 - a) ** 3 / 6, 0.0))
        db = np.where(a < 1, -2 * t + 1.5 * t * a, np.where(a < 2, -0.5 * np.sign(t) * (2 - a) ** 2, 0.0))
        d2 = np.where(a < 1, -2 + 3 * a, np.where(a < 2, 2 - a, 0.0))
        return b, db, d2
    return {"trilinear": hat, "triquadratic": quad, "tricubic": cub}[name]


@pytest.mark.parametrize("name", ["tricubic", "trilinear", "triquadratic"])
def test_hessian_of_tensor_products_matches_closed_form(name):
    """The pair-wise derivative identity through the recurrence (kind 0 for the
    tricubic too) equals the product of closed-form B-spline derivatives."""
    spec = specs.tricubic(closed_form=False) if name == "tricubic" else specs.ALL_3D[name]()
    rng = np.random.default_rng(21)
    # the recurrence over 12 directions is slow: fewer points for the tricubic
    y = rng.uniform(-2.2, 2.2, (12 if name == "tricubic" else 300, 3))
    f = _d2_factors(name)
    b, db, d2 = f(y)
    want = np.zeros((len(y), 6))
    for k, (p, q) in enumerate(_HIDX):
        t = np.ones(len(y))
        for i in range(3):
            if p == q:
                t *= d2[:, i] if i == p else b[:, i]
            else:
                t *= db[:, i] if i in (p, q) else b[:, i]
        want[:, k] = t
    got = oracle.phi_hess(spec, y)
    assert np.max(np.abs(got - want)) < 1e-12


@pytest.mark.parametrize("name", sorted(specs.ALL_3D))
def test_hessian_matches_central_differences_of_gradient(name):
    spec = specs.ALL_3D[name]()
    rng = np.random.default_rng(22)
    y = rng.uniform(-2.0, 2.0, (150, 3))
    H = _hmat(oracle.phi_hess(spec, y))
    fd = np.zeros_like(H)
    fd2 = np.zeros_like(H)
    for i in range(3):
        for h, out in ((1e-5, fd), (2e-5, fd2)):
            e = np.zeros(3)
            e[i] = h
            out[:, i, :] = (oracle.phi_grad(spec, y + e)[1] - oracle.phi_grad(spec, y - e)[1]) / (2 * h)
    # points within a step of a knot plane show up as disagreeing differences
    smooth = np.max(np.abs(fd - fd2), axis=(1, 2)) < 1e-6
    assert smooth.sum() > 100
    assert np.max(np.abs(H[smooth] - fd[smooth])) < 1e-8


@pytest.mark.parametrize("name", ["tricubic", "triquadratic", "bcc_quintic", "bcc_quartic", "fcc6"])
def test_hessian_of_reproduced_quadratic_is_exact(name):
    """Splines of order >= 3 reproduce quadratics up to a constant (the moment
    defect), so the Hessian of sum_n p(n) phi(x - n) is the Hessian of p."""
    spec = _small(ALL[name]())
    sites = _sites_and_grid(spec)
    rng = np.random.default_rng(23)
    Q = rng.normal(size=(3, 3))
    Q = Q + Q.T
    vals = 0.5 * np.einsum("ni,ij,nj->n", sites, Q, sites) + sites @ rng.normal(size=3)
    pts = _interior_pts(rng, 60, 4.5, 6.5 if spec.scale == 1 else 8.5)
    H = _hmat(oracle.eval_sum_hess(spec, vals, pts))
    assert np.max(np.abs(H - Q[None])) < 1e-9


@pytest.mark.parametrize("name", ["bcc_quintic", "bcc_quartic", "fcc6", "triquadratic"])
def test_hessian_transforms_with_the_lattice_symmetries(name):
    """phi(R y) = phi(y) for the signed permutations R, so H(R y) = R H(y) R^T."""
    spec = specs.ALL_3D[name]()
    rng = np.random.default_rng(24)
    y = rng.uniform(-1.8, 1.8, (30, 3))
    H = _hmat(oracle.phi_hess(spec, y))
    for p, s in SIGNED_PERMS_3[::7]:
        R = np.zeros((3, 3))
        for i in range(3):
            R[i, p[i]] = s[i]
        HR = _hmat(oracle.phi_hess(spec, y @ R.T))
        assert np.max(np.abs(HR - np.einsum("ij,njk,lk->nil", R, H, R))) < 1e-11
