"""The tile-staged value kernel (variant stage) for spatially sorted points.

A block bounds the region-of-evaluation sites of its consecutive points; when
their stencils fit one tile it loads that tile with one TMA tensor copy and
evaluates from shared memory, with coordinates shifted by an even (scale 2) or
integer (scale 1) vector of non-negative grid steps.  That shift is exact in
FP32, so every result must equal the plain kernel's bit for bit: with tiles that
fit and tiles that do not, several tiles per block (grid-stride loop, mbarrier
phases), points beyond the arrays, non-finite points, both linear layouts and
volumes whose tensor map cannot be made (those read global memory throughout).
The values are also checked against the FP64 oracle on a sample.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads
from oracle import specs as ospecs

pytestmark = pytest.mark.gpu

TOL = 2e-6
ORACLE_SPEC = {"tricubic": ospecs.tricubic, "trilinear": ospecs.trilinear, "triquadratic": ospecs.triquadratic,
               "bcc_linear": ospecs.bcc_linear, "bcc_quintic": ospecs.bcc_quintic, "bcc_quartic": ospecs.bcc_quartic,
               "voronoi2_bcc": ospecs.voronoi2_bcc, "voronoi2_fcc": ospecs.voronoi2_fcc, "fcc6": ospecs.fcc6}
# extents with ext0 % 4 == 0, so the coset-major rows are whole 16-byte units
EXT = {"tricubic": (40, 36, 30), "trilinear": (40, 32, 30), "triquadratic": (36, 32, 28),
       "bcc_linear": (24, 22, 20), "bcc_quintic": (24, 20, 18), "fcc6": (24, 20, 18)}
NAMES = list(EXT)


def n_cosets(name):
    return len(workloads.LATTICES[workloads.SPLINE_LATTICE[name]][2])


def morton_order_np(p, lo, cell=1.0):
    """Morton (Z-order) permutation of the cells of p, by numpy: bit b of cell
    axis a goes to key bit 3 b + a."""
    q = np.floor((p - lo) / cell).astype(np.int64)
    key = np.zeros(len(p), np.int64)
    for b in range(12):
        for a in range(3):
            key |= ((q[:, a] >> b) & 1) << (3 * b + a)
    return np.argsort(key, kind="stable")


def sorted_points(name, ext, n, seed, margin=1.5, specials=True):
    lat = workloads.SPLINE_LATTICE[name]
    lo, hi = workloads.bounding_box(lat, ext)
    p = workloads.points_uniform(n, lo - margin, hi + margin, seed=seed)
    p = p[morton_order_np(p, lo - margin)]
    if specials:
        p[7] = np.nan
        p[1000, 1] = np.inf
        p[2001] = -3.0e7                       # beyond the coordinate range
        p[n // 2] = (lo - 40.0)                # far outside the arrays
    return np.ascontiguousarray(p, dtype=np.float32)


def volume(name, ext, coef_np, layout, **kw):
    from paper_2102_08518_b300.api import Spline, Volume, relayout
    C = n_cosets(name)
    c = torch.from_numpy(coef_np.astype(np.float32)).cuda()
    if layout == "interleaved":
        c = relayout(c, C, ext, to="interleaved")
    return Volume(Spline(name, "f32", **kw), ext, c.contiguous(), layout=layout)


def bitwise_equal(a, b):
    return torch.equal(a.view(torch.int32), b.view(torch.int32))


@pytest.mark.parametrize("layout", ["interleaved", "coset"])
@pytest.mark.parametrize("name", NAMES)
def test_staged_equals_plain_bitwise(name, layout):
    ext = EXT[name]
    lat = workloads.SPLINE_LATTICE[name]
    coef = workloads.coef_uniform(lat, ext, seed=11)
    pts = torch.from_numpy(sorted_points(name, ext, 200_003, seed=3)).cuda()
    plain = volume(name, ext, coef, layout).eval(pts)
    for kw in ({"stage": 1}, {"stage": 1, "blocks_per_sm": 1}, {"stage": 1, "block": 128}, {"stage": 8},
               {"stage": 16}):
        vs = volume(name, ext, coef, layout, **kw)
        got = vs.eval(pts)
        vs.spline.status()
        assert bitwise_equal(got, plain), kw


@pytest.mark.parametrize("name", ["fcc6", "bcc_quintic", "tricubic"])
def test_staged_unsorted_and_sparse_points(name):
    """Unsorted points: almost no tile fits, the global path runs; a few
    points per block: every tile fits."""
    ext = EXT[name]
    lat = workloads.SPLINE_LATTICE[name]
    coef = workloads.coef_uniform(lat, ext, seed=12)
    lo, hi = workloads.bounding_box(lat, ext)
    plain_v = volume(name, ext, coef, "interleaved")
    staged_v = volume(name, ext, coef, "interleaved", stage=1)
    for n in (1, 31, 257, 40_000):
        pts = torch.from_numpy(workloads.points_uniform(n, lo - 2.0, hi + 2.0, seed=n)).cuda()
        assert bitwise_equal(staged_v.eval(pts), plain_v.eval(pts)), n
    # all points of a block inside one small cube: the tile always fits
    c = (lo + hi) / 2
    pts = torch.from_numpy(workloads.points_uniform(10_000, c - 2.0, c + 2.0, seed=77)).cuda()
    assert bitwise_equal(staged_v.eval(pts), plain_v.eval(pts))
    staged_v.spline.status()


@pytest.mark.parametrize("name", ["fcc6", "bcc_quintic"])
def test_staged_without_tensor_map_reads_global_memory(name):
    """Coset-major rows of ext0 = 22 floats are not a multiple of 16 bytes: no
    tensor map, every block takes the global path, results unchanged."""
    ext = (22, 20, 18)
    lat = workloads.SPLINE_LATTICE[name]
    coef = workloads.coef_uniform(lat, ext, seed=13)
    pts = torch.from_numpy(sorted_points(name, ext, 50_000, seed=4)).cuda()
    plain = volume(name, ext, coef, "coset").eval(pts)
    got = volume(name, ext, coef, "coset", stage=1).eval(pts)
    assert bitwise_equal(got, plain)


@pytest.mark.parametrize("name", NAMES)
def test_staged_matches_oracle(name):
    ext = EXT[name]
    lat = workloads.SPLINE_LATTICE[name]
    coef = workloads.coef_uniform(lat, ext, seed=14)
    p = sorted_points(name, ext, 120_000, seed=5, specials=False)
    got = volume(name, ext, coef, "interleaved", stage=1).eval(torch.from_numpy(p).cuda()).cpu().numpy()
    idx = np.random.default_rng(0).choice(len(p), 1500, replace=False)
    spec = ORACLE_SPEC[name]().with_extent(ext)
    want = oracle.eval_sum(spec, coef.astype(np.float64).ravel(), p[idx].astype(np.float64))
    assert np.max(np.abs(got[idx].astype(np.float64) - want)) <= TOL * np.abs(coef).max()


def test_stage_variant_rejects_what_it_cannot_stage():
    from paper_2102_08518_b300.api import Spline
    from paper_2102_08518_b300._abi import LsError
    for kw, dt, name in (({"stage": 6}, "f32", "fcc6"), ({"stage": 1}, "bf16", "fcc6"),
                         ({"stage": 1, "brick": 1}, "f32", "bcc_quintic"), ({"stage": 1}, "f32", "zp"),
                         ({"stage": 80}, "f32", "fcc6")):
        with pytest.raises(LsError):
            Spline(name, dt, **kw)
