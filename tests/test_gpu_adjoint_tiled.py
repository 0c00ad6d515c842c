"""The tiled adjoint (shared-memory sums per block of spatially sorted points).

A block whose points' stencils fit one tile sums its contributions in shared
memory and adds each touched coefficient once; other blocks take the
per-point path.  The FP32 form must agree with the per-point atomic adjoint
(and the FP64 oracle); the fixed-point form must give the bits of the
untiled fixed-point adjoint, whatever the tiling, because both add the same
integers.  Sorted, unsorted and far-outside points, both linear layouts, and
a bricked volume (which takes the untiled kernels).
"""
import numpy as np
import pytest
import torch

import oracle
import workloads
from oracle import specs as ospecs

pytestmark = pytest.mark.gpu

ORACLE_SPEC = {"tricubic": ospecs.tricubic, "trilinear": ospecs.trilinear, "bcc_linear": ospecs.bcc_linear,
               "bcc_quintic": ospecs.bcc_quintic, "bcc_quartic": ospecs.bcc_quartic,
               "voronoi2_bcc": ospecs.voronoi2_bcc, "voronoi2_fcc": ospecs.voronoi2_fcc, "fcc6": ospecs.fcc6, "zp": ospecs.zp2d}
EXT = {"tricubic": (40, 36, 30), "trilinear": (40, 32, 30), "bcc_linear": (24, 22, 20),
       "bcc_quintic": (24, 20, 18), "fcc6": (24, 20, 18), "zp": (40, 36)}


def n_cosets(name):
    return len(workloads.LATTICES[workloads.SPLINE_LATTICE[name]][2])


def morton_order_np(p, lo):
    q = np.floor(p - lo).astype(np.int64)
    key = np.zeros(len(p), np.int64)
    D = p.shape[1]
    for b in range(12):
        for a in range(D):
            key |= ((q[:, a] >> b) & 1) << (D * b + a)
    return np.argsort(key, kind="stable")


def points(name, ext, n, seed, sort=True):
    lat = workloads.SPLINE_LATTICE[name]
    lo, hi = workloads.bounding_box(lat, ext)
    p = workloads.points_uniform(n, lo - 1.5, hi + 1.5, seed=seed)
    if sort:
        p = p[morton_order_np(p, lo - 1.5)]
    p[n // 3] = lo - 30.0                      # far outside: contributes nothing
    return np.ascontiguousarray(p, dtype=np.float32)


def volume(name, ext, layout="coset", **kw):
    from paper_2102_08518_b300.api import Spline, Volume
    C = n_cosets(name)
    c = torch.zeros(C * int(np.prod(ext)), device="cuda")
    if layout == "bricked":
        kw["brick"] = 1
    return Volume(Spline(name, "f32", **kw), ext, c, layout=layout)


@pytest.mark.parametrize("layout", ["coset", "interleaved"])
@pytest.mark.parametrize("name", list(EXT))
def test_tiled_fixed_point_is_bitwise_the_untiled_fixed_point(name, layout):
    ext = EXT[name]
    vol = volume(name, ext, layout)
    g = torch.from_numpy(np.random.default_rng(1).standard_normal(60_001).astype(np.float32)).cuda()
    for sort in (True, False):
        p = torch.from_numpy(points(name, ext, 60_001, seed=2, sort=sort)).cuda()
        a = vol.adjoint(p, g, deterministic="fixed")
        b = vol.adjoint(p, g, deterministic="fixed", tiled=True)
        assert torch.equal(a, b), sort
        assert torch.equal(b, vol.adjoint(p, g, deterministic="fixed", tiled=True))


@pytest.mark.parametrize("layout", ["coset", "interleaved"])
@pytest.mark.parametrize("name", list(EXT))
def test_tiled_atomic_matches_the_atomic_adjoint(name, layout):
    ext = EXT[name]
    vol = volume(name, ext, layout)
    g = torch.from_numpy(np.random.default_rng(3).standard_normal(80_000).astype(np.float32)).cuda()
    p = torch.from_numpy(points(name, ext, 80_000, seed=4)).cuda()
    a = vol.adjoint(p, g)
    b = vol.adjoint(p, g, tiled=True)
    scale = float(torch.abs(a).max())
    assert float(torch.abs(a - b).max()) <= 1e-5 * max(scale, 1.0)


@pytest.mark.parametrize("name", ["bcc_quintic", "fcc6", "tricubic"])
def test_tiled_adjoint_matches_oracle(name):
    ext = {"bcc_quintic": (8, 8, 6), "fcc6": (8, 6, 8), "tricubic": (10, 10, 8)}[name]
    vol = volume(name, ext, "interleaved" if name != "tricubic" else "coset")
    pts = points(name, ext, 3000, seed=5)
    g = np.random.default_rng(6).standard_normal(len(pts))
    got = vol.adjoint(torch.from_numpy(pts).cuda(), torch.from_numpy(g.astype(np.float32)).cuda(), tiled=True)
    got = got.cpu().numpy().astype(np.float64)
    C = n_cosets(name)
    if name != "tricubic":
        got = np.ascontiguousarray(got.reshape(-1, C).T).ravel()        # interleaved -> coset-major
    spec = ORACLE_SPEC[name]().with_extent(ext)
    want = oracle.adjoint(spec, pts.astype(np.float64), g.astype(np.float32).astype(np.float64))
    assert np.max(np.abs(got - want)) <= 1e-4 * max(1.0, np.abs(want).max())


def test_tiled_modes_on_a_bricked_volume_take_the_untiled_kernels():
    name, ext = "bcc_quintic", (24, 20, 18)
    vol = volume(name, ext, "bricked")
    g = torch.ones(20_000, device="cuda")
    p = torch.from_numpy(points(name, ext, 20_000, seed=7)).cuda()
    assert torch.equal(vol.adjoint(p, g, deterministic="fixed"), vol.adjoint(p, g, deterministic="fixed", tiled=True))


def test_tiled_cg_fit_converges_like_the_untiled_one():
    from paper_2102_08518_b300.api import cg_fit
    name, ext = "bcc_quintic", (16, 16, 16)
    lat = workloads.SPLINE_LATTICE[name]
    lo, hi = workloads.bounding_box(lat, ext)
    pts = points(name, ext, 40_000, seed=8)
    y = torch.from_numpy(np.sin(0.2 * pts[:, 0]) * np.cos(0.15 * pts[:, 1]).astype(np.float32)).float().cuda()
    p = torch.from_numpy(pts).cuda()
    res = []
    for tiled in (False, True):
        vol = volume(name, ext, "interleaved")
        it, hist = cg_fit(vol, p, y, lam=1e-3, max_iter=30, rel_tol=1e-7, deterministic="fixed", tiled=tiled)
        res.append((it, hist, vol.coef.clone() if hasattr(vol, "coef") else None))
    assert res[0][0] == res[1][0]
    assert np.array_equal(res[0][1], res[1][1])          # fixed-point sums: the same bits, the same iterates
