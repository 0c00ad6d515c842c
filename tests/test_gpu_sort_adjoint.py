"""Morton sort, permutation, FP64 dot and the deterministic adjoint on the GPU."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from oracle import specs as ospecs

pytestmark = pytest.mark.gpu

ORACLE_SPEC = {"tricubic": ospecs.tricubic, "trilinear": ospecs.trilinear, "triquadratic": ospecs.triquadratic,
               "bcc_linear": ospecs.bcc_linear, "bcc_quintic": ospecs.bcc_quintic, "bcc_quartic": ospecs.bcc_quartic,
               "voronoi2_bcc": ospecs.voronoi2_bcc, "voronoi2_fcc": ospecs.voronoi2_fcc, "fcc6": ospecs.fcc6,
               "zp": ospecs.zp2d}
SMALL_EXT = {"tricubic": (12, 11, 10), "trilinear": (9, 12, 10), "triquadratic": (11, 9, 12),
             "bcc_linear": (7, 6, 8), "bcc_quintic": (8, 7, 6), "fcc6": (7, 8, 6), "zp": (13, 11)}


def _expected_morton(pts, origin, cell):
    """Keys from the oracle's Morton definition on cells computed in FP32 like the kernel."""
    inv = np.float32(1.0) / np.float32(cell)
    c = np.floor((pts.astype(np.float32) - np.asarray(origin, np.float32)) * inv)
    c = np.clip(c, 0, 1023).astype(np.int64)
    keys = np.array([oracle.morton3(int(a), int(b), int(d)) for a, b, d in c], dtype=np.int64)
    return keys


@pytest.mark.parametrize("n,hi", [(1, 300.0), (1000, 300.0), (4096 * 3 + 17, 300.0), (200003, 300.0),
                                  (200003, 2500.0), (70001, 7.0), (50000, 1.0)])
def test_morton_sort_bit_exact(n, hi):
    """Keys of 30 bits (box 2500 / cell 2: cells clamped at 1023), 24 bits
    (the top digit constant), 6 bits (three constant digits) and one key for
    every point (points in [0, 1) with cell 2: every pass keeps the input
    order)."""
    from paper_2102_08518_b300.api import morton_sort
    rng = np.random.default_rng(n)
    pts = rng.uniform(-5 if hi > 2 else 0, hi, (n, 3)).astype(np.float32)
    pts[: n // 3] = np.round(pts[: n // 3])        # many equal keys: stability matters
    perm, keys = morton_sort(torch.from_numpy(pts).cuda(), origin=(0.0, 0.0, 0.0), cell=2.0, want_keys=True)
    torch.cuda.synchronize()
    want_keys = _expected_morton(pts, (0, 0, 0), 2.0)
    want_perm = np.argsort(want_keys, kind="stable")
    assert np.array_equal(perm.cpu().numpy(), want_perm)
    assert np.array_equal(keys.cpu().numpy().astype(np.int64) & 0xFFFFFFFF, want_keys[want_perm])


@pytest.mark.parametrize("n,width", [(5001, 3), (1, 3), (777, 1), (3000, 2), (4099, 4), (513, 5),
                                     ((1 << 21) + 7, 3)])
def test_permute_rows_roundtrip(n, width):
    """Rows of 1-4 floats (the batched-rows kernels: several rows per thread,
    strided by the grid; n spanning several strides and a ragged end) and a
    wider row (the per-element kernel), forward and inverse."""
    from paper_2102_08518_b300.api import permute_rows
    rng = np.random.default_rng(5 + n + width)
    x = torch.from_numpy(rng.normal(size=(n, width)).astype(np.float32)).cuda()
    perm = torch.from_numpy(rng.permutation(n).astype(np.int32)).cuda()
    y = permute_rows(x, perm)
    assert torch.equal(y, x[perm.long()])
    z = permute_rows(y, perm, inverse=True)
    assert torch.equal(z, x)


def test_dot_f64():
    from paper_2102_08518_b300.api import dot_f64
    rng = np.random.default_rng(6)
    a = rng.normal(size=1_000_003).astype(np.float32)
    b = rng.normal(size=1_000_003).astype(np.float32)
    got = dot_f64(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()).item()
    want = float(np.dot(a.astype(np.float64), b.astype(np.float64)))
    assert abs(got - want) <= 1e-12 * np.sum(np.abs(a.astype(np.float64) * b))


def _vol(name, ext, coef):
    from paper_2102_08518_b300.api import Spline, Volume
    return Volume(Spline(name, "f32"), ext, torch.from_numpy(coef).cuda())


@pytest.mark.parametrize("name", ["tricubic", "trilinear", "triquadratic", "bcc_linear", "bcc_quintic", "fcc6", "zp"])
def test_deterministic_adjoint_matches_oracle_and_is_bitwise_stable(name):
    lat = workloads.SPLINE_LATTICE[name]
    ext = SMALL_EXT[name]
    lo, hi = workloads.bounding_box(lat, ext)
    n = 5000
    pts = workloads.points_uniform(n, lo - 2.0, hi + 2.0, seed=51)
    g = np.random.default_rng(52).normal(size=n).astype(np.float32)
    g[::7] = 0.0
    coef = workloads.coef_uniform(lat, ext, seed=53)
    vol = _vol(name, ext, coef)
    p = torch.from_numpy(pts).cuda()
    gg = torch.from_numpy(g).cuda()
    d1 = vol.adjoint(p, gg, deterministic=True)
    d2 = vol.adjoint(p, gg, deterministic=True)
    da = vol.adjoint(p, gg, deterministic=False)
    torch.cuda.synchronize()
    assert torch.equal(d1, d2)
    spec = ORACLE_SPEC[name]().with_extent(ext)
    want = oracle.adjoint(spec, pts.astype(np.float64), g.astype(np.float64))
    got = d1.cpu().numpy().astype(np.float64)
    scale = max(1.0, np.abs(want).max())
    assert np.max(np.abs(got - want)) <= 2e-5 * scale
    assert np.max(np.abs(da.cpu().numpy() - got)) <= 2e-5 * scale


def test_deterministic_adjoint_large_and_accumulating():
    """2^18 points: bitwise determinism, accumulation into dcoef, the adjoint
    identity <g, A c> = <A^T g, c>; the oracle checks a 2^11-point slice."""
    name, ext = "bcc_quintic", (32, 32, 32)
    coef = workloads.coef_uniform("bcc", ext, seed=61)
    lo, hi = workloads.bounding_box("bcc", ext)
    pts = workloads.points_uniform(1 << 18, lo, hi, seed=62)
    g = np.random.default_rng(63).normal(size=1 << 18).astype(np.float32)
    vol = _vol(name, ext, coef)
    p = torch.from_numpy(pts).cuda()
    gg = torch.from_numpy(g).cuda()
    base = torch.full((vol.n_coef,), 0.5, device="cuda")
    d1 = vol.adjoint(p, gg, dcoef=base.clone(), deterministic=True)
    d2 = vol.adjoint(p, gg, dcoef=base.clone(), deterministic=True)
    torch.cuda.synchronize()
    assert torch.equal(d1, d2)
    f = vol.eval(p)
    lhs = float(torch.dot(f.double(), gg.double()))
    rhs = float(torch.dot((d1 - base).double(), torch.from_numpy(coef.ravel()).cuda().double()))
    assert abs(lhs - rhs) <= 1e-4 * abs(lhs)
    sub = slice(0, 1 << 11)
    ds = vol.adjoint(p[sub], gg[sub], deterministic=True)
    torch.cuda.synchronize()
    spec = ORACLE_SPEC[name]().with_extent(ext)
    want = oracle.adjoint(spec, pts[sub].astype(np.float64), g[sub].astype(np.float64))
    assert np.max(np.abs(ds.cpu().numpy() - want)) <= 2e-5 * max(1.0, np.abs(want).max())


@pytest.mark.parametrize("name", ["tricubic", "trilinear", "triquadratic", "bcc_linear", "bcc_quintic", "fcc6", "zp"])
def test_fixed_point_adjoint_is_bitwise_stable_and_matches_oracle(name):
    """Integer atomics on values rounded to multiples of 2^-s: the same bits on
    every run and for a shuffled point order, and the oracle's sums."""
    lat = workloads.SPLINE_LATTICE[name]
    ext = SMALL_EXT[name]
    lo, hi = workloads.bounding_box(lat, ext)
    n = 6000
    pts = workloads.points_uniform(n, lo - 2.0, hi + 2.0, seed=151)
    g = np.random.default_rng(152).normal(size=n).astype(np.float32)
    coef = workloads.coef_uniform(lat, ext, seed=153)
    vol = _vol(name, ext, coef)
    p, gg = torch.from_numpy(pts).cuda(), torch.from_numpy(g).cuda()
    d1 = vol.adjoint(p, gg, deterministic="fixed")
    d2 = vol.adjoint(p, gg, deterministic="fixed")
    perm = torch.from_numpy(np.random.default_rng(154).permutation(n)).cuda()
    d3 = vol.adjoint(p[perm].contiguous(), gg[perm].contiguous(), deterministic="fixed")
    torch.cuda.synchronize()
    assert torch.equal(d1, d2) and torch.equal(d1, d3)
    spec = ORACLE_SPEC[name]().with_extent(ext)
    want = oracle.adjoint(spec, pts.astype(np.float64), g.astype(np.float64))
    assert np.max(np.abs(d1.cpu().numpy() - want)) <= 2e-5 * max(1.0, np.abs(want).max())


@pytest.mark.parametrize("gscale", [1e-30, 1e-6, 1.0, 1e8, 1e25])
def test_fixed_point_adjoint_scale_follows_gout(gscale):
    """The power-of-two scale adapts to sum|g|: the relative error stays at the
    FP32 level for tiny and huge gradients, and g = 0 adds nothing."""
    name, ext = "bcc_quintic", SMALL_EXT["bcc_quintic"]
    lo, hi = workloads.bounding_box("bcc", ext)
    n = 3000
    pts = workloads.points_uniform(n, lo, hi, seed=161)
    g = (np.random.default_rng(162).normal(size=n) * gscale).astype(np.float32)
    vol = _vol(name, ext, workloads.coef_uniform("bcc", ext, seed=163))
    p = torch.from_numpy(pts).cuda()
    base = torch.full((vol.n_coef,), 0.25, device="cuda")
    d = vol.adjoint(p, torch.from_numpy(g).cuda(), dcoef=base.clone() * gscale, deterministic="fixed")
    z = vol.adjoint(p, torch.zeros(n, device="cuda"), dcoef=base.clone(), deterministic="fixed")
    torch.cuda.synchronize()
    assert torch.equal(z, base)
    spec = ORACLE_SPEC[name]().with_extent(ext)
    want = oracle.adjoint(spec, pts.astype(np.float64), g.astype(np.float64)) + 0.25 * gscale
    got = d.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - want)) <= 2e-5 * np.abs(want).max()
