"""GPU evaluation (ls_eval / ls_eval_grad / ls_adjoint_coef) against the FP64 oracle.

Tolerance: max |f_gpu - f_oracle| <= 2e-6 * ||c||_inf for FP32 arithmetic on
FP32 coefficients (the accuracy target of the benchmark configurations).  The
oracle evaluates at the FP32 input points promoted to FP64.
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
               "voronoi2_bcc": ospecs.voronoi2_bcc, "voronoi2_fcc": ospecs.voronoi2_fcc, "fcc6": ospecs.fcc6,
               "zp": ospecs.zp2d}
SMALL_EXT = {"tricubic": (12, 11, 10), "trilinear": (9, 12, 10), "triquadratic": (11, 9, 12),
             "bcc_linear": (7, 6, 8), "bcc_quintic": (8, 7, 6), "bcc_quartic": (7, 8, 7), "fcc6": (7, 8, 6),
             "zp": (13, 11), "voronoi2_bcc": (6, 7, 6), "voronoi2_fcc": (6, 6, 7)}
ALL_NAMES = ["tricubic", "trilinear", "triquadratic", "bcc_linear", "bcc_quintic", "bcc_quartic", "fcc6", "zp",
             "voronoi2_bcc", "voronoi2_fcc"]
# splines whose gradient jumps across knot planes (C0): gradients are compared off them
C0_SPLINES = ("bcc_linear", "trilinear", "voronoi2_bcc", "voronoi2_fcc")
_SPLINES = {}


def spline(name, dtype="f32", **kw):
    from paper_2102_08518_b300.api import Spline
    key = (name, dtype, tuple(sorted(kw.items())))
    if key not in _SPLINES:
        _SPLINES[key] = Spline(name, dtype, **kw)
    return _SPLINES[key]


def volume(name, ext, coef_np, dtype="f32"):
    from paper_2102_08518_b300.api import Volume, TORCH_DTYPES
    sp = spline(name, dtype)
    c = torch.from_numpy(coef_np).to("cuda", TORCH_DTYPES[dtype]).contiguous()
    return Volume(sp, ext, c)


def oracle_eval(name, ext, coef_np, pts):
    spec = ORACLE_SPEC[name]().with_extent(ext)
    return oracle.eval_sum(spec, coef_np.astype(np.float64).ravel(), pts.astype(np.float64))


def gpu_eval(vol, pts_np):
    p = torch.from_numpy(pts_np).cuda()
    out = vol.eval(p)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("name", ALL_NAMES)
@pytest.mark.parametrize("n", [1, 31, 4133])
def test_small_volume_every_point(name, n):
    """All points, including beyond the arrays (zero extension, checked gathers)."""
    lat = workloads.SPLINE_LATTICE[name]
    ext = SMALL_EXT[name]
    coef = workloads.coef_uniform(lat, ext, seed=11)
    lo, hi = workloads.bounding_box(lat, ext)
    pts = workloads.points_uniform(n, lo - 2.5, hi + 2.5, seed=n)
    got = gpu_eval(volume(name, ext, coef), pts)
    want = oracle_eval(name, ext, coef, pts)
    assert np.max(np.abs(got - want)) <= TOL * np.abs(coef).max()


@pytest.mark.parametrize("name", ["tricubic", "trilinear", "triquadratic", "bcc_linear", "bcc_quintic", "bcc_quartic",
                                  "fcc6", "voronoi2_bcc", "voronoi2_fcc"])
def test_special_points(name):
    """Lattice sites, half-integers, mirror and BSP planes, and the edges."""
    lat = workloads.SPLINE_LATTICE[name]
    ext = SMALL_EXT[name]
    coef = workloads.coef_uniform(lat, ext, seed=12)
    lo, hi = workloads.bounding_box(lat, ext)
    rng = np.random.default_rng(13)
    p = rng.uniform(lo, hi, (600, 3))
    p[:100] = np.round(p[:100])
    p[100:200] = np.round(p[100:200] * 2) / 2
    p[200:300, 1] = p[200:300, 0]
    d = rng.uniform(-0.5, 0.5, 100)
    p[300:400] = np.round(p[300:400]) + np.stack([d, d, 1 - 2 * np.abs(d)], 1) * 0.5
    p[400:450] = np.array(lo)
    p[450:500] = np.array(hi)
    pts = p.astype(np.float32)
    got = gpu_eval(volume(name, ext, coef), pts)
    want = oracle_eval(name, ext, coef, pts)
    assert np.max(np.abs(got - want)) <= TOL * np.abs(coef).max()


def test_non_finite_and_far_points():
    ext = SMALL_EXT["bcc_quintic"]
    coef = workloads.coef_uniform("bcc", ext, seed=14)
    vol = volume("bcc_quintic", ext, coef)
    pts = np.array([[np.nan, 1, 1], [1e9, 2, 2], [-1e30, 0, 0], [5, 5, 5], [np.inf, 0, 0]], np.float32)
    got = gpu_eval(vol, pts)
    assert np.isnan(got[0]) and got[1] == 0.0 and got[2] == 0.0 and got[4] == 0.0
    want = oracle_eval("bcc_quintic", ext, coef, pts[3:4])
    assert abs(got[3] - want[0]) <= TOL * np.abs(coef).max()


def test_zero_points():
    from paper_2102_08518_b300.api import Volume
    ext = SMALL_EXT["fcc6"]
    vol = Volume(spline("fcc6"), ext)
    out = vol.eval(torch.zeros(0, 3, device="cuda"))
    assert out.numel() == 0


# ---------------------------------------------------------------------------
# the benchmark workloads at full size (sampled oracle)
# ---------------------------------------------------------------------------

def _sampled_check(name, ext, coef, pts, n_sample, seed):
    vol = volume(name, ext, coef)
    got = gpu_eval(vol, pts)
    assert np.all(np.isfinite(got))
    idx = np.random.default_rng(seed).choice(len(pts), n_sample, replace=False)
    want = oracle_eval(name, ext, coef, pts[idx])
    err = np.max(np.abs(got[idx] - want))
    assert err <= TOL * np.abs(coef).max(), err
    return got


def test_tricubic_64cubed_all_points():
    ext = (64, 64, 64)
    coef = workloads.coef_uniform("cc", ext, seed=0)
    pts = workloads.points_uniform(1 << 18, [2, 2, 2], [61, 61, 61], seed=0)
    got = gpu_eval(volume("tricubic", ext, coef), pts)
    want = oracle_eval("tricubic", ext, coef, pts)
    assert np.max(np.abs(got - want)) <= TOL * np.abs(coef).max()


@pytest.mark.parametrize("name", ["bcc_linear", "bcc_quintic"])
def test_bcc_128_per_coset_uniform_and_rays(name):
    ext = (128, 128, 128)
    coef = workloads.coef_smooth("bcc", ext, seed=0)
    lo, hi = workloads.inner_box(name, ext)
    uni = workloads.points_uniform(1 << 24, lo, hi, seed=1)
    _sampled_check(name, ext, coef, uni, 1024, 2)
    rays = workloads.points_rays(4096, 4096, lo, hi, seed=3)
    _sampled_check(name, ext, coef, rays, 1024, 4)


def test_fcc_256_box_value_and_gradient():
    ext = (128, 128, 128)
    coef = workloads.coef_uniform("fcc", ext, seed=0)
    lo, hi = workloads.inner_box("fcc6", ext)
    pts = workloads.points_uniform(1 << 26, lo, hi, seed=5)
    _sampled_check("fcc6", ext, coef, pts, 1024, 6)
    # gradient on a slice of the same workload
    vol = volume("fcc6", ext, coef)
    sub = pts[: 1 << 20]
    val, grad = vol.eval_grad(torch.from_numpy(sub).cuda())
    torch.cuda.synchronize()
    idx = np.random.default_rng(7).choice(len(sub), 512, replace=False)
    spec = ORACLE_SPEC["fcc6"]().with_extent(ext)
    f, g = oracle.eval_sum_grad(spec, coef.astype(np.float64).ravel(), sub[idx].astype(np.float64))
    assert np.max(np.abs(val.cpu().numpy()[idx] - f)) <= TOL * np.abs(coef).max()
    assert np.max(np.abs(grad.cpu().numpy()[idx] - g)) <= 1e-5 * np.abs(coef).max()


# ---------------------------------------------------------------------------
# gradient and adjoint on small volumes
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", ALL_NAMES)
def test_gradient_matches_oracle(name):
    lat = workloads.SPLINE_LATTICE[name]
    ext = SMALL_EXT[name]
    coef = workloads.coef_uniform(lat, ext, seed=21)
    lo, hi = workloads.bounding_box(lat, ext)
    pts = workloads.points_uniform(500 if name.startswith("voronoi") else 2000, lo - 1.0, hi + 1.0, seed=22)
    vol = volume(name, ext, coef)
    val, grad = vol.eval_grad(torch.from_numpy(pts).cuda())
    torch.cuda.synchronize()
    spec = ORACLE_SPEC[name]().with_extent(ext)
    f, g = oracle.eval_sum_grad(spec, coef.astype(np.float64).ravel(), pts.astype(np.float64))
    assert np.max(np.abs(val.cpu().numpy() - f)) <= TOL * np.abs(coef).max()
    gg = grad.cpu().numpy()
    if name in C0_SPLINES:
        # C0 spline: the gradient jumps across knot planes; compare off them
        ok = np.ones(len(pts), bool)
        h = 1e-4
        for i in range(3):
            e = np.zeros(3)
            e[i] = h
            fp = oracle.eval_sum(spec, coef.astype(np.float64).ravel(), pts + e)
            fm = oracle.eval_sum(spec, coef.astype(np.float64).ravel(), pts - e)
            # inside a piece the one-sided slopes differ by h |f''|: 0 for the
            # piecewise-linear splines, up to ~1e-3 for the cubic Voronoi pieces
            ok &= np.abs((fp - f) / h - (f - fm) / h) < (1e-2 if name.startswith("voronoi") else 1e-6)
        gg, g = gg[ok], g[ok]
        assert ok.sum() > len(pts) // 2
    assert np.max(np.abs(gg - g)) <= 1e-5 * np.abs(coef).max()


@pytest.mark.parametrize("warp", [False, True])
@pytest.mark.parametrize("name", ALL_NAMES)
def test_adjoint_atomic_matches_oracle(name, warp):
    lat = workloads.SPLINE_LATTICE[name]
    ext = SMALL_EXT[name]
    lo, hi = workloads.bounding_box(lat, ext)
    pts = workloads.points_uniform(3000, lo - 1.0, hi + 1.0, seed=31)
    g = np.random.default_rng(32).normal(size=3000).astype(np.float32)
    coef = workloads.coef_uniform(lat, ext, seed=33)
    vol = volume(name, ext, coef)
    dc = vol.adjoint(torch.from_numpy(pts).cuda(), torch.from_numpy(g).cuda(), warp_aggregated=warp)
    torch.cuda.synchronize()
    spec = ORACLE_SPEC[name]().with_extent(ext)
    want = oracle.adjoint(spec, pts.astype(np.float64), g.astype(np.float64))
    got = dc.cpu().numpy().astype(np.float64)
    tol_adj = 2e-6 * max(1.0, np.abs(want).max()) * 8
    assert np.max(np.abs(got - want)) <= tol_adj
    # dot-product identity with the forward kernel: <A c, g> = <c, A^T g> holds
    # exactly, so the two FP32 results differ by at most their per-value error
    # bounds (forward TOL max|c| per point, adjoint tol_adj per site) weighted
    # by |g| and |c|; the sums themselves may cancel to almost nothing
    fwd = gpu_eval(vol, pts)
    c64 = coef.ravel().astype(np.float64)
    bound = TOL * np.abs(coef).max() * np.abs(g).sum() + tol_adj * np.abs(c64).sum()
    assert abs(fwd @ g.astype(np.float64) - got @ c64) <= bound


@pytest.mark.parametrize("dtype,bound", [("bf16", 2.0 ** -8), ("f16", 2.0 ** -11)])
@pytest.mark.parametrize("name", ["tricubic", "bcc_quintic", "fcc6"])
def test_half_storage(name, dtype, bound):
    """Half-precision storage, FP32 arithmetic: vs the oracle on the rounded
    coefficients (FP32 tolerance) and on the original ones (storage bound)."""
    lat = workloads.SPLINE_LATTICE[name]
    ext = SMALL_EXT[name]
    coef = workloads.coef_uniform(lat, ext, seed=41)
    tdt = {"bf16": torch.bfloat16, "f16": torch.float16}[dtype]
    rounded = torch.from_numpy(coef).to(tdt).float().numpy()
    lo, hi = workloads.bounding_box(lat, ext)
    pts = workloads.points_uniform(3000, lo - 1.0, hi + 1.0, seed=42)
    got = gpu_eval(volume(name, ext, rounded, dtype), pts)
    want_r = oracle_eval(name, ext, rounded, pts)
    want = oracle_eval(name, ext, coef, pts)
    cmax = np.abs(coef).max()
    assert np.max(np.abs(got - want_r)) <= TOL * cmax
    assert np.max(np.abs(got - want)) <= (bound + TOL) * cmax


@pytest.mark.parametrize("pinned", [True, False])
def test_eval_host_multi_matches_device_eval(pinned):
    """Host buffers, several volumes, chunked and overlapped: equal to ls_eval."""
    from paper_2102_08518_b300.api import eval_host_multi
    ext = (16, 16, 16)
    coef_q = workloads.coef_smooth("bcc", ext, seed=1)
    coef_l = workloads.coef_uniform("bcc", ext, seed=2)
    vq, vl = volume("bcc_quintic", ext, coef_q), volume("bcc_linear", ext, coef_l)
    lo, hi = workloads.bounding_box("bcc", ext)
    n = (1 << 20) * 2 + 12345                      # more than two chunks, ragged tail
    pts = workloads.points_uniform(n, lo, hi, seed=3)
    hp = torch.from_numpy(pts)
    outs = [torch.empty(n), torch.empty(n)]
    if pinned:
        hp = hp.pin_memory()
        outs = [o.pin_memory() for o in outs]
    eval_host_multi([vq, vl], hp, outs)
    dp = torch.from_numpy(pts).cuda()
    refq, refl = vq.eval(dp), vl.eval(dp)
    torch.cuda.synchronize()
    assert torch.equal(outs[0], refq.cpu()) and torch.equal(outs[1], refl.cpu())
    out1 = torch.empty(n)
    vq.eval_host(torch.from_numpy(pts), out1)
    assert torch.equal(out1, refq.cpu())


@pytest.mark.parametrize("name", ["bcc_linear", "bcc_quintic", "fcc6", "zp"])
@pytest.mark.parametrize("T", [4, 8])
def test_coherent_reuse_variant_is_bitwise_identical(name, T):
    """Runs of T consecutive points per thread, reusing gathers and the
    coefficient transform while the cell does not change: same bits as the
    one-point-per-thread kernel, for ray-ordered, random and edge points."""
    from paper_2102_08518_b300.api import Spline, Volume
    lat = workloads.SPLINE_LATTICE[name]
    ext = SMALL_EXT[name] if name == "zp" else (24, 24, 24)
    coef = torch.from_numpy(workloads.coef_uniform(lat, ext, seed=71)).cuda()
    lo, hi = workloads.bounding_box(lat, ext)
    sets = [workloads.points_uniform(10007, lo - 2.0, hi + 2.0, seed=72)]
    if len(ext) == 3:
        sets.append(workloads.points_rays(64, 333, lo, hi, seed=73))
    base = Volume(spline(name), ext, coef)
    reuse = Volume(Spline(name, "f32", pts_per_thread=T), ext, coef)
    for pts in sets:
        p = torch.from_numpy(pts).cuda()
        a, b = base.eval(p), reuse.eval(p)
        torch.cuda.synchronize()
        assert torch.equal(a, b)


@pytest.mark.parametrize("name", ["bcc_linear", "bcc_quintic", "fcc6", "zp"])
def test_centroid_expansion_variant(name):
    """The tables expanded about the region centroids (an autotuning choice)."""
    from paper_2102_08518_b300.api import Spline, Volume
    lat = workloads.SPLINE_LATTICE[name]
    ext = SMALL_EXT[name]
    coef = workloads.coef_uniform(lat, ext, seed=81)
    lo, hi = workloads.bounding_box(lat, ext)
    pts = workloads.points_uniform(4000, lo - 2.0, hi + 2.0, seed=82)
    vol = Volume(Spline(name, "f32", expansion="centroid"), ext, torch.from_numpy(coef).cuda())
    got = gpu_eval(vol, pts)
    want = oracle_eval(name, ext, coef, pts)
    assert np.max(np.abs(got - want)) <= TOL * np.abs(coef).max()


@pytest.mark.parametrize("name", ["tricubic", "bcc_quintic", "fcc6", "zp"])
def test_warp_aggregated_adjoint_with_shared_sites(name):
    """Points in clusters of 1..40 copies of a few positions (plus edge points), so
    that lanes of one warp hit the same sites in groups of every size up to 32:
    the shuffle reduction inside the groups must give the oracle's sums."""
    lat = workloads.SPLINE_LATTICE[name]
    ext = SMALL_EXT[name]
    lo, hi = workloads.bounding_box(lat, ext)
    rng = np.random.default_rng(91)
    base = workloads.points_uniform(60, lo - 1.0, hi + 1.0, seed=92)
    reps = rng.integers(1, 41, size=len(base))
    pts = np.repeat(base, reps, axis=0)
    pts[::5] += rng.uniform(-0.01, 0.01, pts[::5].shape).astype(np.float32)
    g = rng.normal(size=len(pts)).astype(np.float32)
    g[::11] = 0.0
    coef = workloads.coef_uniform(lat, ext, seed=93)
    vol = volume(name, ext, coef)
    p, gg = torch.from_numpy(pts).cuda(), torch.from_numpy(g).cuda()
    dw = vol.adjoint(p, gg, warp_aggregated=True)
    da = vol.adjoint(p, gg)
    torch.cuda.synchronize()
    spec = ORACLE_SPEC[name]().with_extent(ext)
    want = oracle.adjoint(spec, pts.astype(np.float64), g.astype(np.float64))
    scale = max(1.0, np.abs(want).max())
    assert np.max(np.abs(dw.cpu().numpy() - want)) <= 2e-5 * scale
    assert np.max(np.abs(da.cpu().numpy() - want)) <= 2e-5 * scale


@pytest.mark.parametrize("name", ["bcc_linear", "bcc_quintic", "fcc6", "zp"])
@pytest.mark.parametrize("block,bps", [(128, 1), (256, 2)])
def test_pipelined_variant(name, block, bps):
    """Gathers of a thread's next point in flight while the current one is
    evaluated: the oracle's values for every point count (odd, even, fewer points
    than threads) and special points (NaN, far away)."""
    from paper_2102_08518_b300.api import Spline, Volume
    lat = workloads.SPLINE_LATTICE[name]
    ext = SMALL_EXT[name]
    coef = workloads.coef_uniform(lat, ext, seed=95)
    lo, hi = workloads.bounding_box(lat, ext)
    sp = Spline(name, "f32", block=block, blocks_per_sm=bps, pipeline=1)
    vol = Volume(sp, ext, torch.from_numpy(coef).cuda())
    plain = volume(name, ext, coef)
    for n in (1, 2, 3, 1000, 148 * block * bps * 3 + 17):
        pts = workloads.points_uniform(n, lo - 2.0, hi + 2.0, seed=n + 96)
        if n > 10:
            pts[5] = np.nan
            pts[7] = 1e9
        got = gpu_eval(vol, pts)
        ref = gpu_eval(plain, pts)
        assert np.array_equal(np.isnan(got), np.isnan(ref))
        ok = ~np.isnan(ref)
        assert np.max(np.abs(got[ok] - ref[ok])) <= 1e-6 * np.abs(coef).max()
        sub = np.flatnonzero(ok)[:600]
        want = oracle_eval(name, ext, coef, pts[sub])
        assert np.max(np.abs(got[sub] - want)) <= TOL * np.abs(coef).max()


@pytest.mark.parametrize("name", ["bcc_linear", "bcc_quintic", "fcc6", "zp"])
@pytest.mark.parametrize("block,producers", [(512, 2), (256, 1), (512, 4)])
def test_warp_specialized_variant(name, block, producers):
    """Producer warps gather into shared-memory slots, consumer warps evaluate:
    the oracle's values and the plain kernel's for point counts below one tile,
    with partial tiles and with several rounds per block; no wait gives up."""
    from paper_2102_08518_b300.api import Spline, Volume
    lat = workloads.SPLINE_LATTICE[name]
    ext = SMALL_EXT[name]
    coef = workloads.coef_uniform(lat, ext, seed=97)
    lo, hi = workloads.bounding_box(lat, ext)
    sp = Spline(name, "f32", block=block, producers=producers)
    vol = Volume(sp, ext, torch.from_numpy(coef).cuda())
    plain = volume(name, ext, coef)
    tile = 32 * (block // 32 - producers)
    for n in (1, 31, tile - 1, tile + 1, 148 * tile * 3 + 77):
        pts = workloads.points_uniform(n, lo - 2.0, hi + 2.0, seed=n + 98)
        if n > 40:
            pts[33] = np.nan
            pts[35] = -1e9
        got = gpu_eval(vol, pts)
        ref = gpu_eval(plain, pts)
        assert np.array_equal(np.isnan(got), np.isnan(ref))
        ok = ~np.isnan(ref)
        assert np.max(np.abs(got[ok] - ref[ok])) <= 1e-6 * np.abs(coef).max()
        sub = np.flatnonzero(ok)[:600]
        want = oracle_eval(name, ext, coef, pts[sub])
        assert np.max(np.abs(got[sub] - want)) <= TOL * np.abs(coef).max()
    sp.status()
