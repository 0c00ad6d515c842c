"""The coset-interleaved and bricked coefficient layouts against the FP64 oracle.

An interleaved volume holds the values of all cosets at one grid index next to
each other (element q * C + j instead of j * P + q); a bricked one cuts the
grid into 2 x 2 x 2 bricks (2 x 2 in 2D), x fastest inside, cosets adjacent.
The arrays here are made from the coset-major ones by numpy reshapes and
transposes, independently of the library's ls_relayout, which is checked bit
for bit on its own.  Every kernel (value, value + gradient, atomic, warp-
aggregated and deterministic adjoints, batched launch, CG fit) must give the
oracle's results with the same tolerances as the coset-major layout.
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
# whole bricks (even extents), so both layouts take them
SMALL_EXT = {"tricubic": (12, 10, 8), "trilinear": (8, 10, 6), "triquadratic": (12, 8, 10),
             "bcc_linear": (8, 6, 8), "bcc_quintic": (8, 6, 6), "bcc_quartic": (6, 8, 6), "fcc6": (8, 8, 6),
             "zp": (12, 10), "voronoi2_bcc": (6, 6, 6), "voronoi2_fcc": (6, 6, 6)}
NAMES = ["tricubic", "trilinear", "triquadratic", "bcc_linear", "bcc_quintic", "bcc_quartic", "fcc6", "zp",
         "voronoi2_bcc", "voronoi2_fcc"]
LAYOUTS = ["interleaved", "bricked"]
# the evaluation kernels also read the shifted bricked copies (3D)
EVAL_LAYOUTS = LAYOUTS + ["bricked_shifted", "bricked_shifted_xyz"]


def n_cosets(name):
    return len(workloads.LATTICES[workloads.SPLINE_LATTICE[name]][2])


def interleave_np(coef, C):
    """coset-major (C arrays of P) -> interleaved, by numpy."""
    return np.ascontiguousarray(coef.reshape(C, -1).T).ravel()


def deinterleave_np(arr, C):
    return np.ascontiguousarray(arr.reshape(-1, C).T).ravel()


def brick_np(coef, C, ext):
    """coset-major -> bricked: axes (C, zh, zl, yh, yl, xh, xl) reordered to
    (zh, yh, xh, zl, yl, xl, C): brick order x fastest, then inside the brick
    x, y, z, then the coset."""
    if len(ext) == 3:
        e0, e1, e2 = ext
        a = coef.reshape(C, e2 // 2, 2, e1 // 2, 2, e0 // 2, 2)
        return np.ascontiguousarray(a.transpose(1, 3, 5, 2, 4, 6, 0)).ravel()
    e0, e1 = ext
    a = coef.reshape(C, e1 // 2, 2, e0 // 2, 2)
    return np.ascontiguousarray(a.transpose(1, 3, 2, 4, 0)).ravel()


def brick_shifted_np(coef, C, ext, xyz=False):
    """coset-major -> the shifted bricked copies: copy s0 + 2 s1 (+ 4 s2) holds
    grid index i at (i0 + s0, i1 + s1, i2 (+ s2)) of a bricked array over
    extents (e0 + 2, e1 + 2, e2 (+ 2)), zero elsewhere."""
    e0, e1, e2 = ext
    a = coef.reshape(C, e2, e1, e0)
    pz = 2 if xyz else 0
    out = []
    for c in range(8 if xyz else 4):
        s0, s1, s2 = c & 1, (c >> 1) & 1, c >> 2
        pad = np.zeros((C, e2 + pz, e1 + 2, e0 + 2), dtype=coef.dtype)
        pad[:, s2:s2 + e2, s1:s1 + e1, s0:s0 + e0] = a
        out.append(brick_np(pad.ravel(), C, (e0 + 2, e1 + 2, e2 + pz)))
    return np.concatenate(out)


def unbrick_np(arr, C, ext):
    if len(ext) == 3:
        e0, e1, e2 = ext
        a = arr.reshape(e2 // 2, e1 // 2, e0 // 2, 2, 2, 2, C)
        return np.ascontiguousarray(a.transpose(6, 0, 3, 1, 4, 2, 5)).ravel()
    e0, e1 = ext
    a = arr.reshape(e1 // 2, e0 // 2, 2, 2, C)
    return np.ascontiguousarray(a.transpose(4, 0, 2, 1, 3)).ravel()


def to_layout_np(coef, C, ext, layout):
    if layout in ("bricked_shifted", "bricked_shifted_xyz"):
        return brick_shifted_np(coef, C, ext, xyz=layout.endswith("xyz"))
    return interleave_np(coef, C) if layout == "interleaved" else brick_np(coef, C, ext)


def from_layout_np(arr, C, ext, layout):
    return deinterleave_np(arr, C) if layout == "interleaved" else unbrick_np(arr, C, ext)


def ivolume(name, ext, coef_np, dtype="f32", layout="interleaved", **kw):
    from paper_2102_08518_b300.api import Spline, Volume, TORCH_DTYPES
    c = torch.from_numpy(to_layout_np(coef_np, n_cosets(name), ext, layout)).to("cuda", TORCH_DTYPES[dtype])
    if layout in ("bricked", "bricked_shifted", "bricked_shifted_xyz"):
        kw["brick"] = {"bricked": 1, "bricked_shifted": 2, "bricked_shifted_xyz": 3}[layout]
    return Volume(Spline(name, dtype, **kw), ext, c.contiguous(), layout=layout)


def test_numpy_brick_maps_are_inverse_and_match_the_definition():
    """The test's own bricked map against the element formula, element by element."""
    for C, ext in ((2, (8, 6, 4)), (1, (4, 2, 2)), (4, (10, 4, 6)), (2, (6, 6)), (1, (2, 2, 2))):
        P = int(np.prod(ext))
        coef = np.arange(C * P, dtype=np.int64)
        b = brick_np(coef, C, ext)
        assert np.array_equal(unbrick_np(b, C, ext), coef)
        e = tuple(ext) + (1,) * (3 - len(ext))
        V = 8 if len(ext) == 3 else 4
        for j in range(C):
            for i2 in range(e[2]):
                for i1 in range(e[1]):
                    for i0 in range(e[0]):
                        q = i0 + e[0] * (i1 + e[1] * i2)
                        bk = i0 // 2 + (e[0] // 2) * (i1 // 2 + (e[1] // 2) * (i2 // 2))
                        w = i0 % 2 + 2 * (i1 % 2) + 4 * (i2 % 2)
                        assert b[(bk * V + w) * C + j] == coef[j * P + q]


def oracle_eval(name, ext, coef_np, pts):
    spec = ORACLE_SPEC[name]().with_extent(ext)
    return oracle.eval_sum(spec, coef_np.astype(np.float64).ravel(), pts.astype(np.float64))


@pytest.mark.parametrize("C,ext", [(1, (100, 101, 99)), (2, (64, 50, 34)), (4, (12, 8, 10)), (2, (36, 22))])
@pytest.mark.parametrize("dtype", [torch.float16, torch.float32, torch.float64])
def test_relayout_matches_numpy_maps(C, ext, dtype):
    from paper_2102_08518_b300.api import relayout
    P = int(np.prod(ext))
    src = (torch.arange(C * P, device="cuda") % 4099).to(dtype) * 0.5 - 7.0
    ref = src.cpu().numpy()
    il = relayout(src, C, ext, to="interleaved")
    assert np.array_equal(il.cpu().numpy(), interleave_np(ref, C))
    assert torch.equal(relayout(il, C, ext, to="coset", src="interleaved"), src)
    if ext[0] % 2 == 0 and ext[1] % 2 == 0 and (len(ext) == 2 or ext[2] % 2 == 0):
        bk = relayout(src, C, ext, to="bricked")
        assert np.array_equal(bk.cpu().numpy(), brick_np(ref, C, ext))
        assert torch.equal(relayout(bk, C, ext, to="interleaved", src="bricked"), il)
        assert torch.equal(relayout(bk, C, ext, to="coset", src="bricked"), src)
        if len(ext) == 3:
            for lay, xyz in (("bricked_shifted", False), ("bricked_shifted_xyz", True)):
                sh = relayout(src, C, ext, to=lay)
                assert np.array_equal(sh.cpu().numpy(), brick_shifted_np(ref, C, ext, xyz))
                assert torch.equal(relayout(sh, C, ext, to="coset", src=lay), src)
                assert torch.equal(relayout(il, C, ext, to=lay, src="interleaved"), sh)


@pytest.mark.parametrize("layout", EVAL_LAYOUTS)
@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("n", [1, 33, 5003])
def test_interleaved_eval_every_point(name, n, layout):
    """Points inside and beyond the arrays (unchecked and bounds-checked gathers)."""
    if layout.startswith("bricked_shifted") and name == "zp":
        pytest.skip("the shifted bricked copies are 3D only")
    lat = workloads.SPLINE_LATTICE[name]
    ext = SMALL_EXT[name]
    coef = workloads.coef_uniform(lat, ext, seed=101)
    lo, hi = workloads.bounding_box(lat, ext)
    pts = workloads.points_uniform(n, lo - 2.5, hi + 2.5, seed=n + 100)
    vol = ivolume(name, ext, coef, layout=layout)
    got = vol.eval(torch.from_numpy(pts).cuda()).cpu().numpy().astype(np.float64)
    want = oracle_eval(name, ext, coef, pts)
    assert np.max(np.abs(got - want)) <= TOL * np.abs(coef).max()


@pytest.mark.parametrize("layout", EVAL_LAYOUTS)
@pytest.mark.parametrize("name", NAMES)
def test_interleaved_gradient(name, layout):
    if layout.startswith("bricked_shifted") and name == "zp":
        pytest.skip("the shifted bricked copies are 3D only")
    if name.startswith("voronoi"):
        pytest.skip("C0 Voronoi-spline gradients: tests/test_gpu_eval.py (coset-major) and the host kernel tests")
    lat = workloads.SPLINE_LATTICE[name]
    ext = SMALL_EXT[name]
    coef = workloads.coef_uniform(lat, ext, seed=102)
    lo, hi = workloads.bounding_box(lat, ext)
    pts = workloads.points_uniform(2000, lo - 1.0, hi + 1.0, seed=103)
    val, grad = ivolume(name, ext, coef, layout=layout).eval_grad(torch.from_numpy(pts).cuda())
    spec = ORACLE_SPEC[name]().with_extent(ext)
    f, g = oracle.eval_sum_grad(spec, coef.astype(np.float64).ravel(), pts.astype(np.float64))
    assert np.max(np.abs(val.cpu().numpy() - f)) <= TOL * np.abs(coef).max()
    gg = grad.cpu().numpy()
    if name in ("bcc_linear", "trilinear"):
        # C0: compare off the knot planes, where both one-sided gradients agree
        h = 1e-4
        ok = np.ones(len(pts), bool)
        for i in range(3):
            e = np.zeros(3)
            e[i] = h
            fp = oracle.eval_sum(spec, coef.astype(np.float64).ravel(), pts + e)
            fm = oracle.eval_sum(spec, coef.astype(np.float64).ravel(), pts - e)
            ok &= np.abs((fp - f) / h - (f - fm) / h) < 1e-6
        gg, g = gg[ok], g[ok]
        assert ok.sum() > 1000
    assert np.max(np.abs(gg - g)) <= 1e-5 * np.abs(coef).max()


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("name", NAMES)
def test_interleaved_adjoints(name, layout):
    """Atomic, warp-aggregated and deterministic adjoints write dcoef in the volume's layout."""
    lat = workloads.SPLINE_LATTICE[name]
    ext = SMALL_EXT[name]
    C = n_cosets(name)
    lo, hi = workloads.bounding_box(lat, ext)
    n = 4000
    pts = workloads.points_uniform(n, lo - 2.0, hi + 2.0, seed=104)
    g = np.random.default_rng(105).normal(size=n).astype(np.float32)
    coef = workloads.coef_uniform(lat, ext, seed=106)
    vol = ivolume(name, ext, coef, layout=layout)
    p, gg = torch.from_numpy(pts).cuda(), torch.from_numpy(g).cuda()
    da = vol.adjoint(p, gg, deterministic=False)
    dw = vol.adjoint(p, gg, warp_aggregated=True)
    d1 = vol.adjoint(p, gg, deterministic=True)
    d2 = vol.adjoint(p, gg, deterministic=True)
    df = vol.adjoint(p, gg, deterministic="fixed")
    torch.cuda.synchronize()
    assert torch.equal(d1, d2)
    spec = ORACLE_SPEC[name]().with_extent(ext)
    want = oracle.adjoint(spec, pts.astype(np.float64), g.astype(np.float64))
    scale = max(1.0, np.abs(want).max())
    for d in (da, dw, d1, df):
        got = from_layout_np(d.cpu().numpy().astype(np.float64), C, ext, layout)
        assert np.max(np.abs(got - want)) <= 2e-5 * scale


def test_upload_converts_dtype_and_layout():
    """ls_volume_upload takes coset-major values and fills an interleaved volume."""
    from paper_2102_08518_b300.api import Spline, Volume
    name, ext = "fcc6", SMALL_EXT["fcc6"]
    coef = workloads.coef_uniform("fcc", ext, seed=107)
    lo, hi = workloads.bounding_box("fcc", ext)
    pts = workloads.points_uniform(3000, lo - 1.0, hi + 1.0, seed=108)
    for dtype, src, layout in (("f32", torch.from_numpy(coef), "interleaved"),
                               ("bf16", torch.from_numpy(coef).double().cuda(), "interleaved"),
                               ("f32", torch.from_numpy(coef).cuda(), "bricked"),
                               ("f16", torch.from_numpy(coef), "bricked")):
        vol = Volume(Spline(name, dtype, brick=int(layout == "bricked")), ext, layout=layout)
        vol.upload(src)
        got = vol.eval(torch.from_numpy(pts).cuda()).cpu().numpy().astype(np.float64)
        rounded = torch.from_numpy(coef).to({"f32": torch.float32, "bf16": torch.bfloat16,
                                             "f16": torch.float16}[dtype]).float().numpy()
        want = oracle_eval(name, ext, rounded, pts)
        assert np.max(np.abs(got - want)) <= TOL * np.abs(coef).max()


def test_batched_plan_mixes_layouts():
    from paper_2102_08518_b300.api import Plan, Spline, Volume
    recipe = workloads.batch_recipe(15, seed=8, edges=(8, 12, 16), log2_lo=4, log2_hi=12)
    sps, vols, pts, outs, refs = {}, [], [], [], []
    for k, it in enumerate(recipe):
        lat = workloads.SPLINE_LATTICE[it.spline]
        C = len(workloads.LATTICES[lat][2])
        sps.setdefault(it.spline, Spline(it.spline, "f32"))
        sps.setdefault(it.spline + "_bk", Spline(it.spline, "f32", brick=1))
        c = workloads.coef_uniform(lat, it.ext, seed=it.seed)
        lo, hi = workloads.bounding_box(lat, it.ext)
        p = torch.from_numpy(workloads.points_uniform(it.n_points, lo - 1.0, hi + 1.0, seed=it.seed + 1)).cuda()
        if k % 3 == 1:
            v = Volume(sps[it.spline], it.ext, torch.from_numpy(interleave_np(c, C)).cuda(), layout="interleaved")
        elif k % 3 == 2 and it.ext[0] % 2 == 0 and it.ext[1] % 2 == 0 and (len(it.ext) < 3 or it.ext[2] % 2 == 0):
            v = Volume(sps[it.spline + "_bk"], it.ext, torch.from_numpy(brick_np(c, C, it.ext)).cuda(),
                       layout="bricked")
        else:
            v = Volume(sps[it.spline], it.ext, torch.from_numpy(c).cuda())
        ref = Volume(sps[it.spline], it.ext, torch.from_numpy(c).cuda()).eval(p)
        vols.append(v)
        pts.append(p)
        outs.append(torch.full((it.n_points,), float("nan"), device="cuda"))
        refs.append(ref)
    assert any(v.layout == "bricked" for v in vols) and any(v.layout == "interleaved" for v in vols)
    plan = Plan(vols, pts, outs, tile=256)
    plan.launch()
    plan.status()
    torch.cuda.synchronize()
    for o, r in zip(outs, refs):
        assert torch.equal(o, r)


@pytest.mark.parametrize("layout", LAYOUTS)
def test_interleaved_cg_fit_equals_coset_major_fit(layout):
    """The fit is the same linear algebra in another order of unknowns: the
    deterministic fits agree to rounding, and both fit the samples."""
    from paper_2102_08518_b300.api import Spline, Volume, cg_fit
    name, ext = "bcc_quintic", (8, 8, 8)
    lo, hi = workloads.bounding_box("bcc", ext)
    pts, y = workloads.gaussian_samples(1 << 13, lo, hi, seed=109)
    p, yy = torch.from_numpy(pts).cuda(), torch.from_numpy(y).cuda()
    va = Volume(Spline(name, "f32"), ext, torch.zeros(2 * 8 ** 3, device="cuda"))
    vb = Volume(Spline(name, "f32", brick=int(layout == "bricked")), ext, torch.zeros(2 * 8 ** 3, device="cuda"),
                layout=layout)
    ia, ha = cg_fit(va, p, yy, lam=1e-4, max_iter=60, rel_tol=0.0, deterministic=True)
    ib, hb = cg_fit(vb, p, yy, lam=1e-4, max_iter=60, rel_tol=0.0, deterministic=True)
    a = va.coef.cpu().numpy()
    b = from_layout_np(vb.coef.cpu().numpy(), 2, ext, layout)
    assert ia == ib == 60
    assert np.max(np.abs(a - b)) <= 1e-3 * np.abs(a).max()
    assert np.allclose(ha, hb, rtol=1e-3)


@pytest.mark.parametrize("layout", LAYOUTS + ["bricked_shifted"])
@pytest.mark.parametrize("name", ["bcc_linear", "bcc_quintic"])
def test_interleaved_bcc_full_size_sampled(name, layout):
    """BCC 2 x 128^3, 2^24 uniform and 2^24 ray points, in the autotuned launch
    configurations; the oracle checks 1024 sampled points per set."""
    from paper_2102_08518_b300.api import Volume, autotune, TUNE_CANDIDATES_SMALL
    ext = (128, 128, 128)
    coef = workloads.coef_smooth("bcc", ext, seed=0)
    lo, hi = workloads.inner_box(name, ext)
    c = torch.from_numpy(to_layout_np(coef, 2, ext, layout)).cuda()
    for ps, pts in (("uniform", workloads.points_uniform(1 << 24, lo, hi, seed=1)),
                    ("rays", workloads.points_rays(4096, 4096, lo, hi, seed=3))):
        p = torch.from_numpy(pts).cuda()
        sp = autotune(name, "f32", ext, c, [p], candidates=TUNE_CANDIDATES_SMALL, tag=f"bcc_step_{ps}",
                      layout=layout)
        got = Volume(sp, ext, c, layout=layout).eval(p).cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(got))
        idx = np.random.default_rng(5).choice(len(pts), 1024, replace=False)
        want = oracle_eval(name, ext, coef, pts[idx])
        assert np.max(np.abs(got[idx] - want)) <= TOL * np.abs(coef).max()


def test_bricked_layout_rejections():
    """Extents that are not whole bricks, and a layout the spline's kernels do not address."""
    from paper_2102_08518_b300 import _abi
    from paper_2102_08518_b300.api import Spline, Volume
    with pytest.raises(_abi.LsError):
        Volume(Spline("bcc_linear", "f32", brick=1), (7, 6, 6), layout="bricked")
    with pytest.raises(_abi.LsError):
        Volume(Spline("bcc_linear", "f32"), (8, 6, 6), layout="bricked")
    with pytest.raises(_abi.LsError):
        Volume(Spline("bcc_linear", "f32", brick=1), (8, 6, 6), layout="interleaved")


def test_shifted_copies_are_read_only():
    """The adjoint and the fit write coefficients; the shifted copies hold four
    of each, so those calls refuse them."""
    name, ext = "bcc_quintic", SMALL_EXT["bcc_quintic"]
    coef = workloads.coef_uniform("bcc", ext, seed=111)
    vol = ivolume(name, ext, coef, layout="bricked_shifted")
    p = torch.zeros(8, 3, device="cuda")
    with pytest.raises(RuntimeError, match="read-only"):
        vol.adjoint(p, torch.ones(8, device="cuda"))


def test_shifted_copies_hessian_and_batched_plan():
    from paper_2102_08518_b300.api import Plan, Spline, Volume
    name, ext = "bcc_quintic", SMALL_EXT["bcc_quintic"]
    coef = workloads.coef_uniform("bcc", ext, seed=112)
    lo, hi = workloads.bounding_box("bcc", ext)
    pts = workloads.points_uniform(3000, lo - 1.0, hi + 1.0, seed=113)
    p = torch.from_numpy(pts).cuda()
    vs = ivolume(name, ext, coef, layout="bricked_shifted")
    vc = Volume(Spline(name, "f32"), ext, torch.from_numpy(coef).cuda())
    f1, g1, h1 = vs.eval_hess(p)
    f2, g2, h2 = vc.eval_hess(p)
    cmax = float(np.abs(coef).max())
    assert torch.max(torch.abs(f1 - f2)) <= 2 * TOL * cmax
    assert torch.max(torch.abs(h1 - h2)) <= 2e-4 * cmax
    out = torch.full((len(pts),), float("nan"), device="cuda")
    plan = Plan([vs], [p], [out], tile=256)
    plan.launch()
    plan.status()
    assert torch.equal(out, vs.eval(p))
