"""The generator's point functions, compiled for the host, against the FP64 oracle.

The generated value, value + gradient and value + gradient + Hessian point
functions are plain arithmetic around a few device intrinsics
(tests/host_kernels.py gives host stand-ins), so their arithmetic and
addressing can be checked on the CPU: every spline, the three coefficient
layouts, the factored and the direct coefficient transform, and the kernel
variants that change the point function (the paper's group size m and depth d
of Algorithm 2, branchy selection of the reference sub-region).  Points reach
2.5 sites beyond the stored arrays (zero extension).  The GPU parity tests
check the compiled kernels.
"""
import numpy as np
import pytest

import oracle
import workloads
from oracle import specs as ospecs

from tests.host_kernels import HostKernels, generated_source
from tests.test_gpu_layout import brick_np, brick_shifted_np, interleave_np

SPEC = {"tricubic": ospecs.tricubic, "trilinear": ospecs.trilinear, "triquadratic": ospecs.triquadratic,
        "bcc_linear": ospecs.bcc_linear, "bcc_quintic": ospecs.bcc_quintic, "bcc_quartic": ospecs.bcc_quartic,
               "voronoi2_bcc": ospecs.voronoi2_bcc, "voronoi2_fcc": ospecs.voronoi2_fcc, "fcc6": ospecs.fcc6, "zp": ospecs.zp2d}
EXT = {"tricubic": (8, 6, 6), "trilinear": (6, 6, 4), "triquadratic": (6, 8, 6), "bcc_linear": (6, 6, 4),
       "bcc_quintic": (8, 6, 6), "bcc_quartic": (6, 8, 6), "fcc6": (6, 6, 6), "zp": (12, 10),
       "voronoi2_bcc": (6, 6, 6), "voronoi2_fcc": (6, 6, 6)}
TOL, GTOL, HTOL = 2e-6, 1e-5, 1e-4


def _case(name, n=1500, seed=2):
    lat = workloads.SPLINE_LATTICE[name]
    ext = EXT[name]
    C = len(workloads.LATTICES[lat][2])
    coef = workloads.coef_uniform(lat, ext, seed=1)
    lo, hi = workloads.bounding_box(lat, ext)
    pts = workloads.points_uniform(n, lo - 2.5, hi + 2.5, seed=seed)
    return lat, ext, C, coef, pts


def _layout(coef, C, ext, layout):
    flat = coef.ravel()
    if layout.startswith("bricked_shifted"):
        return brick_shifted_np(flat, C, ext, xyz=layout.endswith("xyz"))
    return {"coset": flat, "interleaved": interleave_np(flat, C), "bricked": brick_np(flat, C, ext)}[layout]


BRICK = {"coset": 0, "interleaved": 0, "bricked": 1, "bricked_shifted": 2, "bricked_shifted_xyz": 3}


@pytest.mark.parametrize("name", list(SPEC))
@pytest.mark.parametrize("layout", ["coset", "interleaved", "bricked", "bricked_shifted", "bricked_shifted_xyz"])
def test_value_and_gradient(name, layout):
    if layout.startswith("bricked_shifted") and name == "zp":
        pytest.skip("the shifted bricked copies are 3D only")
    voronoi = name.startswith("voronoi")
    lat, ext, C, coef, pts = _case(name, n=200 if voronoi else 1500)
    spec = SPEC[name]().with_extent(ext)
    want, wgrad = oracle.eval_sum_grad(spec, coef.astype(np.float64).ravel(), pts.astype(np.float64))
    hk = HostKernels(name, **({"brick": BRICK[layout]} if BRICK[layout] else {}))
    c = _layout(coef, C, ext, layout)
    f = hk.eval(pts, c, ext, layout, C)
    v, g = hk.eval_grad(pts, c, ext, layout, C)
    cmax = float(np.abs(coef).max())
    assert np.abs(f - want).max() <= TOL * cmax
    assert np.abs(v - want).max() <= TOL * cmax
    if voronoi:
        # the oracle's gradient is a central difference (h = 1e-5): compare where
        # no knot plane lies within the difference step (one-sided slopes agree)
        ok = np.ones(len(pts), bool)
        c64 = coef.astype(np.float64).ravel()
        for i in range(3):
            e = np.zeros(3)
            e[i] = 1e-4
            fp = oracle.eval_sum(spec, c64, pts + e)
            fm = oracle.eval_sum(spec, c64, pts - e)
            ok &= np.abs((fp - want) - (want - fm)) / 1e-4 < 1e-2     # h |f''| inside a cubic piece
        assert ok.sum() > len(pts) // 2
        g, wgrad = g[ok], wgrad[ok]
    assert np.abs(g - wgrad).max() <= GTOL * cmax


@pytest.mark.parametrize("name", ["bcc_quintic", "fcc6", "tricubic", "zp"])
def test_hessian(name):
    lat, ext, C, coef, pts = _case(name, n=200)
    spec = SPEC[name]().with_extent(ext)
    c64 = coef.astype(np.float64).ravel()
    want = oracle.eval_sum_hess(spec, c64, pts.astype(np.float64))
    hk = HostKernels(name)
    f, g, h = hk.eval_hess(pts, coef.ravel(), ext, "coset", C)
    cmax = float(np.abs(coef).max())
    assert np.abs(f - oracle.eval_sum(spec, c64, pts.astype(np.float64))).max() <= TOL * cmax
    if name in ("bcc_quintic", "tricubic"):      # C^2: the Hessian is continuous everywhere
        assert np.abs(h - want).max() <= HTOL * cmax


@pytest.mark.parametrize("name", ["bcc_quintic", "fcc6", "bcc_linear", "zp"])
def test_plain_transform_matches(name):
    """The direct sums over the sites (plain_transform = 1) and the factored
    transform give the oracle's values; the factored one in fewer operations."""
    lat, ext, C, coef, pts = _case(name, n=800)
    spec = SPEC[name]().with_extent(ext)
    want = oracle.eval_sum(spec, coef.astype(np.float64).ravel(), pts.astype(np.float64))
    cmax = float(np.abs(coef).max())
    for var in ({}, {"plain_transform": 1}):
        f = HostKernels(name, **var).eval(pts, coef.ravel(), ext, "coset", C)
        assert np.abs(f - want).max() <= TOL * cmax


def _pt_ops(src, fname):
    i = src.index("void " + fname + "(")
    body = src[i:src.index("\n}\n", i)]
    return body.count("fmaf(") + body.count(" * c") + body.count(" + c") + body.count(" - c")


def test_factored_transform_is_cheaper():
    """BCC quintic: the generator's factored transform needs well under half
    the multiply-adds of the direct sums (1016 nonzeros in the table)."""
    from paper_2102_08518_b300 import api
    fac = generated_source("bcc_quintic")
    pla = generated_source("bcc_quintic", plain_transform=1)
    tag_f = api.kernel_name("bcc_quintic", "f32")
    tag_p = api.kernel_name("bcc_quintic", "f32", plain_transform=1)
    n_f = _pt_ops(fac, "ls_eval_pt__" + tag_f)
    n_p = _pt_ops(pla, "ls_eval_pt__" + tag_p)
    assert n_p >= 1000 and n_f < 0.5 * n_p


@pytest.mark.parametrize("name,var", [("bcc_quintic", {"group": 4, "depth": 2}), ("bcc_quintic", {"group": 8, "depth": 1}),
                                      ("fcc6", {"group": 2, "depth": 4}), ("fcc6", {"branchy": 1}),
                                      ("fcc6", {"branchy": 1, "brick": 1}), ("tricubic", {"group": 8, "depth": 2}),
                                      ("bcc_linear", {"group": 1, "depth": 2}), ("bcc_quintic", {"prefetch": 1}),
                                      ("tricubic", {"prefetch": 1}), ("zp", {"prefetch": 1}),
                                      ("bcc_quintic", {"l2_keep": 1}), ("fcc6", {"l2_keep": 1, "prefetch": 1}),
                                      ("bcc_quintic", {"fma2": 1}), ("fcc6", {"fma2": 1}), ("bcc_quartic", {"fma2": 1}),
                                      ("voronoi2_bcc", {"fma2": 1}), ("bcc_linear", {"fma2": 1}),
                                      ("fcc6", {"fma2": 1, "branchy": 1})])
def test_paper_parameter_variants(name, var):
    """The paper's group size / pipeline depth (Algorithm 2) and branchy
    sub-region selection change the generated point function; each variant
    still gives the oracle's values and gradients."""
    lat, ext, C, coef, pts = _case(name, n=800)
    spec = SPEC[name]().with_extent(ext)
    want, wgrad = oracle.eval_sum_grad(spec, coef.astype(np.float64).ravel(), pts.astype(np.float64))
    layout = "bricked" if var.get("brick") else "coset"
    hk = HostKernels(name, **var)
    c = _layout(coef, C, ext, layout)
    f = hk.eval(pts, c, ext, layout, C)
    v, g = hk.eval_grad(pts, c, ext, layout, C)
    cmax = float(np.abs(coef).max())
    assert np.abs(f - want).max() <= TOL * cmax
    assert np.abs(g - wgrad).max() <= GTOL * cmax


@pytest.mark.parametrize("l2_keep", [0, 1])
@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_reduced_precision_loaders(dtype, l2_keep):
    """BF16 / FP16 storage: the loaders (with and without the L2 evict-last
    policy) widen exactly, so the result equals the oracle fed the rounded
    coefficients."""
    import torch
    name = "bcc_quintic"
    lat, ext, C, coef, pts = _case(name, n=600)
    t = torch.from_numpy(coef.ravel().astype(np.float32)).to(torch.bfloat16 if dtype == "bf16" else torch.float16)
    rounded = t.float().numpy().astype(np.float64)
    raw = t.view(torch.int16).numpy().view(np.uint16)
    spec = SPEC[name]().with_extent(ext)
    want = oracle.eval_sum(spec, rounded, pts.astype(np.float64))
    f = HostKernels(name, dtype, **({"l2_keep": 1} if l2_keep else {})).eval(pts, raw, ext, "coset", C)
    assert np.abs(f - want).max() <= TOL * float(np.abs(rounded).max())


@pytest.mark.parametrize("name", ["bcc_quintic", "fcc6", "voronoi2_bcc"])
def test_paired_fma_transform_gives_the_same_values(name):
    """The paired-FMA transform (fma2 = 1) forms the same sums in the same
    order (a variable only one monomial of a pair reads adds an exact 0), so
    values and gradients equal the scalar transform's."""
    lat, ext, C, coef, pts = _case(name, n=600)
    a, b = HostKernels(name), HostKernels(name, fma2=1)
    fa, ga = a.eval_grad(pts, coef.ravel(), ext, "coset", C)
    fb, gb = b.eval_grad(pts, coef.ravel(), ext, "coset", C)
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)



@pytest.mark.parametrize("name", ["bcc_linear", "bcc_quintic", "fcc6", "voronoi2_bcc", "voronoi2_fcc"])
def test_region_of_evaluation_ties(name):
    """The closed-form nearest site (BCC: the nearer of the even and odd
    candidates; FCC: rounding with the parity fix of D3) on points where
    several sites are nearest: half-integers, the BCC boundary sum |x - c| =
    3/2, integer points with an odd coordinate sum (FCC), lattice sites; the
    value is the oracle's whichever of the tied sites is taken."""
    lat, ext, C, coef, _ = _case(name, n=10)
    lo, hi = workloads.bounding_box(lat, ext)
    rng = np.random.default_rng(7)
    c = rng.integers(2, 2 * min(ext) - 3, (400, 3)).astype(np.float64)
    p = c.copy()
    p[:80] += 0.5                                             # half-integers
    d = rng.uniform(0.0, 1.0, (80, 2))
    p[80:160] = 2 * np.round(c[80:160] / 2) + np.stack([d[:, 0], d[:, 1], 1.5 - d[:, 0] - d[:, 1]], 1)
    p[160:240] = np.round(c[160:240])                         # integer points (odd sums among them)
    p[240:320] = 2 * np.round(c[240:320] / 2)                 # even lattice sites
    p[320:] += rng.choice([-0.5, 0.5], (80, 3))
    pts = np.clip(p, lo, hi).astype(np.float32)
    spec = SPEC[name]().with_extent(ext)
    want = oracle.eval_sum(spec, coef.astype(np.float64).ravel(), pts.astype(np.float64))
    f = HostKernels(name).eval(pts, coef.ravel(), ext, "coset", C)
    assert np.abs(f - want).max() <= TOL * float(np.abs(coef).max())
