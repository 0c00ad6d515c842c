"""The tensor-core value kernel (variant tensor) against the FP64 oracle.

The coefficient transform A = M^T c of a tile of 128 points is one tcgen05
matrix product (three TF32 products for FP32 accuracy; two for BF16 / FP16 storage, whose
values are exact in TF32) instead of per-thread FMAs; everything else is the
FMA kernel's code.  FP32 data also has an FP16 form (tensor_kind 1): each
point's coefficients scaled by a power of two, split into FP16 hi + lo, three
kind::f16 products, the scales undone on the results.  Checked: every non-separable
spline, tile-ragged point counts, points beyond the arrays, non-finite and
far points, both linear layouts and BF16 storage, several tiles per block
(grid-stride loop over the mbarrier phases), and agreement with the FMA
kernel on 2^20 points.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads
from oracle import specs as ospecs

pytestmark = pytest.mark.gpu

TOL = 2e-6
BF16_TOL = 2.0 ** -8 + 2e-6
F16_TOL = 2.0 ** -11 + 2e-6
ORACLE_SPEC = {"bcc_linear": ospecs.bcc_linear, "bcc_quintic": ospecs.bcc_quintic, "bcc_quartic": ospecs.bcc_quartic,
               "voronoi2_bcc": ospecs.voronoi2_bcc, "voronoi2_fcc": ospecs.voronoi2_fcc, "fcc6": ospecs.fcc6,
               "zp": ospecs.zp2d}
EXT = {"bcc_linear": (10, 9, 8), "bcc_quintic": (10, 8, 9), "fcc6": (9, 10, 8), "zp": (14, 12)}
NAMES = list(EXT)


def n_cosets(name):
    return len(workloads.LATTICES[workloads.SPLINE_LATTICE[name]][2])


def volume(name, ext, coef_np, layout="coset", dtype="f32", **kw):
    from paper_2102_08518_b300.api import Spline, TORCH_DTYPES, Volume, relayout
    c = torch.from_numpy(coef_np.astype(np.float32)).cuda()
    if layout == "interleaved":
        c = relayout(c, n_cosets(name), ext, to="interleaved")
    return Volume(Spline(name, dtype, **kw), ext, c.to(TORCH_DTYPES[dtype]).contiguous(), layout=layout)


def oracle_eval(name, ext, coef_np, pts):
    spec = ORACLE_SPEC[name]().with_extent(ext)
    return oracle.eval_sum(spec, coef_np.astype(np.float64).ravel(), pts.astype(np.float64))


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("n", [1, 127, 128, 129, 3001])
def test_tensor_matches_oracle(name, n, kind):
    ext = EXT[name]
    lat = workloads.SPLINE_LATTICE[name]
    coef = workloads.coef_uniform(lat, ext, seed=21)
    lo, hi = workloads.bounding_box(lat, ext)
    pts = workloads.points_uniform(n, lo - 2.5, hi + 2.5, seed=n + 7)
    vol = volume(name, ext, coef, tensor=1, tensor_kind=kind)
    got = vol.eval(torch.from_numpy(pts).cuda()).cpu().numpy().astype(np.float64)
    vol.spline.status()
    want = oracle_eval(name, ext, coef, pts)
    assert np.max(np.abs(got - want)) <= TOL * np.abs(coef).max()


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("name", ["bcc_quintic", "fcc6"])
def test_tensor_special_points(name, kind):
    """NaN gives NaN, infinite and far points give 0, as in the FMA kernel."""
    ext = EXT[name]
    lat = workloads.SPLINE_LATTICE[name]
    coef = workloads.coef_uniform(lat, ext, seed=22)
    lo, hi = workloads.bounding_box(lat, ext)
    pts = workloads.points_uniform(300, lo, hi, seed=3)
    pts[5] = np.nan
    pts[6, 2] = np.inf
    pts[7] = 5.0e6
    pts[8] = lo - 30.0
    vol = volume(name, ext, coef, tensor=1, tensor_kind=kind)
    got = vol.eval(torch.from_numpy(pts).cuda()).cpu().numpy()
    assert np.isnan(got[5]) and got[6] == 0.0 and got[7] == 0.0 and got[8] == 0.0
    keep = np.ones(len(pts), bool)
    keep[5:9] = False
    want = oracle_eval(name, ext, coef, pts[keep])
    assert np.max(np.abs(got[keep] - want)) <= TOL * np.abs(coef).max()
    assert volume(name, ext, coef, tensor=1, tensor_kind=kind).eval(torch.empty(0, 3, device="cuda")).numel() == 0


@pytest.mark.parametrize("layout,dtype", [("interleaved", "f32"), ("coset", "bf16"), ("interleaved", "bf16"),
                                          ("interleaved", "f16")])
@pytest.mark.parametrize("name", ["bcc_quintic", "fcc6"])
def test_tensor_layouts_and_storage(name, layout, dtype):
    ext = EXT[name]
    lat = workloads.SPLINE_LATTICE[name]
    coef = workloads.coef_uniform(lat, ext, seed=23)
    lo, hi = workloads.bounding_box(lat, ext)
    pts = workloads.points_uniform(2000, lo - 2.0, hi + 2.0, seed=9)
    vol = volume(name, ext, coef, layout=layout, dtype=dtype, tensor=1)
    got = vol.eval(torch.from_numpy(pts).cuda()).cpu().numpy().astype(np.float64)
    want = oracle_eval(name, ext, coef, pts)
    tol = {"f32": TOL, "bf16": BF16_TOL, "f16": F16_TOL}[dtype]
    assert np.max(np.abs(got - want)) <= tol * np.abs(coef).max()


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("name", ["bcc_quintic", "fcc6", "bcc_linear"])
def test_tensor_agrees_with_fma_kernel_on_many_points(name, kind):
    """2^20 points, one block per SM (hundreds of tiles per block): both
    kernels approximate the same exact sum."""
    ext = (48, 40, 36)
    lat = workloads.SPLINE_LATTICE[name]
    coef = workloads.coef_uniform(lat, ext, seed=24)
    lo, hi = workloads.bounding_box(lat, ext)
    pts = torch.from_numpy(workloads.points_uniform(1 << 20, lo - 1.0, hi + 1.0, seed=5)).cuda()
    plain = volume(name, ext, coef).eval(pts)
    vt = volume(name, ext, coef, tensor=1, tensor_kind=kind, blocks_per_sm=1)
    got = vt.eval(pts)
    vt.spline.status()
    assert torch.max(torch.abs(got - plain)).item() <= 2 * TOL * float(np.abs(coef).max())
    idx = np.random.default_rng(1).choice(1 << 20, 1000, replace=False)
    want = oracle_eval(name, ext, coef, pts.cpu().numpy()[idx])
    assert np.max(np.abs(got.cpu().numpy()[idx] - want)) <= TOL * np.abs(coef).max()


GRAD_TOL = 1e-5


@pytest.mark.parametrize("kind,slots", [(0, 1), (1, 1), (1, 6)])
@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("n", [1, 129, 3001])
def test_tensor_value_gradient_matches_oracle(name, n, kind, slots):
    """The value + gradient kernel of a tensor-core spline: the same product,
    then the gradient's Horner forms mapped back through the fold (at 6
    slots with the products read back in pieces as the forms need them)."""
    ext = EXT[name]
    lat = workloads.SPLINE_LATTICE[name]
    coef = workloads.coef_uniform(lat, ext, seed=31)
    lo, hi = workloads.bounding_box(lat, ext)
    pts = workloads.points_uniform(n, lo - 2.0, hi + 2.0, seed=n + 17)
    vol = volume(name, ext, coef, layout="interleaved", tensor=slots, tensor_kind=kind)
    val, grad = vol.eval_grad(torch.from_numpy(pts).cuda())
    vol.spline.status()
    spec = ORACLE_SPEC[name]().with_extent(ext)
    want, wgrad = oracle.eval_sum_grad(spec, coef.astype(np.float64).ravel(), pts.astype(np.float64))
    cmax = np.abs(coef).max()
    assert np.max(np.abs(val.cpu().numpy() - want)) <= TOL * cmax
    g = grad.cpu().numpy().astype(np.float64)
    ok = np.ones(len(pts), bool)
    if name == "bcc_linear":
        # C0 spline: the gradient jumps across knot planes; compare off them
        # (one-sided difference quotients of the oracle agree there)
        h = 1e-4
        D = pts.shape[1]
        for q in range(D):
            e = np.zeros(D)
            e[q] = h
            fp = oracle.eval_sum(spec, coef.astype(np.float64).ravel(), pts + e)
            fm = oracle.eval_sum(spec, coef.astype(np.float64).ravel(), pts - e)
            ok &= np.abs((fp - want) / h - (want - fm) / h) < 1e-6
    assert np.max(np.abs(g[ok] - wgrad[ok]), initial=0.0) <= GRAD_TOL * cmax


@pytest.mark.parametrize("name", ["bcc_quintic", "fcc6"])
def test_tensor_value_gradient_agrees_with_fma_kernel(name):
    ext = (48, 40, 36)
    lat = workloads.SPLINE_LATTICE[name]
    coef = workloads.coef_uniform(lat, ext, seed=32)
    lo, hi = workloads.bounding_box(lat, ext)
    pts = torch.from_numpy(workloads.points_uniform(1 << 20, lo - 1.0, hi + 1.0, seed=6)).cuda()
    v0, g0 = volume(name, ext, coef, layout="interleaved").eval_grad(pts)
    vt = volume(name, ext, coef, layout="interleaved", tensor=1)
    v1, g1 = vt.eval_grad(pts)
    _, g2 = vt.eval_grad(pts, want_value=False)
    vt.spline.status()
    cmax = float(np.abs(coef).max())
    assert torch.max(torch.abs(v1 - v0)).item() <= 2 * TOL * cmax
    assert torch.max(torch.abs(g1 - g0)).item() <= 2 * GRAD_TOL * cmax
    assert torch.equal(g1, g2)


@pytest.mark.parametrize("name", ["bcc_quintic", "fcc6", "zp"])
def test_tensor_fp16_form_is_scale_invariant(name):
    """The FP16 form scales each point's coefficients by a power of two and
    undoes it on the results: data scaled by 2^k (within the normal FP32
    range) gives the results scaled by 2^k, bit for bit, values and gradients."""
    ext = EXT[name]
    lat = workloads.SPLINE_LATTICE[name]
    coef = workloads.coef_uniform(lat, ext, seed=41).astype(np.float32)
    coef[np.abs(coef) < 2.0 ** -20] = 2.0 ** -20      # scaled copies stay normal
    lo, hi = workloads.bounding_box(lat, ext)
    pts = torch.from_numpy(workloads.points_uniform(5000, lo - 1.0, hi + 1.0, seed=42)).cuda()
    base = volume(name, ext, coef, layout="interleaved", tensor=1, tensor_kind=1)
    v0, g0 = base.eval_grad(pts)
    for k in (-90, -37, 1, 45, 90):
        vk = volume(name, ext, np.ldexp(coef, k), layout="interleaved", tensor=1, tensor_kind=1)
        f = 2.0 ** k
        assert torch.equal(vk.eval(pts), v0 * f), k
        v, g = vk.eval_grad(pts)
        assert torch.equal(v, v0 * f) and torch.equal(g, g0 * f), k


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("name", ["bcc_quintic", "fcc6"])
def test_tensor_with_coefficients_of_very_different_magnitudes(name, kind):
    """Blocks of the volume scaled by 2^-40, 1 and 2^40: every point's result
    must keep FP32 accuracy relative to its own stencil's coefficients, not to
    the volume's largest one (the FP16 form scales each point's row on its
    own; the TF32 form has FP32's exponent range)."""
    from paper_2102_08518_b300.api import table
    from paper_2102_08518_b300.roofline import stencil_indices
    ext = (16, 12, 12)
    lat = workloads.SPLINE_LATTICE[name]
    coef = workloads.coef_uniform(lat, ext, seed=51).astype(np.float64)
    C = coef.shape[0]
    e2, e1, e0 = np.meshgrid(np.arange(ext[2]), np.arange(ext[1]), np.arange(ext[0]), indexing="ij")
    block = (e0 // 4 + e1 // 4 + e2 // 4) % 3                 # 0, 1, 2 in a 4 x 4 x 4 checkerboard
    coef = coef * np.ldexp(1.0, 40 * (block - 1))[None, :, :, :].repeat(C, axis=0)
    coef = coef.astype(np.float32)
    lo, hi = workloads.bounding_box(lat, ext)
    pts = workloads.points_uniform(4000, lo + 0.5, hi - 0.5, seed=52)
    vol = volume(name, ext, coef, layout="interleaved", tensor=1, tensor_kind=kind)
    val, grad = vol.eval_grad(torch.from_numpy(pts).cuda())
    vol.spline.status()
    spec = ORACLE_SPEC[name]().with_extent(ext)
    want, wgrad = oracle.eval_sum_grad(spec, coef.astype(np.float64).ravel(), pts.astype(np.float64))
    idx = stencil_indices(table(name), ext, pts, "coset")
    flat = np.abs(coef.astype(np.float64).ravel())
    local = np.where(idx >= 0, flat[np.maximum(idx, 0)], 0.0).max(axis=1)
    assert np.all(local > 0)
    err = np.abs(val.cpu().numpy().astype(np.float64) - want) / local
    gerr = np.abs(grad.cpu().numpy().astype(np.float64) - wgrad).max(axis=1) / local
    assert err.max() <= TOL and gerr.max() <= GRAD_TOL
    # the volume's range: points in the small blocks sit 2^80 below the largest coefficient
    assert local.min() < 2.0 ** -30 * np.abs(coef).max()


@pytest.mark.parametrize("kind", [0, 1])
def test_tensor_non_finite_coefficient_reaches_only_its_stencils(kind):
    """FCC: the gathers cover the union of the two reference regions' stencils.
    An infinite coefficient must make exactly the points whose own stencil holds
    it non-finite; the rest stay finite and equal to the FMA kernel's."""
    from paper_2102_08518_b300.api import table
    from paper_2102_08518_b300.roofline import stencil_indices
    name, ext = "fcc6", (10, 10, 10)
    lat = workloads.SPLINE_LATTICE[name]
    coef = workloads.coef_uniform(lat, ext, seed=61)
    flat = coef.reshape(-1)
    site = 2 * int(np.prod(ext)) + 5 + ext[0] * (4 + ext[1] * 5)    # coset 2, grid index (5, 4, 5)
    flat[site] = np.inf
    lo, hi = workloads.bounding_box(lat, ext)
    c = (lo + hi) / 2
    pts = workloads.points_uniform(20000, c - 3.0, c + 3.0, seed=62)
    p = torch.from_numpy(pts).cuda()
    ref = volume(name, ext, coef, layout="interleaved").eval(p).cpu().numpy()
    vt = volume(name, ext, coef, layout="interleaved", tensor=1, tensor_kind=kind)
    got = vt.eval(p).cpu().numpy()
    vt.spline.status()
    holds = (stencil_indices(table(name), ext, pts, "coset") == site).any(axis=1)
    assert 100 < holds.sum() < len(pts) - 100
    assert np.array_equal(~np.isfinite(got), holds)
    assert np.array_equal(~np.isfinite(ref), holds)
    ok = ~holds
    assert np.max(np.abs(got[ok] - ref[ok])) <= 2 * TOL


@pytest.mark.parametrize("slots,kind", [(2, 0), (3, 1), (6, 1), (8, 0)])
def test_tensor_explicit_slot_counts(slots, kind):
    """tensor = S sets the slots per SM (at most what the 512 tensor-memory
    columns hold): every count gives the default's results within the
    tolerance (BCC quintic: 112 columns a slot in the TF32 form, so 8 asks
    for more than fit and gets 4; 80 in the FP16 form)."""
    name = "bcc_quintic"
    ext = (24, 20, 18)
    lat = workloads.SPLINE_LATTICE[name]
    coef = workloads.coef_uniform(lat, ext, seed=71)
    lo, hi = workloads.bounding_box(lat, ext)
    pts = workloads.points_uniform(100_003, lo - 1.0, hi + 1.0, seed=72)
    vt = volume(name, ext, coef, layout="interleaved", tensor=slots, tensor_kind=kind)
    import re
    m = re.search(r"__launch_bounds__\((\d+), 1\) ls_eval__", vt.spline.source())
    assert int(m.group(1)) == 128 * min(slots, 512 // (80 if kind else 112))
    got = vt.eval(torch.from_numpy(pts).cuda()).cpu().numpy().astype(np.float64)
    vt.spline.status()
    idx = np.random.default_rng(3).choice(len(pts), 1500, replace=False)
    want = oracle_eval(name, ext, coef, pts[idx])
    assert np.max(np.abs(got[idx] - want)) <= TOL * np.abs(coef).max()


@pytest.mark.parametrize("name", ["bcc_quintic", "fcc6"])
def test_tensor_slot_count_and_tile_order_do_not_change_results(name):
    """5 slots (all products read back at once) and 6 slots (a large
    spline's products read back in 8-column pieces as the polynomial needs
    them) do the same arithmetic per point: bitwise equal results."""
    ext = (40, 36, 30)
    lat = workloads.SPLINE_LATTICE[name]
    coef = workloads.coef_uniform(lat, ext, seed=81)
    lo, hi = workloads.bounding_box(lat, ext)
    pts = torch.from_numpy(workloads.points_uniform(300_001, lo - 1.0, hi + 1.0, seed=82)).cuda()
    outs = []
    for slots in (1, 6, 2):
        v = volume(name, ext, coef, layout="interleaved", tensor=slots, tensor_kind=1)
        outs.append(v.eval(pts))
        v.spline.status()
    assert torch.equal(outs[0].view(torch.int32), outs[1].view(torch.int32))
    assert torch.equal(outs[0].view(torch.int32), outs[2].view(torch.int32))
