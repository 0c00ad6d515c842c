"""Fused value + gradient + Hessian (ls_eval_hess) against the FP64 oracle.

The oracle's Hessian comes from the box-spline derivative identity applied
twice (pinned in test_oracle_pins against closed forms, central differences of
its gradient and exact quadratic reproduction).  Tolerance: the kernel forms
second derivatives of the per-region polynomial from FP32 monomial
coefficients; their rounding (2^-24 relative) is amplified by the sum of
|second-derivative weights| over the stencil (up to ~40 for the quintic's 32
sites), so the bound used is 1e-4 * ||c||_inf with margin, 2e-6 for values and
1e-5 for gradients as elsewhere.  Splines that are only C^0 or C^1 have a
Hessian that jumps across knot planes: there the comparison keeps the points
whose oracle Hessian is the same a little to either side.
"""
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
EXT = {"tricubic": (9, 8, 10), "trilinear": (9, 12, 10), "triquadratic": (11, 9, 12), "bcc_linear": (6, 7, 6),
       "bcc_quintic": (7, 6, 7), "bcc_quartic": (7, 6, 7), "fcc6": (6, 7, 6), "zp": (13, 11)}
C2 = {"tricubic", "bcc_quintic", "bcc_quartic"}


@pytest.mark.parametrize("name", sorted(EXT))
def test_hessian_matches_oracle(name):
    from paper_2102_08518_b300.api import Spline, Volume
    lat = workloads.SPLINE_LATTICE[name]
    ext = EXT[name]
    coef = workloads.coef_uniform(lat, ext, seed=201)
    lo, hi = workloads.bounding_box(lat, ext)
    n = 400 if name in ("bcc_quintic", "triquadratic") else 1500
    pts = workloads.points_uniform(n, lo - 1.0, hi + 1.0, seed=202)
    vol = Volume(Spline(name, "f32"), ext, torch.from_numpy(coef).cuda())
    val, grad, hess = vol.eval_hess(torch.from_numpy(pts).cuda())
    torch.cuda.synchronize()
    spec = ORACLE_SPEC[name]().with_extent(ext)
    c64 = coef.astype(np.float64).ravel()
    p64 = pts.astype(np.float64)
    f, g = oracle.eval_sum_grad(spec, c64, p64)
    H = oracle.eval_sum_hess(spec, c64, p64)
    cmax = np.abs(coef).max()
    assert np.max(np.abs(val.cpu().numpy() - f)) <= 2e-6 * cmax
    ok = np.ones(n, bool)
    if name not in C2:
        # within one polynomial piece of degree <= 3 the Hessian is affine, so it
        # equals the mean of its values a step to either side; across a knot
        # plane it jumps (gradients likewise, up to the quadratic term)
        d = np.array([0.37, 0.61, 0.70][: len(ext)]) * 1e-4
        hm = 0.5 * (oracle.eval_sum_hess(spec, c64, p64 + d) + oracle.eval_sum_hess(spec, c64, p64 - d))
        gm = 0.5 * (oracle.eval_sum_grad(spec, c64, p64 + d)[1] + oracle.eval_sum_grad(spec, c64, p64 - d)[1])
        ok = np.all(np.abs(hm - H) < 1e-6, axis=1) & np.all(np.abs(gm - g) < 1e-6, axis=1)
        assert ok.sum() > n // 2
    assert np.max(np.abs(grad.cpu().numpy()[ok] - g[ok])) <= 1e-5 * cmax
    assert np.max(np.abs(hess.cpu().numpy()[ok] - H[ok])) <= 1e-4 * cmax


def test_hessian_of_c2_splines_on_knot_planes_and_lattice_sites():
    """C^2 splines: the Hessian is continuous, so points exactly on mirror and
    knot planes and lattice sites must match too."""
    from paper_2102_08518_b300.api import Spline, Volume
    for name in ("tricubic", "bcc_quintic"):
        lat = workloads.SPLINE_LATTICE[name]
        ext = EXT[name]
        coef = workloads.coef_uniform(lat, ext, seed=203)
        lo, hi = workloads.bounding_box(lat, ext)
        rng = np.random.default_rng(204)
        p = rng.uniform(lo, hi, (240, 3))
        p[:60] = np.round(p[:60])
        p[60:120] = np.round(p[60:120] * 2) / 2
        p[120:180, 1] = p[120:180, 0]
        pts = p.astype(np.float32)
        vol = Volume(Spline(name, "f32"), ext, torch.from_numpy(coef).cuda())
        _, _, hess = vol.eval_hess(torch.from_numpy(pts).cuda(), want_value=False, want_grad=False)
        spec = ORACLE_SPEC[name]().with_extent(ext)
        H = oracle.eval_sum_hess(spec, coef.astype(np.float64).ravel(), pts.astype(np.float64))
        assert np.max(np.abs(hess.cpu().numpy() - H)) <= 1e-4 * np.abs(coef).max()


def test_hessian_at_full_size_sampled():
    """BCC quintic 2 x 128^3 (the benchmark's volume), 2^16 points: the oracle
    checks 256 sampled points."""
    from paper_2102_08518_b300.api import Spline, Volume
    ext = (128, 128, 128)
    coef = workloads.coef_smooth("bcc", ext, seed=0)
    lo, hi = workloads.inner_box("bcc_quintic", ext)
    pts = workloads.points_uniform(1 << 16, lo, hi, seed=205)
    vol = Volume(Spline("bcc_quintic", "f32"), ext, torch.from_numpy(coef).cuda())
    p = torch.from_numpy(pts).cuda()
    _, _, hess = vol.eval_hess(p, want_value=False, want_grad=False)
    idx = np.random.default_rng(206).choice(len(pts), 256, replace=False)
    spec = ORACLE_SPEC["bcc_quintic"]().with_extent(ext)
    H = oracle.eval_sum_hess(spec, coef.astype(np.float64).ravel(), pts[idx].astype(np.float64))
    assert np.max(np.abs(hess.cpu().numpy()[idx] - H)) <= 1e-4 * np.abs(coef).max()
