"""Least-squares fit (CGLS) and the autograd wrapper against FP64 references.

The fit is checked against the exact minimiser of ||A c - y||^2 + lam ||c||^2
computed in FP64 on the CPU from the oracle's matrix A[p, n] = phi(x_p - n)
(sparse normal equations, direct solve).  The autograd gradients are checked
against FP64 finite differences of the oracle's naive sum.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla
import torch

import oracle
import workloads
from oracle import specs as ospecs

pytestmark = pytest.mark.gpu

ORACLE_SPEC = {"tricubic": ospecs.tricubic, "bcc_quintic": ospecs.bcc_quintic, "bcc_quartic": ospecs.bcc_quartic,
               "voronoi2_bcc": ospecs.voronoi2_bcc, "voronoi2_fcc": ospecs.voronoi2_fcc, "bcc_linear": ospecs.bcc_linear,
               "fcc6": ospecs.fcc6}


_CASES = {}


def _case(name, ext, nsamp):
    """Samples, the oracle's A, lambda = 1e-6 tr(A^T A) / #unknowns, and the exact minimiser."""
    key = (name, ext, nsamp)
    if key not in _CASES:
        lat = workloads.SPLINE_LATTICE[name]
        lo, hi = workloads.bounding_box(lat, ext)
        pts, y = workloads.gaussian_samples(nsamp, lo, hi, noise=0.01, width=40.0, seed=7)
        spec = ORACLE_SPEC[name]().with_extent(ext)
        r, c, v = oracle.design_triplets(spec, pts.astype(np.float64))
        A = sp.csr_matrix((v, (r, c)), shape=(len(pts), spec.n_coef()))
        lam = 1e-6 * float(A.multiply(A).sum()) / A.shape[1]
        want = spla.spsolve((A.T @ A + lam * sp.identity(A.shape[1])).tocsc(), A.T @ y.astype(np.float64))
        _CASES[key] = (pts, y, A, lam, want)
    return _CASES[key]


@pytest.mark.parametrize("deterministic", [False, True, "fixed"])
@pytest.mark.parametrize("name,ext,nsamp", [("tricubic", (16, 16, 16), 1 << 15),
                                            ("bcc_quintic", (8, 8, 8), 1 << 13)])
def test_cg_fit_matches_exact_least_squares(name, ext, nsamp, deterministic):
    from paper_2102_08518_b300.api import Spline, Volume, cg_fit
    pts, y, A, lam, want = _case(name, ext, nsamp)
    vol = Volume(Spline(name, "f32"), ext, torch.zeros(A.shape[1], device="cuda"))
    it, hist = cg_fit(vol, torch.from_numpy(pts).cuda(), torch.from_numpy(y).cuda(), lam=lam, max_iter=400,
                      rel_tol=1e-6, deterministic=deterministic)
    got = vol.coef.cpu().numpy().astype(np.float64)
    assert 0 < it < 400
    assert hist[-1] <= 1e-6 * np.linalg.norm(A.T @ y) * 1.0001
    # The minimiser is only weakly determined along directions with eigenvalues
    # near lambda (sites with few samples), so the checks are on what the fit
    # determines: the objective and the fitted values A c.
    obj = lambda cc: np.sum((A @ cc - y) ** 2) + lam * np.sum(cc ** 2)
    assert obj(got) <= obj(want) * (1 + 1e-5)
    assert np.max(np.abs(A @ got - A @ want)) <= 1e-3 * np.max(np.abs(A @ want))


@pytest.mark.parametrize("mode", [True, "fixed"])
def test_cg_fit_deterministic_is_bitwise_reproducible(mode):
    from paper_2102_08518_b300.api import Spline, Volume, cg_fit
    name, ext = "bcc_quintic", (8, 8, 8)
    lo, hi = workloads.bounding_box("bcc", ext)
    pts, y = workloads.gaussian_samples(1 << 13, lo, hi, seed=9)
    out = []
    for _ in range(2):
        vol = Volume(Spline(name, "f32"), ext, torch.zeros(2 * 8 ** 3, device="cuda"))
        cg_fit(vol, torch.from_numpy(pts).cuda(), torch.from_numpy(y).cuda(), lam=1e-4, max_iter=30,
               rel_tol=0.0, deterministic=mode)
        out.append(vol.coef.clone())
    assert torch.equal(out[0], out[1])


@pytest.mark.parametrize("name", ["tricubic", "bcc_quintic", "fcc6"])
def test_autograd_matches_fp64_finite_differences(name):
    """L = sum_p g_p f(x_p): dL/dc against central differences in c (exact for a
    linear map), dL/dx against central differences in x of the oracle."""
    from paper_2102_08518_b300.api import Spline, spline_eval
    lat = workloads.SPLINE_LATTICE[name]
    ext = (16, 16, 16) if lat == "cc" else (8, 8, 8)
    coef_np = workloads.coef_uniform(lat, ext, seed=3)
    lo, hi = workloads.inner_box(name, ext)
    pts_np = workloads.points_uniform(512, lo, hi, seed=4)
    g_np = np.random.default_rng(5).normal(size=512)
    spl = Spline(name, "f32")
    coef = torch.from_numpy(coef_np).cuda().requires_grad_(True)
    pts = torch.from_numpy(pts_np).cuda().requires_grad_(True)
    f = spline_eval(spl, ext, coef, pts)
    (f.double() * torch.from_numpy(g_np).cuda()).sum().backward()
    gc = coef.grad.cpu().numpy().ravel().astype(np.float64)
    gx = pts.grad.cpu().numpy().astype(np.float64)
    spec = ORACLE_SPEC[name]().with_extent(ext)
    c64 = coef_np.astype(np.float64).ravel()
    L = lambda cc, xx: float(g_np @ oracle.eval_sum(spec, cc, xx))
    rng = np.random.default_rng(6)
    h = 1e-3
    for n in rng.choice(len(c64), 12, replace=False):
        e = np.zeros_like(c64)
        e[n] = h
        fd = (L(c64 + e, pts_np.astype(np.float64)) - L(c64 - e, pts_np.astype(np.float64))) / (2 * h)
        assert abs(fd - gc[n]) <= 2e-5 * max(1.0, np.abs(gc).max())
    hx = 1e-5
    x64 = pts_np.astype(np.float64)
    for i in range(3):
        e = np.zeros(3)
        e[i] = hx
        fd = g_np * (oracle.eval_sum(spec, c64, x64 + e) - oracle.eval_sum(spec, c64, x64 - e)) / (2 * hx)
        assert np.max(np.abs(fd - gx[:, i])) <= 1e-4 * max(1.0, np.abs(g_np).max())
