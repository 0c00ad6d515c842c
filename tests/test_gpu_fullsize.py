"""Parity at the benchmark's full sizes, in the launch configurations bench.py
times (autotuned kernel variants, the batched plan), on sampled outputs."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from oracle import specs as ospecs

pytestmark = pytest.mark.gpu

ORACLE_SPEC = {"tricubic": ospecs.tricubic, "bcc_linear": ospecs.bcc_linear,
               "bcc_quintic": ospecs.bcc_quintic, "bcc_quartic": ospecs.bcc_quartic,
               "voronoi2_bcc": ospecs.voronoi2_bcc, "voronoi2_fcc": ospecs.voronoi2_fcc, "fcc6": ospecs.fcc6}
TOL = 2e-6


@pytest.mark.parametrize("layout", ["interleaved", "bricked", "coset"])
def test_bench_step_with_autotuned_kernels(layout):
    """The four launches of one bench step (BCC 2x128^3 smooth field, 2^24
    uniform + 2^24 ray points), each with the variant the bench runs in that
    layout: interleaved cosets (the bench's choice for the ray points, where
    the quintic runs the tensor-core kernel), 2x2x2 bricks (its choice for the
    uniform points) and coset-major."""
    from paper_2102_08518_b300.api import TUNE_CANDIDATES_SMALL, Volume, autotune, relayout
    ext = (128, 128, 128)
    coef_np = workloads.coef_smooth("bcc", ext, seed=0)
    lo, hi = workloads.inner_box("bcc_quintic", ext)
    sets = {"uniform": workloads.points_uniform(1 << 24, lo, hi, seed=1),
            "rays": workloads.points_rays(4096, 4096, lo, hi, seed=3)}
    coef = relayout(torch.from_numpy(coef_np).cuda(), 2, ext, to=layout)
    c64 = coef_np.astype(np.float64).ravel()
    for name in ("bcc_linear", "bcc_quintic"):
        spec = ORACLE_SPEC[name]().with_extent(ext)
        for ps, pts in sets.items():
            p = torch.from_numpy(pts).cuda()
            sp = autotune(name, "f32", ext, coef, [p], candidates=TUNE_CANDIDATES_SMALL, tag=f"bcc_step_{ps}",
                          layout=layout)
            out = Volume(sp, ext, coef, layout=layout).eval(p)
            sp.status()
            torch.cuda.synchronize()
            got = out.cpu().numpy().astype(np.float64)
            assert np.all(np.isfinite(got))
            seed = {"uniform": 11, "rays": 13}[ps] + (0 if name == "bcc_linear" else 100)
            idx = np.random.default_rng(seed).choice(len(pts), 768, replace=False)
            want = oracle.eval_sum(spec, c64, pts[idx].astype(np.float64))
            assert np.max(np.abs(got[idx] - want)) <= TOL * np.abs(coef_np).max(), (name, ps, sp.variant)


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_batched_64_volumes_full_size(dtype):
    """The batched configuration (64 volumes, edges {32..256}, mixed splines,
    ~4.8e7 points) as one persistent plan launch; 24 sampled points per volume
    against the oracle on the stored (rounded) coefficients."""
    from paper_2102_08518_b300.api import Plan, Spline, Volume
    tdt = {"bf16": torch.bfloat16, "f16": torch.float16}[dtype]
    recipe = workloads.batch_recipe(64, seed=0)
    sps, vols, pts, outs, coefs = {}, [], [], [], []
    for it in recipe:
        lat = workloads.SPLINE_LATTICE[it.spline]
        if it.spline not in sps:
            sps[it.spline] = Spline(it.spline, dtype)
        c = workloads.coef_uniform_torch(lat, it.ext, seed=it.seed, dtype=tdt)
        lo, hi = workloads.inner_box(it.spline, it.ext)
        vols.append(Volume(sps[it.spline], it.ext, c))
        pts.append(workloads.points_uniform_torch(it.n_points, lo, hi, seed=it.seed + 1))
        outs.append(torch.empty(it.n_points, device="cuda"))
        coefs.append(c)
    plan = Plan(vols, pts, outs, tile=0)
    for o in outs:
        o.fill_(float("nan"))
    plan.launch()
    plan.status()
    torch.cuda.synchronize()
    rng = np.random.default_rng(5)
    for it, c, p, o in zip(recipe, coefs, pts, outs):
        got = o.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(got))
        idx = rng.choice(len(got), min(24, len(got)), replace=False)
        spec = ORACLE_SPEC[it.spline]().with_extent(it.ext)
        c64 = c.float().cpu().numpy().astype(np.float64).ravel()
        want = oracle.eval_sum(spec, c64, p[idx].cpu().numpy().astype(np.float64))
        assert np.max(np.abs(got[idx] - want)) <= TOL * np.abs(c64).max(), it


def test_fcc_sorted_equals_unsorted_full_size():
    """FCC 4x128^3 with 2^26 points: Morton-sorted evaluation scattered back is
    bitwise the unsorted evaluation; sampled oracle check."""
    from paper_2102_08518_b300.api import Spline, Volume, morton_sort, permute_rows
    ext = (128, 128, 128)
    coef = workloads.coef_uniform_torch("fcc", ext, seed=0)
    lo, hi = workloads.inner_box("fcc6", ext)
    p = workloads.points_uniform_torch(1 << 26, lo, hi, seed=5)
    vol = Volume(Spline("fcc6", "f32"), ext, coef)
    f = vol.eval(p)
    perm = morton_sort(p, cell=1.0)
    fs = vol.eval(permute_rows(p, perm))
    back = permute_rows(fs.view(-1, 1), perm, inverse=True).view(-1)
    torch.cuda.synchronize()
    assert torch.equal(back, f)
    idx = np.random.default_rng(6).choice(1 << 26, 512, replace=False)
    spec = ORACLE_SPEC["fcc6"]().with_extent(ext)
    want = oracle.eval_sum(spec, coef.cpu().numpy().astype(np.float64).ravel(),
                           p[idx].cpu().numpy().astype(np.float64))
    assert np.max(np.abs(f[idx].cpu().numpy() - want)) <= TOL * float(coef.abs().max())
