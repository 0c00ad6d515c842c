"""Batched persistent evaluation (one launch over many volumes) on the GPU."""
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
TORCH = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}


def _batch(n_vol, seed, dtypes=("f32", "bf16", "f16"), layout="coset"):
    from paper_2102_08518_b300.api import LAYOUT_BRICK, Spline, Volume, relayout
    recipe = workloads.batch_recipe(n_vol, seed=seed, edges=(8, 12, 16, 24), log2_lo=4, log2_hi=13)
    rng = np.random.default_rng(seed)
    splines, vols, pts, outs, coefs, exts = {}, [], [], [], [], []
    for k, it in enumerate(recipe):
        dt = dtypes[k % len(dtypes)]
        lat = workloads.SPLINE_LATTICE[it.spline]
        if (it.spline, dt) not in splines:
            splines[(it.spline, dt)] = Spline(it.spline, dt, brick=LAYOUT_BRICK[layout])
        c = workloads.coef_uniform(lat, it.ext, seed=it.seed)
        lo, hi = workloads.bounding_box(lat, it.ext)
        n = it.n_points if k != 3 else 0                       # one empty volume
        p = workloads.points_uniform(n, lo - 1.0, hi + 1.0, seed=it.seed + 1)
        ct = torch.from_numpy(c).to("cuda", TORCH[dt]).contiguous()
        cl = ct if layout == "coset" else relayout(ct, len(workloads.LATTICES[lat][2]), it.ext, to=layout)
        vols.append(Volume(splines[(it.spline, dt)], it.ext, cl, layout=layout))
        pts.append(torch.from_numpy(p).cuda())
        outs.append(torch.full((n,), float("nan"), device="cuda"))
        coefs.append(ct.float().cpu().numpy())
        exts.append(it.ext)
    return recipe, splines, vols, pts, outs, coefs, exts


@pytest.mark.parametrize("tile,layout", [(0, "coset"), (100, "coset"), (4096, "coset"), (0, "bricked"),
                                         (100, "bricked_shifted")])
def test_plan_matches_per_volume_kernels_and_oracle(tile, layout):
    """The plan against each volume's own kernel and the oracle, FP32 / BF16 /
    FP16 volumes mixed, in the linear, bricked and shifted-copy layouts (the
    recipe's extents are even)."""
    from paper_2102_08518_b300.api import Plan
    recipe, splines, vols, pts, outs, coefs, exts = _batch(14, seed=3, layout=layout)
    plan = Plan(vols, pts, outs, tile=tile)
    for o in outs:
        o.fill_(float("nan"))
    plan.launch()
    plan.status()
    torch.cuda.synchronize()
    info = plan.info()
    assert info["tile"] > 0 and info["grid"] > 0
    for k, it in enumerate(recipe):
        if pts[k].shape[0] == 0:
            continue
        ref = vols[k].eval(pts[k])
        torch.cuda.synchronize()
        got = outs[k].cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(got))
        cmax = np.abs(coefs[k]).max()
        assert np.max(np.abs(got - ref.cpu().numpy())) <= 1e-6 * cmax
        spec = ORACLE_SPEC[it.spline]().with_extent(exts[k])
        m = min(300, len(got))
        want = oracle.eval_sum(spec, coefs[k].astype(np.float64).ravel(), pts[k][:m].cpu().numpy().astype(np.float64))
        assert np.max(np.abs(got[:m] - want)) <= 2e-6 * cmax


def test_plan_in_cuda_graph_replays():
    from paper_2102_08518_b300.api import Plan
    recipe, splines, vols, pts, outs, coefs, exts = _batch(10, seed=5)
    plan = Plan(vols, pts, outs, tile=1024)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        plan.launch(stream=s)                 # warm-up outside the capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    ref = [o.clone() for o in outs]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.launch(stream=torch.cuda.current_stream())
    for o in outs:
        o.fill_(float("nan"))
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    plan.status()
    for a, b in zip(outs, ref):
        assert torch.equal(a, b)
