"""Every kernel variant the autotuner can hand out, against the FP64 oracle.

The paper's parameter study (Sec. 4.4 and 5: gather group size m, pipeline
depth d, branchy vs predicated selection of the reference sub-region) and the
B300 axes (block size, occupancy, expansion centre, the direct-sum transform)
each change the generated evaluation kernel.  Every entry of the autotuner's
candidate lists and the branchy form of the K = 2 spline are compared with
the oracle on the small-volume every-point set (points 2.5 sites beyond the
arrays: the checked gathers) and on special points (lattice sites, half
integers, mirror and BSP planes, the box corners), at the same tolerance as
the default kernel.
"""
import numpy as np
import pytest
import torch

import workloads
from paper_2102_08518_b300.api import DEFAULT_CANDIDATES, TUNE_CANDIDATES_SMALL, Spline, Volume

from tests.test_gpu_eval import SMALL_EXT, TOL, oracle_eval

pytestmark = pytest.mark.gpu

FMA_CANDIDATES = [c for c in dict.fromkeys(tuple(sorted(c.items())) for c in DEFAULT_CANDIDATES + TUNE_CANDIDATES_SMALL)
                  if not dict(c).get("tensor")]


def _special_points(lo, hi, seed):
    rng = np.random.default_rng(seed)
    p = rng.uniform(lo, hi, (500, 3))
    p[:100] = np.round(p[:100])
    p[100:200] = np.round(p[100:200] * 2) / 2
    p[200:300, 1] = p[200:300, 0]
    d = rng.uniform(-0.5, 0.5, 100)
    p[300:400] = np.round(p[300:400]) + np.stack([d, d, 1 - 2 * np.abs(d)], 1) * 0.5
    p[400:450] = np.array(lo)
    p[450:500] = np.array(hi)
    return p.astype(np.float32)


def _check(name, var, layout="coset"):
    lat = workloads.SPLINE_LATTICE[name]
    ext = SMALL_EXT[name]
    if layout == "bricked":
        ext = tuple(e + (e & 1) for e in ext)
    coef = workloads.coef_uniform(lat, ext, seed=21)
    lo, hi = workloads.bounding_box(lat, ext)
    sets = [workloads.points_uniform(3001, lo - 2.5, hi + 2.5, seed=22), _special_points(lo, hi, 23)]
    v = dict(var)
    exp = v.pop("expansion", "sparse")
    sp = Spline(name, "f32", expansion=exp, **v, **({"brick": 1} if layout == "bricked" else {}))
    c = torch.from_numpy(coef).cuda()
    if layout != "coset":
        from paper_2102_08518_b300.api import relayout
        c = relayout(c, len(workloads.LATTICES[lat][2]), ext, to=layout)
    vol = Volume(sp, ext, c, layout=layout)
    cmax = float(np.abs(coef).max())
    for pts in sets:
        got = vol.eval(torch.from_numpy(pts).cuda()).cpu().numpy().astype(np.float64)
        want = oracle_eval(name, ext, coef, pts)
        assert np.max(np.abs(got - want)) <= TOL * cmax, (name, var, layout)
    sp.status()


@pytest.mark.parametrize("cand", FMA_CANDIDATES, ids=lambda c: "-".join(f"{k}{v}" for k, v in c))
@pytest.mark.parametrize("name", ["bcc_quintic", "fcc6", "bcc_linear"])
def test_autotune_candidates(name, cand):
    _check(name, dict(cand))


@pytest.mark.parametrize("cand", [dict(block=256), dict(block=512), dict(block=256, group=8, depth=2),
                                  dict(block=256, group=4, depth=4)], ids=str)
def test_autotune_candidates_bricked(cand):
    _check("bcc_quintic", cand, layout="bricked")


@pytest.mark.parametrize("var", [dict(branchy=1), dict(branchy=1, block=512), dict(branchy=1, group=4, depth=4),
                                 dict(branchy=1, expansion="centroid")], ids=str)
@pytest.mark.parametrize("layout", ["coset", "interleaved"])
def test_branchy_fcc(var, layout):
    """FCC's two reference sub-regions chosen by a branch instead of a select."""
    _check("fcc6", var, layout)


@pytest.mark.parametrize("var", [dict(branchy=1), dict()], ids=str)
@pytest.mark.parametrize("name", ["voronoi2_bcc", "voronoi2_fcc"])
def test_voronoi_branchy_and_predicated(name, var):
    """The second-order Voronoi splines (five reference sub-regions on BCC)
    with the sub-region chosen by a branch and by selects."""
    _check(name, var)


@pytest.mark.parametrize("var", [dict(group=16, depth=1), dict(group=8, depth=2), dict(group=8, depth=3),
                                 dict(group=4, depth=4)], ids=str)
@pytest.mark.parametrize("name", ["tricubic", "voronoi2_bcc"])
def test_parameter_sweep_variants(name, var):
    """The gather group size m and depth d of the benchmark's parameter sweep
    on the tensor-product spline and on the five-region Voronoi spline."""
    _check(name, var)


@pytest.mark.parametrize("var", [dict(fma2=1), dict(fma2=1, block=512), dict(fma2=1, branchy=1)], ids=str)
@pytest.mark.parametrize("name", ["bcc_quintic", "fcc6", "voronoi2_bcc"])
def test_paired_fma_transform(name, var):
    """The coefficient transform in paired FP32 FMA with constant-bank pairs."""
    if var.get("branchy") and name == "bcc_quintic":
        pytest.skip("one reference sub-region")
    _check(name, var)


@pytest.mark.parametrize("name", ["bcc_quintic", "fcc6", "tricubic", "bcc_linear"])
def test_plain_transform(name):
    """The coefficient transform as direct sums over the sites (the factored
    transform is the default)."""
    _check(name, dict(plain_transform=1))
