"""Linear texture fetch (Sec. 4.4.1) for the tensor-product splines.

Pairs of neighbouring sites become one hardware-interpolated fetch, so the
result carries the texture unit's fixed-point interpolation: each axis'
fraction is kept to 8 bits (off by less than 1/256 when truncated), and a
trilinear value is multilinear in the three fractions with slopes at most
|c_a - c_b| <= 2 ||c||_inf, so a fetch is off by less than 3 * 2 ||c||_inf / 256;
the fetch weights sum to one: |f_tex - f| <= 6 ||c||_inf / 256 (< 2.4e-2).
"""
import numpy as np
import pytest
import torch

import oracle
import workloads
from oracle import specs as ospecs

pytestmark = pytest.mark.gpu

SPECS = {"trilinear": ospecs.trilinear, "triquadratic": ospecs.triquadratic, "tricubic": ospecs.tricubic}
BOUND = 6.0 / 256.0


@pytest.mark.parametrize("name", sorted(SPECS))
def test_linear_fetch_within_the_fixed_point_bound(name):
    from paper_2102_08518_b300.api import Spline, Volume
    ext = (20, 17, 23)
    coef = workloads.coef_uniform("cc", ext, seed=301)
    vol = Volume(Spline(name, "f32"), ext, torch.from_numpy(coef).cuda())
    vol.texture_sync()
    lo, hi = workloads.bounding_box("cc", ext)
    pts = workloads.points_uniform(20000, lo - 2.5, hi + 2.5, seed=302)
    pts[3] = np.nan
    pts[4] = 1e9
    p = torch.from_numpy(pts).cuda()
    got = vol.eval_linear_fetch(p).cpu().numpy().astype(np.float64)
    ref = vol.eval(p).cpu().numpy().astype(np.float64)
    assert np.isnan(got[3]) and got[4] == 0.0
    ok = np.isfinite(ref)
    cmax = np.abs(coef).max()
    assert np.max(np.abs(got[ok] - ref[ok])) <= BOUND * cmax
    want = oracle.eval_sum(SPECS[name]().with_extent(ext), coef.astype(np.float64).ravel(),
                           pts[5:2005].astype(np.float64))
    assert np.max(np.abs(got[5:2005] - want)) <= BOUND * cmax + 2e-6 * cmax
    # the interpolation error is a fraction of the bound on average
    assert np.mean(np.abs(got[ok] - ref[ok])) <= 0.2 * BOUND * cmax


def test_linear_fetch_follows_texture_sync():
    """The texture is a copy: it changes with the coefficients only after a sync."""
    from paper_2102_08518_b300 import _abi
    from paper_2102_08518_b300.api import Spline, Volume
    ext = (16, 16, 16)
    c = torch.from_numpy(workloads.coef_uniform("cc", ext, seed=303)).cuda()
    vol = Volume(Spline("tricubic", "f32"), ext, c)
    p = torch.from_numpy(workloads.points_uniform(4096, [2] * 3, [13] * 3, seed=304)).cuda()
    with pytest.raises(_abi.LsError):
        vol.eval_linear_fetch(p)
    vol.texture_sync()
    a = vol.eval_linear_fetch(p).clone()
    c.mul_(2.0)
    b = vol.eval_linear_fetch(p).clone()
    vol.texture_sync()
    d = vol.eval_linear_fetch(p)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    assert torch.allclose(d, 2.0 * a, rtol=0, atol=2 * BOUND * 2.0)


def test_linear_fetch_rejects_other_splines():
    from paper_2102_08518_b300 import _abi
    from paper_2102_08518_b300.api import Spline, Volume
    vol = Volume(Spline("bcc_linear", "f32"), (8, 8, 8))
    with pytest.raises(_abi.LsError):
        vol.texture_sync()
