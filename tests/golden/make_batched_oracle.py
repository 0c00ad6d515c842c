"""Write the FP64 oracle's values for the batched mixed-precision workload.

The benchmark's batched configuration holds 64 volumes (edges drawn from
{32..256}, splines from {Cartesian tricubic, BCC linear, BCC quintic, FCC
six-direction}) with coefficients U[-1, 1] stored in BF16 and in FP16.  For a
seeded sample of SAMPLE points per volume this script evaluates Eq. 1 with the
oracle on three coefficient sets: the FP32 values, and the same values rounded
to BF16 and to FP16 (round to nearest even).  The benchmark reads the file and
reports, per volume, the batched kernel's error against the oracle on both the
rounded and the original coefficients.  Inputs come from workloads/ (seeded,
no spline arithmetic); values come only from oracle/.

    python tests/golden/make_batched_oracle.py      # rewrites batched_oracle_sample.json
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads  # noqa: E402
from oracle import specs  # noqa: E402

SAMPLE = 32
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "batched_oracle_sample.json")
SPEC = {"tricubic": specs.tricubic, "bcc_linear": specs.bcc_linear, "bcc_quintic": specs.bcc_quintic,
        "fcc6": specs.fcc6}


def to_bf16(c: np.ndarray) -> np.ndarray:
    """FP32 -> BF16 (round to nearest even on the 16 dropped bits), widened back to FP32."""
    b = c.astype(np.float32).view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def to_f16(c: np.ndarray) -> np.ndarray:
    return c.astype(np.float32).astype(np.float16).astype(np.float32)


def sample_points(item) -> np.ndarray:
    lo, hi = workloads.inner_box(item.spline, item.ext)
    return workloads.points_uniform(SAMPLE, lo, hi, seed=item.seed + 7)


def volume_values(item, nthreads: int = 0):
    lat = workloads.SPLINE_LATTICE[item.spline]
    coef = workloads.coef_uniform(lat, item.ext, seed=item.seed)
    pts = sample_points(item).astype(np.float64)
    spec = SPEC[item.spline]().with_extent(item.ext)
    out = {}
    for tag, c in (("f32", coef), ("bf16", to_bf16(coef)), ("f16", to_f16(coef))):
        out[tag] = oracle.eval_sum(spec, c.astype(np.float64).ravel(), pts,
                                   nthreads=nthreads or len(os.sched_getaffinity(0))).tolist()
    out["cmax"] = float(np.abs(coef).max())
    return out


def main():
    recipe = workloads.batch_recipe(64, seed=0)
    vols = []
    for v, it in enumerate(recipe):
        vals = volume_values(it)
        vols.append({"volume": v, "spline": it.spline, "ext": list(it.ext), "seed": it.seed, **vals})
        print(v, it.spline, it.ext, flush=True)
    doc = {"source": "FP64 oracle (oracle/orc.c, Eq. 1) at SAMPLE seeded points per volume of the batched "
                     "workload; written by tests/golden/make_batched_oracle.py",
           "sample_per_volume": SAMPLE, "points_seed": "volume seed + 7 (workloads.points_uniform, inner box)",
           "volumes": vols}
    with open(OUT, "w") as f:
        json.dump(doc, f, indent=0)


if __name__ == "__main__":
    main()
