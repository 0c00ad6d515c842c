"""The stored oracle values of the batched workload (tests/golden) are the
oracle's: a few volumes of each spline are recomputed from their seeded inputs
and must match the file exactly, and the file covers the benchmark's recipe."""
import json
import os

import numpy as np

import workloads
from tests.golden import make_batched_oracle as mk

PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "batched_oracle_sample.json")


def test_file_covers_the_recipe():
    doc = json.load(open(PATH))
    recipe = workloads.batch_recipe(64, seed=0)
    assert len(doc["volumes"]) == len(recipe)
    for g, it in zip(doc["volumes"], recipe):
        assert (g["spline"], tuple(g["ext"]), g["seed"]) == (it.spline, tuple(it.ext), it.seed)
        assert len(g["f32"]) == len(g["bf16"]) == len(g["f16"]) == doc["sample_per_volume"]


def test_values_are_the_oracles():
    doc = json.load(open(PATH))
    recipe = workloads.batch_recipe(64, seed=0)
    seen = set()
    for g, it in zip(doc["volumes"], recipe):
        if it.spline in seen or it.edge > 128:
            continue
        seen.add(it.spline)
        vals = mk.volume_values(it)
        for tag in ("f32", "bf16", "f16"):
            assert np.array_equal(np.asarray(vals[tag]), np.asarray(g[tag])), (it.spline, tag)
        assert vals["cmax"] == g["cmax"]
    assert len(seen) >= 3


def test_bf16_rounding_is_round_to_nearest_even():
    """The script's BF16 rounding against the definition on hand-picked values."""
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -8 + 2 ** -20, -2.5, 3.0e-39], np.float32)
    want = np.array([1.0, 1.0, 1.0 + 4 * 2 ** -8, 1.0 + 2 ** -7, -2.5, 0.0], np.float32)
    got = mk.to_bf16(x)
    assert np.array_equal(got[:5], want[:5])
    assert abs(float(got[5]) - 3.0e-39) <= 2 ** -133
