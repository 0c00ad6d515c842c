"""The oracle's pins catch plausible mistakes planted in the oracle.

Each mutant is a copy of oracle/orc.c with one deliberate error (a flipped
sign, a dropped term, an off-by-one, a transposed operand, wrong centring, a
lost normalisation, a truncated site loop), compiled on the CPU and checked by a
fast subset of the pins in test_oracle_pins.py.  Every mutant must fail at least
one check, and the unmodified source must pass them all.
"""
import ctypes
import json
import math
import os
import subprocess
from fractions import Fraction

import numpy as np
import pytest

import oracle
import oracle.lib as olib
from oracle import specs

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "oracle", "orc.c")

MUTANTS = {
    "recurrence_sign": ("sum += te * a0 + (1.0 - te) * a1;", "sum += te * a0 + (1.0 + te) * a1;"),
    "memo_recurrence_sign": ("sum += T * a0 + ((double)r[d] - T) * a1;", "sum += T * a0 + ((double)r[d] + T) * a1;"),
    "memo_divisor_off_by_one": ("            res = sum / (double)(m - k);", "            res = sum / (double)(m - k + 1);"),
    "factor_support": ("if (!(tau >= 0.0 && tau < 1.0)) return 0.0;", "if (!(tau >= 0.0 && tau < 2.0)) return 0.0;"),
    "shift_sign": ("x[i] -= s[d] * c->dir[d][i];", "x[i] += s[d] * c->dir[d][i];"),
    "dropped_cubic_term": ("return 2.0 / 3.0 - a * a + 0.5 * a * a * a;", "return 2.0 / 3.0 - a * a + 0.5 * a * a;"),
    "centring": ("0.5 * sp->dirs[3 * j + i] : 0.0;", "1.0 * sp->dirs[3 * j + i] : 0.0;"),
    "normalisation": ("double v = sp->detL * memo_eval(&p->full, x);", "double v = memo_eval(&p->full, x);"),
    "gradient_sign": ("(memo_eval(&p->part[n], x) - memo_eval(&p->part[n], xs))",
                      "(memo_eval(&p->part[n], xs) - memo_eval(&p->part[n], x))"),
    "site_loop_truncated": ("if (hi[i] > sp->ext[i] - 1) hi[i] = sp->ext[i] - 1;",
                            "if (hi[i] > sp->ext[i] - 2) hi[i] = sp->ext[i] - 2;"),
    "transposed_solve": ("for (int j = 0; j < k; ++j) a[i][j] = cols[j][i];",
                         "for (int j = 0; j < k; ++j) a[i][j] = cols[i][j];"),
    "basis_weight_dropped": ("if (b[q] == n) T = tb[q];", "if (b[q] == n) T = 0.0;"),
}


def _build(tmp_path, name, src):
    c = tmp_path / f"orc_{name}.c"
    so = tmp_path / f"liborc_{name}.so"
    c.write_text(src)
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
                    "-ffp-contract=off", "-w", "-o", str(so), str(c), "-lm"], check=True)
    return olib.configure(ctypes.CDLL(str(so)))


def _fig1_ok():
    g = json.load(open(os.path.join(HERE, "golden", "fig1_zp_subregion1.json")))
    W = np.array([[float(Fraction(v)) for v in g["weights"][f"c{j}"]] for j in range(7)])
    rng = np.random.default_rng(1)
    coef = rng.uniform(-1, 1, (7, 7))
    c = np.array([coef[3 + s1, 3 + s0] for s0, s1 in g["sites"]])
    spec = specs.zp2d().with_extent((7, 7))
    pts = []
    while len(pts) < 20:
        x = rng.uniform(-0.5, 0.5, 2)
        if x[0] > abs(x[1]):
            pts.append(x)
    pts = np.array(pts)
    got = oracle.eval_sum(spec, coef.ravel(), pts + 3.0)
    want = np.array([c @ (W @ np.array([x[0] ** a * x[1] ** b for a, b in g["monomials"]])) for x in pts])
    return np.max(np.abs(got - want)) < 1e-12


def _checks():
    """Fast pins; each returns True when the oracle behaves."""
    out = {}
    out["fig1"] = _fig1_ok()
    rng = np.random.default_rng(2)
    for name, mk in specs.ALL_3D.items():
        spec = mk().with_extent((10, 10, 10) if mk().scale == 1 else (7, 7, 7))
        pts = rng.uniform(4.5, 6.5 if spec.scale == 1 else 8.5, (20, 3))
        out[f"pu_{name}"] = np.max(np.abs(oracle.eval_sum(spec, np.ones(spec.n_coef()), pts) - 1)) < 1e-12
        y = rng.uniform(-2.0, 2.0, (8, 3))
        base = oracle.phi(mk(), y)
        out[f"sym_{name}"] = np.max(np.abs(oracle.phi(mk(), y[:, [1, 0, 2]] * [-1, 1, 1]) - base)) < 1e-12
        # gradient against central differences of the value
        coef = rng.uniform(-1, 1, spec.n_coef())
        f, g = oracle.eval_sum_grad(spec, coef, pts[:6])
        h = 1e-6
        fd = (oracle.eval_sum(spec, coef, pts[:6] + [h, 0, 0]) - oracle.eval_sum(spec, coef, pts[:6] - [h, 0, 0])) / (2 * h)
        out[f"grad_{name}"] = np.max(np.abs(fd - g[:, 0])) < 1e-5
    # cardinal cubic B-spline (truncated powers) and the recurrence form of the tricubic
    xs = np.linspace(0.1, 3.9, 9)
    tp = lambda x: sum((-1) ** k * math.comb(4, k) * (max(x - k, 0.0) ** 3) for k in range(5)) / 6
    out["cardinal"] = all(abs(oracle.box([[1.0]] * 4, [x]) - tp(x)) < 1e-12 for x in xs)
    y = rng.uniform(-2.2, 2.2, (10, 3))
    out["tricubic_closed"] = np.max(np.abs(oracle.phi(specs.tricubic(True), y) - oracle.phi(specs.tricubic(False), y))) < 1e-12
    out["beta3_values"] = abs(oracle.phi(specs.tricubic(True), [[0, 0, 0]])[0] - 8 / 27) < 1e-14 and \
        abs(oracle.phi(specs.tricubic(True), [[0.5, 0, 0]])[0] - (2 / 3) ** 2 * (2 / 3 - 0.25 + 0.0625)) < 1e-14
    # every stored site, brute force, including points near the array edges
    spec = specs.fcc6().with_extent((5, 5, 5))
    coef = rng.uniform(-1, 1, spec.n_coef())
    allsites = []
    for l in spec.cosets:
        for i2 in range(5):
            for i1 in range(5):
                for i0 in range(5):
                    allsites.append([2 * i0 + l[0], 2 * i1 + l[1], 2 * i2 + l[2]])
    allsites = np.array(allsites, float)
    p = rng.uniform(-1.0, 10.0, (6, 3))
    got = oracle.eval_sum(spec, coef, p)
    want = np.array([coef @ oracle.phi(spec, x[None, :] - allsites) for x in p])
    out["enumeration"] = np.max(np.abs(got - want)) < 1e-12
    return out


@pytest.fixture(scope="module")
def source():
    return open(SRC).read()


def _with_lib(lib):
    saved = olib._lib
    olib._lib = lib
    try:
        return _checks()
    finally:
        olib._lib = saved


def test_unmodified_oracle_passes_the_fast_pins(tmp_path, source):
    res = _with_lib(_build(tmp_path, "orig", source))
    assert all(res.values()), [k for k, v in res.items() if not v]


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_planted_mistake_is_caught(tmp_path, source, mutant):
    old, new = MUTANTS[mutant]
    assert source.count(old) == 1, mutant
    res = _with_lib(_build(tmp_path, mutant, source.replace(old, new)))
    failed = [k for k, v in res.items() if not v]
    assert failed, f"mutant {mutant} passed every fast pin"
