"""CPU checks of the FP32 arithmetic the pair kernel relies on (no GPU).

The kernel's Newtonian tail forms y^3 (r^2 y^2 - A) from the SFU estimate y of
(r^2)^-1/2 and accumulates forces in the scale sigma = -(A - 1), removed in FP64
at the end.  Here the constants are read from the kernel's shared header and the
identity is checked in emulated FP32 (each fused multiply-add rounded once):
after removing sigma the tail must equal r^-3 to a few units in the last place
for every estimate within the SFU's error, i.e. it is one Newton step.
"""
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUH = os.path.join(ROOT, "paper_1810_02916_b300", "csrc", "nf_internal.cuh")


def _constant(name):
    text = open(CUH).read()
    m = re.search(rf"constexpr\s+(?:float|double)\s+{name}\s*=\s*([^;]+);", text)
    assert m, name
    expr = m.group(1).replace("f", "")
    return eval(expr, {"__builtins__": {}})


def _fma32(a, b, c):
    # a*b is exact in float64 for float32 inputs (48 significant bits); adding c
    # (float32, same magnitude range here) stays exact, so one rounding to float32
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def test_scale_constants_are_exact():
    A = np.float32(_constant("kNewtonA"))
    sigma = np.float32(_constant("kForceSigma"))
    unscale = _constant("kForceUnscale")
    assert A == np.float32(5.0 / 3.0)                       # nearest FP32 to 5/3
    assert float(A) == 13981013 * 2.0 ** -23
    assert float(sigma) == -(float(A) - 1.0)                # A - 1 is exact in FP32
    assert float(np.float32(float(A) - 1.0)) == float(A) - 1.0
    assert unscale == 1.0 / float(sigma)


def test_scaled_newton_tail_is_one_newton_step():
    A = np.float32(_constant("kNewtonA"))
    sigma = float(_constant("kForceSigma"))
    rng = np.random.default_rng(3)
    r2 = np.exp(rng.uniform(np.log(1.0), np.log(27.0), 200000)).astype(np.float32)   # far pairs, cell units
    exact = r2.astype(np.float64) ** -1.5
    # estimates within 2^-21 of (r^2)^-1/2, beyond the SFU's stated error
    delta = rng.uniform(-2.0 ** -21, 2.0 ** -21, r2.size)
    y = (r2.astype(np.float64) ** -0.5 * (1.0 + delta)).astype(np.float32)
    yy = (y * y).astype(np.float32)
    g = _fma32(r2, yy, np.full_like(r2, -A))
    f = ((yy * y).astype(np.float32) * g).astype(np.float32)
    rel = np.abs(f.astype(np.float64) / sigma - exact) / exact
    assert rel.max() < 6 * 2.0 ** -24, rel.max()
    # without the Newton factor the raw cube is off by up to 3 delta
    raw = np.abs((yy * y).astype(np.float64) - exact) / exact
    assert raw.max() > 16 * 2.0 ** -24


def test_dropping_the_factor_or_using_the_unrounded_constant_is_caught():
    """Plausible slips in the tail: forgetting 1 + 3e, or removing the scale with
    -(5/3 - 1) instead of the FP32 constant's own value."""
    A = np.float32(_constant("kNewtonA"))
    rng = np.random.default_rng(4)
    r2 = np.exp(rng.uniform(0.0, np.log(27.0), 50000)).astype(np.float32)
    exact = r2.astype(np.float64) ** -1.5
    y = (r2.astype(np.float64) ** -0.5 * (1.0 + rng.uniform(-2.0 ** -22, 2.0 ** -22, r2.size))).astype(np.float32)
    yy = (y * y).astype(np.float32)
    f = ((yy * y).astype(np.float32) * _fma32(r2, yy, np.full_like(r2, -A))).astype(np.float32)
    wrong_scale = np.abs(f / -(2.0 / 3.0) - exact) / exact
    # a consistent bias of 6e-8 in every pair: small per pair, systematic over a sum
    assert np.median(wrong_scale) > 2.0 ** -25
