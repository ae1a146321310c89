"""Host check of the float-float dot product that the SCDM QR update uses for
single-precision candidate columns: q (double) split as qh + ql in float,
each qh a as a rounded product plus its exact error (an fma), ql a rounded,
the running sum as an unevaluated float pair (TwoSum).  Emulated here with
numpy float32 rounding (an fma of floats is exact in double before its one
rounding); checked against exact rational arithmetic: the error stays within
a few 2^-48 of sum |q_i a_i|, where a float dot product would be ~2^-24."""
from fractions import Fraction

import numpy as np
import pytest

f32 = np.float32


def fma32(x, y, z):
    # x y is exact in double for floats x, y; one rounding of the exact x y + z
    # (z is a float, so x y + z differs from the double sum by at most a
    # double rounding, far below float resolution)
    return f32(float(x) * float(y) + float(z))


def ff_dot(q, a):
    sh = sl = f32(0)
    for qi, ai in zip(q, a):
        qh = f32(qi)
        ql = f32(qi - float(qh))
        p = f32(qh * ai)
        e = fma32(qh, ai, -p)
        e = fma32(ql, ai, e)
        s = f32(sh + p)
        bb = f32(s - sh)
        t = f32(f32(sh - f32(s - bb)) + f32(p - bb))
        sl = f32(sl + f32(t + e))
        sh = s
    return float(sh) + float(sl)


@pytest.mark.parametrize("seed,n", [(1, 128), (2, 512), (3, 37)])
def test_float_float_dot_accuracy(seed, n):
    rng = np.random.default_rng(seed)
    q = rng.standard_normal(n)
    q /= np.linalg.norm(q)
    a = rng.standard_normal(n).astype(np.float32)
    exact = sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(q, a))
    scale = float(np.abs(q).dot(np.abs(a.astype(np.float64))))
    err_ff = abs(Fraction(ff_dot(q, a)) - exact) / Fraction(scale)
    assert float(err_ff) < 8 * 2.0 ** -48
    # a plain float dot product for contrast
    s = f32(0)
    for x, y in zip(q, a):
        s = f32(s + f32(f32(x) * y))
    assert float(abs(Fraction(float(s)) - exact) / Fraction(scale)) > float(err_ff)


def test_float_float_dot_cancellation():
    """q nearly orthogonal to a (the residual downdating case): the result is
    still accurate relative to sum |q_i a_i|."""
    rng = np.random.default_rng(4)
    a = rng.standard_normal(256).astype(np.float32)
    q = rng.standard_normal(256)
    q -= q.dot(a.astype(np.float64)) / float(a.astype(np.float64).dot(a)) * a.astype(np.float64)
    q /= np.linalg.norm(q)
    exact = sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(q, a))
    scale = float(np.abs(q).dot(np.abs(a.astype(np.float64))))
    assert float(abs(Fraction(ff_dot(q, a)) - exact) / Fraction(scale)) < 8 * 2.0 ** -48
