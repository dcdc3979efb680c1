"""Host model (numpy float32) of the double-word scalars of the double-float
panel: each FP32 operation is rounded to nearest as on the GPU, and an FMA
is formed exactly in float64 (the products of two 24-bit significands are
exact there) before one rounding to float32.  Checks the accuracy the kernel
comment states (about 44 bits for quotient and square root, ~2^-46 for sum
and product) against float64 / exact-rational references, and that the
double-float multiply-add used by the bulk updates (exact product, two-sum
accumulation) keeps ~2^-46 relative to the sum of |terms| over long dot
products.  Methods: Knuth's two-sum, Dekker's fast two-sum, FMA-exact
products, one Newton correction for the quotient and the square root."""
from fractions import Fraction

import numpy as np
import pytest

f32 = np.float32


def fma(a, b, c):
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def fast(a, b):
    s = f32(a + b)
    return s, f32(b - f32(s - a))


def dw_add(x, y):
    s = f32(x[0] + y[0])
    bb = f32(s - x[0])
    e = f32(f32(x[0] - f32(s - bb)) + f32(y[0] - bb))
    return fast(s, f32(e + f32(x[1] + y[1])))


def dw_mul(x, y):
    p = f32(x[0] * y[0])
    e = fma(x[0], y[1], fma(x[1], y[0], fma(x[0], y[0], -p)))
    return fast(p, e)


def dw_div(x, y):
    q1 = f32(x[0] / y[0])
    r = f32(fma(-q1, y[0], x[0]) + fma(-q1, y[1], x[1]))
    return fast(q1, f32(r / y[0]))


def dw_sqrt(x):
    if not x[0] > 0:
        return f32(0), f32(0)
    s = f32(np.sqrt(x[0]))
    e = f32(fma(-s, s, x[0]) + x[1])
    return fast(s, f32(e / f32(f32(2) * s)))


def split(v):
    hi = f32(v)
    return hi, f32(np.float64(v) - np.float64(hi))


def val(x):
    return Fraction(float(x[0])) + Fraction(float(x[1]))


def rel(x, exact):
    return abs(float((val(x) - exact) / exact))


@pytest.fixture(scope="module")
def samples():
    rng = np.random.default_rng(11)
    a = rng.standard_normal(400) * 10.0 ** rng.integers(-6, 6, 400)
    b = rng.standard_normal(400) * 10.0 ** rng.integers(-6, 6, 400)
    return [(split(x), split(y)) for x, y in zip(a, b)]


def test_product_and_sum(samples):
    for x, y in samples:
        assert rel(dw_mul(x, y), val(x) * val(y)) < 2.0 ** -45
        s = val(x) + val(y)
        if s != 0 and abs(s) > 1e-3 * (abs(val(x)) + abs(val(y))):
            assert rel(dw_add(x, y), s) < 2.0 ** -44


def test_quotient_and_square_root(samples):
    for x, y in samples:
        assert rel(dw_div(x, y), val(x) / val(y)) < 2.0 ** -43
        ax = (f32(abs(x[0])), f32(abs(x[1])) if x[0] * x[1] >= 0 else f32(-abs(x[1])))
        r = dw_sqrt(ax)
        # compare r^2 with the input: relative error of the root ~ half of that
        assert abs(float((val(r) ** 2 - val(ax)) / val(ax))) < 2.0 ** -42


def test_results_are_normalised(samples):
    for x, y in samples:
        for z in (dw_mul(x, y), dw_div(x, y), dw_add(x, y)):
            hi, lo = float(z[0]), float(z[1])
            assert abs(lo) <= abs(hi) * 2.0 ** -23 or hi == 0.0


def df_mac(s, a, b):
    """The bulk updates' multiply-add: exact FMA product, two-sum of the high parts,
    cross terms into the low word."""
    p = f32(a[0] * b[0])
    e = fma(a[0], b[0], -p)
    t = fma(a[0], b[1], fma(a[1], b[0], e))
    hi = f32(s[0] + p)
    bp = f32(hi - s[0])
    err = f32(f32(s[0] - f32(hi - bp)) + f32(p - bp))
    return hi, f32(s[1] + f32(err + t))


@pytest.mark.parametrize("K", [16, 144, 1000])
def test_double_float_dot_product(K):
    rng = np.random.default_rng(K)
    a = rng.standard_normal(K)
    b = rng.standard_normal(K)
    s = (f32(0), f32(0))
    for x, y in zip(a, b):
        s = df_mac(s, split(x), split(y))
    exact = sum(val(split(x)) * val(split(y)) for x, y in zip(a, b))
    scale = sum(abs(val(split(x)) * val(split(y))) for x, y in zip(a, b))
    assert abs(float((val(s) - exact) / scale)) < K * 2.0 ** -46
