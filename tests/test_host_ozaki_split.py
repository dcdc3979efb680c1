"""The digit arithmetic of the tensor-core residual, modelled exactly on the
host (Python integers and fractions): what the kernels compute is

  x = (-1)^s 2^E sum_{l=1..8} d_l 2^{-7l} + r,  d_l in [0, 127],  |r| < 2^{E-56},

with 2^E > max |x| over the row (of H) or column (of Xhat); the slice products
of one level t = k + l summed over a 128-deep window stay below 2^24 (exact in
FP32); and keeping the 36 products with k + l <= 9 reproduces the dot product
to within the bound the kernel's tolerance is derived from.  Error-free
splitting: Ozaki, Ogita, Oishi, Rump (2012)."""
import math
from fractions import Fraction

import numpy as np
import pytest

SL = 8      # slices
WIN = 128   # accumulation window (K)


def scale_exp(maxabs):
    """E with 2^(E-1) <= maxabs < 2^E (normal maxabs), from the exponent field."""
    if maxabs == 0.0:
        return -1022
    m, e = math.frexp(maxabs)  # maxabs = m 2^e, 0.5 <= m < 1
    return e


def digits(x, E):
    """Sign and the eight 7-bit digits of |x| 2^(56-E), truncated (as the kernels)."""
    M = math.floor(abs(Fraction(x)) * Fraction(2) ** (56 - E))
    assert 0 <= M < 2 ** 56
    return (-1 if math.copysign(1.0, x) < 0 else 1), [(M >> (49 - 7 * l)) & 127 for l in range(SL)]


def value(sign, d, E):
    return sign * sum(Fraction(dl) * Fraction(2) ** (E - 7 * (l + 1)) for l, dl in enumerate(d))


def test_scale_exponent_brackets_the_maximum():
    rng = np.random.default_rng(1)
    for v in np.concatenate([rng.uniform(0, 1, 50) * 10.0 ** rng.integers(-30, 30, 50), [1.0, 0.5, 2.0 ** 40]]):
        E = scale_exp(float(v))
        assert 2.0 ** (E - 1) <= v < 2.0 ** E


def test_digits_reconstruct_within_two_to_minus_56():
    rng = np.random.default_rng(2)
    xs = rng.standard_normal(400) * 10.0 ** rng.integers(-8, 8, 400)
    E = scale_exp(float(np.max(np.abs(xs))))
    for x in xs:
        s, d = digits(float(x), E)
        assert all(0 <= dl <= 127 for dl in d)
        assert abs(Fraction(float(x)) - value(s, d, E)) < Fraction(2) ** (E - 56)
    # a value equal to a power of two at the top of the range still fits
    s, d = digits(-0.5, scale_exp(0.5))
    assert d[0] == 64 and s == -1 and value(s, d, 0) == Fraction(-1, 2)


def test_level_window_sums_are_exact_in_fp32():
    # the largest possible window sum of a level: (t - 1) products of 127 x 127, 128 deep
    assert 8 * WIN * 127 * 127 < 2 ** 24
    rng = np.random.default_rng(3)
    d = rng.integers(0, 128, size=(2, WIN, SL))
    sg = rng.choice([-1, 1], size=(2, WIN))
    for t in range(2, SL + 2):
        tot = 0
        for k in range(max(1, t - SL), min(SL, t - 1) + 1):
            tot += int(np.sum(sg[0] * sg[1] * d[0, :, k - 1] * d[1, :, t - k - 1]))
        assert abs(tot) < 2 ** 24
        assert float(np.float32(tot)) == tot


def test_truncated_level_sum_reproduces_the_dot_product():
    """sum_j h_j x_j from the 36 products with k + l <= 9 (levels scaled by
    2^(E_h + E_x - 7t)) is within sqrt-free worst case K * 16 * 2^(E_h + E_x - 56)."""
    rng = np.random.default_rng(4)
    for K in (1, 37, 300):
        h = rng.standard_normal(K) * 10.0 ** rng.integers(-3, 3, K)
        x = rng.standard_normal(K)
        Eh, Ex = scale_exp(float(np.max(np.abs(h)))), scale_exp(float(np.max(np.abs(x))))
        dh = [digits(float(v), Eh) for v in h]
        dx = [digits(float(v), Ex) for v in x]
        exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(h, x))
        approx = Fraction(0)
        for t in range(2, SL + 2):
            L = 0
            for k in range(max(1, t - SL), min(SL, t - 1) + 1):
                l = t - k
                L += sum(sa * sb * da[k - 1] * db[l - 1] for (sa, da), (sb, db) in zip(dh, dx))
            approx += Fraction(L) * Fraction(2) ** (Eh + Ex - 7 * t)
        bound = K * 16 * Fraction(2) ** (Eh + Ex - 56)
        assert abs(approx - exact) <= bound
        # and the bound is far below the scale of the terms
        assert float(bound) <= 1e-14 * 2.0 ** (Eh + Ex) * K


@pytest.mark.parametrize("drop_level", [2, 5, 9])
def test_dropping_a_kept_level_is_detected(drop_level):
    """A plausible slip (one level left out of the recombination) breaks the bound."""
    rng = np.random.default_rng(5)
    K = 64
    h = rng.standard_normal(K)
    x = rng.standard_normal(K)
    Eh, Ex = scale_exp(float(np.max(np.abs(h)))), scale_exp(float(np.max(np.abs(x))))
    dh = [digits(float(v), Eh) for v in h]
    dx = [digits(float(v), Ex) for v in x]
    exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(h, x))
    approx = Fraction(0)
    for t in range(2, SL + 2):
        if t == drop_level:
            continue
        L = sum(sa * sb * da[k - 1] * db[t - k - 1]
                for k in range(max(1, t - SL), min(SL, t - 1) + 1)
                for (sa, da), (sb, db) in zip(dh, dx))
        approx += Fraction(L) * Fraction(2) ** (Eh + Ex - 7 * t)
    assert abs(approx - exact) > K * 16 * Fraction(2) ** (Eh + Ex - 56)
