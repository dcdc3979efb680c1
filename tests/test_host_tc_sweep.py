"""Host models (no GPU) of the tensor-core sweep (SSV_SPLIT and the mixed
path's first solve):

  * its digit arithmetic: eight 7-bit digits per row of H, seven per column of
    a block transform, the 35 products with k + l <= 7 summed per level over a
    128-deep block, every level sum exact in FP32, and the recombination
    2^(E_h + E_p) sum_t 2^(-7 (t + 2)) L_t within about 2^-49 of the row and
    column scales (exact integers and fractions);
  * its block schedule: the first block takes (n - m) mod n_b rows so that every
    later block starts at a multiple of n_b; the rows above each block are
    updated as Z1 P1 + Z2 P2 - sigma E P1 with the shifted-diagonal rows
    r - m + c, c < min(m, n_b,eff); the block transforms' P2 are parked in the
    output rows n - b m .. n - (b - 1) m - 1 and read back by the X-hat back
    pass before it writes over them.  Modelled in float64 with any orthonormal
    null-space basis as the block transform (the result does not depend on
    which), and compared with the oracle's dense solve.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import workloads as W

SDH = 8     # digits of a row of H
SD = 7      # digits of a column of a block transform
LEV = 8     # levels k + l = 0 .. 7
NB = 128    # block rows = K of one update


def scale_exp(maxabs):
    if maxabs == 0.0:
        return -1022
    return math.frexp(maxabs)[1]


def digits(x, E):
    M = math.floor(abs(Fraction(x)) * Fraction(2) ** (56 - E))
    return (-1 if math.copysign(1.0, x) < 0 else 1), [(M >> (49 - 7 * l)) & 127 for l in range(8)]


def level_pairs(t):
    """(k, l) digit pairs of level t: H digit k < 8, transform digit l < 7."""
    return [(k, t - k) for k in range(max(0, t - (SD - 1)), min(SDH - 1, t) + 1)]


def test_level_sums_of_one_block_are_exact_in_fp32():
    counts = [len(level_pairs(t)) for t in range(LEV)]
    assert counts == [1, 2, 3, 4, 5, 6, 7, 7] and sum(counts) == 35
    # the issuers' shares of the products ({7, 1}, {6, 0}, {5, 2}, {4, 3})
    owner = {7: 0, 1: 0, 6: 1, 0: 1, 5: 2, 2: 2, 4: 3, 3: 3}
    shares = [sum(counts[t] for t in range(LEV) if owner[t] == i) for i in range(4)]
    assert shares == [9, 8, 9, 9]
    assert max(counts) * NB * 127 * 127 < 2 ** 24


def test_seven_digit_products_reproduce_the_block_product():
    """sum_c h_c p_c over one block from the 35 digit products (k + l <= 7),
    scaled as the update's epilogue scales them, is within K 2^(E_h + E_p - 48)
    of the exact value: about 2^-49 relative to the row and column scales."""
    rng = np.random.default_rng(11)
    for K in (1, 56, NB):
        h = rng.standard_normal(K) * 10.0 ** rng.integers(-2, 2, K)
        pcol = rng.standard_normal(K) * 0.3
        Eh, Ep = scale_exp(float(np.max(np.abs(h)))), scale_exp(float(np.max(np.abs(pcol))))
        dh = [digits(float(v), Eh) for v in h]
        dp = [digits(float(v), Ep) for v in pcol]
        exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(h, pcol))
        approx = Fraction(0)
        for t in range(LEV):
            L = sum(sa * sb * da[k] * db[l] for k, l in level_pairs(t)
                    for (sa, da), (sb, db) in zip(dh, dp))
            assert abs(L) < 2 ** 24
            approx += Fraction(L) * Fraction(2) ** (Eh + Ep - 7 * (t + 2))
        bound = K * Fraction(2) ** (Eh + Ep - 48)
        assert abs(approx - exact) <= bound
        # the epilogue starts its scale at 2^-14 and divides by 2^7 per level
        assert Fraction(2) ** (-7 * (0 + 2)) == Fraction(1, 2 ** 14)


def test_dropping_the_last_level_is_detected():
    rng = np.random.default_rng(12)
    K = NB
    h = rng.standard_normal(K)
    pcol = rng.standard_normal(K)
    Eh, Ep = scale_exp(float(np.max(np.abs(h)))), scale_exp(float(np.max(np.abs(pcol))))
    dh = [digits(float(v), Eh) for v in h]
    dp = [digits(float(v), Ep) for v in pcol]
    exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(h, pcol))
    approx = Fraction(0)
    for t in range(LEV - 2):   # levels 6 and 7 left out
        L = sum(sa * sb * da[k] * db[l] for k, l in level_pairs(t) for (sa, da), (sb, db) in zip(dh, dp))
        approx += Fraction(L) * Fraction(2) ** (Eh + Ep - 7 * (t + 2))
    assert abs(approx - exact) > K * Fraction(2) ** (Eh + Ep - 48)


def test_eighth_digit_of_h_matters_for_a_dominant_diagonal():
    """A row with one entry 2 and the rest ~0.014 (H of A = -2I + G/sqrt(n)): with
    seven digits of H the small entries keep only about 42 bits; the eighth
    digit brings the row's dot product back within 2^-49 of its scale."""
    rng = np.random.default_rng(13)
    K = NB
    h = rng.standard_normal(K) * 0.014
    h[5] = -2.0
    pcol = rng.standard_normal(K) * 0.1
    Eh, Ep = scale_exp(float(np.max(np.abs(h)))), scale_exp(float(np.max(np.abs(pcol))))
    dh = [digits(float(v), Eh) for v in h]
    dp = [digits(float(v), Ep) for v in pcol]
    exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(h, pcol))

    def approx(ndig_h):
        tot = Fraction(0)
        for t in range(LEV):
            L = sum(sa * sb * da[k] * db[l] for k, l in level_pairs(t) if k < ndig_h
                    for (sa, da), (sb, db) in zip(dh, dp))
            tot += Fraction(L) * Fraction(2) ** (Eh + Ep - 7 * (t + 2))
        return tot

    e8, e7 = abs(approx(8) - exact), abs(approx(7) - exact)
    assert e8 <= K * Fraction(2) ** (Eh + Ep - 48)
    assert e8 < e7


def block_schedule(n, m, nb=NB):
    """[(k, nbe, j0)] of the sweep: the first block (n - m) mod nb rows (nb if 0)."""
    first = (n - m) % nb or nb
    out, k = [], n
    while k > m:
        nbe = first if not out else nb
        out.append((k, nbe, k - m - nbe))
        k -= nbe
    return out


@pytest.mark.parametrize("n,m", [(5000, 16), (300, 3), (17, 16), (144, 16), (145, 1), (1000, 8)])
def test_schedule_aligns_blocks_and_parks_within_the_output(n, m):
    sch = block_schedule(n, m)
    assert sum(nbe for _, nbe, _ in sch) == n - m
    B = len(sch)
    for b, (k, nbe, j0) in enumerate(sch, start=1):
        assert j0 == (B - b) * NB            # fresh columns start at a multiple of n_b
        assert j0 % 32 == 0                  # = a multiple of the digit tiles' depth
        assert 1 <= nbe <= NB and (b == 1 or nbe == NB)
        # parked P2 of step b fits in the output and below the X-hat rows the back
        # pass writes before reading it
        assert n - b * m >= 0
        written_before = j0 + nbe             # back pass writes rows < j0 + nbe at step b
        assert written_before <= n - (b - 1) * m


def null_basis(Z):
    """Orthonormal basis of the right null space of Z (rows x (rows + m))."""
    _, _, vh = np.linalg.svd(Z)
    return vh[Z.shape[0]:].conj().T


def tc_sweep_model(H, R, Ct, sigma, nb=NB):
    """The sweep in the order the tensor-core path runs it, in float64."""
    n, m = R.shape
    p = Ct.shape[0]
    Z1 = np.vstack([Ct, H]).astype(np.complex128)           # original columns, no shift
    Z2 = Z1[:, n - m:].copy()
    for q in range(m):
        Z2[p + n - m + q, q] -= sigma
    ZT = np.zeros((n, m), dtype=np.complex128)
    out = np.zeros((n, m), dtype=np.complex128)              # parking rows, then X-hat
    sch = block_schedule(n, m, nb)
    for b, (k, nbe, j0) in enumerate(sch, start=1):
        r = p + k - nbe
        F = Z1[r:r + nbe, j0:j0 + nbe].copy()
        for t in range(nbe):
            gr = k - nbe + t                                 # global row of block row t
            jc = gr                                          # its diagonal column
            if j0 <= jc < j0 + nbe:
                F[t, jc - j0] -= sigma
        P = null_basis(np.hstack([F, Z2[r:r + nbe]]))
        P1, P2 = P[:nbe], P[nbe:]
        new = Z1[:r, j0:j0 + nbe] @ P1 + Z2[:r] @ P2
        for c in range(min(m, nbe)):                         # diagonal of fresh column c above the block
            new[r - m + c] -= sigma * P1[c]
        Z2[:r] = new
        ZT[j0:j0 + nbe] = P1
        out[n - b * m:n - (b - 1) * m] = P2
    Y = np.linalg.solve(Z2[p:p + m], np.triu(R[:m]))
    G = Z2[:p] @ Y
    z = Y
    B = len(sch)
    for b in range(B, 0, -1):
        k, nbe, j0 = sch[b - 1]
        p2 = out[n - b * m:n - (b - 1) * m].copy()           # read before the rows are written
        out[j0:j0 + nbe] = ZT[j0:j0 + nbe] @ z
        z = p2 @ z
    out[n - m:] = z
    return out, G


@pytest.mark.parametrize("n,m,p", [(300, 3, 2), (200, 16, 16), (17, 16, 4), (144, 16, 3), (145, 1, 1)])
def test_schedule_model_solves_the_reduced_system(ora, n, m, p):
    sysr = W.random_system(n, m, p, seed=900 + n + m)
    H, R, Ct, _ = ora.reduce(sysr.A, sysr.B, sysr.C)
    for sigma in (0.7j, -2.1 + 0.4j):
        X, G = tc_sweep_model(H, R, Ct, sigma)
        Xo, _, _ = ora.reduced_solve(H, R, Ct, [sigma], want="xhat")
        Go, _, _ = ora.reduced_solve(H, R, Ct, [sigma], want="g")
        assert np.linalg.norm(X - Xo[0]) <= 1e-10 * np.linalg.norm(Xo[0])
        assert np.linalg.norm(G - Go[0]) <= 1e-10 * np.linalg.norm(Go[0])


def test_schedule_model_misplaced_diagonal_correction_fails(ora):
    """A shifted-diagonal correction one row off (a plausible slip) is caught."""
    sysr = W.random_system(200, 4, 2, seed=77)
    H, R, Ct, _ = ora.reduce(sysr.A, sysr.B, sysr.C)
    sigma = -1.5 + 0.2j
    Xo, _, _ = ora.reduced_solve(H, R, Ct, [sigma], want="xhat")

    def bad_model():
        n, m = R.shape
        p = Ct.shape[0]
        Z1 = np.vstack([Ct, H]).astype(np.complex128)
        Z2 = Z1[:, n - m:].copy()
        for q in range(m):
            Z2[p + n - m + q, q] -= sigma
        ZT = np.zeros((n, m), dtype=np.complex128)
        P2s = []
        for k, nbe, j0 in block_schedule(n, m):
            r = p + k - nbe
            F = Z1[r:r + nbe, j0:j0 + nbe].copy()
            for t in range(nbe):
                if j0 <= k - nbe + t < j0 + nbe:
                    F[t, k - nbe + t - j0] -= sigma
            P = null_basis(np.hstack([F, Z2[r:r + nbe]]))
            P1, P2 = P[:nbe], P[nbe:]
            new = Z1[:r, j0:j0 + nbe] @ P1 + Z2[:r] @ P2
            for c in range(min(m, nbe)):
                new[r - m + c - 1] -= sigma * P1[c]          # one row too high
            Z2[:r] = new
            ZT[j0:j0 + nbe] = P1
            P2s.append(P2)
        Y = np.linalg.solve(Z2[p:p + m], np.triu(R[:m]))
        X = np.zeros((n, m), dtype=np.complex128)
        z = Y
        for (k, nbe, j0), P2 in reversed(list(zip(block_schedule(n, m), P2s))):
            X[j0:j0 + nbe] = ZT[j0:j0 + nbe] @ z
            z = P2 @ z
        X[n - m:] = z
        return X

    assert np.linalg.norm(bad_model() - Xo[0]) > 1e-6 * np.linalg.norm(Xo[0])


def real_form_B(P2):
    """The real (2m x 2m) operand of Z2 P2 with Z2's row interleaved as
    [Re z_0, Im z_0, Re z_1, ...] and the output interleaved the same way:
    B[2i, 2q] = Re P(i, q), B[2i + 1, 2q] = -Im P(i, q),
    B[2i, 2q + 1] = Im P(i, q), B[2i + 1, 2q + 1] = Re P(i, q)."""
    m = P2.shape[0]
    B = np.zeros((2 * m, 2 * m))
    B[0::2, 0::2] = P2.real
    B[1::2, 0::2] = -P2.imag
    B[0::2, 1::2] = P2.imag
    B[1::2, 1::2] = P2.real
    return B


def test_real_form_of_the_z2_p2_product():
    rng = np.random.default_rng(21)
    for m in (1, 5, 16):
        Z = rng.standard_normal((7, m)) + 1j * rng.standard_normal((7, m))
        P = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
        zr = np.zeros((7, 2 * m))
        zr[:, 0::2], zr[:, 1::2] = Z.real, Z.imag
        out = zr @ real_form_B(P)
        W = Z @ P
        assert np.allclose(out[:, 0::2], W.real) and np.allclose(out[:, 1::2], W.imag)


def float_pair_digits(hi, lo, E):
    """The kernel's digits of x = hi + lo (two FP32 words) relative to 2^E,
    formed from the words' bit fields without FP64: each word contributes its
    24-bit significand shifted to 2^(56 - E) units (truncated toward zero), the
    low word with its own sign."""
    def part(f):
        f = float(np.float32(f))
        if f == 0.0:
            return 0
        mnt, ex = math.frexp(abs(f))          # |f| = mnt 2^ex, 0.5 <= mnt < 1
        mi = int(mnt * 2 ** 24)               # 24-bit significand
        sh = ex - 24 + 56 - E
        v = mi << sh if sh >= 0 else mi >> (-sh)
        return v if f > 0 else -v
    M = part(hi) + part(lo)
    s = -1 if M < 0 else 1
    M = abs(M)
    assert M < 2 ** 56
    return s, [(M >> (49 - 7 * l)) & 127 for l in range(7)]


def test_float_pair_digits_match_the_exact_value():
    rng = np.random.default_rng(22)
    for _ in range(300):
        x = float(rng.standard_normal() * 10.0 ** rng.integers(-3, 3))
        hi = float(np.float32(x))
        lo = float(np.float32(x - hi))
        E = scale_exp(abs(hi) * (1 + 2 ** -23))
        s, d = float_pair_digits(hi, lo, E)
        val = s * sum(Fraction(dl) * Fraction(2) ** (E - 7 * (l + 1)) for l, dl in enumerate(d))
        exact = Fraction(hi) + Fraction(lo)
        assert abs(val - exact) <= Fraction(2) ** (E - 48)
