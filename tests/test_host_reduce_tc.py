"""Host models of the tensor-core reduction and of the fused-level digit products.

1. The two-level blocked reduction (Sec. 2.1, Algorithms 2 and 3, the equations for
   V, T and Y) in the exact order `csrc/reduce_tc.cu` runs it: per mini-block the
   right update by Y and V, the left update by I - V T^T V^T, the Householder QR of
   the mini-block, T's new columns, Y's new columns from A V_s of the block-start
   matrix; per block the right update of the rows above r0 (and of C) from column
   z + m and of the rows r0.. from column z + b, then W = V^T A, Z = T^T W and the left
   update.  With plain FP64 products it must give the oracle's reduced triple
   (Algorithm 1) to 1e-12 after fixing Q's column signs.
2. The digit products, emulated exactly (integer digit planes, level sums below
   2^24 per 128-deep window, 64-bit words, one rounding per word): nine levels give
   an FP64-class product; eight levels, or V's rows at a fixed exponent, are measurably
   worse on long K (the readings behind the kernel's choices).
3. The fused-level issue schedules of every tensor-core kernel cover each digit pair
   exactly once, open every level with the first products of a window, and stay in
   their TMEM columns.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from tests.gpu_util import relerr, sign_matrix

KB = 128  # block width bound of the tensor-core reduction


# ---------------------------------------------------------------------------
# 1. the two-level blocked reduction
# ---------------------------------------------------------------------------
def _panel(P, r0, n, w, wp, pv0, j, c0, V, T, Y, p, tau):
    """One mini-block: P is indexed by matrix row (rows r0..n-1 used), w columns."""
    Ps = P[r0:n, :w].copy()
    if j > 0:
        Ps -= Y[p + r0:p + n, :j] @ V[c0:c0 + w, :j].T              # from the right
        Wm = V[r0:n, :j].T @ Ps                                       # from the left
        Ps -= V[r0:n, :j] @ (np.triu(T[:j, :j]).T @ Wm)
    for t in range(wp):
        rl = pv0 + t - r0
        x = Ps[rl + 1:, t]
        sig = x @ x
        alpha = Ps[rl, t]
        tk = 0.0
        if sig != 0.0:
            nrm = np.sqrt(alpha * alpha + sig)
            beta = -nrm if alpha >= 0 else nrm
            tk = (beta - alpha) / beta
            scal = 1.0 / (alpha - beta)
            wk = Ps[rl, t + 1:] + scal * (Ps[rl + 1:, t + 1:].T @ x)
            v = x * scal
            Ps[rl + 1:, t + 1:] -= tk * np.outer(v, wk)
            Ps[rl, t + 1:] -= tk * wk
            Ps[rl + 1:, t] = v
            Ps[rl, t] = beta
        tau[t] = tk
    P[r0:n, :w] = Ps
    for t in range(wp):
        pr = pv0 + t
        V[:, j + t] = 0.0
        V[pr, j + t] = 1.0
        V[pr + 1:n, j + t] = Ps[pr - r0 + 1:, t]
    S = V[r0:n, :j + wp].T @ V[r0:n, j:j + wp]
    for t in range(wp):
        c = j + t
        T[c, c] = tau[t]
        T[:c, c] = -tau[t] * (np.triu(T[:c, :c]) @ S[:c, t])
    return S


def blocked_reduce(A, B, C):
    n, m = B.shape
    p = C.shape[0]
    E = np.vstack([C, A]).copy()   # C above A: every right update is one product
    R = B.copy()
    kb, ka = min(m, n - 1), max(0, n - m - 1)
    tauB, tauA = np.zeros(max(kb, 1)), np.zeros(max(ka, 1))

    def block(r0, tc0, cs, jb, panels):
        A0 = E.copy()
        V = np.zeros((n, KB))
        T = np.zeros((KB, KB))
        Y = np.zeros((p + n, KB))
        j = 0
        for get_panel, w, wp, pv0, c0, tau in panels:
            S = _panel(get_panel(), r0, n, w, wp, pv0, j, c0, V, T, Y, p, tau)
            AV = A0[:, r0:] @ V[r0:, j:j + wp]                        # Eq. for Y
            Y[:, j:j + wp] = (AV - Y[:, :j] @ S[:j, :]) @ np.triu(T[j:j + wp, j:j + wp])
            j += wp
        if tc0 == cs:
            E[:, cs:] -= Y[:, :jb] @ V[cs:, :jb].T
        else:
            E[:p + r0, tc0:] -= Y[:p + r0, :jb] @ V[tc0:, :jb].T
            E[p + r0:, cs:] -= Y[p + r0:, :jb] @ V[cs:, :jb].T
        if cs < n:
            Wm = V[r0:n, :jb].T @ E[p + r0:p + n, cs:]
            E[p + r0:, cs:] -= V[r0:n, :jb] @ (np.triu(T[:jb, :jb]).T @ Wm)

    if kb > 0:
        block(0, 0, 0, kb, [(lambda: R, m, kb, 0, 0, tauB)])
    b = (KB // m) * m
    for z in range(0, ka, b):
        jb = min(b, ka - z)
        panels = [((lambda c0=z + j, w=min(m, jb - j): E[p:p + n, c0:c0 + w]),
                   min(m, jb - j), min(m, jb - j), z + j + m, z + j, tauA[z + j:z + j + min(m, jb - j)])
                  for j in range(0, jb, m)]
        block(z + m, z + m, z + jb, jb, panels)
    return np.triu(E[p:], -m), np.triu(R), E[:p].copy()


@pytest.mark.parametrize("n,m,p", [(256, 2, 2), (300, 7, 3), (130, 16, 16), (65, 32, 5), (40, 1, 1),
                                   (17, 17, 2), (9, 8, 3), (3, 2, 0), (401, 33, 2), (300, 64, 3)])
def test_blocked_reduction_model_matches_oracle(n, m, p):
    sysr = W.random_system(n, m, p, seed=700 + n + m)
    H, R, Ct = blocked_reduce(sysr.A, sysr.B, sysr.C)
    Ho, Ro, Co, _ = oracle.reduce(sysr.A, sysr.B, sysr.C, want_q=True)
    d = sign_matrix(R, H, Ro, Ho, m)
    assert relerr(H, d[:, None] * Ho * d[None, :]) < 1e-12
    assert relerr(R, d[:, None] * Ro) < 1e-12
    if p:
        assert relerr(Ct, Co * d[None, :]) < 1e-12


# ---------------------------------------------------------------------------
# 2. the digit products, emulated exactly
# ---------------------------------------------------------------------------
def scale_exp(mx):
    """2^E > mx from the exponent field (E = -1022 for zero), per row."""
    _, e = np.frexp(np.asarray(mx, dtype=np.float64))
    return np.where(np.asarray(mx) == 0, -1022, e).astype(np.int64)


def digit_planes(X, E):
    """Eight 7-bit digits of |x| 2^(56 - E) (truncated), with x's sign, as float planes."""
    M = np.floor(np.ldexp(np.abs(X), (56 - E)[:, None]))   # exact: a power-of-two scaling
    return [np.mod(np.floor(np.ldexp(M, -(49 - 7 * l))), 128.0) * np.sign(X) for l in range(8)]


def digit_product(A, B, levels, Ea=None, Eb=None):
    """sum_k A(r, k) B(c, k) as the kernels form it: levels t = a + b < `levels`,
    exact level sums per 128-deep window, exact 64-bit words (levels 0-3, 4-7, 8),
    one rounding per word."""
    Ea = scale_exp(np.abs(A).max(axis=1)) if Ea is None else Ea
    Eb = scale_exp(np.abs(B).max(axis=1)) if Eb is None else Eb
    Pa, Pb = digit_planes(A, Ea), digit_planes(B, Eb)
    words = [0, 0, 0]
    for k0 in range(0, A.shape[1], 128):
        sl = slice(k0, k0 + 128)
        for t in range(levels):
            L = sum(Pa[a][:, sl] @ Pb[t - a][:, sl].T for a in range(max(0, t - 7), min(t, 7) + 1))
            assert np.abs(L).max() < 2 ** 24          # exact in FP32
            w = t // 4
            words[w] = words[w] + L * 2.0 ** (21 - 7 * (t - 4 * w))
    sc = np.ldexp(1.0, Ea[:, None] + Eb[None, :])
    out = 0.0
    for w in (2, 1, 0):
        assert np.abs(words[w]).max() < 2 ** 53 if np.ndim(words[w]) else True
        out = out + words[w] * sc * 2.0 ** (-35 - 28 * w)
    return out


def _err(X, ref):
    return float(np.linalg.norm(X - ref) / np.linalg.norm(ref))


def test_digit_product_nine_levels_is_fp64_class():
    rng = np.random.default_rng(3)
    A, B = rng.standard_normal((40, 640)), rng.standard_normal((30, 640))
    ref = A.astype(np.longdouble) @ B.T.astype(np.longdouble)
    e64 = _err(A @ B.T, ref)
    assert _err(digit_product(A, B, 9), ref) < 4 * max(e64, 2.2e-16)
    assert _err(digit_product(A, B, 8), ref) < 8 * max(e64, 2.2e-16)


def test_nine_levels_matter_for_terms_far_below_the_row_scale():
    # the long products of the reduction: most terms sit far below row max x column max
    rng = np.random.default_rng(4)
    A = rng.standard_normal((32, 1024)) * np.logspace(-4, 0, 1024)[None, :]
    B = rng.standard_normal((16, 1024))
    ref = A.astype(np.longdouble) @ B.T.astype(np.longdouble)
    e8, e9 = _err(digit_product(A, B, 8), ref), _err(digit_product(A, B, 9), ref)
    assert e9 < 2e-15 and e8 > 10 * e9


def test_v_rows_need_their_own_exponent():
    # rows of V across a block's reflectors sit far below the unit pivots
    rng = np.random.default_rng(5)
    Y = rng.standard_normal((64, 128))
    V = rng.standard_normal((48, 128)) * 0.01
    ref = Y.astype(np.longdouble) @ V.T.astype(np.longdouble)
    fixed = digit_product(Y, V, 8, Eb=np.ones(48, dtype=np.int64))
    own = digit_product(Y, V, 8)
    assert _err(own, ref) * 20 < _err(fixed, ref)


def test_words_stay_exact_over_long_k():
    # a window adds below 2^46 to a word; 2^17 windows fit below 2^63
    assert 8 * 128 * 127 ** 2 < 2 ** 24
    assert (2 ** 24) * 2 ** 21 * (1 + 2 ** -7 + 2 ** -14 + 2 ** -21) < 2 ** 46
    assert 2 ** 46 * 2 ** 17 <= 2 ** 63


# ---------------------------------------------------------------------------
# 3. fused-level issue schedules
# ---------------------------------------------------------------------------
def fused_schedule(na, nb_digits, levels, N, zero_plane):
    """(a, b0, c) products of the reduction / sweep form: A digit a against B digits
    b0 .. b0 + c - 1 (c N <= 256), B digit b landing in level a + b; digit index
    nb_digits stands for the zero plane when `zero_plane`."""
    out = []
    for a in range(na):
        nb = levels if a == 0 else min(nb_digits, levels - a)
        if a == 0 and not zero_plane:
            nb = min(nb_digits, levels)
        for b0 in range(0, nb, 256 // N):
            out.append((a, b0, min(256 // N, nb - b0)))
    return out


@pytest.mark.parametrize("name,na,nbd,levels,N,zero", [
    ("reduction rank-b update", 8, 8, 8, 64, False),
    ("reduction A V_s", 8, 8, 9, 16, True),
    ("reduction W", 8, 8, 9, 32, True),
    ("residual, two shifts", 8, 8, 8, 64, False),
    ("sweep Z1 P1", 8, 7, 8, 64, True),
])
def test_fused_schedule_covers_every_pair_once(name, na, nbd, levels, N, zero):
    sched = fused_schedule(na, nbd, levels, N, zero)
    hits = {}
    opened = set()
    for a, b0, c in sched:
        assert c * N <= 256 and (c * N) % 16 == 0
        assert (a + b0 + c) * N <= 512                      # TMEM columns of the levels
        for b in range(b0, b0 + c):
            if b < nbd:
                hits[(a, b)] = hits.get((a, b), 0) + 1
            else:
                assert zero and b == nbd                     # only the zero plane
            if a == 0:
                opened.add(a + b)
    want = {(a, b) for a in range(na) for b in range(nbd) if a + b < levels}
    assert set(hits) == want and all(v == 1 for v in hits.values()), name
    assert opened == set(range(levels)), name               # a = 0 opens every level


@pytest.mark.parametrize("cs,S", [(16, 4), (32, 2)])
def test_fused_z2p2_layout(cs, S):
    # each shift's seven levels side by side: shift l, level t at column 7 cs l + cs t
    cols = set()
    for l in range(S):
        for kd in range(7):
            n = cs * (7 - kd)
            assert n <= 256 and n % 16 == 0
            lo = 7 * cs * l + kd * cs
            cols.update(range(lo, lo + n))
            assert lo + n <= 7 * cs * (l + 1)                # never into the next shift
    assert max(cols) < 512
    # the drain of quarter qt (16 columns): shift (16 qt) // cs, offset (16 qt) % cs
    for qt in range(4):
        l, off = (16 * qt) // cs, (16 * qt) % cs
        assert l < S and off + 16 <= cs
