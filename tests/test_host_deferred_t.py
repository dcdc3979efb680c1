"""X-hat by a backward pass over the stored block transforms (host model of the
multi-column sweep's bookkeeping, same index formulas as the kernel).

The sweep's accumulated column transform T gets, at block step b, the rows
P1_b (the block's fresh columns) while every row set earlier is multiplied by
the step's m x m block P2_b; X-hat = T Y.  The kernel keeps P1_b in T's rows,
parks P2_b in the shift's output rows n - b m .. n - (b-1) m - 1, and forms
  z_B = Y,  X-hat(rows of b) = P1_b z_b,  z_{b-1} = P2_b z_b,
  X-hat(n-m .. n-1) = z_0.
Checked here: the result equals the forward accumulation, the step sequence
recomputed backwards (k_b = n - (b-1) n_b) matches the forward one, every
parked P2 is read before any output write reaches it (n_b >= m), and every
output row is written."""
import numpy as np
import pytest


def forward_and_backward(n, m, nb, seed):
    rng = np.random.default_rng(seed)
    T = np.zeros((n, m))
    T[n - m:, :] = np.eye(m)
    ZT = np.zeros((n, m))
    out = np.full((n, m), np.nan)
    steps = []
    k, b = n, 0
    while k > m:
        b += 1
        nbe = min(nb, k - m)
        j0, lo = k - m - nbe, k - m
        P1, P2 = rng.standard_normal((nbe, m)), rng.standard_normal((m, m))
        T[lo:, :] = T[lo:, :] @ P2
        T[j0:lo, :] = P1
        ZT[j0:lo, :] = P1
        assert n - b * m >= 0, "parking rows exhausted"
        out[n - b * m:n - (b - 1) * m, :] = P2      # parked
        steps.append((k, nbe, j0))
        k -= nbe
    Y = rng.standard_normal((m, m))
    ref = T @ Y
    written = np.zeros(n, bool)
    z = Y.copy()
    for bb in range(b, 0, -1):
        kb = n - (bb - 1) * nb
        nbe_b = min(nb, kb - m)
        j0b = kb - m - nbe_b
        assert (kb, nbe_b, j0b) == steps[bb - 1]
        park = slice(n - bb * m, n - (bb - 1) * m)
        assert not written[park].any(), "a parked P2 was overwritten before it was read"
        p2 = out[park].copy()
        out[j0b:j0b + nbe_b] = ZT[j0b:j0b + nbe_b] @ z
        written[j0b:j0b + nbe_b] = True
        z = p2 @ z
    out[n - m:] = z
    written[n - m:] = True
    return ref, out, written


@pytest.mark.parametrize("n,m,nb", [(300, 3, 64), (129, 1, 64), (257, 16, 16), (96, 8, 64),
                                    (40, 16, 16), (513, 5, 128), (1000, 32, 64), (70, 16, 16),
                                    (33, 16, 16), (17, 16, 16), (200, 32, 32), (5000, 16, 128),
                                    (131, 7, 7), (64, 2, 128)])
def test_backward_pass_equals_forward_accumulation(n, m, nb):
    ref, out, written = forward_and_backward(n, m, nb, seed=n * 7 + m)
    assert written.all()
    assert np.max(np.abs(out - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_parking_needs_nb_at_least_m():
    """With n_b < m the parked blocks can run out of rows or lie under rows
    the backward pass writes first (n_b >= m is sufficient, not necessary):
    the kernel keeps the forward update whenever n_b < m."""
    for n, m, nb in [(200, 16, 8), (400, 32, 20), (300, 10, 9)]:
        with pytest.raises(AssertionError, match="overwritten|exhausted"):
            forward_and_backward(n, m, nb, seed=1)
