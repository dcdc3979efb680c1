"""Pins of the CPU oracle against facts fixed by the mathematics (no GPU).

Each test ties an oracle function to something other than itself:
exact rational brute force, closed forms (diagonal and 2x2-block-diagonal A),
textbook routines for special cases (sigma = 0, m = 1 Hessenberg), block-Krylov
uniqueness of the controller-Hessenberg form, and invariants of Algorithm 1.
"""
import numpy as np
import pytest
import scipy.linalg

import workloads as W
from tests import exact

EPS = np.finfo(np.float64).eps


def relerr(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


# --------------------------------------------------------------------------
# dense_solve: the plain definition X = (A - sigma I)^{-1} B
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n,m,seed", [(1, 1, 1), (3, 2, 2), (5, 1, 3), (6, 3, 4), (8, 2, 5)])
def test_dense_solve_matches_exact_rational(ora, n, m, seed):
    An, Bn, sig, den = W.small_rational_system(n, m, seed)
    A = An / den
    B = Bn / den
    sigma = complex(sig[0], sig[1]) / den
    X, st = ora.dense_solve(A, B, [sigma])
    Xe = exact.solve(exact.shifted(An, den, sig), exact.real_matrix(Bn, den))
    assert Xe is not None and st[0] == 0
    Xe = np.array([[exact.to_complex(z) for z in row] for row in Xe])
    assert relerr(X[0], Xe) < 1e-12


@pytest.mark.parametrize("n,m", [(7, 2), (40, 3)])
def test_dense_solve_diagonal_closed_form(ora, n, m):
    a, sysd = W.diagonal_system(n, m, 2, seed=11)
    sig = W.imag_axis_logspace(-2, 2, 9)
    X, st = ora.dense_solve(sysd.A, sysd.B, sig)
    assert (st == 0).all()
    for j, s in enumerate(sig):
        assert relerr(X[j], sysd.B / (a - s)[:, None]) < 1e-14


def test_dense_solve_sigma_zero_is_linalg_solve(ora):
    sysr = W.random_system(50, 4, 3, seed=12)
    X, st = ora.dense_solve(sysr.A, sysr.B, [0.0])
    assert relerr(X[0], np.linalg.solve(sysr.A, sysr.B)) < 1e-13


def test_dense_solve_conjugate_symmetry(ora):
    sysr = W.random_system(30, 3, 2, seed=13)
    s = -0.7 + 1.3j
    X, _ = ora.dense_solve(sysr.A, sysr.B, [s, np.conj(s)])
    assert relerr(X[1], np.conj(X[0])) < 1e-13


def test_dense_solve_exact_singular_shift(ora):
    a, sysd = W.diagonal_system(6, 2, 2, seed=14)
    X, st = ora.dense_solve(sysd.A, sysd.B, [a[3] + 0j, 1j])
    assert st[0] == ora.STATUS_SINGULAR and np.isnan(X[0]).all()
    assert st[1] == ora.STATUS_OK


# --------------------------------------------------------------------------
# reduce: Algorithm 1 invariants and uniqueness
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n,m,p", [(2, 1, 1), (10, 1, 2), (12, 3, 2), (40, 5, 4), (33, 8, 3),
                                   (7, 7, 2), (9, 8, 1), (65, 16, 16)])
def test_reduce_invariants(ora, n, m, p):
    sysr = W.random_system(n, m, p, seed=100 + n + m)
    H, R, Ct, Q = ora.reduce(sysr.A, sysr.B, sysr.C, want_q=True)
    tol = 50 * n * EPS
    assert np.linalg.norm(Q.T @ Q - np.eye(n)) < tol
    i, j = np.indices((n, n))
    assert (H[i > j + m] == 0).all()                       # stored zeros below m-th subdiagonal
    ib, jb = np.indices((n, m))
    assert (R[ib > jb] == 0).all()                         # R upper triangular
    assert np.linalg.norm(Q.T @ sysr.A @ Q - H) <= tol * np.linalg.norm(sysr.A)
    assert np.linalg.norm(Q.T @ sysr.B - R) <= tol * np.linalg.norm(sysr.B)
    assert np.linalg.norm(sysr.C @ Q - Ct) <= tol * np.linalg.norm(sysr.C)


def _sign_normalize_hess(H, sub):
    """D H D with D = diag(+-1) making the sub-th subdiagonal nonnegative, D[0] = +1."""
    n = H.shape[0]
    d = np.ones(n)
    for i in range(sub, n):
        if H[i, i - sub] * d[i - sub] < 0:
            d[i] = -1.0
    return d[:, None] * H * d[None, :]


def test_reduce_m1_is_textbook_hessenberg(ora):
    """For m = 1 the form is the classic Hessenberg reduction with Q e1 ~ b: by the
    implicit-Q theorem it equals LAPACK's (scipy.linalg.hessenberg) after fixing
    signs, starting from any orthogonal Q0 with first column b / ||b||."""
    n = 24
    sysr = W.random_system(n, 1, 2, seed=21)
    H, R, Ct, Q = ora.reduce(sysr.A, sysr.B, sysr.C, want_q=True)
    Q0, _ = np.linalg.qr(np.hstack([sysr.B, np.eye(n)[:, : n - 1]]))
    H2 = scipy.linalg.hessenberg(Q0.T @ sysr.A @ Q0)
    assert abs(abs(R[0, 0]) - np.linalg.norm(sysr.B)) < 1e-13 * np.linalg.norm(sysr.B)
    Hn = _sign_normalize_hess(H, 1)
    H2n = _sign_normalize_hess(H2, 1)
    # fix the sign of the first basis vector, then everything follows
    assert relerr(Hn, H2n) < 1e-12


@pytest.mark.parametrize("n,m", [(12, 3), (10, 2), (8, 4)])
def test_reduce_spans_block_krylov(ora, n, m):
    """Q(:, 1:k m) is the orthonormal basis of [B, AB, ..., A^{k-1} B] (block-Krylov
    uniqueness of the controller-Hessenberg form), up to column signs."""
    sysr = W.random_system(n, m, 1, seed=31 + n)
    H, R, Ct, Q = ora.reduce(sysr.A, sysr.B, sysr.C, want_q=True)
    blocks = [sysr.B]
    while sum(b.shape[1] for b in blocks) < n:
        blocks.append(sysr.A @ blocks[-1])
    K = np.hstack(blocks)[:, :n]
    QK, RK = np.linalg.qr(K)
    d = np.sign(np.sum(QK * Q, axis=0))
    assert relerr(Q * d[None, :], QK) < 1e-8


# --------------------------------------------------------------------------
# reduced_solve (tier 2) and coordinate invariance
# --------------------------------------------------------------------------

def _random_mhess(n, m, seed, den=8):
    rng = np.random.default_rng(seed)
    Hn = rng.integers(-9, 10, (n, n))
    i, j = np.indices((n, n))
    Hn[i > j + m] = 0
    Rn = rng.integers(-9, 10, (n, m))
    ib, jb = np.indices((n, m))
    Rn[ib > jb] = 0
    return Hn, Rn


@pytest.mark.parametrize("n,m,seed", [(4, 1, 1), (6, 2, 2), (8, 3, 3), (8, 8, 4), (7, 5, 5)])
def test_reduced_solve_matches_exact_rational(ora, n, m, seed):
    den = 8
    Hn, Rn = _random_mhess(n, m, seed, den)
    sig = (3, -5)
    Xh, st, _ = ora.reduced_solve(Hn / den, Rn / den, np.zeros((1, n)), [complex(*sig) / den])
    Xe = exact.solve(exact.shifted(Hn, den, sig), exact.real_matrix(Rn, den))
    Xe = np.array([[exact.to_complex(z) for z in row] for row in Xe])
    assert st[0] == 0
    assert relerr(Xh[0], Xe) < 1e-12


def test_reduced_solve_exact_singular_shift(ora):
    n, m = 6, 2
    rng = np.random.default_rng(5)
    H = np.triu(rng.standard_normal((n, n)))
    R = np.triu(rng.standard_normal((n, m)))
    Xh, st, _ = ora.reduced_solve(H, R, np.ones((1, n)), [H[2, 2] + 0j, 0.5j])
    assert st[0] == ora.STATUS_SINGULAR and st[1] == ora.STATUS_OK


@pytest.mark.parametrize("n,m,p", [(60, 1, 1), (60, 4, 3), (45, 9, 2), (16, 16, 4)])
def test_reduced_solve_equals_dense_in_original_coordinates(ora, n, m, p):
    sysr = W.random_system(n, m, p, seed=200 + n + m)
    sig = np.concatenate([W.imag_axis_logspace(-2, 2, 5), [-2.1 + 0.3j, -1.0 - 0.5j]])
    X, st = ora.dense_solve(sysr.A, sysr.B, sig)
    H, R, Ct, Q = ora.reduce(sysr.A, sysr.B, sysr.C, want_q=True)
    Xh, st2, _ = ora.reduced_solve(H, R, Ct, sig, want="xhat")
    G2, st3, _ = ora.reduced_solve(H, R, Ct, sig, want="g")
    G = ora.transfer(sysr.C, X)
    for j in range(len(sig)):
        assert relerr(Q @ Xh[j], X[j]) < 1e-11
        assert relerr(G2[j], G[j]) < 1e-11


def test_transfer_function_diagonal_residues(ora):
    """G(s) = C (sI - A)^{-1} B = sum_i C(:, i) B(i, :) / (s - a_i) for diagonal A;
    the reduced path's -Ct Xhat must reproduce it."""
    n, m, p = 30, 3, 2
    a, sysd = W.diagonal_system(n, m, p, seed=41)
    H, R, Ct, _ = ora.reduce(sysd.A, sysd.B, sysd.C)
    sig = W.imag_axis_logspace(-2, 2, 11)
    G, st, _ = ora.reduced_solve(H, R, Ct, sig, want="g")
    for j, s in enumerate(sig):
        tf = sum(np.outer(sysd.C[:, i], sysd.B[i, :]) / (s - a[i]) for i in range(n))
        assert relerr(-G[j], tf) < 1e-12


def test_transfer_function_block_diagonal_poles(ora):
    """2x2 blocks [[alpha, beta], [-beta, alpha]] have poles alpha +- i beta with
    eigenvectors [1, +-i]; G(s) = sum over poles of residue / (s - lambda)."""
    nblk, m, p = 12, 2, 3
    alpha, beta, sysb = W.block_diagonal_system(nblk, m, p, seed=42)
    H, R, Ct, _ = ora.reduce(sysb.A, sysb.B, sysb.C)
    sig = np.concatenate([W.imag_axis_logspace(-1, 1, 7), [0.3 - 0.2j]])
    G, st, _ = ora.reduced_solve(H, R, Ct, sig, want="g")
    Gd, _ = ora.dense_solve(sysb.A, sysb.B, sig)
    for j, s in enumerate(sig):
        tf = np.zeros((p, m), dtype=complex)
        for k in range(nblk):
            Ck = sysb.C[:, 2 * k:2 * k + 2]
            Bk = sysb.B[2 * k:2 * k + 2, :]
            for sgn in (+1, -1):
                lam = alpha[k] + sgn * 1j * beta[k]
                v = np.array([1.0, sgn * 1j])            # right eigenvector
                w = np.array([0.5, -sgn * 0.5j])         # left eigenvector, w v = 1
                tf += np.outer(Ck @ v, w @ Bk) / (s - lam)
        assert relerr(-G[j], tf) < 1e-12
        assert relerr(-sysb.C @ Gd[j], tf) < 1e-12


def test_reduced_solve_conjugate_symmetry_and_sigma_zero(ora):
    sysr = W.random_system(40, 3, 2, seed=51)
    H, R, Ct, Q = ora.reduce(sysr.A, sysr.B, sysr.C, want_q=True)
    s = 0.4 + 0.9j
    Xh, _, _ = ora.reduced_solve(H, R, Ct, [s, np.conj(s), 0.0])
    assert relerr(Xh[1], np.conj(Xh[0])) < 1e-13
    assert relerr(Q @ Xh[2], np.linalg.solve(sysr.A, sysr.B)) < 1e-12


def test_hager_condition_estimate_is_tight_lower_bound(ora):
    n, m = 40, 2
    sysr = W.random_system(n, m, 1, seed=61)
    H, R, Ct, _ = ora.reduce(sysr.A, sysr.B, sysr.C)
    sig = np.array([-2.0 + 0.1j, 1j, -1.5 - 0.4j])
    _, _, c1 = ora.reduced_solve(H, R, Ct, sig, cond=True)
    for j, s in enumerate(sig):
        M = H - s * np.eye(n)
        k1 = np.linalg.norm(M, 1) * np.linalg.norm(np.linalg.inv(M), 1)
        assert c1[j] <= k1 * (1 + 1e-10)
        assert c1[j] >= k1 / 10


# --------------------------------------------------------------------------
# dense_solve_vec: a different right-hand side for every shift (Sec. 3.3),
# x = (A - sigma I)^{-1} b and the transposed x = (A - sigma I)^{-T} c
# --------------------------------------------------------------------------

@pytest.mark.parametrize("trans", [False, True])
@pytest.mark.parametrize("n,seed", [(1, 21), (4, 22), (7, 23)])
def test_dense_solve_vec_matches_exact_rational(ora, n, trans, seed):
    from fractions import Fraction as Fr
    An, Bn, sig, den = W.small_rational_system(n, 2, seed)
    rng = np.random.default_rng(seed + 100)
    wr, wi = rng.integers(-5, 6, 2), rng.integers(-5, 6, 2)
    # rhs = B (wr + i wi) / den, exactly representable
    rre = Bn @ wr
    rim = Bn @ wi
    rhs = (rre + 1j * rim) / den
    M = exact.shifted(An.T if trans else An, den, sig)
    b = [[(Fr(int(rre[i]), den), Fr(int(rim[i]), den))] for i in range(n)]
    xe = exact.solve(M, b)
    assert xe is not None
    xe = np.array([exact.to_complex(row[0]) for row in xe])
    X, st = ora.dense_solve_vec(An / den, rhs[None, :], [complex(sig[0], sig[1]) / den], trans=trans)
    assert st[0] == 0
    assert relerr(X[0], xe) < 1e-12


@pytest.mark.parametrize("trans", [False, True])
def test_dense_solve_vec_diagonal_closed_form(ora, trans):
    a, sysd = W.diagonal_system(20, 1, 1, seed=24)
    sig = W.imag_axis_logspace(-1, 1, 5)
    rng = np.random.default_rng(25)
    rhs = rng.standard_normal((5, 20)) + 1j * rng.standard_normal((5, 20))
    X, st = ora.dense_solve_vec(sysd.A, rhs, sig, trans=trans)
    assert (st == 0).all()
    for j, s in enumerate(sig):
        assert relerr(X[j], rhs[j] / (a - s)) < 1e-14


def test_dense_solve_vec_transposed_block_diagonal_closed_form(ora):
    """c-side of the transfer function: x = (A - sigma I)^{-T} C^T chat gives
    x^T B = chat^T C (A - sigma I)^{-1} B = -chat^T G(sigma), with G(s) = C (sI - A)^{-1} B
    in closed form for 2 x 2 blocks [[alpha, beta], [-beta, alpha]]."""
    alpha, beta, sysb = W.block_diagonal_system(6, 2, 3, seed=26)
    sig = np.array([0.4j, -1.1 + 0.7j, 2.5j])
    chat = np.array([1.0 - 0.5j, 0.25j, -2.0])
    rhs = np.tile(sysb.C.T @ chat, (len(sig), 1))
    X, st = ora.dense_solve_vec(sysb.A, rhs, sig, trans=True)
    assert (st == 0).all()
    for j, s in enumerate(sig):
        G = np.zeros((3, 2), dtype=complex)
        for k in range(len(alpha)):
            Ak = np.array([[alpha[k], beta[k]], [-beta[k], alpha[k]]])
            # (sI - Ak)^{-1} = [[s - a, b], [-b, s - a]] / ((s - a)^2 + b^2)
            d = (s - alpha[k]) ** 2 + beta[k] ** 2
            inv = np.array([[s - alpha[k], beta[k]], [-beta[k], s - alpha[k]]]) / d
            sl = slice(2 * k, 2 * k + 2)
            G += sysb.C[:, sl] @ inv @ sysb.B[sl, :]
            assert np.allclose(inv @ (s * np.eye(2) - Ak), np.eye(2))
        assert relerr(X[j] @ sysb.B, -(chat @ G)) < 1e-13


def test_dense_solve_vec_duality_of_the_two_sides(ora):
    """For nonsymmetric A: chat^T C x_b = x_c^T B bhat with x_b = (A - sigma I)^{-1} B bhat
    and x_c = (A - sigma I)^{-T} C^T chat (both are chat^T C (A - sigma I)^{-1} B bhat)."""
    sysr = W.random_system(40, 3, 2, seed=27)
    sig = np.array([0.3j, -2.2 + 0.4j])
    rng = np.random.default_rng(28)
    bhat = rng.standard_normal((2, 3)) + 1j * rng.standard_normal((2, 3))
    chat = rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))
    xb, _ = ora.dense_solve_vec(sysr.A, bhat @ sysr.B.T, sig)
    xc, _ = ora.dense_solve_vec(sysr.A, chat @ sysr.C, sig, trans=True)
    for j in range(2):
        lhs = chat[j] @ (sysr.C @ xb[j])
        rhs = xc[j] @ (sysr.B @ bhat[j])
        assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # and the two sides differ (A is not symmetric): the transpose matters
    xwrong, _ = ora.dense_solve_vec(sysr.A, chat @ sysr.C, sig, trans=False)
    assert abs(xwrong[0] @ (sysr.B @ bhat[0]) - chat[0] @ (sysr.C @ xb[0])) > 1e-6


def test_dense_solve_vec_exact_singular_shift(ora):
    a, sysd = W.diagonal_system(6, 1, 1, seed=29)
    X, st = ora.dense_solve_vec(sysd.A, np.ones((2, 6), dtype=complex), [a[2] + 0j, 0.5j], trans=True)
    assert st[0] == ora.STATUS_SINGULAR and np.isnan(X[0]).all()
    assert st[1] == ora.STATUS_OK


# --------------------------------------------------------------------------
# greedy Givens schedule (Algorithm 9): the paper's worked example and the
# properties any valid schedule must have
# --------------------------------------------------------------------------

def _golden_schedule():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "greedy_givens_m6_nb8.txt")
    steps = []
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        parts = line.split()
        steps.append((int(parts[0]), [tuple(int(v) for v in t.split(",")) for t in parts[1:]]))
    return steps


def test_greedy_schedule_reproduces_the_papers_figure():
    from oracle.givens import greedy_schedule
    gold = _golden_schedule()
    assert [k for k, _ in gold] == list(range(1, 14))
    assert greedy_schedule(8, 14) == [rots for _, rots in gold]


def test_literal_bottom_only_initialisation_does_not_finish():
    """Reading R6: with only the bottom row available at the start, the diagonal
    entries never open up and the schedule stops early (21 of 48 rotations)."""
    from oracle.givens import greedy_schedule
    lit = greedy_schedule(8, 14, initial="bottom_only")
    assert sum(map(len, lit)) < 48


@pytest.mark.parametrize("n_rows,n_cols", [(8, 14), (1, 2), (5, 6), (16, 32), (64, 80), (12, 13), (3, 40)])
def test_greedy_schedule_is_a_valid_rq_order(n_rows, n_cols):
    from oracle.givens import greedy_schedule
    steps = greedy_schedule(n_rows, n_cols)
    d = n_cols - n_rows
    zeroed = {}
    for k, step in enumerate(steps):
        cols = [c for (_, c1, c2) in step for c in (c1, c2)]
        assert len(cols) == len(set(cols)), "rotations of a step share a column"
        for (r, c1, c2) in step:
            assert r <= c1 < c2 <= r + d
            assert (r, c1) not in zeroed and (r, c2) not in zeroed
            if r < n_rows and c1 > r:
                # the entry below must already be zero (it was updated by that rotation)
                assert zeroed.get((r + 1, c1), k) < k
            zeroed[(r, c1)] = k
    assert set(zeroed) == {(r, c) for r in range(1, n_rows + 1) for c in range(r, r + d)}


def test_greedy_schedule_applied_as_givens_rotations_gives_an_rq_factor():
    """Applying the rotations to a random complex trapezoidal block (rows 1..8,
    nonzeros in columns r..14) leaves the first delta columns zero and one
    entry (r, r + delta) on the 'diagonal' of R; the column transform is unitary."""
    from oracle.givens import greedy_schedule
    rng = np.random.default_rng(30)
    nr, ncol = 8, 14
    Z = rng.standard_normal((nr, ncol)) + 1j * rng.standard_normal((nr, ncol))
    Z[np.tril_indices(nr, -1, ncol)] = 0.0
    Z0 = Z.copy()
    Q = np.eye(ncol, dtype=complex)
    for step in greedy_schedule(nr, ncol):
        for (r, c1, c2) in step:
            a, b = Z[r - 1, c1 - 1], Z[r - 1, c2 - 1]
            rho = np.hypot(abs(a), abs(b))
            # [a, b] G = [0, rho] with the unitary G = [[b, conj a], [-a, conj b]] / rho
            G = np.array([[b, np.conj(a)], [-a, np.conj(b)]]) / rho
            Z[:, [c1 - 1, c2 - 1]] = Z[:, [c1 - 1, c2 - 1]] @ G
            Q[:, [c1 - 1, c2 - 1]] = Q[:, [c1 - 1, c2 - 1]] @ G
    d = ncol - nr
    assert np.abs(Z[:, :d]).max() < 1e-12 * np.abs(Z0).max()
    for r in range(nr):
        assert np.abs(Z[r, d:d + r]).max(initial=0.0) < 1e-12 * np.abs(Z0).max()
        assert abs(Z[r, r + d]) > 1e-3
    assert np.linalg.norm(Q.conj().T @ Q - np.eye(ncol)) < 1e-13
    assert np.linalg.norm(Z0 @ Q - Z) < 1e-12 * np.linalg.norm(Z0)


# --------------------------------------------------------------------------
# tf_norm2: ||C (zI - A)^{-1} B||_2, the structured-pseudospectrum function
# --------------------------------------------------------------------------

def test_tf_norm2_single_input_single_output_closed_form(ora):
    """m = p = 1, diagonal A: |sum_i c_i b_i / (z - a_i)|."""
    a, sysd = W.diagonal_system(12, 1, 1, seed=31)
    z = np.array([0.3j, -1.2 + 0.8j, -4.0 - 0.1j])
    X, _ = ora.dense_solve(sysd.A, sysd.B, z)
    nrm = ora.tf_norm2(ora.transfer(sysd.C, X))
    for j, zz in enumerate(z):
        exact = abs(np.sum(sysd.C[0] * sysd.B[:, 0] / (zz - a)))
        assert abs(nrm[j] - exact) <= 1e-13 * exact


def test_tf_norm2_normal_matrix_is_the_inverse_distance_to_the_spectrum(ora):
    """B = C^T = I and A = diag(a): ||(zI - A)^{-1}||_2 = 1 / min_i |z - a_i|, so the
    structured pseudospectrum is the union of the discs of radius eps around a_i."""
    n = 9
    a = -np.linspace(0.5, 3.5, n)
    A = np.diag(a)
    z = np.array([0.2j, -2.0 + 0.05j, -0.9 - 0.4j])
    X, _ = ora.dense_solve(A, np.eye(n), z)
    nrm = ora.tf_norm2(ora.transfer(np.eye(n), X))
    for j, zz in enumerate(z):
        exact = 1.0 / np.min(np.abs(zz - a))
        assert abs(nrm[j] - exact) <= 1e-13 * exact


def test_tf_norm2_single_input_is_the_vector_norm(ora):
    """m = 1: G(z) is a p-vector and its 2-norm is sqrt(sum_k |G_k|^2) in closed form."""
    a, sysd = W.diagonal_system(15, 1, 4, seed=32)
    z = np.array([0.7j, -2.3 + 0.2j])
    X, _ = ora.dense_solve(sysd.A, sysd.B, z)
    nrm = ora.tf_norm2(ora.transfer(sysd.C, X))
    for j, zz in enumerate(z):
        g = sysd.C @ (-sysd.B[:, 0] / (zz - a))  # C (A - zI)^{-1} b
        assert abs(nrm[j] - np.sqrt(np.sum(np.abs(g) ** 2))) <= 1e-13 * nrm[j]


# --------------------------------------------------------------------------
# backward_error: ||(H - sigma I) X - R|| / (||H - sigma I|| ||X|| + ||R||)
# --------------------------------------------------------------------------

def _triu_band(n, m, seed):
    rng = np.random.default_rng(seed)
    return np.triu(rng.standard_normal((n, n)) / np.sqrt(n), -m) - 2.0 * np.eye(n)


@pytest.mark.parametrize("extended", [False, True])
def test_backward_error_of_zero_is_one(ora, extended):
    """X = 0 leaves the whole right-hand side as residual: eta = ||R|| / ||R|| = 1."""
    H = _triu_band(30, 3, 1)
    R = np.triu(np.random.default_rng(2).standard_normal((30, 3)))
    assert ora.backward_error(H, 0.4j, np.zeros((30, 3), complex), R, extended=extended) == pytest.approx(1.0, abs=1e-15)


@pytest.mark.parametrize("extended", [False, True])
def test_backward_error_diagonal_closed_form_solution(ora, extended):
    """Diagonal H: X = R / (d - sigma) row by row solves the system; its backward
    error is at the rounding level of the division."""
    n, m = 50, 4
    d = np.linspace(-3.0, -1.0, n)
    R = np.random.default_rng(3).standard_normal((n, m))
    s = -1.7 + 0.2j
    X = R / (d - s)[:, None]
    assert ora.backward_error(np.diag(d), s, X, R, extended=extended) <= 4 * EPS


@pytest.mark.parametrize("j,q", [(0, 0), (17, 2), (39, 1)])
def test_backward_error_single_entry_perturbation(ora, j, q):
    """X' = X + delta e_j e_q^T for the exact-enough X: the residual is
    -(H - sigma I) e_j delta, so eta = |delta| ||(H - sigma I) e_j|| / den."""
    n, m = 40, 3
    H = _triu_band(n, m, 4)
    R = np.triu(np.random.default_rng(5).standard_normal((n, m)))
    s = 0.3 - 0.8j
    M = H - s * np.eye(n)
    X = scipy.linalg.solve(M, R.astype(complex))
    delta = 1e-5 * (2 - 1j)
    Xp = X.copy()
    Xp[j, q] += delta
    den = np.linalg.norm(M) * np.linalg.norm(Xp) + np.linalg.norm(R)
    want = abs(delta) * np.linalg.norm(M[:, j]) / den
    for ext in (False, True):
        assert ora.backward_error(H, s, Xp, R, extended=ext) == pytest.approx(want, rel=1e-9)


def test_backward_error_extended_agrees_with_fp64_for_large_residuals(ora):
    H = _triu_band(60, 5, 6)
    rng = np.random.default_rng(7)
    R = np.triu(rng.standard_normal((60, 5)))
    X = rng.standard_normal((60, 5)) + 1j * rng.standard_normal((60, 5))
    a = ora.backward_error(H, -1.1 + 0.5j, X, R)
    b = ora.backward_error(H, -1.1 + 0.5j, X, R, extended=True)
    assert a == pytest.approx(b, rel=1e-13)
