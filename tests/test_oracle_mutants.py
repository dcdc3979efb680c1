"""The oracle's pins catch plausible mistakes planted in a copy of the oracle.

Each mutant is a one-line change to oracle/csrc/ssv_oracle.c (a wrong sign, a
transposed operand, a dropped term, an off-by-one band); it is compiled to a
temporary library and run against pin checks taken from test_oracle_pins.  At
least one check must fail for every mutant, and all pass on the real oracle.
"""
import os
import subprocess

import numpy as np
import pytest

import oracle
import workloads as W
from tests import exact

SRC = os.path.join(os.path.dirname(oracle.__file__), "csrc", "ssv_oracle.c")

MUTANTS = {
    "dense_shift_sign": ("M[i + (size_t)i * n] -= sigma[s];", "M[i + (size_t)i * n] += sigma[s];"),
    "dense_backsub_transposed": ("for (int i = 0; i < k; ++i) x[i] -= a[i + (size_t)k * n] * x[k];",
                                 "for (int i = 0; i < k; ++i) x[i] -= a[k + (size_t)i * n] * x[k];"),
    "reduce_C_not_updated": ("    apply_right(Ct, p, p, r0, len, v, tau);\n", "\n"),
    "reduce_reflector_row": ("    int r0 = j + m, len = n - r0;", "    int r0 = j + m - 1, len = n - r0;"),
    "reduce_B_left_missing": ("    apply_left(H, n, i, len, 0, n, v, tau);                  /* A <- H_i A */", ""),
    "reduced_shift_sign": ("for (int i = 0; i < n; ++i) U[(size_t)i * n + i] -= sigma[s];",
                           "for (int i = 0; i < n; ++i) U[(size_t)i * n + i] += sigma[s];"),
    "reduced_band_short": ("      int last = k + m < n - 1 ? k + m : n - 1;\n      int pr = k;",
                           "      int last = k + m - 1 < n - 1 ? k + m - 1 : n - 1;\n      int pr = k;"),
    "vec_transpose_ignored": ("M[i + (size_t)j * n] = trans ? A[j + (size_t)i * lda] : A[i + (size_t)j * lda];",
                              "M[i + (size_t)j * n] = A[i + (size_t)j * lda];"),
    "vec_rhs_column": ("for (int i = 0; i < n; ++i) xs[i] = rhs[i + (size_t)s * ldr];",
                       "for (int i = 0; i < n; ++i) xs[i] = rhs[i];"),
    "transfer_index": ("acc += Ct[i + (size_t)k * ldc] * X[k + (size_t)j * n];",
                       "acc += Ct[k + (size_t)i * ldc] * X[k + (size_t)j * n];"),
}


def _checks(lib):
    """Pin checks run against an oracle library; returns the list of failures."""
    saved = oracle._lib
    oracle._lib = lib
    fails = []
    try:
        # exact rational dense solve
        An, Bn, sig, den = W.small_rational_system(6, 3, 4)
        X, _ = oracle.dense_solve(An / den, Bn / den, [complex(*sig) / den])
        Xe = np.array([[exact.to_complex(z) for z in row]
                       for row in exact.solve(exact.shifted(An, den, sig), exact.real_matrix(Bn, den))])
        if not np.linalg.norm(X[0] - Xe) <= 1e-12 * np.linalg.norm(Xe):
            fails.append("dense exact")
        # reduction invariants
        sysr = W.random_system(14, 3, 2, seed=5)
        H, R, Ct, Q = oracle.reduce(sysr.A, sysr.B, sysr.C, want_q=True)
        n = 14
        tol = 50 * n * 2.2e-16
        i, j = np.indices((n, n))
        if not ((H[i > j + 3] == 0).all() and np.linalg.norm(Q.T @ Q - np.eye(n)) < tol
                and np.linalg.norm(Q.T @ sysr.A @ Q - H) <= tol * np.linalg.norm(sysr.A)
                and np.linalg.norm(Q.T @ sysr.B - R) <= tol * np.linalg.norm(sysr.B)
                and np.linalg.norm(sysr.C @ Q - Ct) <= tol * np.linalg.norm(sysr.C)):
            fails.append("reduce invariants")
        # exact rational reduced solve on an m-Hessenberg matrix
        rng = np.random.default_rng(3)
        Hn = rng.integers(-9, 10, (8, 8))
        ii, jj = np.indices((8, 8))
        Hn[ii > jj + 3] = 0
        Rn = np.triu(rng.integers(-9, 10, (8, 3)))
        Xh, _, _ = oracle.reduced_solve(Hn / 8, Rn / 8, np.zeros((1, 8)), [complex(3, -5) / 8])
        Xe = np.array([[exact.to_complex(z) for z in row]
                       for row in exact.solve(exact.shifted(Hn, 8, (3, -5)), exact.real_matrix(Rn, 8))])
        if not np.linalg.norm(Xh[0] - Xe) <= 1e-12 * np.linalg.norm(Xe):
            fails.append("reduced exact")
        # coordinate invariance of G
        sysr = W.random_system(30, 3, 2, seed=6)
        sig2 = np.array([0.7j, -1.9 + 0.2j])
        Xd, _ = oracle.dense_solve(sysr.A, sysr.B, sig2)
        H, R, Ct, _ = oracle.reduce(sysr.A, sysr.B, sysr.C)
        G, _, _ = oracle.reduced_solve(H, R, Ct, sig2, want="g")
        Gd = oracle.transfer(sysr.C, Xd)
        if not all(np.linalg.norm(G[k] - Gd[k]) <= 1e-11 * np.linalg.norm(Gd[k]) for k in range(2)):
            fails.append("coordinate invariance")
        # per-shift right-hand sides, both sides, exact rational
        from fractions import Fraction as Fr
        An, Bn, sig, den = W.small_rational_system(5, 2, 8)
        rre, rim = Bn @ np.array([2, -1]), Bn @ np.array([1, 3])
        for trans in (False, True):
            xe = exact.solve(exact.shifted(An.T if trans else An, den, sig),
                             [[(Fr(int(rre[i]), den), Fr(int(rim[i]), den))] for i in range(5)])
            xe = np.array([exact.to_complex(row[0]) for row in xe])
            rhs = np.stack([(rre + 1j * rim) / den, np.zeros(5)])
            Xv, _ = oracle.dense_solve_vec(An / den, rhs, [complex(*sig) / den, 0.5j], trans=trans)
            if not np.linalg.norm(Xv[0] - xe) <= 1e-12 * np.linalg.norm(xe) or np.abs(Xv[1]).max() != 0:
                fails.append("vec exact trans=%d" % trans)
    except Exception as e:  # a mutant may also crash a check
        fails.append("exception: %r" % (e,))
    finally:
        oracle._lib = saved
    return fails


def _build_mutant(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, name
    mutated = src.replace(old, new, 1)
    c = tmp_path / ("%s.c" % name)
    so = tmp_path / ("%s.so" % name)
    c.write_text(mutated)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", str(so), str(c), "-lm"],
                   check=True)
    return oracle.load_library(str(so))


def test_real_oracle_passes_the_checks():
    assert _checks(oracle._load()) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    lib = _build_mutant(tmp_path, name, old, new)
    assert _checks(lib) != [], "mutant %s survived every pin" % name


GIVENS_MUTANTS = {
    "partner_smallest_first": ("for c2 in range(r + delta, c1, -1):", "for c2 in range(c1 + 1, r + delta + 1):"),
    "opens_the_row_below": ("                available.add((r - 1, c))", "                available.add((r + 1, c))"),
    "partners_never_return": ("        ready |= busy\n", "\n"),
    "rows_from_the_top": ("for r in range(n_rows, 0, -1):", "for r in range(1, n_rows + 1):"),
}


@pytest.mark.parametrize("name", sorted(GIVENS_MUTANTS))
def test_givens_schedule_mutant_is_caught(name):
    import types

    import oracle.givens as og
    from tests.test_oracle_pins import _golden_schedule
    src = open(og.__file__).read()
    old, new = GIVENS_MUTANTS[name]
    assert src.count(old) == 1, name
    mod = types.ModuleType("givens_mutant")
    exec(compile(src.replace(old, new), "givens_mutant", "exec"), mod.__dict__)
    gold = [rots for _, rots in _golden_schedule()]
    assert og.greedy_schedule(8, 14) == gold
    try:
        got = mod.greedy_schedule(8, 14)
    except Exception:
        return
    assert got != gold, "mutant %s reproduces the figure" % name


BACKWARD_ERROR_MUTANTS = {
    "shift_sign": ("M = H.astype(np.complex128) - sigma * np.eye(n)", "M = H.astype(np.complex128) + sigma * np.eye(n)"),
    "rhs_dropped": ("rn = np.linalg.norm(M @ X - R)", "rn = np.linalg.norm(M @ X)"),
    "rhs_norm_dropped": ("/ (np.linalg.norm(M) * np.linalg.norm(X) + np.linalg.norm(R))",
                         "/ (np.linalg.norm(M) * np.linalg.norm(X))"),
    "ext_coupling_sign": ("er = Hl @ xr - (sr * xr - si * xi)", "er = Hl @ xr - (sr * xr + si * xi)"),
    "ext_imag_shift": ("ei = Hl @ xi - (sr * xi + si * xr)", "ei = Hl @ xi - (sr * xi)"),
}


def _backward_error_checks(fn):
    """The backward-error pins of test_oracle_pins, as a list of failures."""
    from tests import test_oracle_pins as P
    fails = []
    H = P._triu_band(30, 3, 1)
    R = np.triu(np.random.default_rng(2).standard_normal((30, 3)))
    for ext in (False, True):
        try:
            if abs(fn(H, 0.4j, np.zeros((30, 3), complex), R, extended=ext) - 1.0) > 1e-15:
                fails.append("zero %s" % ext)
        except ZeroDivisionError:
            fails.append("zero %s raised" % ext)
    n, m = 40, 3
    H = P._triu_band(n, m, 4)
    R = np.triu(np.random.default_rng(5).standard_normal((n, m)))
    s = 0.3 - 0.8j
    M = H - s * np.eye(n)
    import scipy.linalg
    X = scipy.linalg.solve(M, R.astype(complex))
    delta = 1e-5 * (2 - 1j)
    X[17, 2] += delta
    den = np.linalg.norm(M) * np.linalg.norm(X) + np.linalg.norm(R)
    want = abs(delta) * np.linalg.norm(M[:, 17]) / den
    for ext in (False, True):
        if abs(fn(H, s, X, R, extended=ext) - want) > 1e-9 * want:
            fails.append("single entry %s" % ext)
    return fails


def _backward_error_variant(old, new):
    import inspect
    src = inspect.getsource(oracle.backward_error)
    assert src.count(old) == 1, old
    ns = {"np": np}
    exec(compile(src.replace(old, new), "backward_error_mutant", "exec"), ns)
    return ns["backward_error"]


def test_real_backward_error_passes_its_checks():
    assert _backward_error_checks(oracle.backward_error) == []


@pytest.mark.parametrize("name", sorted(BACKWARD_ERROR_MUTANTS))
def test_backward_error_mutant_is_caught(name):
    fn = _backward_error_variant(*BACKWARD_ERROR_MUTANTS[name])
    with np.errstate(divide="ignore", invalid="ignore"):  # a mutant may divide by zero
        assert _backward_error_checks(fn) != [], "mutant %s survived every pin" % name
