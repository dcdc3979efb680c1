"""CPU oracle for the shifted m-Hessenberg solver (TEST INFRASTRUCTURE ONLY).

This package is the slow, plain, obviously correct reference the CUDA path is
checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline of ``bench.py`` may import it; the product package never does, and the
two share no code.

All arithmetic is IEEE double (complex128), done in ``csrc/ssv_oracle.c``:

* :func:`dense_solve` -- X = (A - sigma I)^{-1} B by LU with partial pivoting
  on the full matrix (the plain definition of the shifted solve, Sec. 1).
* :func:`dense_solve_vec` -- one right-hand side per shift, x = (A - sigma I)^{-1} b
  or x = (A - sigma I)^{-T} c (Sec. 3.3), same LU.
* :func:`tf_norm2` -- ||C (sigma I - A)^{-1} B||_2 per shift (structured pseudospectra,
  Sec. 1), largest singular value of G by the library SVD.
* :func:`reduce` -- controller-Hessenberg form (H, R, Ct[, Q]) of (A, B, C) by
  unblocked Householder reflectors in the order of Algorithm 1 (Sec. 2).
* :func:`reduced_solve` -- Xhat = (H - sigma I)^{-1} R (or G = Ct Xhat) by
  band-limited Gaussian elimination with row pivoting in reduced coordinates,
  plus an optional Hager/Higham estimate of kappa_1(H - sigma I).
* :func:`backward_error` -- the normwise backward error of a given Xhat for
  (H - sigma I) Xhat = R (numpy; optionally with a longdouble residual).

:mod:`oracle.givens` holds the greedy Givens annihilation schedule of
Algorithm 9 (plain Python), pinned by the paper's worked example in
``tests/golden/greedy_givens_m6_nb8.txt``.

Conventions (Sec. 2, Sec. 3): G(sigma) = C X = Ct Xhat with
X = (A - sigma I)^{-1} B; the paper's transfer function is
C (sigma I - A)^{-1} B = -G(sigma).
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

STATUS_OK = 0
STATUS_SINGULAR = 1


def load_library(path):
    """CDLL of an oracle build at `path` with its argument types declared."""
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    I = ctypes.c_int
    lib.ora_dense_solve.argtypes = [I, I, P, I, P, I, I, P, P, P]
    lib.ora_dense_solve_vec.argtypes = [I, P, I, I, P, I, P, I, P, P]
    lib.ora_reduce.argtypes = [I, I, I, P, I, P, I, P, I, P, P, P, P]
    lib.ora_reduced_solve.argtypes = [I, I, I, P, I, P, I, P, I, I, P, I, P, P, P]
    for f in (lib.ora_dense_solve, lib.ora_dense_solve_vec, lib.ora_reduce, lib.ora_reduced_solve):
        f.restype = I
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = load_library(_build.build())
    return _lib


def _f64(a):
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def dense_solve(A, B, sigmas):
    """Return (X, status): X[j] = (A - sigmas[j] I)^{-1} B, complex128 (s, n, m).

    status[j] = 1 where LU met an exactly zero pivot (X[j] is NaN there).
    """
    lib = _load()
    A = _f64(A)
    B = _f64(B)
    if B.ndim == 1:
        B = B[:, None]
    n, m = B.shape
    sig = np.ascontiguousarray(np.asarray(sigmas, dtype=np.complex128).reshape(-1))
    ns = sig.size
    X = np.zeros((ns, m, n), dtype=np.complex128)  # per shift column-major n x m
    st = np.zeros(ns, dtype=np.int32)
    rc = lib.ora_dense_solve(n, m, _ptr(A), n, _ptr(B), n, ns, _ptr(sig), _ptr(X), _ptr(st))
    if rc != 0:
        raise MemoryError("oracle dense_solve failed")
    return np.transpose(X, (0, 2, 1)).copy(), st


def dense_solve_vec(A, rhs, sigmas, trans=False):
    """Return (X, status) with X[j] = (A - sigmas[j] I)^{-1} rhs[j] (trans=False) or
    (A - sigmas[j] I)^{-T} rhs[j] (trans=True, plain transpose); rhs and X (s, n)
    complex128.  status[j] = 1 where LU met an exactly zero pivot (X[j] NaN)."""
    lib = _load()
    A = _f64(A)
    n = A.shape[0]
    sig = np.ascontiguousarray(np.asarray(sigmas, dtype=np.complex128).reshape(-1))
    ns = sig.size
    R = np.ascontiguousarray(np.asarray(rhs, dtype=np.complex128).reshape(ns, n))
    X = np.zeros((ns, n), dtype=np.complex128)
    st = np.zeros(ns, dtype=np.int32)
    rc = lib.ora_dense_solve_vec(n, _ptr(A), n, ns, _ptr(sig), 1 if trans else 0, _ptr(R), n,
                                 _ptr(X), _ptr(st))
    if rc != 0:
        raise MemoryError("oracle dense_solve_vec failed")
    return X, st


def reduce(A, B, C, want_q=False):
    """Controller-Hessenberg form: returns (H, R, Ct, Q or None), all float64.

    H = Q^T A Q is zero below the m-th subdiagonal, R = Q^T B is zero below the
    diagonal (n x m), Ct = C Q (p x n).
    """
    lib = _load()
    A = _f64(A)
    B = _f64(B)
    C = _f64(C)
    n = A.shape[0]
    m = B.shape[1]
    p = C.shape[0]
    H = np.zeros((n, n), order="F")
    R = np.zeros((n, m), order="F")
    Ct = np.zeros((p, n), order="F")
    Q = np.zeros((n, n), order="F") if want_q else None
    rc = lib.ora_reduce(n, m, p, _ptr(A), n, _ptr(B), n, _ptr(C), max(p, 1), _ptr(H), _ptr(R),
                        _ptr(Ct), _ptr(Q))
    if rc != 0:
        raise MemoryError("oracle reduce failed")
    return H, R, Ct, Q


def reduced_solve(H, R, Ct, sigmas, want="xhat", cond=False):
    """Solve (H - sigma I) Xhat = R for every shift in reduced coordinates.

    want="xhat" returns Xhat (s, n, m); want="g" returns G = Ct Xhat (s, p, m).
    Returns (out, status, cond1) with cond1 None unless cond=True.
    """
    lib = _load()
    H = _f64(H)
    R = _f64(R)
    Ct = _f64(Ct)
    n = H.shape[0]
    m = R.shape[1]
    p = Ct.shape[0]
    sig = np.ascontiguousarray(np.asarray(sigmas, dtype=np.complex128).reshape(-1))
    ns = sig.size
    mode = 0 if want == "xhat" else 1
    rows = n if mode == 0 else p
    out = np.zeros((ns, m, rows), dtype=np.complex128)
    st = np.zeros(ns, dtype=np.int32)
    c1 = np.zeros(ns, dtype=np.float64) if cond else None
    rc = lib.ora_reduced_solve(n, m, p, _ptr(H), n, _ptr(R), n, _ptr(Ct), max(p, 1), ns,
                               _ptr(sig), mode, _ptr(out), _ptr(st), _ptr(c1))
    if rc != 0:
        raise MemoryError("oracle reduced_solve failed")
    return np.transpose(out, (0, 2, 1)).copy(), st, c1


def transfer(C, X):
    """G = C X for a stack of solutions X (s, n, m) -> (s, p, m)."""
    return np.einsum("pn,snm->spm", np.asarray(C, dtype=np.float64), X)


def tf_norm2(G):
    """||G(sigma_j)||_2 for a stack G (s, p, m): the quantity whose level sets are the
    structured pseudospectrum of (A, B, C) (Sec. 1, the set of z with
    ||C (zI - A)^{-1} B||_2 >= 1/eps).  Largest singular value by the library SVD."""
    G = np.asarray(G, dtype=np.complex128)
    if G.shape[1] == 0 or G.shape[2] == 0:
        return np.zeros(G.shape[0])
    return np.array([np.linalg.svd(g, compute_uv=False)[0] for g in G])


def backward_error(H, sigma, X, R, extended=False):
    """Normwise backward error of X as a solution of the reduced system
    (H - sigma I) X = R (Sec. 2), the quantity the mixed path certifies:

        ||(H - sigma I) X - R||_F / (||H - sigma I||_F ||X||_F + ||R||_F).

    H real n x n, R n x m, X n x m complex.  With ``extended`` the residual is
    formed in numpy longdouble (real and imaginary parts separately), for
    residuals far below FP64 rounding of the products."""
    H = np.asarray(H, dtype=np.float64)
    n = H.shape[0]
    X = np.asarray(X, dtype=np.complex128)
    R = np.asarray(R)
    M = H.astype(np.complex128) - sigma * np.eye(n)
    if extended:
        Hl = H.astype(np.longdouble)
        xr, xi = X.real.astype(np.longdouble), X.imag.astype(np.longdouble)
        sr, si = np.longdouble(np.real(sigma)), np.longdouble(np.imag(sigma))
        er = Hl @ xr - (sr * xr - si * xi) - np.real(R).astype(np.longdouble)
        ei = Hl @ xi - (sr * xi + si * xr) - np.imag(R).astype(np.longdouble)
        rn = float(np.sqrt(np.sum(er * er + ei * ei)))
    else:
        rn = np.linalg.norm(M @ X - R)
    return rn / (np.linalg.norm(M) * np.linalg.norm(X) + np.linalg.norm(R))
