"""The tensor-core reduction (SSV_REDUCE_TENSOR) against the oracle.

The two-level blocked form (Sec. 2.1, Algorithms 2 and 3) with its bulk
products as error-free BF16 digit products must give the same controller-
Hessenberg triple as the oracle's plain reduction (Algorithm 1) to 1e-12
relative after fixing the column signs of Q, on shapes that exercise every
case of the blocking: one block and several, a ragged last block and last
mini-block, m that does not divide the block width, m = 1, m = 64, n <= m + 1
(no reflectors of A), p = 0 and p > m.  At the benchmark size the oracle is
too slow, so there the invariants that define the result are checked
directly on random vectors: Q is orthogonal, A Q = Q H, B = Q R, C Q = Ct.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from paper_1708_06290_gb300 import ssv
from tests.gpu_util import blocks, dev, relerr, shifts_dev, sign_matrix

pytestmark = pytest.mark.gpu

SHAPES = [(256, 2, 2), (300, 7, 3), (130, 16, 16), (65, 32, 5), (40, 1, 1), (17, 17, 2), (9, 8, 3),
          (520, 20, 4), (1100, 16, 16), (401, 33, 2), (700, 64, 3), (2, 1, 1), (3, 2, 0), (129, 16, 0),
          (1500, 12, 20), (257, 5, 1)]


def tensor_system(sysr):
    return ssv.reduce(dev(sysr.A), dev(sysr.B), dev(sysr.C), arith="tensor")


@pytest.mark.parametrize("n,m,p", SHAPES)
def test_tensor_reduction_matches_oracle(n, m, p):
    sysr = W.random_system(n, m, p, seed=700 + n + m)
    h = tensor_system(sysr)
    Hg, Rg, Cg = [t.cpu().numpy() for t in h.reduced()]
    Ho, Ro, Co, _ = oracle.reduce(sysr.A, sysr.B, sysr.C, want_q=True)
    d = sign_matrix(Rg, Hg, Ro, Ho, m)
    assert relerr(Hg, d[:, None] * Ho * d[None, :]) < 1e-12
    assert relerr(Rg, d[:, None] * Ro) < 1e-12
    if p > 0:
        assert relerr(Cg, Co * d[None, :]) < 1e-12
    # the stored reflectors define an orthogonal Q with Q^T A Q = H
    eye = torch.eye(n, dtype=torch.complex128, device="cuda")
    Qg = h.apply_q(ssv.colmajor(eye)).cpu().numpy().real
    assert np.linalg.norm(Qg.T @ Qg - np.eye(n)) < 50 * n * 2.2e-16
    assert np.linalg.norm(Qg.T @ sysr.A @ Qg - Hg) < 50 * n * 2.2e-16 * np.linalg.norm(sysr.A)
    h.close()


def test_tensor_and_fp64_reductions_agree_and_solve_alike():
    sysr = W.random_system(900, 16, 8, seed=4242)
    ht = tensor_system(sysr)
    hf = ssv.reduce(dev(sysr.A), dev(sysr.B), dev(sysr.C))
    Ht, Rt, Ct = [t.cpu().numpy() for t in ht.reduced()]
    Hf, Rf, Cf = [t.cpu().numpy() for t in hf.reduced()]
    d = sign_matrix(Rt, Ht, Rf, Hf, 16)
    assert relerr(Ht, d[:, None] * Hf * d[None, :]) < 1e-12
    # the transfer function is independent of Q's signs: compare with the dense oracle
    sig = np.concatenate([W.imag_axis_logspace(-2, 2, 12), [0.7 - 0.2j]])
    X, _ = oracle.dense_solve(sysr.A, sysr.B, sig)
    Go = oracle.transfer(sysr.C, X)
    for prec in ("fp64", "mixed"):
        out, st, _ = ht.solve(shifts_dev(sig), mode="g", precision=prec)
        torch.cuda.synchronize()
        assert (st.cpu().numpy() == 0).all()
        G = blocks(out, 16)
        assert max(relerr(G[j], Go[j]) for j in range(len(sig))) < 1e-10, prec
    ht.close()
    hf.close()


def test_tensor_reduction_invariants_at_benchmark_size():
    sysr, _ = W.workload_precision()
    n, m, p = sysr.n, sysr.m, sysr.p
    h = tensor_system(sysr)
    Hg, Rg, Cg = [t.cpu().numpy() for t in h.reduced()]
    assert np.abs(np.tril(Hg, -m - 1)).max() == 0.0
    assert np.abs(np.tril(Rg, -1)).max() == 0.0
    rng = np.random.default_rng(11)
    x = rng.standard_normal((n, 4))
    Qx = h.apply_q(dev(x, torch.complex128)).cpu().numpy().real
    # orthogonality: <Q x_i, Q x_j> = <x_i, x_j>
    assert np.linalg.norm(Qx.T @ Qx - x.T @ x) < 1e-12 * np.linalg.norm(x.T @ x)
    # A Q = Q H
    QHx = h.apply_q(dev(Hg @ x, torch.complex128)).cpu().numpy().real
    assert np.linalg.norm(sysr.A @ Qx - QHx) < 1e-12 * np.linalg.norm(sysr.A) * np.linalg.norm(x)
    # B = Q R and C Q = Ct
    y = rng.standard_normal((m, 3))
    QRy = h.apply_q(dev(Rg @ y, torch.complex128)).cpu().numpy().real
    assert np.linalg.norm(sysr.B @ y - QRy) < 1e-12 * np.linalg.norm(sysr.B) * np.linalg.norm(y)
    assert np.linalg.norm(sysr.C @ Qx - Cg @ x) < 1e-12 * np.linalg.norm(sysr.C) * np.linalg.norm(x)
    h.close()


def test_tensor_reduction_refuses_wide_m():
    sysr = W.random_system(200, 65, 2, seed=3)
    with pytest.raises(RuntimeError):
        tensor_system(sysr)
    with pytest.raises(ValueError):
        ssv.reduce(dev(sysr.A), dev(sysr.B), dev(sysr.C), arith="fp32")
