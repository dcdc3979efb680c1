"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances (floating point, FP64 path): relative error <= 1e-10 against the
oracle for every shift whose estimated kappa_1(H - sigma I) <= 1e6, normwise
backward error <= 1e-12; the reduction matches the oracle's to 1e-12 relative
after fixing the column signs of Q (Householder reflectors are unique up to a
diagonal +-1 when the m-th subdiagonal has no zero entry).
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from paper_1708_06290_gb300 import ssv
from tests.gpu_util import blocks, dev, relerr, shifts_dev, sign_matrix

pytestmark = pytest.mark.gpu

REL_TOL = 1e-10
BWD_TOL = 1e-12
KAPPA_GATE = 1e6


def gpu_system(sysr):
    return ssv.reduce(dev(sysr.A), dev(sysr.B), dev(sysr.C))


@pytest.mark.parametrize("n,m,p", [(256, 2, 2), (300, 7, 3), (130, 16, 16), (65, 32, 5),
                                   (40, 1, 1), (17, 17, 2), (9, 8, 3), (1, 1, 1),
                                   (520, 20, 4), (1100, 16, 16), (700, 1, 3), (401, 33, 2)])
def test_reduce_matches_oracle(n, m, p):
    sysr = W.random_system(n, m, p, seed=700 + n + m)
    h = gpu_system(sysr)
    Hg, Rg, Cg = [t.cpu().numpy() for t in h.reduced()]
    Ho, Ro, Co, Qo = oracle.reduce(sysr.A, sysr.B, sysr.C, want_q=True)
    d = sign_matrix(Rg, Hg, Ro, Ho, m)
    assert relerr(Hg, d[:, None] * Ho * d[None, :]) < 1e-12
    assert relerr(Rg, d[:, None] * Ro) < 1e-12
    assert relerr(Cg, Co * d[None, :]) < 1e-12
    # the GPU's own Q (via apply_q) satisfies Q^T Q = I and Q^T A Q = H
    eye = torch.eye(n, dtype=torch.complex128, device="cuda")
    Qg = h.apply_q(ssv.colmajor(eye)).cpu().numpy().real
    assert np.linalg.norm(Qg.T @ Qg - np.eye(n)) < 50 * n * 2.2e-16
    assert np.linalg.norm(Qg.T @ sysr.A @ Qg - Hg) < 50 * n * 2.2e-16 * np.linalg.norm(sysr.A)


def _check_against_dense(sysr, sig, h, nb=0, modes=("g", "tf", "x"), precision="fp64"):
    X, st = oracle.dense_solve(sysr.A, sysr.B, sig)
    Go = oracle.transfer(sysr.C, X)
    sd = shifts_dev(sig)
    for mode in modes:
        out, status, resid = h.solve(sd, mode=mode, nb=nb, want_resid=True, precision=precision)
        torch.cuda.synchronize()
        res = blocks(out, sysr.m)
        status = status.cpu().numpy()
        resid = resid.cpu().numpy()
        assert (status == 0).all(), (mode, status)
        assert resid.max() <= BWD_TOL, (mode, resid.max())
        for j in range(len(sig)):
            if mode == "g":
                assert relerr(res[j], Go[j]) < REL_TOL, (mode, j)
            elif mode == "tf":
                assert relerr(res[j], -Go[j]) < REL_TOL, (mode, j)
            else:
                assert relerr(res[j], X[j]) < REL_TOL, (mode, j)


def test_small_workload_all_shifts():
    """n = 256, m = p = 2, 64 shifts i*omega, omega = logspace(-2, 2, 64)."""
    sysr, sig = W.workload_small()
    h = gpu_system(sysr)
    _check_against_dense(sysr, sig, h)


@pytest.mark.parametrize("n,m,p,nb", [(517, 3, 2, 64), (200, 8, 4, 16), (333, 16, 3, 64),
                                      (260, 32, 2, 64), (129, 1, 1, 64), (150, 5, 2, 7),
                                      (97, 8, 3, 5), (64, 4, 4, 1), (300, 16, 16, 33)])
def test_ragged_sizes_and_block_widths(n, m, p, nb):
    sysr = W.random_system(n, m, p, seed=900 + n + nb)
    sig = np.concatenate([W.imag_axis_logspace(-2, 2, 5), [-1.7 + 0.4j, -2.6 - 0.2j, 0.3 + 0.1j]])
    h = gpu_system(sysr)
    _check_against_dense(sysr, sig, h, nb=nb)


@pytest.mark.parametrize("n,m", [(12, 12), (13, 12), (20, 19), (6, 1), (2, 1)])
def test_degenerate_shapes(n, m):
    """m = n (no elimination block, dense m x m solve), n = m + 1, tiny n."""
    sysr = W.random_system(n, m, 2, seed=40 + n)
    sig = np.array([0.5j, -1.0 + 0.2j, 3.0j])
    h = gpu_system(sysr)
    _check_against_dense(sysr, sig, h, nb=4)


def test_xhat_matches_oracle_in_reduced_coordinates():
    n, m, p = 410, 6, 3
    sysr = W.random_system(n, m, p, seed=77)
    sig = np.array([0.01j, 0.7j, -2.2 + 0.5j, -1.1 - 0.3j])
    h = gpu_system(sysr)
    Hg, Rg, _ = [t.cpu().numpy() for t in h.reduced()]
    Ho, Ro, Co, _ = oracle.reduce(sysr.A, sysr.B, sysr.C)
    d = sign_matrix(Rg, Hg, Ro, Ho, m)
    Xo, st, cond = oracle.reduced_solve(Ho, Ro, Co, sig, want="xhat", cond=True)
    out, status, _ = h.solve(shifts_dev(sig), mode="xhat")
    Xg = blocks(out, m)
    for j in range(len(sig)):
        assert relerr(Xg[j], d[:, None] * Xo[j]) < REL_TOL


def test_exact_singular_shift_is_reported():
    """A upper triangular, B = [I; 0]: every reflector is the identity, so H = A
    and sigma = A(i, i) makes H - sigma I exactly singular."""
    n, m, p = 40, 3, 2
    rng = np.random.default_rng(5)
    A = np.triu(rng.standard_normal((n, n))) - 2 * np.eye(n)
    B = np.eye(n)[:, :m]
    C = rng.standard_normal((p, n))
    h = ssv.reduce(dev(A), dev(B), dev(C))
    sig = np.array([A[n - 1, n - 1] + 0j, A[17, 17] + 0j, 0.5j])
    _, st_o = oracle.dense_solve(A, B, sig)
    out, status, _ = h.solve(shifts_dev(sig), mode="g")
    status = status.cpu().numpy()
    assert list(st_o) == [1, 1, 0]
    assert status[0] == ssv.SHIFT_SINGULAR and status[1] == ssv.SHIFT_SINGULAR
    assert status[2] == ssv.SHIFT_OK
    g = blocks(out, m)
    assert np.isnan(g[0]).all() and np.isfinite(g[2]).all()


def test_conjugate_symmetry_and_no_shifts():
    sysr = W.random_system(150, 4, 2, seed=81)
    h = gpu_system(sysr)
    s = -0.8 + 1.1j
    out, _, _ = h.solve(shifts_dev([s, np.conj(s)]), mode="x")
    x = blocks(out, 4)
    assert relerr(x[1], np.conj(x[0])) < 1e-13
    out0, st0, _ = h.solve(shifts_dev(np.zeros(0)), mode="g")
    assert out0.shape[1] == 0 and st0.numel() == 0


def test_fp64_workload_sampled():
    """n = 2000, m = p = 8, 1000 shifts i*omega, omega = logspace(-3, 3, 1000):
    all shifts on the GPU, 60 sampled shifts against the tier-2 oracle."""
    sysr, sig = W.workload_fp64()
    h = gpu_system(sysr)
    out, status, resid = h.solve(shifts_dev(sig), mode="g", want_resid=True)
    G = blocks(out, sysr.m)
    assert (status.cpu().numpy() == 0).all()
    assert resid.cpu().numpy().max() <= BWD_TOL
    idx = np.unique(np.linspace(0, len(sig) - 1, 60).astype(int))
    Ho, Ro, Co, _ = oracle.reduce(sysr.A, sysr.B, sysr.C)
    Go, st, cond = oracle.reduced_solve(Ho, Ro, Co, sig[idx], want="g", cond=True)
    for k, j in enumerate(idx):
        if cond[k] <= KAPPA_GATE:
            assert relerr(G[j], Go[k]) < REL_TOL, (j, cond[k])


def test_precision_workload_sampled_fp64():
    """n = 5000, m = p = 16, 2000 shifts on the 50 x 40 grid over [-4,0] x [-2,2]
    (the benchmark's launch), 16 sampled shifts against the tier-2 oracle:
    8 evenly spread, 8 inside the spectral disc |sigma + 2| < 1."""
    sysr, sig = W.workload_precision()
    h = gpu_system(sysr)
    out, status, _ = h.solve(shifts_dev(sig), mode="g")
    G = blocks(out, sysr.m)
    st = status.cpu().numpy()
    inside = np.where(np.abs(sig + 2.0) < 1.0)[0]
    idx = np.concatenate([np.linspace(0, len(sig) - 1, 8).astype(int), inside[:: max(1, len(inside) // 8)][:8]])
    Ho, Ro, Co, _ = oracle.reduce(sysr.A, sysr.B, sysr.C)
    Go, sto, cond = oracle.reduced_solve(Ho, Ro, Co, sig[idx], want="g", cond=True)
    checked = 0
    for k, j in enumerate(idx):
        assert st[j] == sto[k] == 0
        if cond[k] <= KAPPA_GATE:
            assert relerr(G[j], Go[k]) < REL_TOL, (j, cond[k])
            checked += 1
    assert checked >= 8


def test_load_reduced_checkpoint_roundtrip():
    """A handle restored from ssv_get_reduced's output solves exactly like the original;
    it has no Q, so SSV_X is refused."""
    sysr = W.random_system(230, 5, 3, seed=91)
    h = gpu_system(sysr)
    Hg, Rg, Cg = h.reduced()
    h2 = ssv.load_reduced(Hg, Rg, Cg)
    sig = shifts_dev(np.array([0.3j, -1.9 + 0.2j, 2.0j]))
    g1, _, _ = h.solve(sig, mode="g")
    g2, _, _ = h2.solve(sig, mode="g")
    assert torch.equal(g1, g2)
    with pytest.raises(ssv.SsvError):
        h2.solve(sig, mode="x")


# --------------------------------------------------------------------------
# mixed precision: complex64 sweeps + FP64-accurate refinement
# --------------------------------------------------------------------------

def test_mixed_small_workload_all_shifts():
    sysr, sig = W.workload_small()
    h = gpu_system(sysr)
    _check_against_dense(sysr, sig, h, precision="mixed")


@pytest.mark.parametrize("n,m,p,nb", [(517, 3, 2, 64), (200, 8, 4, 16), (333, 16, 3, 64),
                                      (260, 32, 2, 64), (129, 1, 1, 64), (97, 8, 3, 5),
                                      (13, 12, 2, 4), (12, 12, 2, 4)])
def test_mixed_ragged_sizes(n, m, p, nb):
    sysr = W.random_system(n, m, p, seed=900 + n + nb)
    sig = np.concatenate([W.imag_axis_logspace(-2, 2, 5), [-1.7 + 0.4j, -2.6 - 0.2j, 0.3 + 0.1j]])
    h = gpu_system(sysr)
    _check_against_dense(sysr, sig, h, nb=nb, precision="mixed")


def test_mixed_exact_singular_shift_falls_back_and_is_reported():
    n, m, p = 40, 3, 2
    rng = np.random.default_rng(5)
    A = np.triu(rng.standard_normal((n, n))) - 2 * np.eye(n)
    B = np.eye(n)[:, :m]
    C = rng.standard_normal((p, n))
    h = ssv.reduce(dev(A), dev(B), dev(C))
    sig = np.array([A[n - 1, n - 1] + 0j, A[17, 17] + 0j, 0.5j])
    out, status, _ = h.solve(shifts_dev(sig), mode="g", precision="mixed")
    status = status.cpu().numpy()
    assert status[0] == ssv.SHIFT_SINGULAR and status[1] == ssv.SHIFT_SINGULAR
    assert status[2] == ssv.SHIFT_OK


def test_mixed_precision_workload_sampled():
    """n = 5000, m = p = 16, all 2000 grid shifts in mixed precision; every shift
    reaches backward error <= 1e-12 and the sampled shifts match the oracle."""
    sysr, sig = W.workload_precision()
    h = gpu_system(sysr)
    out, status, resid = h.solve(shifts_dev(sig), mode="g", precision="mixed", want_resid=True)
    G = blocks(out, sysr.m)
    st = status.cpu().numpy()
    assert (st == 0).all()
    assert resid.cpu().numpy().max() <= BWD_TOL
    inside = np.where(np.abs(sig + 2.0) < 1.0)[0]
    idx = np.concatenate([np.linspace(0, len(sig) - 1, 8).astype(int), inside[:: max(1, len(inside) // 8)][:8]])
    Ho, Ro, Co, _ = oracle.reduce(sysr.A, sysr.B, sysr.C)
    Go, sto, cond = oracle.reduced_solve(Ho, Ro, Co, sig[idx], want="g", cond=True)
    checked = 0
    for k, j in enumerate(idx):
        if cond[k] <= KAPPA_GATE:
            assert relerr(G[j], Go[k]) < REL_TOL, (j, cond[k])
            checked += 1
    assert checked >= 8


def test_bounded_barrier_times_out_and_device_stays_usable():
    """A grid barrier that one block never reaches gives up after its spin limit:
    the library returns SSV_ETIMEOUT and later work on the device still runs."""
    assert ssv.selftest_barrier(100000) == ssv.SSV_ETIMEOUT
    sysr = W.random_system(60, 2, 2, seed=3)
    h = gpu_system(sysr)
    out, st, _ = h.solve(shifts_dev([0.5j]), mode="g")
    X, _ = oracle.dense_solve(sysr.A, sysr.B, [0.5j])
    assert relerr(blocks(out, 2)[0], oracle.transfer(sysr.C, X)[0]) < REL_TOL


# --------------------------------------------------------------------------
# double-float bulk updates (SSV_DFLOAT): FP64 panels, the updates of the rows
# above each block in FP32 pairs (48-bit class, no refinement)
# --------------------------------------------------------------------------

def test_dfloat_small_workload_all_shifts():
    sysr, sig = W.workload_small()
    h = gpu_system(sysr)
    _check_against_dense(sysr, sig, h, precision="dfloat")


@pytest.mark.parametrize("n,m,p,nb", [(517, 3, 2, 64), (200, 8, 4, 16), (333, 16, 3, 0),
                                      (260, 32, 2, 64), (129, 1, 1, 64), (97, 8, 3, 5), (13, 12, 2, 4)])
def test_dfloat_ragged_sizes(n, m, p, nb):
    sysr = W.random_system(n, m, p, seed=950 + n + nb)
    sig = np.concatenate([W.imag_axis_logspace(-2, 2, 5), [-1.7 + 0.4j, -2.6 - 0.2j, 0.3 + 0.1j]])
    h = gpu_system(sysr)
    _check_against_dense(sysr, sig, h, nb=nb, precision="dfloat")


def test_dfloat_precision_workload_sampled():
    """n = 5000, m = p = 16, all 2000 grid shifts with double-float updates: every
    backward error <= 1e-12 and the sampled shifts match the oracle."""
    sysr, sig = W.workload_precision()
    h = gpu_system(sysr)
    out, status, resid = h.solve(shifts_dev(sig), mode="g", precision="dfloat", want_resid=True)
    G = blocks(out, sysr.m)
    st = status.cpu().numpy()
    assert (st == 0).all()
    assert resid.cpu().numpy().max() <= BWD_TOL
    inside = np.where(np.abs(sig + 2.0) < 1.0)[0]
    idx = np.concatenate([np.linspace(0, len(sig) - 1, 8).astype(int), inside[:: max(1, len(inside) // 8)][:8]])
    Ho, Ro, Co, _ = oracle.reduce(sysr.A, sysr.B, sysr.C)
    Go, sto, cond = oracle.reduced_solve(Ho, Ro, Co, sig[idx], want="g", cond=True)
    checked = 0
    for k, j in enumerate(idx):
        if cond[k] <= KAPPA_GATE:
            assert relerr(G[j], Go[k]) < REL_TOL, (j, cond[k])
            checked += 1
    assert checked >= 8


def test_dfloat_exact_singular_shift_is_reported():
    n, m, p = 40, 3, 2
    rng = np.random.default_rng(5)
    A = np.triu(rng.standard_normal((n, n))) - 2 * np.eye(n)
    B = np.eye(n)[:, :m]
    C = rng.standard_normal((p, n))
    h = ssv.reduce(dev(A), dev(B), dev(C))
    sig = np.array([A[n - 1, n - 1] + 0j, A[17, 17] + 0j, 0.5j])
    out, status, _ = h.solve(shifts_dev(sig), mode="g", precision="dfloat")
    status = status.cpu().numpy()
    assert status[0] == ssv.SHIFT_SINGULAR and status[1] == ssv.SHIFT_SINGULAR
    assert status[2] == ssv.SHIFT_OK


@pytest.mark.parametrize("precision", ["fp64", "dfloat", "mixed"])
def test_nonfinite_input_is_reported_not_hidden(precision):
    """A NaN in A reaches every shift: each status is NONFINITE (or SINGULAR) and no
    output is silently finite-looking garbage with an OK status."""
    sysr = W.random_system(80, 3, 2, seed=44)
    A = sysr.A.copy()
    A[10, 20] = np.nan
    h = ssv.reduce(dev(A), dev(sysr.B), dev(sysr.C))
    out, status, _ = h.solve(shifts_dev([0.5j, -1.0 + 0.2j]), mode="g", precision=precision)
    st = status.cpu().numpy()
    o = out.cpu().numpy()
    assert ((st == ssv.SHIFT_NONFINITE) | (st == ssv.SHIFT_SINGULAR)).all(), st
    assert not np.isfinite(o).all()
