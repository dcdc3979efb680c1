"""The sweep with the trailing update on the tensor cores (SSV_SPLIT, and the
mixed path's tensor-core first solve), through the C ABI, against the oracle.

Same tolerances as the FP64 path: relative error <= 1e-10 against the oracle's
dense solve, normwise backward error <= 1e-12 (from the FP64 residual).  The
shapes span several 128-row tiles of H, several shift groups with a ragged
last group, a partial first block (n - m not a multiple of 128), single-block
systems, and every column stride of a shift group (2m rounded up to 2 .. 32).
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from paper_1708_06290_gb300 import ssv
from tests.gpu_util import blocks, dev, relerr, shifts_dev
from tests.test_gpu_parity import _check_against_dense

pytestmark = pytest.mark.gpu

REL_TOL = 1e-10


def _sig(k):
    return np.concatenate([W.imag_axis_logspace(-2, 2, k), [-1.7 + 0.4j, -2.6 - 0.2j, 0.3 + 0.1j]])


@pytest.mark.parametrize("n,m,p,k", [(256, 2, 2, 61), (700, 8, 5, 10), (1000, 16, 16, 6),
                                     (17, 16, 4, 3), (144, 16, 3, 4), (145, 1, 1, 40),
                                     (300, 12, 2, 5), (513, 5, 3, 7), (390, 3, 16, 9)])
def test_split_matches_dense_oracle(n, m, p, k):
    sysr = W.random_system(n, m, p, seed=1300 + n + m)
    h = ssv.reduce(dev(sysr.A), dev(sysr.B), dev(sysr.C))
    _check_against_dense(sysr, _sig(k), h, precision="split")


def test_split_agrees_with_fp64_and_dfloat_on_the_fp64_workload():
    """n = 2000, m = p = 8, 200 of the 1000 imaginary-axis shifts: the three
    sweeps agree to well within the parity tolerance."""
    sysr, sig = W.workload_fp64()
    sig = sig[::5]
    h = ssv.reduce(dev(sysr.A), dev(sysr.B), dev(sysr.C))
    sd = shifts_dev(sig)
    g64, st64, _ = h.solve(sd, mode="g")
    gsp, stsp, rsp = h.solve(sd, mode="g", precision="split", want_resid=True)
    gdf, _, _ = h.solve(sd, mode="g", precision="dfloat")
    torch.cuda.synchronize()
    assert (stsp.cpu().numpy() == 0).all() and (st64.cpu().numpy() == 0).all()
    assert float(rsp.max()) <= 1e-13
    a, b, c = blocks(gsp, 8), blocks(g64, 8), blocks(gdf, 8)
    assert max(relerr(a[j], b[j]) for j in range(len(sig))) < 1e-11
    assert max(relerr(c[j], b[j]) for j in range(len(sig))) < 1e-11


def test_split_xhat_in_reduced_coordinates_and_repeat_calls():
    """X-hat mode (the mixed path's first solve) on 301 shifts (151 groups of 2,
    the last one half empty), twice in a row: both calls identical, and the
    backward error of every shift from the FP64 residual <= 1e-13."""
    sysr = W.random_system(900, 16, 16, seed=4242)
    h = ssv.reduce(dev(sysr.A), dev(sysr.B), dev(sysr.C))
    sig = np.concatenate([W.pseudospectrum_grid(15, 20), [0.5j]])
    sd = shifts_dev(sig)
    x1, s1, r1 = h.solve(sd, mode="xhat", precision="split", want_resid=True)
    x2, s2, _ = h.solve(sd, mode="xhat", precision="split")
    torch.cuda.synchronize()
    assert torch.equal(x1, x2) and torch.equal(s1, s2)
    assert (s1.cpu().numpy() == 0).all()
    assert float(r1.max()) <= 1e-13, float(r1.max())
    # and against the oracle's tier-2 solve through G = Ct X-hat (coordinate-free)
    Ct = h.reduced()[2].cpu().numpy()
    Ho, Ro, Co, _ = oracle.reduce(sysr.A, sysr.B, sysr.C)
    pick = np.arange(0, len(sig), 23)
    Go, _, k1 = oracle.reduced_solve(Ho, Ro, Co, sig[pick], want="g", cond=True)
    X = blocks(x1, 16)
    for t, j in enumerate(pick):
        if k1[t] <= 1e6:
            assert relerr(Ct @ X[j], Go[t]) < REL_TOL, (j, k1[t])


def test_split_exact_singular_shift_and_nonfinite_input():
    n, m, p = 300, 3, 2
    rng = np.random.default_rng(5)
    A = np.triu(rng.standard_normal((n, n))) - 2 * np.eye(n)
    B = np.eye(n)[:, :m]
    C = rng.standard_normal((p, n))
    h = ssv.reduce(dev(A), dev(B), dev(C))
    sig = np.array([A[n - 1, n - 1] + 0j, A[150, 150] + 0j, 0.5j])
    out, st, _ = h.solve(shifts_dev(sig), mode="g", precision="split")
    torch.cuda.synchronize()
    st = st.cpu().numpy()
    assert st[0] == ssv.SHIFT_SINGULAR and st[1] == ssv.SHIFT_SINGULAR and st[2] == ssv.SHIFT_OK
    assert np.isnan(blocks(out, m)[0]).all()
    A2 = W.random_system(200, 4, 2, seed=3).A.copy()
    A2[50, 60] = np.nan
    sysr = W.random_system(200, 4, 2, seed=3)
    h2 = ssv.reduce(dev(A2), dev(sysr.B), dev(sysr.C))
    _, st2, _ = h2.solve(shifts_dev([0.3j, 1.0j]), mode="g", precision="split")
    torch.cuda.synchronize()
    assert (st2.cpu().numpy() != ssv.SHIFT_OK).all()


def test_split_refuses_what_it_does_not_cover():
    sysr = W.random_system(100, 17, 2, seed=8)
    h = ssv.reduce(dev(sysr.A), dev(sysr.B), dev(sysr.C))
    with pytest.raises(ssv.SsvError):
        h.solve(shifts_dev([0.5j]), mode="g", precision="split")       # m > 16
    sysr = W.random_system(12, 12, 2, seed=9)
    h = ssv.reduce(dev(sysr.A), dev(sysr.B), dev(sysr.C))
    with pytest.raises(ssv.SsvError):
        h.solve(shifts_dev([0.5j]), mode="g", precision="split")       # n = m


@pytest.mark.parametrize("n,m,p", [(700, 8, 5), (1000, 16, 16), (145, 1, 1)])
def test_mixed_with_tensor_first_solve(n, m, p):
    sysr = W.random_system(n, m, p, seed=1500 + n)
    h = ssv.reduce(dev(sysr.A), dev(sysr.B), dev(sysr.C))
    sig = _sig(6)
    X, st0 = oracle.dense_solve(sysr.A, sysr.B, sig)
    Go = oracle.transfer(sysr.C, X)
    ssv.refine_counts(reset=True)
    out, st, resid = h.solve(shifts_dev(sig), mode="g", precision="mixed", first="tensor",
                             want_resid=True)
    torch.cuda.synchronize()
    corr, resolves = ssv.refine_counts(reset=True)
    assert (st.cpu().numpy() == 0).all()
    assert float(resid.max()) <= 1e-12
    assert resolves == 0 and corr <= len(sig)   # the first solve all but certifies
    G = blocks(out, m)
    for j in range(len(sig)):
        assert relerr(G[j], Go[j]) < REL_TOL, j
