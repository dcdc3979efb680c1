"""||C (zI - A)^{-1} B||_2 over shifts (structured pseudospectra, Sec. 1):
ssv_tf_norm2 against the oracle (largest singular value of the oracle's G),
in each precision.  Tolerance: relative 1e-10 (the transfer function's)."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from paper_1708_06290_gb300 import ssv
from tests.gpu_util import dev, shifts_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,m,p", [(200, 3, 5), (150, 8, 2), (130, 16, 16), (90, 1, 1), (120, 32, 32),
                                   (60, 20, 3)])
@pytest.mark.parametrize("precision", ["fp64", "dfloat", "mixed"])
def test_tf_norm2_matches_oracle(n, m, p, precision):
    sysr = W.random_system(n, m, p, seed=1700 + n + m + p)
    sig = np.concatenate([W.imag_axis_logspace(-2, 2, 5), [-1.8 + 0.3j, -2.2 - 0.6j, 0.1j]])
    h = ssv.reduce(dev(sysr.A), dev(sysr.B), dev(sysr.C))
    nrm, st = h.tf_norm2(shifts_dev(sig), precision=precision)
    nrm = nrm.cpu().numpy()
    assert (st.cpu().numpy() == 0).all()
    X, _ = oracle.dense_solve(sysr.A, sysr.B, sig)
    ref = oracle.tf_norm2(oracle.transfer(sysr.C, X))
    assert np.all(np.abs(nrm - ref) <= 1e-10 * ref)


def test_pseudospectrum_grid_of_the_benchmark_system():
    """The 50 x 40 grid of the n = 5000, m = p = 16 workload: sampled norms against
    the tier-2 oracle (kappa gate 1e6), and the structured pseudospectrum for
    eps = 1e-2 contains the grid points nearest the spectral disc."""
    sysr, sig = W.workload_precision()
    h = ssv.reduce(dev(sysr.A), dev(sysr.B), dev(sysr.C))
    nrm, st = h.tf_norm2(shifts_dev(sig))
    nrm = nrm.cpu().numpy()
    assert (st.cpu().numpy() == 0).all() and np.all(nrm > 0)
    idx = np.linspace(0, len(sig) - 1, 12).astype(int)
    Ho, Ro, Co, _ = oracle.reduce(sysr.A, sysr.B, sysr.C)
    Go, _, cond = oracle.reduced_solve(Ho, Ro, Co, sig[idx], want="g", cond=True)
    ref = oracle.tf_norm2(Go)
    for k, j in enumerate(idx):
        if cond[k] <= 1e6:
            assert abs(nrm[j] - ref[k]) <= 1e-10 * ref[k]
    inside = np.abs(sig + 2.0) < 0.9
    assert np.median(nrm[inside]) > np.median(nrm[~inside])
