"""The Givens panel (Sec. 3.2, greedy schedule of Algorithm 9) against the
oracle, and against the default Householder panel.  Tolerances as in
test_gpu_parity (relative 1e-10, backward error 1e-12)."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from paper_1708_06290_gb300 import ssv
from tests.gpu_util import blocks, dev, relerr, shifts_dev

pytestmark = pytest.mark.gpu

REL_TOL = 1e-10
BWD_TOL = 1e-12


@pytest.mark.parametrize("n,m,p,nb", [(256, 2, 2, 0), (300, 7, 3, 32), (130, 16, 16, 0), (97, 3, 2, 5),
                                      (40, 8, 2, 32), (260, 32, 4, 16), (64, 1, 1, 0), (13, 12, 2, 4)])
def test_givens_panel_matches_dense_oracle(n, m, p, nb):
    sysr = W.random_system(n, m, p, seed=1600 + n + m)
    sig = np.concatenate([W.imag_axis_logspace(-2, 2, 6), [-1.7 + 0.4j, 0.3 + 0.1j]])
    h = ssv.reduce(dev(sysr.A), dev(sysr.B), dev(sysr.C))
    X, st = oracle.dense_solve(sysr.A, sysr.B, sig)
    Go = oracle.transfer(sysr.C, X)
    sd = shifts_dev(sig)
    g, status, resid = h.solve(sd, mode="g", nb=nb, want_resid=True, panel="givens")
    x, _, _ = h.solve(sd, mode="x", nb=nb, panel="givens")
    torch.cuda.synchronize()
    assert (status.cpu().numpy() == 0).all()
    assert resid.cpu().numpy().max() <= BWD_TOL
    g, x = blocks(g, m), blocks(x, m)
    for j in range(len(sig)):
        assert relerr(g[j], Go[j]) < REL_TOL, j
        assert relerr(x[j], X[j]) < REL_TOL, j


def test_givens_and_householder_panels_agree_at_the_benchmark_size():
    """n = 5000, m = p = 16: 64 grid shifts solved with both panels agree to
    1e-10 wherever the oracle's kappa_1 estimate is <= 1e6."""
    sysr, sig = W.workload_precision()
    sig = sig[np.linspace(0, len(sig) - 1, 64).astype(int)]
    h = ssv.reduce(dev(sysr.A), dev(sysr.B), dev(sysr.C))
    sd = shifts_dev(sig)
    gh, sth, _ = h.solve(sd, mode="g")
    gg, stg, rg = h.solve(sd, mode="g", panel="givens", want_resid=True)
    assert (stg.cpu().numpy() == 0).all() and (sth.cpu().numpy() == 0).all()
    assert rg.cpu().numpy().max() <= BWD_TOL
    Ho, Ro, Co, _ = oracle.reduce(sysr.A, sysr.B, sysr.C)
    _, _, cond = oracle.reduced_solve(Ho, Ro, Co, sig, want="g", cond=True)
    a, b = blocks(gh, 16), blocks(gg, 16)
    checked = 0
    for j in range(len(sig)):
        if cond[j] <= 1e6:
            assert relerr(b[j], a[j]) < REL_TOL
            checked += 1
    assert checked >= 32


def test_givens_panel_limits_are_refused():
    sysr = W.random_system(100, 4, 2, seed=5)
    h = ssv.reduce(dev(sysr.A), dev(sysr.B), dev(sysr.C))
    with pytest.raises(ssv.SsvError):
        h.solve(shifts_dev([0.5j]), mode="g", nb=64, panel="givens")
    with pytest.raises(ssv.SsvError):
        h.solve(shifts_dev([0.5j]), mode="g", precision="mixed", panel="givens")
