"""Transposed systems (Sec. 3.3): ssv_solve_trans against the oracle.

x_l = (A - sigma_l I)^{-T} C^T chat_l is checked against the plain dense solve
of the transposed system (oracle.dense_solve_vec, trans=True); the duality
chat^T C x_b = x_c^T B bhat ties it to ssv_solve_rhs; at the benchmark size the
c-side values x_c^T B = -chat^T G(sigma) are checked against the tier-2 oracle.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from paper_1708_06290_gb300 import ssv
from tests.gpu_util import dev, relerr, shifts_dev

pytestmark = pytest.mark.gpu

REL_TOL = 1e-10
KAPPA_GATE = 1e6


def _cplx(rows, s, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((rows, s)) + 1j * rng.standard_normal((rows, s))


def _dev_c(b):
    return torch.from_numpy(np.asfortranarray(b)).t().contiguous().t().cuda()


@pytest.mark.parametrize("n,m,p,nb", [(300, 4, 3, 0), (97, 3, 2, 5), (130, 16, 16, 0), (64, 1, 1, 0),
                                      (45, 8, 2, 16), (260, 32, 4, 64)])
def test_solve_trans_matches_dense_oracle(n, m, p, nb):
    sysr = W.random_system(n, m, p, seed=1400 + n + m)
    sig = np.concatenate([W.imag_axis_logspace(-2, 2, 6), [-2.4 + 0.3j, 0.2 - 0.1j]])
    ch = _cplx(p, len(sig), seed=n)
    h = ssv.reduce(dev(sysr.A), dev(sysr.B), dev(sysr.C))
    xo, st = oracle.dense_solve_vec(sysr.A, (sysr.C.T @ ch).T, sig, trans=True)
    assert (st == 0).all()
    sd, cd = shifts_dev(sig), _dev_c(ch)
    x, status = h.solve_trans(sd, cd, mode="x", nb=nb)
    xt, _ = h.solve_trans(sd, cd, mode="xhat", nb=nb)
    torch.cuda.synchronize()
    assert (status.cpu().numpy() == 0).all()
    x = x.cpu().numpy()
    qx = h.apply_q(xt).cpu().numpy()
    for j in range(len(sig)):
        assert relerr(x[:, j], xo[j]) < REL_TOL, j
        assert relerr(qx[:, j], xo[j]) < REL_TOL, j


def test_duality_with_the_per_shift_rhs_solve():
    sysr = W.random_system(400, 6, 5, seed=1501)
    sig = W.imag_axis_logspace(-1, 1.5, 9)
    bh, ch = _cplx(6, 9, 1), _cplx(5, 9, 2)
    h = ssv.reduce(dev(sysr.A), dev(sysr.B), dev(sysr.C))
    sd = shifts_dev(sig)
    xb, _ = h.solve_rhs(sd, _dev_c(bh), mode="x")
    xc, _ = h.solve_trans(sd, _dev_c(ch), mode="x")
    xb, xc = xb.cpu().numpy(), xc.cpu().numpy()
    for j in range(9):
        lhs = ch[:, j] @ (sysr.C @ xb[:, j])
        rhs = xc[:, j] @ (sysr.B @ bh[:, j])
        assert abs(lhs - rhs) <= 1e-11 * abs(lhs)


def test_exact_singular_shift_is_reported():
    n, m, p = 30, 2, 2
    rng = np.random.default_rng(19)
    A = np.triu(rng.standard_normal((n, n))) - 2 * np.eye(n)
    B = np.eye(n)[:, :m]
    C = rng.standard_normal((p, n))
    h = ssv.reduce(dev(A), dev(B), dev(C))
    sig = np.array([A[5, 5] + 0j, 0.4j])
    _, st = h.solve_trans(shifts_dev(sig), _dev_c(_cplx(p, 2, 3)), mode="x")
    st = st.cpu().numpy()
    assert st[0] == ssv.SHIFT_SINGULAR and st[1] == ssv.SHIFT_OK


def test_precision_workload_sampled_c_side_values():
    """n = 5000, m = p = 16, the 2000 grid shifts: x_l^T B = -chat_l^T G(sigma_l)
    against the tier-2 oracle's transfer function (kappa gate 1e6)."""
    sysr, sig = W.workload_precision()
    ch = _cplx(sysr.p, len(sig), seed=5)
    h = ssv.reduce(dev(sysr.A), dev(sysr.B), dev(sysr.C))
    x, st = h.solve_trans(shifts_dev(sig), _dev_c(ch), mode="x")
    assert (st.cpu().numpy() == 0).all()
    x = x.cpu().numpy()
    idx = np.linspace(0, len(sig) - 1, 10).astype(int)
    Ho, Ro, Co, _ = oracle.reduce(sysr.A, sysr.B, sysr.C)
    Go, sto, cond = oracle.reduced_solve(Ho, Ro, Co, sig[idx], want="g", cond=True)
    checked = 0
    for k, j in enumerate(idx):
        if cond[k] <= KAPPA_GATE:
            # x^T B = chat^T C (A - sigma I)^{-1} B = chat^T G with G = C X
            assert relerr(x[:, j] @ sysr.B, ch[:, j] @ Go[k]) < REL_TOL, (j, cond[k])
            checked += 1
    assert checked >= 5


def test_unsupported_modes_are_refused():
    sysr = W.random_system(20, 2, 1, seed=4)
    h = ssv.reduce(dev(sysr.A), dev(sysr.B), dev(sysr.C))
    with pytest.raises(ssv.SsvError):
        h.solve_trans(shifts_dev([0.5j]), _dev_c(np.ones((1, 1), dtype=complex)), mode="g")
