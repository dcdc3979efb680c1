"""The tensor-core residual (error-free BF16 digit splitting of H and Xhat, the
36 slice products accumulated exactly in FP32 by tcgen05.mma) behind
ssv_backward_error(SSV_RESID_TENSOR) and the mixed path's certification.

References: the oracle's backward error with its residual in extended
precision (numpy longdouble), from the handle's own H and R; the FP64-pipe method of the
same entry point at the full benchmark size; and closed forms -- perturbing one
entry of an exact-enough solution by delta changes the residual by exactly
delta times a column of H - sigma I.

Tolerances.  The splitting drops terms below 2^-56 of the row / column
scales, so the residual is accurate to about sqrt(n) 2^-54 ||H|| ||Xhat||; in
backward-error units that is below 5e-15 at n <= 5000.  Residuals far above
that level agree to relative 1e-9."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from paper_1708_06290_gb300 import ssv
from tests.gpu_util import dev, shifts_dev

pytestmark = pytest.mark.gpu

ETA_ABS = 5e-15


def eta_ext(H, R, sig, X, m):
    """Backward error per shift from the oracle, residual in numpy longdouble,
    on the structural part of H (rows <= column + m)."""
    Hs = np.triu(H, -m)
    return np.array([oracle.backward_error(Hs, s, X[:, j * m:(j + 1) * m], R, extended=True)
                     for j, s in enumerate(sig)])


def setup(n, m, p, seed, sig):
    sysr = W.random_system(n, m, p, seed=seed)
    h = ssv.reduce(dev(sysr.A), dev(sysr.B), dev(sysr.C))
    sd = shifts_dev(sig)
    X, st, _ = h.solve(sd, mode="xhat")
    assert (st.cpu().numpy() == 0).all()
    H, R, _ = h.reduced()
    return h, sd, X, H.cpu().numpy(), R.cpu().numpy()


SHIFTS = np.array([0.3j, -1.9 + 0.2j, -2.4 - 0.7j, 5.0j, -0.5 + 1.0j])


@pytest.mark.parametrize("n,m", [(300, 3), (129, 1), (257, 16), (96, 8), (40, 16), (513, 5)])
def test_solution_residual_matches_extended_precision(n, m):
    h, sd, X, H, R = setup(n, m, m, 3100 + n + m, SHIFTS)
    eta = h.backward_error(sd, X).cpu().numpy()
    ref = eta_ext(H, R, SHIFTS, X.cpu().numpy(), m)
    assert np.all(np.isfinite(eta))
    assert np.all(np.abs(eta - ref) <= ETA_ABS), (eta, ref)
    assert np.all(eta <= 1e-14)  # FP64 solutions certify


@pytest.mark.parametrize("n,m", [(300, 3), (257, 16), (129, 1)])
def test_perturbed_and_random_xhat_match_extended_precision(n, m):
    h, sd, X, H, R = setup(n, m, m, 3200 + n + m, SHIFTS)
    rng = np.random.default_rng(n + m)
    Xn = X.cpu().numpy()
    # relative perturbations 1e-9 (backward error ~1e-9) and random Xhat (~1)
    for scale in (1e-9, None):
        if scale is None:
            Xp = rng.standard_normal(Xn.shape) + 1j * rng.standard_normal(Xn.shape)
        else:
            Xp = Xn * (1 + scale * (rng.standard_normal(Xn.shape) + 1j * rng.standard_normal(Xn.shape)))
        Xd = torch.from_numpy(Xp).t().contiguous().t().cuda()
        eta = h.backward_error(sd, Xd).cpu().numpy()
        ref = eta_ext(H, R, SHIFTS, Xp, m)
        assert np.all(np.abs(eta - ref) <= 1e-9 * ref + ETA_ABS), (scale, eta, ref)


def test_single_entry_perturbation_closed_form():
    """X' = X + delta e_j e_q^T: E' - E = -(H - sigma I) e_j delta, so with
    delta >> the solution's own residual, ||E'|| = |delta| ||(H - sigma I) e_j||
    up to that residual (here eta ~ 1e-8, checked to ~1e-6 relative)."""
    n, m = 350, 4
    h, sd, X, H, R = setup(n, m, m, 3301, SHIFTS[:3])
    Xn = X.cpu().numpy().copy()
    delta = 1e-4 * (1 + 1j)
    picks = [(0, 5, 0), (1, 200, 3), (2, n - 1, 2)]
    for sh, j, q in picks:
        Xn[j, sh * m + q] += delta
    Xd = torch.from_numpy(Xn).t().contiguous().t().cuda()
    eta = h.backward_error(sd, Xd).cpu().numpy()
    Hs = np.triu(H, -m)
    r2 = float(np.sum(np.triu(R[:m, :m]) ** 2))
    for sh, j, q in picks:
        s = SHIFTS[sh]
        col = Hs[:, j].astype(complex)
        col[j] -= s
        e = abs(delta) * np.linalg.norm(col)
        m2 = np.linalg.norm(Hs - s * np.eye(n)) ** 2
        den = np.sqrt(m2) * np.linalg.norm(Xn[:, sh * m:(sh + 1) * m]) + np.sqrt(r2)
        # up to the unperturbed solution's own residual and the method's floor
        assert abs(eta[sh] - e / den) <= 1e-9 * e / den + ETA_ABS


def test_nonfinite_shift_is_nan_and_others_unaffected():
    n, m = 200, 2
    h, sd, X, H, R = setup(n, m, m, 3401, SHIFTS)
    Xn = X.cpu().numpy().copy()
    Xn[17, 2 * m + 1] = np.nan
    Xd = torch.from_numpy(Xn).t().contiguous().t().cuda()
    eta = h.backward_error(sd, Xd).cpu().numpy()
    assert np.isnan(eta[2])
    ok = np.arange(len(SHIFTS)) != 2
    ref = eta_ext(H, R, SHIFTS[ok], np.concatenate([Xn[:, j * m:(j + 1) * m] for j in np.where(ok)[0]], 1), m)
    assert np.all(np.abs(eta[ok] - ref) <= ETA_ABS)


def test_benchmark_size_against_fp64_method():
    """n = 5000, m = p = 16, sampled grid shifts: tensor and FP64-pipe methods agree."""
    sysr, sig = W.workload_precision()
    h = ssv.reduce(dev(sysr.A), dev(sysr.B), dev(sysr.C))
    idx = np.linspace(0, len(sig) - 1, 24).astype(int)
    sd = shifts_dev(sig[idx])
    X, st, _ = h.solve(sd, mode="xhat", precision="dfloat")
    e_t = h.backward_error(sd, X, method="tensor").cpu().numpy()
    e_f = h.backward_error(sd, X, method="fp64").cpu().numpy()
    assert np.all(np.abs(e_t - e_f) <= ETA_ABS + 1e-6 * e_f), (e_t, e_f)
    assert np.all(e_t <= 1e-13)


def test_tensor_method_rejects_wide_m():
    sysr = W.random_system(80, 20, 3, seed=3501)
    h = ssv.reduce(dev(sysr.A), dev(sysr.B), dev(sysr.C))
    sd = shifts_dev(SHIFTS[:2])
    X, _, _ = h.solve(sd, mode="xhat")
    with pytest.raises(ssv.SsvError):
        h.backward_error(sd, X, method="tensor")
    e = h.backward_error(sd, X, method="fp64").cpu().numpy()
    assert np.all(e <= 1e-14)
