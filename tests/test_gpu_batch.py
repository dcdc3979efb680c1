"""Many systems in one launch (ssv_solve_many / batch plans), CUDA-graph replay, autotuner.

Every system's result in the batched launch must equal its solo ssv_solve result
(the same per-shift arithmetic runs, only the schedule differs), and match the
oracle within the parity tolerance.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from paper_1708_06290_gb300 import ssv
from tests.gpu_util import blocks, dev, relerr, shifts_dev

pytestmark = pytest.mark.gpu

REL_TOL = 1e-10


def small_batch(nsys=12, seed=77):
    """Scaled-down copy of the batching workload: n ~ U{100..900}, m in {1,2,4,8},
    p = m, 8..60 imaginary-axis shifts."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(nsys):
        n = int(rng.integers(100, 901))
        m = int(rng.choice([1, 2, 4, 8]))
        cnt = int(rng.integers(8, 61))
        om = np.exp(rng.uniform(np.log(1e-3), np.log(1e3), cnt))
        out.append((W.random_system(n, m, m, int(rng.integers(0, 2**31 - 1))), 1j * om))
    return out


@pytest.fixture(scope="module")
def batch():
    systems = small_batch()
    handles = [ssv.reduce(dev(s.A), dev(s.B), dev(s.C)) for s, _ in systems]
    shifts = [shifts_dev(sig) for _, sig in systems]
    return systems, handles, shifts


def test_solve_many_equals_solo_solves(batch):
    systems, handles, shifts = batch
    outs, sts = ssv.solve_many(handles, shifts, mode="g")
    for h, x, o, st in zip(handles, shifts, outs, sts):
        ref, st_ref, _ = h.solve(x, mode="g")
        assert torch.equal(st, st_ref)
        assert torch.equal(o, ref)


@pytest.mark.parametrize("mode", ["g", "xhat"])
def test_solve_many_matches_oracle(batch, mode):
    systems, handles, shifts = batch
    outs, sts = ssv.solve_many(handles, shifts, mode=mode)
    torch.cuda.synchronize()
    for k in (0, 5, 11):
        sysk, sig = systems[k]
        X, _ = oracle.dense_solve(sysk.A, sysk.B, sig)
        got = blocks(outs[k], sysk.m)
        assert (sts[k].cpu().numpy() == 0).all()
        if mode == "g":
            ref = oracle.transfer(sysk.C, X)
            for j in range(len(sig)):
                assert relerr(got[j], ref[j]) < REL_TOL
        else:
            Qx = handles[k].apply_q(outs[k])
            xq = blocks(Qx, sysk.m)
            for j in range(len(sig)):
                assert relerr(xq[j], X[j]) < REL_TOL


def test_batch_plan_replays_in_cuda_graph(batch):
    systems, handles, shifts = batch
    bufs = [x.clone() for x in shifts]
    plan = ssv.BatchPlan(handles, bufs, mode="g")
    stream = torch.cuda.Stream()
    plan.run(stream)            # warm-up outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        plan.run(stream)
    rng = np.random.default_rng(3)
    for rep in range(2):
        new = [shifts_dev(1j * np.exp(rng.uniform(-3, 3, x.numel()))) for x in bufs]
        for b, x in zip(bufs, new):
            b.copy_(x)
        g.replay()
        torch.cuda.synchronize()
        for k in (1, 7):
            ref, _, _ = handles[k].solve(new[k], mode="g")
            assert torch.equal(plan.outs[k], ref)
    plan.close()


def test_autotune_picks_a_candidate_and_keeps_results_correct():
    sysr = W.random_system(1200, 8, 8, seed=19)
    h = ssv.reduce(dev(sysr.A), dev(sysr.B), dev(sysr.C))
    sig = W.imag_axis_logspace(-2, 2, 24)
    nb, ms = ssv.autotune(h, shifts_dev(sig), mode="g")
    assert nb in (32, 48, 64, 96, 128) and ms > 0
    out, st, _ = h.solve(shifts_dev(sig[:6]), mode="g")
    X, _ = oracle.dense_solve(sysr.A, sysr.B, sig[:6])
    ref = oracle.transfer(sysr.C, X)
    got = blocks(out, 8)
    for j in range(6):
        assert relerr(got[j], ref[j]) < REL_TOL


def test_solve_many_mixed_precision(batch):
    systems, handles, shifts = batch
    outs, sts = ssv.solve_many(handles[:4], shifts[:4], mode="g", precision="mixed")
    for k in range(4):
        sysk, sig = systems[k]
        X, _ = oracle.dense_solve(sysk.A, sysk.B, sig)
        ref = oracle.transfer(sysk.C, X)
        got = blocks(outs[k], sysk.m)
        assert (sts[k].cpu().numpy() == 0).all()
        for j in range(len(sig)):
            assert relerr(got[j], ref[j]) < REL_TOL


def test_solve_many_dfloat_equals_solo_dfloat_solves(batch):
    """The double-float updates in the many-systems launch give each system the
    same result as its own SSV_DFLOAT solve, and match the oracle."""
    systems, handles, shifts = batch
    outs, sts = ssv.solve_many(handles, shifts, mode="g", precision="dfloat")
    for k, (h, x, o, st) in enumerate(zip(handles, shifts, outs, sts)):
        ref, st_ref, _ = h.solve(x, mode="g", precision="dfloat")
        assert torch.equal(st, st_ref)
        assert torch.equal(o, ref)
    for k in (0, 5, 11):
        sysk, sig = systems[k]
        X, _ = oracle.dense_solve(sysk.A, sysk.B, sig)
        ref = oracle.transfer(sysk.C, X)
        got = blocks(outs[k], sysk.m)
        for j in range(len(sig)):
            assert relerr(got[j], ref[j]) < REL_TOL
