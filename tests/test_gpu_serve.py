"""Continuous-batching server: results in the mix equal results alone; admission by memory."""
import numpy as np
import pytest
import torch

import workloads as W
from paper_1708_06290_gb300 import ssv
from paper_1708_06290_gb300.serve import Server, make_requests
from tests.gpu_util import dev, shifts_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def handles():
    systems = W.workload_serving_systems(scale=0.08)   # n = 80 .. 800, m = (1, 4, 16)[i % 3]
    return [ssv.reduce(dev(s.A), dev(s.B), dev(s.C)) for s in systems]


def _requests(count, rate, seed):
    reqs = make_requests(W.serving_requests(count, rate, seed=seed))
    for r in reqs:
        r.shifts = r.shifts[:48]
    return reqs


@pytest.mark.parametrize("precision", ["fp64", "dfloat", "mixed"])
def test_each_result_is_the_same_alone_and_in_the_mix(handles, precision):
    reqs = _requests(30, 400.0, seed=11)
    srv = Server(handles, slots=4, mem_budget=2 << 30, max_batch_shifts=96, precision=precision)
    stats = srv.run(reqs, realtime=False)
    assert stats["requests"] == len(reqs)
    assert stats["max_inflight_batches"] >= 2          # micro-batches overlapped on the device
    for r in reqs:
        assert (r.status.cpu().numpy() == 0).all()
        alone, st, _ = handles[r.system].solve(shifts_dev(r.shifts), mode="g", precision=precision)
        torch.cuda.synchronize()
        if precision in ("fp64", "dfloat"):
            assert torch.equal(r.result, alone)
        else:
            a, b = r.result.cpu().numpy(), alone.cpu().numpy()
            assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)


def test_realtime_poisson_latencies_and_memory_admission(handles):
    reqs = _requests(40, 200.0, seed=12)
    fp = [Server(handles).footprint(r) for r in reqs]
    budget = int(3 * max(fp))
    srv = Server(handles, slots=4, mem_budget=budget, max_batch_shifts=128)
    stats = srv.run(reqs, realtime=True)
    assert stats["requests"] == len(reqs)
    assert stats["max_inflight_bytes"] <= budget
    assert stats["p99_ms"] >= stats["p50_ms"] > 0
    assert all(r.t_done >= r.t_arrival for r in reqs)


def test_request_larger_than_budget_is_refused(handles):
    reqs = _requests(3, 100.0, seed=13)
    with pytest.raises(ValueError):
        Server(handles, mem_budget=1024).run(reqs, realtime=False)
