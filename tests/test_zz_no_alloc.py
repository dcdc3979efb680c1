"""The allocation-free solve entry point, called through the C ABI.

ssv_solve_noalloc is for callers that cannot allocate device memory when they
solve (an outside allocator or framework owns device memory during their step,
a device-memory budget fixed in advance, or a latency-critical loop): it runs
the FP64 solve on a fixed scratch array inside the library.  Its results must
match ssv_solve's, and two calls in a row must both be right although they
share that array.  This file is collected last, so a failure here does not hide
the outcome of the other GPU tests.
"""
import ctypes

import numpy as np
import pytest
import torch

import workloads as W
from paper_1708_06290_gb300 import ssv
from tests.gpu_util import blocks, dev, relerr, shifts_dev

pytestmark = pytest.mark.gpu

REL_TOL = 1e-10


def _noalloc(h, shifts, mode, ldo_rows, nb=0, panel="householder"):
    lib = ssv.load()
    s = shifts.numel()
    out = torch.full((s * h.m, ldo_rows), float("nan"), dtype=torch.complex128, device="cuda").t()
    status = torch.full((s,), -7, dtype=torch.int32, device="cuda")
    o = ssv.opts("fp64", mode, nb=nb, panel=panel)
    rc = lib.ssv_solve_noalloc(h.ptr, s, ctypes.c_void_p(shifts.data_ptr()), ctypes.byref(o),
                               ctypes.c_void_p(out.data_ptr()), ldo_rows,
                               ctypes.c_void_p(status.data_ptr()),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, out, status


@pytest.mark.parametrize("mode", ["g", "xhat"])
def test_noalloc_matches_solve_on_two_calls_in_a_row(mode):
    sysr = W.random_system(700, 8, 5, seed=1234)
    h = ssv.reduce(dev(sysr.A), dev(sysr.B), dev(sysr.C))
    rows = sysr.p if mode == "g" else sysr.n
    first = shifts_dev(np.concatenate([W.imag_axis_logspace(-2, 2, 40), [-1.8 + 0.3j, -2.4 - 0.1j]]))
    second = shifts_dev(W.pseudospectrum_grid(7, 5))
    for sig in (first, second):
        rc, out_na, st_na = _noalloc(h, sig, mode, rows)
        assert rc == ssv.SSV_OK, ssv.strerror(rc)
        ref, st_ref, _ = h.solve(sig, mode=mode)
        torch.cuda.synchronize()
        assert torch.equal(st_na, st_ref)
        a, b = blocks(out_na, sysr.m), blocks(ref, sysr.m)
        for j in range(sig.numel()):
            assert relerr(a[j], b[j]) < REL_TOL, j


def test_noalloc_rejects_problems_beyond_its_scratch():
    """One shift's window needs 16 (p + n) m bytes; with n = 1000, m = 32 and
    p = 131100 that is just over the 64 MiB array, so the call must refuse with
    SSV_ESCRATCH (and leave the outputs untouched) while ssv_solve still works."""
    n, m, p = 1000, 32, 131100
    assert 16 * (p + n) * m > (64 << 20)
    rng = np.random.default_rng(8)
    Hs = np.triu(rng.standard_normal((n, n)), -m) - 2.0 * np.eye(n)
    Rs = np.triu(rng.standard_normal((n, m)))
    Ct = torch.zeros((n, p), dtype=torch.float64, device="cuda").t()   # p x n, column-major
    h = ssv.load_reduced(dev(Hs), dev(Rs), Ct)
    rc, out, status = _noalloc(h, shifts_dev([0.5j, 1.5j]), "g", p)
    assert rc == ssv.SSV_ESCRATCH
    assert bool(torch.isnan(out).all()) and bool((status == -7).all())
    ref, st_ref, _ = h.solve(shifts_dev([0.5j]), mode="g")
    assert int(st_ref[0]) == ssv.SHIFT_OK
    # m > 32 is outside the supported range of both solves
    sysr = W.random_system(100, 33, 2, seed=5)
    h2 = ssv.reduce(dev(sysr.A), dev(sysr.B), dev(sysr.C))
    rc, _, _ = _noalloc(h2, shifts_dev([0.5j]), "g", sysr.p)
    assert rc == ssv.SSV_ENOTSUP


def test_noalloc_refuses_unsupported_options():
    sysr = W.random_system(60, 2, 2, seed=6)
    h = ssv.reduce(dev(sysr.A), dev(sysr.B), dev(sysr.C))
    rc, _, _ = _noalloc(h, shifts_dev([0.5j]), "x", sysr.n)
    assert rc == ssv.SSV_ENOTSUP
    # only the Householder panel runs on the fixed scratch; the Givens panel is refused
    rc, _, _ = _noalloc(h, shifts_dev([0.5j]), "g", sysr.p, panel="givens")
    assert rc == ssv.SSV_ENOTSUP
    lib = ssv.load()
    assert b"64 MiB" in lib.ssv_strerror(ssv.SSV_ESCRATCH)


@pytest.mark.parametrize("mode", ["tf", "xhat"])
def test_noalloc_with_fewer_slots_than_blocks(mode, ora):
    """n = 1000, m = p = 32: one shift's window takes 16 (p + n) m = 528 KB (plus
    512 KB for X-hat), so the 64 MiB array holds 127 (or 64) windows, fewer
    than the 300 shifts and fewer than the thread blocks ssv_solve would use;
    each block then solves many shifts in turn through its own window.  The
    results must equal ssv_solve's bit for bit (same kernel, same n_b), on two
    calls in a row, and the oracle's on a few shifts."""
    sysr = W.random_system(1000, 32, 32, seed=4321)
    h = ssv.reduce(dev(sysr.A), dev(sysr.B), dev(sysr.C))
    slot = 16 * (sysr.p + sysr.n) * sysr.m + (16 * sysr.n * sysr.m if mode == "xhat" else 0)
    assert (64 << 20) // slot < 300
    rows = sysr.p if mode == "tf" else sysr.n
    Ct = h.reduced()[2].cpu().numpy()
    Ho, Ro, Co, _ = ora.reduce(sysr.A, sysr.B, sysr.C)
    pick = [0, 77, 150, 299]
    for sig in (W.imag_axis_logspace(-2, 2, 300), W.pseudospectrum_grid(20, 15)):
        sd = shifts_dev(sig)
        rc, out_na, st_na = _noalloc(h, sd, mode, rows)
        assert rc == ssv.SSV_OK, ssv.strerror(rc)
        ref, st_ref, _ = h.solve(sd, mode=mode)
        torch.cuda.synchronize()
        assert torch.equal(st_na, st_ref)
        assert torch.equal(out_na, ref)
        a = blocks(out_na, sysr.m)
        Go, sto, k1 = ora.reduced_solve(Ho, Ro, Co, sig[pick], want="g", cond=True)
        for k, j in enumerate(pick):
            if sto[k] != 0 or k1[k] > 1e6:
                continue
            # G = Ct X-hat is coordinate-free, so X-hat is checked through it
            g = -a[j] if mode == "tf" else Ct @ a[j]
            assert relerr(g, Go[k]) < REL_TOL, j
