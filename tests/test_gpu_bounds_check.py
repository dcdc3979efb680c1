"""The tensor-core sweep and reduction under the bounds-checked debug build (SSV_BOUNDS_CHECK).

compute-sanitizer is not available on the GPU pool, so the library has a debug
variant of its own: every global index of the tensor-core sweep's kernels is
checked against its buffer (an index out of range sets an error bit and every
shift of that solve then reports a non-finite result), its scratch is filled
with NaN before use (a read before the first write poisons the result), and a
canary after the scratch is verified after the last block step.  Small parity
cases (ragged first blocks, single blocks, every shift-group width, repeat
calls, the mixed path) run on that variant in a child process, against the
oracle: a clean pass means no index left its buffer and no scratch was read
before it was written.  The tensor-core reduction's kernels are checked the
same way (an index out of range or a changed canary makes the call fail), on
shapes that reach every blocking case, against the oracle's reduction.
"""
import os
import subprocess
import sys

import pytest

from paper_1708_06290_gb300 import build

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import numpy as np, torch
import oracle, workloads as W
from paper_1708_06290_gb300 import ssv
from tests.gpu_util import blocks, dev, relerr, shifts_dev, sign_matrix
lib = ssv.load()
assert ssv.lib_path() != lib._name, "the debug copy must be the one loaded"
# the tensor-core reduction: an index out of range or a changed canary fails the call
for n, m, p in [(256, 2, 2), (300, 7, 3), (130, 16, 16), (65, 32, 5), (40, 1, 1), (17, 17, 2),
                (9, 8, 3), (3, 2, 0), (401, 33, 2), (300, 64, 3), (700, 16, 5)]:
    sysr = W.random_system(n, m, p, seed=700 + n + m)
    h = ssv.reduce(dev(sysr.A), dev(sysr.B), dev(sysr.C), arith="tensor")
    Hg, Rg, Cg = [t.cpu().numpy() for t in h.reduced()]
    Ho, Ro, Co, _ = oracle.reduce(sysr.A, sysr.B, sysr.C, want_q=True)
    d = sign_matrix(Rg, Hg, Ro, Ho, m)
    assert relerr(Hg, d[:, None] * Ho * d[None, :]) < 1e-12, (n, m, p)
    assert relerr(Rg, d[:, None] * Ro) < 1e-12, (n, m, p)
    if p:
        assert relerr(Cg, Co * d[None, :]) < 1e-12, (n, m, p)
    h.close()
print("bounds-checked tensor-core reduction ok")
cases = [(256, 2, 2, 9), (700, 8, 5, 13), (1000, 16, 16, 5), (17, 16, 4, 3), (144, 16, 3, 4),
         (145, 1, 1, 40), (300, 12, 2, 5), (513, 5, 3, 7), (390, 3, 16, 9)]
for n, m, p, k in cases:
    sysr = W.random_system(n, m, p, seed=2100 + n + m)
    sig = np.concatenate([W.imag_axis_logspace(-2, 2, k), [-1.7 + 0.4j, 0.3 + 0.1j]])
    X, _ = oracle.dense_solve(sysr.A, sysr.B, sig)
    Go = oracle.transfer(sysr.C, X)
    h = ssv.reduce(dev(sysr.A), dev(sysr.B), dev(sysr.C))
    sd = shifts_dev(sig)
    for rep in range(2):
        for prec in ("split", "mixed"):
            out, st, _ = h.solve(sd, mode="g", precision=prec)
            torch.cuda.synchronize()
            st = st.cpu().numpy()
            assert (st == 0).all(), (n, m, p, prec, st)
            G = blocks(out, m)
            worst = max(relerr(G[j], Go[j]) for j in range(len(sig)))
            assert worst < 1e-10, (n, m, p, prec, worst)
        xo, xs, _ = h.solve(sd, mode="xhat", precision="split")
        torch.cuda.synchronize()
        assert (xs.cpu().numpy() == 0).all(), (n, m, p, "xhat")
    h.close()
print("bounds-checked sweep ok:", len(cases), "shapes")
'''


def test_tensor_core_sweep_passes_the_bounds_checked_build():
    lib = build.build(variant="check")
    env = dict(os.environ, SSV_LIBRARY=lib, PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "bounds-checked sweep ok" in r.stdout
    assert "bounds-checked tensor-core reduction ok" in r.stdout
