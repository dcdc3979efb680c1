"""The C ABI library loads and exports every symbol include/ssv.h declares (no GPU).

Only calls that touch no device are made here: option defaults, error strings,
argument validation that fails before any CUDA call, and size queries.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1708_06290_gb300 import build, ssv

    build.build()
    return ssv.load()


def declared_symbols():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if fn.endswith(".h"):
            txt = open(os.path.join(inc, fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names.update(re.findall(r"\b(ssv_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert "ssv_reduce" in names and "ssv_solve" in names
    for nm in names:
        assert hasattr(lib, nm), nm


def test_binding_covers_every_export(lib):
    from paper_1708_06290_gb300 import ssv

    assert set(declared_symbols()) <= set(ssv.EXPORTS)


def test_strerror_and_defaults(lib):
    from paper_1708_06290_gb300 import ssv

    assert lib.ssv_strerror(0) == b"success"
    assert b"invalid" in lib.ssv_strerror(-1)
    assert lib.ssv_strerror(12345) == b"unknown error code"
    o = ssv.Opts()
    lib.ssv_default_opts(ctypes.byref(o))
    assert o.precision == ssv.FP64 and o.mode == ssv.G and o.max_refine == 8 and o.tol == 1e-13
    assert o.first == 2   # SSV_FIRST_TENSOR
    # the C struct and the ctypes mirror agree in size (ssv_opts is passed by pointer)
    assert ctypes.sizeof(ssv.Opts) == 32


def test_argument_validation_needs_no_gpu(lib):
    from paper_1708_06290_gb300 import ssv

    h = ctypes.c_void_p()
    P = ctypes.c_void_p
    fake = P(16)
    # n < 1, m > n, negative p, short leading dimension, NULL output handle
    assert lib.ssv_reduce(0, 1, 1, fake, 1, fake, 1, fake, 1, None, ctypes.byref(h)) == ssv.SSV_EINVAL
    assert lib.ssv_reduce(4, 5, 1, fake, 4, fake, 4, fake, 1, None, ctypes.byref(h)) == ssv.SSV_EINVAL
    assert lib.ssv_reduce(4, 2, -1, fake, 4, fake, 4, fake, 1, None, ctypes.byref(h)) == ssv.SSV_EINVAL
    assert lib.ssv_reduce(4, 2, 1, fake, 3, fake, 4, fake, 1, None, ctypes.byref(h)) == ssv.SSV_EINVAL
    assert lib.ssv_reduce(4, 2, 1, fake, 4, fake, 4, fake, 1, None, None) == ssv.SSV_EINVAL
    # the arithmetic of the reduction's products: FP64 pipe or tensor cores, nothing else
    for arith in (-1, 2, 7):
        assert lib.ssv_reduce_arith(4, 2, 1, fake, 4, fake, 4, fake, 1, arith, None,
                                    ctypes.byref(h)) == ssv.SSV_EINVAL
    assert lib.ssv_reduce_arith(0, 1, 1, fake, 1, fake, 1, fake, 1, ssv.REDUCE_TENSOR, None,
                                ctypes.byref(h)) == ssv.SSV_EINVAL
    assert lib.ssv_reduce_arith(4, 2, 1, fake, 3, fake, 4, fake, 1, ssv.REDUCE_TENSOR, None,
                                ctypes.byref(h)) == ssv.SSV_EINVAL
    assert lib.ssv_solve(None, 1, fake, None, fake, 4, None, None, None) == ssv.SSV_EINVAL
    assert lib.ssv_apply_q(None, 1, fake, 4, fake, 4, None) == ssv.SSV_EINVAL
    bad = ssv.Opts()
    lib.ssv_default_opts(ctypes.byref(bad))
    bad.mode = 9
    b = ctypes.c_size_t()
    assert lib.ssv_footprint(10, 2, 2, 5, ctypes.byref(bad), ctypes.byref(b)) == ssv.SSV_EINVAL
    bad.mode = 0
    bad.first = 7
    assert lib.ssv_footprint(10, 2, 2, 5, ctypes.byref(bad), ctypes.byref(b)) == ssv.SSV_EINVAL
    assert lib.ssv_dims(None, None, None, None) == ssv.SSV_EINVAL
    lib.ssv_destroy(None)


def test_size_queries(lib):
    b = ctypes.c_size_t()
    assert lib.ssv_handle_bytes(100, 4, 3, ctypes.byref(b)) == 0
    assert b.value >= 8 * (100 * 100 + 100 * 4 + 3 * 100)
    assert lib.ssv_footprint(100, 4, 3, 10, None, ctypes.byref(b)) == 0
    assert b.value >= 16 * (103 * 4)
