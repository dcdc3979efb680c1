"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module only draws random numbers and lays out shift sets; it holds none of
the solver's arithmetic, so both the CUDA path and the CPU oracle may consume
its arrays.  Every array is NumPy float64 / complex128, column-major where it
is a matrix, generated from ``numpy.random.default_rng(seed)`` (PCG64).

The systems follow the random LTI systems of the paper's experiments (Sec. 4,
"random systems (A, B, C)") in the form A = -2 I + G / sqrt(n) with G, B, C
i.i.d. N(0, 1): the spectrum of A fills the disc of radius ~1 around -2.
"""
from dataclasses import dataclass

import numpy as np


@dataclass
class System:
    A: np.ndarray  # n x n float64, column-major
    B: np.ndarray  # n x m float64
    C: np.ndarray  # p x n float64

    @property
    def n(self):
        return self.A.shape[0]

    @property
    def m(self):
        return self.B.shape[1]

    @property
    def p(self):
        return self.C.shape[0]


def random_system(n, m, p, seed):
    """A = -2 I + G / sqrt(n), B, C i.i.d. N(0, 1)."""
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((n, n))
    A = -2.0 * np.eye(n) + G / np.sqrt(n)
    B = rng.standard_normal((n, m))
    C = rng.standard_normal((p, n))
    return System(np.asfortranarray(A), np.asfortranarray(B), np.asfortranarray(C))


def diagonal_system(n, m, p, seed):
    """A = diag(a) with distinct negative real a; B, C i.i.d. N(0, 1)."""
    rng = np.random.default_rng(seed)
    a = -np.sort(rng.uniform(0.5, 4.0, n))
    B = rng.standard_normal((n, m))
    C = rng.standard_normal((p, n))
    return a, System(np.asfortranarray(np.diag(a)), np.asfortranarray(B), np.asfortranarray(C))


def block_diagonal_system(nblk, m, p, seed):
    """A = blockdiag([[alpha_k, beta_k], [-beta_k, alpha_k]]) with poles alpha_k +- i beta_k."""
    rng = np.random.default_rng(seed)
    n = 2 * nblk
    alpha = -rng.uniform(0.5, 3.0, nblk)
    beta = rng.uniform(0.2, 2.0, nblk)
    A = np.zeros((n, n))
    for k in range(nblk):
        A[2 * k, 2 * k] = alpha[k]
        A[2 * k, 2 * k + 1] = beta[k]
        A[2 * k + 1, 2 * k] = -beta[k]
        A[2 * k + 1, 2 * k + 1] = alpha[k]
    B = rng.standard_normal((n, m))
    C = rng.standard_normal((p, n))
    return alpha, beta, System(np.asfortranarray(A), np.asfortranarray(B), np.asfortranarray(C))


def small_rational_system(n, m, seed, den=8):
    """Integer numerators on a common denominator (exact in float64), for exact brute force."""
    rng = np.random.default_rng(seed)
    An = rng.integers(-9, 10, (n, n))
    Bn = rng.integers(-9, 10, (n, m))
    sig = (int(rng.integers(-9, 10)), int(rng.integers(1, 10)))  # (re, im) numerators
    return An, Bn, sig, den


# ----------------------------------------------------------------------------
# Shift sets (imaginary-axis frequency sweeps and a pseudospectrum grid).
# ----------------------------------------------------------------------------

def imag_axis_logspace(lo_exp, hi_exp, count):
    """sigma_j = i omega_j with omega log-spaced 10^lo .. 10^hi inclusive."""
    return 1j * np.logspace(lo_exp, hi_exp, count)


def pseudospectrum_grid(nre=50, nim=40, re=(-4.0, 0.0), im=(-2.0, 2.0)):
    """nre x nim grid over [re] x [im], inclusive ends, real index fastest."""
    xr = np.linspace(re[0], re[1], nre)
    yi = np.linspace(im[0], im[1], nim)
    return (xr[None, :] + 1j * yi[:, None]).reshape(-1)


# ----------------------------------------------------------------------------
# The five workloads.
# ----------------------------------------------------------------------------

SEEDS = {"small": 1001, "fp64": 2002, "precision": 3003, "batching": 4004, "serving": 5005}


def workload_small():
    """n=256, m=p=2, 64 shifts i*omega, omega = logspace(-2, 2, 64)."""
    return random_system(256, 2, 2, SEEDS["small"]), imag_axis_logspace(-2, 2, 64)


def workload_fp64():
    """n=2000, m=p=8, 1000 shifts i*omega, omega = logspace(-3, 3, 1000)."""
    return random_system(2000, 8, 8, SEEDS["fp64"]), imag_axis_logspace(-3, 3, 1000)


def workload_precision():
    """n=5000, m=p=16, 2000 shifts on the 50 x 40 grid over [-4, 0] x [-2, 2]."""
    return random_system(5000, 16, 16, SEEDS["precision"]), pseudospectrum_grid()


def workload_batching(nsys=64, seed=None):
    """nsys systems, n ~ U{200..3000}, m uniform in {1,2,4,8}, p = m, shift counts
    floor(exp(U[ln 16, ln 513))), omega log-uniform in [1e-3, 1e3], sigma = i omega."""
    rng = np.random.default_rng(SEEDS["batching"] if seed is None else seed)
    out = []
    for k in range(nsys):
        n = int(rng.integers(200, 3001))
        m = int(rng.choice([1, 2, 4, 8]))
        cnt = int(np.floor(np.exp(rng.uniform(np.log(16), np.log(513)))))
        om = np.exp(rng.uniform(np.log(1e-3), np.log(1e3), cnt))
        sysk = random_system(n, m, m, int(rng.integers(0, 2**31 - 1)))
        out.append((sysk, 1j * om))
    return out


SERVING_N = (1000, 2000, 4000, 6000, 8000, 10000, 10000, 10000)
SERVING_M = (1, 4, 16)


def workload_serving_systems(scale=1.0):
    """The 8 preloaded systems; system i has m = (1, 4, 16)[i mod 3], p = m."""
    rng = np.random.default_rng(SEEDS["serving"])
    out = []
    for i, n in enumerate(SERVING_N):
        n = max(16, int(round(n * scale)))
        m = SERVING_M[i % 3]
        out.append(random_system(n, m, m, int(rng.integers(0, 2**31 - 1))))
    return out


def serving_requests(count, rate_per_s, nsys=8, seed=None):
    """Poisson arrivals: (t_arrival, system index, shifts) with 1..256 shifts
    (count floor(exp(U[0, ln 257)))), omega log-uniform in [1e-2, 1e2]."""
    rng = np.random.default_rng((SEEDS["serving"] + 1) if seed is None else seed)
    t = 0.0
    reqs = []
    for _ in range(count):
        t += rng.exponential(1.0 / rate_per_s)
        sysi = int(rng.integers(0, nsys))
        cnt = int(np.floor(np.exp(rng.uniform(0.0, np.log(257)))))
        om = np.exp(rng.uniform(np.log(1e-2), np.log(1e2), cnt))
        reqs.append((t, sysi, 1j * om))
    return reqs
