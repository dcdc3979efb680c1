"""Helpers for the GPU parity tests: host <-> device marshalling and comparisons."""
import numpy as np
import torch


def dev(a, dtype=torch.float64):
    """Column-major CUDA copy of a NumPy matrix (or a 1-D CUDA vector)."""
    t = torch.from_numpy(np.ascontiguousarray(a))
    if t.dim() == 2:
        t = t.t().contiguous().t()
    return t.to(device="cuda", dtype=dtype)


def shifts_dev(sig):
    return torch.from_numpy(np.asarray(sig, dtype=np.complex128).reshape(-1).copy()).cuda()


def blocks(out, m):
    """(rows, s*m) CUDA complex tensor -> NumPy (s, rows, m)."""
    a = out.cpu().numpy()
    s = a.shape[1] // m
    return np.stack([a[:, j * m:(j + 1) * m] for j in range(s)]) if s else np.zeros((0, a.shape[0], m))


def relerr(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def sign_matrix(Rg, Hg, Ro, Ho, m):
    """D = diag(+-1) with Q_gpu = Q_oracle D, from diag(R) and the m-th subdiagonal of H."""
    n = Hg.shape[0]
    d = np.ones(n)
    for i in range(min(m, n)):
        if Rg[i, i] * Ro[i, i] < 0:
            d[i] = -1.0
    for i in range(m, n):
        a, b = Hg[i, i - m], Ho[i, i - m]
        s = 1.0 if a * b >= 0 else -1.0
        d[i] = s * d[i - m]
    return d
