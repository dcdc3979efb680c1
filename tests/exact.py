"""Exact Gaussian-rational linear algebra for brute-force pins (n <= 8).

Complex numbers are pairs (re, im) of ``fractions.Fraction``.  Gauss-Jordan
elimination with any nonzero pivot gives the exact solution, so a float64
oracle result can be compared against the true value of the rational problem.
"""
from fractions import Fraction as Fr


def cadd(a, b):
    return (a[0] + b[0], a[1] + b[1])


def csub(a, b):
    return (a[0] - b[0], a[1] - b[1])


def cmul(a, b):
    return (a[0] * b[0] - a[1] * b[1], a[0] * b[1] + a[1] * b[0])


def cdiv(a, b):
    d = b[0] * b[0] + b[1] * b[1]
    return ((a[0] * b[0] + a[1] * b[1]) / d, (a[1] * b[0] - a[0] * b[1]) / d)


def czero(a):
    return a[0] == 0 and a[1] == 0


def solve(M, Bm):
    """Solve M X = Bm exactly; M n x n, Bm n x k, lists of complex pairs.

    Returns X as a list of rows, or None when M is singular.
    """
    n = len(M)
    k = len(Bm[0])
    aug = [list(M[i]) + list(Bm[i]) for i in range(n)]
    for c in range(n):
        piv = next((r for r in range(c, n) if not czero(aug[r][c])), None)
        if piv is None:
            return None
        aug[c], aug[piv] = aug[piv], aug[c]
        d = aug[c][c]
        aug[c] = [cdiv(x, d) for x in aug[c]]
        for r in range(n):
            if r != c and not czero(aug[r][c]):
                f = aug[r][c]
                aug[r] = [csub(x, cmul(f, y)) for x, y in zip(aug[r], aug[c])]
    return [row[n:n + k] for row in aug]


def to_complex(z):
    return complex(float(z[0]), float(z[1]))


def shifted(An, den, sig_num):
    """Exact M = A - sigma I with A = An/den, sigma = (re + i im)/den."""
    n = len(An)
    M = [[(Fr(int(An[i][j]), den), Fr(0)) for j in range(n)] for i in range(n)]
    for i in range(n):
        M[i][i] = csub(M[i][i], (Fr(sig_num[0], den), Fr(sig_num[1], den)))
    return M


def real_matrix(Bn, den):
    return [[(Fr(int(x), den), Fr(0)) for x in row] for row in Bn]
