"""Exact rational linear algebra for pinning the oracle on tiny inputs.

Doubles are exact rationals, so (H - lambda I) x = b is solved here without
any rounding by Gaussian elimination over fractions (complex numbers as pairs
of fractions).  Nothing here shares code with the oracle or the CUDA path.
"""
from fractions import Fraction

import numpy as np


class CFrac:
    __slots__ = ("re", "im")

    def __init__(self, re, im=Fraction(0)):
        self.re = Fraction(re)
        self.im = Fraction(im)

    def __add__(self, o):
        return CFrac(self.re + o.re, self.im + o.im)

    def __sub__(self, o):
        return CFrac(self.re - o.re, self.im - o.im)

    def __mul__(self, o):
        return CFrac(self.re * o.re - self.im * o.im, self.re * o.im + self.im * o.re)

    def __truediv__(self, o):
        d = o.re * o.re + o.im * o.im
        return CFrac((self.re * o.re + self.im * o.im) / d, (self.im * o.re - self.re * o.im) / d)

    def is_zero(self):
        return self.re == 0 and self.im == 0

    def to_complex(self):
        return complex(float(self.re), float(self.im))


def exact_solve(H, lam, b, direction=False):
    """Exact solution of (H - lam I) x = b for float64 H, lam, b (complex ok),
    returned as complex128 (rounded once at the end).  direction=True divides
    by the largest real or imaginary magnitude first, so that solutions beyond
    the double range still come back as a (rounded) direction."""
    n = H.shape[0]
    lam = complex(lam)
    M = [[CFrac(Fraction(float(H[i, j]))) for j in range(n)] for i in range(n)]
    for i in range(n):
        M[i][i] = M[i][i] - CFrac(Fraction(lam.real), Fraction(lam.imag))
    bb = np.asarray(b, dtype=np.complex128)
    rhs = [CFrac(Fraction(bb[i].real), Fraction(bb[i].imag)) for i in range(n)]
    for k in range(n):
        p = next(i for i in range(k, n) if not M[i][k].is_zero())
        M[k], M[p] = M[p], M[k]
        rhs[k], rhs[p] = rhs[p], rhs[k]
        for i in range(k + 1, n):
            if M[i][k].is_zero():
                continue
            f = M[i][k] / M[k][k]
            for j in range(k, n):
                M[i][j] = M[i][j] - f * M[k][j]
            rhs[i] = rhs[i] - f * rhs[k]
    x = [None] * n
    for i in range(n - 1, -1, -1):
        s = rhs[i]
        for j in range(i + 1, n):
            s = s - M[i][j] * x[j]
        x[i] = s / M[i][i]
    if direction:
        big = max(max(abs(v.re), abs(v.im)) for v in x)
        if big != 0:
            x = [CFrac(v.re / big, v.im / big) for v in x]
    return np.array([v.to_complex() for v in x])


def read_golden_blocks(path):
    blocks, name, rows = {}, None, []
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line[0].isalpha():
            if name is not None:
                blocks[name] = np.array(rows, dtype=np.float64)
            name, rows = line, []
        else:
            rows.append([float(t) for t in line.split()])
    blocks[name] = np.array(rows, dtype=np.float64)
    return blocks
