"""Test matrices with known eigenvalues.

All matrices are float64 numpy arrays in Fortran (column-major) order, the
layout the C ABI takes.
"""
import numpy as np
import scipy.linalg

from .rng import normal, uniform

# stream ids, so that different uses of one seed draw independent numbers
S_HAAR, S_UPPER, S_PERM, S_EIG, S_JIT, S_B, S_SHIFT, S_IMAG, S_GRADE = range(1, 10)


def haar_orthogonal(n, seed):
    """Haar-distributed orthogonal Q: QR of a Gaussian matrix with the signs of
    R's diagonal moved into Q."""
    G = normal(seed, S_HAAR, n * n).reshape(n, n, order="F")
    Q, R = np.linalg.qr(G)
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return np.asfortranarray(Q * d[None, :])


def quasi_triangular(n, real_eigs, cplx_ab, seed):
    """Quasi-triangular T: 1x1 blocks carry the real eigenvalues, 2x2 blocks
    [[a, b], [-b, a]] carry a +- ib, all other strictly upper entries N(0,1).
    The block order is a seeded random permutation.  Returns (T, diag_order)
    where diag_order lists, for each block in order, ('r', value) or
    ('c', a, b)."""
    real_eigs = list(np.asarray(real_eigs, dtype=np.float64))
    cplx_ab = [tuple(map(float, p)) for p in cplx_ab]
    nb = len(real_eigs) + len(cplx_ab)
    assert len(real_eigs) + 2 * len(cplx_ab) == n
    blocks = [("r", v) for v in real_eigs] + [("c", a, b) for a, b in cplx_ab]
    perm = np.argsort(uniform(seed, S_PERM, nb), kind="stable")
    blocks = [blocks[p] for p in perm]
    T = np.triu(normal(seed, S_UPPER, n * n).reshape(n, n, order="F"), 1)
    i = 0
    for blk in blocks:
        if blk[0] == "r":
            T[i, i] = blk[1]
            i += 1
        else:
            a, b = blk[1], blk[2]
            T[i, i] = a
            T[i, i + 1] = b
            T[i + 1, i] = -b
            T[i + 1, i + 1] = a
            i += 2
    return np.asfortranarray(T), blocks


def hessenberg_reduce(A):
    """LAPACK Hessenberg reduction A = Q0 H Q0^T (the precursor step of the
    method).  Entries below the subdiagonal are exactly zero."""
    H, Q = scipy.linalg.hessenberg(np.asarray(A, dtype=np.float64), calc_q=True)
    H = np.triu(H, -1)
    return np.asfortranarray(H), np.asfortranarray(Q)


def paper_r2_q2(n):
    """R2 and Q2 of the paper's second test problem (Sec. 5.2):
    r2(i,i) = n-i+1, r2(i,j>i) = -n; q2(i,j) = -1 for i-1 = j or (i,j) = (1,n)."""
    R = np.triu(np.full((n, n), -float(n)), 1) + np.diag(np.arange(n, 0, -1, dtype=np.float64))
    Q = np.zeros((n, n))
    for i in range(1, n):
        Q[i, i - 1] = -1.0
    Q[0, n - 1] = -1.0
    return np.asfortranarray(R), np.asfortranarray(Q)


def paper_h2(n, gamma=2.0):
    """The "bad" system H2 = R2 Q2 + gamma I (Sec. 5.2)."""
    R, Q = paper_r2_q2(n)
    return np.asfortranarray(R @ Q + gamma * np.eye(n))


def paper_h3(n, gamma=2.0):
    """The "good" system H3 = R3 Q2 + gamma I with r3(i,i) = n+1-i and
    r3(i,j>i) = 1/2 (Sec. 5.2)."""
    R = np.triu(np.full((n, n), 0.5), 1) + np.diag(np.arange(n, 0, -1, dtype=np.float64))
    _, Q = paper_r2_q2(n)
    return np.asfortranarray(R @ Q + gamma * np.eye(n))


def companion(roots):
    """Upper Hessenberg companion matrix of prod (z - r): first row holds
    -coefficients, ones on the subdiagonal.  The eigenvector of root r is
    (r^(n-1), ..., r, 1)."""
    coeffs = np.poly(np.asarray(roots, dtype=np.float64))  # leading 1
    n = len(roots)
    C = np.zeros((n, n))
    C[0, :] = -coeffs[1:]
    for i in range(1, n):
        C[i, i - 1] = 1.0
    return np.asfortranarray(C)


def graded(H, seed, umax=150.0, monotone=False):
    """D H D^-1 with D = diag(10^u), u uniform in [-umax, umax] per index
    (monotone=True: u decreasing linearly from umax to -umax instead).
    Returns (G, d) with d the diagonal of D.  Hessenberg form is preserved and
    an eigenvector x of H maps to D x."""
    n = H.shape[0]
    if monotone:
        u = np.linspace(umax, -umax, n)
    else:
        u = uniform(seed, S_GRADE, n, -umax, umax)
    d = 10.0 ** u
    G = (d[:, None] * np.asarray(H)) / d[None, :]
    return np.asfortranarray(G), d


def unit_columns(n, ncol, seed, stream=S_B):
    """ncol unit-2-norm N(0,1) columns."""
    B = normal(seed, stream, n * ncol).reshape(n, ncol, order="F")
    B /= np.linalg.norm(B, axis=0)[None, :]
    return np.asfortranarray(B)
