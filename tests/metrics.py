"""Acceptance measures used by the tests (not part of the oracle or the product).

angle: the sign/phase-invariant chordal distance ||x - y (y^H x / |y^H x|)||_2
       between unit vectors x and y.
residual: ||H x - lambda x||_1 / (||H||_1 ||x||_1), the normwise residual whose
          bound is 100 n 2^-53.
"""
import numpy as np

EPS = 2.0 ** -53


def as_vectors(X, wr, wi):
    """Split the column layout (real: 1 column, complex: [re, im]) into a list
    of (lambda, vector) with complex vectors for complex shifts."""
    out, c = [], 0
    for l in range(len(wr)):
        if wi[l] != 0.0:
            out.append((complex(wr[l], wi[l]), X[:, c] + 1j * X[:, c + 1]))
            c += 2
        else:
            out.append((float(wr[l]), X[:, c].astype(np.float64)))
            c += 1
    return out


def angle(x, y):
    x = np.asarray(x, dtype=np.complex128)
    y = np.asarray(y, dtype=np.complex128)
    nx, ny = np.linalg.norm(x), np.linalg.norm(y)
    if nx == 0.0 or ny == 0.0:
        return np.inf
    x = x / nx
    y = y / ny
    d = np.vdot(y, x)
    ph = d / abs(d) if abs(d) > 0 else 1.0
    return float(np.linalg.norm(x - y * ph))


def residual(M, lam, x):
    x = np.asarray(x)
    r = M @ x - lam * x
    return float(np.abs(r).sum() / (np.abs(M).sum(axis=0).max() * np.abs(x).sum()))


def residuals(M, X, wr, wi, status=None):
    res = []
    for l, (lam, x) in enumerate(as_vectors(X, wr, wi)):
        if status is not None and status[l] != 0:
            res.append(np.nan)
            continue
        res.append(residual(M, lam, x))
    return np.array(res)


def separation(eigs, lam):
    """Distance from lam to the nearest other eigenvalue of the list eigs
    (lam itself is one of them)."""
    d = np.sort(np.abs(np.asarray(eigs) - lam))
    return d[1] if len(d) > 1 else np.inf


# Angle gate of the parity tests.  Two normwise backward-stable solves of
# (H - lambda I) x = b whose backward errors are of order n eps ||H|| give
# directions that differ, to first order, by about n eps ||H|| / gap, gap the
# distance of lambda to the nearest other eigenvalue: each of the two lies
# within that of the exact direction, so they lie within twice that of each
# other (C_FO = 2).  Eigenvalues separated by >= 1e-3 ||H||_inf meet the
# acceptance bound 1e-10 itself.
C_FO = 2.0


def first_order_bound(gap, hnorm, n):
    return n * EPS * hnorm / gap if gap > 0 else np.inf


def angle_bound(gap, hnorm, n):
    if gap >= 1e-3 * hnorm:
        return 1e-10
    return max(1e-10, C_FO * first_order_bound(gap, hnorm, n))
