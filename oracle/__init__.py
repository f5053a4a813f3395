"""FP64 CPU oracle for the robust multi-shift shifted-Hessenberg solve.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may use this package; the product path never
does.  It is an independent restatement of the method (Henry's RQ algorithm,
Alg. "henry", with the robust scaling of Sec. 4.1 and the normalization and
backtransform of Alg. "consistency-scaling"), written in plain C in
``hsein_oracle.c`` and wrapped here with ctypes.  It shares no code with the
CUDA library.

Every function here is pinned by tests against values that do not come from
the oracle itself (exact rational solves, closed-form eigenvectors, the
paper's printed 6x6 example, invariants); see tests/test_oracle_*.py.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None
LOG2_OMEGA_DEFAULT = 1000.0


def _load():
    global _lib
    if _lib is None:
        _lib = _bind(ctypes.CDLL(_build.build()))
    return _lib


def swap_library(path):
    """Load the oracle from another build of hsein_oracle.c (used by the
    mutation tests to check that the pins reject planted mistakes).  Returns
    the previously loaded library handle; pass it back to restore."""
    global _lib
    old = _load()
    _lib = path if isinstance(path, ctypes.CDLL) else _bind(ctypes.CDLL(path))
    return old


def _bind(lib):
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    lib.oracle_hnorm_inf.restype = ctypes.c_double
    lib.oracle_hnorm_inf.argtypes = [ctypes.c_int, dp, ctypes.c_int]
    lib.oracle_henry_real.restype = ctypes.c_int
    lib.oracle_henry_real.argtypes = [ctypes.c_int, dp, ctypes.c_int, ctypes.c_double, dp,
                                      ctypes.c_double, ctypes.c_int, dp, ip, dp, dp, dp]
    lib.oracle_henry_cplx.restype = ctypes.c_int
    lib.oracle_henry_cplx.argtypes = [ctypes.c_int, dp, ctypes.c_int, ctypes.c_double,
                                      ctypes.c_double, dp, ctypes.c_double, ctypes.c_int,
                                      dp, ip, dp, dp, dp]
    lib.oracle_backtransform_real.restype = None
    lib.oracle_backtransform_real.argtypes = [ctypes.c_int, dp, dp, dp]
    lib.oracle_backtransform_cplx.restype = None
    lib.oracle_backtransform_cplx.argtypes = [ctypes.c_int, dp, dp, dp]
    lib.oracle_hsein.restype = ctypes.c_int
    lib.oracle_hsein.argtypes = [ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, dp, dp, dp,
                                 ctypes.c_int, dp, ctypes.c_int, ip, ip, ctypes.c_double,
                                 ctypes.c_int, ctypes.c_int]
    lib.oracle_lu_real.restype = ctypes.c_int
    lib.oracle_lu_real.argtypes = [ctypes.c_int, dp, ctypes.c_int, ctypes.c_double, dp,
                                   ctypes.c_double, ctypes.c_int, dp, ip, dp, dp, ip, dp]
    lib.oracle_lu_cplx.restype = ctypes.c_int
    lib.oracle_lu_cplx.argtypes = [ctypes.c_int, dp, ctypes.c_int, ctypes.c_double,
                                   ctypes.c_double, dp, ctypes.c_double, ctypes.c_int,
                                   dp, ip, dp, dp, ip, dp]
    lib.oracle_hsein_lu.restype = ctypes.c_int
    lib.oracle_hsein_lu.argtypes = [ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, dp, dp, dp,
                                    ctypes.c_int, dp, ctypes.c_int, ip, ip, ctypes.c_double,
                                    ctypes.c_int, ctypes.c_int]
    lib.oracle_q0_apply.restype = None
    lib.oracle_q0_apply.argtypes = [ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, dp,
                                    ctypes.c_int, dp, ctypes.c_int, ctypes.c_int]
    lib.oracle_gehrd.restype = None
    lib.oracle_gehrd.argtypes = [ctypes.c_int, dp, ctypes.c_int, dp, ctypes.c_int, dp,
                                 ctypes.c_int, dp]
    return lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _f64(a):
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


def hnorm_inf(H):
    """||H||_inf of an upper Hessenberg matrix (max absolute row sum)."""
    H = _f64(H)
    return _load().oracle_hnorm_inf(H.shape[0], _dp(H), H.shape[0])


def henry_real(H, lam, b, log2_omega=LOG2_OMEGA_DEFAULT, robust=True):
    """One real-shift Henry solve.  Returns (x, e, C, S, replaced) with the
    true solution of (H - lam I) x = b equal to x * 2**e."""
    H = _f64(H)
    n = H.shape[0]
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.empty(n); C = np.empty(n); S = np.empty(n); work = np.empty(2 * n)
    e = np.zeros(1, dtype=np.int32)
    rep = _load().oracle_henry_real(n, _dp(H), n, float(lam), _dp(b), float(log2_omega),
                                    int(bool(robust)), _dp(x), _ip(e), _dp(C), _dp(S), _dp(work))
    return x, int(e[0]), C, S, bool(rep)


def henry_cplx(H, lam, b, log2_omega=LOG2_OMEGA_DEFAULT, robust=True):
    """One complex-shift Henry solve (lam complex, b complex).  Returns
    (x, e, C, S, replaced), C complex, S real."""
    H = _f64(H)
    n = H.shape[0]
    b = np.ascontiguousarray(b, dtype=np.complex128)
    x = np.empty(n, dtype=np.complex128); C = np.empty(n, dtype=np.complex128)
    S = np.empty(n); work = np.empty(2 * n, dtype=np.complex128)
    e = np.zeros(1, dtype=np.int32)
    lam = complex(lam)
    rep = _load().oracle_henry_cplx(n, _dp(H), n, lam.real, lam.imag, _dp(b.view(np.float64)),
                                    float(log2_omega), int(bool(robust)),
                                    _dp(x.view(np.float64)), _ip(e),
                                    _dp(C.view(np.float64)), _dp(S),
                                    _dp(work.view(np.float64)))
    return x, int(e[0]), C, S, bool(rep)


def backtransform_real(C, S, x):
    x = np.array(x, dtype=np.float64)
    _load().oracle_backtransform_real(len(x), _dp(np.ascontiguousarray(C, dtype=np.float64)),
                                      _dp(np.ascontiguousarray(S, dtype=np.float64)), _dp(x))
    return x


def backtransform_cplx(C, S, x):
    x = np.array(x, dtype=np.complex128)
    C = np.ascontiguousarray(C, dtype=np.complex128)
    _load().oracle_backtransform_cplx(len(x), _dp(C.view(np.float64)),
                                      _dp(np.ascontiguousarray(S, dtype=np.float64)),
                                      _dp(x.view(np.float64)))
    return x


def column_offsets(wi):
    """Column of each shift in B/X: real shifts own one column, complex two."""
    wi = np.asarray(wi, dtype=np.float64)
    widths = np.where(wi != 0.0, 2, 1)
    return np.concatenate([[0], np.cumsum(widths)]).astype(np.int64)


def hsein(H, wr, wi, B=None, log2_omega=LOG2_OMEGA_DEFAULT, robust=True, nthreads=0,
          return_exponents=False):
    """Unit-norm eigenvector approximations for every shift (Henry + scaling +
    normalization + backtransform + Varah's convergence test).  Returns
    (X, status) with X of shape (n, ncol); complex shifts own [re, im]."""
    H = _f64(H)
    n = H.shape[0]
    wr = np.ascontiguousarray(wr, dtype=np.float64)
    wi = np.ascontiguousarray(wi, dtype=np.float64)
    m = len(wr)
    ncol = int(column_offsets(wi)[-1])
    X = np.zeros((n, ncol), order="F")
    status = np.zeros(m, dtype=np.int32)
    exps = np.zeros(m, dtype=np.int32)
    if B is None:
        bptr, ldb = None, n
    else:
        B = _f64(B)
        assert B.shape == (n, ncol)
        bptr, ldb = _dp(B), n
    rc = _load().oracle_hsein(n, _dp(H), n, m, _dp(wr), _dp(wi), bptr, ldb, _dp(X), n,
                              _ip(status), _ip(exps), float(log2_omega), int(bool(robust)),
                              int(nthreads))
    if rc != 0:
        raise MemoryError("oracle_hsein failed to allocate")
    if return_exponents:
        return X, status, exps
    return X, status


def lu_real(H, lam, b, log2_omega=LOG2_OMEGA_DEFAULT, robust=True):
    """The LU approach (Sec. 2.1) for one real shift: P (H - lam I) = L U,
    L y = P b, U x = 2^-e y.  Returns (x, e, U packed by rows, L, piv,
    replaced) with the true solution x * 2**e."""
    H = _f64(H)
    n = H.shape[0]
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.empty(n); U = np.empty(n * (n + 1) // 2); Lm = np.empty(n); work = np.empty(n)
    piv = np.zeros(n, dtype=np.int32)
    e = np.zeros(1, dtype=np.int32)
    rep = _load().oracle_lu_real(n, _dp(H), n, float(lam), _dp(b), float(log2_omega),
                                 int(bool(robust)), _dp(x), _ip(e), _dp(U), _dp(Lm), _ip(piv),
                                 _dp(work))
    return x, int(e[0]), U, Lm, piv, bool(rep)


def lu_cplx(H, lam, b, log2_omega=LOG2_OMEGA_DEFAULT, robust=True):
    """Complex counterpart of lu_real (lam and b complex)."""
    H = _f64(H)
    n = H.shape[0]
    b = np.ascontiguousarray(b, dtype=np.complex128)
    x = np.empty(n, dtype=np.complex128); U = np.empty(n * (n + 1) // 2, dtype=np.complex128)
    Lm = np.empty(n, dtype=np.complex128); work = np.empty(n, dtype=np.complex128)
    piv = np.zeros(n, dtype=np.int32)
    e = np.zeros(1, dtype=np.int32)
    lam = complex(lam)
    rep = _load().oracle_lu_cplx(n, _dp(H), n, lam.real, lam.imag, _dp(b.view(np.float64)),
                                 float(log2_omega), int(bool(robust)),
                                 _dp(x.view(np.float64)), _ip(e), _dp(U.view(np.float64)),
                                 _dp(Lm.view(np.float64)), _ip(piv), _dp(work.view(np.float64)))
    return x, int(e[0]), U, Lm, piv, bool(rep)


def hsein_lu(H, wr, wi, B=None, log2_omega=LOG2_OMEGA_DEFAULT, robust=True, nthreads=0,
             return_exponents=False):
    """hsein() with the LU approach of Sec. 2.1 in place of Henry's RQ solve
    (the same outputs: unit-norm columns, status 0 converged / 1 not)."""
    H = _f64(H)
    n = H.shape[0]
    wr = np.ascontiguousarray(wr, dtype=np.float64)
    wi = np.ascontiguousarray(wi, dtype=np.float64)
    m = len(wr)
    ncol = int(column_offsets(wi)[-1])
    X = np.zeros((n, ncol), order="F")
    status = np.zeros(m, dtype=np.int32)
    exps = np.zeros(m, dtype=np.int32)
    if B is None:
        bptr = None
    else:
        B = _f64(B)
        assert B.shape == (n, ncol)
        bptr = _dp(B)
    rc = _load().oracle_hsein_lu(n, _dp(H), n, m, _dp(wr), _dp(wi), bptr, n, _dp(X), n,
                                 _ip(status), _ip(exps), float(log2_omega), int(bool(robust)),
                                 int(nthreads))
    if rc != 0:
        raise MemoryError("oracle_hsein_lu failed to allocate")
    if return_exponents:
        return X, status, exps
    return X, status


def q0_apply(Q, X, nthreads=0):
    """Z = Q X column by column (plain loops)."""
    Q = _f64(Q)
    X = _f64(X)
    n, ncol = X.shape
    Z = np.zeros((n, ncol), order="F")
    _load().oracle_q0_apply(n, _dp(Q), n, ncol, _dp(X), n, _dp(Z), n, int(nthreads))
    return Z


def gehrd(A):
    """Plain Householder reduction A = Q H Q^T.  Returns (H, Q)."""
    A = _f64(A)
    n = A.shape[0]
    H = np.zeros((n, n), order="F"); Q = np.zeros((n, n), order="F")
    work = np.empty(2 * n)
    _load().oracle_gehrd(n, _dp(A), n, _dp(H), n, _dp(Q), n, _dp(work))
    return H, Q


def restart_vector(b, t, b_im=None):
    """Trial starting vector t (t = 1, 2, ...) for a shift whose solve from
    the starting vector b (real; with b_im the complex vector b + i b_im) did
    not converge: the restart of Alg. "hsrq3in" (Sec. 4.2) asks for a new
    start orthogonal to the previous choices.  Reading used here: the
    Householder QR of [b] (real) or [Re b, Im b] (complex) gives an orthogonal
    Q whose leading columns span the previous start; trial t is column
    n+1-t of Q (a real unit vector, orthogonal to b and to the other trials).
    Each reflector is I - 2 w w^T / (w^T w), w = a/||a|| + sign(a_1) e_1, with
    the second reflector acting on rows 2..n; it is skipped when the
    imaginary part lies in the span of the real part (the part outside it is
    below 2^-50 of the whole).  With Re b = 0 the imaginary part leads; with
    b = 0 trial t is e_(n+1-t).  Plain numpy, test infrastructure only."""
    a1 = np.array(b, dtype=np.float64)
    n = a1.shape[0]
    a2 = None if b_im is None else np.array(b_im, dtype=np.float64)
    if a2 is not None and not np.any(a1):
        a1, a2 = a2, a1
    j = n - t  # 0-based column of Q
    y = np.zeros(n)
    y[j] = 1.0
    if not np.any(a1):
        return y

    def reflector(a):
        v = a / np.linalg.norm(a)
        w = v.copy()
        w[0] += 1.0 if v[0] >= 0.0 else -1.0
        return w

    w1 = reflector(a1)
    if a2 is not None:
        u = a2 - 2.0 * (w1 @ a2) / (w1 @ w1) * w1  # P1 a2
        if np.abs(u[1:]).max() > 2.0 ** -50 * np.abs(u).max():
            w2 = reflector(u[1:])
            y[1:] = y[1:] - 2.0 * (w2 @ y[1:]) / (w2 @ w2) * w2  # P2 e_j
    return y - 2.0 * (w1 @ y) / (w1 @ w1) * w1  # P1 y
