"""Pins of the CPU oracle to facts that do not come from the oracle itself.

Each test checks the oracle against one of: an exact rational solve of the
same system, a closed-form eigenvector, the matrices the paper prints for its
second test problem (Sec. 5.2), properties the paper states (unit norm after
the backtransform, c^2 + s^2 = 1, the padding rotation, the triangular factor
(H - lambda I) G_n^T ... G_2^T = R of Sec. 3.1, the "good" system never
scaling and the "bad" one scaling), a library routine, or the normwise
residual bound 100 n eps.
"""
import numpy as np
import pytest

import hsein_inputs as hi
import oracle
from tests.exact import exact_solve, read_golden_blocks
from tests.metrics import EPS, angle, as_vectors, residual, residuals

import os

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def random_hessenberg(n, seed, scale=1.0):
    H = hi.normal(seed, 50, n * n).reshape(n, n, order="F") * scale
    return np.asfortranarray(np.triu(H, -1))


def solve_oracle_real(H, lam, b, **kw):
    x, e, C, S, rep = oracle.henry_real(H, lam, b, **kw)
    return oracle.backtransform_real(C, S, x) * 2.0 ** e


def solve_oracle_cplx(H, lam, b, **kw):
    x, e, C, S, rep = oracle.henry_cplx(H, lam, b, **kw)
    return oracle.backtransform_cplx(C, S, x) * 2.0 ** e


# ------------------------------------------------------------ the norm

def test_hnorm_inf_is_the_maximum_absolute_row_sum():
    # ||H||_inf sets rho = eps ||H||_inf, the pivot replacement and Varah's
    # threshold.  A hand-computed case where the largest row sum (12, row 2,
    # which needs its subdiagonal entry) differs from the largest column sum
    # (11) and from the largest row sum without subdiagonal entries (6)
    H = np.array([[1.0, -2.0, 3.0], [-10.0, 1.0, 1.0], [0.0, 1.0, -1.0]])
    assert oracle.hnorm_inf(H) == 12.0
    assert np.abs(H).sum(axis=0).max() == 11.0
    # non-symmetric random Hessenberg matrices against numpy's matrix norm,
    # with rows and columns of different scales
    for n, seed in ((2, 1), (7, 2), (64, 3), (300, 4)):
        H = random_hessenberg(n, seed)
        H = H * (2.0 ** np.arange(n))[:, None] / (3.0 ** np.arange(n) / 3.0 ** n)[None, :]
        H = np.asfortranarray(H)
        ref = np.linalg.norm(H, np.inf)
        assert abs(oracle.hnorm_inf(H) - ref) <= 2 * n * EPS * ref, (n, oracle.hnorm_inf(H), ref)
        assert abs(np.abs(H).sum(axis=0).max() - ref) > 1e-3 * ref  # the test tells them apart


# ------------------------------------------------------------ exact solves

@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 12])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_real_solve_matches_exact_rational(n, seed):
    H = random_hessenberg(n, seed)
    b = hi.normal(seed, 51, n)
    lam = float(hi.uniform(seed, 52, 1, -2.0, 2.0)[0])
    x = solve_oracle_real(H, lam, b)
    xe = exact_solve(H, lam, b).real
    kappa = np.linalg.cond(H - lam * np.eye(n))
    err = np.linalg.norm(x - xe) / np.linalg.norm(xe)
    assert err <= 4 * n * kappa * EPS, (err, kappa)


@pytest.mark.parametrize("n", [2, 3, 5, 8, 12])
@pytest.mark.parametrize("seed", [4, 5])
def test_complex_solve_matches_exact_rational(n, seed):
    H = random_hessenberg(n, seed)
    b = hi.normal(seed, 51, n) + 1j * hi.normal(seed, 53, n)
    lam = complex(hi.uniform(seed, 52, 1, -2.0, 2.0)[0], hi.uniform(seed, 54, 1, 0.1, 2.0)[0])
    x = solve_oracle_cplx(H, lam, b)
    xe = exact_solve(H, lam, b)
    kappa = np.linalg.cond(H - lam * np.eye(n))
    err = np.linalg.norm(x - xe) / np.linalg.norm(xe)
    assert err <= 4 * n * kappa * EPS, (err, kappa)


@pytest.mark.parametrize("n", [4, 9])
def test_far_shift_is_well_conditioned_to_1e13(n):
    # a shift outside the spectrum: the system is well conditioned and the
    # oracle must agree with the exact solution to 1e-13
    H = random_hessenberg(n, 7)
    lam = 10.0 * np.abs(H).sum(axis=1).max()
    b = hi.normal(7, 51, n)
    x = solve_oracle_real(H, lam, b)
    xe = exact_solve(H, lam, b).real
    assert np.linalg.norm(x - xe) <= 1e-13 * np.linalg.norm(xe)
    xc = solve_oracle_cplx(H, complex(lam, 1.0), b.astype(complex))
    xce = exact_solve(H, complex(lam, 1.0), b)
    assert np.linalg.norm(xc - xce) <= 1e-13 * np.linalg.norm(xce)


# --------------------------------------------------------- closed forms

@pytest.mark.parametrize("n", [2, 3, 5, 8])
def test_companion_eigenvectors_closed_form(n):
    roots = np.arange(1, n + 1, dtype=np.float64)
    C = hi.companion(roots)
    wr = roots.copy()
    wi = np.zeros(n)
    X, status = oracle.hsein(C, wr, wi, B=hi.unit_columns(n, n, seed=n))
    assert np.all(status == 0)
    for l, r in enumerate(roots):
        exact = r ** np.arange(n - 1, -1, -1, dtype=np.float64)
        assert angle(X[:, l], exact) <= 1e-12


def test_paper_h2_example_matches_printed_matrices():
    g = read_golden_blocks(os.path.join(GOLDEN, "paper_h2_n6.txt"))
    R, Q = hi.paper_r2_q2(6)
    assert np.array_equal(R, g["R2"])
    assert np.array_equal(Q, g["Q2"])
    assert np.array_equal(R @ Q, g["H2_MINUS_GAMMA_I"])
    assert np.array_equal(hi.paper_h2(6) - 2.0 * np.eye(6), g["H2_MINUS_GAMMA_I"])


def test_paper_h2_solve_matches_exact_on_printed_matrix():
    g = read_golden_blocks(os.path.join(GOLDEN, "paper_h2_n6.txt"))
    M = g["H2_MINUS_GAMMA_I"]
    b = np.ones(6)
    x = solve_oracle_real(M, 0.0, b)
    xe = exact_solve(M, 0.0, b).real
    assert np.linalg.norm(x - xe) <= 1e-14 * np.linalg.norm(xe)


# ------------------------------------------------------ robust scaling

@pytest.mark.parametrize("n", [16, 64, 256])
@pytest.mark.parametrize("log2_omega", [1000.0, 40.0])
def test_good_system_h3_never_scales(n, log2_omega):
    # Sec. 5.2: the good system never requires numerical scaling
    H = hi.paper_h3(n)
    x, e, C, S, rep = oracle.henry_real(H, 2.0, np.ones(n), log2_omega=log2_omega)
    assert e == 0
    assert np.all(np.isfinite(x))


@pytest.mark.parametrize("n", [32, 48])
def test_bad_system_h2_scales_and_stays_exact(n):
    # Sec. 5.2: the bad system needs frequent scaling; with a lowered overflow
    # threshold the scaling triggers at small n, and the scaled result must
    # still be the exact solution's direction (all rotations are exact here)
    H = hi.paper_h2(n)
    x, e, C, S, rep = oracle.henry_real(H, 2.0, np.ones(n), log2_omega=30.0)
    assert e > 0
    y = oracle.backtransform_real(C, S, x)
    assert np.all(np.isfinite(y))
    xe = exact_solve(H, 2.0, np.ones(n)).real
    assert angle(y, xe) <= 1e-13
    # and the unscaled size really exceeds the lowered threshold
    assert np.log2(np.abs(xe).max()) > 30.0


def test_bad_system_h2_overflows_without_protection():
    n = 1024
    H = hi.paper_h2(n)
    x, e, C, S, rep = oracle.henry_real(H, 2.0, np.ones(n), robust=False)
    assert not np.all(np.isfinite(x))
    x, e, C, S, rep = oracle.henry_real(H, 2.0, np.ones(n), robust=True)
    assert np.all(np.isfinite(x)) and e > 0
    # backward error of the scaled solve: (H - 2I) y = 2^-e b with y the
    # backtransformed x, measured in long double
    y = oracle.backtransform_real(C, S, x).astype(np.longdouble)
    M = (H - 2.0 * np.eye(n)).astype(np.longdouble)
    b = np.ones(n, dtype=np.longdouble) * np.ldexp(np.longdouble(1.0), -e)
    r = np.abs(M @ y - b).sum()
    assert float(r / (np.abs(M).sum(axis=0).max() * np.abs(y).sum())) <= 100 * n * EPS


def test_graded_matrix_overflows_only_without_protection():
    # monotone grading D = diag(10^u), u from 150 down to -150: the exact
    # solution leaves the double range, so the unprotected solve overflows;
    # the protected one stays finite with a small normwise residual (the
    # algorithm is normwise backward stable; with ||G|| ~ 1e300 that is all a
    # shift of size O(1) can promise)
    n = 24
    H0 = random_hessenberg(n, 11)
    G, d = hi.graded(H0, seed=11, umax=150.0, monotone=True)
    ev = np.linalg.eigvals(H0)
    lam = float(ev[np.argmin(np.abs(ev.imag))].real)
    b = hi.normal(11, 51, n)
    with np.errstate(all="ignore"):
        x, e, C, S, rep = oracle.henry_real(G, lam, b, robust=False)
    assert not np.all(np.isfinite(x))
    X, status = oracle.hsein(G, [lam], [0.0], B=b[:, None] / np.linalg.norm(b))
    y = X[:, 0]
    assert status[0] == 0 and np.all(np.isfinite(y)) and abs(np.linalg.norm(y) - 1) < 1e-14
    Gl = G.astype(np.longdouble)
    yl = y.astype(np.longdouble)
    r = np.abs(Gl @ yl - np.longdouble(lam) * yl).sum()
    assert float(r / (np.abs(Gl).sum(axis=0).max() * np.abs(yl).sum())) <= 100 * n * EPS


def test_graded_eigenvector_is_d_times_eigenvector():
    n = 16
    H0 = random_hessenberg(n, 12)
    G, d = hi.graded(H0, seed=12, umax=1.0)
    ev = np.linalg.eigvals(H0)
    lam = float(ev[np.argmin(np.abs(ev.imag))].real)
    b = hi.normal(12, 51, n)
    XH, sH = oracle.hsein(H0, [lam], [0.0], B=b[:, None])
    XG, sG = oracle.hsein(G, [lam], [0.0], B=b[:, None])
    assert sH[0] == 0 and sG[0] == 0
    assert angle(XG[:, 0], d * XH[:, 0]) <= 1e-9


# ------------------------------------------------------------ invariants

@pytest.mark.parametrize("n", [5, 33, 64])
def test_rotations_triangularize_shifted_matrix(n):
    H = random_hessenberg(n, 13)
    lam = 0.37
    x, e, C, S, rep = oracle.henry_real(H, lam, np.ones(n))
    assert C[0] == 1.0 and S[0] == 0.0  # padding rotation of the top-left tile
    assert np.all(np.abs(C ** 2 + S ** 2 - 1.0) <= 4 * EPS)
    M = H - lam * np.eye(n)
    for k in range(n - 1, 0, -1):  # (H - lam I) G_n^T ... G_2^T = R
        G = np.array([[C[k], -S[k]], [S[k], C[k]]])
        M[:, [k - 1, k]] = M[:, [k - 1, k]] @ G
    hn = np.abs(H).sum(axis=1).max()
    assert np.abs(np.tril(M, -1)).max() <= 4 * n * EPS * hn
    assert np.all(np.diag(M)[1:] > 0)  # phi > 0 with the chosen sign


@pytest.mark.parametrize("n", [5, 33])
def test_complex_rotations_triangularize(n):
    H = random_hessenberg(n, 14)
    lam = 0.2 + 0.9j
    x, e, C, S, rep = oracle.henry_cplx(H, lam, np.ones(n, dtype=complex))
    assert C[0] == 1.0 and S[0] == 0.0
    assert np.all(np.abs(np.abs(C) ** 2 + S ** 2 - 1.0) <= 8 * EPS)
    M = (H - lam * np.eye(n)).astype(complex)
    for k in range(n - 1, 0, -1):
        G = np.array([[C[k], -S[k]], [S[k], np.conj(C[k])]])
        M[:, [k - 1, k]] = M[:, [k - 1, k]] @ G
    hn = np.abs(H).sum(axis=1).max() + abs(lam)
    assert np.abs(np.tril(M, -1)).max() <= 8 * n * EPS * hn
    d = np.diag(M)[1:]
    assert np.all(np.abs(d.imag) <= 8 * n * EPS * hn) and np.all(d.real > 0)


def test_output_columns_have_unit_norm_and_small_residual():
    inst = hi.small_instance(80, 8, 6, seed=3)
    X, status = oracle.hsein(inst.H, inst.wr, inst.wi, inst.B)
    offs = hi.column_offsets(inst.wi)
    for l in range(inst.m):
        if status[l] == 0:
            nrm = np.linalg.norm(X[:, offs[l]:offs[l + 1]])
            assert abs(nrm - 1.0) <= 4 * inst.n * EPS
    res = residuals(inst.H, X, inst.wr, inst.wi, status)
    ok = status == 0
    assert ok.sum() >= inst.m - 2
    assert np.nanmax(res[ok]) <= 100 * inst.n * EPS


def test_config0_residuals_and_convergence():
    inst = hi.config0()
    X, status = oracle.hsein(inst.H, inst.wr, inst.wi, inst.B)
    assert np.all(status == 0)
    assert np.nanmax(residuals(inst.H, X, inst.wr, inst.wi)) <= 100 * inst.n * EPS


def test_convergence_flag_far_and_near_shift():
    # Varah's test (Sec. 4.2): a shift far from the spectrum gives a small
    # solution and must be flagged (column zeroed); an eigenvalue must pass
    inst = hi.config0()
    H = inst.H
    far = 1e3 * oracle.hnorm_inf(H)
    X, status = oracle.hsein(H, [far, inst.wr[0]], [0.0, 0.0], B=inst.B[:, :2])
    assert list(status) == [1, 0]
    assert np.all(X[:, 0] == 0.0)
    assert abs(np.linalg.norm(X[:, 1]) - 1.0) <= 1e-13


def test_default_starting_vector_is_rho_e():
    inst = hi.small_instance(40, 4, 2, seed=6)
    X0, s0 = oracle.hsein(inst.H, inst.wr, inst.wi, None)
    rho = EPS * oracle.hnorm_inf(inst.H)
    B = np.zeros((inst.n, inst.ncol))
    offs = hi.column_offsets(inst.wi)
    for l in range(inst.m):
        B[:, offs[l]] = rho  # complex: rho*e in the real part, 0 imaginary
    X1, s1 = oracle.hsein(inst.H, inst.wr, inst.wi, B)
    assert np.array_equal(X0, X1) and np.array_equal(s0, s1)


def test_exact_eigenvalue_pivot_replacement():
    # lambda an exact eigenvalue of an exactly representable H: the final pivot
    # is (numerically) zero and is replaced; the result is the eigenvector
    H = np.array([[2.0, 1.0, 0.0], [1.0, 3.0, 1.0], [0.0, 1.0, 4.0]])
    # eigenvalue 3 has eigenvector (1, 1, -1): H (1, 1, -1) = (3, 3, -3)
    b = np.array([[0.3], [-0.5], [0.8]])
    X, status = oracle.hsein(H, [3.0], [0.0], B=b)
    assert status[0] == 0
    assert angle(X[:, 0], [1.0, 1.0, -1.0]) <= 1e-14
    x, e, C, S, replaced = oracle.henry_real(H, 3.0, b[:, 0])
    assert replaced


def test_q0_apply_matches_matmul():
    rng_Q = hi.haar_orthogonal(20, 3)
    X = hi.normal(3, 60, 20 * 5).reshape(20, 5, order="F")
    Z = oracle.q0_apply(rng_Q, X)
    assert np.allclose(Z, rng_Q @ X, rtol=0, atol=1e-14)


# ------------------------------------------------- Hessenberg reduction

@pytest.mark.parametrize("n", [3, 10, 40])
def test_householder_reduction(n):
    import scipy.linalg
    A = hi.normal(21, 61, n * n).reshape(n, n, order="F")
    H, Q = oracle.gehrd(A)
    assert np.abs(np.tril(H, -2)).max(initial=0.0) == 0.0
    assert np.abs(Q @ H @ Q.T - A).max() <= 10 * n * EPS * np.abs(A).max() * n
    assert np.abs(Q.T @ Q - np.eye(n)).max() <= 10 * n * EPS
    Hs = scipy.linalg.hessenberg(A)
    # unique up to the signs of the reflectors: |H| agrees with LAPACK's
    assert np.allclose(np.abs(H), np.abs(np.triu(Hs, -1)), rtol=1e-10, atol=1e-10 * np.abs(A).max())


# ------------------------------------------------------------ generators

def test_splitmix64_reference_value():
    # seed 0 / stream 0 reduce to the plain SplitMix64 sequence from state 0,
    # whose first output is the published 0xE220A8397B1DCDAF
    assert int(hi.splitmix64(0, 0, 1)[0]) == 0xE220A8397B1DCDAF


def test_generators_are_counter_based():
    a = hi.uniform(5, 3, 100)
    b = hi.uniform(5, 3, 40, start=60)
    assert np.array_equal(a[60:], b)
    z = hi.normal(9, 2, 1000)
    assert abs(z.mean()) < 0.1 and abs(z.std() - 1) < 0.1


def test_config0_structure():
    inst = hi.config0(keep_a=True)
    assert inst.n == 512 and inst.m == 64 and inst.ncol == 64
    assert np.abs(np.tril(inst.H, -2)).max() == 0.0
    assert np.all(inst.H[np.arange(1, 512), np.arange(511)] != 0.0)
    assert np.abs(inst.Q0 @ inst.H @ inst.Q0.T - inst.A).max() <= 1e-10 * np.abs(inst.A).max()
    assert np.allclose(np.linalg.norm(inst.B, axis=0), 1.0)
    # the shifts are eigenvalues of H to working accuracy
    ev = np.linalg.eigvals(inst.H)
    d = np.array([np.min(np.abs(ev - w)) for w in inst.wr])
    assert d.max() <= 1e-8 * np.abs(inst.H).max()


def test_tiny_pivot_division_is_protected():
    # a tiny subdiagonal and a shift that makes the last diagonal entry tiny
    # give a pivot phi ~ 1e-300; dividing a large right-hand side by it
    # overflows unless ProtectDivision rescales first
    H = np.array([[1.0, 2.0, 0.5], [1e-300, 3.0, 1.0], [0.0, 1e-300, 5.0]])
    b = np.array([1.0, 1.0, 1e20])
    with np.errstate(all="ignore"):
        x, e, C, S, rep = oracle.henry_real(H, 5.0, b, robust=False)
    assert not np.all(np.isfinite(x))
    x, e, C, S, rep = oracle.henry_real(H, 5.0, b)
    assert e > 0 and np.all(np.isfinite(x))
    y = oracle.backtransform_real(C, S, x)
    xe = exact_solve(H, 5.0, b, direction=True).real
    assert angle(y, xe) <= 1e-13


def test_bad_system_h2_through_the_driver():
    # the scaled solution of the bad system is astronomically large
    # (exponent far beyond the double range), so Varah's test must pass once
    # the exponent is counted, and the normalized vector must have a tiny
    # residual (Sec. 4.2, Sec. 5.2)
    n = 1024
    H = hi.paper_h2(n)
    X, status, exps = oracle.hsein(H, [2.0], [0.0], B=np.ones((n, 1)) / np.sqrt(n),
                                   return_exponents=True)
    assert status[0] == 0 and exps[0] > 900
    assert np.all(np.isfinite(X)) and abs(np.linalg.norm(X[:, 0]) - 1.0) <= 4 * n * EPS
    assert residual(H, 2.0, X[:, 0]) <= 100 * n * EPS


# ------------------------------------------------- the LU approach (Sec. 2.1)

def _lu_factors(n, U, Lm, piv):
    """Dense P, L, U of P (H - lambda I) = L U from the oracle's packed output:
    row k of U holds columns k..n-1; step k exchanges rows k and k+1 when
    piv[k] and eliminates row k+1 with multiplier Lm[k]."""
    dt = U.dtype
    Ud = np.zeros((n, n), dtype=dt)
    off = 0
    for k in range(n):
        Ud[k, k:] = U[off:off + n - k]
        off += n - k
    # P and L as products of elementary steps: M_{n-2} P_{n-2} ... M_0 P_0 (H - lam I) = U
    Minv = np.eye(n, dtype=dt)  # accumulates (M P)^-1 = P^T M^-1 in order
    for k in range(n - 1):
        Pk = np.eye(n, dtype=dt)
        if piv[k]:
            Pk[[k, k + 1]] = Pk[[k + 1, k]]
        Mk_inv = np.eye(n, dtype=dt)
        Mk_inv[k + 1, k] = Lm[k]
        Minv = Minv @ Pk.T @ Mk_inv
    return Minv, Ud  # H - lam I = Minv U


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 12])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_lu_real_solve_matches_exact_rational(n, seed):
    H = random_hessenberg(n, seed)
    b = hi.normal(seed, 51, n)
    lam = float(hi.uniform(seed, 52, 1, -2.0, 2.0)[0])
    x, e, U, Lm, piv, rep = oracle.lu_real(H, lam, b)
    xe = exact_solve(H, lam, b).real
    kappa = np.linalg.cond(H - lam * np.eye(n))
    err = np.linalg.norm(x * 2.0 ** e - xe) / np.linalg.norm(xe)
    assert err <= 4 * n * kappa * EPS, (err, kappa)


@pytest.mark.parametrize("n", [2, 3, 5, 8, 12])
def test_lu_complex_solve_matches_exact_rational(n):
    H = random_hessenberg(n, 4)
    b = hi.normal(4, 51, n) + 1j * hi.normal(4, 53, n)
    lam = complex(hi.uniform(4, 52, 1, -2.0, 2.0)[0], hi.uniform(4, 54, 1, 0.1, 2.0)[0])
    x, e, U, Lm, piv, rep = oracle.lu_cplx(H, lam, b)
    xe = exact_solve(H, lam, b)
    kappa = np.linalg.cond(H - lam * np.eye(n))
    assert np.linalg.norm(x * 2.0 ** e - xe) / np.linalg.norm(xe) <= 4 * n * kappa * EPS


@pytest.mark.parametrize("cplx", [False, True])
def test_lu_factors_reproduce_the_shifted_matrix_with_bounded_multipliers(cplx):
    # P (H - lambda I) = L U with |l_k| <= 1 (partial pivoting) and U upper
    # triangular; a zero leading entry forces the first interchange
    n = 33
    H = random_hessenberg(n, 17)
    lam = H[0, 0] + (0.5j if cplx else 0.0)
    if cplx:
        x, e, U, Lm, piv, rep = oracle.lu_cplx(H, lam, np.ones(n, dtype=complex))
    else:
        x, e, U, Lm, piv, rep = oracle.lu_real(H, lam, np.ones(n))
    assert np.all(np.abs(Lm[:n - 1]) <= 1.0)
    if not cplx:
        assert piv[0] == 1  # h(0,0) - lambda = 0: the subdiagonal entry must pivot
    Minv, Ud = _lu_factors(n, U, Lm, piv)
    M = H - lam * np.eye(n)
    assert np.abs(Minv @ Ud - M).max() <= 8 * n * EPS * np.abs(M).max()


def test_lu_companion_eigenvectors_closed_form():
    n = 6
    roots = np.arange(1, n + 1, dtype=np.float64)
    C = hi.companion(roots)
    X, status = oracle.hsein_lu(C, roots, np.zeros(n), B=hi.unit_columns(n, n, seed=n))
    assert np.all(status == 0)
    # the roots are one apart: twice the first-order bound n eps ||C|| / gap
    bound = 2 * n * EPS * np.abs(C).sum(axis=1).max()
    for l, r in enumerate(roots):
        assert angle(X[:, l], r ** np.arange(n - 1, -1, -1, dtype=np.float64)) <= bound


def test_lu_scaling_is_needed_and_exact():
    # back-substitution growth of 1e200 per row: the unprotected LU solve
    # overflows, the protected one scales (the exponent carries the growth)
    # and equals the exact solution's direction, real and complex
    n = 6
    H = np.eye(n) + 1e200 * np.triu(np.ones((n, n)), 1) + 1e-3 * np.diag(np.ones(n - 1), -1)
    b = np.ones(n)
    with np.errstate(all="ignore"):
        x, e, U, Lm, piv, rep = oracle.lu_real(H, 0.5, b, robust=False)
    assert not np.all(np.isfinite(x))
    x, e, U, Lm, piv, rep = oracle.lu_real(H, 0.5, b)
    assert e > 0 and np.all(np.isfinite(x))
    assert angle(x / np.abs(x).max(), exact_solve(H, 0.5, b, direction=True).real) <= 1e-13
    bc = b.astype(complex)
    with np.errstate(all="ignore"):
        xc, e, U, Lm, piv, rep = oracle.lu_cplx(H, 0.5 + 0.25j, bc, robust=False)
    assert not np.all(np.isfinite(xc))
    xc, e, U, Lm, piv, rep = oracle.lu_cplx(H, 0.5 + 0.25j, bc)
    assert e > 0 and np.all(np.isfinite(xc))
    assert angle(xc / np.abs(xc).max(), exact_solve(H, 0.5 + 0.25j, bc, direction=True)) <= 1e-13
    # growth in the forward substitution: H - 0 I = L U with L unit lower
    # bidiagonal (-1 below the diagonal, every multiplier -1) and U = I, so
    # x = L^-1 b is the running sum of b; with b near the top of the double
    # range the unprotected forward solve overflows, the protected one gives
    # the closed-form direction (1, 2, ..., n) / ||.||
    m = 9
    H = np.eye(m) - np.diag(np.ones(m - 1), -1)
    b = np.full(m, 1e308)
    with np.errstate(all="ignore"):
        x, e, U, Lm, piv, rep = oracle.lu_real(H, 0.0, b, robust=False)
    assert not np.all(np.isfinite(x))
    x, e, U, Lm, piv, rep = oracle.lu_real(H, 0.0, b)
    assert e > 0 and np.all(np.isfinite(x)) and np.all(piv == 0)
    assert angle(x, np.arange(1.0, m + 1)) <= 4 * m * EPS
    # the bad system of Sec. 5.2 with a lowered threshold: scaling triggers
    # at small n and the direction is exact
    m = 40
    H = hi.paper_h2(m)
    x, e, U, Lm, piv, rep = oracle.lu_real(H, 2.0, np.ones(m), log2_omega=30.0)
    assert e > 0 and np.all(np.isfinite(x))
    assert angle(x, exact_solve(H, 2.0, np.ones(m)).real) <= 1e-13


def test_lu_bad_system_h2_at_full_threshold():
    # at n = 1024 the shift is an eigenvalue of H2 to working accuracy: the
    # final pivot is replaced and the normalized result is an eigenvector
    # (small normwise residual in long double)
    n = 1024
    H = hi.paper_h2(n)
    X, status = oracle.hsein_lu(H, [2.0], [0.0], np.ones((n, 1)) / np.sqrt(n))
    assert status[0] == 0 and np.all(np.isfinite(X))
    y = X[:, 0].astype(np.longdouble)
    M = H.astype(np.longdouble)
    r = np.abs(M @ y - np.longdouble(2.0) * y).sum()
    assert float(r / (np.abs(M).sum(axis=0).max() * np.abs(y).sum())) <= 100 * n * EPS


def test_lu_driver_statuses_and_unit_norm():
    inst = hi.small_instance(60, 4, 3, 9)
    X, status = oracle.hsein_lu(inst.H, inst.wr, inst.wi, inst.B)
    assert np.all(status == 0)
    for lam, x in as_vectors(X, inst.wr, inst.wi):
        assert abs(np.linalg.norm(x) - 1.0) <= 4 * inst.n * EPS
        assert residual(inst.H, lam, x) <= 100 * inst.n * EPS
    far = 1e3 * oracle.hnorm_inf(inst.H)
    X, status = oracle.hsein_lu(inst.H, [far], [0.0], inst.B[:, :1])
    assert status[0] == 1 and np.all(X == 0.0)


# ---------------------------------------------------------------- restart
# Alg. "hsrq3in" (Sec. 4.2): a new starting vector orthogonal to the previous
# choices.  Pins: closed forms at n = 2 (real) and n = 3 (complex: the
# normalized cross product of Re b and Im b), and orthonormality of the
# trials and their orthogonality to the previous start at larger n.

def test_restart_vector_closed_form_real_n2():
    b = np.array([3.0, -4.0])
    y = oracle.restart_vector(b, 1)
    expect = np.array([4.0, 3.0]) / 5.0  # the unit vector orthogonal to b
    assert min(np.abs(y - expect).max(), np.abs(y + expect).max()) <= 1e-15


def test_restart_vector_closed_form_complex_n3():
    br = np.array([1.0, 2.0, -1.0])
    bi = np.array([0.5, -1.0, 3.0])
    y = oracle.restart_vector(br, 1, bi)
    c = np.cross(br, bi)
    c /= np.linalg.norm(c)
    assert min(np.abs(y - c).max(), np.abs(y + c).max()) <= 1e-14


@pytest.mark.parametrize("cplx", [False, True])
def test_restart_vectors_orthonormal_and_orthogonal_to_start(cplx):
    n = 40
    br = hi.normal(71, 1, n)
    bi = hi.normal(72, 1, n) if cplx else None
    T = 6
    Y = np.stack([oracle.restart_vector(br, t, bi) for t in range(1, T + 1)], axis=1)
    assert np.abs(Y.T @ Y - np.eye(T)).max() <= 1e-14
    assert np.abs(br @ Y).max() <= 1e-13 * np.linalg.norm(br)
    if cplx:
        assert np.abs(bi @ Y).max() <= 1e-13 * np.linalg.norm(bi)


def test_restart_vector_degenerate_starts():
    n = 8
    # imaginary part in the span of the real part: only the real part counts
    br = np.arange(1.0, n + 1)
    y = oracle.restart_vector(br, 2, 3.0 * br)
    assert abs(br @ y) <= 1e-13 * np.linalg.norm(br) and abs(np.linalg.norm(y) - 1) <= 1e-15
    # zero real part: the imaginary part leads
    y = oracle.restart_vector(np.zeros(n), 1, br)
    assert abs(br @ y) <= 1e-13 * np.linalg.norm(br)
    # zero start: a unit basis vector
    y = oracle.restart_vector(np.zeros(n), 3)
    assert y[n - 3] == 1.0 and np.abs(y).sum() == 1.0
