"""Restart loop of inverse iteration (Alg. "hsrq3in", Sec. 4.2) and the
per-shift convergence margins, on the GPU against the oracle.

A starting vector b with u^T b = 0 for the left eigenvector u of the shift's
eigenvalue gives one step of inverse iteration no component to amplify, so
the first solve fails Varah's test (the oracle agrees on the same input); the
restart must then converge and match the oracle solved from the oracle's own
trial vector (oracle.restart_vector).  A shift far from the spectrum never
converges, whatever the start.
"""
import math

import numpy as np
import pytest

import hsein_inputs as hi
import oracle
from tests.metrics import EPS, angle, as_vectors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2101_05063_gb300 as hs  # noqa: E402
from tests.metrics import angle_bound, separation  # noqa: E402
from tests.test_gpu_parity import to_dev  # noqa: E402


def _start_without_left_component(H, lam, seed, cplx):
    """A starting vector b (real, or complex as (re, im)) with u^T b = 0 for
    the left eigenvector u of H nearest lam (H^T u = mu u)."""
    w, U = np.linalg.eig(H.T)
    u = U[:, np.argmin(np.abs(w - lam))]
    n = H.shape[0]
    b = hi.normal(seed, 1, n) + (1j * hi.normal(seed, 2, n) if cplx else 0.0)
    b = b - (u @ b) / np.vdot(u, u).real * np.conj(u)
    if cplx:
        return np.stack([b.real, b.imag], axis=1)
    return b.real.reshape(-1, 1)


def _oracle_restart(H, wr, wi, Bcols, tries):
    """The oracle's restart sequence for one shift: trials 1..tries until
    Varah's test passes.  Returns (status, column(s))."""
    b_re = Bcols[:, 0]
    b_im = Bcols[:, 1] if Bcols.shape[1] == 2 else None
    for t in range(1, tries + 1):
        y = oracle.restart_vector(b_re, t, b_im)
        Bt = np.stack([y, np.zeros_like(y)], axis=1) if b_im is not None else y.reshape(-1, 1)
        Xo, so = oracle.hsein(H, np.array([wr]), np.array([wi]), Bt)
        if so[0] == 0:
            return 0, Xo
    return 1, None


@pytest.mark.parametrize("cplx", [False, True])
def test_restart_converges_from_an_orthogonal_start(cplx):
    inst = hi.small_instance(160, 6, 4, 41)
    n, offs = inst.n, hi.column_offsets(inst.wi)
    # the first shift of the wanted kind gets a start without left component
    l = next(i for i in range(inst.m) if (inst.wi[i] != 0) == cplx)
    lam = complex(inst.wr[l], inst.wi[l])
    B = inst.B.copy()
    B[:, offs[l]:offs[l + 1]] = _start_without_left_component(inst.H, lam, 7, cplx)
    Xo, so = oracle.hsein(inst.H, inst.wr, inst.wi, B)
    assert so[l] == 1  # precondition: the start cannot converge (oracle)
    solver = hs.Solver(n, inst.m_real, inst.m_cplx)
    dH, dwr, dwi, dB = to_dev(inst.H), to_dev(inst.wr), to_dev(inst.wi), to_dev(B)
    X, st = solver.solve(dH, dwr, dwi, dB)
    sh = st.cpu().numpy()
    assert sh[l] == 1 and np.array_equal(sh, so)
    X0 = X.cpu().numpy().copy()
    rc, k = solver.restart(dH, dwr, dwi, X, st, B=dB, max_tries=3)
    torch.cuda.synchronize()
    assert (rc, k) == (0, 1)
    sh2 = st.cpu().numpy()
    assert np.all(sh2 == 0)
    Xh = X.cpu().numpy()
    # columns that were not retried are unchanged
    keep = np.ones(Xh.shape[1], dtype=bool)
    keep[offs[l]:offs[l + 1]] = False
    assert np.array_equal(Xh[:, keep], X0[:, keep])
    # the retried column matches the oracle's restart
    s_o, Xr = _oracle_restart(inst.H, inst.wr[l], inst.wi[l], B[:, offs[l]:offs[l + 1]], 3)
    assert s_o == 0
    vo = as_vectors(Xr, np.array([inst.wr[l]]), np.array([inst.wi[l]]))[0][1]
    xg = Xh[:, offs[l]] + 1j * Xh[:, offs[l] + 1] if cplx else Xh[:, offs[l]]
    hn = oracle.hnorm_inf(inst.H)
    gap = separation(inst.eigs, lam)
    bound = angle_bound(gap, hn, n)
    assert angle(xg, vo) <= bound


def test_restart_cannot_fix_a_far_shift():
    inst = hi.small_instance(96, 3, 0, 42)
    hn = oracle.hnorm_inf(inst.H)
    wr = inst.wr.copy()
    wr[1] = 50.0 * hn  # far from every eigenvalue: no start converges
    solver = hs.Solver(inst.n, 3, 0)
    dH, dwr, dwi, dB = to_dev(inst.H), to_dev(wr), to_dev(inst.wi), to_dev(inst.B)
    X, st = solver.solve(dH, dwr, dwi, dB)
    assert st.cpu().numpy()[1] == 1
    rc, k = solver.restart(dH, dwr, dwi, X, st, B=dB, max_tries=4)
    assert (rc, k) == (1, 1)
    sh = st.cpu().numpy()
    assert sh[1] == 1 and sh[0] == 0 and sh[2] == 0
    assert not X.cpu().numpy()[:, 1].any()


def test_restart_default_start_and_split_precision():
    # no B (rho e); a far shift stays unconverged and the others untouched,
    # in the split-precision mode
    inst = hi.small_instance(192, 4, 2, 43)
    hn = oracle.hnorm_inf(inst.H)
    wr = inst.wr.copy()
    j = int(np.nonzero(inst.wi == 0)[0][0])
    wr[j] = -40.0 * hn
    solver = hs.Solver(inst.n, inst.m_real, inst.m_cplx, precision=1)
    dH, dwr, dwi = to_dev(inst.H), to_dev(wr), to_dev(inst.wi)
    X, st = solver.solve(dH, dwr, dwi)
    X0 = X.cpu().numpy().copy()
    rc, k = solver.restart(dH, dwr, dwi, X, st, max_tries=2)
    assert (rc, k) == (1, 1)
    sh = st.cpu().numpy()
    assert sh[j] == 1 and (np.delete(sh, j) == 0).all()
    assert np.array_equal(X.cpu().numpy(), X0)


def test_margins_track_the_oracle():
    # the margin is log2(||x|| / ||b||) - log2(1 / (10 n ||H|| eps)); for
    # shifts equal to eigenvalues it depends on rounding (the distance to the
    # computed spectrum), so it is compared loosely; a bookkeeping error in
    # the scale exponents would show as a gross offset
    inst = hi.small_instance(256, 24, 10, 44)
    n, offs = inst.n, hi.column_offsets(inst.wi)
    solver = hs.Solver(n, inst.m_real, inst.m_cplx, br=32, robust=True, omega_log2=60)
    solver.solve(to_dev(inst.H), to_dev(inst.wr), to_dev(inst.wi), to_dev(inst.B))
    mg = solver.margins().cpu().numpy()
    hn = oracle.hnorm_inf(inst.H)
    thr = -math.log2(10.0 * n * hn * EPS)
    mo = []
    for l in range(inst.m):
        b = inst.B[:, offs[l]:offs[l + 1]]
        if inst.wi[l] == 0:
            x, e = oracle.henry_real(inst.H, inst.wr[l], b[:, 0], log2_omega=60.0)[:2]
        else:
            x, e = oracle.henry_cplx(inst.H, complex(inst.wr[l], inst.wi[l]),
                                     b[:, 0] + 1j * b[:, 1], log2_omega=60.0)[:2]
        mo.append(math.log2(np.linalg.norm(x)) + e - math.log2(np.linalg.norm(b)) - thr)
    d = mg - np.array(mo)
    assert np.median(np.abs(d)) <= 0.5 and np.abs(d).max() <= 3.0, d


def test_restart_full_size_matches_the_oracle():
    # the benchmark workload: whatever shifts fail on this machine's instance
    # are retried, and the outcome matches the oracle's restart sequence
    inst = hi.config1()
    n, offs = inst.n, hi.column_offsets(inst.wi)
    solver = hs.Solver(n, inst.m_real, inst.m_cplx, br=64)
    dH, dwr, dwi, dB = to_dev(inst.H), to_dev(inst.wr), to_dev(inst.wi), to_dev(inst.B)
    X, st = solver.solve(dH, dwr, dwi, dB)
    failed = np.nonzero(st.cpu().numpy())[0]
    rc, k = solver.restart(dH, dwr, dwi, X, st, B=dB, max_tries=3)
    assert k == len(failed)
    sh = st.cpu().numpy()
    Xh = X.cpu().numpy()
    hn = oracle.hnorm_inf(inst.H)
    for l in failed:
        s_o, Xr = _oracle_restart(inst.H, inst.wr[l], inst.wi[l], inst.B[:, offs[l]:offs[l + 1]], 3)
        assert sh[l] == s_o
        if s_o == 0:
            vo = as_vectors(Xr, np.array([inst.wr[l]]), np.array([inst.wi[l]]))[0][1]
            c0 = offs[l]
            xg = Xh[:, c0] + 1j * Xh[:, c0 + 1] if inst.wi[l] != 0 else Xh[:, c0]
            lam = complex(inst.wr[l], inst.wi[l])
            gap = separation(inst.eigs, lam)
            bound = angle_bound(gap, hn, n)
            assert angle(xg, vo) <= bound
    assert rc == (0 if (sh == 0).all() else 1)
