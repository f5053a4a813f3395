"""Power-of-two balancing (hsein_balance / hsein_unbalance), the option that
lets graded matrices use the split-precision products.

Pins: the balanced matrix is exactly D^-1 H D on the Hessenberg pattern
(power-of-two scaling, checked entry by entry); balancing removes a
power-of-two grading; the split-precision solve of a balanced graded matrix
matches the oracle on the same balanced matrix; the map back equals an
extended-precision D x / ||D x||; a serving request on a balanced matrix
equals the standalone solve mapped back.
"""
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


def _graded(inst, u):
    d = 2.0 ** u if u.dtype.kind == "i" else 10.0 ** u
    return np.asfortranarray(inst.H * d[:, None] / d[None, :])


def _row_col_log_ratio(H):
    A = np.abs(H.astype(np.longdouble))
    np.fill_diagonal(A, 0)
    r, c = A.sum(axis=1), A.sum(axis=0)
    return np.abs(np.log2(r / c).astype(np.float64))


def test_balance_is_an_exact_similarity():
    inst = hi.small_instance(150, 4, 2, 31)
    Hg = _graded(inst, hi.uniform(31, 9, inst.n, -120.0, 120.0))
    Hb, e = hs.balance(to_dev(Hg))
    Hb, e = Hb.cpu().numpy(), e.cpu().numpy().astype(np.int64)
    n = inst.n
    i, j = np.indices((n, n))
    expect = np.where(i <= j + 1, np.ldexp(Hg, e[None, :] - e[:, None]), 0.0)
    assert np.array_equal(Hb, expect)


def test_balance_removes_a_power_of_two_grading():
    inst = hi.small_instance(200, 4, 2, 32)
    u = np.rint(hi.uniform(32, 9, inst.n, -400.0, 400.0)).astype(np.int64)
    Hg = _graded(inst, u)
    before = _row_col_log_ratio(Hg).max()
    Hb, e = hs.balance(to_dev(Hg))
    after = _row_col_log_ratio(Hb.cpu().numpy()).max()
    assert before > 100 and after <= max(6.0, _row_col_log_ratio(inst.H).max() + 2)


@pytest.mark.parametrize("n,mr,mc,seed", [(160, 6, 4, 33), (300, 8, 5, 34)])
def test_balanced_split_solve_matches_the_oracle(n, mr, mc, seed):
    # a graded matrix (10^u, u ~ U[-150, 150]) solved on its balanced form
    # with the split-precision products: parity with the oracle on the same
    # balanced matrix, in the balanced basis (the map back is exact up to
    # rounding and pinned separately; in the graded basis the angle is
    # dominated by components that D amplifies, which no FP64 reference
    # resolves)
    inst = hi.small_instance(n, mr, mc, seed)
    Hg = _graded(inst, hi.uniform(seed, 9, n, -150.0, 150.0))
    dHb, e = hs.balance(to_dev(Hg))
    Hb = dHb.cpu().numpy()
    s = hs.Solver(n, mr, mc, precision=1)
    X, st = s.solve(dHb, to_dev(inst.wr), to_dev(inst.wi))
    Xh, sh = X.cpu().numpy(), st.cpu().numpy()
    Xo, so = oracle.hsein(Hb, inst.wr, inst.wi)
    assert np.array_equal(sh, so)
    hn = oracle.hnorm_inf(Hb)
    offs = hi.column_offsets(inst.wi)
    vo = as_vectors(Xo, inst.wr, inst.wi)
    checked = 0
    for l in range(inst.m):
        if sh[l] != 0:
            continue
        c0 = offs[l]
        xg = Xh[:, c0] + 1j * Xh[:, c0 + 1] if inst.wi[l] != 0 else Xh[:, c0]
        gap = separation(inst.eigs, vo[l][0])
        bound = angle_bound(gap, hn, n)
        assert angle(xg, vo[l][1]) <= bound, (l, angle(xg, vo[l][1]), bound)
        checked += 1
    assert checked >= inst.m // 2
    # the balanced matrix is well scaled: the graded one is not
    assert _row_col_log_ratio(Hb).max() < 8 < _row_col_log_ratio(Hg).max()


def test_unbalance_matches_extended_precision():
    n, ncol = 90, 5
    wi = np.array([0.0, 1.5, 0.0, 0.0])  # columns: 1 + 2 + 1 + 1
    X = hi.unit_columns(n, ncol, seed=35)
    X[:, 3] = 0.0  # a not-converged column stays zero
    e = np.rint(hi.uniform(35, 2, n, -600.0, 600.0)).astype(np.int32)
    dX = to_dev(X)
    hs.unbalance(dX, to_dev(wi), torch.as_tensor(e, device="cuda"))
    got = dX.cpu().numpy()
    D = np.ldexp(np.longdouble(1.0), e.astype(np.int64))
    for c0, c1 in [(0, 1), (1, 3), (3, 4), (4, 5)]:
        Y = X[:, c0:c1].astype(np.longdouble) * D[:, None]
        nrm = np.sqrt((Y * Y).sum())
        want = (Y / nrm if nrm > 0 else Y).astype(np.float64)
        assert np.abs(got[:, c0:c1] - want).max() <= 4 * EPS


def test_server_request_on_a_balanced_matrix():
    inst = hi.small_instance(192, 5, 3, 36)
    Hg = _graded(inst, hi.uniform(36, 9, inst.n, -150.0, 150.0))
    dHb, e = hs.balance(to_dev(Hg))
    dwr, dwi = to_dev(inst.wr), to_dev(inst.wi)
    srv = hs.Server(1 << 30, max_jobs=2, max_merge_shifts=64)
    t = srv.submit(dHb, dwr, dwi, precision=1, exps=e)
    while t not in srv.progress(wait=True):
        pass
    X, st = srv.result(t)
    s = hs.Solver(inst.n, inst.m_real, inst.m_cplx, precision=1)
    Xa, sa = s.solve(dHb, dwr, dwi)
    hs.unbalance(Xa, dwi, e)
    assert np.array_equal(st.cpu().numpy(), sa.cpu().numpy())
    assert np.array_equal(X.cpu().numpy(), Xa.cpu().numpy())
