"""The Householder reduction A = Q0 H Q0^T on the GPU (hsein_gehrd), the
precursor step of Sec. 1 that produces H and Q0.

Parity: H and Q0 entry by entry against the oracle's reduction, which takes
the same reflector convention (alpha = -sign(x_1) ||x||), at sizes spanning
several 256-row blocks and 64-column chunks with ragged tails.  Invariants at
every size: exact zeros below the first subdiagonal, Q0^T Q0 = I, Q0 H Q0^T =
A.  Special cases: n = 1 and 2 (no reflector), a triangular A (every column
already reduced: H = A and Q0 = I exactly), a padded leading dimension.  End
to end: A -> (H, Q0) -> solve -> backtransform gives eigenvectors of A.
"""
import numpy as np
import pytest

import hsein_inputs as hi
import oracle
from tests.metrics import EPS

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2101_05063_gb300 as hs  # noqa: E402
from tests.test_gpu_parity import to_dev  # noqa: E402


def _invariants(A, H, Q):
    n = A.shape[0]
    assert np.all(np.tril(H, -2) == 0.0)
    assert np.abs(Q.T @ Q - np.eye(n)).max() <= 20 * n * EPS
    assert np.abs(Q @ H @ Q.T - A).max() <= 20 * n * EPS * np.abs(A).max() * np.sqrt(n)


@pytest.mark.parametrize("n,seed", [(1, 1), (2, 2), (3, 3), (17, 4), (130, 5), (300, 6), (517, 7)])
def test_gehrd_matches_oracle(n, seed):
    A = hi.normal(seed, 62, n * n).reshape(n, n, order="F")
    Hg, Qg = hs.gehrd(to_dev(A))
    Hg, Qg = Hg.cpu().numpy(), Qg.cpu().numpy()
    Ho, Qo = oracle.gehrd(A)
    scale = np.abs(A).max()
    assert np.abs(Hg - Ho).max() <= 1e-10 * scale
    assert np.abs(Qg - Qo).max() <= 1e-10
    _invariants(A, Hg, Qg)


def test_gehrd_triangular_input_is_exact():
    n = 200
    A = np.triu(hi.normal(8, 62, n * n).reshape(n, n, order="F"))
    Hg, Qg = hs.gehrd(to_dev(A))
    assert np.array_equal(Hg.cpu().numpy(), A)
    assert np.array_equal(Qg.cpu().numpy(), np.eye(n))


def test_gehrd_padded_leading_dimension():
    n, lda = 150, 163
    Ap = hi.normal(9, 62, lda * n).reshape(lda, n, order="F")
    dAp = to_dev(Ap)
    dA = dAp[:n, :]  # column-major view with leading dimension lda
    H, Q = hs.gehrd(dA)
    Ho, Qo = oracle.gehrd(np.asfortranarray(Ap[:n, :]))
    assert np.abs(H.cpu().numpy() - Ho).max() <= 1e-10 * np.abs(Ap).max()
    assert np.abs(Q.cpu().numpy() - Qo).max() <= 1e-10
    assert torch.equal(dAp, to_dev(Ap))  # A is not modified


def test_gehrd_argument_errors():
    n = 8
    A = to_dev(np.eye(n))
    rc, wb = hs.hsein_gehrd_workspace(n)
    assert rc == 0 and wb > 0
    assert hs.hsein_gehrd_workspace(0)[0] == -1
    work = torch.empty(wb, dtype=torch.uint8, device="cuda")
    H = torch.empty((n, n), dtype=torch.float64, device="cuda").t()
    st = torch.cuda.current_stream().cuda_stream
    # H aliasing A, too small a workspace, a short leading dimension
    assert hs.hsein_gehrd(n, A.data_ptr(), n, A.data_ptr(), n, H.data_ptr(), n, work.data_ptr(),
                          wb, st) == -1
    assert hs.hsein_gehrd(n, A.data_ptr(), n, H.data_ptr(), n, A.data_ptr() + 0, n,
                          work.data_ptr(), wb, st) == -1
    Q = torch.empty((n, n), dtype=torch.float64, device="cuda").t()
    assert hs.hsein_gehrd(n, A.data_ptr(), n, H.data_ptr(), n, Q.data_ptr(), n, work.data_ptr(),
                          wb - 1, st) == -2
    assert hs.hsein_gehrd(n, A.data_ptr(), n - 1, H.data_ptr(), n, Q.data_ptr(), n,
                          work.data_ptr(), wb, st) == -1


def test_gehrd_then_solve_gives_eigenvectors_of_a():
    inst = hi.small_instance(384, 10, 6, 40, keep_a=True)
    A = inst.A
    dH, dQ = hs.gehrd(to_dev(A))
    s = hs.Solver(inst.n, inst.m_real, inst.m_cplx)
    X, st = s.solve(dH, to_dev(inst.wr), to_dev(inst.wi))
    Z = s.backtransform(dQ, X).cpu().numpy()
    st = st.cpu().numpy()
    assert np.count_nonzero(st == 0) >= inst.m - 1
    offs = hi.column_offsets(inst.wi)
    a1 = np.abs(A).sum(axis=0).max()
    for l in range(inst.m):
        if st[l]:
            continue
        c0 = offs[l]
        if inst.wi[l] != 0:
            lam, z = complex(inst.wr[l], inst.wi[l]), Z[:, c0] + 1j * Z[:, c0 + 1]
        else:
            lam, z = inst.wr[l], Z[:, c0]
        r = np.abs(A @ z - lam * z).sum() / (a1 * np.abs(z).sum())
        assert r <= 100 * inst.n * EPS, (l, r)


@pytest.mark.parametrize("case", ["normal2048", "config1"])
def test_gehrd_full_size_properties(case):
    # sizes whose early steps take the wide tile shapes (two and four rows per
    # thread): invariants on the GPU and |H| against LAPACK's reduction (no
    # oracle run at these sizes)
    import scipy.linalg
    if case == "config1":
        inst = hi.config1(keep_a=True)
        A, Hs = inst.A, inst.H
    else:
        n = 2048
        A = hi.normal(11, 62, n * n).reshape(n, n, order="F")
        Hs = np.triu(scipy.linalg.hessenberg(A), -1)
    n = A.shape[0]
    dA = to_dev(A)
    dH, dQ = hs.gehrd(dA)
    i, j = torch.meshgrid(torch.arange(n, device="cuda"), torch.arange(n, device="cuda"),
                          indexing="ij")
    assert bool((dH[i > j + 1] == 0).all())
    eye = torch.eye(n, dtype=torch.float64, device="cuda")
    assert float((dQ.t() @ dQ - eye).abs().max()) <= 20 * n * EPS
    back = dQ @ dH @ dQ.t()
    assert float((back - dA).abs().max()) <= 20 * n * EPS * float(dA.abs().max()) * np.sqrt(n)
    # |H| agrees with the LAPACK reduction (unique up to reflector signs)
    assert np.abs(np.abs(dH.cpu().numpy()) - np.abs(Hs)).max() <= 1e-8 * np.abs(A).max()
