"""hsein_solve_noalloc: the solve for callers that cannot allocate device
memory (plug-ins whose host framework owns all device memory, real-time
paths that must not call an allocator); it runs on the library's fixed
device array instead of a caller's workspace.

Called through the C ABI; each result must equal hsein_solve's on the same
inputs bit for bit (the same kernels on the same data), on two calls in a
row, and match the oracle within the parity tests' angle gate.  Before the
checked calls, a call on a different instance (another size, complex pairs,
a graded matrix whose solve rescales) leaves its state in the shared array,
so a stale value would show.  A split-precision plan alternates hsein_solve
and hsein_solve_noalloc, so its tensor maps are rebuilt over both
addresses.  This file is collected last so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest

import hsein_inputs as hi
import oracle
from tests.metrics import angle, angle_bound, as_vectors, separation

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2101_05063_gb300 as hs  # noqa: E402


def dev(a):
    return torch.as_tensor(np.asfortranarray(a), dtype=torch.float64).cuda()


def _plan(n, mr, mc, precision=0, omega_log2=1000):
    opt = hs.hsein_default_options()
    opt.precision = precision
    opt.omega_log2 = omega_log2
    return hs.hsein_plan(n, mr, mc, opt)


def _solve(plan, n, ncol, m, d, work=None, wbytes=0):
    """One call through the C ABI: hsein_solve with `work`, or
    hsein_solve_noalloc when work is None.  Returns (X, status) on the host."""
    stream = torch.cuda.current_stream().cuda_stream
    X = torch.full((ncol, n), np.nan, dtype=torch.float64, device="cuda").t()
    st = torch.full((m,), -9, dtype=torch.int32, device="cuda")
    args = (plan, d["H"].data_ptr(), n, d["wr"].data_ptr(), d["wi"].data_ptr(),
            d["B"].data_ptr(), n, X.data_ptr(), n, st.data_ptr())
    if work is None:
        rc = hs.hsein_solve_noalloc(*args, stream)
    else:
        rc = hs.hsein_solve(*args, work.data_ptr(), wbytes, stream)
    assert rc == 0, rc
    torch.cuda.synchronize()
    return X.cpu().numpy(), st.cpu().numpy()


def _graded_call():
    # another size, a graded matrix whose solve rescales (lowered threshold),
    # and a complex shift: its state is what the next call finds in the array
    n = 96
    H0 = np.triu(hi.normal(11, 50, n * n).reshape(n, n, order="F"), -1)
    G, _ = hi.graded(H0, seed=11, umax=150.0, monotone=True)
    ev = np.linalg.eigvals(H0)
    lam_r = float(ev[np.argmin(np.abs(ev.imag))].real)
    lam_c = ev[np.argmax(ev.imag)]
    wr, wi = np.array([lam_r, lam_c.real]), np.array([0.0, lam_c.imag])
    B = hi.unit_columns(n, 3, seed=12)
    plan, _ = _plan(n, 1, 1, omega_log2=40)
    try:
        d = dict(H=dev(G), wr=dev(wr), wi=dev(wi), B=dev(B))
        X, st = _solve(plan, n, 3, 2, d)
        assert np.all(np.isfinite(X)) and np.all((st == 0) | (st == 1))
    finally:
        hs.hsein_plan_destroy(plan)


def _check_against_oracle(inst, X, st):
    Xo, so = oracle.hsein(inst.H, inst.wr, inst.wi, inst.B)
    assert np.array_equal(st, so)
    hn = oracle.hnorm_inf(inst.H)
    for l, ((lam, xg), (_, xo)) in enumerate(zip(as_vectors(X, inst.wr, inst.wi),
                                                as_vectors(Xo, inst.wr, inst.wi))):
        if st[l] == 0:
            assert angle(xg, xo) <= angle_bound(separation(inst.eigs, lam), hn, inst.n), l
        else:
            assert np.all(xg == 0.0)


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_equals_workspace_solve(precision):
    inst = hi.small_instance(300, 20, 12, seed=77)
    n, m, ncol = inst.n, inst.m, inst.ncol
    plan, wbytes = _plan(n, inst.m_real, inst.m_cplx, precision=precision)
    try:
        assert wbytes <= 16 << 20
        d = dict(H=dev(inst.H), wr=dev(inst.wr), wi=dev(inst.wi), B=dev(inst.B))
        work = torch.empty(wbytes, dtype=torch.uint8, device="cuda")
        Xr, sr = _solve(plan, n, ncol, m, d, work, wbytes)
        _check_against_oracle(inst, Xr, sr)
        _graded_call()
        for call in range(2):
            X, st = _solve(plan, n, ncol, m, d)  # no workspace: the fixed array
            assert np.array_equal(st, sr), call
            assert np.array_equal(X, Xr), call
            # back to the caller's workspace on the same plan, then again
            X2, st2 = _solve(plan, n, ncol, m, d, work, wbytes)
            assert np.array_equal(st2, sr) and np.array_equal(X2, Xr), call
    finally:
        hs.hsein_plan_destroy(plan)


def test_noalloc_rejects_plans_beyond_its_array():
    plan, wbytes = hs.hsein_plan(4096, 1024, 0)
    try:
        assert wbytes > 16 << 20
        dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
        p = dummy.data_ptr()
        rc = hs.hsein_solve_noalloc(plan, p, 4096, p, p, p, 4096, p, 4096, p,
                                    torch.cuda.current_stream().cuda_stream)
        assert rc == -2
    finally:
        hs.hsein_plan_destroy(plan)
