"""hsein_solve_noalloc: the solve for callers that cannot allocate device
memory (it runs on the library's fixed device array instead of a workspace).

Called through the C ABI twice in a row on the same inputs; each result must
match hsein_solve's (statuses equal, eigenvectors within the angle bound the
parity tests use), and the second call must not be disturbed by what the
first left in the shared array.  This file is collected last so that a run
stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

import hsein_inputs as hi
from tests.metrics import angle, as_vectors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2101_05063_gb300 as hs  # noqa: E402


def dev(a):
    return torch.as_tensor(np.asfortranarray(a), dtype=torch.float64).cuda()


def test_noalloc_matches_workspace_solve_twice():
    inst = hi.small_instance(300, 20, 12, seed=77)
    n, m, ncol = inst.n, inst.m, inst.ncol
    plan, wbytes = hs.hsein_plan(n, inst.m_real, inst.m_cplx)
    try:
        dH, dwr, dwi, dB = dev(inst.H), dev(inst.wr), dev(inst.wi), dev(inst.B)
        work = torch.empty(wbytes, dtype=torch.uint8, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        Xref = torch.zeros((ncol, n), dtype=torch.float64, device="cuda").t()
        sref = torch.zeros(m, dtype=torch.int32, device="cuda")
        rc = hs.hsein_solve(plan, dH.data_ptr(), n, dwr.data_ptr(), dwi.data_ptr(), dB.data_ptr(), n,
                            Xref.data_ptr(), n, sref.data_ptr(), work.data_ptr(), wbytes, stream)
        assert rc == 0
        torch.cuda.synchronize()
        Xr, sr = Xref.cpu().numpy(), sref.cpu().numpy()
        for call in range(2):
            X = torch.full((ncol, n), np.nan, dtype=torch.float64, device="cuda").t()
            st = torch.full((m,), -9, dtype=torch.int32, device="cuda")
            rc = hs.hsein_solve_noalloc(plan, dH.data_ptr(), n, dwr.data_ptr(), dwi.data_ptr(),
                                        dB.data_ptr(), n, X.data_ptr(), n, st.data_ptr(), stream)
            assert rc == 0, (call, rc)
            torch.cuda.synchronize()
            Xg, sg = X.cpu().numpy(), st.cpu().numpy()
            assert np.array_equal(sg, sr), call
            assert np.all(np.isfinite(Xg))
            for l, ((_, xg), (_, xr)) in enumerate(zip(as_vectors(Xg, inst.wr, inst.wi),
                                                       as_vectors(Xr, inst.wr, inst.wi))):
                if sr[l] == 0:
                    assert angle(xg, xr) <= 1e-10, (call, l)
                else:
                    assert np.all(xg == 0.0)
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
