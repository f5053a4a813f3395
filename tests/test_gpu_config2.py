"""Full-size parity on the precision workload (n = 8192, 2048 real shifts,
eigenvalues U[-n, n] with minimum gap 1e-2), in both precision modes.

The oracle solves a seeded sample of 12 shifts one by one; every converged
column must satisfy the residual bound (FP64 product on the GPU, test
infrastructure only); the split-precision results must also agree with the
FP64 path's (angle bound of the separation gate).
"""
import numpy as np
import pytest

import hsein_inputs as hi
import oracle
from tests.metrics import EPS, angle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2101_05063_gb300 as hs  # noqa: E402
from tests.test_gpu_parity import separation, to_dev  # noqa: E402


@pytest.fixture(scope="module")
def c2():
    inst = hi.config2()
    dev = dict(H=to_dev(inst.H), wr=to_dev(inst.wr), wi=to_dev(inst.wi), B=to_dev(inst.B),
               Q0=to_dev(inst.Q0))
    sample = np.sort(np.argsort(hi.uniform(77, 1, inst.m), kind="stable")[:12])
    Xo, so = oracle.hsein(inst.H, inst.wr[sample], inst.wi[sample], inst.B[:, sample])
    results = {}
    for precision in (0, 1):
        solver = hs.Solver(inst.n, inst.m_real, inst.m_cplx, br=64, precision=precision)
        X, st = solver.solve(dev["H"], dev["wr"], dev["wi"], dev["B"])
        Z = solver.backtransform(dev["Q0"], X)
        HX = dev["H"] @ X
        torch.cuda.synchronize()
        results[precision] = (X.cpu().numpy(), st.cpu().numpy(), Z.cpu().numpy(), HX.cpu().numpy())
        del solver, X, Z, HX
    return inst, sample, Xo, so, results


@pytest.mark.parametrize("precision", [0, 1])
def test_config2_residuals_and_oracle_sample(c2, precision):
    inst, sample, Xo, so, results = c2
    X, st, Z, HX = results[precision]
    n = inst.n
    assert np.all(np.isfinite(X)) and np.all(np.isfinite(Z))
    hn1 = np.abs(inst.H).sum(axis=0).max()
    ok = st == 0
    assert ok.sum() >= inst.m - 8
    for l in np.nonzero(ok)[0]:
        x, hx = X[:, l], HX[:, l]
        r = np.abs(hx - inst.wr[l] * x).sum() / (hn1 * np.abs(x).sum())
        assert r <= 100 * n * EPS, (l, r / (n * EPS))
    assert np.array_equal(st[sample], so)
    hn = oracle.hnorm_inf(inst.H)
    for j, l in enumerate(sample):
        if st[l] != 0:
            continue
        gap = separation(inst.eigs, inst.wr[l])
        bound = 1e-10 if gap >= 1e-3 * hn else max(1e-10, 1e3 * n * EPS * hn / gap)
        assert angle(X[:, l], Xo[:, j]) <= bound, (l, angle(X[:, l], Xo[:, j]), gap)


def test_config2_split_matches_fp64_path(c2):
    inst, sample, Xo, so, results = c2
    X0, s0, Z0, _ = results[0]
    X1, s1, Z1, _ = results[1]
    n = inst.n
    assert np.array_equal(s0, s1)
    hn = oracle.hnorm_inf(inst.H)
    for l in np.nonzero(s0 == 0)[0]:
        gap = separation(inst.eigs, inst.wr[l])
        bound = 1e-10 if gap >= 1e-3 * hn else max(1e-10, 1e3 * n * EPS * hn / gap)
        assert angle(X0[:, l], X1[:, l]) <= bound, l
        assert angle(Z0[:, l], Z1[:, l]) <= bound, l
