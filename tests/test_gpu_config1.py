"""Full-size parity on the benchmark workload (n = 4096, 512 real + 256
complex shifts, tile height 64: the configuration bench.py times).

The oracle solves a seeded sample of 24 shifts one by one (Henry per shift);
those columns must match within the angle bounds.  Every converged column must
satisfy the residual bound (computed here with an FP64 product on the GPU,
test infrastructure only), and every status must match Varah's test recomputed
from the oracle's sampled shifts.
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
from tests.test_gpu_parity import separation, to_dev  # noqa: E402


@pytest.fixture(scope="module")
def c1():
    return hi.config1()


@pytest.mark.parametrize("precision", [0, 1])
def test_config1_full_size(c1, precision):
    inst = c1
    n = inst.n
    solver = hs.Solver(n, inst.m_real, inst.m_cplx, br=64, precision=precision)
    dH = to_dev(inst.H)
    X, status = solver.solve(dH, to_dev(inst.wr), to_dev(inst.wi), to_dev(inst.B))
    Z = solver.backtransform(to_dev(inst.Q0), X)
    torch.cuda.synchronize()
    Xh, sh = X.cpu().numpy(), status.cpu().numpy()
    assert np.all(np.isfinite(Xh))
    # residual of every converged column, FP64 on the device
    offs = hi.column_offsets(inst.wi)
    HX = (dH @ X).cpu().numpy()
    hn1 = np.abs(inst.H).sum(axis=0).max()
    for l in range(inst.m):
        if sh[l] != 0:
            continue
        c0 = offs[l]
        if inst.wi[l] != 0:
            lam = complex(inst.wr[l], inst.wi[l])
            x = Xh[:, c0] + 1j * Xh[:, c0 + 1]
            hx = HX[:, c0] + 1j * HX[:, c0 + 1]
        else:
            lam, x, hx = inst.wr[l], Xh[:, c0], HX[:, c0]
        r = np.abs(hx - lam * x).sum() / (hn1 * np.abs(x).sum())
        assert r <= 100 * n * EPS, (l, r / (n * EPS))
    # z = Q0 x
    Zh = Z.cpu().numpy()
    assert np.abs(Zh - inst.Q0 @ Xh).max() <= 1e-12
    # sampled oracle columns
    rng = np.argsort(hi.uniform(99, 1, inst.m), kind="stable")[:24]
    wr, wi = inst.wr[rng], inst.wi[rng]
    Bs = np.concatenate([inst.B[:, offs[l]:offs[l + 1]] for l in rng], axis=1)
    Xo, so = oracle.hsein(inst.H, wr, wi, Bs)
    assert np.array_equal(so, sh[rng])
    hn = oracle.hnorm_inf(inst.H)
    vo = as_vectors(Xo, wr, wi)
    for j, l in enumerate(rng):
        if sh[l] != 0:
            continue
        c0 = offs[l]
        xg = Xh[:, c0] + 1j * Xh[:, c0 + 1] if inst.wi[l] != 0 else Xh[:, c0]
        lam = vo[j][0]
        gap = separation(inst.eigs, lam)
        bound = 1e-10 if gap >= 1e-3 * hn else max(1e-10, 1e3 * n * EPS * hn / gap)
        assert angle(xg, vo[j][1]) <= bound, (l, lam, angle(xg, vo[j][1]), gap)
