"""Full-size parity on the mixed real/complex workload (n = 4096, 512 real +
256 complex shifts, tile height 64: the configuration bench.py times), in
both precision modes.

The oracle solves every shift one by one (Henry per shift, OpenMP over
shifts).  Every status must match; every converged column must match the
oracle's within the angle gate (tests.metrics.angle_bound) and satisfy the
residual bound 100 n eps (FP64 product on the GPU, test infrastructure only);
z = Q0 x must match numpy's product of the same operands and the oracle's
z within the same gate.  The worst angle / first-order-bound ratio is printed.
"""
import numpy as np
import pytest

import hsein_inputs as hi
import oracle
from tests.metrics import EPS, angle, angle_bound, as_vectors, first_order_bound, separation

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2101_05063_gb300 as hs  # noqa: E402
from tests.test_gpu_parity import to_dev  # noqa: E402


@pytest.fixture(scope="module")
def c1():
    inst = hi.config1()
    Xo, so = oracle.hsein(inst.H, inst.wr, inst.wi, inst.B)
    Zo = oracle.q0_apply(inst.Q0, Xo)
    return inst, Xo, so, Zo


@pytest.mark.parametrize("precision", [0, 1])
def test_config1_full_size(c1, precision):
    inst, Xo, so, Zo = c1
    n = inst.n
    solver = hs.Solver(n, inst.m_real, inst.m_cplx, br=64, precision=precision)
    dH = to_dev(inst.H)
    X, status = solver.solve(dH, to_dev(inst.wr), to_dev(inst.wi), to_dev(inst.B))
    Z = solver.backtransform(to_dev(inst.Q0), X)
    torch.cuda.synchronize()
    Xh, sh, Zh = X.cpu().numpy(), status.cpu().numpy(), Z.cpu().numpy()
    assert np.all(np.isfinite(Xh)) and np.all(np.isfinite(Zh))
    assert np.array_equal(sh, so), np.nonzero(sh != so)
    # residual of every converged column, FP64 on the device
    HX = (dH @ X).cpu().numpy()
    hn1 = np.abs(inst.H).sum(axis=0).max()
    hn = oracle.hnorm_inf(inst.H)
    vg, vo = as_vectors(Xh, inst.wr, inst.wi), as_vectors(Xo, inst.wr, inst.wi)
    hx = as_vectors(HX, inst.wr, inst.wi)
    zg, zo = as_vectors(Zh, inst.wr, inst.wi), as_vectors(Zo, inst.wr, inst.wi)
    worst, worst_x, checked = 0.0, 0.0, 0
    for l in range(inst.m):
        if sh[l] != 0:
            continue
        lam, x = vg[l]
        r = np.abs(hx[l][1] - lam * x).sum() / (hn1 * np.abs(x).sum())
        assert r <= 100 * n * EPS, (l, r / (n * EPS))
        gap = separation(inst.eigs, lam)
        bound = angle_bound(gap, hn, n)
        a = angle(x, vo[l][1])
        assert a <= bound, (l, lam, a, gap, bound)
        az = angle(zg[l][1], zo[l][1])
        assert az <= bound, (l, lam, az, gap, bound)
        worst = max(worst, a / first_order_bound(gap, hn, n))
        worst_x = max(worst_x, a)
        checked += 1
    # z = Q0 x against numpy's product of the same operands
    assert np.abs(Zh - inst.Q0 @ Xh).max() <= 1e-12
    print("config1 precision %d: %d columns vs the oracle, max angle %.3g, worst angle / "
          "(n eps ||H|| / gap) = %.3g" % (precision, checked, worst_x, worst))
