"""The comparison baselines on the GPU against the oracle -- the same
statuses and angles as the tiled path must meet, through the scaling paths,
with the default starting vector, real and complex shifts, and on the
n = 4096 mixed workload (sampled shifts):
  method = 1: Henry's RQ solve per shift, unblocked (Alg. "henry", the RQIN
              of Sec. 5), against the RQ oracle;
  method = 2: the LU approach per shift (Sec. 2.1, LAPACK's inverse
              iteration), against the LU oracle (oracle.hsein_lu) and the RQ
              oracle (both solve the same systems).
"""
import numpy as np
import pytest

import hsein_inputs as hi
import oracle
from tests.metrics import EPS, angle, residual

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2101_05063_gb300 as hs  # noqa: E402
from tests.test_gpu_parity import compare, to_dev  # noqa: E402


def run_henry(H, wr, wi, B, robust=True, omega_log2=1000, method=1):
    wr = np.asarray(wr, dtype=np.float64)
    wi = np.asarray(wi, dtype=np.float64)
    mc = int(np.count_nonzero(wi))
    s = hs.Solver(H.shape[0], len(wr) - mc, mc, robust=robust, omega_log2=omega_log2,
                  method=method)
    X, st = s.solve(to_dev(H), to_dev(wr), to_dev(wi), to_dev(B) if B is not None else None)
    return X.cpu().numpy(), st.cpu().numpy()


@pytest.mark.parametrize("n,mr,mc,seed", [(2, 1, 0, 1), (9, 3, 2, 2), (65, 6, 4, 3), (200, 12, 8, 4),
                                          (333, 9, 0, 5), (300, 0, 10, 6)])
def test_baseline_matches_oracle(n, mr, mc, seed):
    inst = hi.small_instance(max(n, 8), mr, mc, seed) if n > 2 else None
    if inst is None:
        H = np.array([[1.0, 2.0], [3.0, -1.0]])
        wr, wi, B, eigs = np.array([np.sqrt(7.0)]), np.array([0.0]), np.ones((2, 1)), np.array(
            [np.sqrt(7.0), -np.sqrt(7.0)])
    else:
        H, wr, wi, B, eigs = inst.H, inst.wr, inst.wi, inst.B, inst.eigs
    Xg, sg = run_henry(H, wr, wi, B)
    Xo, so = oracle.hsein(H, wr, wi, B)
    compare(H, wr, wi, Xg, sg, Xo, so, eigs)


def test_baseline_default_starting_vector():
    inst = hi.small_instance(150, 10, 6, 21)
    Xg, sg = run_henry(inst.H, inst.wr, inst.wi, None)
    Xo, so = oracle.hsein(inst.H, inst.wr, inst.wi, None)
    compare(inst.H, inst.wr, inst.wi, Xg, sg, Xo, so, inst.eigs)


@pytest.mark.parametrize("n,om", [(48, 30), (200, 60)])
def test_baseline_bad_system_scaling(n, om):
    # the bad system of Sec. 5.2 with lowered thresholds: ProtectDivision and
    # ProtectUpdate rescale the whole vector
    H = hi.paper_h2(n)
    B = np.ones((n, 1)) / np.sqrt(n)
    Xg, sg = run_henry(H, [2.0], [0.0], B, omega_log2=om)
    Xo, so = oracle.hsein(H, [2.0], [0.0], B, log2_omega=om)
    assert sg[0] == 0 and so[0] == 0
    assert np.all(np.isfinite(Xg))
    assert angle(Xg[:, 0], Xo[:, 0]) <= 1e-12
    assert residual(H, 2.0, Xg[:, 0]) <= 100 * n * EPS


def test_baseline_full_size_sample():
    inst = hi.config1()
    n, offs = inst.n, hi.column_offsets(inst.wi)
    rng = np.argsort(hi.uniform(98, 1, inst.m), kind="stable")[:12]
    wr, wi = inst.wr[rng], inst.wi[rng]
    B = np.concatenate([inst.B[:, offs[l]:offs[l + 1]] for l in rng], axis=1)
    Xg, sg = run_henry(inst.H, wr, wi, B)
    Xo, so = oracle.hsein(inst.H, wr, wi, B)
    compare(inst.H, wr, wi, Xg, sg, Xo, so, inst.eigs)
    # every converged column meets the residual bound
    H = to_dev(inst.H)
    HX = (H @ to_dev(Xg)).cpu().numpy()
    hn1 = np.abs(inst.H).sum(axis=0).max()
    o2 = hi.column_offsets(wi)
    for j in range(len(rng)):
        if sg[j]:
            continue
        c0 = o2[j]
        if wi[j] != 0:
            lam = complex(wr[j], wi[j])
            x, hx = Xg[:, c0] + 1j * Xg[:, c0 + 1], HX[:, c0] + 1j * HX[:, c0 + 1]
        else:
            lam, x, hx = wr[j], Xg[:, c0], HX[:, c0]
        assert np.abs(hx - lam * x).sum() / (hn1 * np.abs(x).sum()) <= 100 * n * EPS


# ------------------------------------------------ method 2: the LU approach

def run_lu(H, wr, wi, B, robust=True, omega_log2=1000):
    return run_henry(H, wr, wi, B, robust=robust, omega_log2=omega_log2, method=2)


@pytest.mark.parametrize("n,mr,mc,seed", [(2, 1, 0, 1), (9, 3, 2, 2), (65, 6, 4, 3), (200, 12, 8, 4),
                                          (333, 9, 0, 5), (300, 0, 10, 6), (520, 7, 5, 7)])
def test_lu_baseline_matches_oracles(n, mr, mc, seed):
    if n == 2:
        H = np.array([[1.0, 2.0], [3.0, -1.0]])
        wr, wi, B = np.array([np.sqrt(7.0)]), np.array([0.0]), np.ones((2, 1))
        eigs = np.array([np.sqrt(7.0), -np.sqrt(7.0)])
    else:
        inst = hi.small_instance(n, mr, mc, seed)
        H, wr, wi, B, eigs = inst.H, inst.wr, inst.wi, inst.B, inst.eigs
    Xg, sg = run_lu(H, wr, wi, B)
    Xl, sl = oracle.hsein_lu(H, wr, wi, B)
    compare(H, wr, wi, Xg, sg, Xl, sl, eigs)
    Xo, so = oracle.hsein(H, wr, wi, B)
    compare(H, wr, wi, Xg, sg, Xo, so, eigs)


def test_lu_baseline_default_starting_vector():
    inst = hi.small_instance(150, 10, 6, 21)
    Xg, sg = run_lu(inst.H, inst.wr, inst.wi, None)
    Xl, sl = oracle.hsein_lu(inst.H, inst.wr, inst.wi, None)
    compare(inst.H, inst.wr, inst.wi, Xg, sg, Xl, sl, inst.eigs)


def test_lu_baseline_scaling_paths():
    # back-substitution growth (1e200 per row) and forward-substitution
    # growth (b near the top of the double range): the GPU solve rescales and
    # matches the oracle's direction; the bad system with a lowered threshold
    n = 6
    H = np.eye(n) + 1e200 * np.triu(np.ones((n, n)), 1) + 1e-3 * np.diag(np.ones(n - 1), -1)
    b = np.ones((n, 1))
    Xg, sg = run_lu(H, [0.5], [0.0], b)
    Xl, sl = oracle.hsein_lu(H, [0.5], [0.0], b)
    assert np.all(np.isfinite(Xg)) and sg[0] == sl[0]
    if sl[0] == 0:
        assert angle(Xg[:, 0], Xl[:, 0]) <= 1e-12
    m = 9
    H = np.eye(m) - np.diag(np.ones(m - 1), -1)
    b = np.full((m, 1), 1e308)
    Xg, sg = run_lu(H, [0.0], [0.0], b)
    Xl, sl = oracle.hsein_lu(H, [0.0], [0.0], b)
    assert np.all(np.isfinite(Xg)) and sg[0] == sl[0]
    if sl[0] == 0:
        assert angle(Xg[:, 0], np.arange(1.0, m + 1)) <= 4 * m * EPS
    for n, om in ((48, 30), (200, 60)):
        H = hi.paper_h2(n)
        B = np.ones((n, 1)) / np.sqrt(n)
        Xg, sg = run_lu(H, [2.0], [0.0], B, omega_log2=om)
        Xl, sl = oracle.hsein_lu(H, [2.0], [0.0], B, log2_omega=om)
        assert sg[0] == sl[0] == 0 and np.all(np.isfinite(Xg))
        assert angle(Xg[:, 0], Xl[:, 0]) <= 1e-12
        assert residual(H, 2.0, Xg[:, 0]) <= 100 * n * EPS


def test_lu_baseline_full_size_sample():
    inst = hi.config1()
    offs = hi.column_offsets(inst.wi)
    rng = np.argsort(hi.uniform(97, 1, inst.m), kind="stable")[:12]
    wr, wi = inst.wr[rng], inst.wi[rng]
    B = np.concatenate([inst.B[:, offs[l]:offs[l + 1]] for l in rng], axis=1)
    Xg, sg = run_lu(inst.H, wr, wi, B)
    Xo, so = oracle.hsein(inst.H, wr, wi, B)
    compare(inst.H, wr, wi, Xg, sg, Xo, so, inst.eigs)


def test_lu_baseline_rejects_other_options():
    with pytest.raises(hs.HseinError):
        hs.Solver(64, 2, 0, method=2, precision=1)
    with pytest.raises(hs.HseinError):
        hs.Solver(64, 2, 0, method=2, givens=1)
    with pytest.raises(hs.HseinError):
        hs.Solver(20000, 2, 0, method=2)
