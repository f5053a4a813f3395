"""Parity of the CUDA path with the CPU oracle (run on a GB300).

Every test solves the same seeded input on the GPU (through the C ABI via the
Python binding) and with the oracle, and compares:
  - per-shift status codes (bit-exact: converged / not converged);
  - eigenvectors by the sign/phase-invariant angle: <= 1e-10 for shifts whose
    eigenvalue is separated from the rest of the spectrum by >= 1e-3 ||H||_inf
    (the acceptance bound), and twice the first-order bound n eps ||H|| / gap
    otherwise (tests.metrics.angle_bound);
  - the normwise residual ||H x - lambda x||_1 / (||H||_1 ||x||_1) <= 100 n eps
    for every converged column;
  - Z = Q0 X against numpy's product of the same operands.
"""
import numpy as np
import pytest

import hsein_inputs as hi
import oracle
from tests.metrics import EPS, angle, angle_bound, as_vectors, residual, separation

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2101_05063_gb300 as hs  # noqa: E402


def to_dev(a):
    return torch.as_tensor(np.asfortranarray(a), dtype=torch.float64).cuda()


def run_gpu(inst_H, wr, wi, B, br=64, robust=True, omega_log2=1000, Q0=None, precision=0):
    wr = np.asarray(wr, dtype=np.float64)
    wi = np.asarray(wi, dtype=np.float64)
    mc = int(np.count_nonzero(wi))
    n = inst_H.shape[0]
    solver = hs.Solver(n, len(wr) - mc, mc, br=br, robust=robust, omega_log2=omega_log2,
                       precision=precision)
    X, status = solver.solve(to_dev(inst_H), to_dev(wr), to_dev(wi),
                             None if B is None else to_dev(B))
    Z = solver.backtransform(to_dev(Q0), X) if Q0 is not None else None
    torch.cuda.synchronize()
    Xh = X.cpu().numpy()
    out = (Xh, status.cpu().numpy(), solver)
    if Z is not None:
        out = out + (Z.cpu().numpy(),)
    return out


def compare(H, wr, wi, Xg, sg, Xo, so, eigs=None, hnorm=None, strict_status=True):
    n = H.shape[0]
    hn = hnorm if hnorm is not None else oracle.hnorm_inf(H)
    if strict_status:
        assert np.array_equal(sg, so), (sg, so)
    vg = as_vectors(Xg, wr, wi)
    vo = as_vectors(Xo, wr, wi)
    worst = 0.0
    for l, ((lam, xg), (_, xo)) in enumerate(zip(vg, vo)):
        if so[l] != 0 or sg[l] != 0:
            continue
        assert np.all(np.isfinite(xg))
        assert abs(np.linalg.norm(xg) - 1.0) <= 8 * n * EPS
        r = residual(H, lam, xg)
        assert r <= 100 * n * EPS, (l, r / (n * EPS))
        a = angle(xg, xo)
        gap = separation(eigs, lam) if eigs is not None else np.inf
        bound = angle_bound(gap, hn, n)
        assert a <= bound, (l, lam, a, gap, bound)
        worst = max(worst, a)
    return worst


CASES = [
    # n, m_real, m_cplx, br, seed
    (1, 1, 0, 8, 1),
    (2, 1, 0, 8, 2),
    (3, 1, 1, 8, 3),
    (7, 2, 1, 8, 4),
    (8, 3, 1, 8, 5),
    (9, 3, 2, 8, 6),
    (37, 5, 3, 8, 7),
    (63, 6, 4, 32, 8),
    (64, 6, 4, 32, 9),
    (65, 6, 4, 32, 10),
    (131, 12, 9, 32, 11),
    (200, 20, 10, 64, 12),
    (257, 30, 17, 64, 13),
    (300, 0, 20, 64, 14),
    (300, 33, 0, 64, 15),
    (333, 40, 25, 128, 16),
]


@pytest.mark.parametrize("n,mr,mc,br,seed", CASES)
def test_small_instances_match_oracle(n, mr, mc, br, seed):
    if n == 1:
        H = np.array([[2.5]])
        wr, wi, B = np.array([2.5 + 1e-3]), np.array([0.0]), np.ones((1, 1))
        eigs = np.array([2.5])
    elif n == 2:
        H = np.array([[1.0, 2.0], [0.5, -1.0]])
        ev = np.linalg.eigvals(H)
        wr, wi, B = np.array([ev[0].real]), np.array([0.0]), np.array([[0.6], [0.8]])
        eigs = ev
    else:
        inst = hi.small_instance(n, mr, mc, seed)
        H, wr, wi, B, eigs = inst.H, inst.wr, inst.wi, inst.B, inst.eigs
    Xg, sg, _ = run_gpu(H, wr, wi, B, br=br)
    Xo, so = oracle.hsein(H, wr, wi, B)
    compare(H, wr, wi, Xg, sg, Xo, so, eigs)


@pytest.mark.parametrize("precision,br", [(0, 32), (1, 64)])
def test_many_real_shifts_four_per_warp(precision, br):
    """More real shifts than the GPU has SM sub-partitions for at two shifts
    per warp: the sweep packs four real shifts per warp.  Statuses and
    directions of a seeded sample of shifts against the oracle, and the
    residual of every converged real column."""
    n, mr, mc = 1536, 1300, 20
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert mc + (mr + 1) // 2 > 4 * sms  # the packed layout is the one used
    inst = hi.small_instance(n, mr, mc, 61)
    Xg, sg, _ = run_gpu(inst.H, inst.wr, inst.wi, inst.B, br=br, precision=precision)
    offs = hi.column_offsets(inst.wi)
    pick = np.sort(np.argsort(hi.uniform(62, 0, mr + mc), kind="stable")[:48])
    pick = np.union1d(pick, np.nonzero(inst.wi)[0][:4])  # complex shifts too
    cols = np.concatenate([np.arange(offs[l], offs[l + 1]) for l in pick])
    Xo, so = oracle.hsein(inst.H, inst.wr[pick], inst.wi[pick], inst.B[:, cols])
    compare(inst.H, inst.wr[pick], inst.wi[pick], Xg[:, cols], sg[pick], Xo, so, inst.eigs)
    real = np.nonzero((inst.wi == 0) & (sg == 0))[0]
    rc = np.array([offs[l] for l in real])
    Hd = to_dev(inst.H)
    Xd = to_dev(Xg[:, rc])
    lam = to_dev(inst.wr[real])
    R = Hd @ Xd - Xd * lam
    r = (R.abs().sum(0) / (Hd.abs().sum(0).max() * Xd.abs().sum(0))).max().item()
    assert r <= 100 * n * EPS, r / (n * EPS)
    assert len(real) >= 0.9 * mr


@pytest.mark.parametrize("br", [16, 64])
def test_default_starting_vector(br):
    inst = hi.small_instance(150, 10, 6, 21)
    Xg, sg, _ = run_gpu(inst.H, inst.wr, inst.wi, None, br=br)
    Xo, so = oracle.hsein(inst.H, inst.wr, inst.wi, None)
    compare(inst.H, inst.wr, inst.wi, Xg, sg, Xo, so, inst.eigs)


def test_config0_full_size_with_backtransform():
    inst = hi.config0()
    Xg, sg, _, Zg = run_gpu(inst.H, inst.wr, inst.wi, inst.B, Q0=inst.Q0)
    Xo, so = oracle.hsein(inst.H, inst.wr, inst.wi, inst.B)
    compare(inst.H, inst.wr, inst.wi, Xg, sg, Xo, so, inst.eigs)
    Zref = inst.Q0 @ Xg
    assert np.abs(Zg - Zref).max() <= 1e-13
    Zo = oracle.q0_apply(inst.Q0, Xo)
    hn = oracle.hnorm_inf(inst.H)
    for l in range(inst.m):
        assert sg[l] == 0
        bound = angle_bound(separation(inst.eigs, inst.wr[l]), hn, inst.n)
        assert angle(Zg[:, l], Zo[:, l]) <= bound, l


@pytest.mark.parametrize("n,om", [(48, 30), (96, 40), (200, 60)])
def test_bad_system_h2_scaling_matches_oracle(n, om):
    # the bad system of Sec. 5.2 with a lowered overflow threshold: the
    # scaling paths of the diagonal solve and of the shared-H update run
    H = hi.paper_h2(n)
    B = np.ones((n, 1)) / np.sqrt(n)
    for br in (8, 32):
        Xg, sg, _ = run_gpu(H, [2.0], [0.0], B, br=br, omega_log2=om)
        Xo, so = oracle.hsein(H, [2.0], [0.0], B, log2_omega=om)
        assert sg[0] == 0 and so[0] == 0
        assert np.all(np.isfinite(Xg))
        assert angle(Xg[:, 0], Xo[:, 0]) <= 1e-12
        assert residual(H, 2.0, Xg[:, 0]) <= 100 * n * EPS


def test_bad_system_h2_default_threshold_no_overflow():
    n = 1024
    H = hi.paper_h2(n)
    B = np.ones((n, 1)) / np.sqrt(n)
    Xg, sg, _ = run_gpu(H, [2.0], [0.0], B)
    Xo, so = oracle.hsein(H, [2.0], [0.0], B)
    assert sg[0] == 0 and np.all(np.isfinite(Xg))
    assert angle(Xg[:, 0], Xo[:, 0]) <= 1e-12
    assert residual(H, 2.0, Xg[:, 0]) <= 100 * n * EPS


def test_unprotected_solve_overflows_where_the_protected_one_matches():
    # Sec. 4.1 and Sec. 5.2: the bad system H2 at n = 1024 needs growth far
    # beyond the double range.  Without the protection (robust = 0) the
    # solution overflows: its Varah margin is not finite and the column is
    # returned as not converged (zero), as the oracle's unprotected driver
    # does; with it the solve is finite and matches the oracle
    n = 1024
    H = hi.paper_h2(n)
    B = np.ones((n, 1)) / np.sqrt(n)
    s0 = hs.Solver(n, 1, 0, robust=False)
    X0, st0 = s0.solve(to_dev(H), to_dev(np.array([2.0])), to_dev(np.array([0.0])), to_dev(B),
                       check=False)
    margin0 = s0.margins().cpu().numpy()[0]
    X0, st0 = X0.cpu().numpy(), st0.cpu().numpy()
    with np.errstate(all="ignore"):
        Xu, su = oracle.hsein(H, [2.0], [0.0], B, robust=False)
    assert su[0] == 1 and st0[0] == 1
    assert not np.isfinite(margin0)
    assert np.all(X0 == 0.0)
    s1 = hs.Solver(n, 1, 0, robust=True)
    X1, st1 = s1.solve(to_dev(H), to_dev(np.array([2.0])), to_dev(np.array([0.0])), to_dev(B))
    margin1 = s1.margins().cpu().numpy()[0]
    X1, st1 = X1.cpu().numpy(), st1.cpu().numpy()
    Xo, so = oracle.hsein(H, [2.0], [0.0], B)
    assert st1[0] == 0 and so[0] == 0 and np.isfinite(margin1) and margin1 > 0
    assert np.all(np.isfinite(X1))
    assert angle(X1[:, 0], Xo[:, 0]) <= 1e-12
    assert residual(H, 2.0, X1[:, 0]) <= 100 * n * EPS


def test_good_system_h3_matches():
    # (H3 - 2I) is well conditioned, so one solve is not an eigenvector and
    # both sides must flag it (Varah's test, Sec. 4.2); with eigenvalue
    # shifts of H3 both sides must agree on the vectors
    n = 512
    H = hi.paper_h3(n)
    B = np.ones((n, 1)) / np.sqrt(n)
    Xg, sg, _ = run_gpu(H, [2.0], [0.0], B, omega_log2=30)
    Xo, so = oracle.hsein(H, [2.0], [0.0], B, log2_omega=30)
    assert sg[0] == 1 and so[0] == 1
    ev = np.linalg.eigvals(H)
    real = ev[np.abs(ev.imag) == 0].real
    wr = np.sort(real)[:: max(1, len(real) // 4)][:4]
    cp = ev[ev.imag > 0][:2]
    wr = np.concatenate([wr, cp.real])
    wi = np.concatenate([np.zeros(len(wr) - len(cp)), cp.imag])
    offs = hi.column_offsets(wi)
    Bm = hi.unit_columns(n, int(offs[-1]), seed=5)
    Xg, sg, _ = run_gpu(H, wr, wi, Bm, omega_log2=30)
    Xo, so = oracle.hsein(H, wr, wi, Bm, log2_omega=30)
    compare(H, wr, wi, Xg, sg, Xo, so, ev)


def test_graded_matrix_stays_finite():
    n = 96
    rng_H = np.triu(hi.normal(11, 50, n * n).reshape(n, n, order="F"), -1)
    G, d = hi.graded(rng_H, seed=11, umax=150.0, monotone=True)
    ev = np.linalg.eigvals(rng_H)
    lam = float(ev[np.argmin(np.abs(ev.imag))].real)
    b = hi.normal(11, 51, n)[:, None]
    b /= np.linalg.norm(b)
    Xg, sg, _ = run_gpu(G, [lam], [0.0], b, br=32)
    assert np.all(np.isfinite(Xg))
    if sg[0] == 0:
        Gl = G.astype(np.longdouble)
        y = Xg[:, 0].astype(np.longdouble)
        r = np.abs(Gl @ y - np.longdouble(lam) * y).sum()
        assert float(r / (np.abs(Gl).sum(axis=0).max() * np.abs(y).sum())) <= 100 * n * EPS


def test_device_errors_are_reported():
    inst = hi.small_instance(40, 3, 2, 31)
    # zero subdiagonal -> not unreduced
    H = inst.H.copy()
    H[10, 9] = 0.0
    solver = hs.Solver(40, 3, 2)
    X, st = solver.solve(to_dev(H), to_dev(inst.wr), to_dev(inst.wi), to_dev(inst.B), check=False)
    assert solver.device_status() == -3
    assert np.all(st.cpu().numpy() == 3) and np.all(X.cpu().numpy() == 0.0)
    # non-finite entry
    H = inst.H.copy()
    H[3, 20] = np.nan
    X, st = solver.solve(to_dev(H), to_dev(inst.wr), to_dev(inst.wi), to_dev(inst.B), check=False)
    assert solver.device_status() == -4
    # wrong number of complex shifts
    wi = inst.wi.copy()
    wi[np.nonzero(wi)[0][0]] = 0.0
    X, st = solver.solve(to_dev(inst.H), to_dev(inst.wr), to_dev(wi), to_dev(inst.B), check=False)
    assert solver.device_status() == -7
    # and a clean solve afterwards still works
    X, st = solver.solve(to_dev(inst.H), to_dev(inst.wr), to_dev(inst.wi), to_dev(inst.B))
    assert solver.device_status() in (0, 1)


def test_bounded_wait_runs_out_without_a_fault():
    # the diagonal-tile kernel's wait for its tile copy is bounded: with a
    # limit of one cycle it runs out on purpose (the copy itself is valid and
    # lands; the kernel waits for it before returning), the solve reports
    # HSEIN_ETIMEOUT, every status is HSEIN_COL_INVALID and the output is
    # zero; the context stays usable and the next solve is correct
    inst = hi.small_instance(200, 6, 4, 33)
    s = hs.Solver(inst.n, inst.m_real, inst.m_cplx, wait_limit_cycles=1)
    X, st = s.solve(to_dev(inst.H), to_dev(inst.wr), to_dev(inst.wi), to_dev(inst.B), check=False)
    assert s.device_status() == -6
    assert np.all(st.cpu().numpy() == 3) and np.all(X.cpu().numpy() == 0.0)
    Xg, sg, _ = run_gpu(inst.H, inst.wr, inst.wi, inst.B)
    Xo, so = oracle.hsein(inst.H, inst.wr, inst.wi, inst.B)
    compare(inst.H, inst.wr, inst.wi, Xg, sg, Xo, so, inst.eigs)
    with pytest.raises(hs.HseinError):
        hs.Solver(64, 2, 0, wait_limit_cycles=-1)


def test_far_shift_not_converged_and_zeroed():
    inst = hi.small_instance(64, 4, 0, 41)
    wr = inst.wr.copy()
    wr[1] = 1e3 * oracle.hnorm_inf(inst.H)
    Xg, sg, solver = run_gpu(inst.H, wr, inst.wi, inst.B)
    Xo, so = oracle.hsein(inst.H, wr, inst.wi, inst.B)
    assert sg[1] == 1 and so[1] == 1
    assert np.all(Xg[:, 1] == 0.0)
    assert solver.device_status() == 1


def test_repeatable():
    inst = hi.small_instance(129, 9, 5, 51)
    X1, s1, _ = run_gpu(inst.H, inst.wr, inst.wi, inst.B)
    X2, s2, _ = run_gpu(inst.H, inst.wr, inst.wi, inst.B)
    assert np.array_equal(X1, X2) and np.array_equal(s1, s2)


def _ld_product(Q, X):
    return (np.asarray(Q, dtype=np.longdouble) @ np.asarray(X, dtype=np.longdouble))


@pytest.mark.parametrize("n,ncol,graded", [(512, 64, False), (333, 37, False), (257, 20, True)])
def test_split_precision_backtransform_accuracy(n, ncol, graded):
    # z = Q0 x with the BF16 digit products must be as accurate as the FP64
    # product, measured against a long-double product of the same operands
    Q = hi.haar_orthogonal(n, 3)
    X = hi.unit_columns(n, ncol, seed=4)
    if graded:
        # rows and columns of very different scales exercise the exponents
        Q = Q * (10.0 ** hi.uniform(5, 1, n, -30, 30))[:, None]
        X = X * (10.0 ** hi.uniform(6, 1, ncol, -200, 200))[None, :]
        X[:, 3] = 0.0
    dQ, dX = to_dev(Q), to_dev(X)
    s64 = hs.Solver(n, ncol, 0, precision=0)
    soz = hs.Solver(n, ncol, 0, precision=1)
    Z64 = s64.backtransform(dQ, dX).cpu().numpy()
    Zoz = soz.backtransform(dQ, dX).cpu().numpy()
    Zex = _ld_product(Q, X)
    scale = (np.abs(Q).max(axis=1)[:, None] * np.abs(X).max(axis=0)[None, :]).astype(np.longdouble)
    scale[scale == 0] = 1
    e64 = float(np.max(np.abs(Z64 - Zex) / scale))
    eoz = float(np.max(np.abs(Zoz - Zex) / scale))
    assert np.all(Zoz[:, 3] == 0.0) if graded else True
    assert eoz <= max(4 * e64, 8 * n * EPS), (eoz, e64)


def test_split_precision_pipeline_matches_oracle():
    # the whole split-precision path on the n = 512 workload: statuses,
    # eigenvectors of H and of A (z = Q0 x) against the oracle's within the
    # angle gate, residuals of both against H and A
    inst = hi.config0(keep_a=True)
    solver = hs.Solver(inst.n, inst.m_real, inst.m_cplx, precision=1)
    X, st = solver.solve(to_dev(inst.H), to_dev(inst.wr), to_dev(inst.wi), to_dev(inst.B))
    Z = solver.backtransform(to_dev(inst.Q0), X).cpu().numpy()
    X, st = X.cpu().numpy(), st.cpu().numpy()
    Xo, so = oracle.hsein(inst.H, inst.wr, inst.wi, inst.B)
    Zo = oracle.q0_apply(inst.Q0, Xo)
    compare(inst.H, inst.wr, inst.wi, X, st, Xo, so, inst.eigs)
    hn = oracle.hnorm_inf(inst.H)
    n = inst.n
    for l in range(inst.m):
        assert st[l] == 0
        bound = angle_bound(separation(inst.eigs, inst.wr[l]), hn, n)
        assert angle(Z[:, l], Zo[:, l]) <= bound, l
        assert residual(inst.A, inst.wr[l], Z[:, l]) <= 100 * n * EPS, l


SPLIT_CASES = [(65, 6, 4, 17), (131, 12, 9, 18), (257, 30, 17, 19), (300, 0, 20, 20), (300, 33, 0, 21),
               (520, 40, 25, 22)]


@pytest.mark.parametrize("n,mr,mc,seed", SPLIT_CASES)
def test_split_precision_small_instances_match_oracle(n, mr, mc, seed):
    # the shared-H update and the backtransform on BF16 digit products
    inst = hi.small_instance(n, mr, mc, seed)
    Xg, sg, _, Zg = run_gpu(inst.H, inst.wr, inst.wi, inst.B, precision=1, Q0=inst.Q0)
    Xo, so = oracle.hsein(inst.H, inst.wr, inst.wi, inst.B)
    compare(inst.H, inst.wr, inst.wi, Xg, sg, Xo, so, inst.eigs)
    assert np.abs(Zg - inst.Q0 @ Xg).max() <= 1e-13


@pytest.mark.parametrize("n,om", [(200, 60), (1024, 1000)])
def test_split_precision_bad_system_h2(n, om):
    H = hi.paper_h2(n)
    B = np.ones((n, 1)) / np.sqrt(n)
    Xg, sg, _ = run_gpu(H, [2.0], [0.0], B, omega_log2=om, precision=1)
    Xo, so = oracle.hsein(H, [2.0], [0.0], B, log2_omega=om)
    assert sg[0] == 0 and so[0] == 0 and np.all(np.isfinite(Xg))
    assert angle(Xg[:, 0], Xo[:, 0]) <= 1e-12
    assert residual(H, 2.0, Xg[:, 0]) <= 100 * n * EPS


@pytest.mark.parametrize("precision", [0, 1])
def test_step_graph_matches_the_calls(precision):
    """hsein_graph_create / hsein_graph_launch: the captured step gives the
    results of hsein_solve + hsein_backtransform bitwise, at every launch, and
    follows new contents of its input buffers; the solve-only graph too."""
    inst = hi.small_instance(300, 20, 10, 71)
    H, wr, wi, B, Q0 = (to_dev(inst.H), to_dev(inst.wr), to_dev(inst.wi), to_dev(inst.B),
                        to_dev(inst.Q0))
    s = hs.Solver(inst.n, inst.m_real, inst.m_cplx, precision=precision)
    X0, st0 = s.solve(H, wr, wi, B)
    Z0 = s.backtransform(Q0, X0)
    step = s.graph(H, wr, wi, B, Q0)
    for _ in range(2):
        step.launch()
        torch.cuda.synchronize()
        assert torch.equal(step.status, st0)
        assert torch.equal(step.X, X0)
        assert torch.equal(step.Z, Z0)
    # new starting vectors in the same buffer
    B.copy_(to_dev(np.roll(inst.B, 7, axis=0)))
    X1, st1 = s.solve(H, wr, wi, B)
    Z1 = s.backtransform(Q0, X1)
    step.launch()
    torch.cuda.synchronize()
    assert torch.equal(step.status, st1) and torch.equal(step.X, X1) and torch.equal(step.Z, Z1)
    assert not torch.equal(X1, X0)
    # the solve alone, default starting vector
    Xd, std = s.solve(H, wr, wi, None)
    solve_only = s.graph(H, wr, wi)
    solve_only.launch()
    torch.cuda.synchronize()
    assert solve_only.Z is None
    assert torch.equal(solve_only.status, std) and torch.equal(solve_only.X, Xd)
    Xo, so = oracle.hsein(inst.H, inst.wr, inst.wi, None)
    compare(inst.H, inst.wr, inst.wi, solve_only.X.cpu().numpy(), solve_only.status.cpu().numpy(),
            Xo, so, inst.eigs)


def test_step_graph_rejects_bad_arguments():
    inst = hi.small_instance(64, 3, 1, 72)
    s = hs.Solver(inst.n, inst.m_real, inst.m_cplx)
    H, wr, wi = to_dev(inst.H), to_dev(inst.wr), to_dev(inst.wi)
    with pytest.raises(hs.HseinError) as e:
        s.graph(H, wr, wi, None, to_dev(inst.Q0), Z=torch.empty(0, dtype=torch.float64,
                                                                device="cuda").reshape(0, 0))
    assert e.value.code == -1
    X = torch.empty((inst.ncol, inst.n), dtype=torch.float64, device="cuda").t()
    rc, g = hs.hsein_graph_create(s.plan, H.data_ptr(), 10, wr.data_ptr(), wi.data_ptr(), 0,
                                  inst.n, X.data_ptr(), inst.n, 0, 0, inst.n, 0, inst.n,
                                  s.work.data_ptr(), s.work_bytes)
    assert rc == -1 and not g.value  # ldh < n; no graph is left behind


def test_solve_host_matches_device_path():
    # the end-to-end call from host buffers (hsein_solve_host) gives the
    # device path's results bit for bit (same kernels on the same inputs),
    # twice in a row from pinned memory, then from pageable memory
    inst = hi.small_instance(300, 9, 5, 44)
    n, ncol, m = inst.n, inst.ncol, inst.m
    s = hs.Solver(n, inst.m_real, inst.m_cplx)
    X, st = s.solve(to_dev(inst.H), to_dev(inst.wr), to_dev(inst.wi), to_dev(inst.B))
    Z = s.backtransform(to_dev(inst.Q0), X).cpu().numpy()
    st = st.cpu().numpy()
    pin = lambda a: torch.as_tensor(np.asfortranarray(a), dtype=torch.float64).pin_memory()
    hZ = torch.empty((ncol, n), dtype=torch.float64).pin_memory().t()
    hS = torch.empty(m, dtype=torch.int32).pin_memory()
    for _ in range(2):
        hZ.zero_()
        s.solve_host(pin(inst.H), pin(inst.wr), pin(inst.wi), pin(inst.B), pin(inst.Q0), hZ, hS)
        torch.cuda.synchronize()
        assert np.array_equal(hZ.numpy(), Z)
        assert np.array_equal(hS.numpy(), st)
    # pageable host memory and the default starting vector: the same results
    # as the device path with B = NULL
    X0, st0 = s.solve(to_dev(inst.H), to_dev(inst.wr), to_dev(inst.wi), None)
    Z0 = s.backtransform(to_dev(inst.Q0), X0).cpu().numpy()
    hZ2 = torch.zeros((ncol, n), dtype=torch.float64).t()
    hS2 = torch.zeros(m, dtype=torch.int32)
    cm = lambda a: torch.as_tensor(np.asfortranarray(a), dtype=torch.float64)
    s.solve_host(cm(inst.H), cm(inst.wr), cm(inst.wi), None, cm(inst.Q0), hZ2, hS2)
    torch.cuda.synchronize()
    assert np.array_equal(hZ2.numpy(), Z0) and np.array_equal(hS2.numpy(), st0.cpu().numpy())
    assert s.host_device_status() in (0, 1)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("n,mr,mc,seed", [(64, 3, 2, 53), (130, 6, 4, 51), (300, 9, 5, 52)])
def test_compact_givens_storage_matches_oracle(n, mr, mc, seed, precision):
    # Stewart's compact storage of the rotations (Sec. 4.4): the same results
    # as the oracle, and the same directions as the full storage within each
    # column's angle gate; n x m doubles less workspace
    inst = hi.small_instance(n, mr, mc, seed)
    s0 = hs.Solver(n, mr, mc, precision=precision)
    s1 = hs.Solver(n, mr, mc, precision=precision, givens=1)
    assert s0.work_bytes - s1.work_bytes >= 8 * n * (mr + mc)
    X0, st0 = s0.solve(to_dev(inst.H), to_dev(inst.wr), to_dev(inst.wi), to_dev(inst.B))
    X1, st1 = s1.solve(to_dev(inst.H), to_dev(inst.wr), to_dev(inst.wi), to_dev(inst.B))
    X0, st0, X1, st1 = X0.cpu().numpy(), st0.cpu().numpy(), X1.cpu().numpy(), st1.cpu().numpy()
    Xo, so = oracle.hsein(inst.H, inst.wr, inst.wi, inst.B)
    compare(inst.H, inst.wr, inst.wi, X1, st1, Xo, so, inst.eigs)
    compare(inst.H, inst.wr, inst.wi, X0, st0, Xo, so, inst.eigs)
    assert np.array_equal(st0, st1)
    # full against compact storage, per column.  Directions, not entries: for
    # a shift that equals an eigenvalue to working accuracy, x is about
    # v (u^H b) / delta with delta of the size of the rounding errors, so the
    # sign (real) or phase (complex) of the output is set by rounding, and
    # two correct solves may differ in it
    hn = oracle.hnorm_inf(inst.H)
    for l, ((lam, x0), (_, x1)) in enumerate(zip(as_vectors(X0, inst.wr, inst.wi),
                                                as_vectors(X1, inst.wr, inst.wi))):
        if st0[l] != 0:
            assert np.all(x0 == 0.0) and np.all(x1 == 0.0)
            continue
        bound = angle_bound(separation(inst.eigs, lam), hn, n)
        assert angle(x0, x1) <= bound, (l, lam, angle(x0, x1), bound)


def test_compact_givens_storage_through_the_scaling_paths():
    # the bad system of Sec. 5.2 with a lowered threshold: rescaling on every
    # path, rotations stored compactly
    n = 96
    H = hi.paper_h2(n)
    B = np.ones((n, 1)) / np.sqrt(n)
    s = hs.Solver(n, 1, 0, omega_log2=40, givens=1)
    X, st = s.solve(to_dev(H), to_dev(np.array([2.0])), to_dev(np.array([0.0])), to_dev(B))
    X, st = X.cpu().numpy(), st.cpu().numpy()
    Xo, so = oracle.hsein(H, [2.0], [0.0], B, log2_omega=40)
    assert st[0] == so[0] == 0
    assert angle(X[:, 0], Xo[:, 0]) <= 1e-12


def test_compact_givens_storage_needs_the_tiled_method():
    with pytest.raises(hs.HseinError):
        hs.Solver(64, 2, 0, method=1, givens=1)
    with pytest.raises(hs.HseinError):
        hs.Solver(64, 2, 0, givens=2)
