"""Batches of independent instances in one CUDA graph (hsein_batch_*).

Every instance's results must be bit-identical to hsein_solve on that
instance alone with the same tile height (the batch only changes where and
when the same launches run), whether an instance is one sub-problem or is cut
into blocks of shifts (columns never mix), before and after the autotuner.
Sampled shifts are checked against the oracle.  The full batching workload
(256 instances, n log-uniform in [64, 2048]) is solved once with the residual
bound on every converged column.
"""
import os

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

TILE = {0: lambda n: 64, 1: lambda n: 32 if n < 512 else 64,
        2: lambda n: 16 if n < 256 else (32 if n < 1024 else 64)}


@pytest.fixture(scope="module")
def small_batch():
    sizes = hi.config3_sizes(seed=5, count=14, lo=64, hi=520)
    return [hi.batch_instance(n, k, 5000 + i) for i, (n, k) in enumerate(sizes)]


def _dev(insts):
    return [(to_dev(i.H), to_dev(i.wr), to_dev(i.wi), to_dev(i.B)) for i in insts]


def _alone(inst, dev, br):
    s = hs.Solver(inst.n, inst.m_real, inst.m_cplx, br=br)
    X, st = s.solve(*dev)
    return X.cpu().numpy(), st.cpu().numpy()


@pytest.mark.parametrize("policy,block,streams", [(1, 0, 4), (2, 7, 8), (0, 0, 1)])
def test_batch_equals_each_instance_alone(small_batch, policy, block, streams):
    dev = _dev(small_batch)
    b = hs.Batch(dev, streams=streams, br_policy=policy, shift_block=block)
    cfg, nsub = b.info()
    assert cfg == {"streams": streams, "br_policy": policy, "shift_block": block}
    if block:
        assert nsub > len(small_batch)
    Xs, sts = b.solve()
    b.solve()  # a replay of the captured graph gives the same results
    torch.cuda.synchronize()
    for inst, d, X, st in zip(small_batch, dev, Xs, sts):
        Xa, sa = _alone(inst, d, TILE[policy](inst.n))
        assert np.array_equal(st.cpu().numpy(), sa)
        assert np.array_equal(X.cpu().numpy(), Xa)


def test_batch_matches_the_oracle(small_batch):
    dev = _dev(small_batch)
    b = hs.Batch(dev, streams=8, br_policy=2)
    Xs, sts = b.solve()
    torch.cuda.synchronize()
    for j, (inst, X, st) in enumerate(zip(small_batch, Xs, sts)):
        offs = hi.column_offsets(inst.wi)
        pick = np.argsort(hi.uniform(77, j, inst.m), kind="stable")[:3]
        Bs = np.concatenate([inst.B[:, offs[l]:offs[l + 1]] for l in pick], axis=1)
        Xo, so = oracle.hsein(inst.H, inst.wr[pick], inst.wi[pick], Bs)
        sh, Xh = st.cpu().numpy(), X.cpu().numpy()
        assert np.array_equal(so, sh[pick])
        hn = oracle.hnorm_inf(inst.H)
        vo = as_vectors(Xo, inst.wr[pick], inst.wi[pick])
        for q, l in enumerate(pick):
            if sh[l] != 0:
                continue
            lam = vo[q][0]
            gap = separation(inst.eigs, lam)
            bound = angle_bound(gap, hn, inst.n)
            assert angle(Xh[:, offs[l]], vo[q][1]) <= bound


def test_autotune_picks_a_candidate_and_keeps_results(small_batch):
    dev = _dev(small_batch)
    b = hs.Batch(dev, streams=16, br_policy=1)
    cfg, ms = b.autotune()
    assert ms > 0
    assert cfg["br_policy"] in (0, 1, 2) and cfg["shift_block"] in (0, 512, 256, 128)
    assert cfg["streams"] in (4, 8, 16, 24, 32, 48)
    assert b.info()[0] == cfg
    Xs, sts = b.solve()
    torch.cuda.synchronize()
    for inst, d, X, st in zip(small_batch, dev, Xs, sts):
        Xa, sa = _alone(inst, d, TILE[cfg["br_policy"]](inst.n))
        assert np.array_equal(st.cpu().numpy(), sa)
        assert np.array_equal(X.cpu().numpy(), Xa)


def test_batching_workload_full_size():
    insts = hi.config3(workers=min(16, os.cpu_count() or 1))
    assert len(insts) == 256
    dev = _dev(insts)
    b = hs.Batch(dev, streams=16, br_policy=1)
    cfg, ms = b.autotune()
    Xs, sts = b.solve()
    torch.cuda.synchronize()
    cols = 0
    # statuses of sampled shifts (every non-converged one among them) against
    # the oracle, on eight instances across the size range
    order = np.argsort([i.n for i in insts], kind="stable")
    for j in order[::32]:
        inst, sh = insts[j], sts[j].cpu().numpy()
        pick = sorted(set(np.argsort(hi.uniform(78, int(j), inst.m), kind="stable")[:4].tolist())
                      | set(np.nonzero(sh)[0][:4].tolist()))
        Xo, so = oracle.hsein(inst.H, inst.wr[pick], inst.wi[pick], inst.B[:, pick])
        assert np.array_equal(so, sh[pick]), (inst.n, pick, so, sh[pick])
    for inst, d, X, st in zip(insts, dev, Xs, sts):
        sh = st.cpu().numpy()
        conv = sh == 0
        # residual of every converged column, FP64 on the device
        H = d[0]
        Xd = X[:, np.nonzero(conv)[0].tolist()]
        R = H @ Xd - Xd * d[1][torch.as_tensor(np.nonzero(conv)[0], device=H.device)]
        r = (R.abs().sum(0) / (H.abs().sum(0).max() * Xd.abs().sum(0))).max().item()
        assert r <= 100 * inst.n * EPS, (inst.n, r / (inst.n * EPS))
        cols += int(conv.sum())
    assert cols >= 0.95 * sum(i.m for i in insts)
    print("batching workload: %d converged columns, autotuned %s, %.1f ms" % (cols, cfg, ms))


def test_batch_with_complex_shifts_in_blocks():
    insts = [hi.small_instance(n, mr, mc, 60 + i)
             for i, (n, mr, mc) in enumerate([(96, 5, 4), (200, 9, 7), (130, 0, 6), (75, 8, 0)])]
    dev = _dev(insts)
    b = hs.Batch(dev, streams=3, br_policy=2, shift_block=3)
    Xs, sts = b.solve()
    torch.cuda.synchronize()
    for inst, d, X, st in zip(insts, dev, Xs, sts):
        Xa, sa = _alone(inst, d, TILE[2](inst.n))
        assert np.array_equal(st.cpu().numpy(), sa)
        assert np.array_equal(X.cpu().numpy(), Xa)
