"""The serving loop (hsein_server_*): continuous batching of solve requests.

Each result must equal what hsein_solve gives the request alone (same
precision and tile height), whether the request was fused with others on the
same matrix, waited for memory, or ran while others were on the GPU; requests
that cannot fit the arena are refused at submission; a short real-time
Poisson stream of the serving workload completes with the residual bound on
its converged columns.
"""
import numpy as np
import pytest

import hsein_inputs as hi
from tests.metrics import EPS

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import bench  # noqa: E402
import paper_2101_05063_gb300 as hs  # noqa: E402
from tests.test_gpu_parity import to_dev  # noqa: E402

GB = 1 << 30


@pytest.fixture(scope="module")
def pool():
    p = hi.serving_pool(sizes=(256, 512, 1024), per_size={256: 2, 512: 2, 1024: 2}, seed=9)
    dev = {n: [(to_dev(i.H), to_dev(i.Hg)) for i in lst] for n, lst in p.items()}
    bal = {n: [(to_dev(i.H),) + tuple(hs.balance(to_dev(i.Hg))) for i in lst] for n, lst in p.items()}
    torch.cuda.synchronize()
    dev["balanced"] = bal
    return p, dev


def _alone(H, wr, wi, precision):
    n = H.shape[0]
    mc = int((wi != 0).sum().item())
    s = hs.Solver(n, wr.numel() - mc, mc, br=64, precision=precision)
    X, st = s.solve(H, wr, wi)
    return X.cpu().numpy(), st.cpu().numpy()


def _requests(pool, count, seed):
    reqs = hi.serving_requests(pool, count, seed=seed)
    return reqs


def test_fused_requests_equal_each_alone(pool):
    p, dev = pool
    reqs = _requests(p, 14, 11)
    srv = hs.Server(4 * GB, max_jobs=4, max_merge_shifts=1 << 20)
    tickets = []
    for r in reqs:  # all pending together: requests on one matrix fuse
        H, Hg = dev[r["n"]][r["index"]]
        tickets.append(srv.submit(Hg if r["graded"] else H, to_dev(r["wr"]), to_dev(r["wi"]),
                                  precision=0 if r["graded"] else 1))
    done = set()
    while len(done) < len(tickets):
        done |= set(srv.progress(wait=True))
    st = srv.stats()
    assert st["requests_admitted"] == len(reqs) and st["pending"] == 0 and st["running"] == 0
    assert st["solves_admitted"] < len(reqs)  # some requests shared a solve
    assert st["bytes_in_use"] == 0
    for r, t in zip(reqs, tickets):
        X, s = srv.result(t)
        H, Hg = dev[r["n"]][r["index"]]
        Xa, sa = _alone(Hg if r["graded"] else H, to_dev(r["wr"]), to_dev(r["wi"]),
                        0 if r["graded"] else 1)
        assert np.array_equal(s.cpu().numpy(), sa)
        assert np.array_equal(X.cpu().numpy(), Xa)


def test_admission_waits_for_memory(pool):
    p, dev = pool
    reqs = [r for r in _requests(p, 30, 12) if r["n"] == 1024][:5]
    # an arena for about one n = 1024 solve at a time
    opt = hs.hsein_default_options()
    opt.precision = 1
    big = 0
    for r in reqs:
        mc = int((r["wi"] != 0).sum())
        plan, w = hs.hsein_plan(1024, len(r["wr"]) - mc, mc, opt)
        hs.hsein_plan_destroy(plan)
        big = max(big, w)
    srv = hs.Server(int(big * 1.5), max_jobs=4, max_merge_shifts=1)  # no fusion
    tickets = [srv.submit(dev[1024][r["index"]][0], to_dev(r["wr"]), to_dev(r["wi"]), precision=1)
               for r in reqs]
    peak = 0
    done = set()
    while len(done) < len(tickets):
        st = srv.stats()
        peak = max(peak, st["running"])
        assert st["bytes_in_use"] <= int(big * 1.5)
        done |= set(srv.progress(wait=True))
    assert peak <= 1
    for r, t in zip(reqs, tickets):
        X, s = srv.result(t)
        Xa, sa = _alone(dev[1024][r["index"]][0], to_dev(r["wr"]), to_dev(r["wi"]), 1)
        assert np.array_equal(s.cpu().numpy(), sa) and np.array_equal(X.cpu().numpy(), Xa)


@pytest.mark.parametrize("bypass", [0, 4])
def test_head_of_line_bypass(pool, bypass):
    # an arena for one n = 1024 solve and one n = 256 solve: behind a large
    # request that must wait for memory, a small one waits too in arrival
    # order (bypass 0), or is admitted ahead of it (bypass > 0); every result
    # equals the request's solve alone
    p, dev = pool
    big_r = [r for r in _requests(p, 40, 15) if r["n"] == 1024][:2]
    small_r = [r for r in _requests(p, 40, 16) if r["n"] == 256][:1]
    opt = hs.hsein_default_options()
    opt.precision = 1

    def ws(r):
        mc = int((r["wi"] != 0).sum())
        plan, w = hs.hsein_plan(r["n"], len(r["wr"]) - mc, mc, opt)
        hs.hsein_plan_destroy(plan)
        return w
    wb = max(ws(r) for r in big_r)
    arena = wb + ws(small_r[0]) + (1 << 20)
    assert arena < 2 * min(ws(r) for r in big_r)
    srv = hs.Server(arena, max_jobs=4, max_merge_shifts=1, max_bypass=bypass)
    order = big_r + small_r
    tickets = [srv.submit(dev[r["n"]][r["index"]][0], to_dev(r["wr"]), to_dev(r["wi"]),
                          precision=1) for r in order]
    done = set(srv.progress())  # admission happens here
    st = srv.stats()
    assert st["running"] + len(done) == (2 if bypass else 1)
    while len(done) < len(tickets):
        done |= set(srv.progress(wait=True))
    for r, t in zip(order, tickets):
        X, s = srv.result(t)
        Xa, sa = _alone(dev[r["n"]][r["index"]][0], to_dev(r["wr"]), to_dev(r["wi"]), 1)
        assert np.array_equal(s.cpu().numpy(), sa) and np.array_equal(X.cpu().numpy(), Xa)


def test_oversized_request_is_refused(pool):
    p, dev = pool
    srv = hs.Server(1 << 20, max_jobs=2, max_merge_shifts=64)
    r = [r for r in _requests(p, 30, 13) if r["n"] == 1024][0]
    with pytest.raises(hs.HseinError) as e:
        srv.submit(dev[1024][r["index"]][0], to_dev(r["wr"]), to_dev(r["wi"]), precision=1)
    assert e.value.code == -2


def test_short_poisson_stream(pool):
    p, dev = pool
    reqs = _requests(p, 120, 14)
    srv = hs.Server(8 * GB, max_jobs=8, max_merge_shifts=4096)
    times, results = bench.replay_stream(srv, dev["balanced"], reqs, torch)
    lat = np.array([c - a for a, c in times])
    assert np.all(lat > 0)
    conv = 0
    for j, r in enumerate(reqs):
        X, s = results[j]
        sh = s.cpu().numpy()
        conv += int(sum(2 if w != 0 else 1 for w, st in zip(r["wi"], sh) if st == 0))
        if j % 10:
            continue
        # the result alone, for every tenth request; the residual of the
        # converged columns (FP64 on the device; graded requests in the
        # balanced basis, where the solve ran)
        Hp, Hb, e = dev["balanced"][r["n"]][r["index"]]
        H = Hb if r["graded"] else Hp
        Xa, sa = _alone(H, to_dev(r["wr"]), to_dev(r["wi"]), 1)
        if r["graded"]:
            Xb = to_dev(Xa)
            hs.unbalance(Xb, to_dev(r["wi"]), e)
            Xua = Xb.cpu().numpy()
        else:
            Xua = Xa
        assert np.array_equal(sh, sa) and np.array_equal(X.cpu().numpy(), Xua)
        X = to_dev(Xa)
        offs = hi.column_offsets(r["wi"])
        HX = (H @ X).cpu().numpy()
        Xh = X.cpu().numpy()
        hn1 = H.abs().sum(0).max().item()
        for l in np.nonzero(sh == 0)[0]:
            c0 = offs[l]
            if r["wi"][l] != 0:
                lam = complex(r["wr"][l], r["wi"][l])
                x, hx = Xh[:, c0] + 1j * Xh[:, c0 + 1], HX[:, c0] + 1j * HX[:, c0 + 1]
            else:
                lam, x, hx = r["wr"][l], Xh[:, c0], HX[:, c0]
            res = np.abs(hx - lam * x).sum() / (hn1 * np.abs(x).sum())
            assert res <= 100 * r["n"] * EPS
    print("short stream: %d requests, %d converged columns, p50 %.2f ms p99 %.2f ms, stats %s"
          % (len(reqs), conv, 1e3 * np.percentile(lat, 50), 1e3 * np.percentile(lat, 99),
             srv.stats()))
