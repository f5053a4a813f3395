#!/usr/bin/env python
"""Throughput benchmark: eigenvectors per second on the mixed real/complex
workload (n = 4096; 512 real + 256 complex-conjugate shifts, i.e. 1024
solution columns; quasi-triangular T with known eigenvalues, Haar similarity,
Hessenberg reduction; seeded unit-norm N(0,1) starting vectors).

One step = hsein_solve (all tile columns: diagonal sweeps, shared-H updates,
normalization and Givens backtransform) + hsein_backtransform (z = Q0 x) on
inputs resident in HBM.  H and Q0 (134 MB each) are larger than L2, so no
flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank solves its own seeded instance of the same
size (independent problems, no collective on the data path: weak scaling);
the elapsed time is the maximum over ranks.  Rank 0 prints one JSON line.

--impl reference times the CPU oracle (Henry's algorithm per shift, OpenMP
over shifts) on the host cores on a bounded sample of the same workload.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "eigvecs/s vs plain FP64 GPU at residual≤100nε; tensor-peak %; p50/p99 ms"
UNIT = "eigvecs/s"
EPS = 2.0 ** -53
# FP64 peak of the CUDA cores from unit counts and the clock: GB300's nominal
# 1.25 TFLOP/s at 2070 MHz over 152 SMs is 2 FP64 FMAs (4 flops) per SM per
# clock; the roofline takes that times the SM count times the median SM clock
# sampled during the timed region.  Beside it: the rate the library's DFMA
# probe reaches (hsein_fp64_rate) and the older estimate from the measured
# BF16 peak x the nominal FP64/BF16 ratio 1.25/2250.
FP64_FLOPS_PER_SM_CLK = 4.0
NOMINAL_FP64_OVER_BF16 = 1.25 / 2250.0


_T0 = time.perf_counter()


def log(msg):
    """Progress on stderr (the JSON line is the only stdout output)."""
    sys.stderr.write("[bench %7.1f s] %s\n" % (time.perf_counter() - _T0, msg))
    sys.stderr.flush()


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--br", type=int, default=64)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batching workload")
    ap.add_argument("--batch-steps", type=int, default=5)
    ap.add_argument("--no-serve", action="store_true", help="skip the serving workload")
    ap.add_argument("--serve-requests", type=int, default=20000,
                    help="requests in the serving stream at 200 requests/s (the workload)")
    ap.add_argument("--capacity-requests", type=int, default=1500,
                    help="requests per stream of the serving capacity sweep (0: skip)")
    ap.add_argument("--no-c2", action="store_true", help="skip the n = 8192 precision workload")
    ap.add_argument("--c2-steps", type=int, default=5)
    ap.add_argument("--cpu-sample", type=int, default=256, help="shifts in the oracle sample")
    ap.add_argument("--no-reduction", action="store_true",
                    help="skip timing the Hessenberg reduction A -> (H, Q0)")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return p, "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.strip().split(", ") for r in self.file.read().splitlines() if r.strip()]
        self.file.close()
        os.unlink(self.file.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for name, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(backend="nccl"):
    """Rank, world size and local rank from the launcher's environment; joins
    the process group when there is more than one rank (NCCL on GPUs; gloo for
    host-only runs).  Each rank drives its own GPU."""
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if backend == "nccl":
        torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        if backend == "nccl":
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group(backend)
    return rank, world, local


def _reduce(v, world, op, device):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=op)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world, device="cuda"):
    """The slowest rank's time: the whole job is done when it is."""
    import torch.distributed as dist
    return _reduce(v, world, dist.ReduceOp.MAX if world > 1 else None, device)


def sum_over_ranks(v, world, device="cuda"):
    """Units processed by all ranks together (each rank solves its own
    seeded instance, so their converged-column counts may differ)."""
    import torch.distributed as dist
    return _reduce(v, world, dist.ReduceOp.SUM if world > 1 else None, device)


def rank_seed(rank):
    """Seed of the instance a rank solves (weak scaling: one instance per rank)."""
    return 1 + rank


def update_flops(n, ncol, br):
    """Algorithmic flops of all shared-H products of one solve: for every tile
    column J >= 1 a (p0 x br) times (br x 2 ncol) product."""
    N = (n + br - 1) // br
    b0 = n - (N - 1) * br
    total = 0
    for J in range(1, N):
        p0 = b0 + (J - 1) * br
        total += 2 * p0 * br * 2 * ncol
    return total, N - 1


def diag_flops(inst, br):
    """Algorithmic flops of all diagonal-tile sweeps of one solve (k_diag, one
    launch per tile column): 5 n b_r per solution column, the count of the
    per-column work on the diagonal tiles (Table "flops-vector"; a complex
    shift owns two columns).  Returns (total, launches)."""
    n = inst.n
    N = (n + br - 1) // br
    return 5.0 * n * br * inst.ncol, N


def fp64_peak_tflops(sm_mhz, sms):
    """FP64 CUDA-core peak from unit counts and the sampled SM clock."""
    return FP64_FLOPS_PER_SM_CLK * sms * sm_mhz * 1e6 / 1e12


def spawn_pool(workers, blas_threads):
    """A pool of spawned processes (safe beside an initialized CUDA context)
    whose BLAS uses blas_threads threads, at a lower scheduling priority than
    this process (which generates and measures the headline workload)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    keys = ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    for k in keys:
        os.environ[k] = str(blas_threads)
    try:
        ex = cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn"),
                                    initializer=os.nice, initargs=(10,))
        ex.submit(int, 0).result()  # start the workers with these settings
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return ex


def _gen_config2():
    import hsein_inputs as hi
    t0 = time.perf_counter()
    inst = hi.config2()
    return inst, time.perf_counter() - t0


def _gen_serving_pool():
    import hsein_inputs as hi
    t0 = time.perf_counter()
    pool = hi.serving_pool()
    return pool, time.perf_counter() - t0


def column_vectors(X, wr, wi):
    """[(lambda, vector)] from the column layout (complex: [re, im])."""
    import numpy as np
    out, c = [], 0
    for l in range(len(wr)):
        if wi[l] != 0:
            out.append((complex(wr[l], wi[l]), X[:, c] + 1j * X[:, c + 1]))
            c += 2
        else:
            out.append((float(wr[l]), X[:, c]))
            c += 1
    return out


def chordal_angle(x, y):
    import numpy as np
    x = np.asarray(x, dtype=np.complex128)
    y = np.asarray(y, dtype=np.complex128)
    nx, ny = np.linalg.norm(x), np.linalg.norm(y)
    if nx == 0 or ny == 0:
        return float("inf")
    x, y = x / nx, y / ny
    d = np.vdot(y, x)
    return float(np.linalg.norm(x - y * (d / abs(d) if abs(d) > 0 else 1.0)))


def accuracy_vs_oracle(inst, idx, Xg, sg, Xo, so, hnorm):
    """Angles between the GPU's and the oracle's eigenvectors for the sampled
    shifts idx (Xo, so: the oracle's results for them), the worst ratio to the
    first-order bound n eps ||H|| / gap (gap = distance to the nearest other
    eigenvalue) and whether the statuses agree."""
    import numpy as np
    import hsein_inputs as hi
    offs = hi.column_offsets(inst.wi)
    vo = column_vectors(Xo, inst.wr[idx], inst.wi[idx])
    worst, worst_ratio, worst_sep, n_sep, cnt = 0.0, 0.0, 0.0, 0, 0
    eigs = np.asarray(inst.eigs)
    for j, l in enumerate(idx):
        if sg[l] != 0 or so[j] != 0:
            continue
        c0, c1 = offs[l], offs[l + 1]
        xg = Xg[:, c0] + 1j * Xg[:, c0 + 1] if c1 - c0 == 2 else Xg[:, c0]
        lam = vo[j][0]
        a = chordal_angle(xg, vo[j][1])
        d = np.sort(np.abs(eigs - lam))
        gap = d[1] if len(d) > 1 else np.inf
        worst = max(worst, a)
        worst_ratio = max(worst_ratio, a / (inst.n * EPS * hnorm / gap))
        if gap >= 1e-3 * hnorm:
            n_sep += 1
            worst_sep = max(worst_sep, a)
        cnt += 1
    return {"angle_max_vs_oracle": worst,
            "angle_over_first_order_bound_max": worst_ratio,
            "angle_max_separated": worst_sep if n_sep else None, "separated_columns": n_sep,
            "columns_compared": cnt,
            "status_equal": bool(np.array_equal(np.asarray(sg)[idx], so)),
            "gate": "angle <= 1e-10 (gap >= 1e-3 ||H||_inf), else <= 2 n eps ||H|| / gap"}


def source_hash(relpath):
    with open(os.path.join(ROOT, relpath), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def profiled_traffic(kernel_file, summary):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current source of the kernel; None otherwise."""
    path = os.path.join(ROOT, "profiles", summary)
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("source_sha256") != source_hash(kernel_file):
        return None
    try:
        return float(vals["dram_bytes_per_launch_full_size"])
    except (KeyError, ValueError):
        return None


def cpu_baseline(inst, sample_shifts):
    """The oracle as it stands, on all host cores, on a seeded sample of the
    workload's shifts; returns (columns/s, cores, description)."""
    import numpy as np

    import hsein_inputs as hi
    import oracle
    offs = hi.column_offsets(inst.wi)
    idx = np.sort(np.argsort(hi.uniform(1234, 7, inst.m), kind="stable")[:sample_shifts])
    wr, wi = inst.wr[idx], inst.wi[idx]
    B = np.concatenate([inst.B[:, offs[l]:offs[l + 1]] for l in idx], axis=1)
    oracle.hsein(inst.H[:64, :64], wr[:1] * 0, wi[:1] * 0, None)  # load and warm the library
    t0 = time.perf_counter()
    X, st = oracle.hsein(inst.H, wr, wi, B)
    Z = oracle.q0_apply(inst.Q0, X)
    dt = time.perf_counter() - t0
    cols = X.shape[1]
    cores = os.cpu_count()
    desc = ("%d of %d shifts (%d columns) of the same instance: Henry solve + normalization + "
            "backtransform + z = Q0 x, OpenMP over shifts, %.2f s wall" % (len(idx), inst.m, cols, dt))
    return cols / dt, cores, desc, (idx, X, st)


def run_reference(args):
    """The oracle on the host cores, on the same workload, each step a bounded
    sample of its shifts."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np

    import hsein_inputs as hi
    import oracle
    inst = hi.config1(seed=1)
    offs = hi.column_offsets(inst.wi)
    per_step = 96
    order = np.argsort(hi.uniform(4321, 7, inst.m), kind="stable")

    def step(s):
        idx = order[(s * per_step) % inst.m:(s * per_step) % inst.m + per_step]
        wr, wi = inst.wr[idx], inst.wi[idx]
        B = np.concatenate([inst.B[:, offs[l]:offs[l + 1]] for l in idx], axis=1)
        X, st = oracle.hsein(inst.H, wr, wi, B)
        oracle.q0_apply(inst.Q0, X)
        return X.shape[1]

    for s in range(args.warmup):
        step(s)
    t0 = time.perf_counter()
    cols = 0
    for s in range(args.steps):
        cols += step(args.warmup + s)
    dt = time.perf_counter() - t0
    value = cols / dt
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": workload_config(inst, args.br),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%d shifts per step of the same instance (Henry solve + "
                                   "normalization + backtransform + z = Q0 x)" % per_step},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def measure_batch(args, torch, hs, hi, fp64_peak):
    """The batching workload (256 independent instances, n log-uniform in
    [64, 2048], all real eigenvalues as shifts, FP64 throughout) in one
    captured CUDA graph per batch, configuration chosen by the autotuner."""
    import numpy as np
    t0 = time.perf_counter()
    insts = hi.config3(workers=min(16, os.cpu_count() or 1))
    t_gen = time.perf_counter() - t0
    f = lambda a: torch.as_tensor(np.asfortranarray(a), dtype=torch.float64, device="cuda")
    dev = [(f(i.H), f(i.wr), f(i.wi), f(i.B)) for i in insts]
    b = hs.Batch(dev, streams=16, br_policy=1)
    cfg, ms_tune = b.autotune()
    b.solve()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.batch_steps + 1)]
    evs[0].record(stream)
    for i in range(args.batch_steps):
        b.solve()
        evs[i + 1].record(stream)
    torch.cuda.synchronize()
    per = [evs[i].elapsed_time(evs[i + 1]) for i in range(args.batch_steps)]
    conv = sum(int((st.cpu().numpy() == 0).sum()) for st in b.status)  # real shifts: 1 column each
    total = sum(i.m for i in insts)
    ms = float(np.mean(per))
    # algorithmic flops of the batch at the chosen tile heights: every
    # instance's shared-H products and diagonal-tile sweeps
    pol = cfg.get("br_policy", 0)

    def br_of(n):
        if pol == 1:
            return 32 if n < 512 else 64
        if pol == 2:
            return 16 if n < 256 else (32 if n < 1024 else 64)
        return 64
    flops = 0.0
    for i in insts:
        br = br_of(i.n)
        flops += update_flops(i.n, i.ncol, br)[0] + diag_flops(i, br)[0]
    achieved = flops / (ms * 1e-3) / 1e12
    return {"workload": "256 independent instances, n = round(exp(U[ln 64, ln 2048])), 25%% with "
                        "complex pairs, all real eigenvalues as shifts (%d), FP64" % total,
            "value": conv / (ms * 1e-3), "unit": UNIT, "ms_per_batch": ms,
            "latency": {"p50": float(np.percentile(per, 50)), "p99": float(np.percentile(per, 99)),
                        "unit": "ms", "of": "%d batches" % args.batch_steps},
            "converged_columns": conv, "columns": total, "autotuned": cfg,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": fp64_peak,
                         "unit": "TFLOP/s", "frac": achieved / fp64_peak,
                         "algorithmic_flops": flops,
                         "what": "shared-H products (2 p0 b_r 2 ncol per tile column) + "
                                 "diagonal-tile sweeps (5 n b_r per column), all instances"},
            "autotune_ms_best": ms_tune, "host_launches_per_batch": 1,
            "generation_s": t_gen, "sizes": {"min": min(i.n for i in insts),
                                             "max": max(i.n for i in insts),
                                             "sum": sum(i.n for i in insts)}}


def replay_stream(srv, pool_dev, reqs, torch, keep=True, precision=1):
    """Replay a request stream in real time on a hs.Server: each request is
    submitted at its arrival time (seconds after the start) and progress()
    is driven in between.  pool_dev[n][i] = (H, Hb, e): the matrix, the
    power-of-two balanced form of its graded variant and the balancing
    exponents.  Every request runs with split-precision products; a graded
    one on the balanced matrix (one digit exponent per row could not hold
    the 10^300 range of a graded row), mapped back by the server.  Returns
    per request (arrival,
    completion) host times in seconds since the start, and the results
    {request index: (X, status)} (keep=False: only the status, on the host)."""
    f = lambda a: torch.as_tensor(a, dtype=torch.float64, device="cuda")
    shifts = [(f(r["wr"]), f(r["wi"])) for r in reqs]
    torch.cuda.synchronize()
    t_done = [None] * len(reqs)
    of = {}
    results = {}
    t0 = time.perf_counter()
    i = 0
    while len(results) < len(reqs):
        now = time.perf_counter() - t0
        while i < len(reqs) and reqs[i]["t"] <= now:
            r = reqs[i]
            H, Hb, e = pool_dev[r["n"]][r["index"]]
            # graded requests run on the balanced form of their matrix
            tk = srv.submit(Hb if r["graded"] else H, shifts[i][0], shifts[i][1],
                            precision=precision, exps=e if r["graded"] else None)
            of[tk] = i
            i += 1
        done = srv.progress(wait=(i == len(reqs)))
        now = time.perf_counter() - t0
        for tk in done:
            j = of.pop(tk)
            t_done[j] = now
            X, st = srv.result(tk)
            results[j] = (X, st) if keep else st.cpu().numpy()
        if not done and i < len(reqs):
            time.sleep(max(0.0, min(reqs[i]["t"] - now, 2e-4)))
    return [(r["t"], t_done[j]) for j, r in enumerate(reqs)], results


def measure_serving(args, torch, hs, hi, pool, t_gen):
    """The serving workload: a Poisson stream (200 requests/s) of solves on a
    pre-generated pool, replayed in real time through hs.Server; then the
    capacity sweep: shorter streams at 2, 4 and 8 times the rate, and the
    8-times stream again with FP64 products (precision 0) for every request,
    so that the saturated throughput of the split-precision service stands
    beside the plain FP64 service's."""
    import numpy as np
    f = lambda a: torch.as_tensor(np.asfortranarray(a), dtype=torch.float64, device="cuda")
    pool_dev = {n: [(f(i.H),) + tuple(hs.balance(f(i.Hg))) for i in lst]
                for n, lst in pool.items()}
    torch.cuda.synchronize()
    srv = hs.Server(64 << 30, max_jobs=8, max_merge_shifts=4096)
    # warm-up: one request per size class and kind, outside the stream
    warm = [dict(r, t=0.0) for r in hi.serving_requests(pool, 64, seed=41)]
    seen, wl = set(), []
    for r in warm:
        if (r["n"], r["graded"]) not in seen:
            seen.add((r["n"], r["graded"]))
            wl.append(r)
    replay_stream(srv, pool_dev, wl, torch, keep=False)
    replay_stream(srv, pool_dev, wl, torch, keep=False, precision=0)

    def run(count, rate, precision, seed=4, server=None):
        srv_ = server or srv
        reqs = hi.serving_requests(pool, count, seed=seed, rate=rate)
        s0 = srv_.stats()
        times, status = replay_stream(srv_, pool_dev, reqs, torch, keep=False, precision=precision)
        s1 = srv_.stats()
        lat = np.array([c - a for a, c in times]) * 1e3
        conv = sum(int(sum(2 if w != 0 else 1 for w, st in zip(r["wi"], status[j]) if st == 0))
                   for j, r in enumerate(reqs))
        cols = sum(len(r["wr"]) + int((r["wi"] != 0).sum()) for r in reqs)
        span = max(c for a, c in times)
        return {"rate_per_s": rate, "requests": count,
                "precision": "split" if precision == 1 else "fp64",
                "value": conv / span, "unit": UNIT, "span_s": span,
                "arrival_span_s": reqs[-1]["t"],
                "latency": {"p50": float(np.percentile(lat, 50)),
                            "p99": float(np.percentile(lat, 99)), "unit": "ms"},
                "converged_columns": conv, "columns": cols,
                "requests_admitted": s1["requests_admitted"] - s0["requests_admitted"],
                "solves_admitted": s1["solves_admitted"] - s0["solves_admitted"]}

    main = run(args.serve_requests, 200.0, 1)
    out = {"workload": "Poisson stream, 200 requests/s, %d requests; n uniform over %s, k "
                       "uniform in [1, n/4]; 30%% graded D H D^-1 (u ~ U[-150, 150]) solved "
                       "on their power-of-two balanced form; 30%% with complex pairs; "
                       "split-precision products; rho e starting vectors"
                       % (args.serve_requests, list(hi.SERVE_SIZES)),
           "value": main["value"], "unit": UNIT, "span_s": main["span_s"],
           "latency": dict(main["latency"], of="%d requests, arrival to completion"
                           % args.serve_requests),
           "converged_columns": main["converged_columns"], "columns": main["columns"],
           "requests_admitted": main["requests_admitted"],
           "solves_admitted": main["solves_admitted"],
           "server": {"arena_gb": 64, "max_jobs": 8, "max_merge_shifts": 4096},
           "pool": {str(n): len(v) for n, v in pool.items()}, "generation_s": t_gen,
           "value_is": "converged columns / (last completion - first arrival): the offered "
                       "load while the service keeps up (see capacity)"}
    if args.capacity_requests > 0:
        cap = [run(args.capacity_requests, 200.0 * k, 1, seed=50 + k) for k in (2, 4, 8)]
        cap.append(run(args.capacity_requests, 1600.0, 0, seed=58))
        # the 2x stream again with head-of-line bypass (up to 8 later requests
        # may pass one that does not fit the arena)
        srv_b = hs.Server(64 << 30, max_jobs=8, max_merge_shifts=4096, max_bypass=8)
        byp = run(args.capacity_requests, 400.0, 1, seed=52, server=srv_b)
        del srv_b
        sat = [c for c in cap if c["span_s"] > 1.2 * c["arrival_span_s"]]
        out["capacity"] = {
            "streams": cap,
            "saturated_split_value": max((c["value"] for c in cap if c["precision"] == "split"),
                                         default=None),
            "saturated_fp64_value": cap[-1]["value"],
            "split_over_fp64": cap[2]["value"] / cap[-1]["value"] if cap[-1]["value"] else None,
            "saturated_streams": [(c["rate_per_s"], c["precision"]) for c in sat],
            "bypass_2x": {"p50": byp["latency"]["p50"], "p99": byp["latency"]["p99"],
                          "value": byp["value"], "without_bypass_p99": cap[0]["latency"]["p99"],
                          "how": "the same 2x stream with hsein_server_set_bypass(8)"},
            "how": "%d-request streams at 2x, 4x, 8x the rate (split products) and at 8x with "
                   "FP64 products; a stream whose completion span exceeds its arrival span is "
                   "saturated, and its eigvecs/s is the service's capacity"
                   % args.capacity_requests}
    return out


def measure_reduction(inst, torch, hs, fp64_peak):
    """The precursor step A = Q0 H Q0^T (hsein_gehrd) on the workload's own A:
    two timed calls after one warm-up (CUDA events on the calling stream),
    with invariant checks on the device.  Algorithmic work of the level-2
    reduction with Q0 accumulated: per step 4 m^2 (left reflection of the
    trailing block) + 4 n m (right reflection) + 4 n m (Q0 P) flops,
    m = n - k - 1, i.e. 16/3 n^3 in total."""
    import numpy as np
    n = inst.n
    dA = torch.as_tensor(np.asfortranarray(inst.A), dtype=torch.float64, device="cuda")
    hs.gehrd(dA)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 2
    e0.record()
    for _ in range(reps):
        dH, dQ = hs.gehrd(dA)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    flops = sum(4.0 * (n - k - 1) ** 2 + 8.0 * n * (n - k - 1) for k in range(n - 2))
    achieved = flops / (ms * 1e-3) / 1e12
    eye = torch.eye(n, dtype=torch.float64, device="cuda")
    orth = float((dQ.t() @ dQ - eye).abs().max())
    back = float((dQ @ dH @ dQ.t() - dA).abs().max()) / float(dA.abs().max())
    lapack = float(np.abs(np.abs(dH.cpu().numpy()) - np.abs(inst.H)).max() / np.abs(inst.A).max())
    below = int(torch.count_nonzero(torch.tril(dH, -2)))
    return {"n": n, "ms": ms, "unit": "ms per reduction (A -> H, Q0)",
            "roofline": {"bound": "alu", "achieved": achieved, "peak": fp64_peak,
                         "unit": "TFLOP/s", "frac": achieved / fp64_peak,
                         "algorithmic_flops": flops},
            "gpu_launches": 1 + 4 * (n - 2),
            "checks": {"max_abs_QtQ_minus_I": orth, "max_abs_QHQt_minus_A_over_max_A": back,
                       "max_abs_absH_minus_abs_lapack_H_over_max_A": lapack,
                       "nonzeros_below_subdiagonal": below}}


def residual_max_device(torch, dH, X, wr, wi, status, n):
    """Largest normwise residual ||H x - lambda x||_1 / (||H||_1 ||x||_1) over
    the converged columns, in units of n eps (FP64 on the device)."""
    import numpy as np
    import hsein_inputs as hi
    HX = dH @ X
    hn1 = float(dH.abs().sum(dim=0).max())
    st = status.cpu().numpy()
    offs = hi.column_offsets(wi)
    ok = st == 0
    dev = X.device
    worst = 0.0
    re = np.nonzero(ok & (np.asarray(wi) == 0))[0]
    if len(re):
        c = torch.as_tensor(offs[re], device=dev)
        lam = torch.as_tensor(np.asarray(wr)[re], dtype=torch.float64, device=dev)
        num = (HX[:, c] - X[:, c] * lam).abs().sum(dim=0)
        den = X[:, c].abs().sum(dim=0)
        worst = max(worst, float((num / (hn1 * den)).max()))
    cx = np.nonzero(ok & (np.asarray(wi) != 0))[0]
    if len(cx):
        c = torch.as_tensor(offs[cx], device=dev)
        lr = torch.as_tensor(np.asarray(wr)[cx], dtype=torch.float64, device=dev)
        li = torch.as_tensor(np.asarray(wi)[cx], dtype=torch.float64, device=dev)
        xr, xi, hr, hi_ = X[:, c], X[:, c + 1], HX[:, c], HX[:, c + 1]
        rr = hr - xr * lr + xi * li
        ri = hi_ - xi * lr - xr * li
        num = torch.sqrt(rr * rr + ri * ri).sum(dim=0)
        den = torch.sqrt(xr * xr + xi * xi).sum(dim=0)
        worst = max(worst, float((num / (hn1 * den)).max()))
    return worst / (n * EPS)


def timed_steps(torch, stream, step, steps):
    """Run `steps` steps between CUDA events on `stream` (one event between
    consecutive steps); the per-step times in ms."""
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    evs[0].record(stream)
    for i in range(steps):
        step()
        evs[i + 1].record(stream)
    torch.cuda.synchronize()
    return [evs[i].elapsed_time(evs[i + 1]) for i in range(steps)]


def profiled_steps(torch, hs, solver, stream, step, steps):
    """The same steps again with a CUDA event pair around every launch of the
    solver (the phase breakdown and the per-launch kernel times): the events
    themselves lengthen a step, so the throughput and latency come from the
    plain region and this one supplies the per-kernel figures.  Returns the
    phases and this region's ms per step."""
    hs.hsein_plan_set_profiling(solver.plan, True)
    hs.hsein_plan_profile(solver.plan, reset=True)
    per = timed_steps(torch, stream, step, steps)
    prof = hs.hsein_plan_profile(solver.plan, reset=True)
    hs.hsein_plan_set_profiling(solver.plan, False)
    return prof, float(sum(per)) / steps


def measure_instance(torch, hs, inst, precision, steps, warmup, br=64, keep=False):
    """Time `steps` steps (hsein_solve + hsein_backtransform) of one instance
    in one precision mode, inputs resident in HBM; per-step latency, phases,
    residuals and converged columns."""
    import numpy as np
    import hsein_inputs as hi
    f = lambda a: torch.as_tensor(np.asfortranarray(a), dtype=torch.float64, device="cuda")
    dH, dwr, dwi, dB, dQ = f(inst.H), f(inst.wr), f(inst.wi), f(inst.B), f(inst.Q0)
    n, ncol = inst.n, inst.ncol
    X = torch.empty((ncol, n), dtype=torch.float64, device="cuda").t()
    Z = torch.empty((ncol, n), dtype=torch.float64, device="cuda").t()
    status = torch.empty(inst.m, dtype=torch.int32, device="cuda")
    solver = hs.Solver(n, inst.m_real, inst.m_cplx, br=br, precision=precision)

    def step():
        solver.solve(dH, dwr, dwi, dB, X=X, status=status, check=False)
        solver.backtransform(dQ, X, Z=Z)

    for _ in range(max(3, warmup)):
        step()
    torch.cuda.synchronize()
    if solver.device_status() < 0:
        raise RuntimeError("device status %d" % solver.device_status())
    stream = torch.cuda.current_stream()
    graph = solver.graph(dH, dwr, dwi, dB, dQ, X=X, status=status, Z=Z)
    graph.launch()
    per = timed_steps(torch, stream, graph.launch, steps)
    ms = float(sum(per)) / steps
    ms_eager = float(sum(timed_steps(torch, stream, step, steps))) / steps
    prof, ms_events = profiled_steps(torch, hs, solver, stream, step, steps)
    del graph
    sh = status.cpu().numpy()
    offs = hi.column_offsets(inst.wi)
    conv = int(sum(offs[l + 1] - offs[l] for l in range(inst.m) if sh[l] == 0))
    out = {"value": conv / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
           "latency": {"p50": float(np.percentile(per, 50)), "p99": float(np.percentile(per, 99)),
                       "unit": "ms", "of": "%d steps" % steps,
                       "launch": "one CUDA graph per step"},
           "ms_per_step_eager": ms_eager,
           "residual_max_over_n_eps": residual_max_device(torch, dH, X, inst.wr, inst.wi,
                                                          status, n),
           "not_converged": int((sh != 0).sum()), "converged_columns": conv,
           "phases": {k: {"ms_per_step": v[0] / steps, "launches_per_step": v[1] / steps}
                      for k, v in prof.items()},
           "ms_per_step_with_launch_events": ms_events}
    host = (X.cpu().numpy(), sh) if keep else None
    del solver, dH, dQ, dB, X, Z
    torch.cuda.empty_cache()
    return out, host


def measure_config2(args, torch, hs, inst, t_gen, fp64_peak, bf16_peak):
    """The precision workload (n = 8192, 2048 real shifts): split-precision
    products against FP64 products on the same instance, with the angles of a
    seeded sample of columns against the oracle."""
    import numpy as np
    import hsein_inputs as hi
    import oracle
    sp, (Xs, ss) = measure_instance(torch, hs, inst, 1, args.c2_steps, args.warmup, keep=True)
    fp, (Xf, sf) = measure_instance(torch, hs, inst, 0, 2, 3, keep=True)
    idx = np.sort(np.argsort(hi.uniform(4242, 7, inst.m), kind="stable")[:64])
    Xo, so = oracle.hsein(inst.H, inst.wr[idx], inst.wi[idx], inst.B[:, idx])
    hn = oracle.hnorm_inf(inst.H)
    sp["accuracy"] = accuracy_vs_oracle(inst, idx, Xs, ss, Xo, so, hn)
    fp["accuracy"] = accuracy_vs_oracle(inst, idx, Xf, sf, Xo, so, hn)
    # split against FP64 products, every converged column
    worst = 0.0
    for l in np.nonzero((ss == 0) & (sf == 0))[0]:
        worst = max(worst, chordal_angle(Xs[:, l], Xf[:, l]))
    uf, ul = update_flops(inst.n, inst.ncol, 64)
    q0f = 2.0 * inst.n * inst.n * inst.ncol
    ph = sp["phases"]
    df, dl = diag_flops(inst, 64)
    t_diag = ph["diag_sweep"]["ms_per_step"] / max(1e-9, ph["diag_sweep"]["launches_per_step"])
    sp["roofline_k_diag"] = {"bound": "alu", "achieved": df / dl / (t_diag * 1e-3) / 1e12,
                             "peak": fp64_peak, "unit": "TFLOP/s"}
    sp["roofline_k_diag"]["frac"] = sp["roofline_k_diag"]["achieved"] / fp64_peak
    sp["tensor"] = {
        "peak": bf16_peak, "unit": "TFLOP/s",
        "shared_h_update_frac": 28.0 * uf / (ph["shared_h_update"]["ms_per_step"] * 1e-3) / 1e12
        / bf16_peak,
        "q0_backtransform_frac": 28.0 * q0f / (ph["q0_backtransform"]["ms_per_step"] * 1e-3)
        / 1e12 / bf16_peak}
    t_upd = fp["phases"]["shared_h_update"]["ms_per_step"]
    fp["roofline_k_update"] = {"bound": "alu", "achieved": uf / (t_upd * 1e-3) / 1e12,
                               "peak": fp64_peak, "unit": "TFLOP/s"}
    fp["roofline_k_update"]["frac"] = fp["roofline_k_update"]["achieved"] / fp64_peak
    return {"workload": "n = 8192, 2048 real shifts, eigenvalues U[-n, n] with minimum gap "
                        "1e-2, tile height 64; split-precision products (BF16 digit slices on "
                        "the tensor cores) against FP64 products",
            "split": sp, "fp64": fp,
            "split_over_fp64": sp["value"] / fp["value"] if fp["value"] else None,
            "angle_max_split_vs_fp64": worst, "generation_s": t_gen}


def workload_config(inst, br):
    return {
        "workload": "mixed real/complex shifts: n=4096, 512 real + 256 complex shifts "
                    "(1024 columns), split-precision products (BF16 digit slices on the "
                    "tensor cores; plain_fp64: FP64 products), tile height %d" % br,
        "n": inst.n, "m_real": inst.m_real, "m_cplx": inst.m_cplx, "columns": inst.ncol,
        "br": br, "precision": "split (plain_fp64: fp64)",
        "l2": "no flush: H and Q0 (134 MB each) are larger than L2",
    }


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    import numpy as np
    import torch

    import hsein_inputs as hi
    import paper_2101_05063_gb300 as hs

    rank, world, local = dist_setup()
    # the larger workloads' inputs are generated in spawned processes while
    # the GPU measures the headline workload
    bg, futs = None, {}
    if rank == 0 and world == 1 and (not args.no_c2 or not args.no_serve):
        # one worker, the n = 8192 workload first (it is needed first), all
        # cores for its BLAS
        bg = spawn_pool(1, os.cpu_count() or 1)
        if not args.no_c2:
            futs["c2"] = bg.submit(_gen_config2)
        if not args.no_serve:
            futs["serve"] = bg.submit(_gen_serving_pool)
    dev = torch.device("cuda", local)
    log("generating the n = 4096 workload")
    inst = hi.config1(seed=rank_seed(rank), keep_a=True)
    log("generated")
    n, ncol, m = inst.n, inst.ncol, inst.m
    f = lambda a: torch.as_tensor(np.asfortranarray(a), dtype=torch.float64, device=dev)
    dH, dwr, dwi, dB, dQ = f(inst.H), f(inst.wr), f(inst.wi), f(inst.B), f(inst.Q0)
    X = torch.empty((ncol, n), dtype=torch.float64, device=dev).t()
    Z = torch.empty((ncol, n), dtype=torch.float64, device=dev).t()
    status = torch.empty(m, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    offs = hi.column_offsets(inst.wi)
    hn1 = np.abs(inst.H).sum(axis=0).max()

    def residual_max(sh):
        """Largest normwise residual over the converged columns (FP64 on the
        device), in units of n eps."""
        HX = (dH @ X).cpu().numpy()
        Xh = X.cpu().numpy()
        worst = 0.0
        for l in range(m):
            if sh[l] != 0:
                continue
            c0, c1 = offs[l], offs[l + 1]
            if c1 - c0 == 2:
                lam = complex(inst.wr[l], inst.wi[l])
                x, hx = Xh[:, c0] + 1j * Xh[:, c0 + 1], HX[:, c0] + 1j * HX[:, c0 + 1]
            else:
                lam, x, hx = inst.wr[l], Xh[:, c0], HX[:, c0]
            worst = max(worst, np.abs(hx - lam * x).sum() / (hn1 * np.abs(x).sum()))
        return worst / (n * EPS)

    def measure(precision, sample_clocks, method=0, steps=None, givens=0):
        """Warm up, check, then time `steps` (default args.steps) steps of one
        precision mode / method / rotation storage."""
        nsteps = steps or args.steps
        solver = hs.Solver(n, inst.m_real, inst.m_cplx, br=args.br, precision=precision,
                           device=dev, method=method, givens=givens)

        def step():
            solver.solve(dH, dwr, dwi, dB, X=X, status=status, check=False)
            solver.backtransform(dQ, X, Z=Z)

        for _ in range(max(3, args.warmup)):
            step()
        torch.cuda.synchronize()
        dstat = solver.device_status()
        if dstat < 0:
            raise RuntimeError("device status %d" % dstat)
        sh = status.cpu().numpy()
        worst = residual_max(sh)
        sampler = ClockSampler(torch.cuda.current_device()) if (rank == 0 and sample_clocks) else None
        if sampler:
            sampler.start()
        # the same step captured as one CUDA graph (hsein_graph_create): the
        # throughput and latency are timed through it
        graph = solver.graph(dH, dwr, dwi, dB, dQ, X=X, status=status, Z=Z)
        graph.launch()
        barrier(world)
        torch.cuda.synchronize()
        # one event between consecutive steps: per-step latency and the total
        per_step = timed_steps(torch, stream, graph.launch, nsteps)
        barrier(world)
        ms = float(sum(per_step))
        lat = {"p50": float(np.percentile(per_step, 50)), "p99": float(np.percentile(per_step, 99)),
               "unit": "ms", "of": "%d steps" % nsteps, "launch": "one CUDA graph per step"}
        # the same steps launched kernel by kernel from the host
        lat["ms_per_step_eager"] = float(sum(timed_steps(torch, stream, step, nsteps))) / nsteps
        # the per-launch kernel times (phases, roofline) from a timed region
        # of the same steps with an event pair around every launch
        prof, ms_ev = profiled_steps(torch, hs, solver, stream, step, nsteps)
        lat["ms_per_step_with_launch_events"] = ms_ev
        del graph
        clocks = sampler.stop() if sampler else None
        return solver, step, max_over_ranks(ms, world), prof, worst, sh, clocks, lat

    # ---------------- end to end through the API with host buffers ---------
    pin = lambda a: torch.as_tensor(np.asfortranarray(a), dtype=torch.float64).pin_memory()
    hH, hwr, hwi, hB, hQ = pin(inst.H), pin(inst.wr), pin(inst.wi), pin(inst.B), pin(inst.Q0)
    hZ = torch.empty((ncol, n), dtype=torch.float64).pin_memory().t()
    hS = torch.empty(m, dtype=torch.int32).pin_memory()
    h2d = 8 * (2 * n * n + n * ncol + 2 * m)
    d2h = 8 * n * ncol + 4 * m
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    # the C ABI's end-to-end call (hsein_solve_host): inputs up, solve (Q0's
    # upload overlapped with it on the plan's side stream), backtransform, Z
    # and the status codes down
    def time_e2e(slv):
        slv.solve_host(hH, hwr, hwi, hB, hQ, hZ, hS)
        torch.cuda.synchronize()
        barrier(world)
        e0.record(stream)
        for _ in range(args.steps):
            slv.solve_host(hH, hwr, hwi, hB, hQ, hZ, hS)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        return max_over_ranks(e0.elapsed_time(e1), world)

    def converged_columns(sh_):
        # eigenvectors that pass Varah's test (the others are zeroed columns)
        return int(sum(offs[l + 1] - offs[l] for l in range(m) if sh_[l] == 0))

    # ---------------- the plain FP64 path (the metric's comparison) --------
    log("plain FP64 path")
    solver, step, ms, prof, worst, sh, clocks, lat = measure(0, True)
    X_plain = X.cpu().numpy()
    conv_cols = converged_columns(sh)
    all_cols = sum_over_ranks(conv_cols, world)
    value = all_cols * args.steps / (ms * 1e-3)
    e2e_value = all_cols * args.steps / (time_e2e(solver) * 1e-3)
    del solver

    # ---------------- the split-precision path: the headline ---------------
    log("split-precision path")
    solver_sp, step_sp, ms_sp, prof_sp, worst_sp, sh_sp, clocks_sp, lat_sp = measure(1, True)
    X_sp = X.cpu().numpy()
    conv_sp = converged_columns(sh_sp)
    all_sp = sum_over_ranks(conv_sp, world)
    value_sp = all_sp * args.steps / (ms_sp * 1e-3)
    e2e_value_sp = all_sp * args.steps / (time_e2e(solver_sp) * 1e-3)

    log("restart")
    # restart (Alg. "hsrq3in") of the shifts that did not converge, timed once
    # after a fresh solve: the cost of making every column converge
    step_sp()
    torch.cuda.synchronize()
    r0 = time.perf_counter()
    rc_r, n_retried = solver_sp.restart(dH, dwr, dwi, X, status, B=dB, max_tries=3)
    torch.cuda.synchronize()
    ms_restart = (time.perf_counter() - r0) * 1e3
    sh_r = status.cpu().numpy()
    conv_r = converged_columns(sh_r)
    restart = {"retried_shifts": n_retried, "not_converged_after": int((sh_r != 0).sum()),
               "ms": ms_restart, "clock": "host wall time (the restart synchronizes)",
               "value_with_restart": sum_over_ranks(conv_r, world)
               / ((ms_sp / args.steps + ms_restart) * 1e-3),
               "unit": UNIT}
    del solver_sp

    log("compact storage")
    # the headline path with the rotations stored compactly (Sec. 4.4)
    solver_c, _, ms_c, prof_c, worst_c, sh_c, _, lat_c = measure(1, False, givens=1, steps=5)
    compact = {"value": sum_over_ranks(converged_columns(sh_c), world) * 5 / (ms_c * 1e-3),
               "unit": UNIT, "ms_per_step": ms_c / 5, "residual_max_over_n_eps": worst_c,
               "not_converged": int((sh_c != 0).sum()),
               "workspace_bytes_saved": None,
               "phases": {k: {"ms_per_step": v[0] / 5} for k, v in prof_c.items()}}
    compact["workspace_bytes_saved"] = (
        hs.Solver(n, inst.m_real, inst.m_cplx, br=args.br, precision=1, device=dev).work_bytes
        - solver_c.work_bytes)
    del solver_c

    # the comparison baseline: Henry's solve per shift, unblocked (the RQIN of
    # the paper's experiments), FP64, same workload, same backtransform
    bsteps = 3
    log("per-shift baseline")
    _, _, ms_b, prof_b, worst_b, sh_b, _, lat_b = measure(0, False, method=1, steps=bsteps)
    conv_b = converged_columns(sh_b)
    baseline = {"method": "Henry's RQ solve per shift, unblocked (one thread block per shift "
                          "over the whole matrix), FP64; same prepare, normalization and "
                          "z = Q0 x",
                "value": sum_over_ranks(conv_b, world) * bsteps / (ms_b * 1e-3), "unit": UNIT,
                "ms_per_step": ms_b / bsteps, "residual_max_over_n_eps": worst_b,
                "not_converged": int((sh_b != 0).sum()),
                "phases": {k: {"ms_per_step": v[0] / bsteps} for k, v in prof_b.items()}}

    # the other comparison baseline: the LU approach per shift (Sec. 2.1,
    # LAPACK's inverse iteration), FP64, same workload and backtransform
    log("per-shift LU baseline")
    _, _, ms_l, prof_l, worst_l, sh_l, _, lat_l = measure(0, False, method=2, steps=bsteps)
    lu_baseline = {"method": "LU with partial pivoting per shift (P (H - lambda I) = L U, "
                             "L y = P b, U x = alpha y; one thread block per shift, U kept "
                             "packed in HBM), FP64; same prepare, normalization and z = Q0 x",
                   "value": sum_over_ranks(converged_columns(sh_l), world) * bsteps / (ms_l * 1e-3),
                   "unit": UNIT, "ms_per_step": ms_l / bsteps, "residual_max_over_n_eps": worst_l,
                   "not_converged": int((sh_l != 0).sum()),
                   "phases": {k: {"ms_per_step": v[0] / bsteps} for k, v in prof_l.items()}}

    if rank != 0:
        return
    pk, pk_kind = peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = (clocks_sp or {}).get("sm_mhz") or 2070.0
    fp64_peak = fp64_peak_tflops(sm_mhz, sms)
    log("FP64 probe")
    probe_sampler = ClockSampler(torch.cuda.current_device())
    probe_sampler.start()
    probe, probe_all = hs.fp64_rate(iters=50000, repeats=5)
    probe_clocks = probe_sampler.stop()
    fp64_peak_info = {
        "peak_tflops": fp64_peak,
        "how": "4 flops (2 FP64 FMA) per SM per clock x %d SMs x %.0f MHz (median SM clock "
               "sampled during the timed region)" % (sms, sm_mhz),
        "probe_tflops": probe, "probe_clocks": probe_clocks,
        "probe_how": "hsein_fp64_rate: eight independent DFMA chains per thread, %d threads, "
                     "median of 5 launches (CUDA events)" % (sms * 1024),
        "bf16_derived_tflops": pk["bf16_tflops"] * NOMINAL_FP64_OVER_BF16,
        "bf16_derived_how": "%s bf16 %.1f TFLOP/s x nominal FP64/BF16 ratio 1.25/2250"
                            % (pk_kind, pk["bf16_tflops"])}
    peak_source = "FP64 CUDA cores: unit counts x sampled clock (%.3f TFLOP/s); probe %.3f" % (
        fp64_peak, probe)
    uf, ulaunch = update_flops(n, ncol, args.br)
    q0f = 2.0 * n * n * ncol
    per_phase = lambda pr: {k: {"ms_per_step": v[0] / args.steps,
                                "launches_per_step": v[1] / args.steps} for k, v in pr.items()}
    # plain FP64 path: its dominant kernel is the shared-H product k_update
    # (or z = Q0 x when that takes longer)
    if max(prof, key=lambda k: prof[k][0]) == "q0_backtransform":
        flops_launch = q0f
        t_launch = prof["q0_backtransform"][0] / max(1, prof["q0_backtransform"][1])
        kfile, summary, kname = "paper_2101_05063_gb300/csrc/k_q0.cu", "k_q0_config1.txt", "k_q0"
    else:
        flops_launch = uf / ulaunch
        t_launch = prof["shared_h_update"][0] / max(1, prof["shared_h_update"][1])
        kfile, summary, kname = ("paper_2101_05063_gb300/csrc/k_update.cu",
                                 "k_update_config1.txt", "k_update")
    achieved = flops_launch / (t_launch * 1e-3) / 1e12
    # prepare is five kernels (setup, row sums, tile norms, init, tile
    # staging), six in split mode (+ the digit split of H); z = Q0 x is four
    # in split mode (row maxima, two splits, the product); the other phases
    # are one kernel per recorded launch
    launches = 5 * prof["prepare"][1] + sum(v[1] for k, v in prof.items() if k != "prepare")
    launches_sp = (6 * prof_sp["prepare"][1] + 4 * prof_sp["q0_backtransform"][1]
                   + sum(v[1] for k, v in prof_sp.items()
                         if k not in ("prepare", "q0_backtransform")))
    plain = {
        "value": value, "unit": UNIT, "ms_per_step": ms / args.steps, "latency": lat,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "residual_max_over_n_eps": worst, "not_converged": int((sh != 0).sum()),
        "phases": per_phase(prof), "gpu_launches": launches, "clocks": clocks, "dtype": "f64",
        "roofline": {"kernel": kname, "bound": "alu", "achieved": achieved,
                     "peak": fp64_peak, "unit": "TFLOP/s", "frac": achieved / fp64_peak,
                     "traffic": profiled_traffic(kfile, summary), "peak_source": peak_source,
                     "algorithmic_flops_per_launch": flops_launch,
                     "frac_of_probe": achieved / probe},
    }

    # split path: the digit products run on the BF16 tensor cores; 28 digit
    # pairs per product (7 digits, pairs above the FP64 rounding level)
    t_upd_sp = prof_sp["shared_h_update"][0] / args.steps
    t_q0_sp = prof_sp["q0_backtransform"][0] / args.steps
    tensor_upd = 28.0 * uf / (t_upd_sp * 1e-3) / 1e12
    tensor_q0 = 28.0 * q0f / (t_q0_sp * 1e-3) / 1e12
    tensor = {"peak": pk["bf16_tflops"], "unit": "TFLOP/s",
              "shared_h_update_achieved": tensor_upd,
              "shared_h_update_frac": tensor_upd / pk["bf16_tflops"],
              "q0_backtransform_achieved": tensor_q0,
              "q0_backtransform_frac": tensor_q0 / pk["bf16_tflops"],
              "engine": "tcgen05.mma kind::f16 (bf16 x bf16 -> fp32 in TMEM), TMA-staged tiles"}
    # the split path's dominant kernel: the diagonal-tile sweep k_diag (FP64)
    df, dlaunch = diag_flops(inst, args.br)
    t_diag = prof_sp["diag_sweep"][0] / max(1, prof_sp["diag_sweep"][1])
    achieved_d = df / dlaunch / (t_diag * 1e-3) / 1e12
    bf_d = pk["bf16_tflops"] * NOMINAL_FP64_OVER_BF16
    line = {
        "metric": METRIC, "value": value_sp, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms_sp / args.steps, "latency": lat_sp,
        "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 (bf16 digit-sliced products)", "data": "synthetic",
        "config": workload_config(inst, args.br),
        "vs_plain_fp64_gpu": value_sp / value if value > 0 else None,
        "roofline": {"kernel": "k_diag", "bound": "alu", "achieved": achieved_d,
                     "peak": fp64_peak, "unit": "TFLOP/s", "frac": achieved_d / fp64_peak,
                     "traffic": profiled_traffic("paper_2101_05063_gb300/csrc/k_diag.cu",
                                                 "k_diag_config1.txt"),
                     "peak_source": peak_source,
                     "algorithmic_flops_per_launch": df / dlaunch,
                     "flop_count": "5 n b_r per column per solve (per launch: 5 b_r^2 ncol)",
                     "frac_of_probe": achieved_d / probe,
                     "frac_of_bf16_derived": achieved_d / bf_d,
                     "timed": "average CUDA-event duration of the kernel's launches "
                              "(an event pair around each, on the launching stream) "
                              "over a second timed region of the same %d steps"
                              % args.steps},
        "fp64_peak": fp64_peak_info,
        "tensor": tensor,
        "phases": per_phase(prof_sp),
        "residual_max_over_n_eps": worst_sp,
        "not_converged": int((sh_sp != 0).sum()),
        "clocks": clocks_sp,
        "gpu_launches": launches_sp,
        "e2e": {"value": e2e_value_sp, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "vs_plain_fp64_gpu_e2e": e2e_value_sp / e2e_value if e2e_value > 0 else None},
        "columns_counted": "converged columns only (%d of %d); complex shifts count 2"
                           % (conv_sp, ncol),
        "restart": restart,
        "plain_fp64": plain,
        "per_shift_baseline": baseline,
        "per_shift_lu_baseline": lu_baseline,
        "compact_givens": compact,
    }
    if not args.no_reduction and world == 1:
        log("reduction")
        line["reduction"] = measure_reduction(inst, torch, hs, fp64_peak)
    if world == 1:
        log("n = 512 workload")
        c0 = hi.config0()
        sp0, _ = measure_instance(torch, hs, c0, 1, args.steps, args.warmup)
        fp0, _ = measure_instance(torch, hs, c0, 0, args.steps, args.warmup)
        line["config0"] = {"workload": "n = 512, 64 real shifts (the prescribed eigenvalues), "
                                       "tile height 64", "split": sp0, "fp64": fp0}
    if "c2" in futs:
        log("waiting for the n = 8192 workload")
        c2, t_c2 = futs["c2"].result()
        log("n = 8192 workload")
        line["precision_c2"] = measure_config2(args, torch, hs, c2, t_c2, fp64_peak,
                                               pk["bf16_tflops"])
        del c2
    if not args.no_batch and world == 1:
        log("batching")
        line["batching"] = measure_batch(args, torch, hs, hi, fp64_peak)
    if "serve" in futs:
        log("waiting for the serving pool")
        pool, t_pool = futs["serve"].result()
        log("serving")
        line["serving"] = measure_serving(args, torch, hs, hi, pool, t_pool)
        del pool
    if bg is not None:
        bg.shutdown()
    if not args.no_cpu_baseline and world == 1:
        log("cpu baseline")
        v, cores, desc, (idx, Xo, so) = cpu_baseline(inst, args.cpu_sample)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": desc}
        import oracle
        hn = oracle.hnorm_inf(inst.H)
        line["accuracy"] = accuracy_vs_oracle(inst, idx, X_sp, sh_sp, Xo, so, hn)
        line["plain_fp64"]["accuracy"] = accuracy_vs_oracle(inst, idx, X_plain, sh, Xo, so, hn)
    log("done")
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
