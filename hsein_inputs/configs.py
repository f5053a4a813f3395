"""The workload configurations as seeded synthetic instances.

config0: n = 512, upper triangular T with 64 prescribed eigenvalues evenly
         spaced in [-64, 64] and 448 more evenly spaced in [-512, 512] with
         U(-0.1, 0.1) jitter, strictly upper entries N(0,1); A = Q T Q^T with a
         Haar Q, reduced to Hessenberg H.  64 real shifts equal to the
         prescribed eigenvalues; unit-norm N(0,1) starting vectors.
config1: n = 4096, quasi-triangular T with 1024 real eigenvalues U[-n, n] and
         1536 blocks [[a, b], [-b, a]], a ~ U[-n, n], b ~ U[0.5, 2].
         512 real + 256 complex shifts (one member of each conjugate pair),
         drawn from the prescribed eigenvalues, in a seeded mixed order.
config2: n = 8192, real eigenvalues U[-n, n] with minimum gap >= 1e-2, 2048
         real shifts.
config3: 256 independent instances, n = round(exp(U[ln 64, ln 2048])) each,
         from their own seeds.  A quarter (by a seeded draw) carry complex
         pairs with the config1 recipe (a quarter of the eigenvalues real);
         the others follow config0 at size n (n real eigenvalues evenly
         spaced in [-n, n] with U(-0.1, 0.1) jitter).  Every instance's
         shifts are all of its real eigenvalues.
small_instance: the config1 recipe at any size, for parity tests.

Layout conventions (those of the C ABI): H, Q0 and B are column-major; a real
shift owns one column of B and X, a complex shift two adjacent columns
[re, im]; shifts are given as (wr, wi) with wi != 0 marking a complex shift.
"""
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

from .matrices import (S_B, S_EIG, S_IMAG, S_JIT, S_SHIFT, haar_orthogonal, hessenberg_reduce,
                       quasi_triangular)
from .rng import uniform


@dataclass
class Instance:
    name: str
    n: int
    H: np.ndarray
    Q0: np.ndarray
    wr: np.ndarray
    wi: np.ndarray
    B: np.ndarray
    A: Optional[np.ndarray] = None
    eigs: np.ndarray = field(default_factory=lambda: np.zeros(0, dtype=np.complex128))

    @property
    def m(self):
        return len(self.wr)

    @property
    def m_cplx(self):
        return int(np.count_nonzero(self.wi))

    @property
    def m_real(self):
        return self.m - self.m_cplx

    @property
    def ncol(self):
        return self.m_real + 2 * self.m_cplx


def column_offsets(wi):
    """Column of each shift in B/X: real shifts own one column, complex two."""
    widths = np.where(np.asarray(wi) != 0.0, 2, 1)
    return np.concatenate([[0], np.cumsum(widths)]).astype(np.int64)


def _starting_vectors(n, wi, seed):
    """Unit-2-norm N(0,1) starting vectors; a complex shift's [re, im] pair is
    normalized as one complex vector."""
    offs = column_offsets(wi)
    ncol = int(offs[-1])
    from .rng import normal
    B = normal(seed, S_B, n * ncol).reshape(n, ncol, order="F")
    for l in range(len(wi)):
        c0, c1 = offs[l], offs[l + 1]
        B[:, c0:c1] /= np.linalg.norm(B[:, c0:c1])
    return np.asfortranarray(B)


def _build(name, n, T, seed, wr, wi, keep_a):
    Q = haar_orthogonal(n, seed)
    A = np.asfortranarray(Q @ T @ Q.T)
    H, Q0 = hessenberg_reduce(A)
    B = _starting_vectors(n, wi, seed)
    return Instance(name=name, n=n, H=H, Q0=Q0, wr=np.asarray(wr, dtype=np.float64),
                    wi=np.asarray(wi, dtype=np.float64), B=B, A=A if keep_a else None)


def config0(seed=0, keep_a=False):
    n = 512
    pres = np.linspace(-64.0, 64.0, 64)
    rest = np.linspace(-512.0, 512.0, 448) + uniform(seed, S_JIT, 448, -0.1, 0.1)
    eigs = np.concatenate([pres, rest])
    T, _ = quasi_triangular(n, eigs, [], seed)
    inst = _build("config0", n, T, seed, pres, np.zeros(64), keep_a)
    inst.eigs = eigs.astype(np.complex128)
    return inst


def _mixed_instance(name, n, n_real_eigs, m_real, m_cplx, seed, keep_a, real_lo=None):
    n_pairs = (n - n_real_eigs) // 2
    assert n_real_eigs + 2 * n_pairs == n
    lo = -float(n) if real_lo is None else real_lo
    reals = uniform(seed, S_EIG, n_real_eigs, lo, float(n))
    a = uniform(seed, S_EIG, n_pairs, -float(n), float(n), start=n_real_eigs)
    b = uniform(seed, S_IMAG, n_pairs, 0.5, 2.0)
    T, _ = quasi_triangular(n, reals, list(zip(a, b)), seed)
    # shifts: m_real real eigenvalues and m_cplx pairs, in a seeded mixed order
    pick_r = np.argsort(uniform(seed, S_SHIFT, n_real_eigs), kind="stable")[:m_real]
    pick_c = np.argsort(uniform(seed, S_SHIFT, max(n_pairs, 1), start=n_real_eigs),
                        kind="stable")[:m_cplx]
    wr = np.concatenate([reals[pick_r], a[pick_c]])
    wi = np.concatenate([np.zeros(m_real), b[pick_c]])
    order = np.argsort(uniform(seed, S_SHIFT, m_real + m_cplx, start=3 * n), kind="stable")
    wr, wi = wr[order], wi[order]
    inst = _build(name, n, T, seed, wr, wi, keep_a)
    inst.eigs = np.concatenate([reals, a + 1j * b, a - 1j * b])
    return inst


def config1(seed=1, keep_a=False):
    return _mixed_instance("config1", 4096, 1024, 512, 256, seed, keep_a)


def _gapped_uniform(n, lo, hi, gap, seed):
    """n values uniform in [lo, hi) whose sorted neighbours differ by >= gap:
    offending values are redrawn from fresh counter indices until none is left."""
    vals = uniform(seed, S_EIG, n, lo, hi)
    nxt = n
    while True:
        order = np.argsort(vals, kind="stable")
        s = vals[order]
        bad = np.nonzero(np.diff(s) < gap)[0]
        if len(bad) == 0:
            return vals
        idx = order[bad + 1]
        vals[idx] = uniform(seed, S_EIG, len(idx), lo, hi, start=nxt)
        nxt += len(idx)


def config2(seed=2, keep_a=False):
    n = 8192
    eigs = _gapped_uniform(n, -float(n), float(n), 1e-2, seed)
    T, _ = quasi_triangular(n, eigs, [], seed)
    pick = np.argsort(uniform(seed, S_SHIFT, n), kind="stable")[:2048]
    inst = _build("config2", n, T, seed, eigs[pick], np.zeros(2048), keep_a)
    inst.eigs = eigs.astype(np.complex128)
    return inst


def small_instance(n, m_real, m_cplx, seed, keep_a=False):
    """The config1 recipe at size n: about n/4 real eigenvalues, the rest in
    complex pairs; m_real real and m_cplx complex shifts in mixed order."""
    n_real = max(m_real, n // 4)
    if (n - n_real) % 2:
        n_real += 1
    n_pairs = (n - n_real) // 2
    assert m_cplx <= n_pairs and m_real <= n_real
    return _mixed_instance("small_n%d" % n, n, n_real, m_real, m_cplx, seed, keep_a)


S_SIZE, S_KIND = 20, 21


def config3_sizes(seed=3, count=256, lo=64, hi=2048):
    """(n, has_complex) of every instance of the batching workload."""
    u = uniform(seed, S_SIZE, count)
    ns = np.rint(np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))).astype(int)
    kinds = uniform(seed, S_KIND, count) < 0.25
    return [(int(n), bool(k)) for n, k in zip(ns, kinds)]


def batch_instance(n, has_complex, seed):
    """One instance of the batching workload (see config3)."""
    if has_complex:
        n_real = max(2, n // 4)
        if (n - n_real) % 2:
            n_real += 1
        return _mixed_instance("batch_n%d" % n, n, n_real, n_real, 0, seed, False)
    eigs = np.linspace(-float(n), float(n), n) + uniform(seed, S_JIT, n, -0.1, 0.1)
    T, _ = quasi_triangular(n, eigs, [], seed)
    inst = _build("batch_n%d" % n, n, T, seed, eigs, np.zeros(n), False)
    inst.eigs = eigs.astype(np.complex128)
    return inst


def _batch_instance_star(args):
    return batch_instance(*args)


def config3(seed=3, count=256, lo=64, hi=2048, workers=0):
    """The batching workload: a list of instances (seed of instance i is
    1000 * seed + i + 1).  workers > 1 generates them in a pool of spawned
    processes with single-threaded BLAS; the BLAS thread count changes the
    summation order, so those instances equal the serial ones only up to
    rounding (each is still a valid instance of the recipe)."""
    args = [(n, k, 1000 * seed + i + 1)
            for i, (n, k) in enumerate(config3_sizes(seed, count, lo, hi))]
    if workers and workers > 1:
        import concurrent.futures as cf
        import multiprocessing as mp
        import os
        keys = ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")
        saved = {k: os.environ.get(k) for k in keys}
        for k in keys:
            os.environ[k] = "1"
        try:
            with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
                # largest first, so that the pool drains evenly
                order = sorted(range(len(args)), key=lambda i: -args[i][0])
                done = dict(zip(order, ex.map(_batch_instance_star, [args[i] for i in order])))
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        return [done[i] for i in range(len(args))]
    return [batch_instance(*a) for a in args]


# --------------------------------------------------------------- serving
S_ARRIVE, S_CLASS, S_PICK, S_K, S_KIND4, S_GRADE4, S_SHIFTS4 = 30, 31, 32, 33, 34, 35, 36
SERVE_SIZES = (256, 512, 1024, 2048, 4096, 8192)


def serving_pool(sizes=SERVE_SIZES, per_size=None, seed=4):
    """{n: [instances]}: the matrix pool of the serving workload.  Each is the
    config1 recipe at size n (a quarter of the eigenvalues real, the rest in
    complex pairs); per_size[n] instances per class (default 8 up to n = 2048,
    2 at 4096, 1 at 8192).  Each instance also carries its graded form
    D H D^-1, D = diag(10^u), u ~ U[-150, 150] per index (attribute Hg)."""
    from .matrices import S_GRADE
    pool = {}
    for n in sizes:
        k = (per_size or {}).get(n, 8 if n <= 2048 else (2 if n <= 4096 else 1))
        lst = []
        for j in range(k):
            s = 100000 * seed + 100 * n + j
            n_real = n // 4 + ((n - n // 4) % 2)
            inst = _mixed_instance("serve_n%d_%d" % (n, j), n, n_real, 0, 0, s, False)
            u = uniform(s, S_GRADE, n, -150.0, 150.0)
            d = 10.0 ** u
            inst.Hg = np.asfortranarray(inst.H * d[:, None] / d[None, :])
            inst.n_real = n_real
            lst.append(inst)
        pool[n] = lst
    return pool


def serving_requests(pool, count, seed=4, rate=200.0):
    """The request stream: Poisson arrivals (rate per second), n uniform over
    the pool's size classes, a pool instance uniform in its class, k shifts
    uniform in [1, n/4]; 30% graded (the instance's D H D^-1), 30% with
    complex pairs (ceil(k/2) complex shifts, one member per pair, and
    floor(k/2) real ones), the rest k real shifts; shifts drawn without
    replacement from the instance's eigenvalues.  Starting vectors: rho e.
    Returns a list of dicts (t, n, index, graded, wr, wi)."""
    sizes = sorted(pool)
    ua = uniform(seed, S_ARRIVE, count)
    t = np.cumsum(-np.log(1.0 - ua) / rate)
    cls = (uniform(seed, S_CLASS, count) * len(sizes)).astype(int)
    pick = uniform(seed, S_PICK, count)
    uk = uniform(seed, S_K, count)
    kind = uniform(seed, S_KIND4, count)
    grade = uniform(seed, S_GRADE4, count)
    reqs = []
    for i in range(count):
        n = sizes[cls[i]]
        idx = int(pick[i] * len(pool[n]))
        inst = pool[n][idx]
        k = 1 + int(uk[i] * (n // 4))
        cplx = kind[i] < 0.3
        kc, kr = ((k + 1) // 2, k // 2) if cplx else (0, k)
        reals = inst.eigs[:inst.n_real].real
        pairs = inst.eigs[inst.n_real:inst.n_real + (n - inst.n_real) // 2]
        pr = np.argsort(uniform(seed * 7919 + i, S_SHIFTS4, len(reals)), kind="stable")[:kr]
        pc = np.argsort(uniform(seed * 7919 + i, S_SHIFTS4, len(pairs), start=n), kind="stable")[:kc]
        wr = np.concatenate([reals[pr], pairs[pc].real])
        wi = np.concatenate([np.zeros(kr), pairs[pc].imag])
        reqs.append({"t": float(t[i]), "n": n, "index": idx, "graded": bool(grade[i] < 0.3),
                     "wr": wr, "wi": wi})
    return reqs
