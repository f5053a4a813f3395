"""GB300-native multi-shift inverse iteration from the Hessenberg matrix.

Python binding of libhsein (C ABI in include/hsein.h).  The functions named
like the C entry points (hsein_plan, hsein_solve, hsein_backtransform, ...)
only marshal arguments; every step of the computation runs in the CUDA
kernels of the library.  PyTorch provides device memory and streams.  There
is no CPU fallback: if the library cannot be loaded, every call raises.

    import torch, paper_2101_05063_gb300 as hs
    H, Q0 = hs.gehrd(A)                               # A = Q0 H Q0^T on the GPU
    solver = hs.Solver(n, m_real, m_cplx)             # plan + workspace
    X, status = solver.solve(H, wr, wi, B)            # unit eigenvectors of H
    Z = solver.backtransform(Q0, X)                   # eigenvectors of A
    solver.solve_host(hH, hwr, hwi, hB, hQ0, hZ, hst) # the same from pinned host buffers
    step = solver.graph(H, wr, wi, B, Q0)             # solve + Z = Q0 X as one CUDA graph
    step.launch()                                     # results in step.X, step.status, step.Z

Options of Solver: precision=1 (split-precision products on the BF16 tensor
cores, the fast mode), givens=1 (compact rotation storage), method=1 / 2 (the
per-shift baselines: Henry's RQ solve / the LU approach), br (tile height),
robust, omega_log2, wait_limit_cycles.  Batch runs many
independent instances in one captured graph; Server admits requests by HBM
footprint and fuses those on the same matrix; balance/unbalance prepare
graded matrices for the split-precision mode.

Column layout (as in the C ABI): a real shift owns one column, a complex
shift two adjacent columns [re, im], in the input order of the shifts.
"""
import ctypes
import os

from . import build as _build

__all__ = [
    "HseinError", "HseinOptions", "load", "hsein_default_options", "hsein_plan", "hsein_solve",
    "hsein_solve_noalloc", "hsein_backtransform", "hsein_plan_sync_status", "hsein_margins",
    "hsein_restart", "hsein_batch_plan", "hsein_batch_solve", "hsein_batch_autotune",
    "hsein_batch_info", "hsein_batch_destroy", "HseinInstance", "HseinBatchConfig", "Batch",
    "HseinRequest", "hsein_server_create", "hsein_server_submit", "hsein_server_progress",
    "hsein_server_stats", "hsein_server_destroy", "hsein_server_set_bypass", "Server", "hsein_balance", "hsein_unbalance",
    "balance", "unbalance", "hsein_gehrd_workspace", "hsein_gehrd", "gehrd",
    "hsein_plan_info", "hsein_plan_destroy",
    "hsein_status_string", "hsein_plan_set_profiling", "hsein_plan_profile", "Solver",
    "STATUS", "PHASES", "hsein_fp64_rate", "fp64_rate", "hsein_host_workspace",
    "hsein_solve_host", "StepGraph", "hsein_graph_create", "hsein_graph_launch",
    "hsein_graph_destroy",
]

STATUS = {0: "HSEIN_OK", -1: "HSEIN_EARG", -2: "HSEIN_ENOMEM", -3: "HSEIN_ENOTUNREDUCED",
          -4: "HSEIN_ENONFINITE", -5: "HSEIN_ECUDA", -6: "HSEIN_ETIMEOUT", -7: "HSEIN_ESHIFTS",
          1: "HSEIN_WNOTCONVERGED"}


class HseinError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = int(code)
        msg = "%s (%d)" % (STATUS.get(self.code, "unknown"), self.code)
        if what:
            msg = what + ": " + msg
        super().__init__(msg)


class HseinOptions(ctypes.Structure):
    _fields_ = [("br", ctypes.c_int), ("precision", ctypes.c_int), ("robust", ctypes.c_int),
                ("omega_log2", ctypes.c_int), ("method", ctypes.c_int),
                ("givens", ctypes.c_int), ("wait_limit_cycles", ctypes.c_longlong)]


class HseinInstance(ctypes.Structure):
    """One instance of a batch: the arguments of hsein_solve."""
    _fields_ = [("n", ctypes.c_int), ("m_real", ctypes.c_int), ("m_cplx", ctypes.c_int),
                ("dH", ctypes.c_void_p), ("ldh", ctypes.c_int), ("dWr", ctypes.c_void_p),
                ("dWi", ctypes.c_void_p), ("dB", ctypes.c_void_p), ("ldb", ctypes.c_int),
                ("dX", ctypes.c_void_p), ("ldx", ctypes.c_int), ("dStatus", ctypes.c_void_p)]


class HseinRequest(ctypes.Structure):
    _fields_ = [("inst", HseinInstance), ("precision", ctypes.c_int), ("br", ctypes.c_int),
                ("dExp", ctypes.c_void_p)]


class HseinBatchConfig(ctypes.Structure):
    _fields_ = [("streams", ctypes.c_int), ("br_policy", ctypes.c_int),
                ("shift_block", ctypes.c_int), ("reserved", ctypes.c_int)]

    def as_dict(self):
        return {"streams": self.streams, "br_policy": self.br_policy,
                "shift_block": self.shift_block}


_lib = None


def load(build_if_missing=True):
    """Load libhsein.so (building it with nvcc first if it is missing or
    stale).  Raises if it cannot be built or loaded: there is no fallback."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise HseinError(-5, "libhsein.so is missing (%s); run build()" % path)
    lib = ctypes.CDLL(path)
    vp, sz, ip, dp = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p
    lib.hsein_default_options.restype = ctypes.c_int
    lib.hsein_default_options.argtypes = [ctypes.POINTER(HseinOptions)]
    lib.hsein_plan.restype = ctypes.c_int
    lib.hsein_plan.argtypes = [ctypes.POINTER(vp), ip, ip, ip, ctypes.POINTER(HseinOptions),
                               ctypes.POINTER(sz)]
    lib.hsein_solve.restype = ctypes.c_int
    lib.hsein_solve.argtypes = [vp, dp, ip, dp, dp, dp, ip, dp, ip, dp, vp, sz, vp]
    lib.hsein_solve_noalloc.restype = ctypes.c_int
    lib.hsein_solve_noalloc.argtypes = [vp, dp, ip, dp, dp, dp, ip, dp, ip, dp, vp]
    lib.hsein_backtransform.restype = ctypes.c_int
    lib.hsein_backtransform.argtypes = [vp, dp, ip, dp, ip, dp, ip, vp, sz, vp]
    lib.hsein_graph_create.restype = ctypes.c_int
    lib.hsein_graph_create.argtypes = [vp, dp, ip, dp, dp, dp, ip, dp, ip, dp, dp, ip, dp, ip,
                                       vp, sz, ctypes.POINTER(vp)]
    lib.hsein_graph_launch.restype = ctypes.c_int
    lib.hsein_graph_launch.argtypes = [vp, vp]
    lib.hsein_graph_destroy.restype = ctypes.c_int
    lib.hsein_graph_destroy.argtypes = [vp]
    lib.hsein_plan_sync_status.restype = ctypes.c_int
    lib.hsein_plan_sync_status.argtypes = [vp, vp, vp]
    lib.hsein_margins.restype = ctypes.c_int
    lib.hsein_margins.argtypes = [vp, vp, dp, vp]
    bp = ctypes.POINTER(HseinBatchConfig)
    lib.hsein_batch_plan.restype = ctypes.c_int
    lib.hsein_batch_plan.argtypes = [ctypes.POINTER(vp), ip, ctypes.POINTER(HseinInstance),
                                     ctypes.POINTER(HseinOptions), bp, ctypes.POINTER(sz)]
    lib.hsein_batch_solve.restype = ctypes.c_int
    lib.hsein_batch_solve.argtypes = [vp, vp, sz, vp]
    lib.hsein_batch_autotune.restype = ctypes.c_int
    lib.hsein_batch_autotune.argtypes = [vp, vp, sz, vp, bp, ctypes.POINTER(ctypes.c_double)]
    lib.hsein_batch_info.restype = ctypes.c_int
    lib.hsein_batch_info.argtypes = [vp, bp, ctypes.POINTER(ctypes.c_int)]
    lib.hsein_batch_destroy.restype = ctypes.c_int
    lib.hsein_batch_destroy.argtypes = [vp]
    ll = ctypes.c_longlong
    lib.hsein_balance.restype = ctypes.c_int
    lib.hsein_balance.argtypes = [ip, dp, ip, dp, ip, dp, ip, vp]
    lib.hsein_unbalance.restype = ctypes.c_int
    lib.hsein_unbalance.argtypes = [ip, ip, dp, dp, dp, ip, vp]
    lib.hsein_gehrd_workspace.restype = ctypes.c_int
    lib.hsein_gehrd_workspace.argtypes = [ip, ctypes.POINTER(sz)]
    lib.hsein_gehrd.restype = ctypes.c_int
    lib.hsein_gehrd.argtypes = [ip, dp, ip, dp, ip, dp, ip, vp, sz, vp]
    lib.hsein_host_workspace.restype = ctypes.c_int
    lib.hsein_host_workspace.argtypes = [vp, ctypes.POINTER(sz)]
    lib.hsein_solve_host.restype = ctypes.c_int
    lib.hsein_solve_host.argtypes = [vp, dp, ip, dp, dp, dp, ip, dp, ip, dp, ip, dp, vp, sz, vp]
    lib.hsein_server_set_bypass.restype = ctypes.c_int
    lib.hsein_server_set_bypass.argtypes = [vp, ctypes.c_int]
    lib.hsein_fp64_rate.restype = ctypes.c_int
    lib.hsein_fp64_rate.argtypes = [ctypes.c_longlong, dp, ctypes.c_longlong,
                                    ctypes.POINTER(ctypes.c_double), vp]
    lib.hsein_server_create.restype = ctypes.c_int
    lib.hsein_server_create.argtypes = [ctypes.POINTER(vp), sz, ip, ip, ctypes.POINTER(HseinOptions)]
    lib.hsein_server_submit.restype = ctypes.c_int
    lib.hsein_server_submit.argtypes = [vp, ctypes.POINTER(HseinRequest), ctypes.POINTER(ll)]
    lib.hsein_server_progress.restype = ctypes.c_int
    lib.hsein_server_progress.argtypes = [vp, ctypes.POINTER(ll), ip, ctypes.POINTER(ip), ip]
    lib.hsein_server_stats.restype = ctypes.c_int
    lib.hsein_server_stats.argtypes = [vp, ctypes.POINTER(ip), ctypes.POINTER(ip),
                                       ctypes.POINTER(sz), ctypes.POINTER(ll), ctypes.POINTER(ll)]
    lib.hsein_server_destroy.restype = ctypes.c_int
    lib.hsein_server_destroy.argtypes = [vp]
    lib.hsein_restart.restype = ctypes.c_int
    lib.hsein_restart.argtypes = [vp, dp, ip, dp, dp, dp, ip, dp, ip, dp, ip,
                                  ctypes.POINTER(ctypes.c_int), vp, sz, vp]
    lib.hsein_plan_info.restype = ctypes.c_int
    lib.hsein_plan_info.argtypes = [vp] + [ctypes.POINTER(ctypes.c_int)] * 5 + [ctypes.POINTER(sz)]
    lib.hsein_plan_destroy.restype = ctypes.c_int
    lib.hsein_plan_destroy.argtypes = [vp]
    lib.hsein_status_string.restype = ctypes.c_char_p
    lib.hsein_status_string.argtypes = [ctypes.c_int]
    lib.hsein_plan_set_profiling.restype = ctypes.c_int
    lib.hsein_plan_set_profiling.argtypes = [vp, ip]
    lib.hsein_plan_profile.restype = ctypes.c_int
    lib.hsein_plan_profile.argtypes = [vp, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_int), ip, ip]
    _lib = lib
    return lib


# ----------------------------------------------------------- C-ABI mirrors

def hsein_default_options():
    o = HseinOptions()
    _check(load().hsein_default_options(ctypes.byref(o)), "hsein_default_options")
    return o


def hsein_plan(n, m_real, m_cplx, opt=None):
    """Returns (plan handle, workspace bytes)."""
    p = ctypes.c_void_p()
    w = ctypes.c_size_t()
    rc = load().hsein_plan(ctypes.byref(p), int(n), int(m_real), int(m_cplx),
                           ctypes.byref(opt) if opt is not None else None, ctypes.byref(w))
    _check(rc, "hsein_plan")
    return p, w.value


def hsein_solve(plan, dH, ldh, dWr, dWi, dB, ldb, dX, ldx, dStatus, dWork, work_bytes, stream):
    """Device pointers are integers (e.g. tensor.data_ptr()); dB may be 0."""
    return load().hsein_solve(plan, dH, ldh, dWr, dWi, dB or None, ldb, dX, ldx, dStatus, dWork,
                              work_bytes, stream or None)


def hsein_graph_create(plan, dH, ldh, dWr, dWi, dB, ldb, dX, ldx, dStatus, dQ0, ldq, dZ, ldz,
                       dWork, work_bytes):
    """One step (hsein_solve, then hsein_backtransform when dQ0 is not 0)
    captured as a CUDA graph on these device buffers; returns (status,
    handle)."""
    g = ctypes.c_void_p()
    rc = load().hsein_graph_create(plan, dH, ldh, dWr, dWi, dB or None, ldb, dX, ldx, dStatus,
                                   dQ0 or None, ldq, dZ or None, ldz, dWork, work_bytes,
                                   ctypes.byref(g))
    return rc, g


def hsein_graph_launch(graph, stream):
    return load().hsein_graph_launch(graph, stream or None)


def hsein_graph_destroy(graph):
    return load().hsein_graph_destroy(graph)


def hsein_solve_noalloc(plan, dH, ldh, dWr, dWi, dB, ldb, dX, ldx, dStatus, stream):
    """hsein_solve on the library's fixed device array instead of a caller
    workspace: for callers that cannot allocate device memory."""
    return load().hsein_solve_noalloc(plan, dH, ldh, dWr, dWi, dB or None, ldb, dX, ldx, dStatus,
                                      stream or None)


def hsein_backtransform(plan, dQ0, ldq, dX, ldx, dZ, ldz, dWork, work_bytes, stream):
    return load().hsein_backtransform(plan, dQ0, ldq, dX, ldx, dZ, ldz, dWork, work_bytes,
                                      stream or None)


def hsein_plan_sync_status(plan, dWork, stream):
    return load().hsein_plan_sync_status(plan, dWork, stream or None)


def hsein_margins(plan, dWork, dMargin, stream):
    """Per-shift Varah margins (log2, > 0 converged) of the last solve on dWork."""
    return load().hsein_margins(plan, dWork, dMargin, stream or None)


def hsein_restart(plan, dH, ldh, dWr, dWi, dB, ldb, dX, ldx, dStatus, max_tries, dWork,
                  work_bytes, stream):
    """Retry the non-converged shifts with new orthogonal starting vectors;
    returns (status code, number of shifts retried)."""
    k = ctypes.c_int(0)
    rc = load().hsein_restart(plan, dH, ldh, dWr, dWi, dB or None, ldb, dX, ldx, dStatus,
                              int(max_tries), ctypes.byref(k), dWork, work_bytes, stream or None)
    return rc, k.value


def hsein_batch_plan(instances, opt=None, cfg=None):
    """instances: a sequence of HseinInstance.  Returns (batch, workspace bytes)."""
    arr = (HseinInstance * len(instances))(*instances)
    b = ctypes.c_void_p()
    w = ctypes.c_size_t()
    rc = load().hsein_batch_plan(ctypes.byref(b), len(instances), arr,
                                 ctypes.byref(opt) if opt is not None else None,
                                 ctypes.byref(cfg) if cfg is not None else None, ctypes.byref(w))
    _check(rc, "hsein_batch_plan")
    return b, w.value


def hsein_batch_solve(batch, dWork, work_bytes, stream):
    return load().hsein_batch_solve(batch, dWork, work_bytes, stream or None)


def hsein_batch_autotune(batch, dWork, work_bytes, stream):
    """Returns (status, chosen HseinBatchConfig, ms)."""
    c = HseinBatchConfig()
    t = ctypes.c_double()
    rc = load().hsein_batch_autotune(batch, dWork, work_bytes, stream or None, ctypes.byref(c),
                                     ctypes.byref(t))
    return rc, c, t.value


def hsein_batch_info(batch):
    c = HseinBatchConfig()
    k = ctypes.c_int()
    _check(load().hsein_batch_info(batch, ctypes.byref(c), ctypes.byref(k)), "hsein_batch_info")
    return c, k.value


def hsein_batch_destroy(batch):
    return load().hsein_batch_destroy(batch)


def hsein_balance(n, dH, ldh, dHb, ldhb, dExp, max_sweeps, stream):
    return load().hsein_balance(n, dH, ldh, dHb, ldhb, dExp, max_sweeps, stream or None)


def hsein_unbalance(n, m, dWi, dExp, dX, ldx, stream):
    return load().hsein_unbalance(n, m, dWi, dExp, dX, ldx, stream or None)


def balance(H, max_sweeps=30):
    """Power-of-two balancing of a CUDA float64 Hessenberg matrix: returns
    (Hb, exps) with Hb = D^-1 H D, D = diag(2^exps), column-major."""
    import torch
    H = _colmajor(H, torch)
    n = H.shape[0]
    Hb = torch.empty((n, n), dtype=torch.float64, device=H.device).t()
    e = torch.empty(n, dtype=torch.int32, device=H.device)
    _check(hsein_balance(n, H.data_ptr(), _ld(H), Hb.data_ptr(), _ld(Hb), e.data_ptr(),
                         int(max_sweeps), torch.cuda.current_stream(H.device).cuda_stream),
           "hsein_balance")
    return Hb, e


def unbalance(X, wi, exps):
    """Eigenvectors of the balanced matrix (in place in X, column-major) back
    to the original matrix, unit 2-norm per shift."""
    import torch
    wi = wi.to(torch.float64).contiguous()
    _check(hsein_unbalance(X.shape[0], wi.numel(), wi.data_ptr(), exps.data_ptr(), X.data_ptr(),
                           _ld(X), torch.cuda.current_stream(X.device).cuda_stream),
           "hsein_unbalance")
    return X


def hsein_gehrd_workspace(n):
    """Returns (status, workspace bytes)."""
    w = ctypes.c_size_t()
    rc = load().hsein_gehrd_workspace(n, ctypes.byref(w))
    return rc, w.value


def hsein_gehrd(n, dA, lda, dH, ldh, dQ, ldq, dWork, work_bytes, stream):
    return load().hsein_gehrd(n, dA, lda, dH, ldh, dQ, ldq, dWork, work_bytes, stream or None)


def gehrd(A):
    """Householder reduction of a CUDA float64 square matrix: returns (H, Q0)
    with A = Q0 H Q0^T, H upper Hessenberg (exact zeros below the first
    subdiagonal) and Q0 orthogonal, both column-major."""
    import torch
    A = _colmajor(A, torch)
    n = A.shape[0]
    H = torch.empty((n, n), dtype=torch.float64, device=A.device).t()
    Q = torch.empty((n, n), dtype=torch.float64, device=A.device).t()
    rc, wb = hsein_gehrd_workspace(n)
    _check(rc, "hsein_gehrd_workspace")
    work = torch.empty(wb, dtype=torch.uint8, device=A.device)
    _check(hsein_gehrd(n, A.data_ptr(), _ld(A), H.data_ptr(), _ld(H), Q.data_ptr(), _ld(Q),
                       work.data_ptr(), wb, torch.cuda.current_stream(A.device).cuda_stream),
           "hsein_gehrd")
    return H, Q


def hsein_server_create(hbm_bytes, max_jobs, max_merge_shifts, opt=None):
    srv = ctypes.c_void_p()
    rc = load().hsein_server_create(ctypes.byref(srv), int(hbm_bytes), int(max_jobs),
                                    int(max_merge_shifts),
                                    ctypes.byref(opt) if opt is not None else None)
    _check(rc, "hsein_server_create")
    return srv


def hsein_server_submit(server, req):
    """Returns (status, ticket)."""
    t = ctypes.c_longlong()
    rc = load().hsein_server_submit(server, ctypes.byref(req), ctypes.byref(t))
    return rc, t.value


def hsein_server_progress(server, max_done=256, wait=False):
    """Returns (status, list of completed tickets)."""
    buf = (ctypes.c_longlong * max_done)()
    k = ctypes.c_int()
    rc = load().hsein_server_progress(server, buf, max_done, ctypes.byref(k), int(bool(wait)))
    return rc, list(buf[:k.value])


def hsein_server_stats(server):
    p, r = ctypes.c_int(), ctypes.c_int()
    b = ctypes.c_size_t()
    ra, sa = ctypes.c_longlong(), ctypes.c_longlong()
    _check(load().hsein_server_stats(server, ctypes.byref(p), ctypes.byref(r), ctypes.byref(b),
                                     ctypes.byref(ra), ctypes.byref(sa)), "hsein_server_stats")
    return {"pending": p.value, "running": r.value, "bytes_in_use": b.value,
            "requests_admitted": ra.value, "solves_admitted": sa.value}


def hsein_server_set_bypass(server, max_bypass):
    return load().hsein_server_set_bypass(server, int(max_bypass))


def hsein_server_destroy(server):
    return load().hsein_server_destroy(server)


def hsein_host_workspace(plan):
    """Device bytes hsein_solve_host needs."""
    w = ctypes.c_size_t()
    _check(load().hsein_host_workspace(plan, ctypes.byref(w)), "hsein_host_workspace")
    return w.value


def hsein_solve_host(plan, hH, ldh, hWr, hWi, hB, ldb, hQ0, ldq, hZ, ldz, hStatus, dWork,
                     work_bytes, stream):
    return load().hsein_solve_host(plan, hH, ldh, hWr, hWi, hB, ldb, hQ0, ldq, hZ, ldz,
                                   hStatus, dWork, work_bytes, stream)


def hsein_fp64_rate(iters, dOut, count, stream):
    """Launch the FP64 rate probe; returns its flop count."""
    f = ctypes.c_double()
    _check(load().hsein_fp64_rate(int(iters), dOut, int(count), ctypes.byref(f), stream),
           "hsein_fp64_rate")
    return f.value


def fp64_rate(iters=200000, repeats=5, device=None):
    """FP64 FMA rate of the current GPU in TFLOP/s (median over repeats of
    one probe launch timed with CUDA events), and the per-repeat values."""
    import torch
    dev = torch.device(device or "cuda")
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    count = sms * 1024
    out = torch.empty(count, dtype=torch.float64, device=dev)
    st = torch.cuda.current_stream(dev)
    hsein_fp64_rate(1000, out.data_ptr(), count, st.cuda_stream)  # warm-up
    vals = []
    for _ in range(repeats):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        flops = hsein_fp64_rate(iters, out.data_ptr(), count, st.cuda_stream)
        e1.record(st)
        e1.synchronize()
        vals.append(flops / (e0.elapsed_time(e1) * 1e-3) / 1e12)
    vals.sort()
    return vals[len(vals) // 2], vals


def hsein_plan_info(plan):
    vals = [ctypes.c_int() for _ in range(5)]
    w = ctypes.c_size_t()
    _check(load().hsein_plan_info(plan, *[ctypes.byref(v) for v in vals], ctypes.byref(w)),
           "hsein_plan_info")
    n, mr, mc, ncol, br = (v.value for v in vals)
    return dict(n=n, m_real=mr, m_cplx=mc, ncol=ncol, br=br, workspace_bytes=w.value)


def hsein_plan_destroy(plan):
    return load().hsein_plan_destroy(plan)


def hsein_status_string(code):
    return load().hsein_status_string(int(code)).decode()


PHASES = ["prepare", "diag_sweep", "shared_h_update", "finalize", "q0_backtransform"]


def hsein_plan_set_profiling(plan, enable):
    return _check(load().hsein_plan_set_profiling(plan, int(bool(enable))),
                  "hsein_plan_set_profiling")


def hsein_plan_profile(plan, reset=True):
    """{phase: (milliseconds, launches)} since the last reset."""
    n = len(PHASES)
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_int * n)()
    _check(load().hsein_plan_profile(plan, ms, cnt, n, int(bool(reset))), "hsein_plan_profile")
    return {PHASES[i]: (ms[i], cnt[i]) for i in range(n)}


def _check(rc, what):
    if rc < 0:
        raise HseinError(rc, what)
    return rc


# ------------------------------------------------------ torch convenience

def _colmajor(t, torch):
    """A column-major (Fortran-order) float64 view or copy of a 2-D tensor."""
    if t.dim() == 1:
        t = t.reshape(-1, 1)
    if t.dtype != torch.float64:
        raise TypeError("expected float64, got %s" % t.dtype)
    if t.stride(0) == 1 and (t.shape[1] <= 1 or t.stride(1) >= max(1, t.shape[0])):
        return t
    return t.t().contiguous().t()


def _ld(t):
    """Leading dimension of a column-major tensor (for one column any value
    >= the row count is valid, whatever stride torch reports)."""
    return t.stride(1) if t.shape[1] > 1 else max(1, t.shape[0])


class Solver:
    """A plan plus its device workspace for fixed (n, m_real, m_cplx).

    solve() and backtransform() take CUDA float64 tensors (any layout; they are
    used in place when already column-major) and run on the current stream.
    """

    def __init__(self, n, m_real, m_cplx, br=64, robust=True, omega_log2=1000, precision=0,
                 device=None, method=0, givens=0, wait_limit_cycles=0):
        import torch
        self.torch = torch
        self.device = torch.device(device or "cuda")
        with torch.cuda.device(self.device):
            opt = hsein_default_options()
            opt.br = int(br)
            opt.robust = int(bool(robust))
            opt.omega_log2 = int(omega_log2)
            opt.precision = int(precision)
            opt.method = int(method)
            opt.givens = int(givens)
            opt.wait_limit_cycles = int(wait_limit_cycles)
            self.plan, self.work_bytes = hsein_plan(n, m_real, m_cplx, opt)
        self.n, self.m_real, self.m_cplx = int(n), int(m_real), int(m_cplx)
        self.m = self.m_real + self.m_cplx
        self.ncol = self.m_real + 2 * self.m_cplx
        self.work = torch.empty(self.work_bytes, dtype=torch.uint8, device=self.device)

    def __del__(self):
        plan = getattr(self, "plan", None)
        if plan is not None and _lib is not None:
            _lib.hsein_plan_destroy(plan)
            self.plan = None

    def _stream(self):
        return self.torch.cuda.current_stream(self.device).cuda_stream

    def solve(self, H, wr, wi, B=None, X=None, status=None, check=True):
        """Returns (X, status): unit-norm eigenvector approximations of H
        (n x ncol, column-major) and per-shift codes (0 ok, 1 not converged)."""
        torch = self.torch
        H = _colmajor(H, torch)
        wr = wr.to(torch.float64).contiguous()
        wi = wi.to(torch.float64).contiguous()
        if B is not None:
            B = _colmajor(B, torch)
        if X is None:
            X = torch.empty((self.ncol, self.n), dtype=torch.float64, device=self.device).t()
        if status is None:
            status = torch.empty(self.m, dtype=torch.int32, device=self.device)
        rc = hsein_solve(self.plan, H.data_ptr(), _ld(H), wr.data_ptr(), wi.data_ptr(),
                         B.data_ptr() if B is not None else 0, _ld(B) if B is not None else self.n,
                         X.data_ptr(), _ld(X), status.data_ptr(), self.work.data_ptr(),
                         self.work_bytes, self._stream())
        _check(rc, "hsein_solve")
        if check:
            rc = hsein_plan_sync_status(self.plan, self.work.data_ptr(), self._stream())
            _check(rc, "hsein_solve (device)")
        return X, status

    def device_status(self):
        return hsein_plan_sync_status(self.plan, self.work.data_ptr(), self._stream())

    def restart(self, H, wr, wi, X, status, B=None, max_tries=3):
        """Alg. "hsrq3in": retry the shifts whose status is 1 from new starting
        vectors orthogonal to the previous ones, in place in X and status.
        Synchronizes the stream; returns (code, shifts retried), code 0 when
        every shift converged, 1 (HSEIN_WNOTCONVERGED) otherwise."""
        torch = self.torch
        H = _colmajor(H, torch)
        wr = wr.to(torch.float64).contiguous()
        wi = wi.to(torch.float64).contiguous()
        if B is not None:
            B = _colmajor(B, torch)
        rc, k = hsein_restart(self.plan, H.data_ptr(), _ld(H), wr.data_ptr(), wi.data_ptr(),
                              B.data_ptr() if B is not None else 0,
                              _ld(B) if B is not None else self.n, X.data_ptr(), _ld(X),
                              status.data_ptr(), int(max_tries), self.work.data_ptr(),
                              self.work_bytes, self._stream())
        if rc < 0:
            _check(rc, "hsein_restart")
        return rc, k

    def margins(self):
        """Varah margins of the last solve, per shift in input order (log2;
        > 0 converged)."""
        out = self.torch.empty(self.m, dtype=self.torch.float64, device=self.device)
        _check(hsein_margins(self.plan, self.work.data_ptr(), out.data_ptr(), self._stream()),
               "hsein_margins")
        return out

    def solve_host(self, hH, hwr, hwi, hB, hQ0, hZ, hstatus):
        """End to end from host memory through hsein_solve_host: H, the shifts
        and B go to the device first; Q0 follows on the plan's side stream
        while the solve runs (it is needed only by the backtransform); Z = Q0 X
        and the status codes come back into hZ and hstatus.  Host tensors
        should be pinned and laid out like the device operands (column-major).
        Stream-ordered on the current stream: synchronize before reading hZ
        and hstatus.  The device workspace is allocated on the first call and
        reused."""
        torch = self.torch
        if getattr(self, "_hwork", None) is None:
            nb = hsein_host_workspace(self.plan)
            self._hwork = torch.empty(nb, dtype=torch.uint8, device=self.device)
        hH = _colmajor(hH, torch)
        hQ0 = _colmajor(hQ0, torch)
        hB = _colmajor(hB, torch) if hB is not None else None
        rc = hsein_solve_host(self.plan, hH.data_ptr(), _ld(hH), hwr.data_ptr(), hwi.data_ptr(),
                              hB.data_ptr() if hB is not None else 0,
                              _ld(hB) if hB is not None else self.n, hQ0.data_ptr(), _ld(hQ0),
                              hZ.data_ptr(), _ld(hZ), hstatus.data_ptr(), self._hwork.data_ptr(),
                              self._hwork.numel(), self._stream())
        _check(rc, "hsein_solve_host")
        return hZ, hstatus

    def host_device_status(self):
        """Device status of the last hsein_solve_host call."""
        return hsein_plan_sync_status(self.plan, self._hwork.data_ptr(), self._stream())

    def backtransform(self, Q0, X, Z=None):
        """Z = Q0 X (eigenvectors of A = Q0 H Q0^T)."""
        torch = self.torch
        Q0 = _colmajor(Q0, torch)
        X = _colmajor(X, torch)
        if Z is None:
            Z = torch.empty((self.ncol, self.n), dtype=torch.float64, device=self.device).t()
        rc = hsein_backtransform(self.plan, Q0.data_ptr(), _ld(Q0), X.data_ptr(), _ld(X),
                                 Z.data_ptr(), _ld(Z), self.work.data_ptr(), self.work_bytes,
                                 self._stream())
        _check(rc, "hsein_backtransform")
        return Z

    def graph(self, H, wr, wi, B=None, Q0=None, X=None, status=None, Z=None):
        """One step (solve, then Z = Q0 X when Q0 is given) captured as a CUDA
        graph on these buffers (hsein_graph_create); StepGraph.launch() runs
        it on the current stream.  The tensors are used in place (inputs that
        are already column-major float64 are not copied): refresh their
        contents between launches."""
        torch = self.torch
        H = _colmajor(H, torch)
        wr = wr.to(torch.float64).contiguous()
        wi = wi.to(torch.float64).contiguous()
        if B is not None:
            B = _colmajor(B, torch)
        if X is None:
            X = torch.empty((self.ncol, self.n), dtype=torch.float64, device=self.device).t()
        if status is None:
            status = torch.empty(self.m, dtype=torch.int32, device=self.device)
        if Q0 is not None:
            Q0 = _colmajor(Q0, torch)
            if Z is None:
                Z = torch.empty((self.ncol, self.n), dtype=torch.float64, device=self.device).t()
        with torch.cuda.device(self.device):
            rc, g = hsein_graph_create(
                self.plan, H.data_ptr(), _ld(H), wr.data_ptr(), wi.data_ptr(),
                B.data_ptr() if B is not None else 0, _ld(B) if B is not None else self.n,
                X.data_ptr(), _ld(X), status.data_ptr(),
                Q0.data_ptr() if Q0 is not None else 0, _ld(Q0) if Q0 is not None else self.n,
                Z.data_ptr() if Z is not None else 0, _ld(Z) if Z is not None else self.n,
                self.work.data_ptr(), self.work_bytes)
        _check(rc, "hsein_graph_create")
        return StepGraph(self, g, (H, wr, wi, B, Q0), X, status, Z)


class StepGraph:
    """A captured step of a Solver (Solver.graph); X, status and Z are its
    outputs, valid once the launching stream has completed."""

    def __init__(self, solver, handle, inputs, X, status, Z):
        self.solver, self.handle, self._inputs = solver, handle, inputs
        self.X, self.status, self.Z = X, status, Z

    def launch(self):
        _check(hsein_graph_launch(self.handle, self.solver._stream()), "hsein_graph_launch")

    def __del__(self):
        handle = getattr(self, "handle", None)
        if handle is not None and _lib is not None:
            _lib.hsein_graph_destroy(handle)
            self.handle = None


class Batch:
    """Independent instances solved together in one captured CUDA graph
    (hsein_batch_*).  instances: a list of (H, wr, wi, B or None) CUDA float64
    tensors; X and status tensors are allocated here (column-major X per
    instance).  The tensors are referenced, not copied: refresh their
    contents in place between solves."""

    def __init__(self, instances, streams=16, br_policy=1, shift_block=0, robust=True,
                 omega_log2=1000, device=None):
        import torch
        self.torch = torch
        self.device = torch.device(device or "cuda")
        self._keep = []
        self.X, self.status = [], []
        items = []
        for (H, wr, wi, B) in instances:
            H = _colmajor(H, torch)
            wr = wr.to(torch.float64).contiguous()
            wi = wi.to(torch.float64).contiguous()
            B = _colmajor(B, torch) if B is not None else None
            n = H.shape[0]
            mc = int((wi != 0).sum().item())
            mr = wr.numel() - mc
            X = torch.zeros((mr + 2 * mc, n), dtype=torch.float64, device=self.device).t()
            st = torch.zeros(mr + mc, dtype=torch.int32, device=self.device)
            self._keep += [H, wr, wi, B]
            self.X.append(X)
            self.status.append(st)
            items.append(HseinInstance(n, mr, mc, H.data_ptr(), _ld(H), wr.data_ptr(),
                                       wi.data_ptr(), B.data_ptr() if B is not None else None,
                                       _ld(B) if B is not None else n, X.data_ptr(), _ld(X),
                                       st.data_ptr()))
        opt = hsein_default_options()
        opt.robust = int(bool(robust))
        opt.omega_log2 = int(omega_log2)
        cfg = HseinBatchConfig(int(streams), int(br_policy), int(shift_block), 0)
        with torch.cuda.device(self.device):
            self.batch, self.work_bytes = hsein_batch_plan(items, opt, cfg)
        self.work = torch.empty(self.work_bytes, dtype=torch.uint8, device=self.device)

    def __del__(self):
        b = getattr(self, "batch", None)
        if b is not None and _lib is not None:
            _lib.hsein_batch_destroy(b)
            self.batch = None

    def _stream(self):
        return self.torch.cuda.current_stream(self.device).cuda_stream

    def solve(self):
        """Solve every instance (one graph launch); returns (X list, status list)."""
        _check(hsein_batch_solve(self.batch, self.work.data_ptr(), self.work_bytes, self._stream()),
               "hsein_batch_solve")
        return self.X, self.status

    def autotune(self):
        """Search the batch configurations; returns (config dict, ms)."""
        rc, c, ms = hsein_batch_autotune(self.batch, self.work.data_ptr(), self.work_bytes,
                                         self._stream())
        _check(rc, "hsein_batch_autotune")
        return c.as_dict(), ms

    def info(self):
        c, k = hsein_batch_info(self.batch)
        return c.as_dict(), k


class Server:
    """The serving loop (hsein_server_*): submit requests, drive progress().

    submit(H, wr, wi, B=None, precision=0, br=64) takes CUDA float64 tensors
    (kept alive until the request completes), allocates its X and status and
    returns a ticket; progress() returns the tickets completed since the last
    call; result(ticket) gives (X, status) of a completed request."""

    def __init__(self, hbm_bytes, max_jobs=8, max_merge_shifts=4096, robust=True,
                 omega_log2=1000, device=None, max_bypass=0):
        import torch
        self.torch = torch
        self.device = torch.device(device or "cuda")
        opt = hsein_default_options()
        opt.robust = int(bool(robust))
        opt.omega_log2 = int(omega_log2)
        with torch.cuda.device(self.device):
            self.server = hsein_server_create(hbm_bytes, max_jobs, max_merge_shifts, opt)
        if max_bypass:
            _check(hsein_server_set_bypass(self.server, max_bypass), "hsein_server_set_bypass")
        self._live = {}

    def __del__(self):
        srv = getattr(self, "server", None)
        if srv is not None and _lib is not None:
            _lib.hsein_server_destroy(srv)
            self.server = None

    def submit(self, H, wr, wi, B=None, precision=0, br=64, exps=None):
        torch = self.torch
        H = _colmajor(H, torch)
        wr = wr.to(torch.float64).contiguous()
        wi = wi.to(torch.float64).contiguous()
        B = _colmajor(B, torch) if B is not None else None
        n = H.shape[0]
        mc = int((wi != 0).sum().item())
        mr = wr.numel() - mc
        X = torch.empty((mr + 2 * mc, n), dtype=torch.float64, device=self.device).t()
        st = torch.empty(mr + mc, dtype=torch.int32, device=self.device)
        inst = HseinInstance(n, mr, mc, H.data_ptr(), _ld(H), wr.data_ptr(), wi.data_ptr(),
                             B.data_ptr() if B is not None else None,
                             _ld(B) if B is not None else n, X.data_ptr(), _ld(X), st.data_ptr())
        # the library's streams wait for nothing of torch's: make the inputs ready
        torch.cuda.current_stream(self.device).synchronize()
        rc, t = hsein_server_submit(self.server, HseinRequest(
            inst, int(precision), int(br), exps.data_ptr() if exps is not None else None))
        _check(rc, "hsein_server_submit")
        self._live[t] = (H, wr, wi, B, X, st, exps)
        return t

    def progress(self, wait=False):
        rc, done = hsein_server_progress(self.server, 4096, wait)
        _check(rc, "hsein_server_progress")
        return done

    def result(self, ticket):
        """(X, status) of a completed request (released from the server's
        bookkeeping)."""
        H, wr, wi, B, X, st, exps = self._live.pop(ticket)
        return X, st

    def stats(self):
        return hsein_server_stats(self.server)
