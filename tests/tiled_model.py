"""A numpy model of the CUDA path's single-pass tiled schedule (no scaling).

It mirrors the kernels' formulas step by step -- per-tile Henry sweep and
solve, z = G^H [0; x], the prefix weights w_k = c_k prod_{i<k} s_i and
pi = prod s_i, and the fused update
    B   <- B - A Z' - R~ z_br + lambda rho' e_last
    R~  <- A W + pi R~ - lambda c_0 e_last
over the rows above each tile -- so that the host-side algebra of the design
can be checked against the oracle without a GPU.  Test infrastructure only.
"""
import numpy as np


def tiled_solve(H, lam, b, br):
    """Solution of (H - lam I) x = b (complex arithmetic throughout) by the
    single-pass tiled schedule; returns (x_backtransformed, C, S)."""
    H = np.asarray(H, dtype=np.float64)
    n = H.shape[0]
    lam = complex(lam)
    N = (n + br - 1) // br
    b0 = n - (N - 1) * br
    start = [0] + [b0 + (J - 1) * br for J in range(1, N)]
    height = [b0] + [br] * (N - 1)
    X = np.array(b, dtype=np.complex128)
    Rt = H[:, n - 1].astype(np.complex128)
    Rt[n - 1] -= lam
    C = np.zeros(n, dtype=np.complex128)
    S = np.zeros(n)
    for J in range(N - 1, -1, -1):
        p0, bt = start[J], height[J]
        v = Rt[p0:p0 + bt].copy()
        x = X[p0:p0 + bt].copy()
        for k in range(bt - 1, 0, -1):
            h = H[p0 + k, p0 + k - 1]
            r = np.hypot(h, abs(v[k]))
            c, s = v[k] / r, -h / r
            C[p0 + k], S[p0 + k] = c, s
            x[k] /= r
            t = H[p0:p0 + k, p0 + k - 1].astype(np.complex128)
            t[k - 1] -= lam
            Rcol = -s * t + np.conj(c) * v[:k]
            x[:k] -= x[k] * Rcol
            v[:k] = c * t + s * v[:k]
        if p0 > 0:
            h = H[p0, p0 - 1]
            r = np.hypot(h, abs(v[0]))
            c0, s0 = v[0] / r, -h / r
            x[0] /= r
        else:
            c0, s0 = 1.0, 0.0
            x[0] /= v[0]
        C[p0], S[p0] = c0, s0
        X[p0:p0 + bt] = x
        if p0 == 0:
            break
        # Z' and W
        cs, ss = C[p0:p0 + bt], S[p0:p0 + bt]
        Zp = np.zeros(bt, dtype=np.complex128)
        W = np.zeros(bt, dtype=np.complex128)
        Zp[0] = -ss[0] * x[0]
        tau = np.conj(cs[0]) * x[0]
        W[0] = cs[0]
        pr = ss[0]
        for k in range(1, bt):
            Zp[k] = cs[k] * tau - ss[k] * x[k]
            tau = ss[k] * tau + np.conj(cs[k]) * x[k]
            W[k] = cs[k] * pr
            pr *= ss[k]
        zbr, pi = tau, pr
        A = H[:p0, p0 - 1:p0 - 1 + bt]
        Rold = Rt[:p0].copy()
        X[:p0] = X[:p0] - A @ Zp - Rold * zbr
        X[p0 - 1] += lam * Zp[0]
        Rt[:p0] = A @ W + pi * Rold
        Rt[p0 - 1] -= lam * c0
    # backtransform
    y = X.copy()
    tau = y[0]
    for k in range(1, n):
        yk = y[k]
        y[k - 1] = C[k] * tau - S[k] * yk
        tau = S[k] * tau + np.conj(C[k]) * yk
    y[n - 1] = tau
    return y, C, S
