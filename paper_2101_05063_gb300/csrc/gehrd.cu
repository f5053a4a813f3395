// Householder reduction A = Q0 H Q0^T on the GPU (include/hsein.h,
// hsein_gehrd): the step that produces the Hessenberg matrix and Q0 the solve
// and the backtransform take (Sec. 1).  Level 2, one reflector
// P = I - beta v v^T per step k, applied from both sides and to Q0.  The
// two-sided product is written as one rank-2 update,
//     P H P = H - v yh^T - z v^T,  y = beta H^T v,  z = beta H v,
//     yh = y - gamma v,  gamma = beta v^T z,
// so each step streams the trailing columns of H and Q0 twice: a read pass
// for the column dots (y), the row sums (z) and Q0 v, and a read-write pass
// for the update.  Partial sums go to per-block slots summed in a fixed
// order (no atomics): the result is bitwise reproducible.
//
//  k_reflector  one block: x = H(k+1:n, k), alpha = -sign(x_1) ||x||
//               (max-scaled norm), v = x - alpha e_1 (zero above row k+1),
//               beta = 2 / v^T v = 1 / (||x|| (||x|| + |x_1|))
//  k_dots       tiles of 32 NCH columns x 256 RPT rows: row sums of H and Q0
//               against v (per column block), column dots v^T H (per row
//               block; a butterfly reduce-scatter across the warp)
//  k_combine    z = beta sum zp, q = beta sum qp, y = beta sum yp, per-block
//               partials of v^T z; column k becomes (alpha, 0, ..., 0)
//  k_apply      H(:, j) -= v yh_j + z v_j, Q0(:, j) -= q v_j for j > k
#include "../../include/hsein.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>

namespace {

constexpr int kT = 256;  // threads per block
constexpr int kTC = 32;  // columns per k_dots tile
constexpr int kCC = 32;  // columns per k_apply block
constexpr int kApplyG = 4;  // columns per load group of k_apply

struct GState {
    double alpha, beta;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int ceil_div(int a, int b) { return (a + b - 1) / b; }

// workspace carve-up (all offsets 256-byte aligned)
struct Work {
    double *v, *z, *q, *y, *zp, *qp, *yp, *gp;
    GState* g;
    size_t bytes;
};

Work carve(int n, char* base) {
    const size_t nb = align256(sizeof(double) * (size_t)n);
    const int cbmax = ceil_div(n, kTC), rbmax = ceil_div(n, kT), gbmax = ceil_div(n, 32);
    size_t off = 0;
    Work w{};
    auto take = [&](size_t bytes) {
        char* p = base ? base + off : nullptr;
        off += align256(bytes);
        return p;
    };
    w.v = reinterpret_cast<double*>(take(nb));
    w.z = reinterpret_cast<double*>(take(nb));
    w.q = reinterpret_cast<double*>(take(nb));
    w.y = reinterpret_cast<double*>(take(nb));
    w.zp = reinterpret_cast<double*>(take(nb * cbmax));
    w.qp = reinterpret_cast<double*>(take(nb * cbmax));
    w.yp = reinterpret_cast<double*>(take(nb * rbmax));
    w.gp = reinterpret_cast<double*>(take(sizeof(double) * gbmax));
    w.g = reinterpret_cast<GState*>(take(sizeof(GState)));
    w.bytes = off;
    return w;
}

template <int T>
__device__ double block_sum(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < T / 32; ++w) t += red[w];
    return t;
}
template <int T>
__device__ double block_max(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < T / 32; ++w) t = fmax(t, red[w]);
    return t;
}

__global__ void k_identity(int n, double* Q, int ldq) {
    const int j = blockIdx.x;
    for (int i = threadIdx.x; i < n; i += blockDim.x) Q[i + (size_t)j * ldq] = i == j ? 1.0 : 0.0;
}

constexpr int kTR = 256;  // threads of k_reflector

// One block.  The largest |x_i| is an integer maximum of the bit patterns
// (monotonic for non-negative doubles); the sum of squares is scaled by the
// exact power of two 2^-e, e = the exponent of that maximum.  Only warp 0
// combines the per-warp results (FP64 work on one SM is the cost here).
__global__ void __launch_bounds__(kTR)
k_reflector(int n, int k, const double* __restrict__ H, int ldh, double* __restrict__ v,
            GState* g) {
    __shared__ unsigned long long redm[kTR / 32];
    __shared__ double reds[kTR / 32];
    __shared__ double bc[2];
    const double* x = H + (size_t)k * ldh;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    unsigned long long mb = 0;
    for (int i = k + 1 + tid; i < n; i += kTR)
        mb = max(mb, (unsigned long long)__double_as_longlong(x[i]) & 0x7FFFFFFFFFFFFFFFull);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
    if (lane == 0) redm[w] = mb;
    __syncthreads();
    mb = redm[0];
#pragma unroll
    for (int q = 1; q < kTR / 32; ++q) mb = max(mb, redm[q]);
    const double m = __longlong_as_double((long long)mb);
    // e kept above -1020 so that 2^-e stays finite
    const int em = m > 0.0 ? max(ilogb(m), -1020) : 0;
    const double sc = scalbn(1.0, -em);
    double ss = 0.0;
    for (int i = k + 1 + tid; i < n; i += kTR) {
        const double t = x[i] * sc;
        ss = fma(t, t, ss);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if (lane == 0) reds[w] = ss;
    __syncthreads();
    if (w == 0) {
        double t = lane < kTR / 32 ? reds[lane] : 0.0;
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) {
            const double nx = m > 0.0 ? scalbn(sqrt(t), em) : 0.0, x0 = x[k + 1];
            // a zero column keeps its (signed) zero: no reflection, beta = 0
            const double alpha = nx == 0.0 ? x0 : (x0 >= 0.0 ? -nx : nx);
            // v^T v = ||x||^2 - 2 alpha x_1 + alpha^2 = 2 ||x|| (||x|| + |x_1|)
            const double beta = nx > 0.0 ? 1.0 / (nx * (nx + fabs(x0))) : 0.0;
            bc[0] = x0 - alpha;
            g->alpha = alpha;
            g->beta = beta;
        }
    }
    __syncthreads();
    const double v1 = bc[0];
    for (int i = tid; i < n; i += kTR) v[i] = i <= k ? 0.0 : (i == k + 1 ? v1 : x[i]);
}

// Butterfly reduce-scatter: every lane enters with 32 values c[0..31] (one
// per column); afterwards c[0] of lane L holds the warp's sum for column L.
__device__ __forceinline__ void warp_reduce_scatter32(double (&c)[kTC]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const bool hi = (lane & s) != 0;  // this lane keeps the upper half
#pragma unroll
        for (int t = 0; t < s; ++t) {
            const double keep = hi ? c[t + s] : c[t];
            const double send = hi ? c[t] : c[t + s];
            c[t] = keep + __shfl_xor_sync(0xffffffffu, send, s);
        }
    }
}

// read pass over the columns j0 .. j0 + 32 NCH - 1 (j0 = k+1 + 32 NCH cb)
// and the rows rb 256 RPT + 256 s + tid, s < RPT, of H and Q0: row sums
// against v accumulate over the column chunks (one partial per column
// block), column dots v^T H are reduced per chunk across the block (one
// partial per row block).  Rows <= k carry v_i = 0: a warp whose rows all lie
// there skips the column-dot products.
template <int RPT, int NCH>
__global__ void __launch_bounds__(kT, 2)
k_dots(int n, int k, const double* __restrict__ H, int ldh, const double* __restrict__ Q, int ldq,
       const double* __restrict__ v, double* __restrict__ zp, double* __restrict__ qp,
       double* __restrict__ yp, int ldp) {
    __shared__ double vs[NCH * kTC];
    __shared__ double red[kT / 32][kTC];
    const int cb = blockIdx.x, rb = blockIdx.y, tid = threadIdx.x;
    const int lane = tid & 31, w = tid >> 5;
    const int jb = k + 1 + cb * NCH * kTC;
    for (int t = tid; t < NCH * kTC; t += kT) vs[t] = jb + t < n ? v[jb + t] : 0.0;
    __syncthreads();
    const int i0 = rb * kT * RPT + tid;
    int ri[RPT];
    bool dot[RPT];  // warp-uniform: some row of this warp lies below row k
    double vi[RPT], rs[RPT], rq[RPT];
#pragma unroll
    for (int s = 0; s < RPT; ++s) {
        const int i = i0 + s * kT;
        ri[s] = min(i, n - 1);  // a row past n reads row n-1 with v = 0
        vi[s] = i < n ? v[i] : 0.0;
        dot[s] = i0 - lane + s * kT + 31 > k;
        rs[s] = 0.0;
        rq[s] = 0.0;
    }
    // first row slot whose warp has rows below row k (RPT: none); the FP64
    // pipe charges a predicated-off instruction like an executed one, so
    // the column-dot products are branched around, not predicated
    int sd = RPT;
#pragma unroll
    for (int s = RPT - 1; s >= 0; --s)
        if (dot[s]) sd = s;
#pragma unroll 1
    for (int ch = 0; ch < NCH; ++ch) {
        const int j0 = jb + ch * kTC;
        if (j0 >= n) break;
        const int nc = min(kTC, n - j0);
        const double* Hb = H + (size_t)j0 * ldh;
        const double* Qb = Q + (size_t)j0 * ldq;
        const double* vc = vs + ch * kTC;
        double c[kTC];
        auto sweep = [&](auto SDc) {
            constexpr int SD = decltype(SDc)::value;
#pragma unroll
            for (int t = 0; t < kTC; ++t) {
                c[t] = 0.0;
                if (t < nc) {
                    const double vt = vc[t];
#pragma unroll
                    for (int s = 0; s < RPT; ++s) {
                        const double h = Hb[ri[s] + (size_t)t * ldh];
                        rs[s] = fma(h, vt, rs[s]);
                        if (s >= SD) c[t] = fma(vi[s], h, c[t]);
                        rq[s] = fma(Qb[ri[s] + (size_t)t * ldq], vt, rq[s]);
                    }
                }
            }
        };
        switch (sd) {  // every slot from sd on needs the column dots
            case 0: sweep(std::integral_constant<int, 0>{}); break;
            case 1: if constexpr (RPT > 1) { sweep(std::integral_constant<int, 1>{}); break; }
            [[fallthrough]];
            case 2: if constexpr (RPT > 2) { sweep(std::integral_constant<int, 2>{}); break; }
            [[fallthrough]];
            case 3: if constexpr (RPT > 3) { sweep(std::integral_constant<int, 3>{}); break; }
            [[fallthrough]];
            default: sweep(std::integral_constant<int, RPT>{});
        }
        if (sd < RPT) warp_reduce_scatter32(c);  // else c is all zero
        __syncthreads();  // the previous chunk's red[] has been read
        red[w][lane] = c[0];
        __syncthreads();
        if (tid < nc) {
            double t = 0.0;
#pragma unroll
            for (int r = 0; r < kT / 32; ++r) t += red[r][tid];
            yp[(size_t)rb * ldp + j0 + tid] = t;
        }
    }
#pragma unroll
    for (int s = 0; s < RPT; ++s) {
        const int i = i0 + s * kT;
        if (i < n) {
            zp[(size_t)cb * ldp + i] = rs[s];
            qp[(size_t)cb * ldp + i] = rq[s];
        }
    }
}

constexpr int kTCB = 32;  // threads per k_combine block

__global__ void __launch_bounds__(kTCB)
k_combine(int n, int k, double* __restrict__ H, int ldh, const double* __restrict__ v,
          const double* __restrict__ zp, const double* __restrict__ qp,
          const double* __restrict__ yp, int ldp, int ncb, int nrb, double* __restrict__ z,
          double* __restrict__ q, double* __restrict__ y, double* __restrict__ gp,
          const GState* __restrict__ g) {
    const int i = blockIdx.x * kTCB + threadIdx.x;
    const double beta = g->beta;
    double part = 0.0;
    if (i < n) {
        // four independent partial sums, added in a fixed order
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0, b0 = 0.0, b1 = 0.0, b2 = 0.0, b3 = 0.0;
        int b = 0;
        for (; b + 4 <= ncb; b += 4) {
            a0 += zp[(size_t)b * ldp + i];
            a1 += zp[(size_t)(b + 1) * ldp + i];
            a2 += zp[(size_t)(b + 2) * ldp + i];
            a3 += zp[(size_t)(b + 3) * ldp + i];
            b0 += qp[(size_t)b * ldp + i];
            b1 += qp[(size_t)(b + 1) * ldp + i];
            b2 += qp[(size_t)(b + 2) * ldp + i];
            b3 += qp[(size_t)(b + 3) * ldp + i];
        }
        for (; b < ncb; ++b) {
            a0 += zp[(size_t)b * ldp + i];
            b0 += qp[(size_t)b * ldp + i];
        }
        const double sz = ((a0 + a1) + (a2 + a3)) * beta;
        z[i] = sz;
        q[i] = ((b0 + b1) + (b2 + b3)) * beta;
        part = v[i] * sz;
        if (i > k) {
            double sy = 0.0;
            for (int r = 0; r < nrb; ++r) sy += yp[(size_t)r * ldp + i];
            y[i] = sy * beta;
            // the reduced column
            H[i + (size_t)k * ldh] = i == k + 1 ? g->alpha : 0.0;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (threadIdx.x == 0) gp[blockIdx.x] = part;
}

template <int G>
__global__ void __launch_bounds__(kT, 16 / G)
k_apply(int n, int k, double* __restrict__ H, int ldh, double* __restrict__ Q, int ldq,
        const double* __restrict__ v, const double* __restrict__ z, const double* __restrict__ q,
        const double* __restrict__ y, const double* __restrict__ gp, int ngp,
        const GState* __restrict__ g) {
    __shared__ double vs[kCC], ys[kCC];
    __shared__ double gam;
    const int tid = threadIdx.x;
    const int j0 = k + 1 + blockIdx.y * kCC;
    const int nc = min(kCC, n - j0);
    if (tid < 32) {
        double t = 0.0;
        for (int b = tid; b < ngp; b += 32) t += gp[b];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (tid == 0) gam = g->beta * t;
    }
    __syncthreads();
    if (tid < kCC) {
        const double vj = tid < nc ? v[j0 + tid] : 0.0;
        vs[tid] = vj;
        ys[tid] = tid < nc ? fma(-gam, vj, y[j0 + tid]) : 0.0;
    }
    __syncthreads();
    const int i = blockIdx.x * kT + tid;
    if (i >= n) return;
    const double vi = v[i], zi = z[i], qi = q[i];
    double* Hb = H + (size_t)j0 * ldh + i;
    double* Qb = Q + (size_t)j0 * ldq + i;
    // groups of G columns: every load of a group is issued before its
    // stores (the compiler cannot reorder loads past stores into the same
    // arrays), so each thread keeps 2 G loads in flight
    const bool below = i > k;  // v_i = 0 above: the right-hand term only
#pragma unroll 1
    for (int t0 = 0; t0 < nc; t0 += G) {
        double hv[G], qv[G];
        if (t0 + G <= nc) {
#pragma unroll
            for (int u = 0; u < G; ++u) {
                hv[u] = Hb[(size_t)(t0 + u) * ldh];
                qv[u] = Qb[(size_t)(t0 + u) * ldq];
            }
            if (below) {
#pragma unroll
                for (int u = 0; u < G; ++u) hv[u] = fma(-vi, ys[t0 + u], fma(-zi, vs[t0 + u], hv[u]));
            } else {
#pragma unroll
                for (int u = 0; u < G; ++u) hv[u] = fma(-zi, vs[t0 + u], hv[u]);
            }
#pragma unroll
            for (int u = 0; u < G; ++u) {
                qv[u] = fma(-qi, vs[t0 + u], qv[u]);
                Hb[(size_t)(t0 + u) * ldh] = hv[u];
                Qb[(size_t)(t0 + u) * ldq] = qv[u];
            }
        } else {
            for (int t = t0; t < nc; ++t) {
                Hb[(size_t)t * ldh] = fma(-vi, ys[t], fma(-zi, vs[t], Hb[(size_t)t * ldh]));
                Qb[(size_t)t * ldq] = fma(-qi, vs[t], Qb[(size_t)t * ldq]);
            }
        }
    }
}

}  // namespace

extern "C" {

hsein_status hsein_gehrd_workspace(int n, size_t* workspace_bytes) {
    if (n < 1 || !workspace_bytes) return HSEIN_EARG;
    *workspace_bytes = carve(n, nullptr).bytes;
    return HSEIN_OK;
}

hsein_status hsein_gehrd(int n, const double* dA, int lda, double* dH, int ldh, double* dQ,
                         int ldq, void* dWork, size_t work_bytes, void* stream) {
    if (n < 1 || !dA || lda < n || !dH || ldh < n || !dQ || ldq < n || !dWork) return HSEIN_EARG;
    if ((const void*)dH == (const void*)dA || (const void*)dQ == (const void*)dA ||
        (const void*)dQ == (const void*)dH)
        return HSEIN_EARG;
    if (reinterpret_cast<uintptr_t>(dWork) & 255) return HSEIN_EARG;
    const Work w = carve(n, static_cast<char*>(dWork));
    if (work_bytes < w.bytes) return HSEIN_ENOMEM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemcpy2DAsync(dH, sizeof(double) * ldh, dA, sizeof(double) * lda, sizeof(double) * n, n,
                          cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return HSEIN_ECUDA;
    k_identity<<<n, kT, 0, s>>>(n, dQ, ldq);
    const int ldp = (int)(align256(sizeof(double) * (size_t)n) / sizeof(double));
    const int rbs = ceil_div(n, kT), cbs = ceil_div(n, kTCB);
    for (int k = 0; k + 2 < n; ++k) {
        const int m = n - k - 1;
        k_reflector<<<1, kTR, 0, s>>>(n, k, dH, ldh, w.v, w.g);
        // more rows per thread (fewer cross-lane reductions, fewer partials)
        // while the grid still fills the GPU (thresholds from a sweep of the
        // tile shapes at n = 4096 on GB300)
        const int ncb = ceil_div(m, kTC);
        int nrb;
        if ((long long)ncb * ceil_div(n, 4 * kT) >= 256) {
            nrb = ceil_div(n, 4 * kT);
            k_dots<4, 1><<<dim3(ncb, nrb), kT, 0, s>>>(n, k, dH, ldh, dQ, ldq, w.v, w.zp, w.qp,
                                                       w.yp, ldp);
        } else if ((long long)ncb * ceil_div(n, 2 * kT) >= 200) {
            nrb = ceil_div(n, 2 * kT);
            k_dots<2, 1><<<dim3(ncb, nrb), kT, 0, s>>>(n, k, dH, ldh, dQ, ldq, w.v, w.zp, w.qp,
                                                       w.yp, ldp);
        } else {
            nrb = rbs;
            k_dots<1, 1><<<dim3(ncb, nrb), kT, 0, s>>>(n, k, dH, ldh, dQ, ldq, w.v, w.zp, w.qp,
                                                       w.yp, ldp);
        }
        k_combine<<<cbs, kTCB, 0, s>>>(n, k, dH, ldh, w.v, w.zp, w.qp, w.yp, ldp, ncb, nrb, w.z,
                                       w.q, w.y, w.gp, w.g);
        k_apply<kApplyG><<<dim3(rbs, ceil_div(m, kCC)), kT, 0, s>>>(n, k, dH, ldh, dQ, ldq, w.v, w.z, w.q,
                                                            w.y, w.gp, cbs, w.g);
    }
    return cudaGetLastError() == cudaSuccess ? HSEIN_OK : HSEIN_ECUDA;
}

}  // extern "C"
