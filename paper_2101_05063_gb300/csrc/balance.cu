// Power-of-two balancing of a Hessenberg matrix and the map of eigenvectors
// back (include/hsein.h: hsein_balance, hsein_unbalance).  Graded inputs
// D H D^-1 put entries of very different scale into one row, which one
// power-of-two exponent per row of a digit split cannot represent; after
// Hb = D'^-1 H D' with D' = diag(2^e) the split-precision products apply
// (the balancing step of Parlett and Reinsch's method, radix 2).
//
//  k_balance        one block: sweeps i = 0..n-1; the off-diagonal 1-norms
//                   r_i (row) and c_i (column) of the current scaled matrix
//                   are block reductions of |h| 2^(difference of exponents),
//                   kept as (exponent, scaled sum) so that nothing overflows;
//                   2^k with k nearest to log2(sqrt(r_i / c_i)) is accepted
//                   when it lowers r_i + c_i by 5% or more
//  k_balance_apply  Hb = D^-1 H D (exact power-of-two scaling)
//  k_unbalance      per shift: D x scaled by 2^-max exponent, normalized
#include "../../include/hsein.h"
#include "common.cuh"

#include <climits>
#include <cmath>

namespace hsein {
namespace {

constexpr int kThreads = 1024;

// nonnegative value s 2^E (s == 0: zero), with 1 <= s < 2n after additions
struct Acc {
    int E;
    double s;
};

__device__ inline Acc acc_add(Acc a, int te, double mt) {
    if (mt == 0.0) return a;
    if (a.s == 0.0) return Acc{te, mt};
    if (te > a.E) {
        a.s = scalbn(a.s, a.E - te) + mt;
        a.E = te;
    } else {
        a.s += scalbn(mt, te - a.E);
    }
    return a;
}
// + |h| 2^d
__device__ inline Acc acc_add_scaled(Acc a, double h, int d) {
    if (h == 0.0) return a;
    const int eh = ilogb(h);
    return acc_add(a, eh + d, scalbn(fabs(h), -eh));
}
__device__ inline Acc acc_merge(Acc a, Acc b) { return b.s == 0.0 ? a : acc_add(a, b.E, b.s); }
__device__ inline double acc_log2(Acc a) { return a.s == 0.0 ? -HUGE_VAL : a.E + log2(a.s); }

__device__ Acc block_acc(Acc a, Acc* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        Acc b{__shfl_xor_sync(0xffffffffu, a.E, o), __shfl_xor_sync(0xffffffffu, a.s, o)};
        a = acc_merge(a, b);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = a;
    __syncthreads();
    Acc t{0, 0.0};
    for (int w = 0; w < kThreads / 32; ++w) t = acc_merge(t, red[w]);
    return t;
}

__global__ void __launch_bounds__(kThreads)
k_balance(int n, const double* __restrict__ H, int ldh, int* __restrict__ e, int max_sweeps) {
    __shared__ Acc redc[kThreads / 32], redr[kThreads / 32];
    __shared__ int changed;
    for (int i = threadIdx.x; i < n; i += kThreads) e[i] = 0;
    __syncthreads();
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        if (threadIdx.x == 0) changed = 0;
        __syncthreads();
        for (int i = 0; i < n; ++i) {
            const int ei = e[i];
            Acc c{0, 0.0}, r{0, 0.0};
            // column i: rows 0 .. min(i+1, n-1); row i: columns max(i-1, 0) .. n-1
            const int jc = min(i + 1, n - 1), jr = max(i - 1, 0);
            for (int j = threadIdx.x; j <= jc; j += kThreads)
                if (j != i) c = acc_add_scaled(c, H[j + (size_t)i * ldh], ei - e[j]);
            for (int j = jr + threadIdx.x; j < n; j += kThreads)
                if (j != i) r = acc_add_scaled(r, H[i + (size_t)j * ldh], e[j] - ei);
            c = block_acc(c, redc);
            r = block_acc(r, redr);
            if (threadIdx.x == 0 && c.s != 0.0 && r.s != 0.0) {
                const double lc = acc_log2(c), lr = acc_log2(r);
                const int k = (int)rint(0.5 * (lr - lc));
                if (k != 0) {
                    // c 2^k + r 2^-k < 0.95 (c + r), relative to the larger of c, r
                    const double L = fmax(lc, lr);
                    const double before = exp2(lc - L) + exp2(lr - L);
                    const double after = exp2(lc - L + k) + exp2(lr - L - k);
                    if (after < 0.95 * before) {
                        e[i] = ei + k;
                        changed = 1;
                    }
                }
            }
            __syncthreads();
        }
        if (!changed) break;
        __syncthreads();
    }
}

// Hb(i, j) = H(i, j) 2^(e_j - e_i) on the Hessenberg pattern, 0 below it
__global__ void k_balance_apply(int n, const double* __restrict__ H, int ldh,
                                double* __restrict__ Hb, int ldhb, const int* __restrict__ e) {
    const int j = blockIdx.x;
    const int ej = e[j];
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double v = i <= j + 1 ? scalbn(H[i + (size_t)j * ldh], ej - e[i]) : 0.0;
        Hb[i + (size_t)j * ldhb] = v;
    }
}

__global__ void __launch_bounds__(256)
k_unbalance(int n, int m, const double* __restrict__ wi, const int* __restrict__ e,
            double* __restrict__ X, int ldx) {
    __shared__ int s_red[8];
    __shared__ double s_sum[8];
    const int l = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // column of shift l: l plus the complex shifts before it
    int cnt = 0;
    for (int q = tid; q < l; q += 256) cnt += wi[q] != 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (lane == 0) s_red[warp] = cnt;
    __syncthreads();
    int col = l;
    for (int w = 0; w < 8; ++w) col += s_red[w];
    __syncthreads();
    const int nc = wi[l] != 0.0 ? 2 : 1;
    double* x0 = X + (size_t)col * ldx;
    // largest exponent of D x over the shift's columns
    int mx = INT_MIN;
    for (int c = 0; c < nc; ++c)
        for (int i = tid; i < n; i += 256) {
            const double v = x0[i + (size_t)c * ldx];
            if (v != 0.0) mx = max(mx, ilogb(v) + e[i]);
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) s_red[warp] = mx;
    __syncthreads();
    mx = INT_MIN;
    for (int w = 0; w < 8; ++w) mx = max(mx, s_red[w]);
    if (mx == INT_MIN) return;  // a zero (not converged) column stays zero
    // y = D x 2^-mx (every |y_i| < 2), then y / ||y||_2
    double ss = 0.0;
    for (int c = 0; c < nc; ++c)
        for (int i = tid; i < n; i += 256) {
            const double y = scalbn(x0[i + (size_t)c * ldx], e[i] - mx);
            ss += y * y;
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    __syncthreads();
    if (lane == 0) s_sum[warp] = ss;
    __syncthreads();
    double tot = 0.0;
    for (int w = 0; w < 8; ++w) tot += s_sum[w];
    const double r = 1.0 / sqrt(tot);
    for (int c = 0; c < nc; ++c)
        for (int i = tid; i < n; i += 256) {
            double* p = x0 + i + (size_t)c * ldx;
            *p = scalbn(*p, e[i] - mx) * r;
        }
}

}  // namespace
}  // namespace hsein

extern "C" {

hsein_status hsein_balance(int n, const double* dH, int ldh, double* dHb, int ldhb, int* dExp,
                           int max_sweeps, void* stream) {
    if (n < 1 || !dH || ldh < n || !dHb || ldhb < n || !dExp || max_sweeps < 0) return HSEIN_EARG;
    if ((const void*)dHb == (const void*)dH) return HSEIN_EARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    hsein::k_balance<<<1, hsein::kThreads, 0, s>>>(n, dH, ldh, dExp, max_sweeps);
    hsein::k_balance_apply<<<n, 256, 0, s>>>(n, dH, ldh, dHb, ldhb, dExp);
    return cudaGetLastError() == cudaSuccess ? HSEIN_OK : HSEIN_ECUDA;
}

hsein_status hsein_unbalance(int n, int m, const double* dWi, const int* dExp, double* dX,
                             int ldx, void* stream) {
    if (n < 1 || m < 1 || !dWi || !dExp || !dX || ldx < n) return HSEIN_EARG;
    hsein::k_unbalance<<<m, 256, 0, static_cast<cudaStream_t>(stream)>>>(n, m, dWi, dExp, dX, ldx);
    return cudaGetLastError() == cudaSuccess ? HSEIN_OK : HSEIN_ECUDA;
}

}  // extern "C"
