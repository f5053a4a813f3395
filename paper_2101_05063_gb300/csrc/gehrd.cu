// Householder reduction A = Q0 H Q0^T on the GPU (include/hsein.h,
// hsein_gehrd): the step that produces the Hessenberg matrix and Q0 the solve
// and the backtransform take (Sec. 1).  Level-2 form: step k forms the
// reflector of column k and applies it from both sides and to Q0, each
// pass streaming the trailing part of H (and Q0) once; the n - 2 steps are
// bound by memory bandwidth.
//
//  k_reflector   one block: v = x - alpha e_1 for x = H(k+1:n, k),
//                alpha = -sign(x_1) ||x|| (max-scaled norm),
//                beta = 2 / (v^T v) = 1 / (||x|| (||x|| + |x_1|)); clears u, uq
//  k_left        one block per column j >= k: H(k+1:n, j) -= beta (v^T H(k+1:n, j)) v;
//                column k itself becomes (alpha, 0, ..., 0) exactly
//  k_right_gemv  u = H(:, k+1:n) v, uq = Q0(:, k+1:n) v (column chunks, atomics)
//  k_rank1       H(:, j) -= beta u v_j, Q0(:, j) -= beta uq v_j for j > k
#include "../../include/hsein.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

namespace {

constexpr int kT = 256;
constexpr int kChunk = 64;  // columns per block of k_right_gemv

struct GState {
    double alpha, beta;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

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

__global__ void __launch_bounds__(1024)
k_reflector(int n, int k, const double* __restrict__ H, int ldh, double* __restrict__ v,
            double* __restrict__ u, double* __restrict__ uq, GState* g) {
    __shared__ double red[32];
    const double* x = H + (size_t)k * ldh;
    const int tid = threadIdx.x;
    double m = 0.0;
    for (int i = k + 1 + tid; i < n; i += 1024) m = fmax(m, fabs(x[i]));
    m = block_max<1024>(m, red);
    double ss = 0.0;
    if (m > 0.0)
        for (int i = k + 1 + tid; i < n; i += 1024) {
            const double t = x[i] / m;
            ss += t * t;
        }
    ss = block_sum<1024>(ss, red);
    const double nx = m * sqrt(ss), x0 = x[k + 1];
    // a zero column keeps its (signed) zero: no reflection, beta = 0
    const double alpha = nx == 0.0 ? x0 : (x0 >= 0.0 ? -nx : nx);
    // v^T v = ||x||^2 - 2 alpha x_1 + alpha^2 = 2 ||x|| (||x|| + |x_1|)
    const double beta = nx > 0.0 ? 1.0 / (nx * (nx + fabs(x0))) : 0.0;
    for (int i = tid; i < n; i += 1024) {
        v[i] = i <= k ? 0.0 : (i == k + 1 ? x0 - alpha : x[i]);
        u[i] = 0.0;
        uq[i] = 0.0;
    }
    if (tid == 0) {
        g->alpha = alpha;
        g->beta = beta;
    }
}

__global__ void __launch_bounds__(kT)
k_left(int n, int k, double* __restrict__ H, int ldh, const double* __restrict__ v,
       const GState* __restrict__ g) {
    __shared__ double red[kT / 32];
    const int j = k + blockIdx.x;
    double* col = H + (size_t)j * ldh;
    if (j == k) {
        // the reduced column: (alpha, 0, ..., 0) below the diagonal
        for (int i = k + 1 + threadIdx.x; i < n; i += kT) col[i] = i == k + 1 ? g->alpha : 0.0;
        return;
    }
    double d = 0.0;
    for (int i = k + 1 + threadIdx.x; i < n; i += kT) d += v[i] * col[i];
    d = g->beta * block_sum<kT>(d, red);
    for (int i = k + 1 + threadIdx.x; i < n; i += kT) col[i] -= d * v[i];
}

__global__ void __launch_bounds__(kT)
k_right_gemv(int n, int k, const double* __restrict__ H, int ldh, const double* __restrict__ Q,
             int ldq, const double* __restrict__ v, double* __restrict__ u, double* __restrict__ uq) {
    const int i = blockIdx.x * kT + threadIdx.x;
    if (i >= n) return;
    const int j0 = k + 1 + blockIdx.y * kChunk, j1 = min(n, j0 + kChunk);
    double su = 0.0, sq = 0.0;
    for (int j = j0; j < j1; ++j) {
        const double vj = v[j];
        su = fma(H[i + (size_t)j * ldh], vj, su);
        sq = fma(Q[i + (size_t)j * ldq], vj, sq);
    }
    atomicAdd(u + i, su);
    atomicAdd(uq + i, sq);
}

__global__ void __launch_bounds__(kT)
k_rank1(int n, int k, double* __restrict__ H, int ldh, double* __restrict__ Q, int ldq,
        const double* __restrict__ v, const double* __restrict__ u, const double* __restrict__ uq,
        const GState* __restrict__ g) {
    const int i = blockIdx.x * kT + threadIdx.x;
    if (i >= n) return;
    const double b = g->beta, ui = u[i], uqi = uq[i];
    for (int j = k + 1 + blockIdx.y; j < n; j += gridDim.y) {
        const double f = b * v[j];
        H[i + (size_t)j * ldh] -= ui * f;
        Q[i + (size_t)j * ldq] -= uqi * f;
    }
}

}  // namespace

extern "C" {

hsein_status hsein_gehrd_workspace(int n, size_t* workspace_bytes) {
    if (n < 1 || !workspace_bytes) return HSEIN_EARG;
    *workspace_bytes = 3 * align256(sizeof(double) * (size_t)n) + 256;
    return HSEIN_OK;
}

hsein_status hsein_gehrd(int n, const double* dA, int lda, double* dH, int ldh, double* dQ,
                         int ldq, void* dWork, size_t work_bytes, void* stream) {
    if (n < 1 || !dA || lda < n || !dH || ldh < n || !dQ || ldq < n || !dWork) return HSEIN_EARG;
    if ((const void*)dH == (const void*)dA || (const void*)dQ == (const void*)dA ||
        (const void*)dQ == (const void*)dH)
        return HSEIN_EARG;
    if (reinterpret_cast<uintptr_t>(dWork) & 255) return HSEIN_EARG;
    size_t need = 0;
    hsein_gehrd_workspace(n, &need);
    if (work_bytes < need) return HSEIN_ENOMEM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char* w = static_cast<char*>(dWork);
    const size_t vb = align256(sizeof(double) * (size_t)n);
    double* v = reinterpret_cast<double*>(w);
    double* u = reinterpret_cast<double*>(w + vb);
    double* uq = reinterpret_cast<double*>(w + 2 * vb);
    GState* g = reinterpret_cast<GState*>(w + 3 * vb);
    if (cudaMemcpy2DAsync(dH, sizeof(double) * ldh, dA, sizeof(double) * lda, sizeof(double) * n, n,
                          cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return HSEIN_ECUDA;
    k_identity<<<n, kT, 0, s>>>(n, dQ, ldq);
    const int rb = (n + kT - 1) / kT;
    for (int k = 0; k + 2 < n; ++k) {
        k_reflector<<<1, 1024, 0, s>>>(n, k, dH, ldh, v, u, uq, g);
        k_left<<<n - k, kT, 0, s>>>(n, k, dH, ldh, v, g);
        k_right_gemv<<<dim3(rb, (n - k - 1 + kChunk - 1) / kChunk), kT, 0, s>>>(n, k, dH, ldh, dQ,
                                                                                 ldq, v, u, uq);
        k_rank1<<<dim3(rb, std::min(n - k - 1, 65535)), kT, 0, s>>>(n, k, dH, ldh, dQ, ldq, v, u, uq, g);
    }
    return cudaGetLastError() == cudaSuccess ? HSEIN_OK : HSEIN_ECUDA;
}

}  // extern "C"
