// Restart of inverse iteration for the shifts that did not converge
// (Alg. "hsrq3in", Sec. 4.2): a new starting vector orthogonal to the
// previous choices, solved again for just those shifts.
//
// The paper asks only for orthogonality.  The vectors used here: for a real
// shift with previous starting vector b, trial t (t = 1, 2, ...) is column
// n+1-t of the Householder reflector P = I - 2 w w^T / (w^T w),
// w = b/||b|| + sign(b_1) e_1, whose first column is -sign(b_1) b/||b||; the
// other columns are orthonormal and orthogonal to b, so every trial is
// orthogonal to b and to the earlier trials.  For a complex shift with
// b = b_re + i b_im the trial is column n+1-t of P1 P2, the Householder QR of
// [b_re b_im] (P2 acts on rows 2..n); columns 3..n are real vectors orthogonal
// to both parts, hence b^H x = 0.  Trials are unit vectors (the starting
// vector's scale does not enter Varah's test).
//
//  k_restart_trial   one block per retried shift: its shift and its trial
//                    starting vector(s) into the compact sub-problem
//  k_restart_scatter one block per retried shift: a converged sub-solution
//                    replaces the zeroed columns of X, status becomes 0
#include "common.cuh"

namespace hsein {
namespace {

constexpr int kThreads = 256;

// sum over the block (fixed reduction order)
__device__ double block_sum(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) t += red[w];
    return t;
}
__device__ double block_max(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) t = fmax(t, red[w]);
    return t;
}

// Householder vector of the unit vector v (length len, stride 1) into w:
// w = v + sign(v_0) e_0; returns 2 / (w^T w)
__device__ double householder(const double* v, double* w, int len, double* red) {
    const double s0 = v[0] >= 0.0 ? 1.0 : -1.0;
    __syncthreads();  // every thread has read v[0] before w (possibly v) is written
    double acc = 0.0;
    for (int i = threadIdx.x; i < len; i += kThreads) {
        const double wi = v[i] + (i == 0 ? s0 : 0.0);
        w[i] = wi;
        acc += wi * wi;
    }
    return 2.0 / block_sum(acc, red);
}

// v = a / ||a|| with a max-scaling against overflow; false if a == 0
__device__ bool unit(const double* a, double* v, int len, double* red) {
    double m = 0.0;
    for (int i = threadIdx.x; i < len; i += kThreads) m = fmax(m, fabs(a[i]));
    m = block_max(m, red);
    if (!(m > 0.0)) return false;
    double acc = 0.0;
    for (int i = threadIdx.x; i < len; i += kThreads) {
        const double u = a[i] / m;
        v[i] = u;
        acc += u * u;
    }
    const double r = 1.0 / sqrt(block_sum(acc, red));
    for (int i = threadIdx.x; i < len; i += kThreads) v[i] *= r;
    __syncthreads();
    return true;
}

// map: per retried shift {input index l, column in X, column in B_sub, complex}
__global__ void __launch_bounds__(kThreads)
k_restart_trial(int n, int t, const int* __restrict__ map, const double* __restrict__ wr,
                const double* __restrict__ wi, const double* __restrict__ B, int ldb,
                double* __restrict__ wr_s, double* __restrict__ wi_s, double* __restrict__ Bs,
                double* __restrict__ scratch) {
    __shared__ double red[kThreads / 32];
    const int j = blockIdx.x;
    const int l = map[4 * j], uc = map[4 * j + 1], us = map[4 * j + 2], cplx = map[4 * j + 3];
    // per-block scratch: a1, a2, v1 (= w1), v2 (= w2), y: 5 n doubles
    double* a1 = scratch + (size_t)j * 5 * n;
    double* a2 = a1 + n;
    double* w1 = a2 + n;
    double* w2 = w1 + n;
    double* y = w2 + n;
    if (threadIdx.x == 0) {
        wr_s[j] = wr[l];
        wi_s[j] = wi[l];
    }
    for (int i = threadIdx.x; i < n; i += kThreads) {
        a1[i] = B ? B[i + (size_t)uc * ldb] : 1.0;  // the default start is a multiple of e
        a2[i] = (cplx && B) ? B[i + (size_t)(uc + 1) * ldb] : 0.0;
    }
    __syncthreads();
    double* out = Bs + (size_t)us * n;
    // the trial's position: column jc (0-based) of the orthogonal factor
    const int jc = n - t;
    bool ok1 = unit(a1, w1, n, red);
    if (!ok1 && cplx) {  // b_re = 0: the imaginary part leads
        for (int i = threadIdx.x; i < n; i += kThreads) {
            const double tmp = a1[i];
            a1[i] = a2[i];
            a2[i] = tmp;
        }
        __syncthreads();
        ok1 = unit(a1, w1, n, red);
    }
    if (!ok1) {
        // zero previous start: any unit vector is orthogonal to it
        for (int i = threadIdx.x; i < n; i += kThreads) out[i] = i == jc ? 1.0 : 0.0;
        if (cplx)
            for (int i = threadIdx.x; i < n; i += kThreads) out[i + n] = 0.0;
        return;
    }
    const double beta1 = householder(w1, w1, n, red);  // w1 in place of v1
    __syncthreads();
    // y = e_jc, or for a complex shift P2 e_jc (P2 on rows 1..n-1)
    for (int i = threadIdx.x; i < n; i += kThreads) y[i] = i == jc ? 1.0 : 0.0;
    __syncthreads();
    if (cplx) {
        // u = P1 a2; P2 from u(1:n-1) unless a2 lies in span(a1)
        double acc = 0.0;
        for (int i = threadIdx.x; i < n; i += kThreads) acc += w1[i] * a2[i];
        const double d = beta1 * block_sum(acc, red);
        for (int i = threadIdx.x; i < n; i += kThreads) a2[i] -= d * w1[i];
        __syncthreads();
        double m = 0.0, ma = 0.0;
        for (int i = threadIdx.x; i < n; i += kThreads) {
            if (i > 0) m = fmax(m, fabs(a2[i]));
            ma = fmax(ma, fabs(a2[i]));
        }
        m = block_max(m, red);
        ma = block_max(ma, red);
        // the part of a2 outside span(a1) is numerically zero: P2 = I
        if (m > 0x1p-50 * ma && unit(a2 + 1, w2, n - 1, red)) {
            const double beta2 = householder(w2, w2, n - 1, red);
            __syncthreads();
            const double c = beta2 * w2[jc - 1];  // w2^T e_(jc-1)
            for (int i = threadIdx.x; i < n - 1; i += kThreads) y[i + 1] -= c * w2[i];
            __syncthreads();
        }
    }
    // trial = P1 y
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += kThreads) acc += w1[i] * y[i];
    const double d = beta1 * block_sum(acc, red);
    for (int i = threadIdx.x; i < n; i += kThreads) out[i] = y[i] - d * w1[i];
    if (cplx)
        for (int i = threadIdx.x; i < n; i += kThreads) out[i + n] = 0.0;
}

__global__ void __launch_bounds__(kThreads)
k_restart_scatter(int n, const int* __restrict__ map, const double* __restrict__ Xs,
                  const int* __restrict__ st_s, double* __restrict__ X, int ldx,
                  int* __restrict__ status) {
    const int j = blockIdx.x;
    if (st_s[j] != 0) return;
    const int l = map[4 * j], uc = map[4 * j + 1], us = map[4 * j + 2], cplx = map[4 * j + 3];
    const int nc = cplx ? 2 : 1;
    for (int c = 0; c < nc; ++c)
        for (int i = threadIdx.x; i < n; i += kThreads)
            X[i + (size_t)(uc + c) * ldx] = Xs[i + (size_t)(us + c) * n];
    if (threadIdx.x == 0) status[l] = 0;
}

}  // namespace

size_t restart_scratch_bytes(int n, int k) { return (size_t)k * 5 * n * sizeof(double); }

void launch_restart_trial(int n, int t, int k, const int* map, const double* wr, const double* wi,
                          const double* B, int ldb, double* wr_s, double* wi_s, double* Bs,
                          double* scratch, cudaStream_t s) {
    k_restart_trial<<<k, kThreads, 0, s>>>(n, t, map, wr, wi, B, ldb, wr_s, wi_s, Bs, scratch);
}

void launch_restart_scatter(int n, int k, const int* map, const double* Xs, const int* st_s,
                            double* X, int ldx, int* status, cudaStream_t s) {
    k_restart_scatter<<<k, kThreads, 0, s>>>(n, map, Xs, st_s, X, ldx, status);
}

}  // namespace hsein
