// K5: z = Q0 x for every solution column (Sec. 1: H = Q0^T A Q0, so an
// eigenvector x of H gives the eigenvector Q0 x of A).  A plain FP64 product
// Z = Q0 X (n x n times n x ncol); complex shifts are two real columns.
//
// FP64 path: CUDA-core DFMA.  CTA tile 64 x 64, K step 16, 16 x 16 threads,
// each 4 consecutive rows x 4 consecutive columns; the next K step is
// prefetched into registers while the current one is multiplied.
#include "common.cuh"

namespace hsein {
namespace {

constexpr int kTM = 64, kTN = 64, kTK = 16;

__global__ void __launch_bounds__(256)
k_q0(int n, int ncol, const double* __restrict__ Q, int ldq, const double* __restrict__ X,
     int ldx, double* __restrict__ Z, int ldz) {
    __shared__ __align__(16) double As[2][kTK][kTM];
    __shared__ __align__(16) double Bs[2][kTK][kTN];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int r0 = blockIdx.x * kTM, c0 = blockIdx.y * kTN;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    // each thread loads 4 A values (rows r, k) and 4 B values (k, cols)
    double ra[4], rb[4];
    auto load = [&](int k0) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            int idx = tid + 256 * u;  // 0..1023
            int kk = idx / kTM, r = idx % kTM;
            int gi = r0 + r, gk = k0 + kk;
            ra[u] = (gi < n && gk < n) ? Q[gi + (size_t)gk * ldq] : 0.0;
            int c = idx / kTK, k2 = idx % kTK;
            int gc = c0 + c, gk2 = k0 + k2;
            rb[u] = (gc < ncol && gk2 < n) ? X[gk2 + (size_t)gc * ldx] : 0.0;
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            int idx = tid + 256 * u;
            As[buf][idx / kTM][idx % kTM] = ra[u];
            Bs[buf][idx % kTK][idx / kTK] = rb[u];
        }
    };
    int nk = (n + kTK - 1) / kTK;
    load(0);
    store(0);
    __syncthreads();
    for (int t = 0; t < nk; ++t) {
        const int buf = t & 1;
        if (t + 1 < nk) load((t + 1) * kTK);
#pragma unroll
        for (int kk = 0; kk < kTK; ++kk) {
            const double2 a01 = *reinterpret_cast<const double2*>(&As[buf][kk][4 * ty]);
            const double2 a23 = *reinterpret_cast<const double2*>(&As[buf][kk][4 * ty + 2]);
            const double2 b01 = *reinterpret_cast<const double2*>(&Bs[buf][kk][4 * tx]);
            const double2 b23 = *reinterpret_cast<const double2*>(&Bs[buf][kk][4 * tx + 2]);
            const double av[4] = {a01.x, a01.y, a23.x, a23.y};
            const double bv[4] = {b01.x, b01.y, b23.x, b23.y};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
        }
        if (t + 1 < nk) store(buf ^ 1);
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        int gc = c0 + 4 * tx + j;
        if (gc >= ncol) continue;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int gi = r0 + 4 * ty + i;
            if (gi < n) Z[gi + (size_t)gc * ldz] = acc[i][j];
        }
    }
}

}  // namespace

void launch_q0(const Layout& L, const double* Q, int ldq, const double* X, int ldx, double* Z,
               int ldz, cudaStream_t s) {
    dim3 grid((L.n + kTM - 1) / kTM, (L.ncol + kTN - 1) / kTN);
    k_q0<<<grid, 256, 0, s>>>(L.n, L.ncol, Q, ldq, X, ldx, Z, ldz);
}

}  // namespace hsein
