// Measurement helper, outside the method: the rate of FP64 fused multiply-
// adds this GPU sustains on its CUDA cores, the denominator of the FP64
// rooflines.  Every thread runs eight independent FMA chains (enough
// independent work to cover the dependent-FMA latency on every SM
// sub-partition), and writes their sum so that nothing is optimized away.
#include "../../include/hsein.h"

#include <cuda_runtime.h>

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kThreads) k_fp64_rate(long long iters, double m, double c,
                                                        double* __restrict__ out) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    double a[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = 1.0 + (double)(t * kChains + j) * 0x1p-40;
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += a[j];
    out[t] = s;
}

}  // namespace

extern "C" hsein_status hsein_fp64_rate(long long iters, double* dOut, long long count,
                                        double* flops, void* stream) {
    if (iters < 1 || !dOut || count < kThreads || count % kThreads != 0 || count > (1LL << 31))
        return HSEIN_EARG;
    // a contraction towards c / (1 - m) = 1: values stay near 1, no
    // subnormals, no overflow, whatever the iteration count
    const double m = 0.5, c = 0.5;
    k_fp64_rate<<<(unsigned)(count / kThreads), kThreads, 0, static_cast<cudaStream_t>(stream)>>>(
        iters, m, c, dOut);
    if (cudaGetLastError() != cudaSuccess) return HSEIN_ECUDA;
    if (flops) *flops = 2.0 * kChains * (double)iters * (double)count;
    return HSEIN_OK;
}
