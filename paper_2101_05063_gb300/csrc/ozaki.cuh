// Split-precision (Ozaki-style) products on the BF16 tensor cores.
//
// A double a with a power-of-two scale 2^E (|a| < 2^E, one E per row of the
// left operand or per column of the right one) is written as
//     a = 2^E * sum_{i=0}^{S-1} d_i 2^(-7-8i),   d_i integer in [-128, 128],
// i.e. a 55-bit fixed-point integer cut into balanced base-256 digits.  Every
// digit is exact in BF16 (8 significant bits), so a digit-pair product summed
// over k is an exact integer as long as the FP32 accumulator stays below 2^24.
// A dot product is then
//     sum_k a_k b_k = 2^(E+F-14) sum_d 2^(-8d) S_d,   S_d = sum_k sum_{i+j=d} d_i d'_j,
// and the pairs with i + j >= S are dropped (their weight is below the FP64
// rounding level).  S_0..S_3 are converted exactly to a 64-bit integer every
// kKc values of k (4 products x 128 x 2^14 < 2^24); S_4..S_6 stay in FP32,
// whose relative rounding there is below 2^-53 of the result.
//
// The splitting uses integer operations on the bit pattern only, so it does
// not load GB300's FP64 pipe.
#pragma once

#include <cuda_bf16.h>
#include <cstdint>

namespace hsein {
namespace oz {

constexpr int kS = 7;      // digits per value (7 + 8*6 = 55 bits)
constexpr int kKc = 128;   // exact FP32 chunk for diagonals 0..3
constexpr int kTopDiag = 4;

// exponent E with |v| < 2^E for the largest magnitude v of a row/column
// (0 for an all-zero vector)
__device__ inline int scale_exponent(double vmax) {
    if (!(vmax > 0.0)) return 0;
    return ilogb(vmax) + 1;
}

// the kS balanced digits of a relative to 2^E (|a| < 2^E), most significant first
__device__ inline void split_digits(double a, int E, int* d) {
    long long bits = __double_as_longlong(a);
    int ea = (int)((bits >> 52) & 0x7FF);
    long long mant = bits & ((1LL << 52) - 1);
    if (ea != 0) mant |= (1LL << 52);
    int eff = ea != 0 ? ea : 1;
    // V = round(|a| 2^(55 - E)) = round(mant 2^(eff - 1075 - E + 55))
    int sh = eff - 1075 - E + 55;
    long long V;
    if (mant == 0) {
        V = 0;
    } else if (sh >= 0) {
        V = mant << sh;  // sh <= 2 because |a| < 2^E
    } else if (sh > -63) {
        V = (mant + (1LL << (-sh - 1))) >> (-sh);
    } else {
        V = 0;
    }
    if (bits < 0) V = -V;
#pragma unroll
    for (int i = kS - 1; i >= 1; --i) {
        int di = (int)((V + 128) & 255) - 128;
        d[i] = di;
        V = (V - di) >> 8;
    }
    d[0] = (int)V;
}

}  // namespace oz

// host launchers
size_t ozq0_workspace_bytes(int n, int ncol);
// false if the TMA tensor maps could not be encoded; a device-side abort
// (a wait that timed out) lowers *err to -5
bool launch_ozaki_q0(int n, int ncol, const double* Q, int ldq, const double* X, int ldx,
                     double* Z, int ldz, void* ws, int* err, cudaStream_t s);
cudaError_t ozaki_configure();

}  // namespace hsein
