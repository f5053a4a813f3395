// z = Q0 x as a split-precision product on the BF16 tensor cores (the
// "precision" mode of the backtransform).  See ozaki.cuh for the number
// format.  Steps:
//   k_oz_rowmax     max |Q0(r,:)| per row (exponent of the row)
//   k_oz_split_rows Q0 -> kS BF16 digit matrices, k-contiguous rows
//   k_oz_split_cols X  -> kS BF16 digit matrices per column, with exponents
//   k_oz_gemm       the 28 digit-pair products (i + j < kS) with mma.sync
//                   m16n8k16 BF16 -> FP32, exact integer accumulation of the
//                   leading diagonals, FP64 recombination once per output.
#include "common.cuh"
#include "ozaki.cuh"

namespace hsein {
namespace {

using oz::kKc;
using oz::kS;

constexpr int BM = 64, BN = 64, BK = 32, STAGES = 3;
constexpr int kTileElems = BM * BK;                 // per digit matrix, per operand
constexpr int kStageBytes = 2 * kS * kTileElems * 2;  // A and B, kS digits, bf16
constexpr int kSmemBytes = STAGES * kStageBytes;

struct OzLayout {
    int Mp, Np, Kp;
    size_t off_A, off_B, off_E, off_F, off_rmax, total;
};

__host__ __device__ inline OzLayout oz_layout(int n, int ncol) {
    OzLayout o;
    o.Mp = (n + BM - 1) / BM * BM;
    o.Np = (ncol + BN - 1) / BN * BN;
    o.Kp = (n + BK - 1) / BK * BK;
    size_t off = 0;
    auto take = [&](size_t b) {
        size_t at = off;
        off = (off + b + 255) & ~(size_t)255;
        return at;
    };
    o.off_A = take((size_t)kS * o.Mp * o.Kp * 2);
    o.off_B = take((size_t)kS * o.Np * o.Kp * 2);
    o.off_E = take((size_t)o.Mp * 4);
    o.off_F = take((size_t)o.Np * 4);
    o.off_rmax = take((size_t)o.Mp * 8);
    o.total = off;
    return o;
}

__global__ void k_oz_rowmax(int n, int K, const double* __restrict__ A, int lda,
                            unsigned long long* __restrict__ rmax) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int k0 = blockIdx.y * 256, k1 = min(K, k0 + 256);
    if (r >= n) return;
    double m = 0.0;
    for (int k = k0; k < k1; ++k) m = fmax(m, fabs(A[r + (size_t)k * lda]));
    atomic_max_nonneg(rmax + r, m);
}

// Q0 (n x K, column-major) -> digits [kS][Mp][Kp]; tile 32 rows x 32 k
__global__ void k_oz_split_rows(int n, int K, const double* __restrict__ A, int lda,
                                const unsigned long long* __restrict__ rmax, int* __restrict__ E,
                                __nv_bfloat16* __restrict__ dig, int Mp, int Kp) {
    __shared__ __nv_bfloat16 sd[kS][32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    const int r0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
    const int r = r0 + tx;
    int e = 0;
    if (r < n) e = oz::scale_exponent(bits_to_double(rmax[r]));
    if (r < Mp && blockIdx.y == 0 && ty == 0) E[r] = e;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        int kk = ty + 8 * j, k = k0 + kk;
        int d[kS];
        double a = (r < n && k < K) ? A[r + (size_t)k * lda] : 0.0;
        oz::split_digits(a, e, d);
#pragma unroll
        for (int i = 0; i < kS; ++i) sd[i][tx][kk] = __float2bfloat16_rn((float)d[i]);
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        int rr = ty + 8 * j;
#pragma unroll
        for (int i = 0; i < kS; ++i)
            dig[((size_t)i * Mp + r0 + rr) * Kp + k0 + tx] = sd[i][rr][tx];
    }
}

// X (K x N, column-major) -> digits [kS][Np][Kp] and column exponents
__global__ void k_oz_split_cols(int K, int N, const double* __restrict__ B, int ldb,
                                int* __restrict__ F, __nv_bfloat16* __restrict__ dig, int Np,
                                int Kp) {
    const int c = blockIdx.x;
    __shared__ double red[32];
    double m = 0.0;
    if (c < N)
        for (int k = threadIdx.x; k < K; k += blockDim.x) m = fmax(m, fabs(B[k + (size_t)c * ldb]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (threadIdx.x == 0) red[0] = v;
    }
    __syncthreads();
    const int e = oz::scale_exponent(red[0]);
    if (threadIdx.x == 0) F[c] = e;
    for (int k = threadIdx.x; k < Kp; k += blockDim.x) {
        int d[kS];
        double b = (c < N && k < K) ? B[k + (size_t)c * ldb] : 0.0;
        oz::split_digits(b, e, d);
#pragma unroll
        for (int i = 0; i < kS; ++i)
            dig[((size_t)i * Np + c) * Kp + k] = __float2bfloat16_rn((float)d[i]);
    }
}

__device__ inline uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ inline void cp_async16(uint32_t dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src));
}

__device__ inline void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2,
                               uint32_t& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ inline void mma_bf16(float* c, const uint32_t* a, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// byte offset of 16-byte chunk c of row r inside a [rows][BK] bf16 tile
// (64-byte rows; XOR swizzle keeps ldmatrix conflict-free)
__device__ inline uint32_t tile_off(int r, int c) {
    return (uint32_t)(r * 64 + ((c ^ ((r >> 1) & 3)) << 4));
}

__global__ void __launch_bounds__(256, 1)
k_oz_gemm(int n, int ncol, OzLayout o, const void* __restrict__ wsp, double* __restrict__ Z,
          int ldz) {
    extern __shared__ __align__(128) unsigned char smem[];
    const char* wsb = static_cast<const char*>(wsp);
    const __nv_bfloat16* gA = reinterpret_cast<const __nv_bfloat16*>(wsb + o.off_A);
    const __nv_bfloat16* gB = reinterpret_cast<const __nv_bfloat16*>(wsb + o.off_B);
    const int* gE = reinterpret_cast<const int*>(wsb + o.off_E);
    const int* gF = reinterpret_cast<const int*>(wsb + o.off_F);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n0 = blockIdx.x * BN, m0 = blockIdx.y * BM;
    const int wm = warp & 1, wn = warp >> 1;  // warp tile 32 rows x 16 cols
    const uint32_t sbase = smem_u32(smem);
    const int nK = o.Kp / BK;

    auto load_stage = [&](int stage, int kt) {
        const uint32_t st = sbase + stage * kStageBytes;
        const int k0 = kt * BK;
        // A: kS x 64 rows x 4 chunks; B: kS x 64 rows x 4 chunks
        for (int idx = tid; idx < 2 * kS * 64 * 4; idx += 256) {
            int c = idx & 3, r = (idx >> 2) & 63, t = idx >> 8;  // t in [0, 2 kS)
            int i = t % kS;
            bool isB = t >= kS;
            const __nv_bfloat16* src =
                isB ? gB + ((size_t)i * o.Np + n0 + r) * o.Kp + k0 + 8 * c
                    : gA + ((size_t)i * o.Mp + m0 + r) * o.Kp + k0 + 8 * c;
            uint32_t dst = st + (isB ? kS * kTileElems * 2 : 0) + i * kTileElems * 2 + tile_off(r, c);
            cp_async16(dst, src);
        }
    };

    float acc[kS][2][2][4];
    long long top[2][2][4];
#pragma unroll
    for (int d = 0; d < kS; ++d)
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[d][a][b][e] = 0.f;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int e = 0; e < 4; ++e) top[a][b][e] = 0;

    auto flush_top = [&]() {
#pragma unroll
        for (int d = 0; d < oz::kTopDiag; ++d)
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int b = 0; b < 2; ++b)
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        top[a][b][e] += (long long)__float2int_rn(acc[d][a][b][e]) * (1LL << (8 * (oz::kTopDiag - 1 - d)));
                        acc[d][a][b][e] = 0.f;
                    }
    };

#pragma unroll
    for (int s = 0; s < STAGES - 1; ++s) {
        if (s < nK) load_stage(s, s);
        asm volatile("cp.async.commit_group;\n" ::);
    }
    const int chunk_steps = kKc / BK;
    for (int kt = 0; kt < nK; ++kt) {
        asm volatile("cp.async.wait_group %0;\n" ::"n"(STAGES - 2));
        __syncthreads();
        const uint32_t st = sbase + (kt % STAGES) * kStageBytes;
        const uint32_t sA = st, sB = st + kS * kTileElems * 2;
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
#pragma unroll
            for (int i = 0; i < kS; ++i) {
                uint32_t af[2][4];
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    int mi = lane >> 3;
                    int r = wm * 32 + mt * 16 + (mi & 1) * 8 + (lane & 7);
                    int c = (kk >> 3) + (mi >> 1);
                    ldsm_x4(sA + i * kTileElems * 2 + tile_off(r, c), af[mt][0], af[mt][1], af[mt][2],
                            af[mt][3]);
                }
#pragma unroll
                for (int j = 0; j < kS - i; ++j) {
                    uint32_t b0, b1, b2, b3;
                    int mi = lane >> 3;
                    int r = wn * 16 + (mi >> 1) * 8 + (lane & 7);
                    int c = (kk >> 3) + (mi & 1);
                    ldsm_x4(sB + j * kTileElems * 2 + tile_off(r, c), b0, b1, b2, b3);
#pragma unroll
                    for (int mt = 0; mt < 2; ++mt) {
                        mma_bf16(acc[i + j][mt][0], af[mt], b0, b1);
                        mma_bf16(acc[i + j][mt][1], af[mt], b2, b3);
                    }
                }
            }
        }
        const int nxt = kt + STAGES - 1;
        if (nxt < nK) load_stage(nxt % STAGES, nxt);
        asm volatile("cp.async.commit_group;\n" ::);
        if ((kt + 1) % chunk_steps == 0) flush_top();
    }
    if (nK % chunk_steps != 0) flush_top();
    asm volatile("cp.async.wait_group 0;\n" ::);

    // recombination: 2^(E+F-14) (top 2^-24 + S4 2^-32 + S5 2^-40 + S6 2^-48)
    const int g = lane >> 2, t4 = lane & 3;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int r = m0 + wm * 32 + mt * 16 + g + ((e >> 1) << 3);
                const int c = n0 + wn * 16 + nt * 8 + 2 * t4 + (e & 1);
                if (r < n && c < ncol) {
                    double v = (double)top[mt][nt][e] * 0x1p-24;
                    v = fma((double)acc[4][mt][nt][e], 0x1p-32, v);
                    v = fma((double)acc[5][mt][nt][e], 0x1p-40, v);
                    v = fma((double)acc[6][mt][nt][e], 0x1p-48, v);
                    Z[r + (size_t)c * ldz] = scalbn(v, gE[r] + gF[c] - 14);
                }
            }
}

}  // namespace

size_t ozq0_workspace_bytes(int n, int ncol) { return oz_layout(n, ncol).total; }

void launch_ozaki_q0(int n, int ncol, const double* Q, int ldq, const double* X, int ldx,
                     double* Z, int ldz, void* ws, cudaStream_t s) {
    const OzLayout o = oz_layout(n, ncol);
    char* w = static_cast<char*>(ws);
    unsigned long long* rmax = reinterpret_cast<unsigned long long*>(w + o.off_rmax);
    int* E = reinterpret_cast<int*>(w + o.off_E);
    int* F = reinterpret_cast<int*>(w + o.off_F);
    __nv_bfloat16* dA = reinterpret_cast<__nv_bfloat16*>(w + o.off_A);
    __nv_bfloat16* dB = reinterpret_cast<__nv_bfloat16*>(w + o.off_B);
    cudaMemsetAsync(rmax, 0, (size_t)o.Mp * 8, s);
    dim3 g0((n + 127) / 128, (n + 255) / 256);
    k_oz_rowmax<<<g0, 128, 0, s>>>(n, n, Q, ldq, rmax);
    dim3 g1(o.Mp / 32, o.Kp / 32);
    k_oz_split_rows<<<g1, dim3(32, 8), 0, s>>>(n, n, Q, ldq, rmax, E, dA, o.Mp, o.Kp);
    k_oz_split_cols<<<o.Np, 256, 0, s>>>(n, ncol, X, ldx, F, dB, o.Np, o.Kp);
    dim3 g2(o.Np / BN, o.Mp / BM);
    k_oz_gemm<<<g2, 256, kSmemBytes, s>>>(n, ncol, o, ws, Z, ldz);
}

cudaError_t ozaki_configure() {
    return cudaFuncSetAttribute(k_oz_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
}

}  // namespace hsein
