// z = Q0 x as a split-precision product on the BF16 tensor cores (the
// "precision" mode of the backtransform).  See ozaki.cuh for the number
// format.  Steps:
//   k_oz_rowmax     max |Q0(r,:)| per row (exponent of the row)
//   k_oz_split_rows Q0 -> kS BF16 digit matrices, k-contiguous rows
//   k_oz_split_cols X  -> kS BF16 digit matrices per column, with exponents
//   k_oz_gemm       the 28 digit-pair products (i + j < kS) on the 5th-gen
//                   tensor cores: TMA brings 32-wide K slices of all 7 digit
//                   matrices of both operands into shared memory (2 stages);
//                   one thread issues tcgen05.mma BF16 x BF16 -> FP32 into 7
//                   diagonal accumulators in TMEM (10 MMAs per K-step, each A
//                   digit against a run of B digits); epilogue warps fold the
//                   leading diagonals into exact int64 every 256 of K and
//                   recombine in FP64 once per output.
#include "common.cuh"
#include "ozaki.cuh"
#include "tc.cuh"

namespace hsein {
namespace {

using oz::kS;

constexpr int BM = 128, BN = 64, BK = 32, STAGES = 2;
constexpr int kABytes = kS * BM * BK * 2;             // one stage of A digits (7 x 8 KB)
constexpr int kBBytes = kS * BN * BK * 2;             // one stage of B digits (7 x 4 KB)
constexpr int kStageBytes = kABytes + kBBytes;
constexpr int kSmemBytes = STAGES * kStageBytes + 1024;  // + alignment slack
constexpr int kChunkBlocks = 256 / BK;  // exact FP32 span of diagonals 0..3 (4 x 256 x 2^14 <= 2^24)
constexpr int kTmemCols = 512;          // 7 diagonals x 64 columns, rounded to a power of two

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

// One K-step of the digit products, as MMAs of A digit i against the B digits
// j0 .. j0+nj-1.  The B digit matrices sit one after another in shared memory
// (64 rows each), so they form one operand with N = 64 nj, and its output
// columns land on the diagonal accumulators i+j0 .. i+j0+nj-1 directly.  The
// first six pieces touch only diagonals >= kTopDiag; they are issued before
// the epilogue has released diagonals 0..3 of the previous chunk.
struct Piece {
    int i, j0, nj;
};
constexpr int kPieces = 10, kLowPieces = 6;
__constant__ const Piece kPiece[kPieces] = {{0, 4, 3}, {1, 4, 2}, {2, 4, 1}, {4, 0, 3}, {5, 0, 2},
                                            {6, 0, 1}, {0, 0, 4}, {1, 0, 4}, {2, 0, 4}, {3, 0, 4}};
constexpr int kEpiWarps = 8;  // two per TMEM lane quarter, 32 columns each
constexpr int kThreads = 64 + 32 * kEpiWarps;

__global__ void __launch_bounds__(kThreads, 1)
k_oz_gemm(int n, int ncol, OzLayout o, const __grid_constant__ CUtensorMap mapA,
          const __grid_constant__ CUtensorMap mapB, const void* __restrict__ wsp,
          double* __restrict__ Z, int ldz, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], accf, acce, mdone;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;
    // 1024-byte aligned stage buffers (the swizzle atoms assume it)
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const char* wsb = static_cast<const char*>(wsp);
    const int* gE = reinterpret_cast<const int*>(wsb + o.off_E);
    const int* gF = reinterpret_cast<const int*>(wsb + o.off_F);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n0 = blockIdx.x * BN, m0 = blockIdx.y * BM;
    const int nK = o.Kp / BK;
    const int nchunks = (nK + kChunkBlocks - 1) / kChunkBlocks;

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(&accf, 1);
        tc::mbar_init(&acce, kEpiWarps);
        tc::mbar_init(&mdone, 1);
        abort_flag = 0;
        tc::mbar_fence_init();
    }
    if (warp == 1) tc::tmem_alloc(&tmem_slot, kTmemCols);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = tmem_slot;
    int last_kb[STAGES];  // producer: last K slice loaded into each stage
#pragma unroll
    for (int s = 0; s < STAGES; ++s) last_kb[s] = -1;

    if (warp == 0) {
        // ---- producer: TMA of the 7 digit matrices of A and B per K slice
        if (lane == 0) {
            for (int kb = 0; kb < nK && !abort_flag; ++kb) {
                const int s = kb % STAGES;
                if (kb >= STAGES && !tc::mbar_wait(&empty[s], ((kb / STAGES) - 1) & 1)) {
                    abort_flag = 1;
                    break;
                }
                unsigned char* st = smem + s * kStageBytes;
                tc::mbar_expect_tx(&full[s], kStageBytes);
                tc::tma_load_3d(st, &mapA, kb * BK, m0, 0, &full[s]);
                tc::tma_load_3d(st + kABytes, &mapB, kb * BK, n0, 0, &full[s]);
                last_kb[s] = kb;
            }
        }
    } else if (warp == 1) {
        // ---- MMA issue: 10 pieces x 2 K-steps per K slice
        if (lane == 0) {
            for (int kb = 0; kb < nK && !abort_flag; ++kb) {
                const int s = kb % STAGES, c = kb / kChunkBlocks;
                const bool chunk_start = kb % kChunkBlocks == 0;
                if (!tc::mbar_wait(&full[s], (kb / STAGES) & 1)) {
                    abort_flag = 1;
                    break;
                }
                tc::tc_fence_after();
                const uint32_t sa = tc::su32(smem + s * kStageBytes), sb = sa + kABytes;
                for (int p = 0; p < kPieces; ++p) {
                    if (p == kLowPieces && chunk_start && c > 0) {
                        // diagonals 0..3 restart: wait until the epilogue has read them
                        if (!tc::mbar_wait(&acce, (c - 1) & 1)) {
                            abort_flag = 1;
                            break;
                        }
                        tc::tc_fence_after();
                    }
                    const Piece pc = kPiece[p];
                    const uint32_t idesc = tc::idesc_bf16(BM, BN * pc.nj);
                    // the piece that zero-initialises its diagonals: {0,4,3} at
                    // the first slice, {0,0,4} at the first slice of each chunk
                    const bool init = pc.i == 0 && (pc.j0 == 0 ? chunk_start : kb == 0);
#pragma unroll
                    for (int ks = 0; ks < BK / 16; ++ks) {
                        const uint64_t da = tc::smem_desc(sa + pc.i * (BM * BK * 2) + ks * 32, 512, 4);
                        const uint64_t db = tc::smem_desc(sb + pc.j0 * (BN * BK * 2) + ks * 32, 512, 4);
                        tc::mma_bf16(tmem + (pc.i + pc.j0) * BN, da, db, idesc,
                                     (init && ks == 0) ? 0u : 1u);
                    }
                }
                if (abort_flag) break;
                tc::mma_commit(&empty[s]);
                if (kb % kChunkBlocks == kChunkBlocks - 1 || kb == nK - 1) tc::mma_commit(&accf);
            }
        }
    } else {
        // ---- epilogue: lane quarter q of TMEM = rows 32q .. 32q+31 of the
        // tile; half h of the 64 columns
        const int q = warp & 3, h = (warp - 2) >> 2;
        const int row = m0 + 32 * q + lane;
        const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16) + 32 * h;
        long long top[32];
#pragma unroll
        for (int c = 0; c < 32; ++c) top[c] = 0;
        bool ok = true;
        for (int c = 0; c < nchunks; ++c) {
            if (!__all_sync(0xffffffffu, tc::mbar_wait(&accf, c & 1))) {
                ok = false;
                abort_flag = 1;
                break;
            }
            tc::tc_fence_after();
#pragma unroll
            for (int d = 0; d < oz::kTopDiag; ++d) {
                uint32_t v[2][16];
                tc::tmem_ld16(tl + d * BN, v[0]);
                tc::tmem_ld16(tl + d * BN + 16, v[1]);
                tc::tmem_wait_ld();
#pragma unroll
                for (int t = 0; t < 32; ++t)
                    top[t] += (long long)__float2int_rn(__uint_as_float(v[t >> 4][t & 15]))
                              << (8 * (oz::kTopDiag - 1 - d));
            }
            tc::tc_fence_before();
            __syncwarp();
            if (c + 1 < nchunks && lane == 0) tc::mbar_arrive(&acce);
        }
        if (ok) {
            // the remaining diagonals (FP32 over all of K) and the recombination
            // 2^(E+F-14) (top 2^-24 + S4 2^-32 + S5 2^-40 + S6 2^-48)
            const int er = row < n ? gE[row] : 0;
#pragma unroll
            for (int c0 = 0; c0 < 32; c0 += 16) {
                uint32_t v4[16], v5[16], v6[16];
                tc::tmem_ld16(tl + 4 * BN + c0, v4);
                tc::tmem_ld16(tl + 5 * BN + c0, v5);
                tc::tmem_ld16(tl + 6 * BN + c0, v6);
                tc::tmem_wait_ld();
#pragma unroll
                for (int t = 0; t < 16; ++t) {
                    const int col = n0 + 32 * h + c0 + t;
                    if (row < n && col < ncol) {
                        double v = (double)top[c0 + t] * 0x1p-24;
                        v = fma((double)__uint_as_float(v4[t]), 0x1p-32, v);
                        v = fma((double)__uint_as_float(v5[t]), 0x1p-40, v);
                        v = fma((double)__uint_as_float(v6[t]), 0x1p-48, v);
                        Z[row + (size_t)col * ldz] = scalbn(v, er + gF[col] - 14);
                    }
                }
            }
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 1 && lane == 0) {
        // every MMA this thread issued has retired before TMEM is released
        tc::mma_commit(&mdone);
        if (!tc::mbar_wait(&mdone, 0)) abort_flag = 1;
    }
    if (warp == 0 && lane == 0 && abort_flag) {
        // after an abort, let the copies still in flight land (bounded wait)
#pragma unroll
        for (int s = 0; s < STAGES; ++s)
            if (last_kb[s] >= 0) tc::mbar_wait(&full[s], (last_kb[s] / STAGES) & 1);
    }
    __syncthreads();
    if (abort_flag && tid == 0) atomicMin(err, -5);  // reported as HSEIN_ECUDA
    if (warp == 1) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, kTmemCols);
    }
}

}  // namespace

size_t ozq0_workspace_bytes(int n, int ncol) { return oz_layout(n, ncol).total + 256; }

bool launch_ozaki_q0(int n, int ncol, const double* Q, int ldq, const double* X, int ldx,
                     double* Z, int ldz, void* ws, int* err, cudaStream_t s) {
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
    CUtensorMap mA, mB;
    const uint64_t dimA[3] = {(uint64_t)o.Kp, (uint64_t)o.Mp, (uint64_t)kS};
    const uint64_t strA[2] = {(uint64_t)o.Kp * 2, (uint64_t)o.Mp * o.Kp * 2};
    const uint32_t boxA[3] = {BK, BM, kS};
    const uint64_t dimB[3] = {(uint64_t)o.Kp, (uint64_t)o.Np, (uint64_t)kS};
    const uint64_t strB[2] = {(uint64_t)o.Kp * 2, (uint64_t)o.Np * o.Kp * 2};
    const uint32_t boxB[3] = {BK, BN, kS};
    if (!encode_bf16_map_3d(&mA, dA, dimA, strA, boxA, 64) ||
        !encode_bf16_map_3d(&mB, dB, dimB, strB, boxB, 64))
        return false;
    dim3 g2(o.Np / BN, o.Mp / BM);
    k_oz_gemm<<<g2, kThreads, kSmemBytes, s>>>(n, ncol, o, mA, mB, ws, Z, ldz, err);
    return true;
}

cudaError_t ozaki_configure() {
    return cudaFuncSetAttribute(k_oz_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
}

}  // namespace hsein
