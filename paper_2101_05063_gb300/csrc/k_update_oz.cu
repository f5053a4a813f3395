// Split-precision variant of K3, the shared-H update (precision = 1, b_r = 64).
//
//  k_oz_split_h   once per solve: every block A_J = H(1:p0(J), J^-) the
//                 update of tile column J reads is cut into kS BF16 digit
//                 matrices with one power-of-two exponent per (row, J), so
//                 rows of different magnitude keep their own scale.
//  k_update_oz    A_J [Z'|W] from the digit products of A_J and of the
//                 [Z'|W] digits k_diag wrote (one exponent per product
//                 column), on the 5th-generation tensor cores: TMA brings
//                 the seven 128 x 64 digit tiles of A_J into shared memory
//                 once per CTA and streams 32-column digit tiles of [Z'|W]
//                 through two stages; one thread issues tcgen05.mma (BF16 x
//                 BF16 -> FP32) into seven diagonal accumulators in TMEM,
//                 double-buffered so that the epilogue of one tile overlaps
//                 the products of the next.  With K = b_r = 64 every diagonal
//                 sum stays below 2^24 (7 x 64 x 2^14), so all of them are
//                 exact integers; they are folded into two int64 and
//                 recombined in FP64 once per output.  The epilogue is that
//                 of the FP64 k_update (the robust update of Sec. 3 and the
//                 cross-over reduction of the tiled algorithm).
#include "common.cuh"
#include "ozaki.cuh"
#include "tc.cuh"

#include <type_traits>

#include <algorithm>

namespace hsein {
namespace {

using oz::kS;
constexpr int kBr = 64;  // tile height this path supports
constexpr int TBM = 128;  // rows of A_J per tile (the TMEM lanes)
constexpr int TBN = 32;   // product columns per tile (16 solution columns)
constexpr int kABytes = kS * TBM * kBr * 2;  // seven 128 x 64 digit tiles of A_J
constexpr int kBBytes = kS * TBN * kBr * 2;  // seven 32 x 64 digit tiles of [Z'|W]
constexpr int kSmem = kABytes + 2 * kBBytes + 1024;  // + alignment slack
constexpr int kAccCols = 256;  // one accumulator set: 7 diagonals x 32 columns, padded
constexpr int kEpiWarps = 16;  // four per TMEM lane quarter, one 8-column group each
constexpr int kThreads = 64 + 32 * kEpiWarps;  // producer, MMA issuer, epilogue

__global__ void k_oz_split_h(Layout L, void* work, const double* __restrict__ H, int ldh) {
    const DevState* st = ws<DevState>(work, L.off_state);
    if (st->status < 0) return;
    const int J = blockIdx.y + 1;
    const int p0 = tile_start(L, J);
    const int r0 = blockIdx.x * 32;
    if (r0 >= p0) return;
    __nv_bfloat16* hd = ws<__nv_bfloat16>(work, L.off_hd);
    int* he = ws<int>(work, L.off_he);
    const size_t P = (size_t)(J - 1) * L.b0 + (size_t)kBr * (J - 1) * (J - 2) / 2;
    __shared__ __nv_bfloat16 sd[kS][32][kBr + 2];
    __shared__ double smax[8][32];
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    const int r = r0 + tx;
    const int c0 = p0 - 1;  // first column of J^-
    double m = 0.0;
    if (r < p0)
        for (int k = ty; k < kBr; k += 8) m = fmax(m, fabs(H[r + (size_t)(c0 + k) * ldh]));
    smax[ty][tx] = m;
    __syncthreads();
    double rm = 0.0;
#pragma unroll
    for (int t = 0; t < 8; ++t) rm = fmax(rm, smax[t][tx]);
    const int e = oz::scale_exponent(rm);
    if (ty == 0 && r < p0) he[P + r] = e;
    for (int k = ty; k < kBr; k += 8) {
        int d[kS];
        double a = r < p0 ? H[r + (size_t)(c0 + k) * ldh] : 0.0;
        oz::split_digits(a, e, d);
#pragma unroll
        for (int i = 0; i < kS; ++i) sd[i][tx][k] = __float2bfloat16_rn((float)d[i]);
    }
    __syncthreads();
    // write rows r0..r0+31 (k contiguous), digit-major inside block J
    for (int idx = ty * 32 + tx; idx < kS * 32 * (kBr / 2); idx += 256) {
        int kp = idx % (kBr / 2), rr = (idx / (kBr / 2)) % 32, i = idx / (32 * (kBr / 2));
        int gr = r0 + rr;
        if (gr < p0) {
            __nv_bfloat162 v;
            v.x = sd[i][rr][2 * kp];
            v.y = sd[i][rr][2 * kp + 1];
            *reinterpret_cast<__nv_bfloat162*>(hd + kS * kBr * P + ((size_t)i * p0 + gr) * kBr + 2 * kp) = v;
        }
    }
}


// RN(top + low 2^-24) 2^k from the two exact integer parts, built with
// integer operations only (GB300's FP64 pipe is the scarce resource of the
// epilogue).  |top| < 2^45 and |low| < 2^39, so V = top 2^24 + low has at
// most 70 bits.  While |top| < 2^38, V fits a 64-bit integer as it is;
// beyond, W = |V| >> 7 with the dropped bits OR-ed into its last bit (a
// rounding to odd with at least 55 bits, whose rounding to 53 bits is the
// rounding of V).  Results outside the normal range take scalbn.
__device__ inline double fixed_to_double(long long top, long long low, int k) {
    const bool big = (unsigned long long)(top + (1LL << 38)) >= (1ULL << 39);
    bool neg;
    unsigned long long M;
    int sh;
    if (!big) {
        const long long V = top * (1LL << 24) + low;
        neg = V < 0;
        M = (unsigned long long)(neg ? -V : V);
        sh = 0;
    } else {
        neg = top < 0;
        const long long t = neg ? -top : top, l = neg ? -low : low;  // |V| = t 2^24 + l
        M = (unsigned long long)(t * (1LL << 17) + (l >> 7)) | ((l & 127) != 0 ? 1ULL : 0ULL);
        sh = 7;
    }
    if (M == 0) return 0.0;
    const int lz = __clzll((long long)M);
    const unsigned long long Mn = M << lz;  // leading bit at 63
    unsigned long long mant = Mn >> 11;     // 53 bits
    const unsigned rb = (unsigned)(Mn & 0x7FF);
    if (rb > 0x400u || (rb == 0x400u && (mant & 1))) ++mant;  // to nearest, ties to even
    const int E = (63 - lz) + sh - 24 + k;  // value = (mant / 2^52) 2^E
    if (E >= -1022 && E <= 1022) {
        // the implicit bit of mant (or its carry to 2^53) lands in the exponent field
        const unsigned long long bits =
            ((unsigned long long)neg << 63) + ((unsigned long long)(E + 1022) << 52) + mant;
        return __longlong_as_double((long long)bits);
    }
    const double m = (double)mant;
    return scalbn(neg ? -m : m, E - 52);
}

// exact recombination of product column c from its seven diagonal sums
// (FP32 bit patterns read from TMEM): 2^(e-14) sum_d 2^(-8d) S_d.  With
// |S_d| <= (d+1) 64 2^14 the pairs S_0 256 + S_1, S_2 256 + S_3 and
// S_4 256 + S_5 fit in 32-bit integers.
__device__ inline double recombine(const uint32_t (&a)[kS][4], int c, int e) {
    int S[kS];
#pragma unroll
    for (int d = 0; d < kS; ++d) S[d] = __float2int_rn(__uint_as_float(a[d][c]));
    const int t1 = S[0] * 256 + S[1], t2 = S[2] * 256 + S[3], t3 = S[4] * 256 + S[5];
    const long long top = (long long)t1 * 65536 + t2;  // |top| < 2^45
    const long long low = (long long)t3 * 256 + S[6];  // |low| < 2^39
    return fixed_to_double(top, low, e - 14 - 24);
}

// an upper bound of |v| as the high word of its bit pattern, rounded up
// (orders like the magnitude; (bound << 32) reads back as a double >= |v|)
__device__ inline uint32_t mag_hi(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFULL;
    return (uint32_t)(b >> 32) + ((uint32_t)b != 0 ? 1u : 0u);
}

__host__ __device__ inline size_t hd_block(const Layout& L, int J) {
    // rows of all blocks A_1 .. A_{J-1} before block J
    return (size_t)(J - 1) * L.b0 + (size_t)kBr * (J - 1) * (J - 2) / 2;
}

// grid: x = 128-row tiles of A_J, y = groups of tiles_per_cta consecutive
// 32-column tiles of [Z'|W]
__global__ void __launch_bounds__(kThreads, 1)
k_update_oz(Layout L, void* work, int J, int tiles_per_cta, const __grid_constant__ CUtensorMap mapA,
            const __grid_constant__ CUtensorMap mapB) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t afull, bfull[2], bempty[2], tfull[2], tempty[2], mdone;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;
    DevState* st = ws<DevState>(work, L.off_state);
    if (st->status < 0) return;
    const int p0 = tile_start(L, J);
    const int m0 = blockIdx.x * TBM;
    const int t_begin = blockIdx.y * tiles_per_cta;
    const int ntl = min(2 * L.ncolp / TBN - t_begin, tiles_per_cta);
    if (ntl <= 0) return;
    unsigned char* sA = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    unsigned char* sB = sA + kABytes;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        tc::mbar_init(&afull, 1);
        for (int s = 0; s < 2; ++s) {
            tc::mbar_init(&bfull[s], 1);
            tc::mbar_init(&bempty[s], 1);
            tc::mbar_init(&tfull[s], 1);
            tc::mbar_init(&tempty[s], kEpiWarps);
        }
        tc::mbar_init(&mdone, 1);
        abort_flag = 0;
        tc::mbar_fence_init();
    }
    if (warp == 1) tc::tmem_alloc(&tmem_slot, 2 * kAccCols);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = tmem_slot;
    int last_t[2] = {-1, -1};  // producer: last tile loaded into each B stage

    if (warp == 0) {
        // ---- producer: A_J digits once, [Z'|W] digit tiles through two stages
        if (lane == 0) {
            tc::mbar_expect_tx(&afull, kABytes);
            tc::tma_load_3d(sA, &mapA, 0, m0, 0, &afull);
            for (int t = 0; t < ntl && !abort_flag; ++t) {
                const int s = t & 1;
                if (t >= 2 && !tc::mbar_wait(&bempty[s], ((t >> 1) - 1) & 1)) {
                    abort_flag = 1;
                    break;
                }
                tc::mbar_expect_tx(&bfull[s], kBBytes);
                tc::tma_load_3d(sB + s * kBBytes, &mapB, 0, (t_begin + t) * TBN, 0, &bfull[s]);
                last_t[s] = t;
            }
        }
    } else if (warp == 1) {
        // ---- MMA issue: A digit i against B digits 0..6-i in one MMA of
        // N = 32 (7 - i), written to the diagonal accumulators i .. 6
        if (lane == 0) {
            if (!tc::mbar_wait(&afull, 0)) abort_flag = 1;
            for (int t = 0; t < ntl && !abort_flag; ++t) {
                const int s = t & 1;
                if (!tc::mbar_wait(&bfull[s], (t >> 1) & 1) ||
                    (t >= 2 && !tc::mbar_wait(&tempty[s], ((t >> 1) - 1) & 1))) {
                    abort_flag = 1;
                    break;
                }
                tc::tc_fence_after();
                const uint32_t sa = tc::su32(sA), sb = tc::su32(sB + s * kBBytes);
#pragma unroll
                for (int i = 0; i < kS; ++i) {
                    const uint32_t idesc = tc::idesc_bf16(TBM, TBN * (kS - i));
#pragma unroll
                    for (int ks = 0; ks < kBr / 16; ++ks) {
                        const uint64_t da = tc::smem_desc(sa + i * (TBM * kBr * 2) + ks * 32, 1024, 2);
                        const uint64_t db = tc::smem_desc(sb + ks * 32, 1024, 2);
                        tc::mma_bf16(tmem + s * kAccCols + i * TBN, da, db, idesc,
                                     (i == 0 && ks == 0) ? 0u : 1u);
                    }
                }
                tc::mma_commit(&bempty[s]);
                tc::mma_commit(&tfull[s]);
            }
        }
    } else {
        // ---- epilogue: TMEM lane quarter q = rows 32q .. 32q+31 of the tile,
        // one row per thread; warp group g takes product columns 8g .. 8g+7
        // (4 solution columns).  The element-wise update is that of the FP64
        // k_update.
        const int q = warp & 3, g = (warp - 2) >> 2;
        const int gi = m0 + 32 * q + lane;
        const bool rv = gi < p0, last = gi == p0 - 1;
        const bool last_warp = m0 + 32 * q <= p0 - 1 && p0 - 1 < m0 + 32 * q + 32;
        const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16);
        const Epi* epi = ws<Epi>(work, L.off_epi);
        double* X = ws<double>(work, L.off_X);
        double* R = ws<double>(work, L.off_R);
        const int* zf = ws<int>(work, L.off_zwf);
        const int ea = rv ? ws<int>(work, L.off_he)[hd_block(L, J) + gi] : 0;
        unsigned long long* bmax = ws<unsigned long long>(work, L.off_bmax);
        unsigned long long* rmax = ws<unsigned long long>(work, L.off_rmax);
        const size_t ldw = L.ldw;
        for (int t = 0; t < ntl; ++t) {
            const int s = t & 1;
            const int gc = (t_begin + t) * TBN + 8 * g;  // first product column of the group
            const int sc = gc >> 1;                      // its first solution column
            // operands that do not depend on the products: issued before the wait
            int ez[8];
            {
                const int4 z0 = *reinterpret_cast<const int4*>(zf + gc);
                const int4 z1 = *reinterpret_cast<const int4*>(zf + gc + 4);
                ez[0] = ea + z0.x, ez[1] = ea + z0.y, ez[2] = ea + z0.z, ez[3] = ea + z0.w;
                ez[4] = ea + z1.x, ez[5] = ea + z1.y, ez[6] = ea + z1.z, ez[7] = ea + z1.w;
            }
            double xv[4], rv4[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const bool ok = rv && sc + k < L.ncol;
                const size_t ix = gi + (size_t)(sc + k) * ldw;
                xv[k] = ok ? X[ix] : 0.0;
                rv4[k] = ok ? R[ix] : 0.0;
            }
            if (lane < 2) {
                // the group's shift parameters (at most 4 consecutive entries)
                const int q0 = sc < 2 * L.mc ? (sc >> 1) : L.mc + (sc - 2 * L.mc);
                if (q0 < L.m) {
                    const char* pf = reinterpret_cast<const char*>(epi + q0) + 128 * lane;
                    asm volatile("prefetch.global.L1 [%0];\n" ::"l"(pf));
                }
            }
            if (!__all_sync(0xffffffffu, tc::mbar_wait(&tfull[s], (t >> 1) & 1))) {
                abort_flag = 1;
                break;
            }
            tc::tc_fence_after();
            uint32_t mb[4] = {0, 0, 0, 0}, mr[4] = {0, 0, 0, 0};
            // two halves of 4 product columns: one pair of solution columns
            // each.  The warp that holds row p0-1 runs its own instance with
            // that row's constant terms; every other warp runs none of them
            // (as selects they would cost every lane FP64 adds)
            auto halves = [&](auto LASTc) {
            constexpr bool LASTW = decltype(LASTc)::value;
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                uint32_t a[kS][4];
#pragma unroll
                for (int d = 0; d < kS; ++d)
                    tc::tmem_ld4(tl + s * kAccCols + d * TBN + 8 * g + 4 * u, a[d]);
                tc::tmem_wait_ld();
                if (u == 1) {
                    // this warp is done with the accumulator set
                    tc::tc_fence_before();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&tempty[s]);
                }
                double z[4];  // A_J Z' and A_J W of the pair, interleaved
#pragma unroll
                for (int c = 0; c < 4; ++c) z[c] = recombine(a, c, ez[4 * u + c]);
                const int sp = sc + 2 * u;  // even solution column of the pair
                if (!rv || sp >= L.ncol) continue;
                if (sp < 2 * L.mc) {
                    // complex pair (re, im) of one shift; z_br (complex) times R~
                    const Epi E = epi[sp >> 1];
                    const size_t ir = gi + (size_t)sp * ldw, ii = ir + ldw;
                    const double ur = rv4[2 * u], ui = rv4[2 * u + 1], br = xv[2 * u], bi = xv[2 * u + 1];
                    double vbr = fma(ui, E.zbr_im, fma(-ur, E.zbr_re, fma(br, E.fB, -z[0])));
                    double vbi = fma(-ui, E.zbr_re, fma(-ur, E.zbr_im, fma(bi, E.fB, -z[2])));
                    double vrr = fma(E.pi, ur, z[1]), vri = fma(E.pi, ui, z[3]);
                    if (LASTW && last) {
                        vbr += E.cz_re;
                        vbi += E.cz_im;
                        vrr -= E.cw_re;
                        vri -= E.cw_im;
                    }
                    X[ir] = vbr;
                    X[ii] = vbi;
                    R[ir] = vrr;
                    R[ii] = vri;
                    mb[2 * u] = mag_hi(vbr);
                    mb[2 * u + 1] = mag_hi(vbi);
                    mr[2 * u] = mag_hi(vrr);
                    mr[2 * u + 1] = mag_hi(vri);
                } else {
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        const int sk = sp + k;
                        if (sk >= L.ncol) break;
                        const Epi E = epi[L.mc + (sk - 2 * L.mc)];
                        const size_t ix = gi + (size_t)sk * ldw;
                        const double u_ = rv4[2 * u + k];
                        double vb = fma(-u_, E.zbr_re, fma(xv[2 * u + k], E.fB, -z[2 * k]));
                        double vr = fma(E.pi, u_, z[2 * k + 1]);
                        if (LASTW && last) {
                            vb += E.cz_re;
                            vr -= E.cw_re;
                        }
                        X[ix] = vb;
                        R[ix] = vr;
                        mb[2 * u + k] = mag_hi(vb);
                        mr[2 * u + k] = mag_hi(vr);
                    }
                }
            }
            };
            if (last_warp) halves(std::true_type{});
            else halves(std::false_type{});
            {
                // per-shift maxima over the warp's 32 rows; lanes 0..7 post them
                uint32_t mine = 0;
#pragma unroll
                for (int v = 0; v < 8; ++v) {
                    const uint32_t m = __reduce_max_sync(0xffffffffu, v < 4 ? mb[v] : mr[v - 4]);
                    if (lane == v) mine = m;
                }
                const int sv = sc + (lane & 3);
                if (lane < 8 && sv < L.ncol && mine != 0) {
                    const int qq = sv < 2 * L.mc ? (sv >> 1) : L.mc + (sv - 2 * L.mc);
                    atomicMax((lane >> 2 ? rmax : bmax) + qq, (unsigned long long)mine << 32);
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
        // after an abort, let the copies still in flight land (bounded waits)
        tc::mbar_wait(&afull, 0);
        for (int s = 0; s < 2; ++s)
            if (last_t[s] >= 0) tc::mbar_wait(&bfull[s], (last_t[s] >> 1) & 1);
    }
    __syncthreads();
    if (abort_flag && tid == 0) set_error(st, -5);  // HSEIN_ECUDA
    if (warp == 1) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, 2 * kAccCols);
    }
}

}  // namespace

size_t oz_update_hd_elems(const Layout& L) {
    // rows of all blocks A_1 .. A_{N-1}
    return L.N <= 1 ? 0 : hd_block(L, L.N);
}

void launch_split_h(const Layout& L, void* work, const double* H, int ldh, cudaStream_t s) {
    if (L.N <= 1) return;
    dim3 grid((L.n + 31) / 32, L.N - 1);
    k_oz_split_h<<<grid, dim3(32, 8), 0, s>>>(L, work, H, ldh);
}

bool encode_update_oz_maps(const Layout& L, void* work, CUtensorMap* mapsA, CUtensorMap* mapB) {
    const __nv_bfloat16* hd = ws<__nv_bfloat16>(work, L.off_hd);
    for (int J = 1; J < L.N; ++J) {
        const uint64_t p0 = (uint64_t)tile_start(L, J);
        const uint64_t dims[3] = {(uint64_t)kBr, p0, (uint64_t)kS};
        const uint64_t strides[2] = {(uint64_t)kBr * 2, p0 * kBr * 2};
        const uint32_t box[3] = {(uint32_t)kBr, (uint32_t)TBM, (uint32_t)kS};
        if (!encode_bf16_map_3d(&mapsA[J], hd + kS * kBr * hd_block(L, J), dims, strides, box, 128))
            return false;
    }
    const uint64_t ncz = 2 * (uint64_t)L.ncolp;
    const uint64_t dims[3] = {(uint64_t)kBr, ncz, (uint64_t)kS};
    const uint64_t strides[2] = {(uint64_t)kBr * 2, ncz * kBr * 2};
    const uint32_t box[3] = {(uint32_t)kBr, (uint32_t)TBN, (uint32_t)kS};
    return encode_bf16_map_3d(mapB, ws<__nv_bfloat16>(work, L.off_zwd), dims, strides, box, 128);
}

void launch_update_oz(const Layout& L, void* work, int J, int num_sms, const CUtensorMap& mapA,
                      const CUtensorMap& mapB, cudaStream_t s) {
    const int p0 = tile_start(L, J);
    if (p0 <= 0) return;
    // tiles per CTA: the fewest tile times for the busiest SM (one CTA per
    // SM at a time; each CTA also pays about one tile time to load A_J)
    const int mt = (p0 + TBM - 1) / TBM, nt = 2 * L.ncolp / TBN;
    int per = nt;
    long best = -1;
    for (int c = 1; c <= nt; ++c) {
        const long ctas = (long)mt * ((nt + c - 1) / c);
        const long cost = (ctas + num_sms - 1) / num_sms * (c + 1);
        if (best < 0 || cost < best) best = cost, per = c;
    }
    dim3 grid(mt, (nt + per - 1) / per);
    k_update_oz<<<grid, kThreads, kSmem, s>>>(L, work, J, per, mapA, mapB);
}

cudaError_t update_oz_configure() {
    return cudaFuncSetAttribute(k_update_oz, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
}

}  // namespace hsein
