// Split-precision variant of K3, the shared-H update (precision = 1, b_r = 64).
//
//  k_oz_split_h   once per solve: every block A_J = H(1:p0(J), J^-) the
//                 update of tile column J reads is cut into kS BF16 digit
//                 matrices with one power-of-two exponent per (row, J), so
//                 rows of different magnitude keep their own scale.
//  k_update_oz    A_J [Z'|W] from the digit products of A_J and of the
//                 [Z'|W] digits k_diag wrote (one exponent per product
//                 column), on the BF16 tensor cores (mma.sync m16n8k16,
//                 FP32 accumulation).  With K = b_r = 64 every diagonal sum
//                 stays below 2^24 (7 x 64 x 2^14), so all of them are exact
//                 integers; they are folded into two int64 and recombined in
//                 FP64 once per output.  The epilogue is that of the FP64
//                 k_update (eq. "robust-update" and the cross-over reduction
//                 of Alg. "tiled-reduction2").
#include "common.cuh"
#include "ozaki.cuh"

namespace hsein {
namespace {

using oz::kS;
constexpr int kBr = 64;  // tile height this path supports
constexpr int BM = 64, BN = 64;
constexpr int kTile = BM * kBr;  // bf16 elements of one digit tile (64 rows x 64 k)
constexpr int kSmem = 2 * kS * kTile * 2;

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

__device__ inline uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ inline void cp_async16_zfill(uint32_t dst, const void* src, bool valid) {
    int n = valid ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(n));
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
// 128-byte rows (64 bf16), 8 chunks of 16 bytes, XOR swizzle by row
__device__ inline uint32_t tile_off(int r, int c) { return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4)); }

// exact recombination: 2^(e-14) sum_d 2^(-8d) S_d from the exact FP32 sums
__device__ inline double combine(const float (&acc)[kS][2][2][4], int mt, int nt, int el, int e) {
    long long top = 0, low = 0;
#pragma unroll
    for (int d = 0; d < 4; ++d) top += (long long)__float2int_rn(acc[d][mt][nt][el]) * (1LL << (8 * (3 - d)));
#pragma unroll
    for (int d = 4; d < kS; ++d) low += (long long)__float2int_rn(acc[d][mt][nt][el]) * (1LL << (8 * (kS - 1 - d)));
    double v = fma((double)low, 0x1p-24, (double)top);  // in units of 2^-24 of the top
    return scalbn(v, e - 14 - 24);
}

__global__ void __launch_bounds__(256, 1)
k_update_oz(Layout L, void* work, int J) {
    extern __shared__ __align__(128) unsigned char smem[];
    const DevState* st = ws<DevState>(work, L.off_state);
    if (st->status < 0) return;
    const int p0 = tile_start(L, J);
    const int r0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 1, wn = warp >> 1;
    const size_t P = (size_t)(J - 1) * L.b0 + (size_t)kBr * (J - 1) * (J - 2) / 2;
    const __nv_bfloat16* hd = ws<__nv_bfloat16>(work, L.off_hd) + kS * kBr * P;
    const int* he = ws<int>(work, L.off_he) + P;
    const __nv_bfloat16* zd = ws<__nv_bfloat16>(work, L.off_zwd);
    const int* zf = ws<int>(work, L.off_zwf);
    const int ncz = 2 * L.ncolp;
    const uint32_t sA = smem_u32(smem), sB = sA + kS * kTile * 2;
    for (int idx = tid; idx < 2 * kS * 64 * 8; idx += 256) {
        int c = idx & 7, r = (idx >> 3) & 63, t = idx >> 9;  // t in [0, 2 kS)
        if (t < kS) {
            bool ok = r0 + r < p0;
            const __nv_bfloat16* src = hd + ((size_t)t * p0 + (ok ? r0 + r : 0)) * kBr + 8 * c;
            cp_async16_zfill(sA + t * kTile * 2 + tile_off(r, c), src, ok);
        } else {
            int i = t - kS;
            const __nv_bfloat16* src = zd + ((size_t)i * ncz + n0 + r) * kBr + 8 * c;
            cp_async16_zfill(sB + i * kTile * 2 + tile_off(r, c), src, true);
        }
    }
    asm volatile("cp.async.commit_group;\n" ::);
    asm volatile("cp.async.wait_group 0;\n" ::);
    __syncthreads();

    float acc[kS][2][2][4];
#pragma unroll
    for (int d = 0; d < kS; ++d)
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[d][a][b][e] = 0.f;
#pragma unroll
    for (int kk = 0; kk < kBr; kk += 16) {
#pragma unroll
        for (int i = 0; i < kS; ++i) {
            uint32_t af[2][4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                int mi = lane >> 3;
                int r = wm * 32 + mt * 16 + (mi & 1) * 8 + (lane & 7);
                int c = (kk >> 3) + (mi >> 1);
                ldsm_x4(sA + i * kTile * 2 + tile_off(r, c), af[mt][0], af[mt][1], af[mt][2], af[mt][3]);
            }
#pragma unroll
            for (int j = 0; j < kS - i; ++j) {
                uint32_t b0, b1, b2, b3;
                int mi = lane >> 3;
                int r = wn * 16 + (mi >> 1) * 8 + (lane & 7);
                int c = (kk >> 3) + (mi & 1);
                ldsm_x4(sB + j * kTile * 2 + tile_off(r, c), b0, b1, b2, b3);
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    mma_bf16(acc[i + j][mt][0], af[mt], b0, b1);
                    mma_bf16(acc[i + j][mt][1], af[mt], b2, b3);
                }
            }
        }
    }

    // ---------------- epilogue (as in k_update) ---------------------------
    const Epi* epi = ws<Epi>(work, L.off_epi);
    double* X = ws<double>(work, L.off_X);
    double* R = ws<double>(work, L.off_R);
    const int g = lane >> 2, t4 = lane & 3;
    double mb[2] = {0.0, 0.0}, mr[2] = {0.0, 0.0};  // per n-tile
    double nb[2][2][2], nr[2][2][2];                // [mt][nt][row half]
    int gis[2][2];
    // phase A: all loads and arithmetic
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
        const int gc = n0 + wn * 16 + nt * 8 + 2 * t4;  // product column of Z'
        const int sc = gc >> 1;                          // solution column
        const bool valid_col = sc < L.ncol;
        const bool cplx = sc < 2 * L.mc;
        const int q = cplx ? (sc >> 1) : L.mc + (sc - 2 * L.mc);
        const bool is_im = cplx && (sc & 1);
        const int scre = cplx ? (sc & ~1) : sc;
        Epi E;
        if (valid_col) E = epi[q];
        const int fz = zf[gc], fw = zf[gc + 1];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int row = wm * 32 + mt * 16 + g + 8 * h;
                const int gi = r0 + row;
                gis[mt][h] = gi;
                nb[mt][nt][h] = 0.0;
                nr[mt][nt][h] = 0.0;
                if (!(valid_col && gi < p0)) continue;
                const int ea = he[gi];
                const double az = combine(acc, mt, nt, 2 * h, ea + fz);
                const double aw = combine(acc, mt, nt, 2 * h + 1, ea + fw);
                const bool last = gi == p0 - 1;
                const double b_ = X[gi + (size_t)sc * L.ldw];
                if (cplx) {
                    const double ur = R[gi + (size_t)scre * L.ldw];
                    const double ui = R[gi + (size_t)(scre + 1) * L.ldw];
                    const double u = is_im ? ui : ur;
                    // z_br (complex) times R~: re = ur zr - ui zi, im = ur zi + ui zr
                    double rz = is_im ? (ur * E.zbr_im + ui * E.zbr_re) : (ur * E.zbr_re - ui * E.zbr_im);
                    double vb = fma(b_, E.fB, -az) - rz;
                    double vr = fma(E.pi, u, aw);
                    if (last) {
                        vb += is_im ? E.cz_im : E.cz_re;
                        vr -= is_im ? E.cw_im : E.cw_re;
                    }
                    nb[mt][nt][h] = vb;
                    nr[mt][nt][h] = vr;
                } else {
                    const double u = R[gi + (size_t)sc * L.ldw];
                    double vb = fma(b_, E.fB, -az) - u * E.zbr_re;
                    double vr = fma(E.pi, u, aw);
                    if (last) {
                        vb += E.cz_re;
                        vr -= E.cw_re;
                    }
                    nb[mt][nt][h] = vb;
                    nr[mt][nt][h] = vr;
                }
                mb[nt] = fmax(mb[nt], fabs(nb[mt][nt][h]));
                mr[nt] = fmax(mr[nt], fabs(nr[mt][nt][h]));
            }
    }
    __syncwarp();  // every lane has read R~ before any lane overwrites it
    // phase B: stores
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
        const int sc = (n0 + wn * 16 + nt * 8 + 2 * t4) >> 1;
        if (sc >= L.ncol) continue;
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int gi = gis[mt][h];
                if (gi < p0) {
                    X[gi + (size_t)sc * L.ldw] = nb[mt][nt][h];
                    R[gi + (size_t)sc * L.ldw] = nr[mt][nt][h];
                }
            }
    }
    // per-shift maxima: over the 8 row groups of the warp, then the 2 row warps
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int o = 4; o < 32; o <<= 1) {
            mb[nt] = fmax(mb[nt], __shfl_xor_sync(0xffffffffu, mb[nt], o));
            mr[nt] = fmax(mr[nt], __shfl_xor_sync(0xffffffffu, mr[nt], o));
        }
    __syncthreads();
    double* red = reinterpret_cast<double*>(smem);  // [2 wm][2 kinds][32 solution cols]
    if (g == 0) {
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            int cl = wn * 8 + nt * 4 + t4;  // solution column within the tile (0..31)
            red[(wm * 2 + 0) * 32 + cl] = mb[nt];
            red[(wm * 2 + 1) * 32 + cl] = mr[nt];
        }
    }
    __syncthreads();
    if (tid < 64) {
        const int which = tid >> 5, cl = tid & 31;
        double v = fmax(red[(0 * 2 + which) * 32 + cl], red[(1 * 2 + which) * 32 + cl]);
        const int sc = (n0 >> 1) + cl;
        if (sc < L.ncol) {
            int q = sc < 2 * L.mc ? (sc >> 1) : L.mc + (sc - 2 * L.mc);
            unsigned long long* dst = ws<unsigned long long>(work, which ? L.off_rmax : L.off_bmax);
            atomic_max_nonneg(dst + q, v);
        }
    }
}

}  // namespace

size_t oz_update_hd_elems(const Layout& L) {
    const size_t Nm1 = (size_t)L.N;  // P(N) = sum over J = 1..N-1 of p0(J)
    size_t P = (Nm1 - 1) * L.b0 + (size_t)kBr * (Nm1 - 1) * (Nm1 - 2) / 2;
    if (L.N <= 1) P = 0;
    return P;
}

void launch_split_h(const Layout& L, void* work, const double* H, int ldh, cudaStream_t s) {
    if (L.N <= 1) return;
    dim3 grid((L.n + 31) / 32, L.N - 1);
    k_oz_split_h<<<grid, dim3(32, 8), 0, s>>>(L, work, H, ldh);
}

void launch_update_oz(const Layout& L, void* work, int J, cudaStream_t s) {
    const int p0 = tile_start(L, J);
    if (p0 <= 0) return;
    dim3 grid((p0 + BM - 1) / BM, (2 * L.ncolp) / BN);
    k_update_oz<<<grid, 256, kSmem, s>>>(L, work, J);
}

cudaError_t update_oz_configure() {
    return cudaFuncSetAttribute(k_update_oz, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
}

}  // namespace hsein
