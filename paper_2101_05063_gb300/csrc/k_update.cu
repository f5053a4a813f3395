// K3: the shared-H update of all rows above diagonal tile J, for every shift.
//
// With A = H(1:p0, J^-) (columns p0-1 .. p0+bt-2, shared by all shifts) and
// the per-shift operand [Z'|W] built by k_diag, one product A [Z'|W] serves
// both the back-substitution update of eq. "update" / Alg. "tile-update"
// (B -= A Z' + R~ z_br - lambda rho' e_last, with the robust rescaling of
// eq. "robust-update") and the reduction of the cross-over column of Alg.
// "tiled-reduction2" (R~ = A W + pi R~ - lambda c_0 e_last).  Columns of the
// product come in pairs (Z', W) per solution column, so the thread that owns
// a solution column owns both and reads R~ once.  Complex shifts own two
// solution columns [re, im] (Sec. 4.3): real H times a complex z is a real
// product with two columns.
//
// The epilogue also emits max |B(1:p0, q)| and max |R~(1:p0, q)| per shift,
// the bounds the next tile's ProtectUpdate needs.
//
// This is the FP64 path: CUDA-core DFMA (GB300's FP64 tensor rate is no
// higher than its DFMA rate).  CTA tile 64 rows x 64 product columns,
// 16 x 16 threads, each 4 consecutive rows x 4 consecutive columns.
#include "common.cuh"

namespace hsein {
namespace {

constexpr int kTM = 64, kTN = 64;

__global__ void __launch_bounds__(256)
k_update(Layout L, void* work, const double* __restrict__ H, int ldh, int J) {
    extern __shared__ __align__(16) double smem[];
    const DevState* st = ws<DevState>(work, L.off_state);
    if (st->status < 0) return;
    const int p0 = tile_start(L, J);
    const int bt = tile_height(L, J);
    const int r0 = blockIdx.x * kTM;
    const int c0 = blockIdx.y * kTN;
    const size_t ldzw = 2 * (size_t)L.ncolp;
    const double* ZW = ws<double>(work, L.off_ZW);
    double* As = smem;                    // [bt][64] rows of A, k-major
    double* Bs = smem + (size_t)bt * kTM;  // [bt][64]
    const int tid = threadIdx.x;
    for (int idx = tid; idx < bt * kTM; idx += 256) {
        int kk = idx / kTM, r = idx % kTM;
        int gi = r0 + r;
        As[idx] = gi < p0 ? H[gi + (size_t)(p0 - 1 + kk) * ldh] : 0.0;
        Bs[idx] = ZW[(size_t)kk * ldzw + c0 + r];
    }
    __syncthreads();
    const int tx = tid & 15, ty = tid >> 4;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (int kk = 0; kk < bt; ++kk) {
        const double2 a01 = *reinterpret_cast<const double2*>(As + kk * kTM + 4 * ty);
        const double2 a23 = *reinterpret_cast<const double2*>(As + kk * kTM + 4 * ty + 2);
        const double2 b01 = *reinterpret_cast<const double2*>(Bs + kk * kTN + 4 * tx);
        const double2 b23 = *reinterpret_cast<const double2*>(Bs + kk * kTN + 4 * tx + 2);
        const double av[4] = {a01.x, a01.y, a23.x, a23.y};
        const double bv[4] = {b01.x, b01.y, b23.x, b23.y};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }

    // ---------------- epilogue -------------------------------------------
    const Epi* epi = ws<Epi>(work, L.off_epi);
    double* X = ws<double>(work, L.off_X);
    double* R = ws<double>(work, L.off_R);
    const int pair = (c0 >> 2) + tx;  // solution columns 2*pair, 2*pair+1
    const int sc0 = 2 * pair;
    const bool cplx = sc0 < 2 * L.mc;
    double mb[2] = {0.0, 0.0}, mr[2] = {0.0, 0.0};
    const int row0 = r0 + 4 * ty;
    if (cplx) {
        const int q = pair;
        const Epi E = epi[q];
        double* xre = X + (size_t)sc0 * L.ldw;
        double* xim = X + (size_t)(sc0 + 1) * L.ldw;
        double* rre = R + (size_t)sc0 * L.ldw;
        double* rim = R + (size_t)(sc0 + 1) * L.ldw;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int gi = row0 + i;
            if (gi < p0) {
                const double br_ = xre[gi], bi_ = xim[gi], ur = rre[gi], ui = rim[gi];
                const bool last = gi == p0 - 1;
                double nbr = fma(br_, E.fB, -acc[i][0]) - (ur * E.zbr_re - ui * E.zbr_im);
                double nbi = fma(bi_, E.fB, -acc[i][2]) - (ur * E.zbr_im + ui * E.zbr_re);
                double nrr = fma(E.pi, ur, acc[i][1]);
                double nri = fma(E.pi, ui, acc[i][3]);
                if (last) {
                    nbr += E.cz_re;
                    nbi += E.cz_im;
                    nrr -= E.cw_re;
                    nri -= E.cw_im;
                }
                xre[gi] = nbr;
                xim[gi] = nbi;
                rre[gi] = nrr;
                rim[gi] = nri;
                mb[0] = fmax(mb[0], fmax(fabs(nbr), fabs(nbi)));
                mr[0] = fmax(mr[0], fmax(fabs(nrr), fabs(nri)));
            }
        }
    } else {
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int sc = sc0 + j;
            if (sc >= L.ncol) continue;
            const int q = L.mc + (sc - 2 * L.mc);
            const Epi E = epi[q];
            double* xc = X + (size_t)sc * L.ldw;
            double* rc = R + (size_t)sc * L.ldw;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int gi = row0 + i;
                if (gi < p0) {
                    const double b_ = xc[gi], u = rc[gi];
                    const bool last = gi == p0 - 1;
                    double nb = fma(b_, E.fB, -acc[i][2 * j]) - u * E.zbr_re;
                    double nr = fma(E.pi, u, acc[i][2 * j + 1]);
                    if (last) {
                        nb += E.cz_re;
                        nr -= E.cw_re;
                    }
                    xc[gi] = nb;
                    rc[gi] = nr;
                    mb[j] = fmax(mb[j], fabs(nb));
                    mr[j] = fmax(mr[j], fabs(nr));
                }
            }
        }
    }
    // per-shift maxima: reduce over the 16 row groups, one atomic per column
    __syncthreads();
    double* red = smem;  // [2][16][32]
    red[(0 * 16 + ty) * 32 + 2 * tx] = mb[0];
    red[(0 * 16 + ty) * 32 + 2 * tx + 1] = mb[1];
    red[(1 * 16 + ty) * 32 + 2 * tx] = mr[0];
    red[(1 * 16 + ty) * 32 + 2 * tx + 1] = mr[1];
    __syncthreads();
    if (tid < 64) {
        const int which = tid >> 5, cl = tid & 31;
        double v = 0.0;
        for (int t = 0; t < 16; ++t) v = fmax(v, red[(which * 16 + t) * 32 + cl]);
        const int sc = (c0 >> 1) + cl;  // solution column
        if (sc < L.ncol) {
            int q = sc < 2 * L.mc ? (sc >> 1) : L.mc + (sc - 2 * L.mc);
            unsigned long long* dst = ws<unsigned long long>(work, which ? L.off_rmax : L.off_bmax);
            // complex shifts: both columns fold into the same shift's bound
            atomic_max_nonneg(dst + q, v);
        }
    }
}

}  // namespace

void launch_update(const Layout& L, void* work, const double* H, int ldh, int J, cudaStream_t s) {
    const int p0 = tile_start(L, J);
    if (p0 <= 0) return;
    dim3 grid((p0 + kTM - 1) / kTM, (2 * L.ncolp) / kTN);
    size_t smem = 2 * (size_t)L.br * kTM * sizeof(double);
    if (smem < 2 * 16 * 32 * sizeof(double)) smem = 2 * 16 * 32 * sizeof(double);
    k_update<<<grid, 256, smem, s>>>(L, work, H, ldh, J);
}

// the limit is per kernel, not per plan: configure it for the largest tile
// height, so that plans of different heights can be used in any order
cudaError_t update_configure(int br) {
    (void)br;
    size_t smem = 2 * (size_t)kMaxBr * kTM * sizeof(double);
    if (smem < 2 * 16 * 32 * sizeof(double)) smem = 2 * 16 * 32 * sizeof(double);
    return cudaFuncSetAttribute(k_update, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

}  // namespace hsein
