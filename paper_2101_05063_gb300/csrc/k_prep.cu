// Step a0 of the solve: checks, norms, prescale and initial state.
//
//  k_setup    one block: clears the device state, maps input shifts to the
//             internal order (complex shifts first, Sec. 4.3 interleaved
//             [re, im] storage), checks the count of complex shifts and that
//             every shift is finite.
//  k_rowpart  partial absolute row sums of H by column chunk; the chunks are
//             exactly the column ranges J^- = j-1 : j+b_r-2 of the tile
//             columns (Alg. "tiled-reduction"), so one pass gives both
//             ||H||_inf and the norms ||H(1:p0, J^-)||_inf that bound the
//             shared-H updates (ProtectUpdate's ||H||_inf, Alg.
//             "robust-tile-update").  Also checks finiteness and that H is
//             unreduced (Sec. 1).
//  k_rownorm  reduces the chunks: ||H||_inf and the per-tile-column table.
//  k_init     per shift: the power-of-two prescale of H and the shift, the
//             first cross-over column r~ = h(:,n) - lambda e_n (Alg.
//             "tiled-reduction", its initialization), the working copy of the
//             starting vector (or rho e, rho = eps ||H||_inf, Sec. 4.2), its
//             2-norm, and the first bounds for the robust update.
#include "common.cuh"

#include <cfloat>

namespace hsein {
namespace {

constexpr int kSetupThreads = 1024;
constexpr double kEps = 0x1p-53;
constexpr int kPrescaleLog2 = 1010;  // ||H'||_inf + |lambda'| < 2^1010 after prescale

__device__ int block_exclusive_scan(int v, int* smem_warp, int* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int nw = blockDim.x >> 5;
        int w = lane < nw ? smem_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) smem_warp[lane] = w;  // inclusive prefix of warp sums
    }
    __syncthreads();
    int before = (warp > 0 ? smem_warp[warp - 1] : 0) + x - v;
    *total = smem_warp[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before;
}

__global__ void k_setup(Layout L, void* work, const double* __restrict__ wr,
                        const double* __restrict__ wi) {
    DevState* st = ws<DevState>(work, L.off_state);
    int* qsrc = ws<int>(work, L.off_qsrc);
    int* qcol = ws<int>(work, L.off_qcol);
    unsigned long long* anorm = ws<unsigned long long>(work, L.off_anorm);
    __shared__ int sw[32];
    __shared__ int s_bad;
    if (threadIdx.x == 0) {
        st->status = 0;
        st->hexp = 0;
        st->ncplx_found = 0;
        st->hscale = 1.0;
        st->hnorm = 0.0;
        st->hnorm_bits = 0ull;
        st->lammax_bits = 0ull;
        s_bad = 0;
    }
    for (int J = threadIdx.x; J < L.N; J += blockDim.x) anorm[J] = 0ull;
    __syncthreads();
    int nc_before = 0, col_before = 0;
    for (int base = 0; base < L.m; base += blockDim.x) {
        int l = base + threadIdx.x;
        bool valid = l < L.m;
        double a = valid ? wr[l] : 0.0, b = valid ? wi[l] : 0.0;
        int isc = (valid && b != 0.0) ? 1 : 0;
        if (valid && !(isfinite(a) && isfinite(b))) atomicOr(&s_bad, 1);
        if (valid) atomic_max_nonneg(&st->lammax_bits, fabs(a) + fabs(b));
        int tc, tw;
        int c_ex = block_exclusive_scan(isc, sw, &tc);
        int w_ex = block_exclusive_scan(valid ? 1 + isc : 0, sw, &tw);
        if (valid) {
            int ncb = nc_before + c_ex;            // complex shifts before l
            int nrb = l - ncb;                     // real shifts before l
            int q = isc ? ncb : L.mc + nrb;
            bool inrange = isc ? (ncb < L.mc) : (nrb < L.mr);
            if (inrange) {
                qsrc[q] = l;
                qcol[q] = col_before + w_ex;
            }
        }
        nc_before += tc;
        col_before += tw;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        st->ncplx_found = nc_before;
        if (s_bad) set_error(st, -4);
        else if (nc_before != L.mc) set_error(st, -7);
    }
}

// column chunk c: 0 -> [0, b0-1); J in [1, N-1] -> J^- = [p0-1, p0-1+br); N -> [n-1, n)
__device__ inline void chunk_range(const Layout& L, int c, int* j0, int* j1) {
    if (c == 0) {
        *j0 = 0;
        *j1 = L.b0 - 1;
    } else if (c < L.N) {
        int p0 = tile_start(L, c);
        *j0 = p0 - 1;
        *j1 = p0 - 1 + L.br;
    } else {
        *j0 = L.n - 1;
        *j1 = L.n;
    }
}

__global__ void k_rowpart(Layout L, void* work, const double* __restrict__ H, int ldh) {
    DevState* st = ws<DevState>(work, L.off_state);
    double* part = ws<double>(work, L.off_rowpart);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (i >= L.n) return;
    int j0, j1;
    chunk_range(L, c, &j0, &j1);
    if (j0 < i - 1) j0 = i - 1;  // entries below the subdiagonal are not read
    // the finiteness and zero tests read the exponent and magnitude bits
    // (integer operations; on GB300 an FP64 compare costs an FP64 pipe slot)
    double s = 0.0;
    bool finite = true, zero_sub = false;
    for (int j = j0; j < j1; ++j) {
        const double h = H[i + (size_t)j * ldh];
        const unsigned long long m = abs_bits(h);
        finite = finite && m < 0x7FF0000000000000ULL;
        if (j == i - 1 && m == 0) zero_sub = true;
        s += fabs(h);
    }
    part[i + (size_t)c * L.n] = s;
    if (!finite) set_error(st, -4);
    if (zero_sub) set_error(st, -3);
}

__global__ void k_rownorm(Layout L, void* work, int row_blocks) {
    DevState* st = ws<DevState>(work, L.off_state);
    const double* part = ws<double>(work, L.off_rowpart);
    unsigned long long* anorm = ws<unsigned long long>(work, L.off_anorm);
    __shared__ double red[32];
    double best = 0.0;
    if ((int)blockIdx.x < row_blocks) {
        int i = blockIdx.x * blockDim.x + threadIdx.x;
        if (i < L.n) {
            double s = 0.0;
            for (int c = 0; c <= L.N; ++c) s += part[i + (size_t)c * L.n];  // fixed order
            best = s;
        }
    } else {
        int J = blockIdx.x - row_blocks + 1;  // 1 .. N-1
        int p0 = tile_start(L, J);
        for (int i = threadIdx.x; i < p0; i += blockDim.x)
            best = fmax(best, part[i + (size_t)J * L.n]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (threadIdx.x == 0) {
            if ((int)blockIdx.x < row_blocks) atomic_max_nonneg(&st->hnorm_bits, v);
            else anorm[blockIdx.x - row_blocks + 1] = (unsigned long long)__double_as_longlong(v);
        }
    }
}

__global__ void k_init(Layout L, void* work, const double* __restrict__ H, int ldh,
                       const double* __restrict__ wr, const double* __restrict__ wi,
                       const double* __restrict__ B, int ldb) {
    DevState* st = ws<DevState>(work, L.off_state);
    if (st->status < 0) return;
    const int q = blockIdx.x;
    const int* qsrc = ws<int>(work, L.off_qsrc);
    const int* qcol = ws<int>(work, L.off_qcol);
    double* lam = ws<double>(work, L.off_lam);
    double* bnorm = ws<double>(work, L.off_bnorm);
    int* eB = ws<int>(work, L.off_eB);
    unsigned long long* bmax = ws<unsigned long long>(work, L.off_bmax);
    unsigned long long* rmax = ws<unsigned long long>(work, L.off_rmax);
    double* X = ws<double>(work, L.off_X);
    double* R = ws<double>(work, L.off_R);

    // prescale: H' = 2^-s H with ||H'||_inf + max|lambda'| < 2^kPrescaleLog2
    const double hn = bits_to_double(st->hnorm_bits);
    const double lm = bits_to_double(st->lammax_bits);
    int lb = max(log2_bound(hn), log2_bound(lm)) + 1;
    int s = max(0, lb - kPrescaleLog2);
    const double hscale = ldexp(1.0, -s);
    if (q == 0 && threadIdx.x == 0) {
        st->hexp = s;
        st->hscale = hscale;
        st->hnorm = hn * hscale;
    }
    const int l = qsrc[q];
    const bool cplx = q < L.mc;
    const double lre = wr[l] * hscale, lim = cplx ? wi[l] * hscale : 0.0;
    if (threadIdx.x == 0) {
        lam[2 * q] = lre;
        lam[2 * q + 1] = lim;
        eB[q] = 0;
    }
    const int c = qcolumn(L, q);
    const int uc = qcol[q];
    const double rho = kEps * hn;  // default starting vector rho*e (Sec. 4.2)
    // pass 1: X = B, R~ = h(:, n) - lambda e_n, and the largest magnitudes
    // (integer maxima of the bit patterns: no FP64 work)
    unsigned long long xm = 0, rm = 0;
    for (int i = threadIdx.x; i < L.n; i += blockDim.x) {
        const double b0 = B ? B[i + (size_t)uc * ldb] : rho;
        X[i + (size_t)c * L.ldw] = b0;
        xm = max(xm, abs_bits(b0));
        // h(i, n) prescaled (the factor is 1 unless ||H|| is huge), minus
        // lambda' on row n
        double r0 = H[i + (size_t)(L.n - 1) * ldh];
        if (s != 0) r0 *= hscale;
        if (i == L.n - 1) r0 -= lre;
        R[i + (size_t)c * L.ldw] = r0;
        rm = max(rm, abs_bits(r0));
        if (cplx) {
            const double b1 = B ? B[i + (size_t)(uc + 1) * ldb] : 0.0;
            X[i + (size_t)(c + 1) * L.ldw] = b1;
            xm = max(xm, abs_bits(b1));
            const double r1 = (i == L.n - 1) ? -lim : 0.0;
            R[i + (size_t)(c + 1) * L.ldw] = r1;
            rm = max(rm, abs_bits(r1));
        }
    }
    __shared__ unsigned long long s_x[32], s_r[32];
    __shared__ double s_t[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        xm = max(xm, __shfl_xor_sync(0xffffffffu, xm, o));
        rm = max(rm, __shfl_xor_sync(0xffffffffu, rm, o));
    }
    if (lane == 0) {
        s_x[warp] = xm;
        s_r[warp] = rm;
    }
    __syncthreads();
    xm = s_x[0];
    rm = s_r[0];
    for (int w = 1; w < nw; ++w) {
        xm = max(xm, s_x[w]);
        rm = max(rm, s_r[w]);
    }
    // pass 2: ||b||_2 = 2^e sqrt(sum (b_i 2^-e)^2), 2^e the scale of the
    // largest |b_i| (exact power-of-two scaling; the column is re-read from
    // cache)
    const int e = norm_exp(xm);
    const double sc = pow2(-e);
    double ss = 0.0;
    for (int i = threadIdx.x; i < L.n; i += blockDim.x) {
        const double t0 = X[i + (size_t)c * L.ldw] * sc;
        ss = fma(t0, t0, ss);
        if (cplx) {
            const double t1 = X[i + (size_t)(c + 1) * L.ldw] * sc;
            ss = fma(t1, t1, ss);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if (lane == 0) s_t[warp] = ss;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < nw; ++w) t += s_t[w];
        bnorm[q] = xm == 0 ? 0.0 : sqrt(t) * pow2(e);
        bmax[q] = xm;
        rmax[q] = rm;
    }
}

}  // namespace

void launch_prepare(const Layout& L, void* work, const double* H, int ldh, const double* wr,
                    const double* wi, const double* B, int ldb, int omega_log2, cudaStream_t s) {
    (void)omega_log2;
    k_setup<<<1, kSetupThreads, 0, s>>>(L, work, wr, wi);
    const int rt = 128;
    dim3 g1((L.n + rt - 1) / rt, L.N + 1);
    k_rowpart<<<g1, rt, 0, s>>>(L, work, H, ldh);
    const int nt = 256;
    int row_blocks = (L.n + nt - 1) / nt;
    k_rownorm<<<row_blocks + (L.N - 1), nt, 0, s>>>(L, work, row_blocks);
    k_init<<<L.m, 256, 0, s>>>(L, work, H, ldh, wr, wi, B, ldb);
}

}  // namespace hsein
