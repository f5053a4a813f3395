// Comparison baseline (hsein_options.method = 2): the LU approach of
// LAPACK's inverse iteration (Sec. 2.1) per shift.  P (H - lambda I) = L U
// with partial pivoting, L y = P b, U x = 2^-e y, the first iteration with
// the given starting vector (the system the RQ solve answers), in FP64.
//
// One thread block per shift.  The matrix is first copied row-major and
// prescaled (k_lu_rows), so that row k+1 of H, which elimination step k
// reads, is contiguous.  For a Hessenberg matrix the pivot search at step k
// is between two rows: w, the row carried down, held in shared memory, and
// row k+1 of H - lambda I; the one whose entry in column k has the larger
// magnitude (compared by squares) becomes row k of U, written row-packed to
// the block's slot of the workspace, and the other is eliminated with
// |l_k| <= 1 and carried down.  Thread 0 takes the pivot decision for the
// next step right after updating w(k+1), and carries the forward
// substitution y (registers for y(k), y(k+1); the next entry of b is
// prefetched one step ahead), so one barrier per step suffices.  The back
// substitution is row-oriented: per row a block reduction of U(i, i+1:) x,
// coalesced reads of the packed row.  Robustness (Sec. 4.1): one integer
// exponent for the whole vector; the forward step halves the vector when
// |y(k+1)| + |y(k)| could exceed 2^omega; before each row's dot product the
// bound 2^bx (|x| < 2^bx) times the row's largest magnitude (recorded as an
// integer maximum of bit patterns during the elimination) times its length
// is kept below 2^omega, and each division is preceded by ProtectDivision.
// The result, its exponent and identity rotations are written in the layout
// of the tiled path, so the same normalization and Varah test follow
// (k_finalize; its Givens backtransform is the identity here).
#include "common.cuh"

namespace hsein {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

// the decision of one elimination step, published by thread 0
struct Dec {
    double lr, li;  // multiplier l_k
    int swap;       // row k+1 becomes row k of U
    int q;          // forward substitution: exponent added before this step (0: none)
};

__device__ inline int lbits(unsigned long long b) {
    // floor(log2 v) + 1 for the non-negative double with bit pattern b
    // (normal numbers; subnormals and 0 get the bound of the smallest normal)
    const int ex = (int)((b >> 52) & 0x7FF);
    return max(ex, 1) - 1022;
}
__device__ inline unsigned long long cabs_bits(double re, double im) {
    // bit pattern of |re| + |im| rounded up: an upper bound of the modulus
    return abs_bits(fabs(re) + fabs(im)) + 1;
}

// Smith's division (ar + i ai) / (br + i bi)
__device__ inline void cdiv(double ar, double ai, double br, double bi, double& cr, double& ci) {
    if (fabs(br) >= fabs(bi)) {
        const double r = bi / br, d = br + bi * r;
        cr = (ar + ai * r) / d;
        ci = (ai - ar * r) / d;
    } else {
        const double r = br / bi, d = bi + br * r;
        cr = (ar * r + ai) / d;
        ci = (ai * r - ar) / d;
    }
}

__global__ void k_lu_rows(Layout L, void* work, const double* __restrict__ H, int ldh) {
    const DevState* st = ws<DevState>(work, L.off_state);
    if (st->status < 0) return;
    __shared__ double tile[32][33];
    const int n = L.n;
    const double hscale = st->hscale;
    double* Hr = ws<double>(work, L.off_hr);
    const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int j = j0 + r, i = i0 + threadIdx.x;
        tile[r][threadIdx.x] = (i < n && j < n && j + 1 >= i) ? H[i + (size_t)j * ldh] * hscale : 0.0;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += 8) {
        const int i = i0 + r, j = j0 + threadIdx.x;
        if (i < n && j < n) Hr[(size_t)i * n + j] = tile[threadIdx.x][r];
    }
}

template <bool CPLX>
__global__ void __launch_bounds__(kThreads)
k_lu(Layout L, void* work, int q_first, int robust, int om) {
    extern __shared__ double sw[];  // w, later x / y: n entries (complex: re, im interleaved)
    __shared__ Dec dec[2];
    __shared__ double red[kWarps][2];
    __shared__ int s_back[2][2];  // back substitution: exponent added, bound of |x(i)|
    DevState* dst = ws<DevState>(work, L.off_state);
    if (dst->status < 0) return;
    const int slot = blockIdx.x, q = q_first + slot;
    const int n = L.n, tid = threadIdx.x;
    const double hnorm = dst->hnorm;
    const double* lamv = ws<double>(work, L.off_lam);
    const double lre = lamv[2 * q], lim = CPLX ? lamv[2 * q + 1] : 0.0;
    const int col = qcolumn(L, q);
    double* xr = ws<double>(work, L.off_X) + (size_t)col * L.ldw;
    double* xi = xr + L.ldw;
    const double* Hr = ws<double>(work, L.off_hr);
    char* sbase = ws<char>(work, L.off_lu) + (size_t)slot * L.lu_slot_bytes;
    double* U = reinterpret_cast<double*>(sbase);  // packed rows, complex entries (re, im)
    unsigned long long* rmax =
        reinterpret_cast<unsigned long long*>(sbase + (size_t)n * (n + 1) / 2 * 16);
    const double omega = ldexp(1.0, om);
    auto rowoff = [&](int k) { return (size_t)k * n - (size_t)k * (k - 1) / 2; };
    auto W = [&](int j) -> double& { return sw[CPLX ? 2 * j : j]; };
    auto Wi = [&](int j) -> double& { return sw[2 * j + 1]; };

    // ---- elimination with the fused forward substitution -------------------
    for (int j = tid; j < n; j += kThreads) {
        W(j) = Hr[j] - (j == 0 ? lre : 0.0);
        if (CPLX) Wi(j) = j == 0 ? -lim : 0.0;
        rmax[j] = 0ull;
    }
    int e = 0;  // exponent of the vector (forward and back substitution)
    // thread 0: y(k) and the prefetched y(k+1) (scaled by 2^-e), written to x
    double yr = 0.0, yi = 0.0, nr = 0.0, ni = 0.0;
    if (tid == 0) {
        yr = xr[0];
        yi = CPLX ? xi[0] : 0.0;
        if (n > 1) {
            nr = xr[1];
            ni = CPLX ? xi[1] : 0.0;
        }
    }
    __syncthreads();
    // thread 0: the decision of step k from w(k) and h(k+1,k), the pivot into
    // U, and the forward step on y
    auto decide = [&](int k) {
        const double tr = Hr[(size_t)(k + 1) * n + k];  // subdiagonal: no shift
        const double wr = W(k), wi = CPLX ? Wi(k) : 0.0;
        const double tt = tr * tr, ww = CPLX ? fma(wr, wr, wi * wi) : wr * wr;
        const int swap = tt > ww;
        const double pr = swap ? tr : wr, pi = swap ? 0.0 : wi;
        const double orr = swap ? wr : tr, oi = swap ? wi : 0.0;
        double lr, li = 0.0;
        if (CPLX) cdiv(orr, oi, pr, pi, lr, li);
        else lr = orr / pr;
        double* Uk = U + 2 * rowoff(k);
        Uk[0] = pr;
        Uk[1] = pi;
        // forward step: y(k), y(k+1) exchanged if swap, y(k+1) -= l y(k)
        double ar = yr, ai = yi, br = nr, bi = ni;
        if (swap) {
            ar = nr;
            ai = ni;
            br = yr;
            bi = yi;
        }
        int qf = 0;
        if (robust) {
            const double mb = CPLX ? fabs(br) + fabs(bi) : fabs(br);
            const double ma = CPLX ? fabs(ar) + fabs(ai) : fabs(ar);
            if (mb > omega - ma) {  // halve the vector (rare)
                qf = 1;
                ar *= 0.5;
                ai *= 0.5;
                br *= 0.5;
                bi *= 0.5;
            }
        }
        br = fma(-lr, ar, br);
        if (CPLX) {
            br = fma(li, ai, br);
            bi = fma(-lr, ai, fma(-li, ar, bi));
        }
        xr[k] = ar;  // y(k) is final
        if (CPLX) xi[k] = ai;
        yr = br;
        yi = bi;
        if (k + 2 < n) {  // the next entry of b, with the exponent so far
            nr = xr[k + 2];
            ni = CPLX ? xi[k + 2] : 0.0;
        }
        dec[k & 1] = Dec{lr, li, swap, qf};
    };
    if (tid == 0 && n > 1) decide(0);
    __syncthreads();
    for (int k = 0; k + 1 < n; ++k) {
        const Dec D = dec[k & 1];
        if (D.q) {
            // the forward step halved y: the written entries y(0..k-1) and
            // the unread b(k+2..) follow (thread 0 holds the rest in registers)
            for (int j = tid; j < n; j += kThreads) {
                if (j < k || j >= k + 2) {
                    xr[j] *= 0.5;
                    if (CPLX) xi[j] *= 0.5;
                }
            }
            if (tid == 0) {
                nr *= 0.5;
                ni *= 0.5;
            }
            e += 1;
            __syncthreads();
        }
        double* Uk = U + 2 * rowoff(k);
        const double* hrow = Hr + (size_t)(k + 1) * n;
        unsigned long long mx = abs_bits(CPLX ? fabs(Uk[0]) + fabs(Uk[1]) : Uk[0]) + 1;
        mx = tid == 0 ? mx : 0ull;
        for (int j = k + 1 + tid; j < n; j += kThreads) {
            const double tr = hrow[j] - (j == k + 1 ? lre : 0.0);
            const double ti = (CPLX && j == k + 1) ? -lim : 0.0;
            const double wr = W(j), wi = CPLX ? Wi(j) : 0.0;
            const double ur = D.swap ? tr : wr, ui = D.swap ? ti : wi;
            const double orr = D.swap ? wr : tr, oi = D.swap ? wi : ti;
            Uk[2 * (j - k)] = ur;
            Uk[2 * (j - k) + 1] = ui;
            mx = max(mx, CPLX ? cabs_bits(ur, ui) : abs_bits(ur));
            if (CPLX) {
                W(j) = fma(-D.lr, ur, fma(D.li, ui, orr));
                Wi(j) = fma(-D.lr, ui, fma(-D.li, ur, oi));
            } else {
                W(j) = fma(-D.lr, ur, orr);
            }
            if (j == k + 1 && k + 2 < n) decide(k + 1);  // tid 0 owns column k+1
        }
        // the row's largest magnitude: warp maxima, one atomic per warp
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((tid & 31) == 0 && mx) atomicMax(rmax + k, mx);
        __syncthreads();
    }
    // the last pivot: an exactly singular or tiny one is replaced by
    // eps ||H'|| with its phase (+ for 0)
    if (tid == 0) {
        double pr = W(n - 1), pi = CPLX ? Wi(n - 1) : 0.0;
        const double small = 0x1p-53 * hnorm;
        const double pa = CPLX ? hypot(pr, pi) : fabs(pr);
        if (pa < small) {
            if (pa > 0.0) {
                pr *= small / pa;
                pi *= small / pa;
            } else {
                pr = small;
                pi = 0.0;
            }
        }
        double* Un = U + 2 * rowoff(n - 1);
        Un[0] = pr;
        Un[1] = pi;
        atomicMax(rmax + (n - 1), CPLX ? cabs_bits(pr, pi) : abs_bits(pr));
        xr[n - 1] = yr;  // the last entry of y
        if (CPLX) xi[n - 1] = yi;
    }
    __syncthreads();

    // ---- back substitution, row-oriented, x and the rest of y in shared
    // memory ------------------------------------------------------------------
    for (int j = tid; j < n; j += kThreads) {
        W(j) = xr[j];
        if (CPLX) Wi(j) = xi[j];
    }
    int bx = kNegInfLog;  // |x(i+1:)| < 2^bx (every thread keeps the same bound)
    if (tid == 0) s_back[1][0] = s_back[1][1] = 0;
    __syncthreads();
    // scale every entry but `skip` by 2^-sq (exact)
    auto scale_all = [&](int sq, int skip) {
        const double f = ldexp(1.0, -sq);
        for (int j = tid; j < n; j += kThreads) {
            if (j == skip) continue;
            W(j) *= f;
            if (CPLX) Wi(j) *= f;
        }
    };
    for (int i = n - 1; i >= 0; --i) {
        // the previous row's division may have rescaled (thread 0 decided):
        // every entry but that row's new x, which was computed scaled
        const int qd = s_back[(i + 1) & 1][0];
        const int lx = s_back[(i + 1) & 1][1];
        if (i < n - 1) {
            if (qd) {
                scale_all(qd, i + 1);
                e += qd;
                bx -= qd;
            }
            bx = max(bx, lx);
        }
        // ProtectUpdate for the row: |y(i)| + |U(i, i+1:)| |x| < 2^omega
        // with |U(i, i+1:) x| < 2^(lb(max|U(i,:)|) + ceil(log2(n-i)) + bx)
        if (robust && i < n - 1) {
            const int lu = lbits(rmax[i]) + (32 - __clz(n - i - 1)) + (CPLX ? 1 : 0);
            const int need = lu + bx + 1 - om;
            if (need > 0) {
                __syncthreads();  // every read of the previous row's x is done
                scale_all(need, -1);
                e += need;
                bx -= need;
                __syncthreads();
            }
        }
        const double* Ui = U + 2 * rowoff(i);
        double sr = 0.0, si = 0.0;
        for (int j = i + 1 + tid; j < n; j += kThreads) {
            const double ur = Ui[2 * (j - i)];
            if (CPLX) {
                const double ui = Ui[2 * (j - i) + 1];
                sr = fma(ur, W(j), fma(-ui, Wi(j), sr));
                si = fma(ur, Wi(j), fma(ui, W(j), si));
            } else {
                sr = fma(ur, W(j), sr);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sr += __shfl_xor_sync(0xffffffffu, sr, o);
            if (CPLX) si += __shfl_xor_sync(0xffffffffu, si, o);
        }
        if ((tid & 31) == 0) {
            red[tid >> 5][0] = sr;
            red[tid >> 5][1] = si;
        }
        __syncthreads();
        if (tid == 0) {
            double dr = 0.0, di = 0.0;
            for (int w = 0; w < kWarps; ++w) {
                dr += red[w][0];
                di += red[w][1];
            }
            double ar = W(i) - dr, ai = CPLX ? Wi(i) - di : 0.0;
            const double pr = Ui[0], pi = CPLX ? Ui[1] : 0.0;
            int qd2 = 0;
            if (robust) {  // ProtectDivision: |s| / |u(i,i)| < 2^omega
                const double pa = CPLX ? fabs(pr) + fabs(pi) : fabs(pr);
                const double ma = CPLX ? fabs(ar) + fabs(ai) : fabs(ar);
                // |s| / |u| <= 2 ma / pa for complex (|.|_1 against the modulus)
                const int lq = lbits(abs_bits(ma)) - (lbits(abs_bits(pa)) - 1) + (CPLX ? 1 : 0);
                qd2 = max(0, lq - om);
                if (qd2) {
                    ar = ldexp(ar, -qd2);
                    ai = ldexp(ai, -qd2);
                }
            }
            double xr0, xi0 = 0.0;
            if (CPLX) cdiv(ar, ai, pr, pi, xr0, xi0);
            else xr0 = ar / pr;
            W(i) = xr0;
            if (CPLX) Wi(i) = xi0;
            s_back[i & 1][0] = qd2;
            s_back[i & 1][1] = CPLX ? lbits(cabs_bits(xr0, xi0)) : lbits(abs_bits(xr0));
        }
        __syncthreads();
    }
    // the last division's rescale applies to the rest of the vector
    if (s_back[0][0]) {
        scale_all(s_back[0][0], 0);
        e += s_back[0][0];
    }
    __syncthreads();

    // ---- results in the tiled path's layout -------------------------------
    double* Cr = ws<double>(work, L.off_Cr) + (size_t)q * n;
    double* Ci = ws<double>(work, L.off_Ci) + (size_t)q * n;
    double* Sv = ws<double>(work, L.off_S) + (size_t)q * n;
    for (int j = tid; j < n; j += kThreads) {
        xr[j] = W(j);
        if (CPLX) {
            xi[j] = Wi(j);
            Ci[j] = 0.0;
        }
        Cr[j] = 1.0;  // identity rotations: no Givens backtransform
        Sv[j] = 0.0;
    }
    if (tid == 0) {
        int* etile = ws<int>(work, L.off_etile);
        for (int J = 0; J < L.N; ++J) etile[(size_t)J * L.m + q] = e;
    }
}

}  // namespace

size_t lu_slot_bytes(int n) {
    const size_t b = (size_t)n * (n + 1) / 2 * 16 + (size_t)n * 8;
    return (b + 255) & ~(size_t)255;
}

size_t lu_smem_bytes(int n, bool cplx) { return (size_t)n * (cplx ? 16 : 8); }

void launch_lu(const Layout& L, void* work, const double* H, int ldh, int robust, int omega_log2,
               cudaStream_t s) {
    dim3 g((L.n + 31) / 32, (L.n + 31) / 32);
    k_lu_rows<<<g, dim3(32, 8), 0, s>>>(L, work, H, ldh);
    // chunks of at most L.lu_slots shifts, complex shifts first
    for (int q0 = 0; q0 < L.mc; q0 += L.lu_slots) {
        const int cnt = min(L.lu_slots, L.mc - q0);
        k_lu<true><<<cnt, kThreads, lu_smem_bytes(L.n, true), s>>>(L, work, q0, robust, omega_log2);
    }
    for (int q0 = L.mc; q0 < L.m; q0 += L.lu_slots) {
        const int cnt = min(L.lu_slots, L.m - q0);
        k_lu<false><<<cnt, kThreads, lu_smem_bytes(L.n, false), s>>>(L, work, q0, robust,
                                                                      omega_log2);
    }
}

cudaError_t lu_configure(int n) {
    const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(k_lu<true>, a, (int)lu_smem_bytes(n, true));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_lu<false>, a, (int)lu_smem_bytes(n, false));
}

}  // namespace hsein
