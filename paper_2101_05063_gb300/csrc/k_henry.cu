// Comparison baseline (hsein_options.method = 1): Henry's RQ solve of
// (H - lambda I) x = b per shift, unblocked (Alg. "henry"), the RQIN of the
// paper's experiments (Sec. 5).  One thread block per shift walks
// k = n-1 .. 1 over the whole matrix, reading column k-1 of H at every step:
// level-2 work, every shift re-reads the upper Hessenberg part of H.  Warp 0
// forms the rotation and the step's scalars and publishes them in shared
// memory; every warp then updates its rows of x and of the working column v
// (x -= a v - b t, v = c t + s v, t = h(:, k-1) - lambda e_(k-1), with
// a = x(k) conj(c), b = x(k) s).  Robustness as in the tiled sweep: one
// integer exponent, ProtectDivision before x(k) / phi, ProtectUpdate with an
// integer bound on |x| refined by an exact maximum when it fails
// (Sec. 4.1).  The solution, its exponent and the rotations are written in
// the layout the tiled path uses, so the same normalization, Varah test and
// Givens backtransform (k_finalize) follow.
#include "common.cuh"

namespace hsein {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

// bound on log2 |v| (v < 2^L); kNegInfLog for 0
__device__ inline int lbnd(double v) { return log2_bound(fabs(v)); }

__device__ int block_max_int(int v, int* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    int t = kNegInfLog;
    for (int w = 0; w < kWarps; ++w) t = max(t, red[w]);
    return t;
}

// the step's scalars, written by warp 0
struct Step {
    double cr, ci, s, xr, xi;  // rotation and x(k) / phi
    int sq;                    // power-of-two rescale of the whole x first (0: none)
};

template <bool CPLX>
__global__ void __launch_bounds__(kThreads)
k_henry(Layout L, void* work, const double* __restrict__ H, int ldh, int q_first, int robust,
        int om) {
    __shared__ Step st_s;
    __shared__ int red[kWarps];
    DevState* dst = ws<DevState>(work, L.off_state);
    if (dst->status < 0) return;
    const int q = q_first + blockIdx.x;
    const int n = L.n, tid = threadIdx.x;
    const double hscale = dst->hscale, hnorm = dst->hnorm;
    const double* lamv = ws<double>(work, L.off_lam);
    const double lre = lamv[2 * q], lim = CPLX ? lamv[2 * q + 1] : 0.0;
    const int col = qcolumn(L, q);
    double* xr = ws<double>(work, L.off_X) + (size_t)col * L.ldw;
    double* xi = xr + L.ldw;
    double* vr = ws<double>(work, L.off_R) + (size_t)col * L.ldw;
    double* vi = vr + L.ldw;
    double* Cr = ws<double>(work, L.off_Cr) + (size_t)q * n;
    double* Ci = ws<double>(work, L.off_Ci) + (size_t)q * n;
    double* Sv = ws<double>(work, L.off_S) + (size_t)q * n;
    const int LRb = lbnd(hnorm + fabs(lre) + fabs(lim));  // |R(i,k)| < 2^LRb
    auto lb2 = [&](double a, double b) {
        return CPLX ? max(lbnd(a), lbnd(b)) + 1 : lbnd(a);
    };
    auto xmax_exact = [&]() {
        int b = kNegInfLog;
        for (int i = tid; i < n; i += kThreads) b = max(b, lb2(xr[i], CPLX ? xi[i] : 0.0));
        return block_max_int(b, red);
    };
    auto rescale_all = [&](int sq) {
        for (int i = tid; i < n; i += kThreads) {
            xr[i] = scalbn(xr[i], -sq);
            if (CPLX) xi[i] = scalbn(xi[i], -sq);
        }
    };
    int e = ws<int>(work, L.off_eB)[q];
    int bx = xmax_exact();

    for (int k = n - 1; k >= 1; --k) {
        __syncthreads();  // the previous step's rows (among them row k) are done
        // ---- the step's scalars (warp 0); an overflow guard that needs the
        // whole vector is reported in st_s.sq and done by every thread
        if (tid < 32) {
            const double vkr = vr[k], vki = CPLX ? vi[k] : 0.0;
            double xkr = xr[k], xki = CPLX ? xi[k] : 0.0;
            double hs = H[k + (size_t)(k - 1) * ldh] * hscale, a0 = vkr, a1 = vki, sc = 1.0;
            int eh = max(lbnd(hs), lbnd(a0));
            if (CPLX) eh = max(eh, lbnd(a1));
            if (eh > 500 || eh < -500) {
                sc = scalbn(1.0, -eh);
                hs *= sc;
                a0 *= sc;
                a1 *= sc;
            }
            const double ss = CPLX ? fma(a0, a0, fma(a1, a1, hs * hs)) : fma(a0, a0, hs * hs);
            const double rr = rsqrt(ss);
            const double rinv = rr * sc;
            int sq = 0;
            if (robust) {  // ProtectDivision: |x(k)| / phi < 2^om
                sq = max(0, lb2(xkr, xki) + lbnd(rinv) - om);
                xkr = scalbn(xkr, -sq);
                xki = scalbn(xki, -sq);
            }
            if (tid == 0) {
                st_s.cr = a0 * rr;
                st_s.ci = CPLX ? a1 * rr : 0.0;
                st_s.s = -hs * rr;
                st_s.xr = xkr * rinv;
                st_s.xi = CPLX ? xki * rinv : 0.0;
                st_s.sq = sq;
            }
        }
        __syncthreads();
        Step S = st_s;
        if (S.sq) {  // rare: rescale the whole vector before the division
            rescale_all(S.sq);
            e += S.sq;
            bx -= S.sq;
        }
        if (robust) {
            // ProtectUpdate: |x| + |R| |x(k)| < 2^om, the bound refined by an
            // exact maximum only when it fails (every thread decides alike)
            const int lx = lb2(S.xr, S.xi);
            int nb = max(bx, LRb + lx) + 1;
            if (nb > om) {
                __syncthreads();  // x rescaled above is complete
                bx = max(xmax_exact(), lx);
                nb = max(bx, LRb + lx) + 1;
                if (nb > om) {
                    const int sq2 = nb - om;
                    __syncthreads();
                    rescale_all(sq2);
                    S.xr = scalbn(S.xr, -sq2);
                    S.xi = scalbn(S.xi, -sq2);
                    e += sq2;
                    nb = om;
                }
            }
            bx = nb;
        }
        // a = x(k) conj(c), b = x(k) s
        const double ar = CPLX ? fma(S.xr, S.cr, S.xi * S.ci) : S.xr * S.cr;
        const double ai = CPLX ? fma(S.xi, S.cr, -S.xr * S.ci) : 0.0;
        const double bR = S.xr * S.s, bI = CPLX ? S.xi * S.s : 0.0;
        __syncthreads();  // every thread has read row k (and rescaled it) before it is final
        if (tid == 0) {
            xr[k] = S.xr;
            if (CPLX) xi[k] = S.xi;
            Cr[k] = S.cr;
            if (CPLX) Ci[k] = S.ci;
            Sv[k] = S.s;
        }
        // ---- rows i < k
        const double* hc = H + (size_t)(k - 1) * ldh;
        for (int i = tid; i < k; i += kThreads) {
            double tr = hc[i] * hscale, ti = 0.0;
            if (i == k - 1) {
                tr -= lre;
                ti = -lim;
            }
            if (CPLX) {
                const double ur = vr[i], ui = vi[i];
                // x += b t - a v  (t complex only on the diagonal)
                xr[i] = fma(-ar, ur, fma(ai, ui, fma(bR, tr, fma(-bI, ti, xr[i]))));
                xi[i] = fma(-ar, ui, fma(-ai, ur, fma(bI, tr, fma(bR, ti, xi[i]))));
                // v = c t + s v
                vr[i] = fma(S.cr, tr, fma(-S.ci, ti, S.s * ur));
                vi[i] = fma(S.ci, tr, fma(S.cr, ti, S.s * ui));
            } else {
                const double u = vr[i];
                xr[i] = fma(-ar, u, fma(bR, tr, xr[i]));
                vr[i] = fma(S.cr, tr, S.s * u);
            }
        }
    }
    __syncthreads();
    // ---- final pivot r11 = v(0); an exactly singular or tiny pivot is
    // replaced by eps ||H'|| with its phase (+ for 0)
    if (tid < 32) {
        double pr = vr[0], pi = CPLX ? vi[0] : 0.0;
        double x0r = xr[0], x0i = CPLX ? xi[0] : 0.0;
        const double small = 0x1p-53 * hnorm;
        double pa = CPLX ? hypot(pr, pi) : fabs(pr);
        if (pa < small) {
            if (pa > 0.0) {
                pr *= small / pa;
                pi *= small / pa;
            } else {
                pr = small;
                pi = 0.0;
            }
            pa = small;
        }
        int sq = 0;
        if (robust) sq = max(0, lb2(x0r, x0i) - (lbnd(pa) - 1) - om);
        if (tid == 0) {
            st_s.sq = sq;
            st_s.cr = pr;
            st_s.ci = pi;
        }
    }
    __syncthreads();
    const int sq0 = st_s.sq;
    if (sq0) {
        rescale_all(sq0);
        e += sq0;
    }
    __syncthreads();
    if (tid == 0) {
        const double pr = st_s.cr, pi = st_s.ci;
        double x0r = xr[0], x0i = CPLX ? xi[0] : 0.0;
        if (CPLX) {
            // Smith's division
            double nr, ni;
            if (fabs(pr) >= fabs(pi)) {
                const double rt = pi / pr, d = pr + pi * rt;
                nr = (x0r + x0i * rt) / d;
                ni = (x0i - x0r * rt) / d;
            } else {
                const double rt = pr / pi, d = pi + pr * rt;
                nr = (x0r * rt + x0i) / d;
                ni = (x0i * rt - x0r) / d;
            }
            xr[0] = nr;
            xi[0] = ni;
            Ci[0] = 0.0;
        } else {
            xr[0] = x0r / pr;
        }
        Cr[0] = 1.0;  // padding rotation of the top row
        Sv[0] = 0.0;
        int* etile = ws<int>(work, L.off_etile);
        for (int J = 0; J < L.N; ++J) etile[(size_t)J * L.m + q] = e;
    }
}

}  // namespace

void launch_henry(const Layout& L, void* work, const double* H, int ldh, int robust,
                  int omega_log2, cudaStream_t s) {
    if (L.mc > 0) k_henry<true><<<L.mc, kThreads, 0, s>>>(L, work, H, ldh, 0, robust, omega_log2);
    if (L.mr > 0)
        k_henry<false><<<L.mr, kThreads, 0, s>>>(L, work, H, ldh, L.mc, robust, omega_log2);
}

}  // namespace hsein
