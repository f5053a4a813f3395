// K1: per-shift work on one diagonal tile J (rows p0 .. p0+bt-1).
//
// One warp per shift; lane l owns the tile rows l, l+32, ... .  The H tile
// H(J, J^-) (columns p0-1 .. p0+bt-2, prescaled) sits in shared memory and is
// shared by the warps (shifts) of the block.
//
// Phase 1 (Alg. "tiled-reduction1" fused with Alg. "solve", i.e. Henry's
// Alg. "henry" restricted to the tile): for k = bt-1 .. 1 the rotation with
// [h(k,k-1) v(k)] G^H = [0 phi] is formed (Sec. 3.1 eq. "givens"; complex:
// eq. "cgivens" with c = v/phi, s = -h/phi), x(k) is divided by phi, column k
// of R (-s t + conj(c) v, t = h(:,k-1) - lambda e_{k-1}) updates the rows
// above it, and the working column becomes c t + s v.  Row 0 is closed by the
// rotation against h(p0, p0-1) (the left cross-over, Alg. "solve") or, on the
// top-left tile, by the division by v(0) (padding rotation c = 1, s = 0).
// Robustness (Sec. 4.1, Alg. "robust-solve"): the tile segment carries one
// exponent e (stored = true * 2^-e); a division that could exceed 2^omega is
// preceded by a power-of-two rescale (ProtectDivision), and so is an update
// whose bound |x| + |R(i,k)| |x(k)| could (ProtectUpdate); |R(i,k)| is bounded
// by ||H'||_inf + |lambda'| because R's rows are rows of H' - lambda' I times
// a unitary matrix.
//
// Phase 2 (Alg. "tile-update" lines building rho and z, and the weights of
// Alg. "tiled-reduction2" written as one product): z = G_{p0+bt-1}^H ...
// G_{p0}^H [0; x] gives Z' = [rho'; z(1:bt-1)] and z_br, and the off-diagonal
// reduction of the cross-over column unrolls to R~_left = A w + pi R~_right
// - lambda c_0 e_last with w_k = c_k prod_{i<k} s_i and pi = prod s_i.  Then
// the common exponent of the rows above is chosen (the consistent scaling
// min(alpha, beta) of Alg. "robust-tile-update" and one ProtectUpdate over
// all three linear updates of eq. "robust-update"), and [Z'|W] plus the
// epilogue constants are written for the shared-H product (k_update).
#include "common.cuh"
#include "ozaki.cuh"

namespace hsein {
namespace {

constexpr int kWarps = 4;

__device__ inline double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// q >= 0 such that 2^-q * xabs / dabs <= 2^om (dabs > 0); uses exponents only
__device__ inline int div_scale(double xabs, double dabs, int om) {
    if (dabs >= 1.0 || xabs == 0.0) return 0;
    if (xabs <= dabs * ldexp(1.0, om)) return 0;
    int q = log2_bound(xabs) - ilogb(dabs) - om;
    return q < 1 ? 1 : q;
}

// q >= 0 such that 2^-q (xb + rb * xk) <= 2^om, or 0 if already below
__device__ inline int upd_scale(double xb, double rb, double xk, int om) {
    double nb = fma(rb, xk, xb);
    if (nb <= ldexp(1.0, om)) return 0;
    int lq = max(log2_bound(xb), log2_bound(rb) + log2_bound(xk)) + 1 - om;
    return lq < 1 ? 1 : lq;
}

template <int T, bool CPLX>
__device__ void tile_shift(const Layout& L, void* work, const double* __restrict__ Hs, int J,
                           int p0, int bt, int q, int robust, int om, double* sm) {
    const int lane = threadIdx.x & 31;
    const int br = L.br;
    const DevState* st = ws<DevState>(work, L.off_state);
    const double* lamv = ws<double>(work, L.off_lam);
    int* eB = ws<int>(work, L.off_eB);
    int* etile = ws<int>(work, L.off_etile);
    unsigned long long* bmaxv = ws<unsigned long long>(work, L.off_bmax);
    unsigned long long* rmaxv = ws<unsigned long long>(work, L.off_rmax);
    const unsigned long long* anorm = ws<unsigned long long>(work, L.off_anorm);
    Epi* epi = ws<Epi>(work, L.off_epi);
    double* X = ws<double>(work, L.off_X);
    double* R = ws<double>(work, L.off_R);
    double* Cr = ws<double>(work, L.off_Cr);
    double* Ci = ws<double>(work, L.off_Ci);
    double* Sv = ws<double>(work, L.off_S);
    double* ZW = ws<double>(work, L.off_ZW);

    // per-warp shared scratch: c (re, im), s, x (re, im), Z' (re, im), W (re, im)
    double* s_cr = sm;
    double* s_ci = sm + br;
    double* s_s = sm + 2 * br;
    double* s_xr = sm + 3 * br;
    double* s_xi = sm + 4 * br;

    const double hscale = st->hscale;
    const double hnorm = st->hnorm;
    const double lre = lamv[2 * q], lim = CPLX ? lamv[2 * q + 1] : 0.0;
    const int col = qcolumn(L, q);
    const double Omega = ldexp(1.0, om);
    const double Rb = hnorm + fabs(lre) + fabs(lim);  // bound on |R(i,k)|

    double vr[T], vi[T], xr[T], xi[T];
#pragma unroll
    for (int t = 0; t < T; ++t) {
        int i = lane + 32 * t;
        bool ok = i < bt;
        vr[t] = ok ? R[p0 + i + (size_t)col * L.ldw] : 0.0;
        xr[t] = ok ? X[p0 + i + (size_t)col * L.ldw] : 0.0;
        if (CPLX) {
            vi[t] = ok ? R[p0 + i + (size_t)(col + 1) * L.ldw] : 0.0;
            xi[t] = ok ? X[p0 + i + (size_t)(col + 1) * L.ldw] : 0.0;
        } else {
            vi[t] = 0.0;
            xi[t] = 0.0;
        }
    }
    const int eB0 = eB[q];
    int e = eB0;
    double xbound = 0.0;
#pragma unroll
    for (int t = 0; t < T; ++t) xbound = fmax(xbound, fabs(xr[t]) + fabs(xi[t]));
    xbound = warp_max(xbound);

    auto rescale = [&](int sq, double& ar, double& ai) {
#pragma unroll
        for (int t = 0; t < T; ++t) {
            xr[t] = scalbn(xr[t], -sq);
            if (CPLX) xi[t] = scalbn(xi[t], -sq);
        }
        ar = scalbn(ar, -sq);
        if (CPLX) ai = scalbn(ai, -sq);
        xbound = scalbn(xbound, -sq);
        e += sq;
    };

    // ---------------- phase 1: sweep k = bt-1 .. 1 -----------------------
#pragma unroll
    for (int sl = T - 1; sl >= 0; --sl) {
        for (int kk = 31; kk >= 0; --kk) {
            const int k = sl * 32 + kk;
            if (k >= bt || k == 0) continue;
            double vkr = __shfl_sync(0xffffffffu, vr[sl], kk);
            double xkr = __shfl_sync(0xffffffffu, xr[sl], kk);
            double vki = 0.0, xki = 0.0;
            if (CPLX) {
                vki = __shfl_sync(0xffffffffu, vi[sl], kk);
                xki = __shfl_sync(0xffffffffu, xi[sl], kk);
            }
            const double h = Hs[k * br + k];  // h(p0+k, p0+k-1)
            double rinv = CPLX ? rhypot(h, hypot(vkr, vki)) : rhypot(h, vkr);
            const double cr = vkr * rinv, ci = vki * rinv, s = -h * rinv;
            if (robust) {
                double xa = fabs(xkr) + fabs(xki);
                if (rinv > 1.0) {
                    int sq = div_scale(xa, 1.0 / rinv, om);
                    if (sq) rescale(sq, xkr, xki);
                }
            }
            xkr *= rinv;
            xki *= rinv;
            if (robust) {
                double xa = fabs(xkr) + fabs(xki);
                if (!(fma(Rb, xa, xbound) <= Omega)) {
                    double ex = 0.0;
#pragma unroll
                    for (int t = 0; t < T; ++t) ex = fmax(ex, fabs(xr[t]) + fabs(xi[t]));
                    xbound = fmax(warp_max(ex), xa);
                    int sq = upd_scale(xbound, Rb, xa, om);
                    if (sq) {
                        rescale(sq, xkr, xki);
                        xa = fabs(xkr) + fabs(xki);
                    }
                }
                xbound = fma(Rb, xa, xbound);
            }
            // rows i < k: R(i,k) = -s t + conj(c) v ; x -= R x(k) ; v = c t + s v
#pragma unroll
            for (int t = 0; t <= sl; ++t) {
                const int i = lane + 32 * t;
                if (t < sl || lane < kk) {
                    double tr = Hs[k * br + i] - (i == k - 1 ? lre : 0.0);
                    double ti = (CPLX && i == k - 1) ? -lim : 0.0;
                    if (CPLX) {
                        // conj(c) v = (cr v_r + ci v_i) + i (cr v_i - ci v_r)
                        double rr = fma(cr, vr[t], fma(ci, vi[t], -s * tr));
                        double ri = fma(cr, vi[t], fma(-ci, vr[t], -s * ti));
                        // x -= R * xk (complex)
                        xr[t] = fma(-rr, xkr, fma(ri, xki, xr[t]));
                        xi[t] = fma(-rr, xki, fma(-ri, xkr, xi[t]));
                        // v = c t + s v
                        double nvr = fma(cr, tr, fma(-ci, ti, s * vr[t]));
                        double nvi = fma(cr, ti, fma(ci, tr, s * vi[t]));
                        vr[t] = nvr;
                        vi[t] = nvi;
                    } else {
                        double rr = fma(cr, vr[t], -s * tr);
                        xr[t] = fma(-rr, xkr, xr[t]);
                        vr[t] = fma(cr, tr, s * vr[t]);
                    }
                }
            }
            if (lane == kk) {
                xr[sl] = xkr;
                if (CPLX) xi[sl] = xki;
            }
            if (lane == 0) {
                s_cr[k] = cr;
                s_ci[k] = ci;
                s_s[k] = s;
            }
        }
    }

    // ---------------- row 0: left rotation or final pivot ----------------
    {
        double v0r = __shfl_sync(0xffffffffu, vr[0], 0);
        double v0i = CPLX ? __shfl_sync(0xffffffffu, vi[0], 0) : 0.0;
        double x0r = __shfl_sync(0xffffffffu, xr[0], 0);
        double x0i = CPLX ? __shfl_sync(0xffffffffu, xi[0], 0) : 0.0;
        double c0r, c0i, s0;
        if (p0 > 0) {
            const double h = Hs[0];  // h(p0, p0-1)
            double rinv = CPLX ? rhypot(h, hypot(v0r, v0i)) : rhypot(h, v0r);
            c0r = v0r * rinv;
            c0i = v0i * rinv;
            s0 = -h * rinv;
            if (robust && rinv > 1.0) {
                int sq = div_scale(fabs(x0r) + fabs(x0i), 1.0 / rinv, om);
                if (sq) rescale(sq, x0r, x0i);
            }
            x0r *= rinv;
            x0i *= rinv;
        } else {
            c0r = 1.0;
            c0i = 0.0;
            s0 = 0.0;
            // final pivot r11 = v(0); an exactly singular or tiny pivot is
            // replaced by eps ||H'||_inf with the pivot's phase (+ for 0)
            const double small = 0x1p-53 * hnorm;
            double pr = v0r, pi = v0i;
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
            if (robust) {
                int sq = div_scale(fabs(x0r) + fabs(x0i), pa, om);
                if (sq) rescale(sq, x0r, x0i);
            }
            if (CPLX) {
                // Smith's division (x0r + i x0i) / (pr + i pi)
                double nr, ni;
                if (fabs(pr) >= fabs(pi)) {
                    double r = pi / pr, d = pr + pi * r;
                    nr = (x0r + x0i * r) / d;
                    ni = (x0i - x0r * r) / d;
                } else {
                    double r = pr / pi, d = pi + pr * r;
                    nr = (x0r * r + x0i) / d;
                    ni = (x0i * r - x0r) / d;
                }
                x0r = nr;
                x0i = ni;
            } else {
                x0r /= pr;
            }
        }
        if (lane == 0) {
            xr[0] = x0r;
            if (CPLX) xi[0] = x0i;
            s_cr[0] = c0r;
            s_ci[0] = c0i;
            s_s[0] = s0;
        }
    }
    __syncwarp();

    // ---------------- outputs of phase 1 ---------------------------------
#pragma unroll
    for (int t = 0; t < T; ++t) {
        int i = lane + 32 * t;
        if (i < bt) {
            X[p0 + i + (size_t)col * L.ldw] = xr[t];
            s_xr[i] = xr[t];
            if (CPLX) {
                X[p0 + i + (size_t)(col + 1) * L.ldw] = xi[t];
                s_xi[i] = xi[t];
            }
        }
    }
    for (int i = lane; i < bt; i += 32) {
        size_t g = (size_t)q * L.n + p0 + i;
        Cr[g] = s_cr[i];
        Sv[g] = s_s[i];
        if (CPLX) Ci[g] = s_ci[i];
    }
    if (lane == 0) etile[(size_t)J * L.m + q] = e;
    __syncwarp();
    if (p0 == 0) return;

    // ---------------- phase 2: [Z'|W], scale exponent, epilogue ----------
    double* s_zr = s_xr;  // Z' and W overwrite the x and c scratch in place
    double* s_zi = s_xi;
    if (lane == 0) {
        // z = G^H [0; x]: rho' = -s_0 x_0, tau = conj(c_0) x_0, then
        // (Z'(k), tau) = (c_k tau - s_k x_k, s_k tau + conj(c_k) x_k)
        double c0r = s_cr[0], c0i = s_ci[0], s0 = s_s[0];
        double x0r = s_xr[0], x0i = CPLX ? s_xi[0] : 0.0;
        double tr = c0r * x0r + c0i * x0i;
        double ti = CPLX ? (c0r * x0i - c0i * x0r) : 0.0;
        double rhor = -s0 * x0r, rhoi = -s0 * x0i;
        s_zr[0] = rhor;
        if (CPLX) s_zi[0] = rhoi;
        double zmax = CPLX ? hypot(rhor, rhoi) : fabs(rhor);
        // W (prefix products) is written into the cosine scratch in place
        double pr = s0;  // prod of s_i for i < k
        // w_0 = c_0 stays in s_cr[0], s_ci[0]
        for (int k = 1; k < bt; ++k) {
            double ckr = s_cr[k], cki = s_ci[k], sk = s_s[k];
            double xkr = s_xr[k], xki = CPLX ? s_xi[k] : 0.0;
            double zr = ckr * tr - cki * ti - sk * xkr;
            double zi = CPLX ? (ckr * ti + cki * tr - sk * xki) : 0.0;
            // tau <- s tau + conj(c) x
            double ntr = sk * tr + ckr * xkr + cki * xki;
            double nti = CPLX ? (sk * ti + ckr * xki - cki * xkr) : 0.0;
            tr = ntr;
            ti = nti;
            s_zr[k] = zr;
            if (CPLX) s_zi[k] = zi;
            zmax = fmax(zmax, CPLX ? hypot(zr, zi) : fabs(zr));
            s_cr[k] = ckr * pr;  // w_k = c_k prod_{i<k} s_i
            s_ci[k] = cki * pr;
            pr *= sk;
        }
        const double pi_ = pr;
        const double zbr_r = tr, zbr_i = ti;

        // consistent exponent for the rows above (Alg. "robust-tile-update"):
        // B_new = B 2^(eB-e) - (A Z' + R~ z_br - lambda rho' e_last) 2^(ex-e)
        const int ex = e;
        int enew = max(eB0, ex);
        if (robust) {
            const int cadd = CPLX ? 1 : 0;
            const double An = bits_to_double(anorm[J]) * hscale;
            const double bm = bits_to_double(bmaxv[q]);
            const double rm = bits_to_double(rmaxv[q]);
            const double la = CPLX ? hypot(lre, lim) : fabs(lre);
            const double rh = CPLX ? hypot(rhor, rhoi) : fabs(rhor);
            const double zb = CPLX ? hypot(zbr_r, zbr_i) : fabs(zbr_r);
            int lt = max(log2_bound(An) + log2_bound(zmax),
                         max(log2_bound(rm) + cadd + log2_bound(zb), log2_bound(la) + log2_bound(rh))) + 2;
            int lb = log2_bound(bm) + cadd;
            int need = max(lb + eB0, lt + ex) + 1 - om;
            enew = max(enew, need);
        }
        const double fB = ldexp(1.0, eB0 - enew);
        const double fZ = ldexp(1.0, ex - enew);
        eB[q] = enew;
        bmaxv[q] = 0ull;
        rmaxv[q] = 0ull;
        Epi E;
        E.fB = fB;
        E.pi = pi_;
        E.zbr_re = zbr_r * fZ;
        E.zbr_im = zbr_i * fZ;
        // lambda' rho' fZ and lambda' c_0
        E.cz_re = (lre * rhor - lim * rhoi) * fZ;
        E.cz_im = (lre * rhoi + lim * rhor) * fZ;
        E.cw_re = lre * s_cr[0] - lim * s_ci[0];
        E.cw_im = lre * s_ci[0] + lim * s_cr[0];
        epi[q] = E;
        s_s[0] = fZ * hscale;  // reuse: factor for Z'
    }
    __syncwarp();
    const double fz = s_s[0];
    const size_t ldzw = 2 * (size_t)L.ncolp;
    if (!L.oz) {
        for (int k = lane; k < bt; k += 32) {
            double* row = ZW + (size_t)k * ldzw + 2 * (size_t)col;
            if (CPLX) {
                row[0] = s_zr[k] * fz;
                row[1] = s_cr[k] * hscale;
                row[2] = s_zi[k] * fz;
                row[3] = s_ci[k] * hscale;
            } else {
                row[0] = s_zr[k] * fz;
                row[1] = s_cr[k] * hscale;
            }
        }
    } else {
        // [Z'|W] as BF16 digits with one exponent per product column
        __nv_bfloat16* zd = ws<__nv_bfloat16>(work, L.off_zwd);
        int* zf = ws<int>(work, L.off_zwf);
        const int ncols = CPLX ? 4 : 2;
        for (int cc = 0; cc < ncols; ++cc) {
            const double* src = (cc & 1) ? ((cc & 2) ? s_ci : s_cr) : ((cc & 2) ? s_zi : s_zr);
            const double f = (cc & 1) ? hscale : fz;
            double v0 = lane < bt ? src[lane] * f : 0.0;
            double v1 = lane + 32 < bt ? src[lane + 32] * f : 0.0;
            double m = warp_max(fmax(fabs(v0), fabs(v1)));
            const int e = oz::scale_exponent(m);
            const int gc = 2 * col + cc;
            if (lane == 0) zf[gc] = e;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int k = lane + 32 * h;
                if (k < br) {
                    int d[oz::kS];
                    oz::split_digits(h ? v1 : v0, e, d);
#pragma unroll
                    for (int i = 0; i < oz::kS; ++i)
                        zd[((size_t)i * ldzw + gc) * br + k] = __float2bfloat16_rn((float)d[i]);
                }
            }
        }
    }
}

template <int T>
__global__ void __launch_bounds__(kWarps * 32)
k_diag(Layout L, void* work, const double* __restrict__ H, int ldh, int J, int robust, int om) {
    extern __shared__ __align__(16) double smem[];
    const DevState* st = ws<DevState>(work, L.off_state);
    if (st->status < 0) return;
    const int br = L.br;
    double* Hs = smem;  // [br cols][br rows]
    double* scratch = smem + (size_t)br * br + (size_t)(threadIdx.x >> 5) * 5 * br;
    const int p0 = tile_start(L, J);
    const int bt = tile_height(L, J);
    const double hscale = st->hscale;
    for (int idx = threadIdx.x; idx < bt * bt; idx += blockDim.x) {
        int cc = idx / bt, i = idx % bt;
        int gc = p0 - 1 + cc;
        double v = 0.0;
        if (gc >= 0 && i <= cc) v = H[p0 + i + (size_t)gc * ldh] * hscale;
        Hs[cc * br + i] = v;
    }
    __syncthreads();
    const int q = blockIdx.x * kWarps + (threadIdx.x >> 5);
    if (q >= L.m) return;
    if (q < L.mc)
        tile_shift<T, true>(L, work, Hs, J, p0, bt, q, robust, om, scratch);
    else
        tile_shift<T, false>(L, work, Hs, J, p0, bt, q, robust, om, scratch);
}

}  // namespace

void launch_diag(const Layout& L, void* work, const double* H, int ldh, int J, int robust,
                 int omega_log2, cudaStream_t s) {
    int grid = (L.m + kWarps - 1) / kWarps;
    size_t smem = ((size_t)L.br * L.br + (size_t)kWarps * 5 * L.br) * sizeof(double);
    if (L.br <= 32) {
        k_diag<1><<<grid, kWarps * 32, smem, s>>>(L, work, H, ldh, J, robust, omega_log2);
    } else if (L.br <= 64) {
        k_diag<2><<<grid, kWarps * 32, smem, s>>>(L, work, H, ldh, J, robust, omega_log2);
    } else {
        k_diag<4><<<grid, kWarps * 32, smem, s>>>(L, work, H, ldh, J, robust, omega_log2);
    }
}

// dynamic shared memory above 48 KB needs an opt-in per kernel
cudaError_t diag_configure(int br) {
    size_t smem = ((size_t)br * br + (size_t)kWarps * 5 * br) * sizeof(double);
    cudaError_t e = cudaSuccess;
    if (br <= 32) e = cudaFuncSetAttribute(k_diag<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    else if (br <= 64) e = cudaFuncSetAttribute(k_diag<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    else e = cudaFuncSetAttribute(k_diag<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return e;
}

}  // namespace hsein
