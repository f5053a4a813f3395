// K1: per-shift work on one diagonal tile J (rows p0 .. p0+bt-1).
//
// Layout: a group of LPS lanes serves one shift and owns the tile rows
// r, r+LPS, r+2 LPS, ... (r = lane % LPS); a warp holds 32/LPS shifts.  GB300
// issues FP64 work per warp instruction whatever the number of active lanes,
// so the per-step rotation serves every shift of the warp at once, the
// update loop only runs the row slots that still hold rows above the pivot,
// and all overflow bookkeeping runs on integer exponents.  The
// diagonal tile (staged once per solve, contiguous and prescaled) arrives in
// shared memory with one bulk asynchronous copy completed on an mbarrier.
//
// Phase 1 (Alg. "tiled-reduction1" fused with Alg. "solve", i.e. Henry's
// Alg. "henry" restricted to the tile): for k = bt-1 .. 1 the rotation with
// [h(k,k-1) v(k)] G^H = [0 phi] is formed (eq. "givens"; complex: eq.
// "cgivens" with c = v/phi, s = -h/phi, phi = sqrt(h^2 + |v|^2)), x(k) is
// divided by phi, column k of R (conj(c) v - s t, t = h(:,k-1) - lambda
// e_{k-1}) updates the rows above it, and the working column becomes
// c t + s v.  With a = x(k) conj(c) and b = x(k) s the two updates of a row
// are x -= a v - b t and v = c t + s v.  Row 0 is closed by the rotation
// against h(p0, p0-1) (the left cross-over, Alg. "solve") or, on the
// top-left tile, by the division by v(0) (padding rotation c = 1, s = 0).
// Robustness (Sec. 4.1, Alg. "robust-solve"): the tile segment carries one
// exponent e (stored = true * 2^-e).  An integer bound 2^bx on |x| is kept;
// a division whose result could exceed 2^omega is preceded by a
// power-of-two rescale (ProtectDivision), and so is an update whose bound
// |x| + |R(i,k)| |x(k)| could (ProtectUpdate); |R(i,k)| <= ||H'||_inf +
// |lambda'| because R's rows are rows of H' - lambda' I times a unitary
// matrix.  Only a bound that fails is refined by an exact maximum.
//
// Phase 2 (Alg. "tile-update" lines building rho and z, and the weights of
// Alg. "tiled-reduction2" written as one product): z = G_{p0+bt-1}^H ...
// G_{p0}^H [0; x] gives Z' = [rho'; z(1:bt-1)] and z_br, and the off-diagonal
// reduction of the cross-over column unrolls to R~_left = A w + pi R~_right
// - lambda c_0 e_last with w_k = c_k prod_{i<k} s_i and pi = prod s_i.  Then
// the common exponent of the rows above is chosen (the consistent scaling
// min(alpha, beta) of Alg. "robust-tile-update" and one ProtectUpdate over
// all three linear updates of eq. "robust-update"), and [Z'|W] plus the
// epilogue constants are written for the shared-H product.
#include "common.cuh"
#include "ozaki.cuh"

#include <type_traits>

namespace hsein {
namespace {

constexpr unsigned kFull = 0xffffffffu;
// after a wait has run out, the tile copy in flight still lands in this
// block's shared memory: the block waits up to this many more cycles for it
// before it returns
constexpr long long kDrainCycles = 1LL << 32;

// floor(log2|v|) + 1 (v < 2^L) from the exponent bits; kNegInfLog for 0
__device__ inline int lbound(double v) {
    const int ex = (int)((__double_as_longlong(v) >> 52) & 0x7FF);
    if (ex != 0) return ex - 1022;
    return v == 0.0 ? kNegInfLog : ilogb(v) + 1;
}

// f(integral_constant<I>), f(integral_constant<I-1>), ..., f(integral_constant<0>)
template <int I, class F>
__device__ __forceinline__ void static_down(F&& f) {
    if constexpr (I >= 0) {
        f(std::integral_constant<int, I>{});
        static_down<I - 1>(f);
    }
}

template <int LPS>
__device__ inline int group_max_int(int v) {
#pragma unroll
    for (int o = 1; o < LPS; o <<= 1) v = max(v, __shfl_xor_sync(kFull, v, o));
    return v;
}
template <int LPS>
__device__ inline double group_max(double v) {
#pragma unroll
    for (int o = 1; o < LPS; o <<= 1) v = fmax(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

// LPS lanes per shift (32 / LPS shifts per warp), RPL rows per lane
// -v by flipping the sign bit (exact).  Used for the negated values that
// feed the rotation's selects: the sweep's step measured shorter this way
// than with the compiler's own negation (same FP64 instruction count, a
// different schedule)
__device__ inline double negd(double v) {
    return __longlong_as_double(__double_as_longlong(v) ^ (long long)0x8000000000000000ULL);
}

template <int LPS, int RPL, bool CPLX>
__device__ void tile_group(const Layout& L, void* work, const double* __restrict__ Hs, int J,
                           int p0, int bt, int q, bool qok, int robust, int om, double* sm) {
    const int lane = threadIdx.x & 31, r = lane & (LPS - 1), gbase = lane & ~(LPS - 1);
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

    // per-group shared scratch: c (re, im), s, x (re, im), shifted diagonal,
    // squared subdiagonal
    double* s_cr = sm;
    double* s_ci = sm + br;
    double* s_s = sm + 2 * br;
    double* s_xr = sm + 3 * br;
    double* s_xi = sm + 4 * br;

    const double hscale = st->hscale;
    const double hnorm = st->hnorm;
    const double lre = qok ? lamv[2 * q] : 0.0;
    const double lim = (CPLX && qok) ? lamv[2 * q + 1] : 0.0;
    const int col = qok ? qcolumn(L, q) : 0;
    const int LRb = lbound(hnorm + fabs(lre) + fabs(lim));  // |R(i,k)| < 2^LRb
    const int cadd = CPLX ? 1 : 0;                            // |z| <= |re| + |im|
    // integer bound of a (complex) value's magnitude
    auto lb2 = [&](double a, double b) { return CPLX ? max(lbound(a), lbound(b)) + 1 : lbound(a); };

    double vr[RPL], vi[RPL], xr[RPL], xi[RPL];
    // the tile rows of the working column and of x (global memory is not
    // written before phase 1 ends, so a re-run of the sweep reloads them)
    auto load_slots = [&]() {
#pragma unroll
        for (int t = 0; t < RPL; ++t) {
            const int i = r + LPS * t;
            const bool ok = qok && i < bt;
            vr[t] = ok ? R[p0 + i + (size_t)col * L.ldw] : 0.0;
            xr[t] = ok ? X[p0 + i + (size_t)col * L.ldw] : 0.0;
            vi[t] = (CPLX && ok) ? R[p0 + i + (size_t)(col + 1) * L.ldw] : 0.0;
            xi[t] = (CPLX && ok) ? X[p0 + i + (size_t)(col + 1) * L.ldw] : 0.0;
        }
    };
    load_slots();
    const int eB0 = qok ? eB[q] : 0;
    int e = eB0;
    auto xmax_bound = [&]() {
        int b = kNegInfLog;
#pragma unroll
        for (int t = 0; t < RPL; ++t) b = max(b, lb2(xr[t], xi[t]));
        return group_max_int<LPS>(b);
    };
    int bx = xmax_bound();
    auto rescale = [&](int sq, double& ar, double& ai) {
#pragma unroll
        for (int t = 0; t < RPL; ++t) {
            xr[t] = scalbn(xr[t], -sq);
            if (CPLX) xi[t] = scalbn(xi[t], -sq);
        }
        ar = scalbn(ar, -sq);
        if (CPLX) ai = scalbn(ai, -sq);
        bx -= sq;
        e += sq;
    };

    // ---------------- phase 1: sweep k = bt-1 .. 1 -----------------------
    // Step k forms the rotation of the pivot row k (lane k % LPS, slot
    // k / LPS) lane-parallel: one FP64 multiply gives c, s and x(k)/phi in
    // different lanes of the group and one more gives a and b, each followed
    // by a shuffle, instead of every lane computing every scalar.  The rows
    // above are then updated: the slot that holds row k-1 (the next pivot) at
    // once, the slots below it one step later, in the same instruction stream
    // as the next rotation, whose dependency chain would otherwise leave the
    // FP64 pipe idle.
    // The sweep runs first with the unscaled, unprotected rotation and no
    // per-step decision: each step only records, with integer tests of
    // exponent fields, whether the overflow scaling of phi or a protection
    // step (ProtectDivision / ProtectUpdate) could be needed (conservative
    // tests).  If any lane recorded one, the tile's rows are reloaded and the
    // sweep runs again the careful way, where every step decides for the
    // whole warp and recomputes the rotation with scaling and protection
    // when needed; that gives the first run's values whenever nothing
    // rescales.
    double* s_d = sm + 5 * br;   // h(i,i) - Re(lambda): the shifted diagonal
    double* s_h2 = sm + 6 * br;  // h(k,k-1)^2, the rotation's constant term
    for (int i = r; i + 1 < bt; i += LPS) s_d[i] = Hs[(i + 1) * br + i] - lre;
    for (int k = r; k < bt; k += LPS) s_h2[k] = Hs[(size_t)k * br + k] * Hs[(size_t)k * br + k];
    __syncwarp();
    const int role = r;
    // fast-path exponent bound, integer only: floor(log2|v|) + 1 for normal v;
    // for zero and subnormal v the bound of the smallest normal number
    auto lbf = [](double v) {
        const int ex = (int)((__double_as_longlong(v) >> 52) & 0x7FF);
        return max(ex, 1) - 1022;
    };
    auto lbf2 = [&](double a, double b) { return CPLX ? max(lbf(a), lbf(b)) + 1 : lbf(a); };

    auto sweep = [&](auto FASTc) -> bool {
        constexpr bool FAST = decltype(FASTc)::value;
        bool bad = false;  // FAST: some step may have needed the careful treatment
        // the rotation waiting for the slots below the pivot slot (identity at first)
        double p_ar = 0.0, p_ai = 0.0, p_bR = 0.0, p_bI = 0.0, p_cr = 0.0, p_ci = 0.0, p_s = 1.0;
        const double* p_col = Hs;

        auto apply_pending = [&](auto NPc) {
            constexpr int NP = decltype(NPc)::value;
#pragma unroll
            for (int t = 0; t < NP; ++t) {
                const double tr = p_col[r + LPS * t];
                if (CPLX) {
                    xr[t] = fma(-p_ar, vr[t], fma(p_ai, vi[t], fma(p_bR, tr, xr[t])));
                    xi[t] = fma(-p_ar, vi[t], fma(-p_ai, vr[t], fma(p_bI, tr, xi[t])));
                    const double nvr = fma(p_cr, tr, p_s * vr[t]);
                    const double nvi = fma(p_ci, tr, p_s * vi[t]);
                    vr[t] = nvr;
                    vi[t] = nvi;
                } else {
                    xr[t] = fma(-p_ar, vr[t], fma(p_bR, tr, xr[t]));
                    vr[t] = fma(p_cr, tr, p_s * vr[t]);
                }
            }
        };

        // one step; TK = slot of the pivot row k, PEEL = the step with k % LPS == 0
        // (row k-1 then sits in slot TK-1)
        auto step = [&](auto TKc, auto PEELc, int rk) {
            constexpr int TK = decltype(TKc)::value;
            constexpr bool PEEL = decltype(PEELc)::value;
            constexpr int US = PEEL ? TK - 1 : TK;  // slot of row k-1
            const int k = LPS * TK + rk;
            const int src = gbase | rk;
            const double vkr = __shfl_sync(kFull, vr[TK], src);
            const double xkr = __shfl_sync(kFull, xr[TK], src);
            const double vki = CPLX ? __shfl_sync(kFull, vi[TK], src) : 0.0;
            const double xki = CPLX ? __shfl_sync(kFull, xi[TK], src) : 0.0;
            const double* Hcol = Hs + (size_t)k * br;  // h(:, k-1) of the tile
            const double hs = Hcol[k];                 // h(k, k-1)
            apply_pending(std::integral_constant<int, TK>{});

            // rotation (eq. "givens" / "cgivens"): 1/phi = rsqrt(h^2 + |v|^2)
            const double h2 = s_h2[k];
            const double ss = CPLX ? fma(vkr, vkr, fma(vki, vki, h2)) : fma(vkr, vkr, h2);
            const double rr = rsqrt(ss);
            double m1;
            const double nhs = negd(hs);
            if (CPLX)
                m1 = role == 0 ? vkr : role == 1 ? vki : role == 2 ? nhs : role == 3 ? xkr : xki;
            else
                m1 = role == 0 ? vkr : role == 1 ? nhs : xkr;
            const double f1 = m1 * rr;
            double cr = __shfl_sync(kFull, f1, gbase);
            double ci = CPLX ? __shfl_sync(kFull, f1, gbase | 1) : 0.0;
            double s = __shfl_sync(kFull, f1, gbase | (CPLX ? 2 : 1));
            double xkr1 = __shfl_sync(kFull, f1, gbase | (CPLX ? 3 : 2));
            double xki1 = CPLX ? __shfl_sync(kFull, f1, gbase | 4) : 0.0;
            // a = x(k) conj(c), b = x(k) s
            double f2;
            if (CPLX) {
                const double u0 = (role & 1) ? xki1 : xkr1;
                const double v0 = role < 2 ? cr : s;
                const double u1 = role == 0 ? xki1 : role == 1 ? negd(xkr1) : 0.0;
                const double v1 = role < 2 ? ci : 0.0;
                f2 = fma(u0, v0, u1 * v1);
            } else {
                f2 = xkr1 * (role == 0 ? cr : s);
            }
            double ar = __shfl_sync(kFull, f2, gbase);
            double ai = CPLX ? __shfl_sync(kFull, f2, gbase | 1) : 0.0;
            double bR = __shfl_sync(kFull, f2, gbase | (CPLX ? 2 : 1));
            double bI = CPLX ? __shfl_sync(kFull, f2, gbase | 3) : 0.0;

            if constexpr (FAST) {
                // integer tests only: phi^2 outside [2^-1000, 2^1000] (the
                // squares need the power-of-two prescale), |x(k)/phi| or the
                // update bound at or above 2^omega (a protection step)
                const int es = (int)((__double_as_longlong(ss) >> 52) & 0x7FF);
                bool need = es < 23 || es > 2022;
                if (robust) {
                    const int lx = lbf2(xkr1, xki1);
                    const int nb = max(bx, LRb + lx) + 1;
                    need = need || lx >= om || nb > om;
                    bx = nb;
                }
                bad = bad || need;
            } else {
                int eh = max(lbound(hs), lbound(vkr));
                if (CPLX) eh = max(eh, lbound(vki));
                bool need = eh > 500 || eh < -500;
                int nb = 0;
                if (robust) {
                    const int sq = lb2(xkr, xki) + lbound(rr) - om;  // ProtectDivision
                    nb = max(bx, LRb + lb2(xkr1, xki1)) + 1;          // ProtectUpdate
                    need = need || sq > 0 || nb > om;
                }
                if (__any_sync(kFull, need)) {
                    // careful step: phi with a power-of-two prescale against
                    // overflow, then the protections with rescaling of x
                    double hsc = hs, vsr = vkr, vsi = vki, sc = 1.0;
                    if (eh > 500 || eh < -500) {
                        sc = exact_pow2(min(-eh, 1023));  // eh in [-1073, 1024]: 2^-eh, finite
                        hsc *= sc;
                        vsr *= sc;
                        if (CPLX) vsi *= sc;
                    }
                    const double ss2 =
                        CPLX ? fma(vsr, vsr, fma(vsi, vsi, hsc * hsc)) : fma(vsr, vsr, hsc * hsc);
                    const double rr2 = rsqrt(ss2);
                    cr = vsr * rr2;
                    s = -hsc * rr2;
                    ci = CPLX ? vsi * rr2 : 0.0;
                    const double rinv = rr2 * sc;
                    xkr1 = xkr;
                    xki1 = xki;
                    if (robust) {
                        const int sq = lb2(xkr1, xki1) + lbound(rinv) - om;
                        if (sq > 0) rescale(sq, xkr1, xki1);
                    }
                    xkr1 *= rinv;
                    if (CPLX) xki1 *= rinv;
                    if (robust) {
                        const int lx = lb2(xkr1, xki1);
                        int nb2 = max(bx, LRb + lx) + 1;
                        const bool refine = nb2 > om;
                        // the exact maximum is a shuffle over the group: every lane of
                        // the warp takes part whenever any group needs it
                        if (__any_sync(kFull, refine)) {
                            const int bexact = xmax_bound();
                            if (refine) {
                                bx = max(bexact, lx);
                                nb2 = max(bx, LRb + lx) + 1;
                                if (nb2 > om) {
                                    rescale(nb2 - om, xkr1, xki1);
                                    nb2 = om;
                                }
                            }
                        }
                        bx = nb2;
                    }
                    ar = CPLX ? fma(xkr1, cr, xki1 * ci) : xkr1 * cr;
                    ai = CPLX ? fma(xki1, cr, -xkr1 * ci) : 0.0;
                    bR = xkr1 * s;
                    bI = CPLX ? xki1 * s : 0.0;
                } else if (robust) {
                    bx = nb;
                }
            }
            if (L.compact) {
                // the canonical rotation (what compact storage recovers); a and b
                // do not change with the flip
                const unsigned long long f = canon_mask<CPLX>(cr, ci, s);
                cr = flip_if(cr, f);
                ci = flip_if(ci, f);
                s = flip_if(s, f);
                xkr1 = flip_if(xkr1, f);
                xki1 = flip_if(xki1, f);
            }
            // row k is final
            if (r == rk) {
                xr[TK] = xkr1;
                if (CPLX) xi[TK] = xki1;
                s_cr[k] = cr;
                if (CPLX) s_ci[k] = ci;
                s_s[k] = s;
            }
            // slot US now (it holds row k-1, whose t entry is the shifted
            // diagonal h(k-1,k-1) - lambda): x -= a v - b t, v = c t + s v
            {
                const int i = r + LPS * US;
                const bool dg = i == k - 1;
                if (PEEL || r < rk) {
                    const double tr = dg ? s_d[i] : Hcol[i];
                    if (CPLX) {
                        const double dli = dg ? lim : 0.0;  // t = tr - i lim on the diagonal
                        xr[US] = fma(bI, dli, fma(-ar, vr[US], fma(ai, vi[US], fma(bR, tr, xr[US]))));
                        xi[US] = fma(-bR, dli, fma(-ar, vi[US], fma(-ai, vr[US], fma(bI, tr, xi[US]))));
                        const double nvr = fma(ci, dli, fma(cr, tr, s * vr[US]));
                        const double nvi = fma(-cr, dli, fma(ci, tr, s * vi[US]));
                        vr[US] = nvr;
                        vi[US] = nvi;
                    } else {
                        xr[US] = fma(-ar, vr[US], fma(bR, tr, xr[US]));
                        vr[US] = fma(cr, tr, s * vr[US]);
                    }
                }
            }
            // the slots below US take this rotation at the next step
            p_ar = ar;
            p_ai = ai;
            p_bR = bR;
            p_bI = bI;
            p_cr = cr;
            p_ci = ci;
            p_s = s;
            p_col = Hcol;
        };

        auto block = [&](auto TKc) {
            constexpr int TK = decltype(TKc)::value;
            for (int rk = LPS - 1; rk >= 1; --rk) {
                if (LPS * TK + rk >= bt) continue;
                step(TKc, std::false_type{}, rk);
            }
            if constexpr (TK >= 1) {
                if (LPS * TK < bt) step(TKc, std::true_type{}, 0);
            }
        };
        static_down<RPL - 1>(block);
        return bad;
    };
    if (__any_sync(kFull, sweep(std::true_type{}))) {
        load_slots();
        e = eB0;
        bx = xmax_bound();
        sweep(std::false_type{});
    }

    // ---------------- row 0: left rotation or final pivot ----------------
    {
        double v0r = __shfl_sync(kFull, vr[0], gbase);
        double v0i = CPLX ? __shfl_sync(kFull, vi[0], gbase) : 0.0;
        double x0r = __shfl_sync(kFull, xr[0], gbase);
        double x0i = CPLX ? __shfl_sync(kFull, xi[0], gbase) : 0.0;
        double c0r, c0i, s0;
        if (p0 > 0) {
            double hs = Hs[0], vsr = v0r, vsi = v0i, sc = 1.0;  // h(p0, p0-1)
            int eh = max(lbound(hs), lbound(vsr));
            if (CPLX) eh = max(eh, lbound(vsi));
            if (eh > 500 || eh < -500) {
                sc = exact_pow2(min(-eh, 1023));  // eh in [-1073, 1024]: 2^-eh, finite
                hs *= sc;
                vsr *= sc;
                vsi *= sc;
            }
            const double ss = CPLX ? fma(vsr, vsr, fma(vsi, vsi, hs * hs)) : fma(vsr, vsr, hs * hs);
            const double rr = rsqrt(ss);
            c0r = vsr * rr;
            c0i = CPLX ? vsi * rr : 0.0;
            s0 = -hs * rr;
            const double rinv = rr * sc;
            if (robust) {
                const int sq = lb2(x0r, x0i) + lbound(rinv) - om;
                if (sq > 0) rescale(sq, x0r, x0i);
            }
            x0r *= rinv;
            x0i *= rinv;
            if (L.compact) {
                const unsigned long long f = canon_mask<CPLX>(c0r, c0i, s0);
                c0r = flip_if(c0r, f);
                c0i = flip_if(c0i, f);
                s0 = flip_if(s0, f);
                x0r = flip_if(x0r, f);
                x0i = flip_if(x0i, f);
            }
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
                const int sq = lb2(x0r, x0i) - (lbound(pa) - 1) - om;
                if (sq > 0) rescale(sq, x0r, x0i);
            }
            if (CPLX) {
                // Smith's division (x0r + i x0i) / (pr + i pi)
                double nr, ni;
                if (fabs(pr) >= fabs(pi)) {
                    double rt = pi / pr, d = pr + pi * rt;
                    nr = (x0r + x0i * rt) / d;
                    ni = (x0i - x0r * rt) / d;
                } else {
                    double rt = pr / pi, d = pi + pr * rt;
                    nr = (x0r * rt + x0i) / d;
                    ni = (x0i * rt - x0r) / d;
                }
                x0r = nr;
                x0i = ni;
            } else {
                x0r /= pr;
            }
        }
        if (r == 0) {
            xr[0] = x0r;
            if (CPLX) xi[0] = x0i;
            s_cr[0] = c0r;
            s_ci[0] = c0i;
            s_s[0] = s0;
        }
    }

    // ---------------- outputs of phase 1 ---------------------------------
#pragma unroll
    for (int t = 0; t < RPL; ++t) {
        const int i = r + LPS * t;
        if (i < bt) {
            s_xr[i] = xr[t];
            if (CPLX) s_xi[i] = xi[t];
            if (qok) {
                X[p0 + i + (size_t)col * L.ldw] = xr[t];
                if (CPLX) X[p0 + i + (size_t)(col + 1) * L.ldw] = xi[t];
            }
        }
    }
    __syncwarp();
    if (qok) {
        for (int i = r; i < bt; i += LPS) {
            const size_t gi = (size_t)q * L.n + p0 + i;
            if (L.compact) {  // Stewart's storage (Sec. 4.4)
                if (CPLX) givens_pack_cplx(s_cr[i], s_ci[i], s_s[i], Cr[gi], Ci[gi]);
                else Cr[gi] = givens_pack_real(s_cr[i], s_s[i]);
            } else {
                Cr[gi] = s_cr[i];
                Sv[gi] = s_s[i];
                if (CPLX) Ci[gi] = s_ci[i];
            }
        }
        if (r == 0) etile[(size_t)J * L.m + q] = e;
    }
    __syncwarp();
    if (p0 == 0) return;

    // ---------------- phase 2: [Z'|W] by a parallel scan ------------------
    // tau_k = s_k tau_{k-1} + conj(c_k) x_k (tau_0 = conj(c_0) x_0) is an
    // affine recurrence and P_k = prod_{i<=k} s_i a product recurrence: each
    // lane composes the maps of a contiguous chunk of rows, the group scans
    // the chunks, then each lane emits Z'(k) = c_k tau_{k-1} - s_k x_k
    // (Z'(0) = rho' = -s_0 x_0) and w_k = c_k P_{k-1} (w_0 = c_0) for its rows.
    double* s_zr = s_xr;  // Z' and W overwrite the x and c scratch in place
    double* s_zi = s_xi;
    const int cs = (bt + LPS - 1) / LPS;
    const int a0 = min(bt, r * cs), a1 = min(bt, a0 + cs);
    double mA = 1.0, mBr = 0.0, mBi = 0.0, mP = 1.0;
    for (int k = a0; k < a1; ++k) {
        const double ckr = s_cr[k], sk = s_s[k], xkr = s_xr[k];
        const double cki = CPLX ? s_ci[k] : 0.0, xki = CPLX ? s_xi[k] : 0.0;
        const double gr = CPLX ? fma(ckr, xkr, cki * xki) : ckr * xkr;
        const double gi = CPLX ? fma(ckr, xki, -cki * xkr) : 0.0;
        const double a = k == 0 ? 0.0 : sk;
        mA *= a;
        mBr = fma(a, mBr, gr);
        if (CPLX) mBi = fma(a, mBi, gi);
        mP *= sk;
    }
    // inclusive scan over the group (earlier chunks applied first)
#pragma unroll
    for (int o = 1; o < LPS; o <<= 1) {
        const double pA = __shfl_up_sync(kFull, mA, o, LPS);
        const double pBr = __shfl_up_sync(kFull, mBr, o, LPS);
        const double pBi = CPLX ? __shfl_up_sync(kFull, mBi, o, LPS) : 0.0;
        const double pP = __shfl_up_sync(kFull, mP, o, LPS);
        if (r >= o) {
            mBr = fma(mA, pBr, mBr);
            if (CPLX) mBi = fma(mA, pBi, mBi);
            mA *= pA;
            mP *= pP;
        }
    }
    double tr = __shfl_up_sync(kFull, mBr, 1, LPS);  // tau entering the chunk
    double ti = CPLX ? __shfl_up_sync(kFull, mBi, 1, LPS) : 0.0;
    double P = __shfl_up_sync(kFull, mP, 1, LPS);     // prod of s_i before the chunk
    if (r == 0) {
        tr = 0.0;
        ti = 0.0;
        P = 1.0;
    }
    double zmax = 0.0;
    for (int k = a0; k < a1; ++k) {
        const double ckr = s_cr[k], sk = s_s[k], xkr = s_xr[k];
        const double cki = CPLX ? s_ci[k] : 0.0, xki = CPLX ? s_xi[k] : 0.0;
        double zr, zi;
        if (k == 0) {
            zr = -sk * xkr;
            zi = CPLX ? -sk * xki : 0.0;
            tr = CPLX ? fma(ckr, xkr, cki * xki) : ckr * xkr;
            ti = CPLX ? fma(ckr, xki, -cki * xkr) : 0.0;
        } else {
            zr = CPLX ? fma(ckr, tr, fma(-cki, ti, -sk * xkr)) : fma(ckr, tr, -sk * xkr);
            zi = CPLX ? fma(ckr, ti, fma(cki, tr, -sk * xki)) : 0.0;
            const double ntr = CPLX ? fma(sk, tr, fma(ckr, xkr, cki * xki)) : fma(sk, tr, ckr * xkr);
            const double nti = CPLX ? fma(sk, ti, fma(ckr, xki, -cki * xkr)) : 0.0;
            tr = ntr;
            ti = nti;
        }
        s_zr[k] = zr;
        if (CPLX) s_zi[k] = zi;
        zmax = fmax(zmax, CPLX ? fmax(fabs(zr), fabs(zi)) : fabs(zr));
        s_cr[k] = ckr * P;  // w_k = c_k prod_{i<k} s_i (w_0 = c_0)
        if (CPLX) s_ci[k] = cki * P;
        P *= sk;
    }
    zmax = group_max<LPS>(zmax);
    const int last = gbase + (bt - 1) / cs;
    const double zbr_r = __shfl_sync(kFull, tr, last);
    const double zbr_i = CPLX ? __shfl_sync(kFull, ti, last) : 0.0;
    const double pi_ = __shfl_sync(kFull, P, last);
    __syncwarp();
    if (r == 0) {
        const double rhor = s_zr[0], rhoi = CPLX ? s_zi[0] : 0.0;
        // consistent exponent for the rows above (Alg. "robust-tile-update"):
        // B_new = B 2^(eB-e) - (A Z' + R~ z_br - lambda rho' e_last) 2^(ex-e)
        const int ex = e;
        int enew = max(eB0, ex);
        if (robust && qok) {
            const double An = bits_to_double(anorm[J]) * hscale;
            const double bm = bits_to_double(bmaxv[q]);
            const double rm = bits_to_double(rmaxv[q]);
            const double la = fabs(lre) + fabs(lim);
            const double rh = fabs(rhor) + fabs(rhoi);
            const double zb = fabs(zbr_r) + fabs(zbr_i);
            const int lt = max(log2_bound(An) + log2_bound(zmax) + cadd,
                               max(log2_bound(rm) + cadd + log2_bound(zb),
                                   log2_bound(la) + log2_bound(rh))) + 2;
            const int lbm = log2_bound(bm) + cadd;
            const int need = max(lbm + eB0, lt + ex) + 1 - om;
            enew = max(enew, need);
        }
        const double fB = ldexp(1.0, eB0 - enew);
        const double fZ = ldexp(1.0, ex - enew);
        if (qok) {
            eB[q] = enew;
            bmaxv[q] = 0ull;
            rmaxv[q] = 0ull;
            Epi E;
            E.fB = fB;
            E.pi = pi_;
            E.zbr_re = zbr_r * fZ;
            E.zbr_im = zbr_i * fZ;
            // lambda' rho' fZ and lambda' c_0 (s_cr[0] = w_0 = c_0)
            E.cz_re = (lre * rhor - lim * rhoi) * fZ;
            E.cz_im = (lre * rhoi + lim * rhor) * fZ;
            E.cw_re = lre * s_cr[0] - lim * s_ci[0];
            E.cw_im = lre * s_ci[0] + lim * s_cr[0];
            epi[q] = E;
        }
        s_s[0] = fZ * hscale;  // reuse: factor for Z'
    }
    __syncwarp();
    const double fz = s_s[0];
    const size_t ldzw = 2 * (size_t)L.ncolp;
    if (!L.oz) {
        if (qok) {
            for (int k = r; k < bt; k += LPS) {
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
        }
    } else {
        // [Z'|W] as BF16 digits with one exponent per product column
        __nv_bfloat16* zd = ws<__nv_bfloat16>(work, L.off_zwd);
        int* zf = ws<int>(work, L.off_zwf);
        const int ncols = CPLX ? 4 : 2;
        for (int cc = 0; cc < ncols; ++cc) {
            const double* srcv = (cc & 1) ? ((cc & 2) ? s_ci : s_cr) : ((cc & 2) ? s_zi : s_zr);
            const double f = (cc & 1) ? hscale : fz;
            double m = 0.0;
            for (int k = r; k < bt; k += LPS) m = fmax(m, fabs(srcv[k] * f));
            m = group_max<LPS>(m);  // every lane takes part (shuffle)
            if (!qok) continue;
            const int es = oz::scale_exponent(m);
            const int gc = 2 * col + cc;
            if (r == 0) zf[gc] = es;
            for (int k = r; k < br; k += LPS) {
                int d[oz::kS];
                oz::split_digits(k < bt ? srcv[k] * f : 0.0, es, d);
#pragma unroll
                for (int i = 0; i < oz::kS; ++i)
                    zd[((size_t)i * ldzw + gc) * br + k] = __float2bfloat16_rn((float)d[i]);
            }
        }
    }
}

__device__ inline uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

template <int LPSC, int RPLC, int LPSR, int RPLR>
__global__ void __launch_bounds__(32)
k_diag(Layout L, void* work, int J, int robust, int om, int nbc, long long wait_limit) {
    extern __shared__ __align__(128) double smem[];
    __shared__ __align__(8) unsigned long long mbar;
    DevState* st = ws<DevState>(work, L.off_state);
    if (st->status < 0) return;
    const int br = L.br;
    const int lane = threadIdx.x;
    const int p0 = tile_start(L, J);
    const int bt = tile_height(L, J);
    double* Hs = smem;  // [br cols][br rows], column cc = global column p0-1+cc
    // one bulk copy of the staged (contiguous, prescaled) tile
    const double* tile = ws<double>(work, L.off_dt) + (size_t)J * br * br;
    const uint32_t bytes = (uint32_t)((size_t)bt * br * sizeof(double));
    const uint32_t mb = smem_u32(&mbar);
    if (lane == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
    }
    __syncwarp();
    const long long t0 = clock64();  // the wait is bounded from the copy's issue
    if (lane == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mb), "r"(bytes));
        asm volatile(
            "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                smem_u32(Hs)),
            "l"(tile), "r"(bytes), "r"(mb)
            : "memory");
    }
    // bounded wait: once wait_limit cycles have passed (checked before every
    // poll) the error is recorded, and the block keeps waiting, at most
    // kDrainCycles more, only so that the copy in flight lands before it
    // returns
    bool expired = false;
    for (;;) {
        const long long el = clock64() - t0;
        if (!expired && el >= wait_limit) {
            expired = true;
            if (lane == 0) set_error(st, -6);  // HSEIN_ETIMEOUT
        }
        if (expired && el >= wait_limit + kDrainCycles) return;
        uint32_t done = 0;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mb)
            : "memory");
        if (done) break;
    }
    if (expired) return;
    const int b = blockIdx.x;
    if (b < nbc) {
        constexpr int G = 32 / LPSC;
        const int g = lane / LPSC;
        const int q = G * b + g;
        double* scratch = smem + (size_t)br * br + (size_t)g * 7 * br;
        tile_group<LPSC, RPLC, true>(L, work, Hs, J, p0, bt, q, q < L.mc, robust, om, scratch);
    } else {
        constexpr int G = 32 / LPSR;
        const int g = lane / LPSR;
        const int q = L.mc + G * (b - nbc) + g;
        double* scratch = smem + (size_t)br * br + (size_t)g * 7 * br;
        tile_group<LPSR, RPLR, false>(L, work, Hs, J, p0, bt, q, q < L.m, robust, om, scratch);
    }
}

// stage every diagonal tile H(J, J^-) once per solve: contiguous, column
// cc = global column p0-1+cc, prescaled, zero below the subdiagonal (those
// entries of H are not read)
__global__ void k_stage_tiles(Layout L, void* work, const double* __restrict__ H, int ldh) {
    const DevState* st = ws<DevState>(work, L.off_state);
    if (st->status < 0) return;
    const int J = blockIdx.x;
    const int br = L.br;
    const int p0 = tile_start(L, J), bt = tile_height(L, J);
    const double hscale = st->hscale;
    double* dt = ws<double>(work, L.off_dt) + (size_t)J * br * br;
    for (int idx = threadIdx.x; idx < bt * br; idx += blockDim.x) {
        const int cc = idx / br, i = idx % br;
        const int gc = p0 - 1 + cc;
        double v = 0.0;
        if (i < bt && gc >= 0 && i <= cc) v = H[p0 + i + (size_t)gc * ldh] * hscale;
        dt[idx] = v;
    }
}

}  // namespace

void launch_stage_tiles(const Layout& L, void* work, const double* H, int ldh, cudaStream_t s) {
    k_stage_tiles<<<L.N, 256, 0, s>>>(L, work, H, ldh);
}

// lanes per shift: complex shifts take a whole warp; real shifts take a whole
// warp too while one warp per shift fits on the GPU's SM sub-partitions (a
// warp's step is bound by its own FP64 issue, so fewer shifts per warp give
// shorter steps: n = 512, 64 shifts, 0.71 -> 0.61 ms per step), half of one
// otherwise, or a quarter of one when half-warps would give more warps than
// the GPU has sub-partitions: two warps on one sub-partition take longer per
// step than one warp with twice the shifts (n = 8192, 2048 real shifts:
// 18.9 -> 13.5 ms per solve).  One or four shifts per warp need tile heights
// up to 64.
constexpr int kLpsC = 32;

int diag_lanes_real(const Layout& L, int num_sms) {
    if (L.br <= 64 && L.mc + L.mr <= 4 * num_sms) return 32;
    const int warps_half = L.mc + (L.mr + 1) / 2;
    return (L.br <= 64 && warps_half > 4 * num_sms) ? 8 : 16;
}

static int pow2_at_least(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

template <int RC, int RR, int LPSR>
static void launch_t(const Layout& L, void* work, int J, int robust, int om, int nbc, int grid,
                     size_t smem, long long wl, cudaStream_t s) {
    k_diag<kLpsC, RC, LPSR, RR><<<grid, 32, smem, s>>>(L, work, J, robust, om, nbc, wl);
}

// the staged tile, then 7 br doubles of scratch per shift group of a warp
static size_t diag_smem(int br, int lpsr) {
    return ((size_t)br * br + (size_t)(32 / lpsr) * 7 * br) * sizeof(double);
}

void launch_diag(const Layout& L, void* work, int J, int robust, int omega_log2,
                 long long wait_limit, cudaStream_t s) {
    const int lpsr = L.lps_real;
    const int nbc = (L.mc + (32 / kLpsC) - 1) / (32 / kLpsC);
    const int nbr = (L.mr + (32 / lpsr) - 1) / (32 / lpsr);
    const size_t smem = diag_smem(L.br, lpsr);
    const int grid = nbc + nbr;
    const int om = omega_log2;
    // rows per lane, rounded up to a power of two: complex br/32, real br/lpsr
    if (lpsr == 32) {
        if (L.br <= 32) launch_t<1, 1, 32>(L, work, J, robust, om, nbc, grid, smem, wait_limit, s);
        else launch_t<2, 2, 32>(L, work, J, robust, om, nbc, grid, smem, wait_limit, s);
        return;
    }
    if (lpsr == 8) {
        switch (pow2_at_least((L.br + 7) / 8)) {
            case 1: launch_t<1, 1, 8>(L, work, J, robust, om, nbc, grid, smem, wait_limit, s); break;
            case 2: launch_t<1, 2, 8>(L, work, J, robust, om, nbc, grid, smem, wait_limit, s); break;
            case 4: launch_t<1, 4, 8>(L, work, J, robust, om, nbc, grid, smem, wait_limit, s); break;
            default: launch_t<2, 8, 8>(L, work, J, robust, om, nbc, grid, smem, wait_limit, s); break;
        }
        return;
    }
    switch (pow2_at_least((L.br + 15) / 16)) {
        case 1: launch_t<1, 1, 16>(L, work, J, robust, om, nbc, grid, smem, wait_limit, s); break;
        case 2: launch_t<1, 2, 16>(L, work, J, robust, om, nbc, grid, smem, wait_limit, s); break;
        case 4: launch_t<2, 4, 16>(L, work, J, robust, om, nbc, grid, smem, wait_limit, s); break;
        default: launch_t<4, 8, 16>(L, work, J, robust, om, nbc, grid, smem, wait_limit, s); break;
    }
}

// dynamic shared memory above 48 KB needs an opt-in per kernel; the limit is
// per kernel instance, not per plan, so each instance is configured for the
// largest tile height it serves (plans of different heights coexist)
cudaError_t diag_configure(int br) {
    const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaSuccess;
    switch (pow2_at_least((br + 15) / 16)) {
        case 1: e = cudaFuncSetAttribute(k_diag<kLpsC, 1, 16, 1>, a, (int)diag_smem(16, 16)); break;
        case 2: e = cudaFuncSetAttribute(k_diag<kLpsC, 1, 16, 2>, a, (int)diag_smem(32, 16)); break;
        case 4: e = cudaFuncSetAttribute(k_diag<kLpsC, 2, 16, 4>, a, (int)diag_smem(64, 16)); break;
        default: e = cudaFuncSetAttribute(k_diag<kLpsC, 4, 16, 8>, a, (int)diag_smem(kMaxBr, 16)); break;
    }
    if (e != cudaSuccess || br > 64) return e;
    e = br <= 32 ? cudaFuncSetAttribute(k_diag<kLpsC, 1, 32, 1>, a, (int)diag_smem(32, 32))
                 : cudaFuncSetAttribute(k_diag<kLpsC, 2, 32, 2>, a, (int)diag_smem(64, 32));
    if (e != cudaSuccess) return e;
    switch (pow2_at_least((br + 7) / 8)) {
        case 1: return cudaFuncSetAttribute(k_diag<kLpsC, 1, 8, 1>, a, (int)diag_smem(8, 8));
        case 2: return cudaFuncSetAttribute(k_diag<kLpsC, 1, 8, 2>, a, (int)diag_smem(16, 8));
        case 4: return cudaFuncSetAttribute(k_diag<kLpsC, 1, 8, 4>, a, (int)diag_smem(32, 8));
        default: return cudaFuncSetAttribute(k_diag<kLpsC, 2, 8, 8>, a, (int)diag_smem(64, 8));
    }
}

}  // namespace hsein
