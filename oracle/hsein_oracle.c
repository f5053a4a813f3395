/*
 * hsein_oracle.c -- plain, slow FP64 CPU oracle for the robust multi-shift
 * solve of shifted Hessenberg systems (Schwarz, "Robust level-3 BLAS Inverse
 * Iteration from the Hessenberg Matrix", arXiv 2101.05063).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code, header or constant with the CUDA
 * library; it is an independent restatement of the method.
 *
 * What it computes, per shift lambda (real or complex):
 *   x = (H - lambda I)^{-1} b, normalized to ||x||_2 = 1, by Henry's RQ
 *   algorithm (Alg. "henry", Sec. 2.2): a column-by-column sweep of Givens
 *   rotations from the right, fused with column-oriented back substitution,
 *   followed by the Givens backtransform (eq. "backtransform", Sec. 3.2).
 *   Robustness (Sec. 4.1) is added the way the paper describes it: the whole
 *   solution vector carries one scale factor 2^-e (an integer exponent e),
 *   every division is guarded by ProtectDivision and every linear update by
 *   ProtectUpdate, and the final vector is normalized with a DNRM2-style
 *   scaled 2-norm before the backtransform (Alg. "consistency-scaling").
 *   Complex shifts use the complex Givens rotation of eq. "cgivens"
 *   (c complex, s real) and complex arithmetic (Sec. 4.3).
 *   Convergence follows Varah's criterion as restated in Sec. 4.2.
 *
 * There are no tiles here: the tiled algorithm equals Henry's algorithm in
 * exact arithmetic (end of Sec. 3.2), so the untiled form is the definition.
 *
 * Readings of passages the paper leaves open:
 *  - Givens sign: phi = +sqrt(h^2 + |v|^2) > 0, c = v/phi, s = -h/phi.
 *  - ProtectUpdate / ProtectDivision are cited but not printed (Sec. 4.1);
 *    the formulas below are derived from the no-overflow requirement with
 *    powers of two so that every rescaling is exact.
 *  - Scale factors are integer exponents, not doubles in (0,1].
 *  - An exactly singular (or tiny) final pivot |r11| < eps*||H||_inf is
 *    replaced by eps*||H||_inf carrying the pivot's sign (+ for 0), the
 *    small-pivot treatment LAPACK's inverse iteration documents.
 *  - The backtransform includes the final entry x(n) <- tau that Alg. "henry"
 *    and Alg. "consistency-scaling" omit.
 *  - eps = 2^-53 (unit roundoff).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <float.h>
#include <complex.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_EPS 0x1p-53

typedef double _Complex zdouble;

/* ---------------------------------------------------------------- helpers */

/* ||H||_inf: maximum absolute row sum of the n x n upper Hessenberg H. */
double oracle_hnorm_inf(int n, const double *H, int ldh)
{
    double best = 0.0;
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        int j0 = i > 0 ? i - 1 : 0;
        for (int j = j0; j < n; ++j) s += fabs(H[i + (size_t)j * ldh]);
        if (s > best) best = s;
    }
    return best;
}

/* smallest integer q with 2^q >= v, for v > 0 */
static int ceil_log2(double v)
{
    int ex;
    double m = frexp(v, &ex); /* v = m 2^ex, m in [0.5, 1) */
    return (m == 0.5) ? ex - 1 : ex;
}

/*
 * ProtectUpdate (Sec. 4.1): returns q >= 0 such that with xi = 2^-q the update
 * xi*b - t*(xi*x) cannot exceed omega in magnitude, where b bounds the vector
 * that is updated, t bounds the column it is updated with and x is the scalar
 * multiplier; b, t, x <= omega is assumed.
 *   x <= 1: t*x <= omega - b  -> 1; otherwise 1/2.
 *   x >  1: t <= (omega-b)/x  -> 1; otherwise 2^-(ceil(log2 x)+1) <= 1/(2x).
 * In both rejected cases xi*b <= omega/2 and t*xi*x <= omega/2.
 */
static int protect_update(double b, double t, double x, double omega)
{
    if (x <= 1.0) {
        if (t * x <= omega - b) return 0;
        return 1;
    }
    if (t <= (omega - b) / x) return 0;
    return ceil_log2(x) + 1;
}

/*
 * ProtectDivision (Sec. 4.1): returns q >= 0 such that (2^-q b)/t <= omega for
 * b <= omega, t > 0.  Only a divisor below one can cause growth.
 */
static int protect_division(double b, double t, double omega)
{
    if (t < 1.0 && b > t * omega) return ceil_log2(b / (t * omega));
    return 0;
}

/* DNRM2-style scaled 2-norm of the real vector x (Alg. "consistency-scaling",
 * its norm loop): running maximum xmax and scaled sum t. */
static double scaled_nrm2(int n, const double *x, int stride)
{
    double xmax = 0.0, t = 0.0;
    for (int i = 0; i < n; ++i) {
        double a = fabs(x[(size_t)i * stride]);
        if (a == 0.0) continue;
        if (xmax < a) {
            double r = xmax / a;
            t = 1.0 + t * r * r;
            xmax = a;
        } else {
            double r = a / xmax;
            t += r * r;
        }
    }
    return xmax * sqrt(t);
}

/* the same for a complex vector: every real and imaginary part is one entry */
static double scaled_nrm2_z(int n, const zdouble *x)
{
    double xmax = 0.0, t = 0.0;
    for (int i = 0; i < 2 * n; ++i) {
        double a = fabs(((const double *)x)[i]);
        if (a == 0.0) continue;
        if (xmax < a) {
            double r = xmax / a;
            t = 1.0 + t * r * r;
            xmax = a;
        } else {
            double r = a / xmax;
            t += r * r;
        }
    }
    return xmax * sqrt(t);
}

/* Smith's complex division a / b (b != 0). */
static zdouble zdiv_smith(zdouble a, zdouble b)
{
    double ar = creal(a), ai = cimag(a), br = creal(b), bi = cimag(b);
    if (fabs(br) >= fabs(bi)) {
        double r = bi / br, d = br + bi * r;
        return ((ar + ai * r) / d) + I * ((ai - ar * r) / d);
    } else {
        double r = br / bi, d = bi + br * r;
        return ((ar * r + ai) / d) + I * ((ai * r - ar) / d);
    }
}

static double zabs(zdouble z) { return hypot(creal(z), cimag(z)); }

/* ------------------------------------------------------- real shift solve */

/*
 * Henry's RQ solve of (H - lambda I) x = 2^-e b for one real shift, with the
 * robust scaling described in the file header.  On return x holds the scaled
 * solution (true solution = x * 2^e), *e_out the exponent, and C[k], S[k] the
 * rotation G_k that combines columns k-1 and k (0-based; C[0]=1, S[0]=0 is the
 * padding of the top-left tile, Sec. 3.2).  robust=0 disables all protection
 * (used to show that unprotected solves overflow).  work: 2n doubles.
 * Returns 0, or 1 when the final pivot was replaced (A10 reading).
 */
int oracle_henry_real(int n, const double *H, int ldh, double lambda,
                      const double *b, double log2_omega, int robust,
                      double *x, int *e_out, double *C, double *S,
                      double *work)
{
    const double omega = ldexp(1.0, (int)log2_omega);
    const double hnorm = oracle_hnorm_inf(n, H, ldh);
    double *v = work, *rcol = work + n;
    int e = 0, replaced = 0;

    for (int i = 0; i < n; ++i) {
        x[i] = b[i];
        v[i] = H[i + (size_t)(n - 1) * ldh];
    }
    v[n - 1] -= lambda;

    for (int k = n - 1; k >= 1; --k) {
        /* Givens rotation with [h(k,k-1) v(k)] G^T = [0 phi] */
        double h = H[k + (size_t)(k - 1) * ldh];
        double phi = hypot(h, v[k]);
        double c = v[k] / phi, s = -h / phi;
        C[k] = c;
        S[k] = s;
        /* x(k) <- x(k) / r(k,k) with r(k,k) = phi */
        if (robust) {
            int q = protect_division(fabs(x[k]), phi, omega);
            if (q) {
                for (int i = 0; i < n; ++i) x[i] = ldexp(x[i], -q);
                e += q;
            }
        }
        x[k] /= phi;
        /* column k of R above the diagonal: -s*t + c*v, t = h(:,k-1) - lambda e_{k-1} */
        double rmax = 0.0, xmax = 0.0;
        for (int i = 0; i < k; ++i) {
            double t = H[i + (size_t)(k - 1) * ldh] - (i == k - 1 ? lambda : 0.0);
            rcol[i] = c * v[i] - s * t;
            if (fabs(rcol[i]) > rmax) rmax = fabs(rcol[i]);
            if (fabs(x[i]) > xmax) xmax = fabs(x[i]);
        }
        if (robust) {
            int q = protect_update(xmax, rmax, fabs(x[k]), omega);
            if (q) {
                for (int i = 0; i < n; ++i) x[i] = ldexp(x[i], -q);
                e += q;
            }
        }
        /* back substitution with the new column, then the next working column */
        for (int i = 0; i < k; ++i) {
            double t = H[i + (size_t)(k - 1) * ldh] - (i == k - 1 ? lambda : 0.0);
            x[i] -= x[k] * rcol[i];
            v[i] = c * t + s * v[i];
        }
    }
    C[0] = 1.0;
    S[0] = 0.0;
    double r11 = v[0];
    double small = ORACLE_EPS * hnorm;
    if (fabs(r11) < small) {
        r11 = copysign(small, r11);
        replaced = 1;
    }
    if (robust) {
        int q = protect_division(fabs(x[0]), fabs(r11), omega);
        if (q) {
            for (int i = 0; i < n; ++i) x[i] = ldexp(x[i], -q);
            e += q;
        }
    }
    x[0] /= r11;
    *e_out = e;
    return replaced;
}

/* Givens backtransform y = G_n^T(...(G_2^T x)) in place (eq. "backtransform"). */
void oracle_backtransform_real(int n, const double *C, const double *S, double *x)
{
    double tau = x[0];
    for (int k = 1; k < n; ++k) {
        double xk = x[k];
        x[k - 1] = C[k] * tau - S[k] * xk;
        tau = S[k] * tau + C[k] * xk;
    }
    x[n - 1] = tau;
}

/* ----------------------------------------------------- complex shift solve */

/*
 * Complex counterpart (Sec. 4.3): x, b are complex; C is complex, S real.
 * G_k^H = [[c, -s], [s, conj(c)]] on columns k-1, k; with h = h(k,k-1) real
 * and v(k) complex: r = sqrt(h^2 + |v(k)|^2), c = v(k)/r, s = -h/r gives
 * [h v(k)] G^H = [0 r].  Column k of R is -s*t + conj(c)*v and the next
 * working column is c*t + s*v.  The solution vector carries one exponent.
 */
int oracle_henry_cplx(int n, const double *H, int ldh, double lre, double lim,
                      const zdouble *b, double log2_omega, int robust,
                      zdouble *x, int *e_out, zdouble *C, double *S,
                      zdouble *work)
{
    const double omega = ldexp(1.0, (int)log2_omega);
    const double hnorm = oracle_hnorm_inf(n, H, ldh);
    const zdouble lambda = lre + I * lim;
    zdouble *v = work, *rcol = work + n;
    int e = 0, replaced = 0;

    for (int i = 0; i < n; ++i) {
        x[i] = b[i];
        v[i] = H[i + (size_t)(n - 1) * ldh];
    }
    v[n - 1] -= lambda;

    for (int k = n - 1; k >= 1; --k) {
        double h = H[k + (size_t)(k - 1) * ldh];
        double r = hypot(h, zabs(v[k]));
        zdouble c = v[k] / r;
        double s = -h / r;
        C[k] = c;
        S[k] = s;
        if (robust) {
            int q = protect_division(zabs(x[k]), r, omega);
            if (q) {
                for (int i = 0; i < n; ++i) x[i] = ldexp(creal(x[i]), -q) + I * ldexp(cimag(x[i]), -q);
                e += q;
            }
        }
        x[k] /= r;
        double rmax = 0.0, xmax = 0.0;
        for (int i = 0; i < k; ++i) {
            zdouble t = H[i + (size_t)(k - 1) * ldh] - (i == k - 1 ? lambda : 0.0);
            rcol[i] = conj(c) * v[i] - s * t;
            if (zabs(rcol[i]) > rmax) rmax = zabs(rcol[i]);
            if (zabs(x[i]) > xmax) xmax = zabs(x[i]);
        }
        if (robust) {
            int q = protect_update(xmax, rmax, zabs(x[k]), omega);
            if (q) {
                for (int i = 0; i < n; ++i) x[i] = ldexp(creal(x[i]), -q) + I * ldexp(cimag(x[i]), -q);
                e += q;
            }
        }
        for (int i = 0; i < k; ++i) {
            zdouble t = H[i + (size_t)(k - 1) * ldh] - (i == k - 1 ? lambda : 0.0);
            x[i] -= x[k] * rcol[i];
            v[i] = c * t + s * v[i];
        }
    }
    C[0] = 1.0;
    S[0] = 0.0;
    zdouble r11 = v[0];
    double small = ORACLE_EPS * hnorm;
    if (zabs(r11) < small) {
        double a = zabs(r11);
        r11 = (a > 0.0) ? r11 * (small / a) : small;
        replaced = 1;
    }
    if (robust) {
        int q = protect_division(zabs(x[0]), zabs(r11), omega);
        if (q) {
            for (int i = 0; i < n; ++i) x[i] = ldexp(creal(x[i]), -q) + I * ldexp(cimag(x[i]), -q);
            e += q;
        }
    }
    x[0] = zdiv_smith(x[0], r11);
    *e_out = e;
    return replaced;
}

/* complex backtransform: (y(k-1), y(k)) <- (c tau - s y(k), s tau + conj(c) y(k)) */
void oracle_backtransform_cplx(int n, const zdouble *C, const double *S, zdouble *x)
{
    zdouble tau = x[0];
    for (int k = 1; k < n; ++k) {
        zdouble xk = x[k];
        x[k - 1] = C[k] * tau - S[k] * xk;
        tau = S[k] * tau + conj(C[k]) * xk;
    }
    x[n - 1] = tau;
}

/* ------------------------------------------------------------- the driver */

/*
 * Full oracle for m shifts (wr[l] + i*wi[l]; wi[l] != 0 marks a complex shift,
 * of which only one member of the conjugate pair is passed).  Column layout of
 * B and X: a real shift owns one column, a complex shift two adjacent columns
 * [re, im], in input order.  B == NULL selects the starting vector rho*e with
 * rho = eps*||H||_inf (Sec. 4.2).  On return X holds unit-norm eigenvector
 * approximations (zeroed where not converged), status[l] = 0 converged,
 * 1 not converged; exps[l] the scale exponent of the solve (may be NULL).
 * Varah's criterion (Sec. 4.2): ||x1||_2 / ||x0||_2 > 1/(10 n ||H||_inf eps),
 * evaluated in log2 with the exponent so that nothing overflows.
 * nthreads <= 0 uses the OpenMP default.
 */
int oracle_hsein(int n, const double *H, int ldh, int m, const double *wr,
                 const double *wi, const double *B, int ldb, double *X, int ldx,
                 int *status, int *exps, double log2_omega, int robust,
                 int nthreads)
{
    int *col = (int *)malloc(sizeof(int) * (size_t)(m + 1));
    if (!col) return -1;
    col[0] = 0;
    for (int l = 0; l < m; ++l) col[l + 1] = col[l] + (wi[l] != 0.0 ? 2 : 1);
    const double hnorm = oracle_hnorm_inf(n, H, ldh);
    const double rho = ORACLE_EPS * hnorm;
    const double log2_thresh = -log2(10.0 * n * hnorm * ORACLE_EPS);
    int err = 0;

#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
#endif
    for (int l = 0; l < m; ++l) {
        int c0 = col[l], e = 0;
        if (wi[l] == 0.0) {
            double *b = (double *)malloc(sizeof(double) * (size_t)n * 5);
            if (!b) { err |= 1; continue; }
            double *x = b + n, *Cs = b + 2 * (size_t)n, *Ss = b + 3 * (size_t)n;
            double *work = (double *)malloc(sizeof(double) * 2 * (size_t)n);
            if (!work) { free(b); err |= 1; continue; }
            for (int i = 0; i < n; ++i) b[i] = B ? B[i + (size_t)c0 * ldb] : rho;
            double b2 = scaled_nrm2(n, b, 1);
            oracle_henry_real(n, H, ldh, wr[l], b, log2_omega, robust, x, &e, Cs, Ss, work);
            double nrm = scaled_nrm2(n, x, 1);
            int conv = (nrm > 0.0) && (log2(nrm) + e - log2(b2) > log2_thresh);
            for (int i = 0; i < n; ++i) x[i] = (nrm > 0.0) ? x[i] / nrm : 0.0;
            oracle_backtransform_real(n, Cs, Ss, x);
            for (int i = 0; i < n; ++i) X[i + (size_t)c0 * ldx] = conv ? x[i] : 0.0;
            status[l] = conv ? 0 : 1;
            free(work);
            free(b);
        } else {
            zdouble *b = (zdouble *)malloc(sizeof(zdouble) * (size_t)n * 5);
            double *Ss = (double *)malloc(sizeof(double) * (size_t)n);
            if (!b || !Ss) { free(b); free(Ss); err |= 1; continue; }
            zdouble *x = b + n, *Cs = b + 2 * (size_t)n, *work = b + 3 * (size_t)n;
            for (int i = 0; i < n; ++i)
                b[i] = B ? (B[i + (size_t)c0 * ldb] + I * B[i + (size_t)(c0 + 1) * ldb]) : rho;
            double b2 = scaled_nrm2_z(n, b);
            oracle_henry_cplx(n, H, ldh, wr[l], wi[l], b, log2_omega, robust, x, &e, Cs, Ss, work);
            double nrm = scaled_nrm2_z(n, x);
            int conv = (nrm > 0.0) && (log2(nrm) + e - log2(b2) > log2_thresh);
            for (int i = 0; i < n; ++i) x[i] = (nrm > 0.0) ? x[i] / nrm : 0.0;
            oracle_backtransform_cplx(n, Cs, Ss, x);
            for (int i = 0; i < n; ++i) {
                X[i + (size_t)c0 * ldx] = conv ? creal(x[i]) : 0.0;
                X[i + (size_t)(c0 + 1) * ldx] = conv ? cimag(x[i]) : 0.0;
            }
            status[l] = conv ? 0 : 1;
            free(Ss);
            free(b);
        }
        if (exps) exps[l] = e;
    }
    free(col);
    return err ? -1 : 0;
}

/* ------------------------------------------- the LU comparison approach */

/*
 * The LU approach of LAPACK's inverse iteration (Sec. 2.1, the "LU
 * Factorization" paragraph): P (H - lambda I) = L U with partial pivoting,
 * then L y = P b and U x = 2^-e y, for the given starting vector b (the same
 * system the RQ solve answers).  For a Hessenberg matrix the pivot search at
 * step k is between two rows only: w, the row carried down (row k of
 * H - lambda I once the earlier eliminations have acted on it), and row k+1
 * of H - lambda I.  The one whose entry in column k has the larger magnitude
 * becomes row k of U (ties keep w); the other is eliminated with the
 * multiplier l_k = (its entry) / (the pivot), |l_k| <= 1, and is carried down.
 * U is kept row-packed in Upk (row k holds columns k..n-1, n(n+1)/2 entries),
 * l_k in L[k] and the interchange in piv[k].  A final pivot below
 * eps ||H||_inf is replaced by eps ||H||_inf with its sign (the treatment of
 * the RQ solve; every other pivot has magnitude >= |h(k+1,k)| > 0).
 * Robustness (Sec. 4.1 applied to both substitutions, one exponent e for the
 * whole vector): before y(k+1) -= l_k y(k) the vector is halved when
 * |y(k+1)| + |y(k)| could exceed omega; the back substitution is the column
 * form of Henry's solve, with ProtectDivision before each division by a
 * pivot and ProtectUpdate before each column update.  On return x holds the
 * scaled solution (true solution = x * 2^e).  work: n doubles.
 * Returns 0, or 1 when the final pivot was replaced.
 */
static double packed_u(const double *Upk, int n, int i, int j)
{
    /* rows 0..i-1 hold n, n-1, ..., n-i+1 entries */
    size_t off = (size_t)i * n - (size_t)i * (i - 1) / 2;
    return Upk[off + (size_t)(j - i)];
}

int oracle_lu_real(int n, const double *H, int ldh, double lambda, const double *b,
                   double log2_omega, int robust, double *x, int *e_out, double *Upk,
                   double *L, int *piv, double *work)
{
    const double omega = ldexp(1.0, (int)log2_omega);
    const double hnorm = oracle_hnorm_inf(n, H, ldh);
    double *w = work;
    int e = 0, replaced = 0;

    /* factorization */
    for (int j = 0; j < n; ++j) w[j] = H[(size_t)j * ldh] - (j == 0 ? lambda : 0.0);
    for (int k = 0; k + 1 < n; ++k) {
        size_t off = (size_t)k * n - (size_t)k * (k - 1) / 2;
        double t_k = H[k + 1 + (size_t)k * ldh];  /* row k+1 of H - lambda I, column k */
        int swap = fabs(t_k) > fabs(w[k]);
        piv[k] = swap;
        double pivot = swap ? t_k : w[k];
        double other = swap ? w[k] : t_k;
        double l = other / pivot;
        L[k] = l;
        Upk[off] = pivot;
        for (int j = k + 1; j < n; ++j) {
            double t = H[k + 1 + (size_t)j * ldh] - (j == k + 1 ? lambda : 0.0);
            double u = swap ? t : w[j];
            double o = swap ? w[j] : t;
            Upk[off + (size_t)(j - k)] = u;
            w[j] = o - l * u;
        }
    }
    {
        size_t off = (size_t)(n - 1) * n - (size_t)(n - 1) * (n - 2) / 2;
        double r = w[n - 1];
        double small = ORACLE_EPS * hnorm;
        if (fabs(r) < small) {
            r = copysign(small, r);
            replaced = 1;
        }
        Upk[off] = r;
    }

    /* forward substitution L y = P b (y kept in x) */
    for (int i = 0; i < n; ++i) x[i] = b[i];
    for (int k = 0; k + 1 < n; ++k) {
        if (piv[k]) {
            double t = x[k];
            x[k] = x[k + 1];
            x[k + 1] = t;
        }
        if (robust && fabs(x[k + 1]) > omega - fabs(x[k])) {
            for (int i = 0; i < n; ++i) x[i] = ldexp(x[i], -1);
            e += 1;
        }
        x[k + 1] -= L[k] * x[k];
    }

    /* back substitution U x = 2^-e y, column by column */
    for (int i = n - 1; i >= 0; --i) {
        double uii = packed_u(Upk, n, i, i);
        if (robust) {
            int q = protect_division(fabs(x[i]), fabs(uii), omega);
            if (q) {
                for (int j = 0; j < n; ++j) x[j] = ldexp(x[j], -q);
                e += q;
            }
        }
        x[i] /= uii;
        if (i == 0) break;
        if (robust) {
            double umax = 0.0, xmax = 0.0;
            for (int j = 0; j < i; ++j) {
                double u = fabs(packed_u(Upk, n, j, i));
                if (u > umax) umax = u;
                if (fabs(x[j]) > xmax) xmax = fabs(x[j]);
            }
            int q = protect_update(xmax, umax, fabs(x[i]), omega);
            if (q) {
                for (int j = 0; j < n; ++j) x[j] = ldexp(x[j], -q);
                e += q;
            }
        }
        for (int j = 0; j < i; ++j) x[j] -= x[i] * packed_u(Upk, n, j, i);
    }
    *e_out = e;
    return replaced;
}

static size_t packed_off(int n, int i) { return (size_t)i * n - (size_t)i * (i - 1) / 2; }

/* the complex counterpart (Sec. 4.3): lambda and b complex, H real; pivots
 * compared by modulus, divisions by Smith's method */
int oracle_lu_cplx(int n, const double *H, int ldh, double lre, double lim, const zdouble *b,
                   double log2_omega, int robust, zdouble *x, int *e_out, zdouble *Upk,
                   zdouble *L, int *piv, zdouble *work)
{
    const double omega = ldexp(1.0, (int)log2_omega);
    const double hnorm = oracle_hnorm_inf(n, H, ldh);
    const zdouble lambda = lre + I * lim;
    zdouble *w = work;
    int e = 0, replaced = 0;

    for (int j = 0; j < n; ++j) w[j] = H[(size_t)j * ldh] - (j == 0 ? lambda : 0.0);
    for (int k = 0; k + 1 < n; ++k) {
        size_t off = packed_off(n, k);
        zdouble t_k = H[k + 1 + (size_t)k * ldh];
        int swap = zabs(t_k) > zabs(w[k]);
        piv[k] = swap;
        zdouble pivot = swap ? t_k : w[k];
        zdouble other = swap ? w[k] : t_k;
        zdouble l = zdiv_smith(other, pivot);
        L[k] = l;
        Upk[off] = pivot;
        for (int j = k + 1; j < n; ++j) {
            zdouble t = H[k + 1 + (size_t)j * ldh] - (j == k + 1 ? lambda : 0.0);
            zdouble u = swap ? t : w[j];
            zdouble o = swap ? w[j] : t;
            Upk[off + (size_t)(j - k)] = u;
            w[j] = o - l * u;
        }
    }
    {
        zdouble r = w[n - 1];
        double small = ORACLE_EPS * hnorm;
        double a = zabs(r);
        if (a < small) {
            r = (a > 0.0) ? r * (small / a) : small;
            replaced = 1;
        }
        Upk[packed_off(n, n - 1)] = r;
    }
    for (int i = 0; i < n; ++i) x[i] = b[i];
    for (int k = 0; k + 1 < n; ++k) {
        if (piv[k]) {
            zdouble t = x[k];
            x[k] = x[k + 1];
            x[k + 1] = t;
        }
        if (robust && zabs(x[k + 1]) > omega - zabs(x[k])) {
            for (int i = 0; i < n; ++i) x[i] = ldexp(creal(x[i]), -1) + I * ldexp(cimag(x[i]), -1);
            e += 1;
        }
        x[k + 1] -= L[k] * x[k];
    }
    for (int i = n - 1; i >= 0; --i) {
        zdouble uii = Upk[packed_off(n, i)];
        if (robust) {
            int q = protect_division(zabs(x[i]), zabs(uii), omega);
            if (q) {
                for (int j = 0; j < n; ++j) x[j] = ldexp(creal(x[j]), -q) + I * ldexp(cimag(x[j]), -q);
                e += q;
            }
        }
        x[i] = zdiv_smith(x[i], uii);
        if (i == 0) break;
        if (robust) {
            double umax = 0.0, xmax = 0.0;
            for (int j = 0; j < i; ++j) {
                double u = zabs(Upk[packed_off(n, j) + (size_t)(i - j)]);
                if (u > umax) umax = u;
                if (zabs(x[j]) > xmax) xmax = zabs(x[j]);
            }
            int q = protect_update(xmax, umax, zabs(x[i]), omega);
            if (q) {
                for (int j = 0; j < n; ++j) x[j] = ldexp(creal(x[j]), -q) + I * ldexp(cimag(x[j]), -q);
                e += q;
            }
        }
        for (int j = 0; j < i; ++j) x[j] -= x[i] * Upk[packed_off(n, j) + (size_t)(i - j)];
    }
    *e_out = e;
    return replaced;
}

/*
 * Driver of the LU approach for m shifts, with the interface and outputs of
 * oracle_hsein (unit-norm columns, Varah's test with the exponent, zeroed
 * columns where it fails).  There is no Givens backtransform: U x = y solves
 * for x directly.  Each shift needs a packed U of n(n+1)/2 entries.
 */
int oracle_hsein_lu(int n, const double *H, int ldh, int m, const double *wr,
                    const double *wi, const double *B, int ldb, double *X, int ldx,
                    int *status, int *exps, double log2_omega, int robust, int nthreads)
{
    int *col = (int *)malloc(sizeof(int) * (size_t)(m + 1));
    if (!col) return -1;
    col[0] = 0;
    for (int l = 0; l < m; ++l) col[l + 1] = col[l] + (wi[l] != 0.0 ? 2 : 1);
    const double hnorm = oracle_hnorm_inf(n, H, ldh);
    const double rho = ORACLE_EPS * hnorm;
    const double log2_thresh = -log2(10.0 * n * hnorm * ORACLE_EPS);
    const size_t np = (size_t)n * (n + 1) / 2;
    int err = 0;

#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
#endif
    for (int l = 0; l < m; ++l) {
        int c0 = col[l], e = 0;
        int *piv = (int *)malloc(sizeof(int) * (size_t)n);
        if (!piv) { err |= 1; continue; }
        if (wi[l] == 0.0) {
            double *b = (double *)malloc(sizeof(double) * ((size_t)n * 4 + np));
            if (!b) { free(piv); err |= 1; continue; }
            double *x = b + n, *Lm = b + 2 * (size_t)n, *work = b + 3 * (size_t)n;
            double *Upk = b + 4 * (size_t)n;
            for (int i = 0; i < n; ++i) b[i] = B ? B[i + (size_t)c0 * ldb] : rho;
            double b2 = scaled_nrm2(n, b, 1);
            oracle_lu_real(n, H, ldh, wr[l], b, log2_omega, robust, x, &e, Upk, Lm, piv, work);
            double nrm = scaled_nrm2(n, x, 1);
            int conv = (nrm > 0.0) && (log2(nrm) + e - log2(b2) > log2_thresh);
            for (int i = 0; i < n; ++i) X[i + (size_t)c0 * ldx] = conv ? x[i] / nrm : 0.0;
            status[l] = conv ? 0 : 1;
            free(b);
        } else {
            zdouble *b = (zdouble *)malloc(sizeof(zdouble) * ((size_t)n * 4 + np));
            if (!b) { free(piv); err |= 1; continue; }
            zdouble *x = b + n, *Lm = b + 2 * (size_t)n, *work = b + 3 * (size_t)n;
            zdouble *Upk = b + 4 * (size_t)n;
            for (int i = 0; i < n; ++i)
                b[i] = B ? (B[i + (size_t)c0 * ldb] + I * B[i + (size_t)(c0 + 1) * ldb]) : rho;
            double b2 = scaled_nrm2_z(n, b);
            oracle_lu_cplx(n, H, ldh, wr[l], wi[l], b, log2_omega, robust, x, &e, Upk, Lm, piv,
                           work);
            double nrm = scaled_nrm2_z(n, x);
            int conv = (nrm > 0.0) && (log2(nrm) + e - log2(b2) > log2_thresh);
            for (int i = 0; i < n; ++i) {
                X[i + (size_t)c0 * ldx] = conv ? creal(x[i]) / nrm : 0.0;
                X[i + (size_t)(c0 + 1) * ldx] = conv ? cimag(x[i]) / nrm : 0.0;
            }
            status[l] = conv ? 0 : 1;
            free(b);
        }
        free(piv);
        if (exps) exps[l] = e;
    }
    free(col);
    return err ? -1 : 0;
}

/* z = Q0 x for every column (the map from eigenvectors of H to those of A,
 * Sec. 1).  Plain triple loop, OpenMP over columns. */
void oracle_q0_apply(int n, const double *Q, int ldq, int ncol, const double *X,
                     int ldx, double *Z, int ldz, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(static)
#endif
    for (int j = 0; j < ncol; ++j) {
        for (int i = 0; i < n; ++i) Z[i + (size_t)j * ldz] = 0.0;
        for (int k = 0; k < n; ++k) {
            double xk = X[k + (size_t)j * ldx];
            for (int i = 0; i < n; ++i) Z[i + (size_t)j * ldz] += Q[i + (size_t)k * ldq] * xk;
        }
    }
}

/*
 * Plain Householder reduction to upper Hessenberg form: A = Q H Q^T with Q
 * orthogonal (the precursor step H = Q0^T A Q0 of Sec. 1).  A is n x n
 * column-major and is not modified; H and Q are outputs.  Entries of H below
 * the first subdiagonal are set to exactly zero.  work: 2n doubles.
 */
void oracle_gehrd(int n, const double *A, int lda, double *H, int ldh, double *Q,
                  int ldq, double *work)
{
    double *v = work, *w = work + n;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            H[i + (size_t)j * ldh] = A[i + (size_t)j * lda];
            Q[i + (size_t)j * ldq] = (i == j) ? 1.0 : 0.0;
        }
    for (int k = 0; k + 2 < n; ++k) {
        /* reflector P = I - 2 v v^T / (v^T v) that zeroes H(k+2:n, k) */
        double nx = 0.0;
        for (int i = k + 1; i < n; ++i) nx = hypot(nx, H[i + (size_t)k * ldh]);
        if (nx == 0.0) continue;
        double x0 = H[k + 1 + (size_t)k * ldh];
        double alpha = (x0 >= 0.0) ? -nx : nx;
        for (int i = 0; i < n; ++i) v[i] = 0.0;
        for (int i = k + 1; i < n; ++i) v[i] = H[i + (size_t)k * ldh];
        v[k + 1] -= alpha;
        double vv = 0.0;
        for (int i = k + 1; i < n; ++i) vv += v[i] * v[i];
        if (vv == 0.0) continue;
        /* H <- P H : H(:,j) -= (2/vv) v (v^T H(:,j)) */
        for (int j = 0; j < n; ++j) {
            double d = 0.0;
            for (int i = k + 1; i < n; ++i) d += v[i] * H[i + (size_t)j * ldh];
            d *= 2.0 / vv;
            for (int i = k + 1; i < n; ++i) H[i + (size_t)j * ldh] -= d * v[i];
        }
        /* H <- H P and Q <- Q P : row-wise */
        for (int i = 0; i < n; ++i) {
            double d = 0.0, dq = 0.0;
            for (int j = k + 1; j < n; ++j) {
                d += H[i + (size_t)j * ldh] * v[j];
                dq += Q[i + (size_t)j * ldq] * v[j];
            }
            w[i] = d * 2.0 / vv;
            double fq = dq * 2.0 / vv;
            for (int j = k + 1; j < n; ++j) Q[i + (size_t)j * ldq] -= fq * v[j];
        }
        for (int i = 0; i < n; ++i)
            for (int j = k + 1; j < n; ++j) H[i + (size_t)j * ldh] -= w[i] * v[j];
        for (int i = k + 2; i < n; ++i) H[i + (size_t)k * ldh] = 0.0;
        H[k + 1 + (size_t)k * ldh] = alpha;
    }
}
