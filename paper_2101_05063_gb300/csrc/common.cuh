// Internal declarations shared by the translation units of libhsein.
//
// Data layout in the caller's workspace (every block 256-byte aligned):
//   DevState                      scalars: device status, ||H||_inf, prescale
//   int   qsrc[m]                 internal shift q -> input position l
//   int   qcol[m]                 internal shift q -> first user column
//   double lam[2m]                prescaled shifts (re, im) by internal shift
//   double bnorm[m]               ||b_q||_2 of the starting vector
//   int   eB[m]                   exponent shared by the unfinished rows
//   int   etile[N*m]              exponent of every finished tile segment
//   u64   bmax[m], rmax[m]        max |B(1:p0,q)|, max |R~(1:p0,q)| (double bits)
//   Epi   epi[m]                  per-shift epilogue parameters of the update
//   u64   anorm[N]                max row sum of H(1:p0, J^-) (double bits)
//   double rowpart[n*(N+1)]       per-row partial sums of |H| by column chunk
//   double X[ldw*ncolp]           working solution, internal column order
//   double R[ldw*ncolp]           live cross-over columns R~ (one per column)
//   double Cr[n*m], Ci[n*m], S[n*m]  Givens rotations (Sec. 3.1, eq. givens)
//   double ZW[br*2*ncolp]         operand [Z'|W] of the shared-H product
//   double dt[N*br*br]            the diagonal tiles H(J, J^-), staged contiguously
// split-precision update only (BF16 digits, see ozaki.cuh):
//   bf16  hd[7 * br * P]          digits of every block H(1:p0(J), J^-), P = sum p0
//   int   he[P]                   their row exponents
//   bf16  zwd[7 * 2ncolp * br]    digits of [Z'|W], k-contiguous per column
//   int   zwf[2ncolp]             their column exponents
//
// Internal column order: the m_cplx complex shifts first (two columns each,
// starting at even columns), then the m_real real shifts; ncolp pads the
// column count to a multiple of 32.
#pragma once

#include <cuda.h>

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace hsein {

constexpr int kMaxBr = 128;
constexpr int kNegInfLog = -100000;  // log2 bound of zero

struct DevState {
    int status;        // 0 ok, < 0 device error, 1 some column not converged
    int hexp;          // prescale exponent s >= 0 (H' = 2^-s H)
    int ncplx_found;   // number of wi != 0 seen
    int pad0;
    double hscale;     // 2^-s
    double hnorm;      // ||H'||_inf (prescaled)
    unsigned long long hnorm_bits;   // ||H||_inf of the raw matrix, as bits
    unsigned long long lammax_bits;  // max |lambda| of the raw shifts, as bits
};

struct Epi {
    double fB;          // 2^(eB_old - eB_new): rescales B(1:p0)
    double pi;          // prod of the tile's sines (multiplies R~)
    double zbr_re, zbr_im;   // last entry of z (multiplies R~ in the B update)
    double cz_re, cz_im;     // lambda' * rho' (row p0-1 of the B update)
    double cw_re, cw_im;     // lambda' * c_0  (row p0-1 of the R~ update)
};

struct Layout {
    int n, m, mr, mc, ncol, ncolp, br, N, b0, ldw;
    size_t off_state, off_qsrc, off_qcol, off_lam, off_bnorm, off_eB, off_etile, off_bmax,
        off_rmax, off_epi, off_anorm, off_rowpart, off_X, off_R, off_Cr, off_Ci, off_S, off_ZW,
        off_dt, off_hd, off_he, off_zwd, off_zwf, off_margin, off_oz, off_hr, off_lu, total;
    int oz;       // 1: split-precision shared-H update (BF16 digits), 0: FP64
    int compact;  // 1: Givens rotations stored compactly (Stewart's scheme)
    int lu_slots;          // per-shift LU baseline: shifts factored at once
    size_t lu_slot_bytes;  // and the workspace of one (packed U, row maxima)
    int lps_real;          // lanes per real shift in the diagonal-tile sweep (16 or 8)
};

// first row of tile J (tile 0 is the ragged top-left tile of height b0)
__host__ __device__ inline int tile_start(const Layout& L, int J) {
    return J == 0 ? 0 : L.b0 + (J - 1) * L.br;
}
__host__ __device__ inline int tile_height(const Layout& L, int J) {
    return J == 0 ? L.b0 : L.br;
}
// internal column of internal shift q
__host__ __device__ inline int qcolumn(const Layout& L, int q) {
    return q < L.mc ? 2 * q : 2 * L.mc + (q - L.mc);
}

template <typename T>
__host__ __device__ inline T* ws(void* base, size_t off) {
    return reinterpret_cast<T*>(static_cast<char*>(base) + off);
}

// upper bound on log2(v): v < 2^L for v > 0 finite; kNegInfLog for v == 0
__device__ inline int log2_bound(double v) {
    if (!(v > 0.0)) return kNegInfLog;
    return ilogb(v) + 1;
}

__device__ inline void atomic_max_nonneg(unsigned long long* addr, double v) {
    // non-negative doubles order like their bit patterns
    atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

__device__ inline double bits_to_double(unsigned long long b) {
    return __longlong_as_double((long long)b);
}

// |v| as an order-preserving integer: the bit pattern without the sign
__device__ inline unsigned long long abs_bits(double v) {
    return (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFULL;
}

// 2^d exactly (from the exponent field where 2^d is normal)
__device__ inline double pow2(int d) {
    if (d >= -1022 && d <= 1023) return __longlong_as_double((long long)(d + 1023) << 52);
    return ldexp(1.0, d);
}

// 2^d for -1074 <= d <= 1023 from the bit pattern alone (normal and
// subnormal powers of two), no library call
__device__ inline double exact_pow2(int d) {
    return d >= -1022 ? __longlong_as_double((long long)(d + 1023) << 52)
                      : __longlong_as_double(1LL << (d + 1074));
}

// ---- Givens rotations: canonical sign and compact storage (Sec. 4.4) ----
// A rotation (c, s) and its negation (-c, -s) (with phi -> -phi and
// x(k) -> -x(k)) serve the solve equally well; the solution of
// (H - lambda I) x = b is the same.  With compact storage the sweep keeps
// the canonical one:
// real rotations have the larger of |c|, |s| positive, complex rotations
// (c complex, s real) have s >= 0.  Stewart's compact storage recovers
// exactly the canonical rotation: it keeps the smaller quantity (halved)
// or twice the reciprocal of the larger one, and recomputes the other from
// c^2 + s^2 = 1 by a well-conditioned square root.

constexpr unsigned long long kSignBit = 0x8000000000000000ULL;

__device__ inline double flip_if(double v, unsigned long long f) {
    return __longlong_as_double(__double_as_longlong(v) ^ (long long)f);
}

// sign-bit mask that makes the rotation canonical (0: keep it)
template <bool CPLX>
__device__ inline unsigned long long canon_mask(double cr, double ci, double s) {
    (void)ci;
    const unsigned long long sb = (unsigned long long)__double_as_longlong(s);
    if (CPLX) return sb & kSignBit;  // s >= 0
    const unsigned long long cb = (unsigned long long)__double_as_longlong(cr);
    return (sb & ~kSignBit) < (cb & ~kSignBit) ? (cb & kSignBit) : (sb & kSignBit);
}

// one number for a canonical real rotation: s/2 (|s| < |c|, c > 0; |value|
// < 0.36), 1 (c = 0, s = 1), or 2/c (|c| <= |s|, s > 0; |value| >= 2.8)
__device__ inline double givens_pack_real(double c, double s) {
    if (fabs(s) < fabs(c)) return 0.5 * s;
    return c == 0.0 ? 1.0 : 2.0 / c;
}
__device__ inline void givens_unpack_real(double r, double& c, double& s) {
    if (r == 1.0) {
        c = 0.0;
        s = 1.0;
    } else if (fabs(r) < 1.0) {
        s = 2.0 * r;
        c = sqrt(fma(-s, s, 1.0));
    } else {
        c = 2.0 / r;
        s = sqrt(fma(-c, c, 1.0));
    }
}

// two numbers for a canonical complex rotation (s >= 0): the first encodes
// (|c|, s) as above with the sign of Re c in its sign bit, the second the
// direction c/|c| taken with Re >= 0 (encoded like a real rotation, with
// +-1 for a purely imaginary direction), 0 when c = 0
__device__ inline void givens_pack_cplx(double cr, double ci, double s, double& r1, double& r2) {
    const double a = sqrt(fma(cr, cr, ci * ci));
    const double e = s < a ? 0.5 * s : (a == 0.0 ? 1.0 : 2.0 / a);
    r1 = copysign(e, cr);
    if (a == 0.0) {
        r2 = 0.0;
        return;
    }
    const double wr = fabs(cr) / a, wi = copysign(1.0, cr) * ci / a;  // w = sign(Re c) c / |c|
    if (fabs(wi) < wr) r2 = 0.5 * wi;
    else r2 = wr == 0.0 ? (wi > 0.0 ? 1.0 : -1.0) : copysign(2.0 / wr, wi);
}
__device__ inline void givens_unpack_cplx(double r1, double r2, double& cr, double& ci,
                                          double& s) {
    const double r = fabs(r1);
    double a;
    if (r == 1.0) {
        a = 0.0;
        s = 1.0;
    } else if (r < 1.0) {
        s = 2.0 * r;
        a = sqrt(fma(-s, s, 1.0));
    } else {
        a = 2.0 / r;
        s = sqrt(fma(-a, a, 1.0));
    }
    if (a == 0.0) {
        cr = 0.0;
        ci = 0.0;
        return;
    }
    double wr, wi;
    const double q = fabs(r2);
    if (q == 1.0) {
        wr = 0.0;
        wi = r2;
    } else if (q < 1.0) {
        wi = 2.0 * r2;
        wr = sqrt(fma(-wi, wi, 1.0));
    } else {
        wr = 2.0 / q;
        wi = copysign(sqrt(fma(-wr, wr, 1.0)), r2);
    }
    const double g = copysign(a, r1);  // c = sign(Re c) |c| w
    cr = g * wr;
    ci = g * wi;
}

// exponent of the scale 2^e for a norm whose largest magnitude has the bit
// pattern mbits: 2^e <= max < 2^(e+1), e kept above -1020 so 2^-e is finite
__device__ inline int norm_exp(unsigned long long mbits) {
    return mbits == 0 ? 0 : max(ilogb(bits_to_double(mbits)), -1020);
}

__device__ inline void set_error(DevState* st, int code) {
    atomicMin(&st->status, code);
}

// host launchers (one per translation unit)
void launch_prepare(const Layout& L, void* work, const double* H, int ldh, const double* wr,
                    const double* wi, const double* B, int ldb, int omega_log2, cudaStream_t s);
void launch_diag(const Layout& L, void* work, int J, int robust, int omega_log2,
                 long long wait_limit, cudaStream_t s);
// lanes per real shift for the sweep of this layout on a GPU with num_sms SMs
int diag_lanes_real(const Layout& L, int num_sms);
void launch_update(const Layout& L, void* work, const double* H, int ldh, int J, cudaStream_t s);
// per-shift LU comparison baseline (method 2)
size_t lu_slot_bytes(int n);
void launch_lu(const Layout& L, void* work, const double* H, int ldh, int robust, int omega_log2,
               cudaStream_t s);
cudaError_t lu_configure(int n);
// split-precision update: tensor maps of the A_J digit blocks (mapsA[1..N-1])
// and of the [Z'|W] digits for the workspace at `work`
bool encode_update_oz_maps(const Layout& L, void* work, CUtensorMap* mapsA, CUtensorMap* mapB);
void launch_update_oz(const Layout& L, void* work, int J, int num_sms, const CUtensorMap& mapA,
                      const CUtensorMap& mapB, cudaStream_t s);
void launch_stage_tiles(const Layout& L, void* work, const double* H, int ldh, cudaStream_t s);
void launch_split_h(const Layout& L, void* work, const double* H, int ldh, cudaStream_t s);
size_t oz_update_hd_elems(const Layout& L);
void launch_finalize(const Layout& L, void* work, double* X, int ldx, int* status,
                     cudaStream_t s);
// comparison baseline: Henry's solve per shift, unblocked (csrc/k_henry.cu)
void launch_henry(const Layout& L, void* work, const double* H, int ldh, int robust,
                  int omega_log2, cudaStream_t s);
// restart of non-converged shifts (csrc/restart.cu)
size_t restart_scratch_bytes(int n, int k);
void launch_restart_trial(int n, int t, int k, const int* map, const double* wr, const double* wi,
                          const double* B, int ldb, double* wr_s, double* wi_s, double* Bs,
                          double* scratch, cudaStream_t s);
void launch_restart_scatter(int n, int k, const int* map, const double* Xs, const int* st_s,
                            double* X, int ldx, int* status, cudaStream_t s);
void launch_q0(const Layout& L, const double* Q, int ldq, const double* X, int ldx, double* Z,
               int ldz, cudaStream_t s);

}  // namespace hsein
