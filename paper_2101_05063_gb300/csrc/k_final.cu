// K4: RBacktransform (Alg. "consistency-scaling", eq. "robust-backtransform")
// plus the convergence test of Sec. 4.2, one thread block per shift.
//
//  1. alpha_min: the largest tile exponent e_max; every tile segment is
//     brought to it by an exact power-of-two factor (consistency scaling).
//  2. Scaled 2-norm: the largest magnitude (integer maximum of the bit
//     patterns), then the sum of squares scaled by its power of two, reduced
//     across the block in a fixed order.
//  3. Varah's test: ||x||_2 2^e_max / ||b||_2 > 1 / (10 n ||H||_inf eps),
//     evaluated in log2.  A column that fails is set to zero (Sec. 4.2).
//  4. y = G_n^H (... (G_2^H (x / ||x||))): the recurrence
//        y(k-1) = c_k tau - s_k x_k,   tau <- s_k tau + conj(c_k) x_k
//     is a first-order linear recurrence in tau, so each thread composes the
//     affine maps of its chunk of rows, a block scan combines the chunks and
//     each thread then emits its outputs.
// Output goes to the caller's X in input column order; dStatus per shift.
#include "common.cuh"

namespace hsein {
namespace {

constexpr int kThreads = 256;

// affine map tau -> a tau + (br + i bi), a real
struct Aff {
    double a, br, bi;
};
// apply f then g
__device__ inline Aff aff_then(Aff f, Aff g) {
    return Aff{g.a * f.a, fma(g.a, f.br, g.br), fma(g.a, f.bi, g.bi)};
}

template <bool CPLX>
__device__ void finalize_shift(const Layout& L, void* work, int q, double* __restrict__ Xo,
                               int ldx, int* __restrict__ status) {
    const DevState* st = ws<DevState>(work, L.off_state);
    DevState* stw = ws<DevState>(work, L.off_state);
    const int* qsrc = ws<int>(work, L.off_qsrc);
    const int* qcol = ws<int>(work, L.off_qcol);
    const int* etile = ws<int>(work, L.off_etile);
    const double* bnorm = ws<double>(work, L.off_bnorm);
    const double* X = ws<double>(work, L.off_X);
    const double* Cr = ws<double>(work, L.off_Cr);
    const double* Ci = ws<double>(work, L.off_Ci);
    const double* Sv = ws<double>(work, L.off_S);
    __shared__ int s_emax;
    __shared__ unsigned long long s_mb[32];
    __shared__ double s_t[32];
    __shared__ Aff s_aff[32];
    __shared__ int s_conv;
    __shared__ double s_scale;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = L.n;
    const int col = qcolumn(L, q);
    const double* xr = X + (size_t)col * L.ldw;
    const double* xi = X + (size_t)(col + 1) * L.ldw;
    const double* cr = Cr + (size_t)q * n;
    const double* ci = Ci + (size_t)q * n;
    const double* sv = Sv + (size_t)q * n;  // not read with compact storage
    // rotation k as stored by the sweep (compact: Stewart's scheme, Sec. 4.4)
    auto rot = [&](int k, double& c_r, double& c_i, double& s_) {
        if (L.compact) {
            if (CPLX) {
                givens_unpack_cplx(cr[k], ci[k], c_r, c_i, s_);
            } else {
                givens_unpack_real(cr[k], c_r, s_);
                c_i = 0.0;
            }
        } else {
            c_r = cr[k];
            c_i = CPLX ? ci[k] : 0.0;
            s_ = sv[k];
        }
    };

    if (tid == 0) {
        int em = etile[q];
        for (int J = 1; J < L.N; ++J) em = max(em, etile[(size_t)J * L.m + q]);
        s_emax = em;
    }
    __syncthreads();
    const int emax = s_emax;
    const int cs = (n + kThreads - 1) / kThreads;
    const int a0 = min(n, tid * cs), a1 = min(n, a0 + cs);
    // the consistency factor 2^(e_tile - e_max) of the tile of each row, for
    // rows a0, a0+1, ... in turn: the tile index is found once per pass and
    // then advanced at tile boundaries
    struct Factor {
        int J, next;
        double f;
    };
    auto factor_at = [&](int J) { return pow2(etile[(size_t)J * L.m + q] - emax); };
    auto factor_start = [&]() {
        Factor t;
        t.J = a0 < L.b0 ? 0 : 1 + (a0 - L.b0) / L.br;
        t.next = tile_start(L, t.J + 1);
        t.f = t.J < L.N ? factor_at(t.J) : 1.0;
        return t;
    };
    auto factor = [&](Factor& t, int i) {
        if (i == t.next) {
            ++t.J;
            t.next += L.br;
            t.f = factor_at(t.J);
        }
        return t.f;
    };
    // scaled 2-norm of the consistently scaled column: the largest magnitude
    // as an integer maximum of bit patterns, then sum (v_i 2^-e)^2 with the
    // exact power-of-two scale 2^e of that maximum (no division per element)
    unsigned long long mb = 0;
    Factor ft = factor_start();
    for (int i = a0; i < a1; ++i) {
        const double f = factor(ft, i);
        mb = max(mb, abs_bits(xr[i] * f));
        if (CPLX) mb = max(mb, abs_bits(xi[i] * f));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
    if (lane == 0) s_mb[warp] = mb;
    __syncthreads();
    mb = s_mb[0];
    for (int w = 1; w < kThreads / 32; ++w) mb = max(mb, s_mb[w]);
    const int ne = norm_exp(mb);
    const double nsc = pow2(-ne);
    double ss = 0.0;
    ft = factor_start();
    for (int i = a0; i < a1; ++i) {
        const double g = factor(ft, i) * nsc;
        const double t0 = xr[i] * g;
        ss = fma(t0, t0, ss);
        if (CPLX) {
            const double t1 = xi[i] * g;
            ss = fma(t1, t1, ss);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if (lane == 0) s_t[warp] = ss;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) t += s_t[w];
        const double nrm = mb == 0 ? 0.0 : sqrt(t) * pow2(ne);
        const double thr = -log2(10.0 * n * st->hnorm * 0x1p-53);
        const double margin = nrm > 0.0 ? log2(nrm) + emax - log2(bnorm[q]) - thr : -HUGE_VAL;
        int conv = margin > 0.0;
        ws<double>(work, L.off_margin)[qsrc[q]] = margin;
        s_conv = conv;
        s_scale = conv ? 1.0 / nrm : 0.0;
    }
    __syncthreads();
    const int uc = qcol[q];
    double* yr = Xo + (size_t)uc * ldx;
    double* yi = Xo + (size_t)(uc + 1) * ldx;
    if (!s_conv) {
        for (int i = tid; i < n; i += kThreads) {
            yr[i] = 0.0;
            if (CPLX) yi[i] = 0.0;
        }
        if (tid == 0) {
            status[qsrc[q]] = 1;
            atomicCAS(&stw->status, 0, 1);
        }
        return;
    }
    const double inv = s_scale;
    // chunk map: tau_out = a tau_in + b over rows a0..a1-1
    Aff f{1.0, 0.0, 0.0};
    ft = factor_start();
    for (int k = a0; k < a1; ++k) {
        double g = factor(ft, k) * inv;
        double yk_r = xr[k] * g, yk_i = CPLX ? xi[k] * g : 0.0;
        Aff step;
        if (k == 0) {
            step = Aff{0.0, yk_r, yk_i};
        } else {
            double c_r, c_i, s;
            rot(k, c_r, c_i, s);
            // conj(c) y
            step = Aff{s, c_r * yk_r + c_i * yk_i, c_r * yk_i - c_i * yk_r};
        }
        f = aff_then(f, step);
    }
    // inclusive scan of chunk maps across the block (warp shuffles, then warps)
    Aff inc = f;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        Aff p{__shfl_up_sync(0xffffffffu, inc.a, o), __shfl_up_sync(0xffffffffu, inc.br, o),
              __shfl_up_sync(0xffffffffu, inc.bi, o)};
        if (lane >= o) inc = aff_then(p, inc);
    }
    if (lane == 31) s_aff[warp] = inc;
    __syncthreads();
    if (tid == 0) {
        Aff run = s_aff[0];
        for (int w = 1; w < kThreads / 32; ++w) {
            run = aff_then(run, s_aff[w]);
            s_aff[w] = run;
        }
    }
    __syncthreads();
    // exclusive prefix for this thread: warps before, then lanes before
    Aff ex{1.0, 0.0, 0.0};
    if (warp > 0) ex = s_aff[warp - 1];
    Aff lanepre{__shfl_up_sync(0xffffffffu, inc.a, 1), __shfl_up_sync(0xffffffffu, inc.br, 1),
                __shfl_up_sync(0xffffffffu, inc.bi, 1)};
    if (lane > 0) ex = aff_then(ex, lanepre);
    double tr = ex.br, ti = ex.bi;  // tau entering row a0 (the map applied to 0)
    ft = factor_start();
    for (int k = a0; k < a1; ++k) {
        double g = factor(ft, k) * inv;
        double yk_r = xr[k] * g, yk_i = CPLX ? xi[k] * g : 0.0;
        if (k == 0) {
            tr = yk_r;
            ti = yk_i;
            continue;
        }
        double c_r, c_i, s;
        rot(k, c_r, c_i, s);
        // y(k-1) = c tau - s y_k
        double outr = c_r * tr - c_i * ti - s * yk_r;
        double outi = c_r * ti + c_i * tr - s * yk_i;
        yr[k - 1] = outr;
        if (CPLX) yi[k - 1] = outi;
        double ntr = s * tr + c_r * yk_r + c_i * yk_i;
        double nti = s * ti + c_r * yk_i - c_i * yk_r;
        tr = ntr;
        ti = nti;
    }
    if (a1 == n && a0 < a1) {
        yr[n - 1] = tr;
        if (CPLX) yi[n - 1] = ti;
    }
    if (tid == 0) status[qsrc[q]] = 0;
}

__global__ void __launch_bounds__(kThreads)
k_finalize(Layout L, void* work, double* __restrict__ Xo, int ldx, int* __restrict__ status) {
    const DevState* st = ws<DevState>(work, L.off_state);
    const int q = blockIdx.x;
    if (st->status < 0) {
        // the solve did not run: mark every shift invalid, zero the output
        if (q < L.m && threadIdx.x == 0) status[q] = 3;
        for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < (size_t)L.n * L.ncol;
             idx += (size_t)gridDim.x * blockDim.x) {
            size_t c = idx / L.n, i = idx % L.n;
            Xo[i + c * ldx] = 0.0;
        }
        return;
    }
    if (q < L.mc) finalize_shift<true>(L, work, q, Xo, ldx, status);
    else finalize_shift<false>(L, work, q, Xo, ldx, status);
}

}  // namespace

void launch_finalize(const Layout& L, void* work, double* X, int ldx, int* status,
                     cudaStream_t s) {
    k_finalize<<<L.m, kThreads, 0, s>>>(L, work, X, ldx, status);
}

}  // namespace hsein
