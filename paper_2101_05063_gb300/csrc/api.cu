// Host side of the C ABI declared in include/hsein.h: argument checks, the
// workspace layout and the launch sequence of one solve.
//
// Launch sequence of hsein_solve (all on the caller's stream):
//   prepare (setup, row sums, tile norms, init)            -- step a0
//   for J = N-1 .. 1:  k_diag(J)  then  k_update(J)          -- steps a1..a4
//   k_diag(0)                                               -- top-left tile
//   k_finalize                                              -- step a5
// The tile columns are walked once from right to left: the cross-over
// columns needed by the update of tile column J are produced by the same
// product that performs that update, so only one n x ncol buffer of
// cross-over columns is live (the paper stores N of them per shift,
// Sec. 4.4, and must group shifts because of it).
#include "../../include/hsein.h"
#include "common.cuh"
#include "ozaki.cuh"

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <new>
#include <vector>

namespace hsein {
cudaError_t diag_configure(int br);
cudaError_t update_configure(int br);
cudaError_t update_oz_configure();
}  // namespace hsein

using hsein::Layout;

struct hsein_plan_s {
    Layout L;
    hsein_options opt;
    int device;
    int num_sms = 0;
    // split precision: TMA tensor maps of the digit operands, encoded for the
    // workspace address they were last used with
    const void* maps_work = nullptr;
    std::vector<CUtensorMap> mapsA;
    CUtensorMap mapB;
    // measurement: one (phase, start, end) record per launch while enabled
    int profiling = 0;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    std::vector<int> rec_phase;
    // hsein_solve_host: a side stream for the upload of Q0, and events that
    // order it after the previous call's backtransform and before this one's
    cudaStream_t side = nullptr;
    cudaEvent_t ev_q0 = nullptr, ev_done = nullptr;
    // hsein_solve_host: the solve on the device copies captured as a graph,
    // for the workspace and starting-vector choice it was captured with
    hsein_graph_s* host_graph = nullptr;
    const void* host_graph_work = nullptr;
    bool host_graph_b = false;
};

// a captured step (hsein_graph_create)
struct hsein_graph_s {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// the LU baseline keeps the carried row (complex) in shared memory
constexpr int kLuMaxN = 14336;

// the per-shift LU baseline keeps the packed U factors of this many bytes at
// most (the shifts are factored in chunks that fit)
constexpr size_t kLuBudget = size_t(16) << 30;

void make_layout(Layout* L, int n, int mr, int mc, int br, int precision, int givens,
                 int method) {
    L->n = n;
    L->mr = mr;
    L->mc = mc;
    L->m = mr + mc;
    L->ncol = mr + 2 * mc;
    L->ncolp = (L->ncol + 31) / 32 * 32;
    L->br = br;
    L->N = (n + br - 1) / br;
    L->b0 = n - (L->N - 1) * br;
    L->ldw = (n + 7) / 8 * 8;
    L->lps_real = 16;  // set for the plan's GPU by hsein_plan
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align256(o + bytes);
        return at;
    };
    const size_t m = (size_t)L->m, N = (size_t)L->N, nn = (size_t)n;
    L->off_state = take(sizeof(hsein::DevState));
    L->off_qsrc = take(sizeof(int) * m);
    L->off_qcol = take(sizeof(int) * m);
    L->off_lam = take(sizeof(double) * 2 * m);
    L->off_bnorm = take(sizeof(double) * m);
    L->off_eB = take(sizeof(int) * m);
    L->off_etile = take(sizeof(int) * N * m);
    L->off_bmax = take(sizeof(unsigned long long) * m);
    L->off_rmax = take(sizeof(unsigned long long) * m);
    L->off_epi = take(sizeof(hsein::Epi) * m);
    L->off_anorm = take(sizeof(unsigned long long) * N);
    L->off_rowpart = take(sizeof(double) * nn * (N + 1));
    L->off_X = take(sizeof(double) * (size_t)L->ldw * L->ncolp);
    L->off_R = take(sizeof(double) * (size_t)L->ldw * L->ncolp);
    L->off_Cr = take(sizeof(double) * nn * m);
    L->off_Ci = take(sizeof(double) * nn * (size_t)(mc > 0 ? mc : 1));
    L->compact = givens;
    L->off_S = take(givens ? 0 : sizeof(double) * nn * m);  // compact: no separate s
    L->off_ZW = take(sizeof(double) * (size_t)br * 2 * L->ncolp);
    L->off_dt = take(sizeof(double) * N * br * br);
    L->off_margin = take(sizeof(double) * m);
    L->oz = precision == 1 ? 1 : 0;
    {
        const size_t P = L->oz ? hsein::oz_update_hd_elems(*L) : 0;
        L->off_hd = take(2 * (size_t)hsein::oz::kS * br * P);
        L->off_he = take(sizeof(int) * P);
        L->off_zwd = take(L->oz ? 2 * (size_t)hsein::oz::kS * 2 * L->ncolp * br : 0);
        L->off_zwf = take(L->oz ? sizeof(int) * 2 * (size_t)L->ncolp : 0);
    }
    // buffers of the split-precision backtransform follow the solve's state,
    // which stays readable (hsein_plan_sync_status) after the backtransform
    L->off_oz = o;
    if (precision == 1) o = align256(o + hsein::ozq0_workspace_bytes(n, L->ncol));
    // per-shift LU baseline: H row-major, and one slot (packed U, row maxima)
    // per shift factored at once
    L->lu_slots = 0;
    L->lu_slot_bytes = 0;
    L->off_hr = o;
    L->off_lu = o;
    if (method == 2) {
        L->lu_slot_bytes = hsein::lu_slot_bytes(n);
        const size_t fit = std::max<size_t>(1, kLuBudget / L->lu_slot_bytes);
        L->lu_slots = (int)std::min<size_t>(fit, (size_t)std::max(mr, mc));
        L->off_hr = take(sizeof(double) * nn * nn);
        L->off_lu = take(L->lu_slot_bytes * (size_t)L->lu_slots);
        o = align256(o);
    }
    L->total = o;
}

bool aligned256(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 255) == 0; }

// room for one retried shift of hsein_restart (map, shift, status, two
// starting-vector and two solution columns, trial scratch) beside the
// sub-problem's own workspace, which is never larger than the plan's
size_t restart_reserve(int n) {
    return 8 * 256 + 4 * align256(sizeof(double) * 2 * (size_t)n) +
           align256(hsein::restart_scratch_bytes(n, 1));
}

cudaEvent_t next_event(hsein_plan_s* p) {
    if (p->used == p->pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        p->pool.push_back(e);
    }
    return p->pool[p->used++];
}

// brackets one launch with events when profiling is on
struct PhaseScope {
    hsein_plan_s* p;
    cudaStream_t s;
    PhaseScope(hsein_plan_s* plan, int phase, cudaStream_t stream) : p(plan), s(stream) {
        if (!p->profiling) return;
        cudaEvent_t e = next_event(p);
        if (e) {
            cudaEventRecord(e, s);
            p->rec_phase.push_back(phase);
        }
    }
    ~PhaseScope() {
        if (!p->profiling) return;
        cudaEvent_t e = next_event(p);
        if (e) cudaEventRecord(e, s);
    }
};

}  // namespace

namespace hsein {
// the device a plan was created on (the device whose kernel settings it made)
int plan_device(const hsein_plan_s* p) { return p->device; }
}  // namespace hsein

extern "C" {

hsein_status hsein_default_options(hsein_options* opt) {
    if (!opt) return HSEIN_EARG;
    *opt = hsein_options{};
    opt->br = 64;
    opt->precision = 0;
    opt->robust = 1;
    opt->omega_log2 = 1000;
    opt->wait_limit_cycles = 1LL << 32;
    return HSEIN_OK;
}

hsein_status hsein_plan(hsein_plan_t* plan, int n, int m_real, int m_cplx,
                        const hsein_options* opt, size_t* workspace_bytes) {
    if (!plan) return HSEIN_EARG;
    *plan = nullptr;
    if (n < 1 || m_real < 0 || m_cplx < 0 || m_real + m_cplx < 1) return HSEIN_EARG;
    if ((long long)m_real + 2LL * m_cplx > (1LL << 30)) return HSEIN_EARG;
    hsein_options o;
    hsein_default_options(&o);
    if (opt) {
        if (opt->br != 0) o.br = opt->br;
        o.precision = opt->precision;
        o.robust = opt->robust;
        if (opt->omega_log2 != 0) o.omega_log2 = opt->omega_log2;
        o.method = opt->method;
        o.givens = opt->givens;
        if (opt->wait_limit_cycles != 0) o.wait_limit_cycles = opt->wait_limit_cycles;
    }
    if (o.wait_limit_cycles < 1 || o.wait_limit_cycles > (1LL << 60)) return HSEIN_EARG;
    if (o.method < 0 || o.method > 2) return HSEIN_EARG;
    if (o.method != 0 && o.precision != 0) return HSEIN_EARG;  // the baselines are FP64
    if (o.method == 2 && n > kLuMaxN) return HSEIN_EARG;       // its row w in shared memory
    if (o.givens != 0 && o.givens != 1) return HSEIN_EARG;
    if (o.givens == 1 && o.method != 0) return HSEIN_EARG;  // the baseline stores c and s
    if (o.br < 8 || o.br > hsein::kMaxBr || o.br % 8 != 0) return HSEIN_EARG;
    if (o.precision != 0 && o.precision != 1) return HSEIN_EARG;
    if (o.precision == 1 && o.br != 64) return HSEIN_EARG;  // digit tiles are 64 wide
    if (o.robust != 0 && o.robust != 1) return HSEIN_EARG;
    if (o.omega_log2 < 16 || o.omega_log2 > 1000) return HSEIN_EARG;
    hsein_plan_s* p = new (std::nothrow) hsein_plan_s;
    if (!p) return HSEIN_ENOMEM;
    make_layout(&p->L, n, m_real, m_cplx, o.br, o.precision, o.givens, o.method);
    p->opt = o;
    if (cudaGetDevice(&p->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess ||
        hsein::diag_configure(o.br) != cudaSuccess || hsein::update_configure(o.br) != cudaSuccess ||
        hsein::ozaki_configure() != cudaSuccess || hsein::update_oz_configure() != cudaSuccess ||
        (o.method == 2 && hsein::lu_configure(n) != cudaSuccess)) {
        cudaGetLastError();
        delete p;
        return HSEIN_ECUDA;
    }
    p->L.lps_real = hsein::diag_lanes_real(p->L, p->num_sms);
    if (workspace_bytes) *workspace_bytes = p->L.total + restart_reserve(n);
    *plan = p;
    return HSEIN_OK;
}

hsein_status hsein_plan_info(hsein_plan_t plan, int* n, int* m_real, int* m_cplx, int* ncol,
                             int* br, size_t* workspace_bytes) {
    if (!plan) return HSEIN_EARG;
    if (n) *n = plan->L.n;
    if (m_real) *m_real = plan->L.mr;
    if (m_cplx) *m_cplx = plan->L.mc;
    if (ncol) *ncol = plan->L.ncol;
    if (br) *br = plan->L.br;
    if (workspace_bytes) *workspace_bytes = plan->L.total + restart_reserve(plan->L.n);
    return HSEIN_OK;
}

hsein_status hsein_solve(hsein_plan_t plan, const double* dH, int ldh, const double* dWr,
                         const double* dWi, const double* dB, int ldb, double* dX, int ldx,
                         int* dStatus, void* dWork, size_t work_bytes, void* stream) {
    if (!plan) return HSEIN_EARG;
    const Layout& L = plan->L;
    if (!dH || ldh < L.n || !dWr || !dWi || !dX || ldx < L.n || !dStatus) return HSEIN_EARG;
    if (dB && ldb < L.n) return HSEIN_EARG;
    if (!dWork || !aligned256(dWork)) return HSEIN_EARG;
    if (work_bytes < L.total) return HSEIN_ENOMEM;
    if ((const void*)dX == (const void*)dH || (dB && (const void*)dX == (const void*)dB))
        return HSEIN_EARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int robust = plan->opt.robust, om = plan->opt.omega_log2;
    if (L.oz && plan->maps_work != dWork) {
        plan->mapsA.resize(L.N);
        if (!hsein::encode_update_oz_maps(L, dWork, plan->mapsA.data(), &plan->mapB)) {
            plan->maps_work = nullptr;
            return HSEIN_ECUDA;
        }
        plan->maps_work = dWork;
    }
    if (plan->opt.method != 0) {
        // comparison baselines, per shift over the whole matrix: Henry's RQ
        // solve (1) or the LU approach (2)
        {
            PhaseScope ps(plan, 0, s);
            hsein::launch_prepare(L, dWork, dH, ldh, dWr, dWi, dB, ldb, om, s);
        }
        {
            PhaseScope ps(plan, 1, s);
            if (plan->opt.method == 1) hsein::launch_henry(L, dWork, dH, ldh, robust, om, s);
            else hsein::launch_lu(L, dWork, dH, ldh, robust, om, s);
        }
        {
            PhaseScope ps(plan, 3, s);
            hsein::launch_finalize(L, dWork, dX, ldx, dStatus, s);
        }
        if (cudaGetLastError() != cudaSuccess) return HSEIN_ECUDA;
        return HSEIN_OK;
    }
    {
        PhaseScope ps(plan, 0, s);
        hsein::launch_prepare(L, dWork, dH, ldh, dWr, dWi, dB, ldb, om, s);
        hsein::launch_stage_tiles(L, dWork, dH, ldh, s);
        if (L.oz) hsein::launch_split_h(L, dWork, dH, ldh, s);
    }
    for (int J = L.N - 1; J >= 1; --J) {
        {
            PhaseScope ps(plan, 1, s);
            hsein::launch_diag(L, dWork, J, robust, om, plan->opt.wait_limit_cycles, s);
        }
        PhaseScope ps(plan, 2, s);
        if (L.oz)
            hsein::launch_update_oz(L, dWork, J, plan->num_sms, plan->mapsA[J], plan->mapB, s);
        else
            hsein::launch_update(L, dWork, dH, ldh, J, s);
    }
    {
        PhaseScope ps(plan, 1, s);
        hsein::launch_diag(L, dWork, 0, robust, om, plan->opt.wait_limit_cycles, s);
    }
    {
        PhaseScope ps(plan, 3, s);
        hsein::launch_finalize(L, dWork, dX, ldx, dStatus, s);
    }
    if (cudaGetLastError() != cudaSuccess) return HSEIN_ECUDA;
    return HSEIN_OK;
}

hsein_status hsein_backtransform(hsein_plan_t plan, const double* dQ0, int ldq, const double* dX,
                                 int ldx, double* dZ, int ldz, void* dWork, size_t work_bytes,
                                 void* stream) {
    if (!plan) return HSEIN_EARG;
    const Layout& L = plan->L;
    if (!dQ0 || ldq < L.n || !dX || ldx < L.n || !dZ || ldz < L.n) return HSEIN_EARG;
    if ((const void*)dZ == (const void*)dX || (const void*)dZ == (const void*)dQ0) return HSEIN_EARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (plan->opt.precision == 1) {
        if (!dWork || !aligned256(dWork)) return HSEIN_EARG;
        if (work_bytes < L.total) return HSEIN_ENOMEM;
        PhaseScope ps(plan, 4, s);
        int* status_word = reinterpret_cast<int*>(static_cast<char*>(dWork) + L.off_state +
                                                  offsetof(hsein::DevState, status));
        if (!hsein::launch_ozaki_q0(L.n, L.ncol, dQ0, ldq, dX, ldx, dZ, ldz,
                                    static_cast<char*>(dWork) + L.off_oz, status_word, s))
            return HSEIN_ECUDA;
    } else {
        PhaseScope ps(plan, 4, s);
        hsein::launch_q0(L, dQ0, ldq, dX, ldx, dZ, ldz, s);
    }
    if (cudaGetLastError() != cudaSuccess) return HSEIN_ECUDA;
    return HSEIN_OK;
}

// Restart loop of Alg. "hsrq3in": the host reads the status array, then for
// trial t = 1, 2, ... solves the shifts that are still not converged again
// from the trial starting vectors of csrc/restart.cu, as a sub-problem with
// its own (host-only) plan whose workspace, shifts, starting vectors and
// results are carved out of dWork.
hsein_status hsein_restart(hsein_plan_t plan, const double* dH, int ldh, const double* dWr,
                           const double* dWi, const double* dB, int ldb, double* dX, int ldx,
                           int* dStatus, int max_tries, int* n_retried, void* dWork,
                           size_t work_bytes, void* stream) {
    if (!plan) return HSEIN_EARG;
    const Layout& L = plan->L;
    if (!dH || ldh < L.n || !dWr || !dWi || !dX || ldx < L.n || !dStatus || max_tries < 0)
        return HSEIN_EARG;
    if (dB && ldb < L.n) return HSEIN_EARG;
    if (!dWork || !aligned256(dWork)) return HSEIN_EARG;
    if (work_bytes < L.total + restart_reserve(L.n)) return HSEIN_ENOMEM;
    if (n_retried) *n_retried = 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int n = L.n, m = L.m;
    std::vector<int> st(m);
    std::vector<double> wi(m);
    if (cudaStreamSynchronize(s) != cudaSuccess ||
        cudaMemcpy(st.data(), dStatus, sizeof(int) * m, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(wi.data(), dWi, sizeof(double) * m, cudaMemcpyDeviceToHost) != cudaSuccess)
        return HSEIN_ECUDA;
    std::vector<int> ucol(m), failed;
    for (int l = 0, c = 0; l < m; ++l) {
        ucol[l] = c;
        c += wi[l] != 0.0 ? 2 : 1;
        if (st[l] == HSEIN_COL_INVALID) return HSEIN_ECUDA;
        if (st[l] == HSEIN_COL_NOT_CONVERGED) failed.push_back(l);
    }
    if (n_retried) *n_retried = (int)failed.size();
    // trial columns n+1-t of the orthogonal factors: t <= n-2 (complex), n-1 (real)
    const int tmax = std::min(max_tries, n - 2);
    for (int t = 1; t <= tmax && !failed.empty(); ++t) {
        std::vector<int> still;
        size_t pos = 0;
        while (pos < failed.size()) {
            // the largest chunk whose sub-problem and buffers fit in dWork
            int k = (int)(failed.size() - pos);
            hsein_plan_t sub = nullptr;
            size_t subw = 0, off_map = 0, off_wr = 0, off_wi = 0, off_st = 0, off_b = 0,
                   off_x = 0, off_sc = 0, end = 0;
            for (;;) {
                int kr = 0, kc = 0;
                for (int j = 0; j < k; ++j) (wi[failed[pos + j]] != 0.0 ? kc : kr)++;
                const size_t ncs = (size_t)kr + 2 * (size_t)kc;
                const hsein_status rc = hsein_plan(&sub, n, kr, kc, &plan->opt, nullptr);
                if (rc != HSEIN_OK) return rc;
                subw = sub->L.total;  // what the sub-solve needs (no restart reserve)
                size_t o = align256(subw);
                auto take = [&](size_t b) {
                    size_t at = o;
                    o = align256(o + b);
                    return at;
                };
                off_map = take(sizeof(int) * 4 * (size_t)k);
                off_wr = take(sizeof(double) * k);
                off_wi = take(sizeof(double) * k);
                off_st = take(sizeof(int) * k);
                off_b = take(sizeof(double) * (size_t)n * ncs);
                off_x = take(sizeof(double) * (size_t)n * ncs);
                off_sc = take(hsein::restart_scratch_bytes(n, k));
                end = o;
                if (end <= work_bytes) break;
                hsein_plan_destroy(sub);
                sub = nullptr;
                if (k == 1) return HSEIN_ENOMEM;
                k = (k + 1) / 2;
            }
            char* w = static_cast<char*>(dWork);
            std::vector<int> map(4 * (size_t)k);
            for (int j = 0, us = 0; j < k; ++j) {
                const int l = failed[pos + j];
                const int cp = wi[l] != 0.0 ? 1 : 0;
                map[4 * j] = l;
                map[4 * j + 1] = ucol[l];
                map[4 * j + 2] = us;
                map[4 * j + 3] = cp;
                us += cp ? 2 : 1;
            }
            int* dmap = reinterpret_cast<int*>(w + off_map);
            double* wr_s = reinterpret_cast<double*>(w + off_wr);
            double* wi_s = reinterpret_cast<double*>(w + off_wi);
            int* st_s = reinterpret_cast<int*>(w + off_st);
            double* Bs = reinterpret_cast<double*>(w + off_b);
            double* Xs = reinterpret_cast<double*>(w + off_x);
            double* scr = reinterpret_cast<double*>(w + off_sc);
            hsein_status rc = HSEIN_OK;
            if (cudaMemcpy(dmap, map.data(), sizeof(int) * map.size(), cudaMemcpyHostToDevice) !=
                cudaSuccess)
                rc = HSEIN_ECUDA;
            if (rc == HSEIN_OK) {
                hsein::launch_restart_trial(n, t, k, dmap, dWr, dWi, dB, ldb, wr_s, wi_s, Bs, scr, s);
                rc = hsein_solve(sub, dH, ldh, wr_s, wi_s, Bs, n, Xs, n, st_s, dWork, subw, stream);
            }
            if (rc == HSEIN_OK) {
                hsein::launch_restart_scatter(n, k, dmap, Xs, st_s, dX, ldx, dStatus, s);
                std::vector<int> sts(k);
                if (cudaMemcpyAsync(sts.data(), st_s, sizeof(int) * k, cudaMemcpyDeviceToHost, s) !=
                        cudaSuccess ||
                    cudaStreamSynchronize(s) != cudaSuccess)
                    rc = HSEIN_ECUDA;
                for (int j = 0; j < k && rc == HSEIN_OK; ++j) {
                    if (sts[j] == HSEIN_COL_INVALID) rc = HSEIN_ECUDA;
                    else if (sts[j] != HSEIN_COL_OK) still.push_back(failed[pos + j]);
                }
            }
            hsein_plan_destroy(sub);
            if (rc != HSEIN_OK) return rc;
            pos += k;
        }
        failed.swap(still);
    }
    if (cudaGetLastError() != cudaSuccess) return HSEIN_ECUDA;
    return failed.empty() ? HSEIN_OK : HSEIN_WNOTCONVERGED;
}

// the device copies of hsein_solve_host's operands, after the solve's own
// workspace: H and Q0 (n x n), B, X and Z (n x ncol, leading dimension n),
// the shifts and the statuses
namespace {
struct HostLayout {
    size_t off_h, off_q, off_b, off_x, off_z, off_wr, off_wi, off_st, total;
};
HostLayout host_layout(const Layout& L) {
    HostLayout h;
    size_t o = align256(L.total);
    auto take = [&](size_t b) {
        size_t at = o;
        o = align256(o + b);
        return at;
    };
    const size_t n = L.n, nc = L.ncol, m = L.m;
    h.off_h = take(sizeof(double) * n * n);
    h.off_q = take(sizeof(double) * n * n);
    h.off_b = take(sizeof(double) * n * nc);
    h.off_x = take(sizeof(double) * n * nc);
    h.off_z = take(sizeof(double) * n * nc);
    h.off_wr = take(sizeof(double) * m);
    h.off_wi = take(sizeof(double) * m);
    h.off_st = take(sizeof(int) * m);
    h.total = o;
    return h;
}
}  // namespace

hsein_status hsein_host_workspace(hsein_plan_t plan, size_t* workspace_bytes) {
    if (!plan || !workspace_bytes) return HSEIN_EARG;
    *workspace_bytes = host_layout(plan->L).total;
    return HSEIN_OK;
}

hsein_status hsein_solve_host(hsein_plan_t plan, const double* hH, int ldh, const double* hWr,
                              const double* hWi, const double* hB, int ldb, const double* hQ0,
                              int ldq, double* hZ, int ldz, int* hStatus, void* dWork,
                              size_t work_bytes, void* stream) {
    if (!plan) return HSEIN_EARG;
    const Layout& L = plan->L;
    if (!hH || ldh < L.n || !hWr || !hWi || !hQ0 || ldq < L.n || !hZ || ldz < L.n || !hStatus)
        return HSEIN_EARG;
    if (hB && ldb < L.n) return HSEIN_EARG;
    if (!dWork || !aligned256(dWork)) return HSEIN_EARG;
    const HostLayout h = host_layout(L);
    if (work_bytes < h.total) return HSEIN_ENOMEM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!plan->side) {
        if (cudaStreamCreateWithFlags(&plan->side, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&plan->ev_q0, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&plan->ev_done, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return HSEIN_ECUDA;
        }
    }
    char* w = static_cast<char*>(dWork);
    double* dH = reinterpret_cast<double*>(w + h.off_h);
    double* dQ = reinterpret_cast<double*>(w + h.off_q);
    double* dB = reinterpret_cast<double*>(w + h.off_b);
    double* dX = reinterpret_cast<double*>(w + h.off_x);
    double* dZ = reinterpret_cast<double*>(w + h.off_z);
    double* dWr = reinterpret_cast<double*>(w + h.off_wr);
    double* dWi = reinterpret_cast<double*>(w + h.off_wi);
    int* dSt = reinterpret_cast<int*>(w + h.off_st);
    const size_t n = L.n, nc = L.ncol, m = L.m, row = sizeof(double) * n;
    // the solve's inputs on the caller's stream; Q0 (needed only by the
    // backtransform) on the side stream meanwhile, once the previous call's
    // backtransform has read the device copy
    bool ok = cudaMemcpy2DAsync(dH, row, hH, sizeof(double) * ldh, row, n, cudaMemcpyHostToDevice,
                                s) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(dWr, hWr, sizeof(double) * m, cudaMemcpyHostToDevice, s) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(dWi, hWi, sizeof(double) * m, cudaMemcpyHostToDevice, s) == cudaSuccess;
    if (hB)
        ok = ok && cudaMemcpy2DAsync(dB, row, hB, sizeof(double) * ldb, row, nc,
                                     cudaMemcpyHostToDevice, s) == cudaSuccess;
    ok = ok && cudaStreamWaitEvent(plan->side, plan->ev_done, 0) == cudaSuccess;
    ok = ok && cudaMemcpy2DAsync(dQ, row, hQ0, sizeof(double) * ldq, row, n,
                                 cudaMemcpyHostToDevice, plan->side) == cudaSuccess;
    ok = ok && cudaEventRecord(plan->ev_q0, plan->side) == cudaSuccess;
    if (!ok) return HSEIN_ECUDA;
    // the solve on the device copies: as a graph captured at the first call
    // with this workspace (one launch instead of one per kernel), or launch
    // by launch while the plan records per-launch profiling events
    hsein_status rc = HSEIN_OK;
    if (plan->profiling) {
        rc = hsein_solve(plan, dH, (int)n, dWr, dWi, hB ? dB : nullptr, (int)n, dX, (int)n, dSt,
                         dWork, L.total, stream);
    } else {
        if (!plan->host_graph || plan->host_graph_work != dWork ||
            plan->host_graph_b != (hB != nullptr)) {
            hsein_graph_destroy(plan->host_graph);
            plan->host_graph = nullptr;
            rc = hsein_graph_create(plan, dH, (int)n, dWr, dWi, hB ? dB : nullptr, (int)n, dX,
                                    (int)n, dSt, nullptr, 0, nullptr, 0, dWork, L.total,
                                    &plan->host_graph);
            plan->host_graph_work = dWork;
            plan->host_graph_b = hB != nullptr;
        }
        if (rc == HSEIN_OK) rc = hsein_graph_launch(plan->host_graph, stream);
    }
    if (rc != HSEIN_OK) return rc;
    if (cudaStreamWaitEvent(s, plan->ev_q0, 0) != cudaSuccess) return HSEIN_ECUDA;
    rc = hsein_backtransform(plan, dQ, (int)n, dX, (int)n, dZ, (int)n, dWork, L.total, stream);
    if (rc != HSEIN_OK) return rc;
    ok = cudaEventRecord(plan->ev_done, s) == cudaSuccess;
    ok = ok && cudaMemcpy2DAsync(hZ, sizeof(double) * ldz, dZ, row, row, nc,
                                 cudaMemcpyDeviceToHost, s) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(hStatus, dSt, sizeof(int) * m, cudaMemcpyDeviceToHost, s) == cudaSuccess;
    return ok ? HSEIN_OK : HSEIN_ECUDA;
}

hsein_status hsein_margins(hsein_plan_t plan, const void* dWork, double* dMargin, void* stream) {
    if (!plan || !dWork || !dMargin) return HSEIN_EARG;
    const char* src = static_cast<const char*>(dWork) + plan->L.off_margin;
    if (cudaMemcpyAsync(dMargin, src, sizeof(double) * plan->L.m, cudaMemcpyDeviceToDevice,
                        static_cast<cudaStream_t>(stream)) != cudaSuccess)
        return HSEIN_ECUDA;
    return HSEIN_OK;
}

hsein_status hsein_plan_sync_status(hsein_plan_t plan, const void* dWork, void* stream) {
    if (!plan || !dWork) return HSEIN_EARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int st = 0;
    const char* base = static_cast<const char*>(dWork) + plan->L.off_state;
    if (cudaMemcpyAsync(&st, base + offsetof(hsein::DevState, status), sizeof(int),
                        cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return HSEIN_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return HSEIN_ECUDA;
    return static_cast<hsein_status>(st);
}

hsein_status hsein_plan_set_profiling(hsein_plan_t plan, int enable) {
    if (!plan) return HSEIN_EARG;
    plan->profiling = enable ? 1 : 0;
    return HSEIN_OK;
}

hsein_status hsein_plan_profile(hsein_plan_t plan, double* ms, int* launches, int nphases,
                                int reset) {
    if (!plan || nphases < 0 || nphases > HSEIN_NUM_PHASES) return HSEIN_EARG;
    for (int i = 0; i < nphases; ++i) {
        if (ms) ms[i] = 0.0;
        if (launches) launches[i] = 0;
    }
    const size_t nrec = plan->rec_phase.size();
    if (nrec > 0) {
        if (cudaEventSynchronize(plan->pool[2 * nrec - 1]) != cudaSuccess) return HSEIN_ECUDA;
        for (size_t r = 0; r < nrec; ++r) {
            float t = 0.0f;
            if (cudaEventElapsedTime(&t, plan->pool[2 * r], plan->pool[2 * r + 1]) != cudaSuccess)
                return HSEIN_ECUDA;
            int ph = plan->rec_phase[r];
            if (ph < nphases) {
                if (ms) ms[ph] += t;
                if (launches) launches[ph] += 1;
            }
        }
    }
    if (reset) {
        plan->used = 0;
        plan->rec_phase.clear();
    }
    return HSEIN_OK;
}

hsein_status hsein_graph_create(hsein_plan_t plan, const double* dH, int ldh, const double* dWr,
                                const double* dWi, const double* dB, int ldb, double* dX, int ldx,
                                int* dStatus, const double* dQ0, int ldq, double* dZ, int ldz,
                                void* dWork, size_t work_bytes, hsein_graph_t* graph) {
    if (!graph) return HSEIN_EARG;
    *graph = nullptr;
    if (!plan || (dQ0 && !dZ)) return HSEIN_EARG;
    // a capture stream of its own (the legacy default stream cannot be
    // captured); thread-local mode, so other threads' CUDA calls meanwhile
    // do not invalidate the capture
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return HSEIN_ECUDA;
    const int profiling = plan->profiling;
    plan->profiling = 0;
    hsein_status rc = HSEIN_OK;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        rc = HSEIN_ECUDA;
    } else {
        rc = hsein_solve(plan, dH, ldh, dWr, dWi, dB, ldb, dX, ldx, dStatus, dWork, work_bytes, cs);
        if (rc == HSEIN_OK && dQ0)
            rc = hsein_backtransform(plan, dQ0, ldq, dX, ldx, dZ, ldz, dWork, work_bytes, cs);
        if (cudaStreamEndCapture(cs, &g) != cudaSuccess && rc == HSEIN_OK) rc = HSEIN_ECUDA;
    }
    plan->profiling = profiling;
    hsein_graph_s* h = nullptr;
    if (rc == HSEIN_OK) {
        h = new (std::nothrow) hsein_graph_s;
        if (!h) rc = HSEIN_ENOMEM;
        else if (cudaGraphInstantiate(&h->exec, g, 0) != cudaSuccess) rc = HSEIN_ECUDA;
    }
    if (rc != HSEIN_OK) {
        delete h;
        h = nullptr;
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
    } else {
        h->graph = g;
    }
    cudaStreamDestroy(cs);
    *graph = h;
    return rc;
}

hsein_status hsein_graph_launch(hsein_graph_t graph, void* stream) {
    if (!graph || !graph->exec) return HSEIN_EARG;
    return cudaGraphLaunch(graph->exec, static_cast<cudaStream_t>(stream)) == cudaSuccess
               ? HSEIN_OK
               : HSEIN_ECUDA;
}

hsein_status hsein_graph_destroy(hsein_graph_t graph) {
    if (graph) {
        if (graph->exec) cudaGraphExecDestroy(graph->exec);
        if (graph->graph) cudaGraphDestroy(graph->graph);
    }
    delete graph;
    return HSEIN_OK;
}

hsein_status hsein_plan_destroy(hsein_plan_t plan) {
    if (plan) {
        for (cudaEvent_t e : plan->pool) cudaEventDestroy(e);
        if (plan->ev_q0) cudaEventDestroy(plan->ev_q0);
        if (plan->ev_done) cudaEventDestroy(plan->ev_done);
        if (plan->side) cudaStreamDestroy(plan->side);
        hsein_graph_destroy(plan->host_graph);
    }
    delete plan;
    return HSEIN_OK;
}

const char* hsein_status_string(hsein_status status) {
    switch (status) {
        case HSEIN_OK: return "ok";
        case HSEIN_EARG: return "invalid argument";
        case HSEIN_ENOMEM: return "out of memory or workspace too small";
        case HSEIN_ENOTUNREDUCED: return "H is reduced: a subdiagonal entry is zero";
        case HSEIN_ENONFINITE: return "H or a shift is not finite";
        case HSEIN_ECUDA: return "CUDA error";
        case HSEIN_ETIMEOUT: return "a bounded wait on the device ran out";
        case HSEIN_ESHIFTS: return "number of complex shifts differs from the plan";
        case HSEIN_WNOTCONVERGED: return "some columns did not converge (set to zero)";
    }
    return "unknown status";
}

}  // extern "C"
