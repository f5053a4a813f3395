// Serving runtime (include/hsein.h, hsein_server_*): a request loop with
// continuous batching, host-side over the library's C ABI.
//
//  - one device arena (cudaMalloc once, first-fit with coalescing) holds the
//    workspace of every solve in flight and the gathered arrays of fused
//    requests: admission is by HBM footprint;
//  - a pool of streams, one per solve in flight, so admitted solves overlap
//    on the device while new requests keep arriving;
//  - requests on the same matrix that are pending together are fused into
//    one solve of the union of their shift sets: their shifts and starting
//    vectors are gathered into the arena (device-to-device copies on the
//    solve's stream), one hsein_solve runs, and the columns and statuses are
//    scattered back to each request's buffers.  Every column of the solve
//    depends only on its own shift and starting vector, so each request gets
//    exactly what hsein_solve gives it alone.
// The caller drives it from one thread (submit / progress).
#include "../../include/hsein.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <deque>
#include <iterator>
#include <map>
#include <new>
#include <vector>

namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kNoBlock = ~(size_t)0;
constexpr int kMaxJobs = 64;

// first-fit allocator over one device allocation; offsets are 256-aligned
class Arena {
  public:
    bool init(size_t bytes) {
        size_ = bytes & ~(size_t)255;
        if (size_ == 0 || cudaMalloc(&base_, size_) != cudaSuccess) {
            cudaGetLastError();
            base_ = nullptr;
            return false;
        }
        free_[0] = size_;
        return true;
    }
    void release() {
        if (base_) cudaFree(base_);
        base_ = nullptr;
    }
    size_t alloc(size_t bytes) {
        bytes = align256(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            const size_t off = it->first, rem = it->second - bytes;
            free_.erase(it);
            if (rem) free_[off + bytes] = rem;
            used_ += bytes;
            return off;
        }
        return kNoBlock;
    }
    void free(size_t off, size_t bytes) {
        bytes = align256(bytes);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    char* ptr(size_t off) const { return static_cast<char*>(base_) + off; }
    size_t size() const { return size_; }
    size_t used() const { return used_; }

  private:
    void* base_ = nullptr;
    size_t size_ = 0, used_ = 0;
    std::map<size_t, size_t> free_;
};

struct Pending {
    long long ticket;
    hsein_request req;
};

struct Job {
    std::vector<long long> tickets;
    hsein_plan_t plan = nullptr;
    size_t off = 0, bytes = 0;
    int slot = -1;
};

int shifts(const hsein_request& r) { return r.inst.m_real + r.inst.m_cplx; }
int columns(const hsein_request& r) { return r.inst.m_real + 2 * r.inst.m_cplx; }

// requests that can share one solve
bool same_solve(const hsein_request& a, const hsein_request& b) {
    return a.inst.dH == b.inst.dH && a.inst.n == b.inst.n && a.inst.ldh == b.inst.ldh &&
           a.dExp == b.dExp &&
           a.precision == b.precision && a.br == b.br && (a.inst.dB == nullptr) == (b.inst.dB == nullptr);
}

hsein_options options_for(const hsein_options& base, const hsein_request& r) {
    hsein_options o = base;
    o.precision = r.precision;
    o.br = r.precision == 1 ? 64 : (r.br ? r.br : 64);
    return o;
}

}  // namespace

struct hsein_server_s {
    Arena arena;
    hsein_options opt;
    int max_jobs = 0, max_merge = 0;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    std::vector<bool> busy;
    std::deque<Pending> pending;
    std::vector<Job> running;
    std::deque<long long> finished;
    long long next_ticket = 1;
    long long req_admitted = 0, solves_admitted = 0;
    // head-of-line bypass: later requests admitted while the oldest one does
    // not fit, at most max_bypass of them per oldest request
    int max_bypass = 0;
    long long head_ticket = 0;
    int head_bypassed = 0;
};

namespace {

// workspace + gathered arrays of a solve of `group` (indices into pending)
hsein_status footprint(const hsein_server_s* S, const std::vector<size_t>& group,
                       hsein_plan_t* plan, size_t* ws, size_t* total) {
    const hsein_request& h = S->pending[group[0]].req;
    int mr = 0, mc = 0;
    for (size_t i : group) {
        mr += S->pending[i].req.inst.m_real;
        mc += S->pending[i].req.inst.m_cplx;
    }
    const hsein_options o = options_for(S->opt, h);
    size_t w = 0;
    const hsein_status rc = hsein_plan(plan, h.inst.n, mr, mc, &o, &w);
    if (rc != HSEIN_OK) return rc;
    size_t t = align256(w);
    if (group.size() > 1) {
        const size_t m = (size_t)mr + mc, nc = (size_t)mr + 2 * (size_t)mc, n = h.inst.n;
        t += 2 * align256(sizeof(double) * m) + align256(sizeof(int) * m) +
             align256(sizeof(double) * n * nc) * (h.inst.dB ? 2 : 1);
    }
    *ws = w;
    *total = t;
    return HSEIN_OK;
}

hsein_status launch(hsein_server_s* S, const std::vector<size_t>& group, hsein_plan_t plan,
                    size_t ws, size_t off, size_t total, int slot) {
    cudaStream_t s = S->streams[slot];
    const hsein_request& h = S->pending[group[0]].req;
    const int n = h.inst.n;
    char* base = S->arena.ptr(off);
    hsein_status rc = HSEIN_OK;
    if (group.size() == 1) {
        const hsein_instance& in = h.inst;
        rc = hsein_solve(plan, in.dH, in.ldh, in.dWr, in.dWi, in.dB, in.ldb, in.dX, in.ldx,
                         in.dStatus, base, ws, s);
    } else {
        int M = 0, NC = 0;
        for (size_t i : group) {
            M += shifts(S->pending[i].req);
            NC += columns(S->pending[i].req);
        }
        size_t o = align256(ws);
        auto take = [&](size_t b) {
            char* p = base + o;
            o += align256(b);
            return p;
        };
        double* wr = reinterpret_cast<double*>(take(sizeof(double) * M));
        double* wi = reinterpret_cast<double*>(take(sizeof(double) * M));
        int* st = reinterpret_cast<int*>(take(sizeof(int) * M));
        double* X = reinterpret_cast<double*>(take(sizeof(double) * (size_t)n * NC));
        double* B = h.inst.dB ? reinterpret_cast<double*>(take(sizeof(double) * (size_t)n * NC)) : nullptr;
        (void)total;
        bool ok = true;
        int m0 = 0, c0 = 0;
        for (size_t i : group) {
            const hsein_instance& in = S->pending[i].req.inst;
            const int m = in.m_real + in.m_cplx, nc = in.m_real + 2 * in.m_cplx;
            ok = ok && cudaMemcpyAsync(wr + m0, in.dWr, sizeof(double) * m, cudaMemcpyDeviceToDevice, s) == cudaSuccess;
            ok = ok && cudaMemcpyAsync(wi + m0, in.dWi, sizeof(double) * m, cudaMemcpyDeviceToDevice, s) == cudaSuccess;
            if (B)
                ok = ok && cudaMemcpy2DAsync(B + (size_t)c0 * n, sizeof(double) * n, in.dB,
                                             sizeof(double) * in.ldb, sizeof(double) * n, nc,
                                             cudaMemcpyDeviceToDevice, s) == cudaSuccess;
            m0 += m;
            c0 += nc;
        }
        if (!ok) return HSEIN_ECUDA;
        rc = hsein_solve(plan, h.inst.dH, h.inst.ldh, wr, wi, B, n, X, n, st, base, ws, s);
        m0 = c0 = 0;
        for (size_t i : group) {
            if (rc != HSEIN_OK) break;
            const hsein_instance& in = S->pending[i].req.inst;
            const int m = in.m_real + in.m_cplx, nc = in.m_real + 2 * in.m_cplx;
            ok = ok && cudaMemcpy2DAsync(in.dX, sizeof(double) * in.ldx, X + (size_t)c0 * n,
                                         sizeof(double) * n, sizeof(double) * n, nc,
                                         cudaMemcpyDeviceToDevice, s) == cudaSuccess;
            ok = ok && cudaMemcpyAsync(in.dStatus, st + m0, sizeof(int) * m, cudaMemcpyDeviceToDevice, s) == cudaSuccess;
            m0 += m;
            c0 += nc;
        }
        if (rc == HSEIN_OK && !ok) rc = HSEIN_ECUDA;
    }
    // eigenvectors of a balanced matrix back to the caller's matrix
    for (size_t i : group) {
        if (rc != HSEIN_OK) break;
        const hsein_request& r = S->pending[i].req;
        if (r.dExp)
            rc = hsein_unbalance(n, shifts(r), r.inst.dWi, r.dExp, r.inst.dX, r.inst.ldx, s);
    }
    if (rc == HSEIN_OK && cudaEventRecord(S->events[slot], s) != cudaSuccess) rc = HSEIN_ECUDA;
    return rc;
}

hsein_status retire(hsein_server_s* S) {
    for (size_t j = 0; j < S->running.size();) {
        Job& job = S->running[j];
        const cudaError_t e = cudaEventQuery(S->events[job.slot]);
        if (e == cudaErrorNotReady) {
            ++j;
            continue;
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            return HSEIN_ECUDA;
        }
        S->arena.free(job.off, job.bytes);
        hsein_plan_destroy(job.plan);
        S->busy[job.slot] = false;
        for (long long t : job.tickets) S->finished.push_back(t);
        S->running.erase(S->running.begin() + j);
    }
    return HSEIN_OK;
}

// admit pending request h (and the later pending requests that can share its
// solve) into `slot` if its footprint fits the arena; *done tells whether it
// did
hsein_status try_admit(hsein_server_s* S, size_t h, int slot, bool* done) {
    *done = false;
    std::vector<size_t> group{h};
    int M = shifts(S->pending[h].req);
    for (size_t i = h + 1; i < S->pending.size(); ++i) {
        const hsein_request& r = S->pending[i].req;
        if (same_solve(r, S->pending[h].req) && M + shifts(r) <= S->max_merge) {
            group.push_back(i);
            M += shifts(r);
        }
    }
    // the largest prefix of the group whose footprint fits the arena now
    hsein_plan_t plan = nullptr;
    size_t ws = 0, total = 0, off = kNoBlock;
    for (;;) {
        const hsein_status rc = footprint(S, group, &plan, &ws, &total);
        if (rc != HSEIN_OK) return rc;
        off = S->arena.alloc(total);
        if (off != kNoBlock) break;
        hsein_plan_destroy(plan);
        plan = nullptr;
        if (group.size() == 1) return HSEIN_OK;  // does not fit now
        group.pop_back();
    }
    Job job;
    job.plan = plan;
    job.off = off;
    job.bytes = total;
    job.slot = slot;
    for (size_t i : group) job.tickets.push_back(S->pending[i].ticket);
    const hsein_status rc = launch(S, group, plan, ws, off, total, slot);
    if (rc != HSEIN_OK) {
        S->arena.free(off, total);
        hsein_plan_destroy(plan);
        return rc;
    }
    S->busy[slot] = true;
    S->running.push_back(job);
    S->req_admitted += (long long)group.size();
    S->solves_admitted += 1;
    for (auto it = group.rbegin(); it != group.rend(); ++it)
        S->pending.erase(S->pending.begin() + (std::ptrdiff_t)*it);
    *done = true;
    return HSEIN_OK;
}

// how many pending requests behind the oldest one are looked at for a bypass
constexpr size_t kBypassScan = 64;

hsein_status admit(hsein_server_s* S) {
    while (!S->pending.empty()) {
        int slot = -1;
        for (int k = 0; k < S->max_jobs; ++k)
            if (!S->busy[k]) {
                slot = k;
                break;
            }
        if (slot < 0) return HSEIN_OK;
        // the oldest request and the later ones that can share its solve
        const long long head = S->pending[0].ticket;
        bool done = false;
        hsein_status rc = try_admit(S, 0, slot, &done);
        if (rc != HSEIN_OK) return rc;
        if (done) continue;
        // it does not fit: wait for memory (arrival order is kept), unless
        // later requests may bypass it
        if (S->head_ticket != head) {
            S->head_ticket = head;
            S->head_bypassed = 0;
        }
        if (S->head_bypassed >= S->max_bypass) return HSEIN_OK;
        const size_t lim = std::min(S->pending.size(), kBypassScan + 1);
        for (size_t h = 1; h < lim && !done; ++h) {
            rc = try_admit(S, h, slot, &done);
            if (rc != HSEIN_OK) return rc;
        }
        if (!done) return HSEIN_OK;
        S->head_bypassed += 1;
    }
    return HSEIN_OK;
}

void destroy(hsein_server_s* S) {
    for (Job& j : S->running) {
        cudaEventSynchronize(S->events[j.slot]);
        hsein_plan_destroy(j.plan);
    }
    for (cudaStream_t s : S->streams)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : S->events)
        if (e) cudaEventDestroy(e);
    S->arena.release();
    delete S;
}

}  // namespace

extern "C" {

hsein_status hsein_server_set_bypass(hsein_server_t server, int max_bypass) {
    if (!server || max_bypass < 0) return HSEIN_EARG;
    server->max_bypass = max_bypass;
    return HSEIN_OK;
}

hsein_status hsein_server_create(hsein_server_t* server, size_t hbm_bytes, int max_jobs,
                                 int max_merge_shifts, const hsein_options* opt) {
    if (!server) return HSEIN_EARG;
    *server = nullptr;
    if (max_jobs < 1 || max_jobs > kMaxJobs || max_merge_shifts < 1) return HSEIN_EARG;
    hsein_server_s* S = new (std::nothrow) hsein_server_s;
    if (!S) return HSEIN_ENOMEM;
    if (opt) S->opt = *opt;
    else hsein_default_options(&S->opt);
    S->max_jobs = max_jobs;
    S->max_merge = max_merge_shifts;
    S->streams.assign(max_jobs, nullptr);
    S->events.assign(max_jobs, nullptr);
    S->busy.assign(max_jobs, false);
    bool ok = true;
    for (int k = 0; k < max_jobs && ok; ++k)
        ok = cudaStreamCreateWithFlags(&S->streams[k], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&S->events[k], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        destroy(S);
        return HSEIN_ECUDA;
    }
    if (!S->arena.init(hbm_bytes)) {
        destroy(S);
        return HSEIN_ENOMEM;
    }
    *server = S;
    return HSEIN_OK;
}

hsein_status hsein_server_submit(hsein_server_t S, const hsein_request* req, long long* ticket) {
    if (!S || !req || !ticket) return HSEIN_EARG;
    const hsein_instance& in = req->inst;
    const int m = in.m_real + in.m_cplx;
    if (in.n < 1 || in.m_real < 0 || in.m_cplx < 0 || m < 1 || !in.dH || in.ldh < in.n ||
        !in.dWr || !in.dWi || !in.dX || in.ldx < in.n || !in.dStatus ||
        (in.dB && in.ldb < in.n) || (req->precision != 0 && req->precision != 1))
        return HSEIN_EARG;
    // its footprint alone must fit the arena
    const hsein_options o = options_for(S->opt, *req);
    hsein_plan_t p = nullptr;
    size_t w = 0;
    const hsein_status rc = hsein_plan(&p, in.n, in.m_real, in.m_cplx, &o, &w);
    if (rc != HSEIN_OK) return rc;
    hsein_plan_destroy(p);
    if (align256(w) > S->arena.size()) return HSEIN_ENOMEM;
    *ticket = S->next_ticket++;
    S->pending.push_back(Pending{*ticket, *req});
    return HSEIN_OK;
}

hsein_status hsein_server_progress(hsein_server_t S, long long* done, int max_done, int* n_done,
                                   int wait) {
    if (!S || (max_done > 0 && !done)) return HSEIN_EARG;
    if (n_done) *n_done = 0;
    hsein_status rc = retire(S);
    if (rc == HSEIN_OK) rc = admit(S);
    if (rc == HSEIN_OK && wait && S->finished.empty() && !S->running.empty()) {
        if (cudaEventSynchronize(S->events[S->running.front().slot]) != cudaSuccess) {
            cudaGetLastError();
            return HSEIN_ECUDA;
        }
        rc = retire(S);
        if (rc == HSEIN_OK) rc = admit(S);
    }
    if (rc != HSEIN_OK) return rc;
    int k = 0;
    while (k < max_done && !S->finished.empty()) {
        done[k++] = S->finished.front();
        S->finished.pop_front();
    }
    if (n_done) *n_done = k;
    return HSEIN_OK;
}

hsein_status hsein_server_stats(hsein_server_t S, int* pending, int* running, size_t* bytes_in_use,
                                long long* requests_admitted, long long* solves_admitted) {
    if (!S) return HSEIN_EARG;
    if (pending) *pending = (int)S->pending.size();
    if (running) *running = (int)S->running.size();
    if (bytes_in_use) *bytes_in_use = S->arena.used();
    if (requests_admitted) *requests_admitted = S->req_admitted;
    if (solves_admitted) *solves_admitted = S->solves_admitted;
    return HSEIN_OK;
}

hsein_status hsein_server_destroy(hsein_server_t S) {
    if (!S) return HSEIN_EARG;
    destroy(S);
    return HSEIN_OK;
}

}  // extern "C"
