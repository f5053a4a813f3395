// Batches of independent instances in one CUDA graph (include/hsein.h,
// hsein_batch_*): host-side runtime over the library's own C ABI.
//
// The paper solves one matrix at a time and groups the shifts of that matrix
// so that the cross-over columns of one group fit a workspace (Sec. 4.4,
// Alg. "hsrq3infinal").  Here a batch is many matrices; every instance, or
// every block of at most cfg.shift_block of its shifts, becomes a
// sub-problem with its own plan (tile height by cfg.br_policy) and its own
// slice of one workspace.  Sub-problems are assigned longest first to the
// least loaded of cfg.streams chains (LPT), and the whole batch -- a fork
// from the caller's stream, the chains' hsein_solve launch sequences, a join
// -- is captured once into a CUDA graph that later solves replay, so a batch
// of hundreds of small instances costs one graph launch on the host and runs
// its chains concurrently on the GPU.
#include "../../include/hsein.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <new>
#include <vector>

namespace {

struct Task {
    int inst;          // instance index
    int first, count;  // shifts [first, first + count) of the instance
    int col;           // first solution column of those shifts
    int mr, mc;        // real / complex shifts among them
    double cost;       // estimated work, for the chain assignment
};

struct Sub {
    hsein_plan_t plan = nullptr;
    size_t off = 0, bytes = 0;  // slice of the workspace
};

constexpr int kMaxStreams = 64;

int tile_height(int policy, int n) {
    switch (policy) {
        case 1: return n < 512 ? 32 : 64;
        case 2: return n < 256 ? 16 : (n < 1024 ? 32 : 64);
        default: return 64;
    }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bool valid_config(const hsein_batch_config& c) {
    return c.streams >= 1 && c.streams <= kMaxStreams && c.br_policy >= 0 && c.br_policy <= 2 &&
           c.shift_block >= 0;
}

}  // namespace

struct hsein_batch_s {
    std::vector<hsein_instance> inst;
    std::vector<std::vector<double>> wi;  // host copy of every instance's shifts' imaginary parts
    hsein_options opt;
    hsein_batch_config cfg;
    std::vector<Task> tasks;
    std::vector<Sub> subs;
    std::vector<std::vector<int>> chains;
    size_t total = 0;
    std::vector<cudaStream_t> streams;
    // the graph is captured and launched on a private stream (the caller's
    // may be the legacy default stream, which cannot capture), ordered
    // after and before the caller's stream by ev_in / ev_out
    cudaStream_t origin = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> joins;
    cudaGraphExec_t exec = nullptr;
    const void* exec_work = nullptr;
};

namespace {

void free_subs(hsein_batch_s* b) {
    for (Sub& s : b->subs)
        if (s.plan) hsein_plan_destroy(s.plan);
    b->subs.clear();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    b->exec_work = nullptr;
}

// split every instance into blocks of at most `block` shifts (0: one block)
std::vector<Task> make_tasks(const hsein_batch_s* b, int block) {
    std::vector<Task> t;
    for (int i = 0; i < (int)b->inst.size(); ++i) {
        const hsein_instance& in = b->inst[i];
        const int m = in.m_real + in.m_cplx;
        const int w = block > 0 ? block : m;
        int col = 0;
        for (int f = 0; f < m; f += w) {
            Task k{};
            k.inst = i;
            k.first = f;
            k.count = std::min(w, m - f);
            k.col = col;
            for (int l = f; l < f + k.count; ++l) (b->wi[i][l] != 0.0 ? k.mc : k.mr)++;
            col += k.mr + 2 * k.mc;
            const double n = in.n, nc = k.mr + 2 * k.mc;
            k.cost = n * n * nc + 64.0 * n * nc;  // update products + diagonal sweeps
            t.push_back(k);
        }
    }
    return t;
}

// workspace of a configuration without keeping its plans
hsein_status config_bytes(const hsein_batch_s* b, const hsein_batch_config& c, size_t* bytes) {
    size_t tot = 0;
    for (const Task& k : make_tasks(b, c.shift_block)) {
        hsein_options o = b->opt;
        o.br = tile_height(c.br_policy, b->inst[k.inst].n);
        hsein_plan_t p = nullptr;
        size_t w = 0;
        const hsein_status rc = hsein_plan(&p, b->inst[k.inst].n, k.mr, k.mc, &o, &w);
        if (rc != HSEIN_OK) return rc;
        hsein_plan_destroy(p);
        tot += align256(w);
    }
    *bytes = tot;
    return HSEIN_OK;
}

// plans, workspace slices and chains of configuration c
hsein_status apply_config(hsein_batch_s* b, const hsein_batch_config& c) {
    free_subs(b);
    b->cfg = c;
    b->tasks = make_tasks(b, c.shift_block);
    b->subs.resize(b->tasks.size());
    size_t off = 0;
    for (size_t j = 0; j < b->tasks.size(); ++j) {
        const Task& k = b->tasks[j];
        hsein_options o = b->opt;
        o.br = tile_height(c.br_policy, b->inst[k.inst].n);
        size_t w = 0;
        const hsein_status rc = hsein_plan(&b->subs[j].plan, b->inst[k.inst].n, k.mr, k.mc, &o, &w);
        if (rc != HSEIN_OK) {
            free_subs(b);
            return rc;
        }
        b->subs[j].off = off;
        b->subs[j].bytes = w;
        off += align256(w);
    }
    b->total = off;
    // longest processing time first, each to the least loaded chain
    std::vector<int> order(b->tasks.size());
    for (size_t j = 0; j < order.size(); ++j) order[j] = (int)j;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int z) { return b->tasks[a].cost > b->tasks[z].cost; });
    const int K = std::min<int>(c.streams, std::max<int>(1, (int)order.size()));
    b->chains.assign(K, {});
    std::vector<double> load(K, 0.0);
    for (int j : order) {
        const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        b->chains[k].push_back(j);
        load[k] += b->tasks[j].cost;
    }
    return HSEIN_OK;
}

hsein_status capture(hsein_batch_s* b, void* dWork, cudaStream_t s) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    b->exec_work = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return HSEIN_ECUDA;
    }
    hsein_status rc = HSEIN_OK;
    if (cudaEventRecord(b->fork, s) != cudaSuccess) rc = HSEIN_ECUDA;
    const int K = (int)b->chains.size();
    for (int k = 0; k < K && rc == HSEIN_OK; ++k)
        if (cudaStreamWaitEvent(b->streams[k], b->fork, 0) != cudaSuccess) rc = HSEIN_ECUDA;
    for (int k = 0; k < K && rc == HSEIN_OK; ++k) {
        for (int j : b->chains[k]) {
            const Task& t = b->tasks[j];
            const hsein_instance& in = b->inst[t.inst];
            const Sub& sb = b->subs[j];
            rc = hsein_solve(sb.plan, in.dH, in.ldh, in.dWr + t.first, in.dWi + t.first,
                             in.dB ? in.dB + (size_t)t.col * in.ldb : nullptr, in.ldb,
                             in.dX + (size_t)t.col * in.ldx, in.ldx, in.dStatus + t.first,
                             static_cast<char*>(dWork) + sb.off, sb.bytes, b->streams[k]);
            if (rc != HSEIN_OK) break;
        }
    }
    for (int k = 0; k < K; ++k) {
        // the join always runs, so that the capture can end cleanly
        cudaEventRecord(b->joins[k], b->streams[k]);
        cudaStreamWaitEvent(s, b->joins[k], 0);
    }
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(s, &g);
    if (rc == HSEIN_OK && (ec != cudaSuccess || !g)) rc = HSEIN_ECUDA;
    if (rc == HSEIN_OK && cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
        b->exec = nullptr;
        rc = HSEIN_ECUDA;
    }
    if (g) cudaGraphDestroy(g);
    if (rc != HSEIN_OK) {
        cudaGetLastError();
        return rc;
    }
    b->exec_work = dWork;
    return HSEIN_OK;
}

void destroy(hsein_batch_s* b) {
    free_subs(b);
    for (cudaStream_t s : b->streams)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->joins)
        if (e) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->origin) cudaStreamDestroy(b->origin);
    delete b;
}

// the candidate set the autotuner searches (coordinate-wise, in this order)
const int kPolicies[] = {0, 1, 2};
const int kBlocks[] = {0, 512, 256, 128};
const int kStreams[] = {4, 8, 16, 24, 32, 48};

}  // namespace

extern "C" {

hsein_status hsein_batch_plan(hsein_batch_t* batch, int count, const hsein_instance* inst,
                              const hsein_options* opt, const hsein_batch_config* cfg,
                              size_t* workspace_bytes) {
    if (!batch) return HSEIN_EARG;
    *batch = nullptr;
    if (count < 1 || !inst) return HSEIN_EARG;
    hsein_batch_config c{16, 1, 0, 0};
    if (cfg) c = *cfg;
    if (c.streams == 0) c.streams = 16;
    if (!valid_config(c)) return HSEIN_EARG;
    hsein_batch_s* b = new (std::nothrow) hsein_batch_s;
    if (!b) return HSEIN_ENOMEM;
    if (opt) b->opt = *opt;
    else hsein_default_options(&b->opt);
    b->inst.assign(inst, inst + count);
    b->wi.resize(count);
    for (int i = 0; i < count; ++i) {
        const hsein_instance& in = inst[i];
        const int m = in.m_real + in.m_cplx;
        if (in.n < 1 || in.m_real < 0 || in.m_cplx < 0 || m < 1 || !in.dH || in.ldh < in.n ||
            !in.dWr || !in.dWi || !in.dX || in.ldx < in.n || !in.dStatus ||
            (in.dB && in.ldb < in.n)) {
            destroy(b);
            return HSEIN_EARG;
        }
        b->wi[i].resize(m);
        if (cudaMemcpy(b->wi[i].data(), in.dWi, sizeof(double) * m, cudaMemcpyDeviceToHost) !=
            cudaSuccess) {
            destroy(b);
            return HSEIN_ECUDA;
        }
        int mc = 0;
        for (double v : b->wi[i]) mc += v != 0.0;
        if (mc != in.m_cplx) {
            destroy(b);
            return HSEIN_ESHIFTS;
        }
    }
    // the largest workspace over every configuration the autotuner may pick
    size_t most = 0;
    for (int pol : kPolicies)
        for (int blk : kBlocks) {
            hsein_batch_config cc = c;
            cc.br_policy = pol;
            cc.shift_block = blk;
            size_t w = 0;
            const hsein_status rc = config_bytes(b, cc, &w);
            if (rc != HSEIN_OK) {
                destroy(b);
                return rc;
            }
            most = std::max(most, w);
        }
    size_t w = 0;
    hsein_status rc = config_bytes(b, c, &w);
    if (rc == HSEIN_OK) rc = apply_config(b, c);
    if (rc != HSEIN_OK) {
        destroy(b);
        return rc;
    }
    b->streams.resize(kMaxStreams, nullptr);
    b->joins.resize(kMaxStreams, nullptr);
    bool ok = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) == cudaSuccess &&
              cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking) == cudaSuccess;
    for (int k = 0; k < kMaxStreams && ok; ++k)
        ok = cudaStreamCreateWithFlags(&b->streams[k], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&b->joins[k], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        destroy(b);
        return HSEIN_ECUDA;
    }
    if (workspace_bytes) *workspace_bytes = std::max(most, w);
    *batch = b;
    return HSEIN_OK;
}

hsein_status hsein_batch_solve(hsein_batch_t b, void* dWork, size_t work_bytes, void* stream) {
    if (!b || !dWork || (reinterpret_cast<uintptr_t>(dWork) & 255)) return HSEIN_EARG;
    if (work_bytes < b->total) return HSEIN_ENOMEM;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaEventRecord(b->ev_in, s) != cudaSuccess ||
        cudaStreamWaitEvent(b->origin, b->ev_in, 0) != cudaSuccess) {
        cudaGetLastError();
        return HSEIN_ECUDA;
    }
    if (!b->exec || b->exec_work != dWork) {
        const hsein_status rc = capture(b, dWork, b->origin);
        if (rc != HSEIN_OK) return rc;
    }
    if (cudaGraphLaunch(b->exec, b->origin) != cudaSuccess ||
        cudaEventRecord(b->ev_out, b->origin) != cudaSuccess ||
        cudaStreamWaitEvent(s, b->ev_out, 0) != cudaSuccess) {
        cudaGetLastError();
        return HSEIN_ECUDA;
    }
    return HSEIN_OK;
}

hsein_status hsein_batch_autotune(hsein_batch_t b, void* dWork, size_t work_bytes, void* stream,
                                  hsein_batch_config* chosen, double* ms_out) {
    if (!b || !dWork) return HSEIN_EARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return HSEIN_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return HSEIN_ECUDA;
    }
    hsein_status rc = HSEIN_OK;
    // median of three timed replays after one untimed one
    auto time_config = [&](const hsein_batch_config& c, double* t) -> hsein_status {
        hsein_status r = apply_config(b, c);
        if (r == HSEIN_OK && work_bytes < b->total) r = HSEIN_ENOMEM;
        if (r == HSEIN_OK) r = hsein_batch_solve(b, dWork, work_bytes, stream);
        double v[3] = {0, 0, 0};
        for (int i = 0; i < 3 && r == HSEIN_OK; ++i) {
            float f = 0.f;
            if (cudaEventRecord(e0, s) != cudaSuccess ||
                hsein_batch_solve(b, dWork, work_bytes, stream) != HSEIN_OK ||
                cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&f, e0, e1) != cudaSuccess)
                r = HSEIN_ECUDA;
            v[i] = f;
        }
        std::sort(v, v + 3);
        *t = v[1];
        return r;
    };
    hsein_batch_config best = b->cfg;
    double tbest = 0.0;
    rc = time_config(best, &tbest);
    // coordinate search: tile-height policy, then shift blocks, then chains
    for (int dim = 0; dim < 3 && rc == HSEIN_OK; ++dim) {
        const int* vals = dim == 0 ? kPolicies : dim == 1 ? kBlocks : kStreams;
        const int nv = dim == 0 ? (int)(sizeof(kPolicies) / sizeof(int))
                     : dim == 1 ? (int)(sizeof(kBlocks) / sizeof(int))
                                : (int)(sizeof(kStreams) / sizeof(int));
        hsein_batch_config base = best;
        for (int i = 0; i < nv && rc == HSEIN_OK; ++i) {
            hsein_batch_config c = base;
            (dim == 0 ? c.br_policy : dim == 1 ? c.shift_block : c.streams) = vals[i];
            if (c.br_policy == best.br_policy && c.shift_block == best.shift_block &&
                c.streams == best.streams)
                continue;
            double t = 0.0;
            rc = time_config(c, &t);
            if (rc == HSEIN_OK && t < tbest) {
                tbest = t;
                best = c;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != HSEIN_OK) return rc;
    rc = apply_config(b, best);
    if (rc != HSEIN_OK) return rc;
    if (chosen) *chosen = best;
    if (ms_out) *ms_out = tbest;
    return HSEIN_OK;
}

hsein_status hsein_batch_info(hsein_batch_t b, hsein_batch_config* cfg, int* subproblems) {
    if (!b) return HSEIN_EARG;
    if (cfg) *cfg = b->cfg;
    if (subproblems) *subproblems = (int)b->tasks.size();
    return HSEIN_OK;
}

hsein_status hsein_batch_destroy(hsein_batch_t b) {
    if (!b) return HSEIN_EARG;
    destroy(b);
    return HSEIN_OK;
}

}  // extern "C"
