// lpb_serve.cu -- the serving loop of include/lpb_serve.h: one worker thread
// per attached matrix admits requests into the matrix's lanes between
// intervals (continuous batching), runs one interval on each of its lanes
// with work (on the matrix's own stream, so the matrices overlap on the
// device), collects finished LPs and moves stalled requests to the polish
// lane.  Every step of the method runs in the kernels; this file schedules.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>

#include "lpb_engine.h"
#include "lpb_serve.h"

using namespace lpb;

namespace {

using Clock = std::chrono::steady_clock;

enum ReqState { kPending = 0, kRunning = 1, kDone = 2, kFailed = 3 };

struct Request {
    int64_t id = 0;
    int matrix = 0;
    int count = 0;
    double tol = 0.0;
    int64_t max_iter = 0;
    std::vector<lpb_lp_spec> specs;
    std::vector<double> warm_x, warm_y;
    int64_t warm_request = -1;
    int warm_lp = 0;
    // device
    lpb_lp_spec* specs_dev = nullptr;
    double* x_dev = nullptr;
    double* y_dev = nullptr;
    double* wx_dev = nullptr;
    double* wy_dev = nullptr;
    std::vector<lpb_lp_result> res;
    GroupRun g;
    int lane = 0;  // 0: FP32 lane, 1: polish lane
    int state = kPending;
    bool polished = false;
    double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
    int64_t footprint = 0;
    bool charged = false;  // footprint counted against the budget
    bool released = false;
};

struct Matrix {
    lpb_ctx* h = nullptr;
    Lane lane32, lanep;
    std::vector<GroupRun*> g32, gp;
    std::deque<Request*> pending;
    std::vector<Request*> running;
    int polish_prec = kPrecDfl;
    bool in_flight = false;  // an interval is queued on the handle's stream
};

}  // namespace

struct lpb_server {
    lpb_server_options opt{};
    int device = 0;
    Clock::time_point t0;
    std::vector<std::thread> workers;  // one per attached matrix
    int in_flight = 0;                  // matrices with device work queued
    Clock::time_point busy_since;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    lpb_err fatal_code = LPB_OK;
    std::string fatal_msg;
    std::vector<std::unique_ptr<Matrix>> mats;
    std::map<int64_t, std::unique_ptr<Request>> reqs;
    // released result buffers, freed by the worker between intervals: only
    // the worker enqueues work on the matrices' streams, which it captures
    // into CUDA graphs (an enqueue from another thread would join a capture)
    std::vector<std::pair<int, void*>> to_free;
    int64_t next_id = 0;
    int64_t budget = 0, used = 0;
    lpb_server_stats st{};
    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

int64_t lane_bytes(const lpb_ctx* h, int cols, int prec) {
    const int64_t ts = prec == kPrecF32 ? 4 : 8;
    const int64_t mr = h->m > 0 ? h->m : 1;
    return (int64_t)cols * (5 * (int64_t)h->n + 5 * mr) * ts + (int64_t)cols * 256;
}

int64_t request_bytes(const lpb_ctx* h, const Request& r) {
    int64_t b = (int64_t)r.count * ((int64_t)h->n + h->m) * 8 + (int64_t)r.count * (int64_t)sizeof(lpb_lp_spec);
    if (!r.warm_x.empty()) b += (int64_t)r.warm_x.size() * 8;
    if (!r.warm_y.empty()) b += (int64_t)r.warm_y.size() * 8;
    return b;
}

// Request buffers are stream-ordered allocations on the matrix's stream:
// cudaMalloc / cudaFree would synchronize the whole device and stall the
// other matrices' intervals.
void free_request_dev(Request& r, cudaStream_t s) {
    if (r.specs_dev) cudaFreeAsync(r.specs_dev, s);
    if (r.wx_dev) cudaFreeAsync(r.wx_dev, s);
    if (r.wy_dev) cudaFreeAsync(r.wy_dev, s);
    r.specs_dev = nullptr;
    r.wx_dev = r.wy_dev = nullptr;
}

void free_request_results(Request& r, cudaStream_t s) {
    if (r.x_dev) cudaFreeAsync(r.x_dev, s);
    if (r.y_dev) cudaFreeAsync(r.y_dev, s);
    r.x_dev = r.y_dev = nullptr;
}

// Device buffers and admission of request r into its matrix's FP32 lane.
lpb_err admit(Matrix& M, Request& r, int gid, int slot0, const double* warm_src_x,
              const double* warm_src_y) {
    lpb_ctx* h = M.h;
    cudaStream_t s = h->stream;
    const int n = h->n, m = h->m;
    LPB_CU(cudaMallocAsync((void**)&r.specs_dev, sizeof(lpb_lp_spec) * r.count, s));
    LPB_CU(cudaMemcpyAsync(r.specs_dev, r.specs.data(), sizeof(lpb_lp_spec) * r.count, cudaMemcpyHostToDevice, s));
    LPB_CU(cudaMallocAsync((void**)&r.x_dev, sizeof(double) * (size_t)n * r.count, s));
    LPB_CU(cudaMallocAsync((void**)&r.y_dev, sizeof(double) * (size_t)(m > 0 ? m : 1) * r.count, s));
    LPB_CU(cudaMemsetAsync(r.x_dev, 0, sizeof(double) * (size_t)n * r.count, s));
    LPB_CU(cudaMemsetAsync(r.y_dev, 0, sizeof(double) * (size_t)(m > 0 ? m : 1) * r.count, s));
    const double *wx = nullptr, *wy = nullptr;
    int64_t wsx = n, wsy = m;
    if (!r.warm_x.empty()) {
        LPB_CU(cudaMallocAsync((void**)&r.wx_dev, sizeof(double) * r.warm_x.size(), s));
        LPB_CU(cudaMemcpyAsync(r.wx_dev, r.warm_x.data(), sizeof(double) * r.warm_x.size(), cudaMemcpyHostToDevice, s));
        wx = r.wx_dev;
    }
    if (!r.warm_y.empty() && m > 0) {
        LPB_CU(cudaMallocAsync((void**)&r.wy_dev, sizeof(double) * r.warm_y.size(), s));
        LPB_CU(cudaMemcpyAsync(r.wy_dev, r.warm_y.data(), sizeof(double) * r.warm_y.size(), cudaMemcpyHostToDevice, s));
        wy = r.wy_dev;
    }
    if (warm_src_x) {
        // the parent's iterate, kept on the device, for every LP
        wx = warm_src_x;
        wy = m > 0 ? warm_src_y : nullptr;
        wsx = 0;
        wsy = 0;
    }
    r.res.assign(r.count, lpb_lp_result{});
    r.g = GroupRun{};
    r.g.id = gid;
    r.g.count = r.count;
    r.g.slot0 = slot0;
    r.g.max_iter = r.max_iter;
    r.g.res = r.res.data();
    r.g.x_dev = r.x_dev;
    r.g.y_dev = r.y_dev;
    r.lane = 0;
    return lane_admit<float>(h, M.lane32, r.g, r.specs_dev, wx, wy, wsx, wsy, r.tol, s, M.g32);
}

template <typename TP>
lpb_err run_polish_interval(Matrix& M, lpb_profile* prof) {
    return lane_interval<TP>(M.h, M.lanep, M.h->opt.check_every, 0, M.h->stream, prof);
}
template <typename TP>
lpb_err collect_polish(Matrix& M, lpb_profile* prof) {
    return lane_collect<TP>(M.h, M.lanep, M.gp, M.h->stream, prof);
}

// Admissions into matrix M's FP32 lane (FIFO; a request waits for its warm
// source, for free columns, a group id, residual slots and budget).
lpb_err admit_pending(lpb_server* srv, Matrix& M, bool& did_work) {
    for (;;) {
        Request* r = nullptr;
        const double *wsx = nullptr, *wsy = nullptr;
        int gid = -1, slot0 = -1;
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            if (M.pending.empty()) return LPB_OK;
            r = M.pending.front();
            if (r->warm_request >= 0) {
                auto it = srv->reqs.find(r->warm_request);
                if (it == srv->reqs.end() || it->second->released || it->second->state == kFailed) {
                    r->state = kFailed;
                    M.pending.pop_front();
                    srv->cv_done.notify_all();
                    continue;
                }
                if (it->second->state != kDone) return LPB_OK;
                const Request& w = *it->second;
                wsx = w.x_dev + (size_t)r->warm_lp * M.h->n;
                wsy = M.h->m > 0 ? w.y_dev + (size_t)r->warm_lp * M.h->m : nullptr;
            }
            if (M.lane32.cap - M.lane32.ncol < r->count) return LPB_OK;
            gid = lane_free_group(M.lane32, M.g32);
            slot0 = lane_find_slots(M.lane32, r->count);
            if (gid < 0 || slot0 < 0) return LPB_OK;
            if (srv->used + r->footprint > srv->budget) return LPB_OK;
            srv->used += r->footprint;
            r->charged = true;
            M.pending.pop_front();
        }
        const bool busy = M.lane32.ncol > 0 || M.lanep.ncol > 0;
        lpb_err rc = admit(M, *r, gid, slot0, wsx, wsy);
        std::lock_guard<std::mutex> lk(srv->mu);
        if (rc != LPB_OK) {
            r->state = kFailed;
            free_request_dev(*r, M.h->stream);
            free_request_results(*r, M.h->stream);
            srv->used -= r->footprint;
            r->charged = false;
            srv->cv_done.notify_all();
            // a bad record fails its request only; anything else stops the server
            if (rc == LPB_ERR_INVALID_ARG || rc == LPB_ERR_BAD_INDEX) continue;
            return rc;
        }
        r->t_admit = srv->now();
        r->state = kRunning;
        if (busy) srv->st.admitted_while_busy += 1;
        did_work = true;
        if (r->g.live == 0) {
            r->state = kDone;
            r->t_done = r->t_admit;
            free_request_dev(*r, M.h->stream);
            srv->st.done += 1;
            srv->cv_done.notify_all();
        } else {
            M.running.push_back(r);
        }
    }
}

// Launches one interval on each of M's lanes with work (async on M's stream).
lpb_err launch(Matrix& M, lpb_server_stats& add, lpb_profile& prof) {
    const int ce = M.h->opt.check_every;
    if (M.lane32.ncol > 0) {
        add.column_iters += (int64_t)M.lane32.ncol * ce;
        lpb_err rc = lane_interval<float>(M.h, M.lane32, ce, M.lanep.cap > 0 ? M.h->opt.polish_stall_checks : 0,
                                          M.h->stream, &prof);
        if (rc != LPB_OK) return rc;
        add.intervals += 1;
        M.in_flight = true;
    }
    if (M.lanep.ncol > 0) {
        add.column_iters += (int64_t)M.lanep.ncol * ce;
        lpb_err rc = M.polish_prec == kPrecDfl ? run_polish_interval<dfloat>(M, &prof)
                                               : run_polish_interval<double>(M, &prof);
        if (rc != LPB_OK) return rc;
        add.intervals += 1;
        M.in_flight = true;
    }
    return LPB_OK;
}

// M's interval has completed: statuses, extraction, compaction, moves of
// stalled requests to the polish lane, finished requests.
lpb_err finish(lpb_server* srv, Matrix& M, lpb_server_stats& add, lpb_profile& prof) {
    M.in_flight = false;
    lpb_err rc;
    if (M.lane32.ncol > 0 && (rc = lane_collect<float>(M.h, M.lane32, M.g32, M.h->stream, &prof)) != LPB_OK)
        return rc;
    if (M.lanep.ncol > 0) {
        rc = M.polish_prec == kPrecDfl ? collect_polish<dfloat>(M, &prof) : collect_polish<double>(M, &prof);
        if (rc != LPB_OK) return rc;
    }
    bool moved = false;
    for (Request* r : M.running) {
        if (r->lane != 0 || r->g.live == 0 || !r->g.stalled || M.lanep.cap == 0) continue;
        if (M.lanep.cap - M.lanep.ncol < r->g.live) continue;
        const int gid = lane_free_group(M.lanep, M.gp);
        const int slot0 = lane_find_slots(M.lanep, r->count);
        if (gid < 0 || slot0 < 0) continue;
        rc = M.polish_prec == kPrecDfl
                 ? lane_migrate<dfloat>(M.h, M.lane32, M.lanep, r->g, gid, slot0, M.h->stream, M.g32)
                 : lane_migrate<double>(M.h, M.lane32, M.lanep, r->g, gid, slot0, M.h->stream, M.g32);
        if (rc != LPB_OK) return rc;
        if ((int)M.gp.size() <= gid) M.gp.resize(gid + 1, nullptr);
        M.gp[gid] = &r->g;
        r->lane = 1;
        moved = true;
        std::lock_guard<std::mutex> lk(srv->mu);
        r->polished = true;
        add.migrations += 1;
    }
    // the extraction copies of finished requests complete before they are reported
    bool any_done = false;
    for (Request* r : M.running) any_done |= r->g.live == 0;
    if (any_done || moved) LPB_CU(cudaStreamSynchronize(M.h->stream));
    if (!any_done) return LPB_OK;
    std::lock_guard<std::mutex> lk(srv->mu);
    std::vector<Request*> still;
    for (Request* r : M.running) {
        if (r->g.live > 0) {
            still.push_back(r);
            continue;
        }
        r->state = kDone;
        r->t_done = srv->now();
        free_request_dev(*r, M.h->stream);
        srv->st.done += 1;
        for (const auto& x : r->res)
            if (x.status == LPB_OPTIMAL || x.status == LPB_PRIMAL_INFEASIBLE || x.status == LPB_DUAL_INFEASIBLE)
                srv->st.lps_solved += 1;
    }
    M.running.swap(still);
    srv->cv_done.notify_all();
    return LPB_OK;
}

// device-busy time: some matrix has an interval in flight
void mark_in_flight(lpb_server* srv, int delta) {
    std::lock_guard<std::mutex> lk(srv->mu);
    const int before = srv->in_flight;
    srv->in_flight += delta;
    if (before == 0 && srv->in_flight > 0) srv->busy_since = Clock::now();
    if (before > 0 && srv->in_flight == 0)
        srv->st.busy_s += std::chrono::duration<double>(Clock::now() - srv->busy_since).count();
}

// One pass of matrix M's worker: once its interval has completed it is
// collected, takes in admissions and launches its next interval at once.
lpb_err step_matrix(lpb_server* srv, Matrix& M, int mi, bool& did_work) {
    did_work = false;
    std::vector<void*> frees;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        std::vector<std::pair<int, void*>> keep;
        for (const auto& f : srv->to_free) {
            if (f.first == mi) frees.push_back(f.second);
            else keep.push_back(f);
        }
        srv->to_free.swap(keep);
    }
    for (void* p : frees) LPB_CU(cudaFreeAsync(p, M.h->stream));
    lpb_server_stats add{};
    lpb_profile prof{};
    lpb_err rc;
    if (M.in_flight) {
        const cudaError_t q = cudaStreamQuery(M.h->stream);
        if (q == cudaErrorNotReady) return LPB_OK;
        if (q != cudaSuccess) return cuda_fail(q, "cudaStreamQuery");
        mark_in_flight(srv, -1);
        if ((rc = finish(srv, M, add, prof)) != LPB_OK) return rc;
        did_work = true;
    }
    if ((rc = admit_pending(srv, M, did_work)) != LPB_OK) return rc;
    if ((rc = launch(M, add, prof)) != LPB_OK) return rc;
    if (M.in_flight) {
        mark_in_flight(srv, +1);
        did_work = true;
    }
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->st.intervals += add.intervals;
    srv->st.column_iters += add.column_iters;
    srv->st.migrations += add.migrations;
    srv->st.kernels += prof.kernels;
    return LPB_OK;
}

// The worker of one attached matrix.  Matrices advance independently: each
// has its own thread, stream and lanes, so a small matrix's short intervals
// are not held back by the host work (collection, admission, launches) of
// the others.
void worker_main(lpb_server* srv, Matrix* M, int mi) {
    cudaSetDevice(srv->device);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            if (srv->stop || srv->fatal_code != LPB_OK) return;
        }
        bool did = false;
        lpb_err rc = step_matrix(srv, *M, mi, did);
        if (rc != LPB_OK) {
            std::lock_guard<std::mutex> lk(srv->mu);
            if (srv->fatal_code == LPB_OK) {
                srv->fatal_code = rc;
                srv->fatal_msg = lpb_last_error();
            }
            for (auto& kv : srv->reqs)
                if (kv.second->state == kPending || kv.second->state == kRunning) kv.second->state = kFailed;
            srv->cv_done.notify_all();
            srv->cv_work.notify_all();
            return;
        }
        if (M->in_flight) {
            // device work outstanding: poll again shortly
            if (!did) std::this_thread::sleep_for(std::chrono::microseconds(20));
        } else if (!did) {
            std::unique_lock<std::mutex> lk(srv->mu);
            if (srv->stop) return;
            srv->cv_work.wait_for(lk, std::chrono::milliseconds(2));
        }
    }
}

}  // namespace

extern "C" {

void lpb_server_default_options(lpb_server_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->hbm_budget_bytes = 0;
    o->lane_columns = 256;
    o->polish_columns = 64;
    o->max_groups = 64;
    o->device = -1;
}

lpb_err lpb_server_create(const lpb_server_options* opt, lpb_server_t* out) {
    if (!out) return fail(LPB_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    lpb_server_options o;
    lpb_server_default_options(&o);
    if (opt) o = *opt;
    if (o.lane_columns < 1 || o.polish_columns < 0 || o.max_groups < 1 || o.hbm_budget_bytes < 0)
        return fail(LPB_ERR_INVALID_ARG, "bad server option");
    int dev = o.device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return fail(LPB_ERR_CUDA, "no CUDA device");
    if (cudaSetDevice(dev) != cudaSuccess) return fail(LPB_ERR_CUDA, "cannot use the CUDA device");
    lpb_server* srv = new (std::nothrow) lpb_server();
    if (!srv) return fail(LPB_ERR_OOM, "host allocation failed");
    srv->opt = o;
    srv->device = dev;
    srv->t0 = Clock::now();
    int64_t budget = o.hbm_budget_bytes;
    if (budget == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            delete srv;
            return fail(LPB_ERR_CUDA, "cudaMemGetInfo failed");
        }
        budget = (int64_t)(0.8 * (double)fr);
    }
    srv->budget = budget;
    srv->st.hbm_budget_bytes = budget;
    *out = srv;
    return LPB_OK;
}

lpb_err lpb_server_attach(lpb_server_t srv, lpb_handle h, int32_t* matrix_id) {
    if (!srv || !h || !matrix_id) return fail(LPB_ERR_INVALID_ARG, "null argument");
    if (h->device != srv->device) return fail(LPB_ERR_INVALID_ARG, "handle is on another device");
    if (h->opt.precision != LPB_MIXED) return fail(LPB_ERR_INVALID_ARG, "serving runs FP32 iterates (LPB_MIXED)");
    std::unique_ptr<Matrix> M(new (std::nothrow) Matrix());
    if (!M) return fail(LPB_ERR_OOM, "host allocation failed");
    M->h = h;
    M->polish_prec = polish_dfloat(h) ? kPrecDfl : kPrecF64;
    const int pcols = polish_enabled(h) ? srv->opt.polish_columns : 0;
    const int64_t need = lane_bytes(h, srv->opt.lane_columns, kPrecF32) +
                         (pcols > 0 ? lane_bytes(h, pcols, M->polish_prec) : 0);
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (srv->fatal_code != LPB_OK) return fail(srv->fatal_code, "server stopped: " + srv->fatal_msg);
        if (srv->used + need > srv->budget) return fail(LPB_ERR_OOM, "the lanes exceed the server's HBM budget");
        srv->used += need;
    }
    lpb_err rc = lane_reserve(h, M->lane32, kPrecF32, srv->opt.lane_columns, srv->opt.max_groups);
    if (rc == LPB_OK && pcols > 0) rc = lane_reserve(h, M->lanep, M->polish_prec, pcols, srv->opt.max_groups);
    if (rc == LPB_OK) rc = ensure_check_ws(h, std::max(M->lane32.cap, M->lanep.cap));
    if (rc == LPB_OK) {
        // the server launches intervals plainly: its lanes change shape at
        // almost every interval (admissions, completions, moves), so a
        // captured graph would rarely be replayed; per-interval event timing
        // is not collected
        h->opt.profile = 0;
        h->opt.use_graphs = 0;
        h->opt.use_pdl = 0;
    }
    std::lock_guard<std::mutex> lk(srv->mu);
    if (rc != LPB_OK) {
        srv->used -= need;
        lane_free(M->lane32);
        lane_free(M->lanep);
        return rc;
    }
    *matrix_id = (int32_t)srv->mats.size();
    Matrix* mp = M.get();
    srv->mats.push_back(std::move(M));
    srv->st.hbm_used_bytes = srv->used;
    srv->workers.emplace_back(worker_main, srv, mp, (int)*matrix_id);
    return LPB_OK;
}

lpb_err lpb_server_submit(lpb_server_t srv, const lpb_request* q, int64_t* request_id) {
    if (!srv || !q || !request_id) return fail(LPB_ERR_INVALID_ARG, "null argument");
    std::unique_ptr<Request> r(new (std::nothrow) Request());
    if (!r) return fail(LPB_ERR_OOM, "host allocation failed");
    lpb_ctx* h = nullptr;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (q->matrix_id < 0 || q->matrix_id >= (int)srv->mats.size()) return fail(LPB_ERR_INVALID_ARG, "bad matrix_id");
        h = srv->mats[q->matrix_id]->h;
    }
    if (q->num_lps < 1 || q->num_lps > srv->opt.lane_columns || !q->specs)
        return fail(LPB_ERR_INVALID_ARG, "num_lps must be in [1, lane_columns] with specs");
    if (!(q->tol > 0.0) || !std::isfinite(q->tol)) return fail(LPB_ERR_INVALID_ARG, "tol must be positive and finite");
    if (q->max_iter < 1) return fail(LPB_ERR_INVALID_ARG, "max_iter must be >= 1");
    for (int32_t k = 0; k < q->num_lps; ++k) {
        const lpb_lp_spec& sp = q->specs[k];
        if (sp.kind < 0 || sp.kind > 2) return fail(LPB_ERR_INVALID_ARG, "override kind must be 0, 1 or 2");
        if (sp.kind != 0 && (sp.var < 0 || sp.var >= h->n))
            return fail(LPB_ERR_BAD_INDEX, "an override names a variable outside [0, n)");
        if (sp.kind == 1 && (std::isnan(sp.lo) || std::isnan(sp.hi)))
            return fail(LPB_ERR_INVALID_ARG, "NaN override bound");
        if (sp.kind == 2 && !std::isfinite(sp.sign)) return fail(LPB_ERR_INVALID_ARG, "non-finite objective sign");
    }
    const int ce = h->opt.check_every;
    r->matrix = q->matrix_id;
    r->count = q->num_lps;
    r->tol = q->tol;
    r->max_iter = (q->max_iter + ce - 1) / ce * ce;
    r->specs.assign(q->specs, q->specs + q->num_lps);
    if (q->warm_x) r->warm_x.assign(q->warm_x, q->warm_x + (size_t)h->n * q->num_lps);
    if (q->warm_y && h->m > 0) r->warm_y.assign(q->warm_y, q->warm_y + (size_t)h->m * q->num_lps);
    r->warm_request = q->warm_request;
    r->warm_lp = q->warm_lp;
    r->footprint = request_bytes(h, *r);
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->fatal_code != LPB_OK) return fail(srv->fatal_code, "server stopped: " + srv->fatal_msg);
    if (r->warm_request >= 0) {
        auto it = srv->reqs.find(r->warm_request);
        if (it == srv->reqs.end() || it->second->released)
            return fail(LPB_ERR_INVALID_ARG, "warm_request is unknown or released");
        if (it->second->matrix != r->matrix) return fail(LPB_ERR_INVALID_ARG, "warm_request is on another matrix");
        if (r->warm_lp < 0 || r->warm_lp >= it->second->count) return fail(LPB_ERR_INVALID_ARG, "bad warm_lp");
    }
    if (r->footprint > srv->budget) return fail(LPB_ERR_OOM, "the request alone exceeds the HBM budget");
    r->id = srv->next_id++;
    r->t_submit = srv->now();
    *request_id = r->id;
    srv->mats[r->matrix]->pending.push_back(r.get());
    srv->reqs[r->id] = std::move(r);
    srv->st.submitted += 1;
    srv->cv_work.notify_all();
    return LPB_OK;
}

lpb_err lpb_server_poll(lpb_server_t srv, int64_t id, int32_t* done) {
    if (!srv || !done) return fail(LPB_ERR_INVALID_ARG, "null argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(id);
    if (it == srv->reqs.end()) return fail(LPB_ERR_INVALID_ARG, "unknown request");
    *done = it->second->state >= kDone ? 1 : 0;
    return LPB_OK;
}

lpb_err lpb_server_wait(lpb_server_t srv, int64_t id, double timeout_s) {
    if (!srv) return fail(LPB_ERR_INVALID_ARG, "null server");
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(id);
    if (it == srv->reqs.end()) return fail(LPB_ERR_INVALID_ARG, "unknown request");
    Request* r = it->second.get();
    auto pred = [&] { return r->state >= kDone; };
    if (timeout_s < 0) {
        srv->cv_done.wait(lk, pred);
    } else if (!srv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred)) {
        return fail(LPB_ERR_TIMEOUT, "request not finished within the timeout");
    }
    if (r->state == kFailed)
        return fail(srv->fatal_code != LPB_OK ? srv->fatal_code : LPB_ERR_INVALID_ARG,
                    srv->fatal_code != LPB_OK ? "server stopped: " + srv->fatal_msg
                                              : std::string("request failed (its warm start was released or failed)"));
    return LPB_OK;
}

lpb_err lpb_server_result(lpb_server_t srv, int64_t id, int32_t lp, lpb_lp_result* res, double* x, double* y) {
    if (!srv) return fail(LPB_ERR_INVALID_ARG, "null server");
    Request* r = nullptr;
    int n = 0, m = 0;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        auto it = srv->reqs.find(id);
        if (it == srv->reqs.end()) return fail(LPB_ERR_INVALID_ARG, "unknown request");
        r = it->second.get();
        if (r->state != kDone) return fail(LPB_ERR_INVALID_ARG, "request not done");
        if (r->released) return fail(LPB_ERR_INVALID_ARG, "request released");
        if (lp < 0 || lp >= r->count) return fail(LPB_ERR_INVALID_ARG, "lp index out of range");
        n = srv->mats[r->matrix]->h->n;
        m = srv->mats[r->matrix]->h->m;
    }
    if (res) *res = r->res[lp];
    cudaSetDevice(srv->device);
    if (x) LPB_CU(cudaMemcpy(x, r->x_dev + (size_t)lp * n, sizeof(double) * n, cudaMemcpyDeviceToHost));
    if (y && m > 0) LPB_CU(cudaMemcpy(y, r->y_dev + (size_t)lp * m, sizeof(double) * m, cudaMemcpyDeviceToHost));
    return LPB_OK;
}

lpb_err lpb_server_results(lpb_server_t srv, int64_t id, lpb_lp_result* res) {
    if (!srv || !res) return fail(LPB_ERR_INVALID_ARG, "null argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(id);
    if (it == srv->reqs.end()) return fail(LPB_ERR_INVALID_ARG, "unknown request");
    if (it->second->state != kDone) return fail(LPB_ERR_INVALID_ARG, "request not done");
    std::memcpy(res, it->second->res.data(), sizeof(lpb_lp_result) * it->second->count);
    return LPB_OK;
}

lpb_err lpb_server_request_info(lpb_server_t srv, int64_t id, lpb_request_info* info) {
    if (!srv || !info) return fail(LPB_ERR_INVALID_ARG, "null argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(id);
    if (it == srv->reqs.end()) return fail(LPB_ERR_INVALID_ARG, "unknown request");
    const Request& r = *it->second;
    std::memset(info, 0, sizeof(*info));
    info->state = r.state;
    info->num_lps = r.count;
    info->t_submit = r.t_submit;
    info->t_admit = r.t_admit;
    info->t_done = r.t_done;
    info->footprint_bytes = r.footprint;
    info->polished = r.polished ? 1 : 0;
    if (r.state == kDone) {
        for (const auto& x : r.res) {
            info->iters = std::max<int64_t>(info->iters, x.iters);
            if (x.status == LPB_OPTIMAL) info->optimal += 1;
            else if (x.status == LPB_PRIMAL_INFEASIBLE || x.status == LPB_DUAL_INFEASIBLE) info->infeasible += 1;
            else if (x.status == LPB_ITERATION_LIMIT) info->iteration_limit += 1;
            else info->other += 1;
        }
    }
    return LPB_OK;
}

lpb_err lpb_server_release(lpb_server_t srv, int64_t id) {
    if (!srv) return fail(LPB_ERR_INVALID_ARG, "null server");
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(id);
    if (it == srv->reqs.end()) return fail(LPB_ERR_INVALID_ARG, "unknown request");
    Request& r = *it->second;
    if (r.state < kDone) return fail(LPB_ERR_INVALID_ARG, "request still pending or running");
    if (r.released) return LPB_OK;
    // a pending request that warm-starts from this one keeps it alive
    for (auto& mp : srv->mats)
        for (const Request* p : mp->pending)
            if (p->warm_request == id) return fail(LPB_ERR_INVALID_ARG, "a pending request warm-starts from it");
    if (r.x_dev) srv->to_free.emplace_back(r.matrix, r.x_dev);
    if (r.y_dev) srv->to_free.emplace_back(r.matrix, r.y_dev);
    r.x_dev = r.y_dev = nullptr;
    r.released = true;
    srv->cv_work.notify_all();
    if (r.charged) srv->used -= r.footprint;
    r.charged = false;
    srv->st.hbm_used_bytes = srv->used;
    return LPB_OK;
}

lpb_err lpb_server_stats_get(lpb_server_t srv, lpb_server_stats* st) {
    if (!srv || !st) return fail(LPB_ERR_INVALID_ARG, "null argument");
    std::lock_guard<std::mutex> lk(srv->mu);
    *st = srv->st;
    st->hbm_used_bytes = srv->used;
    st->hbm_budget_bytes = srv->budget;
    return LPB_OK;
}

void lpb_server_destroy(lpb_server_t srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
        srv->cv_work.notify_all();
    }
    for (auto& w : srv->workers)
        if (w.joinable()) w.join();
    cudaSetDevice(srv->device);
    for (auto& mp : srv->mats) {
        if (mp->h && mp->h->stream) cudaStreamSynchronize(mp->h->stream);
        lane_free(mp->lane32);
        lane_free(mp->lanep);
    }
    for (auto& kv : srv->reqs) {
        cudaStream_t s = srv->mats[kv.second->matrix]->h->stream;
        free_request_dev(*kv.second, s);
        free_request_results(*kv.second, s);
        cudaStreamSynchronize(s);
    }
    for (const auto& f : srv->to_free) {
        cudaStream_t s = srv->mats[f.first]->h->stream;
        cudaFreeAsync(f.second, s);
        cudaStreamSynchronize(s);
    }
    delete srv;
}

}  // extern "C"
