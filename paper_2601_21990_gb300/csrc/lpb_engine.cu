// lpb_engine.cu -- lanes, restart groups and the interval loop on the host
// side.  Every step of the method runs in the kernels of lpb_iter.cu and
// lpb_check.cu; this file allocates, launches, and moves O(columns + groups)
// records between checks (Sec. 5: the batch stays on the device, only
// per-LP flags cross to the host).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>

#include "lpb_engine.h"

namespace lpb {

namespace {

size_t rup(size_t v, size_t a) { return (v + a - 1) / a * a; }

template <typename P>
cudaError_t dmalloc(std::vector<void*>& list, P** out, size_t bytes) {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes ? bytes : 1);
    if (e == cudaSuccess) list.push_back(p);
    *out = (P*)p;
    return e;
}

template <typename T> constexpr int prec_of() {
    return std::is_same<T, float>::value ? kPrecF32 : std::is_same<T, double>::value ? kPrecF64 : kPrecDfl;
}

template <typename T> const T* pick(const double* d64, const float* d32, const dfloat* ddf);
template <> const double* pick<double>(const double* d64, const float*, const dfloat*) { return d64; }
template <> const float* pick<float>(const double*, const float* d32, const dfloat*) { return d32; }
template <> const dfloat* pick<dfloat>(const double*, const float*, const dfloat* ddf) { return ddf; }

template <typename T>
IterData<T> iter_data(const lpb_ctx* h, const Lane& ln) {
    IterData<T> d{};
    d.A = h->A;
    d.At = h->At;
    d.a_vals = pick<T>(h->A.v64, h->A.v32, h->a_dfl);
    d.at_vals = pick<T>(h->At.v64, h->At.v32, h->at_dfl);
    d.c = pick<T>(h->cs, h->cs32, h->cs_dfl);
    d.xl = pick<T>(h->xls, h->xls32, h->xls_dfl);
    d.xu = pick<T>(h->xus, h->xus32, h->xus_dfl);
    d.l = pick<T>(h->ls, h->ls32, h->ls_dfl);
    d.u = pick<T>(h->us, h->us32, h->us_dfl);
    d.col.kind = ln.ckind;
    d.col.var = ln.cvar;
    d.col.grp = ln.cgrp;
    d.col.lo = (T*)ln.clo;
    d.col.hi = (T*)ln.chi;
    d.col.c = (T*)ln.cc;
    d.col.tau = (T*)ln.ctau;
    d.col.sigma = (T*)ln.csigma;
    return d;
}

template <typename T>
IterBufs<T> iter_bufs(const Lane& ln) {
    IterBufs<T> b{};
    b.X = (T*)ln.X;
    b.X0 = (T*)ln.X0;
    b.Xbar = (T*)ln.Xbar;
    b.Y = (T*)ln.Y;
    b.Y0 = (T*)ln.Y0;
    b.Xh = (T*)ln.Xh;
    b.DX = (T*)ln.DX;
    b.G = nullptr;
    b.Yh = (T*)ln.Yh;
    b.DY = (T*)ln.DY;
    b.DYp = (T*)ln.DYp;
    return b;
}

void set_result(lpb_lp_result& r, const ColRecord& rc, int status, int64_t iters, int64_t restarts) {
    r.status = status;
    r.restarts = (int32_t)restarts;
    r.iters = iters;
    r.obj = rc.obj;
    r.dual_obj = rc.dual_obj;
    r.rel_primal = rc.rel_primal;
    r.rel_dual = rc.rel_dual;
    r.rel_gap = rc.rel_gap;
    r.safe_bound = rc.safe;
}

// Removes the columns `gone` (ascending) from the lane by moving live tail
// columns into their places; the moves run on the device.
// idle: the caller has synchronized s since it last queued copies from the
// lane's pinned move lists.
template <typename T>
lpb_err compact(lpb_ctx* h, Lane& ln, const std::vector<int>& gone, cudaStream_t s, lpb_profile* prof,
                bool idle = false) {
    if (gone.empty()) return LPB_OK;
    // the pinned move lists may still be read by copies queued earlier
    if (!idle) LPB_CU(cudaStreamSynchronize(s));
    const int ncol = ln.ncol;
    std::vector<char> is_gone(ncol, 0);
    for (int f : gone) is_gone[f] = 1;
    const int ncol2 = ncol - (int)gone.size();
    int* src = ln.mv_h;
    int* dst = ln.mv_h + ln.cap;
    int cnt = 0, tail = ncol - 1;
    for (int f : gone) {
        if (f >= ncol2) break;
        while (is_gone[tail]) --tail;
        src[cnt] = tail;
        dst[cnt] = f;
        ln.col_group[f] = ln.col_group[tail];
        ln.col_lp[f] = ln.col_lp[tail];
        ++cnt;
        --tail;
    }
    for (int j = ncol2; j < ncol; ++j) {
        ln.col_group[j] = -1;
        ln.col_lp[j] = -1;
    }
    ln.ncol = ncol2;
    if (cnt == 0) return LPB_OK;
    LPB_CU(cudaMemcpyAsync(ln.mv, src, sizeof(int) * cnt, cudaMemcpyHostToDevice, s));
    LPB_CU(cudaMemcpyAsync(ln.mv + ln.cap, dst, sizeof(int) * cnt, cudaMemcpyHostToDevice, s));
    const CheckData cd = lane_check_data(h, ln, 0);
    LPB_CU(launch_compact<T>(iter_bufs<T>(ln), h->n, h->m, ln.cap, ln.mv, ln.mv + ln.cap, cnt, iter_data<T>(h, ln).col,
                             cd.col, s));
    if (prof) {
        prof->compactions += 1;
        prof->kernels += 2;
    }
    return LPB_OK;
}

// a group whose LPs have all left the lane: its id and slots are free again
lpb_err retire_group(Lane& ln, GroupRun& g, cudaStream_t s) {
    for (int q = 0; q < g.count; ++q) ln.slot_used[g.slot0 + q] = 0;
    LPB_CU(cudaMemsetAsync(ln.ctl + g.id, 0, sizeof(Control), s));
    ln.ctl_h[g.id].active = 0;
    return LPB_OK;
}

}  // namespace

lpb_err fail(lpb_err code, const std::string& msg) {
    set_last_error(msg.c_str());
    return code;
}

lpb_err cuda_fail(cudaError_t e, const char* what) {
    return fail(e == cudaErrorMemoryAllocation ? LPB_ERR_OOM : LPB_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

bool polish_enabled(const lpb_ctx* h) { return h->opt.precision == LPB_MIXED && h->opt.fp64_polish; }
bool polish_dfloat(const lpb_ctx* h) { return polish_enabled(h) && h->opt.polish_arith == LPB_POLISH_DFLOAT; }

void lane_free(Lane& ln) {
    if (ln.exec) cudaGraphExecDestroy(ln.exec);
    ln.exec = nullptr;
    for (void* p : ln.allocs) cudaFree(p);
    ln.allocs.clear();
    if (ln.rec_h) cudaFreeHost(ln.rec_h);
    if (ln.ctl_h) cudaFreeHost(ln.ctl_h);
    if (ln.mv_h) cudaFreeHost(ln.mv_h);
    if (ln.optr_h) cudaFreeHost(ln.optr_h);
    const int prec = ln.prec;
    ln = Lane{};
    ln.prec = prec;
}

lpb_err lane_reserve(lpb_ctx* h, Lane& ln, int prec, int cap, int gcap) {
    cap = (int)rup((size_t)std::max(cap, 1), 4);
    gcap = std::max(gcap, 1);
    if (ln.cap >= cap && ln.gcap >= gcap && ln.prec == prec) return LPB_OK;
    if (ln.ncol > 0) return fail(LPB_ERR_INVALID_ARG, "a lane in use cannot be resized");
    lane_free(ln);
    ln.prec = prec;
    auto& L = ln.allocs;
    const size_t tsz = prec == kPrecF32 ? sizeof(float) : prec == kPrecF64 ? sizeof(double) : sizeof(dfloat);
    const size_t n = (size_t)h->n, mr = h->m > 0 ? (size_t)h->m : 1;
    const int ce = h->opt.check_every;
    const int nslot = 2 * cap;
    // the primal iterate itself is not stored (the steps rebuild it from Xbar
    // and X0); the checks of the literal restart reading need it
    void** xs[] = {&ln.X0, &ln.Xbar, &ln.Xh, &ln.DX};
    for (void** q : xs) LPB_CU(dmalloc(L, (char**)q, n * cap * tsz));
    if (!h->opt.restart_to_pdhg_output) LPB_CU(dmalloc(L, (char**)&ln.X, n * cap * tsz));
    void** ys[] = {&ln.Y, &ln.Y0, &ln.Yh, &ln.DY, &ln.DYp};
    for (void** q : ys) LPB_CU(dmalloc(L, (char**)q, mr * cap * tsz));
    void** cs[] = {&ln.clo, &ln.chi, &ln.cc, &ln.ctau, &ln.csigma};
    for (void** q : cs) LPB_CU(dmalloc(L, (char**)q, tsz * cap));
    int** is[] = {&ln.ckind, &ln.cvar, &ln.cgrp, &ln.cslot, &ln.k_stall};
    for (int** q : is) LPB_CU(dmalloc(L, q, sizeof(int) * cap));
    double** ds[] = {&ln.k_lo, &ln.k_hi, &ln.k_c, &ln.k_w, &ln.k_best};
    for (double** q : ds) LPB_CU(dmalloc(L, q, sizeof(double) * cap));
    LPB_CU(dmalloc(L, &ln.rec, sizeof(ColRecord) * cap));
    LPB_CU(dmalloc(L, &ln.ctl, sizeof(Control) * gcap));
    LPB_CU(cudaMemset(ln.ctl, 0, sizeof(Control) * gcap));
    LPB_CU(dmalloc(L, &ln.flags, sizeof(int) * 4));
    LPB_CU(cudaMemset(ln.flags, 0, sizeof(int) * 4));
    LPB_CU(dmalloc(L, &ln.hal64, sizeof(double) * 2 * (size_t)gcap * (ce + 1)));
    LPB_CU(dmalloc(L, &ln.hal32, sizeof(float) * 2 * (size_t)gcap * (ce + 1)));
    LPB_CU(dmalloc(L, &ln.haldf, sizeof(dfloat) * 2 * (size_t)gcap * (ce + 1)));
    LPB_CU(dmalloc(L, &ln.rscr, sizeof(double) * nslot));
    LPB_CU(dmalloc(L, &ln.rtag, sizeof(int) * nslot));
    LPB_CU(cudaMemset(ln.rtag, 0, sizeof(int) * nslot));
    LPB_CU(dmalloc(L, &ln.mv, sizeof(int) * 4 * cap));
    LPB_CU(dmalloc(L, &ln.optr, sizeof(double*) * 2 * cap));
    LPB_CU(cudaMallocHost((void**)&ln.rec_h, sizeof(ColRecord) * cap));
    LPB_CU(cudaMallocHost((void**)&ln.ctl_h, sizeof(Control) * gcap));
    std::memset(ln.ctl_h, 0, sizeof(Control) * gcap);
    LPB_CU(cudaMallocHost((void**)&ln.mv_h, sizeof(int) * 4 * cap));
    LPB_CU(cudaMallocHost((void**)&ln.optr_h, sizeof(double*) * 2 * cap));
    ln.cap = cap;
    ln.gcap = gcap;
    ln.ncol = 0;
    ln.col_group.assign(cap, -1);
    ln.col_lp.assign(cap, -1);
    ln.slot_used.assign(nslot, 0);
    return LPB_OK;
}

void free_long_scratch(lpb_ctx* h) {
    if (h->lr_part) cudaFree(h->lr_part);
    if (h->lr_ticket) cudaFree(h->lr_ticket);
    h->lr_part = nullptr;
    h->lr_ticket = nullptr;
    for (Csr* c : {&h->A, &h->At}) {
        c->part = nullptr;
        c->ticket = nullptr;
        c->ntix = 0;
    }
}

lpb_err ensure_long_scratch(lpb_ctx* h, int cap, bool force) {
    // partial sums: [segment][cap] of the widest iterate type (8 bytes);
    // tickets: one per (long row, column tile), at most cap / 2 + 1 tiles
    if (!force && cap <= h->lr_cap) return LPB_OK;
    LPB_CU(cudaStreamSynchronize(h->stream));
    free_long_scratch(h);
    h->lr_cap = 0;
    if (cap <= 0) return LPB_OK;
    const int ntix = cap / 2 + 1;
    const size_t segs = (size_t)h->A.n_lblocks + h->At.n_lblocks;
    const size_t rows = (size_t)h->A.n_long + h->At.n_long;
    if (segs > 0) {
        LPB_CU(cudaMalloc(&h->lr_part, segs * (size_t)cap * 8));
        LPB_CU(cudaMalloc((void**)&h->lr_ticket, rows * ntix * sizeof(unsigned)));
        LPB_CU(cudaMemsetAsync(h->lr_ticket, 0, rows * ntix * sizeof(unsigned), h->stream));
    }
    char* part = (char*)h->lr_part;
    unsigned* tick = h->lr_ticket;
    for (Csr* c : {&h->A, &h->At}) {
        c->ntix = ntix;
        c->part = c->n_lblocks > 0 ? part : nullptr;
        c->ticket = c->n_long > 0 ? tick : nullptr;
        part += (size_t)c->n_lblocks * cap * 8;
        tick += (size_t)c->n_long * ntix;
    }
    h->lr_cap = cap;
    h->ws_epoch += 1;  // captured intervals hold the old scratch pointers
    return LPB_OK;
}

lpb_err ensure_check_ws(lpb_ctx* h, int cap) {
    if (cap > h->lr_cap) {
        lpb_err rc = ensure_long_scratch(h, std::max(cap, h->ws_cap), false);
        if (rc != LPB_OK) return rc;
    }
    if (cap <= h->ws_cap) return LPB_OK;
    for (void* p : h->ws_allocs) cudaFree(p);
    h->ws_allocs.clear();
    h->ws_cap = 0;
    const size_t mr = h->m > 0 ? (size_t)h->m : 1;
    auto& L = h->ws_allocs;
    LPB_CU(dmalloc(L, &h->P, sizeof(double) * 2 * mr * cap));
    LPB_CU(dmalloc(L, &h->Q, sizeof(double) * 3 * (size_t)h->n * cap));
    LPB_CU(dmalloc(L, &h->partials, sizeof(double) * (size_t)kNumStats * kReduceBlocks * cap));
    LPB_CU(dmalloc(L, &h->colsum, sizeof(double) * (size_t)kNumStats * cap));
    h->ws_cap = cap;
    h->ws_epoch += 1;  // captured intervals hold the old workspace pointers
    return LPB_OK;
}

lpb_err ensure_specs(lpb_ctx* h, int count) {
    if (count <= h->specs_cap) return LPB_OK;
    if (h->specs_dev) cudaFree(h->specs_dev);
    h->specs_dev = nullptr;
    h->specs_cap = 0;
    const int cap = (int)rup((size_t)std::max(count, 1), 64);
    LPB_CU(cudaMalloc((void**)&h->specs_dev, sizeof(lpb_lp_spec) * cap));
    h->specs_cap = cap;
    return LPB_OK;
}

int lane_find_slots(const Lane& ln, int count) {
    const int ns = (int)ln.slot_used.size();
    int run = 0;
    for (int q = 0; q < ns; ++q) {
        run = ln.slot_used[q] ? 0 : run + 1;
        if (run >= count) return q - count + 1;
    }
    return count == 0 ? 0 : -1;
}

int lane_free_group(const Lane& ln, const std::vector<GroupRun*>& groups) {
    for (int g = 0; g < ln.gcap; ++g)
        if (g >= (int)groups.size() || groups[g] == nullptr) return g;
    return -1;
}

CheckData lane_check_data(const lpb_ctx* h, const Lane& ln, int stall_checks) {
    CheckData d{};
    d.A = h->A;
    d.At = h->At;
    d.m = h->m;
    d.n = h->n;
    d.d_r = h->d_r;
    d.d_c = h->d_c;
    d.c = h->c;
    d.xl = h->xl;
    d.xu = h->xu;
    d.l = h->l;
    d.u = h->u;
    d.col.kind = ln.ckind;
    d.col.var = ln.cvar;
    d.col.lo = ln.k_lo;
    d.col.hi = ln.k_hi;
    d.col.c = ln.k_c;
    d.col.w = ln.k_w;
    d.col.grp = ln.cgrp;
    d.col.slot = ln.cslot;
    d.col.best = ln.k_best;
    d.col.stall = ln.k_stall;
    d.eta = h->eta;
    d.beta_s = h->opt.beta_s;
    d.beta_n = h->opt.beta_n;
    d.beta_a = h->opt.beta_a;
    d.theta = h->opt.theta;
    d.mnorm_sign = h->opt.mnorm_sign;
    d.detect_inf = h->opt.detect_infeasibility;
    d.restart_to_output = h->opt.restart_to_pdhg_output;
    d.robust_rc = h->opt.reduced_cost == LPB_RC_ROBUST;
    d.stall_checks = stall_checks;
    d.check_every = h->opt.check_every;
    d.ctl = ln.ctl;
    d.gcap = ln.gcap;
    d.hal64 = ln.hal64;
    d.hal32 = ln.hal32;
    d.haldf = ln.haldf;
    d.rscr = ln.rscr;
    d.rtag = ln.rtag;
    d.flags = ln.flags;
    d.f_dr = h->f_dr;
    d.f_dc = h->f_dc;
    d.f_idr = h->f_idr;
    d.f_idc = h->f_idc;
    d.f_c = h->f_c;
    d.f_xl = h->f_xl;
    d.f_xu = h->f_xu;
    d.f_l = h->f_l;
    d.f_u = h->f_u;
    return d;
}

double step_bytes(int prec, int nnz, int m, int n, bool primal, bool check, int ncol) {
    const double ts = prec == kPrecF32 ? 4.0 : 8.0;
    const double rows = primal ? n : m, cols = primal ? m : n;
    double b = (4.0 + ts) * nnz + 4.0 * (rows + 1);
    // gathered block once, plus the row-side operands: primal reads Xbar, X0
    // and writes Xbar; dual reads Y, Y0 and writes Y; a check writes x^, dx
    // (primal) or y^, dy, Pi_B(dy) (dual)
    b += ts * ncol * (cols + rows * 3.0 + (check ? (primal ? 2.0 : 3.0) * rows : 0.0));
    return b;
}

void add_interval_times(lpb_ctx* h, int L, lpb_profile* prof) {
    if (!prof || !h->opt.profile) return;
    float ms = 0.f;
    for (int t = 0; t < L; ++t) {
        if (cudaEventElapsedTime(&ms, h->events[3 * t], h->events[3 * t + 1]) == cudaSuccess) prof->ms[0] += ms;
        if (cudaEventElapsedTime(&ms, h->events[3 * t + 1], h->events[3 * t + 2]) == cudaSuccess) prof->ms[1] += ms;
    }
    if (cudaEventElapsedTime(&ms, h->events[3 * L], h->events[3 * L + 1]) == cudaSuccess) prof->ms[2] += ms;
    if (cudaEventElapsedTime(&ms, h->events[3 * L + 1], h->events[3 * L + 2]) == cudaSuccess) prof->ms[3] += ms;
}

template <typename T>
lpb_err lane_admit(lpb_ctx* h, Lane& ln, GroupRun& g, const lpb_lp_spec* specs_dev, const double* wx,
                   const double* wy, int64_t wsx, int64_t wsy, double tol, cudaStream_t s,
                   std::vector<GroupRun*>& groups) {
    const int c0 = ln.ncol, count = g.count;
    if (c0 + count > ln.cap) return fail(LPB_ERR_INVALID_ARG, "lane has too few free columns");
    if (g.id < 0 || g.id >= ln.gcap) return fail(LPB_ERR_INVALID_ARG, "bad group id");
    if (g.slot0 < 0 || g.slot0 + count > (int)ln.slot_used.size()) return fail(LPB_ERR_INVALID_ARG, "bad slots");
    const double eps_inf = h->opt.eps_infeas >= 0.0 ? h->opt.eps_infeas : tol;
    const double tol_dual = h->opt.eps_dual >= 0.0 ? h->opt.eps_dual : tol;
    const CheckData cd = lane_check_data(h, ln, 0);
    LPB_CU(launch_admit<T>(cd, iter_data<T>(h, ln), iter_bufs<T>(ln), ln.cap, c0, count, g.id, g.slot0, specs_dev, wx,
                           wy, wsx, wsy, h->c_norm_base, h->b_norm, tol, eps_inf, tol_dual, g.max_iter, ln.rec, s));
    if (count > 0)
        LPB_CU(cudaMemcpyAsync(ln.rec_h + c0, ln.rec + c0, sizeof(ColRecord) * count, cudaMemcpyDeviceToHost, s));
    LPB_CU(cudaMemcpyAsync(ln.ctl_h + g.id, ln.ctl + g.id, sizeof(Control), cudaMemcpyDeviceToHost, s));
    LPB_CU(cudaStreamSynchronize(s));
    if (ln.ctl_h[g.id].error) {
        const int code = ln.ctl_h[g.id].error;
        LPB_CU(cudaMemsetAsync(ln.ctl + g.id, 0, sizeof(Control), s));
        ln.ctl_h[g.id].active = 0;
        return fail((lpb_err)code, code == LPB_ERR_BAD_INDEX ? "an override names a variable outside [0, n)"
                                                              : "an override record has an invalid kind or value");
    }
    for (int q = 0; q < count; ++q) {
        ln.slot_used[g.slot0 + q] = 1;
        ln.col_group[c0 + q] = g.id;
        ln.col_lp[c0 + q] = q;
    }
    if ((int)groups.size() <= g.id) groups.resize(g.id + 1, nullptr);
    groups[g.id] = &g;
    ln.ncol = c0 + count;
    g.live = count;
    g.K = 0;
    g.stalled = false;
    // LPs infeasible from their overrides alone (lo > hi) finish now
    std::vector<int> gone;
    for (int q = 0; q < count; ++q) {
        const ColRecord& rc = ln.rec_h[c0 + q];
        if (rc.status >= 0) {
            set_result(g.res[q], rc, rc.status, 0, 0);
            gone.push_back(c0 + q);
        }
    }
    g.live -= (int)gone.size();
    lpb_err rc = compact<T>(h, ln, gone, s, nullptr);
    if (rc != LPB_OK) return rc;
    if (g.live == 0) {
        if ((rc = retire_group(ln, g, s)) != LPB_OK) return rc;
        groups[g.id] = nullptr;
    }
    return LPB_OK;
}

namespace {

// The check of lane ln after an interval of L iterations, then the copies
// of the per-column and per-group records to their pinned mirrors.
template <typename T>
lpb_err queue_check(lpb_ctx* h, Lane& ln, int L, int stall_checks, cudaStream_t s, cudaEvent_t* ev) {
    const CheckData cd = lane_check_data(h, ln, stall_checks);
    LPB_CU(launch_check<T>(cd, iter_bufs<T>(ln), ln.cap, ln.ncol, L, h->P, h->Q, h->partials, h->colsum, ln.rec,
                           iter_data<T>(h, ln).col, s, ev));
    LPB_CU(cudaMemcpyAsync(ln.rec_h, ln.rec, sizeof(ColRecord) * ln.ncol, cudaMemcpyDeviceToHost, s));
    LPB_CU(cudaMemcpyAsync(ln.ctl_h, ln.ctl, sizeof(Control) * ln.gcap, cudaMemcpyDeviceToHost, s));
    return LPB_OK;
}

// Queues the L iterations of an interval, the check and the copies of the
// per-column and per-group records.
template <typename T>
lpb_err queue_interval(lpb_ctx* h, Lane& ln, int L, int stall_checks, int uni, bool timed, cudaStream_t s) {
    const int ld = ln.cap, ce = h->opt.check_every;
    const IterData<T> id = iter_data<T>(h, ln);
    const IterBufs<T> ib = iter_bufs<T>(ln);
    const T* hal = pick<T>(ln.hal64, ln.hal32, ln.haldf);
    const bool pdl = h->opt.use_pdl != 0;
    for (int t = 0; t < L; ++t)
        LPB_CU(launch_iteration<T>(id, ib, ld, ln.ncol, hal, t, ce, uni, t == L - 1, pdl, s,
                                   timed ? &h->events[3 * t] : nullptr));
    return queue_check<T>(h, ln, L, stall_checks, s, timed ? &h->events[3 * L] : nullptr);
}

// the group of every active column of the lane, or -1
int lane_uni(const Lane& ln) {
    int uni = ln.ncol > 0 ? ln.col_group[0] : -1;
    for (int j = 1; j < ln.ncol && uni >= 0; ++j)
        if (ln.col_group[j] != uni) uni = -1;
    return uni;
}

// Captures what queue() puts on stream s as a CUDA graph and makes *exec
// replay it: updated in place when the topology allows, else instantiated
// anew.
template <typename Q>
lpb_err capture_into(cudaGraphExec_t* exec, cudaStream_t s, Q queue) {
    cudaGraph_t g = nullptr;
    LPB_CU(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    const lpb_err rc = queue();
    const cudaError_t e = cudaStreamEndCapture(s, &g);
    if (rc != LPB_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    LPB_CU(e);
    if (*exec) {
        cudaGraphExecUpdateResultInfo info{};
        if (cudaGraphExecUpdate(*exec, g, &info) != cudaSuccess) {
            cudaGetLastError();
            cudaGraphExecDestroy(*exec);
            *exec = nullptr;
        }
    }
    if (!*exec) {
        const cudaError_t ei = cudaGraphInstantiate(exec, g, 0);
        if (ei != cudaSuccess) {
            cudaGraphDestroy(g);
            *exec = nullptr;
            return cuda_fail(ei, "cudaGraphInstantiate");
        }
    }
    cudaGraphDestroy(g);
    return LPB_OK;
}

// launches, kernels and algorithmic bytes of one interval of lane ln
template <typename T>
void count_interval(const lpb_ctx* h, const Lane& ln, int L, lpb_profile* prof) {
    if (!prof) return;
    const int m = h->m;
    for (int t = 0; t < L; ++t) {
        const bool chk = t == L - 1;
        prof->launches[0] += 1;
        prof->launches[1] += m > 0 ? 1 : 0;
        prof->kernels += m > 0 ? 2 : 1;
        prof->bytes[0] += step_bytes(prec_of<T>(), h->nnz, m, h->n, true, chk, ln.ncol);
        prof->bytes[1] += step_bytes(prec_of<T>(), h->nnz, m, h->n, false, chk, ln.ncol);
    }
    prof->launches[2] += m > 0 ? 2 : 1;
    prof->launches[3] += 1;
    prof->checks += 1;
    prof->kernels += (m > 0 ? 2 : 1) + (m > 0 ? 1 : 0) + 1 + 1 + 1 + (m > 0 ? 2 : 1);
}

}  // namespace

template <typename T>
lpb_err lane_interval(lpb_ctx* h, Lane& ln, int L, int stall_checks, cudaStream_t s, lpb_profile* prof) {
    const int ce = h->opt.check_every;
    const bool timed = prof && h->opt.profile && (int)h->events.size() >= 3 * ce + 3;
    const int uni = lane_uni(ln);
    if (!h->opt.use_graphs || timed) {
        lpb_err rc = queue_interval<T>(h, ln, L, stall_checks, uni, timed, s);
        if (rc != LPB_OK) return rc;
    } else {
        // one CUDA graph per interval shape, replayed while the shape holds;
        // a new shape updates the executable graph in place when it can
        const GraphKey key = interval_key(h, ln, L, stall_checks, uni, (int)sizeof(T));
        if (!ln.exec || !(ln.gkey == key)) {
            const lpb_err rc = capture_into(&ln.exec, s, [&] { return queue_interval<T>(h, ln, L, stall_checks, uni, false, s); });
            if (rc != LPB_OK) return rc;
            ln.gkey = key;
        }
        LPB_CU(cudaGraphLaunch(ln.exec, s));
    }
    count_interval<T>(h, ln, L, prof);
    return LPB_OK;
}

void joint_graph_free(JointGraph& jg) {
    if (jg.exec) cudaGraphExecDestroy(jg.exec);
    jg.exec = nullptr;
    jg.keys.clear();
    jg.seen.clear();
}

template <typename T>
lpb_err joint_interval(lpb_ctx* const* hs, Lane* const* lns, const int* stall_checks, int count, int L,
                       cudaStream_t s, JointGraph& jg, lpb_profile* const* profs) {
    std::vector<IterPart<T>> parts(count);
    std::vector<GraphKey> keys(count);
    for (int i = 0; i < count; ++i) {
        const lpb_ctx* h = hs[i];
        const Lane& ln = *lns[i];
        IterPart<T>& q = parts[i];
        q.d = iter_data<T>(h, ln);
        q.b = iter_bufs<T>(ln);
        q.ld = ln.cap;
        q.ncol = ln.ncol;
        q.ce = h->opt.check_every;
        q.uni = lane_uni(ln);
        q.hal = pick<T>(ln.hal64, ln.hal32, ln.haldf);
        keys[i] = interval_key(h, ln, L, stall_checks[i], q.uni, (int)sizeof(T));
    }
    const bool pdl = hs[0]->opt.use_pdl != 0;
    auto queue = [&]() -> lpb_err {
        for (int t = 0; t < L; ++t) LPB_CU(launch_iteration_multi<T>(parts.data(), count, t, t == L - 1, pdl, s));
        for (int i = 0; i < count; ++i) {
            const lpb_err rc = queue_check<T>(hs[i], *lns[i], L, stall_checks[i], s, nullptr);
            if (rc != LPB_OK) return rc;
        }
        return LPB_OK;
    };
    // one graph per joint shape (every lane's interval key, in order), taken
    // once the shape has held for an interval: with several lanes some lane
    // compacts at most checks, and a graph replayed once does not repay its
    // capture
    const bool replay = hs[0]->opt.use_graphs && jg.exec && jg.keys == keys;
    const bool capture = hs[0]->opt.use_graphs && !replay && jg.seen == keys;
    if (replay || capture) {
        if (capture) {
            const lpb_err rc = capture_into(&jg.exec, s, queue);
            if (rc != LPB_OK) return rc;
            jg.keys = keys;
        }
        LPB_CU(cudaGraphLaunch(jg.exec, s));
    } else {
        const lpb_err rc = queue();
        if (rc != LPB_OK) return rc;
    }
    jg.seen = keys;
    for (int i = 0; i < count; ++i) count_interval<T>(hs[i], *lns[i], L, profs ? profs[i] : nullptr);
    return LPB_OK;
}

template <typename T>
lpb_err lane_collect(lpb_ctx* h, Lane& ln, std::vector<GroupRun*>& groups, cudaStream_t s, lpb_profile* prof,
                     bool idle) {
    for (int gi = 0; gi < (int)groups.size(); ++gi) {
        GroupRun* g = groups[gi];
        if (!g) continue;
        g->K = ln.ctl_h[gi].K;
        g->stalled = ln.ctl_h[gi].stalled != 0;
    }
    std::vector<int> fin;
    for (int j = 0; j < ln.ncol; ++j) {
        const int gi = ln.col_group[j];
        GroupRun* g = groups[gi];
        const Control& c = ln.ctl_h[gi];
        int sj = ln.rec_h[j].status;
        if (sj < 0 && c.K >= g->max_iter) sj = LPB_ITERATION_LIMIT;
        if (sj >= 0) {
            set_result(g->res[ln.col_lp[j]], ln.rec_h[j], sj, c.K, c.restarts - c.restart);
            fin.push_back(j);
        }
    }
    if (fin.empty()) return LPB_OK;
    const int cnt = (int)fin.size();
    if (!idle) LPB_CU(cudaStreamSynchronize(s));  // pinned lists free for reuse
    int* cols = ln.mv_h + 2 * ln.cap;
    for (int f = 0; f < cnt; ++f) {
        const int j = fin[f];
        const GroupRun* g = groups[ln.col_group[j]];
        const size_t lp = (size_t)ln.col_lp[j];
        cols[f] = j;
        ln.optr_h[f] = g->x_dev ? g->x_dev + lp * h->n : nullptr;
        ln.optr_h[cnt + f] = g->y_dev && h->m > 0 ? g->y_dev + lp * h->m : nullptr;
    }
    LPB_CU(cudaMemcpyAsync(ln.mv + 2 * ln.cap, cols, sizeof(int) * cnt, cudaMemcpyHostToDevice, s));
    LPB_CU(cudaMemcpyAsync(ln.optr, ln.optr_h, sizeof(double*) * 2 * cnt, cudaMemcpyHostToDevice, s));
    const CheckData cd = lane_check_data(h, ln, 0);
    LPB_CU(launch_extract<T>(cd, iter_bufs<T>(ln), ln.cap, ln.mv + 2 * ln.cap, ln.optr, cnt, h->xl, h->xu, s));
    if (prof) prof->kernels += 1;
    for (int j : fin) groups[ln.col_group[j]]->live -= 1;
    std::vector<int> done_groups;
    for (int j : fin) {
        const int gi = ln.col_group[j];
        if (groups[gi] && groups[gi]->live == 0 &&
            std::find(done_groups.begin(), done_groups.end(), gi) == done_groups.end())
            done_groups.push_back(gi);
    }
    // the extraction's copies read the column and pointer lists, not the
    // move lists that the compaction fills
    lpb_err rc = compact<T>(h, ln, fin, s, prof, idle);
    if (rc != LPB_OK) return rc;
    for (int gi : done_groups) {
        if ((rc = retire_group(ln, *groups[gi], s)) != LPB_OK) return rc;
        groups[gi] = nullptr;
    }
    return LPB_OK;
}

template <typename TD>
lpb_err lane_migrate(lpb_ctx* h, Lane& src, Lane& dst, GroupRun& g, int id_dst, int slot0_dst, cudaStream_t s,
                     std::vector<GroupRun*>& src_groups) {
    std::vector<int> sc;
    for (int j = 0; j < src.ncol; ++j)
        if (src.col_group[j] == g.id) sc.push_back(j);
    const int cnt = (int)sc.size();
    if (dst.ncol + cnt > dst.cap) return fail(LPB_ERR_INVALID_ARG, "polish lane has too few free columns");
    if (id_dst < 0 || id_dst >= dst.gcap) return fail(LPB_ERR_INVALID_ARG, "bad polish group id");
    LPB_CU(cudaStreamSynchronize(s));  // pinned lists free for reuse
    LPB_CU(cudaMemcpyAsync(dst.ctl + id_dst, src.ctl + g.id, sizeof(Control), cudaMemcpyDeviceToDevice, s));
    const CheckData dcd = lane_check_data(h, dst, 0);
    LPB_CU(launch_group_moved(dcd, id_dst, slot0_dst, s));
    int* scol = src.mv_h + 2 * src.cap;
    int* dcol = src.mv_h + 3 * src.cap;
    for (int q = 0; q < cnt; ++q) {
        scol[q] = sc[q];
        dcol[q] = dst.ncol + q;
    }
    if (cnt > 0) {
        LPB_CU(cudaMemcpyAsync(src.mv + 2 * src.cap, scol, sizeof(int) * 2 * src.cap, cudaMemcpyHostToDevice, s));
        const CheckData scd = lane_check_data(h, src, 0);
        LPB_CU(launch_migrate<TD>(scd, iter_bufs<float>(src), src.cap, dcd, iter_bufs<TD>(dst), dst.cap,
                                  iter_data<TD>(h, dst).col, src.mv + 2 * src.cap, src.mv + 3 * src.cap, cnt, id_dst,
                                  slot0_dst - g.slot0, s));
    }
    for (int q = 0; q < cnt; ++q) {
        dst.col_group[dst.ncol + q] = id_dst;
        dst.col_lp[dst.ncol + q] = src.col_lp[sc[q]];
    }
    for (int q = 0; q < g.count; ++q) dst.slot_used[slot0_dst + q] = 1;
    dst.ncol += cnt;
    // the group leaves the FP32 lane
    lpb_err rc = compact<float>(h, src, sc, s, nullptr);
    if (rc != LPB_OK) return rc;
    if ((rc = retire_group(src, g, s)) != LPB_OK) return rc;
    src_groups[g.id] = nullptr;
    g.id = id_dst;
    g.slot0 = slot0_dst;
    g.live = cnt;
    g.stalled = false;
    LPB_CU(cudaMemcpyAsync(dst.ctl_h + id_dst, dst.ctl + id_dst, sizeof(Control), cudaMemcpyDeviceToHost, s));
    return LPB_OK;
}

template <typename T> IterData<T> lane_iter_data(const lpb_ctx* h, const Lane& ln) { return iter_data<T>(h, ln); }
template <typename T> IterBufs<T> lane_iter_bufs(const Lane& ln) { return iter_bufs<T>(ln); }
template <typename T> const T* lane_hal(const Lane& ln) { return pick<T>(ln.hal64, ln.hal32, ln.haldf); }

#define LPB_ENGINE_INSTANTIATE(T)                                                                                  \
    template lpb_err lane_admit<T>(lpb_ctx*, Lane&, GroupRun&, const lpb_lp_spec*, const double*, const double*,  \
                                   int64_t, int64_t, double, cudaStream_t, std::vector<GroupRun*>&);               \
    template lpb_err lane_interval<T>(lpb_ctx*, Lane&, int, int, cudaStream_t, lpb_profile*);                      \
    template lpb_err lane_collect<T>(lpb_ctx*, Lane&, std::vector<GroupRun*>&, cudaStream_t, lpb_profile*, bool);    \
    template IterData<T> lane_iter_data<T>(const lpb_ctx*, const Lane&);                                            \
    template IterBufs<T> lane_iter_bufs<T>(const Lane&);                                                            \
    template const T* lane_hal<T>(const Lane&);
LPB_ENGINE_INSTANTIATE(float)
LPB_ENGINE_INSTANTIATE(double)
LPB_ENGINE_INSTANTIATE(dfloat)
template lpb_err joint_interval<float>(lpb_ctx* const*, Lane* const*, const int*, int, int, cudaStream_t,
                                       JointGraph&, lpb_profile* const*);
template lpb_err joint_interval<double>(lpb_ctx* const*, Lane* const*, const int*, int, int, cudaStream_t,
                                        JointGraph&, lpb_profile* const*);
template lpb_err joint_interval<dfloat>(lpb_ctx* const*, Lane* const*, const int*, int, int, cudaStream_t,
                                        JointGraph&, lpb_profile* const*);
template lpb_err lane_migrate<double>(lpb_ctx*, Lane&, Lane&, GroupRun&, int, int, cudaStream_t,
                                      std::vector<GroupRun*>&);
template lpb_err lane_migrate<dfloat>(lpb_ctx*, Lane&, Lane&, GroupRun&, int, int, cudaStream_t,
                                      std::vector<GroupRun*>&);

}  // namespace lpb
