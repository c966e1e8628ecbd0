// lpb_api.cu -- the C ABI (include/lpb.h): handle set-up, the batched solve
// loop, extraction of results.  Host code here only validates arguments,
// allocates, launches and moves O(N) per-LP records between checks; every
// step of the method runs in the kernels of lpb_setup.cu, lpb_iter.cu and
// lpb_check.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lpb_internal.h"

using namespace lpb;

namespace {

thread_local std::string g_err;

lpb_err fail(lpb_err code, const std::string& msg) {
    g_err = msg;
    return code;
}

lpb_err cuda_fail(cudaError_t e, const char* what) {
    return fail(e == cudaErrorMemoryAllocation ? LPB_ERR_OOM : LPB_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define CU(call)                                              \
    do {                                                      \
        cudaError_t _e = (call);                              \
        if (_e != cudaSuccess) return cuda_fail(_e, #call);   \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (dev >= 0 && dev != prev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

size_t rup(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace

struct lpb_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    lpb_options opt{};
    int m = 0, n = 0, nnz = 0;
    Csr A, At;
    double *d_r = nullptr, *d_c = nullptr;
    double *c = nullptr, *l = nullptr, *u = nullptr, *xl = nullptr, *xu = nullptr;
    double *cs = nullptr, *ls = nullptr, *us = nullptr, *xls = nullptr, *xus = nullptr;
    float *cs32 = nullptr, *ls32 = nullptr, *us32 = nullptr, *xls32 = nullptr, *xus32 = nullptr;
    // double-float copies for the checks of FP32 iterates
    df *f_dr = nullptr, *f_dc = nullptr, *f_idr = nullptr, *f_idc = nullptr, *f_c = nullptr;
    df *f_xl = nullptr, *f_xu = nullptr, *f_l = nullptr, *f_u = nullptr;
    double eta = 0.0, norm_est = 0.0, c_norm_base = 0.0, b_norm = 0.0, setup_ms = 0.0;
    int power_iters = 0;
    std::vector<void*> fixed_allocs;
    // per-capacity workspace
    int cap = 0, ld = 0;
    std::vector<void*> ws_allocs;
    // iterate buffers and per-column parameters in each precision: [0] FP32
    // (mixed path), [1] FP64 (FP64 path, and the mixed path's FP64 polish)
    struct Set {
        void *X = nullptr, *X0 = nullptr, *Xbar = nullptr, *Xh = nullptr, *DX = nullptr;
        void *Y = nullptr, *Y0 = nullptr, *Yh = nullptr, *DY = nullptr, *DYp = nullptr;
        void *clo = nullptr, *chi = nullptr, *cc = nullptr, *ctau = nullptr, *csigma = nullptr;
    } set[2];
    double *P = nullptr, *Q = nullptr, *partials = nullptr, *colsum = nullptr;
    int *ckind = nullptr, *cvar = nullptr, *clp = nullptr, *k_stall = nullptr;
    double *k_lo = nullptr, *k_hi = nullptr, *k_c = nullptr, *k_w = nullptr, *k_best = nullptr;
    double* hal64 = nullptr;   // Halpern weights of the next interval
    float* hal32 = nullptr;
    ColRecord* rec = nullptr;
    Control* ctl = nullptr;
    int* mv = nullptr;
    lpb_lp_spec* specs_dev = nullptr;
    ColRecord* rec_h = nullptr;
    Control* ctl_h = nullptr;
    int* mv_h = nullptr;
    std::vector<cudaEvent_t> events;
};

struct lpb_batch {
    int device = 0;
    int num_lps = 0, m = 0, n = 0;
    std::vector<lpb_lp_result> res;
    double* x = nullptr;
    double* y = nullptr;
    lpb_profile prof{};
};

namespace {

template <typename P>
cudaError_t dmalloc(std::vector<void*>& list, P** out, size_t count) {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, count ? count : 1);
    if (e == cudaSuccess) list.push_back(p);
    *out = (P*)p;
    return e;
}

void free_list(std::vector<void*>& list) {
    for (void* p : list) cudaFree(p);
    list.clear();
}

void free_workspace(lpb_ctx* h) {
    free_list(h->ws_allocs);
    if (h->rec_h) cudaFreeHost(h->rec_h);
    if (h->ctl_h) cudaFreeHost(h->ctl_h);
    if (h->mv_h) cudaFreeHost(h->mv_h);
    h->rec_h = nullptr;
    h->ctl_h = nullptr;
    h->mv_h = nullptr;
    h->cap = h->ld = 0;
}

bool polish_enabled(const lpb_ctx* h) { return h->opt.precision == LPB_MIXED && h->opt.fp64_polish; }

lpb_err ensure_workspace(lpb_ctx* h, int num_lps) {
    if (num_lps <= h->cap) return LPB_OK;
    free_workspace(h);
    const int cap = (int)rup((size_t)num_lps, 4);
    const int ld = cap;
    const size_t mr = h->m > 0 ? (size_t)h->m : 1;
    auto& L = h->ws_allocs;
    for (int p = 0; p < 2; ++p) {
        const bool need = p == 1 ? (h->opt.precision == LPB_FP64 || polish_enabled(h)) : h->opt.precision == LPB_MIXED;
        if (!need) continue;
        const size_t tsz = p == 0 ? sizeof(float) : sizeof(double);
        auto& S = h->set[p];
        void** xs[] = {&S.X, &S.X0, &S.Xbar, &S.Xh, &S.DX};
        for (void** q : xs) CU(dmalloc(L, (char**)q, (size_t)h->n * ld * tsz));
        void** ys[] = {&S.Y, &S.Y0, &S.Yh, &S.DY, &S.DYp};
        for (void** q : ys) CU(dmalloc(L, (char**)q, mr * ld * tsz));
        void** cs[] = {&S.clo, &S.chi, &S.cc, &S.ctau, &S.csigma};
        for (void** q : cs) CU(dmalloc(L, (char**)q, tsz * ld));
    }
    CU(dmalloc(L, &h->P, sizeof(double) * 2 * mr * ld));
    CU(dmalloc(L, &h->Q, sizeof(double) * 3 * (size_t)h->n * ld));
    CU(dmalloc(L, &h->partials, sizeof(double) * (size_t)kNumStats * kReduceBlocks * ld));
    CU(dmalloc(L, &h->colsum, sizeof(double) * (size_t)kNumStats * ld));
    CU(dmalloc(L, &h->ckind, sizeof(int) * ld));
    CU(dmalloc(L, &h->cvar, sizeof(int) * ld));
    CU(dmalloc(L, &h->clp, sizeof(int) * ld));
    CU(dmalloc(L, &h->k_stall, sizeof(int) * ld));
    CU(dmalloc(L, &h->k_lo, sizeof(double) * ld));
    CU(dmalloc(L, &h->k_hi, sizeof(double) * ld));
    CU(dmalloc(L, &h->k_c, sizeof(double) * ld));
    CU(dmalloc(L, &h->k_w, sizeof(double) * ld));
    CU(dmalloc(L, &h->k_best, sizeof(double) * ld));
    CU(dmalloc(L, &h->hal64, sizeof(double) * 2 * (size_t)h->opt.check_every));
    CU(dmalloc(L, &h->hal32, sizeof(float) * 2 * (size_t)h->opt.check_every));
    CU(dmalloc(L, &h->rec, sizeof(ColRecord) * ld));
    CU(dmalloc(L, &h->ctl, sizeof(Control)));
    CU(dmalloc(L, &h->mv, sizeof(int) * 4 * ld));
    CU(dmalloc(L, &h->specs_dev, sizeof(lpb_lp_spec) * ld));
    CU(cudaMallocHost((void**)&h->rec_h, sizeof(ColRecord) * ld));
    CU(cudaMallocHost((void**)&h->ctl_h, sizeof(Control)));
    CU(cudaMallocHost((void**)&h->mv_h, sizeof(int) * 4 * ld));
    h->cap = cap;
    h->ld = ld;
    return LPB_OK;
}

template <typename T> const T* pick(const double* d64, const float* d32);
template <> const double* pick<double>(const double* d64, const float*) { return d64; }
template <> const float* pick<float>(const double*, const float* d32) { return d32; }
template <typename T> constexpr int set_of() { return sizeof(T) == sizeof(float) ? 0 : 1; }

template <typename T>
IterData<T> iter_data(const lpb_ctx* h) {
    const auto& S = h->set[set_of<T>()];
    IterData<T> d{};
    d.A = h->A;
    d.At = h->At;
    d.a_vals = pick<T>(h->A.v64, h->A.v32);
    d.at_vals = pick<T>(h->At.v64, h->At.v32);
    d.c = pick<T>(h->cs, h->cs32);
    d.xl = pick<T>(h->xls, h->xls32);
    d.xu = pick<T>(h->xus, h->xus32);
    d.l = pick<T>(h->ls, h->ls32);
    d.u = pick<T>(h->us, h->us32);
    d.col.kind = h->ckind;
    d.col.var = h->cvar;
    d.col.lo = (T*)S.clo;
    d.col.hi = (T*)S.chi;
    d.col.c = (T*)S.cc;
    d.col.tau = (T*)S.ctau;
    d.col.sigma = (T*)S.csigma;
    return d;
}

template <typename T>
IterBufs<T> iter_bufs(const lpb_ctx* h) {
    const auto& S = h->set[set_of<T>()];
    IterBufs<T> b{};
    b.X = (T*)S.X;
    b.X0 = (T*)S.X0;
    b.Xbar = (T*)S.Xbar;
    b.Y = (T*)S.Y;
    b.Y0 = (T*)S.Y0;
    b.Xh = (T*)S.Xh;
    b.DX = (T*)S.DX;
    b.G = nullptr;
    b.Yh = (T*)S.Yh;
    b.DY = (T*)S.DY;
    b.DYp = (T*)S.DYp;
    return b;
}

CheckData check_data(const lpb_ctx* h, double tol) {
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
    d.col.kind = h->ckind;
    d.col.var = h->cvar;
    d.col.lo = h->k_lo;
    d.col.hi = h->k_hi;
    d.col.c = h->k_c;
    d.col.w = h->k_w;
    d.col.lp = h->clp;
    d.col.best = h->k_best;
    d.col.stall = h->k_stall;
    d.eta = h->eta;
    d.beta_s = h->opt.beta_s;
    d.beta_n = h->opt.beta_n;
    d.beta_a = h->opt.beta_a;
    d.theta = h->opt.theta;
    d.mnorm_sign = h->opt.mnorm_sign;
    d.eps_inf = h->opt.eps_infeas >= 0.0 ? h->opt.eps_infeas : tol;
    d.tol = tol;
    d.detect_inf = h->opt.detect_infeasibility;
    d.restart_to_output = h->opt.restart_to_pdhg_output;
    d.stall_checks = 0;
    d.check_every = h->opt.check_every;
    d.hal64 = h->hal64;
    d.hal32 = h->hal32;
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

double step_bytes(bool fp32, int nnz, int m, int n, bool primal, bool check, int ncol) {
    const double ts = fp32 ? 4.0 : 8.0;
    const double rows = primal ? n : m, cols = primal ? m : n;
    double b = (4.0 + ts) * nnz + 4.0 * (rows + 1);
    // gathered block once, plus the row-side operands: primal reads X, X0 and
    // writes X, Xbar; dual reads Y, Y0 and writes Y; a check writes x^, dx
    // (primal) or y^, dy, Pi_B(dy) (dual)
    b += ts * ncol * (cols + rows * (primal ? 4.0 : 3.0) + (check ? (primal ? 2.0 : 3.0) * rows : 0.0));
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
}

// State of one solve that survives a change of iterate precision.
struct SolveState {
    std::vector<int> colmap;  // column -> LP index
    int ncol = 0;
    int64_t K = 0;            // iterations done
    bool done = false;
};

template <typename T>
lpb_err compact(lpb_ctx* h, SolveState& st, const std::vector<int>& fin, lpb_profile& prof) {
    if (fin.empty()) return LPB_OK;
    const int ncol = st.ncol;
    std::vector<char> is_fin(ncol, 0);
    for (int f : fin) is_fin[f] = 1;
    const int ncol2 = ncol - (int)fin.size();
    int* src = h->mv_h;
    int* dst = h->mv_h + h->ld;
    int cnt = 0, tail = ncol - 1;
    for (int f : fin) {
        if (f >= ncol2) break;
        while (is_fin[tail]) --tail;
        src[cnt] = tail;
        dst[cnt] = f;
        st.colmap[f] = st.colmap[tail];
        ++cnt;
        --tail;
    }
    st.ncol = ncol2;
    if (cnt == 0) return LPB_OK;
    CU(cudaMemcpyAsync(h->mv, src, sizeof(int) * cnt, cudaMemcpyHostToDevice, h->stream));
    CU(cudaMemcpyAsync(h->mv + h->ld, dst, sizeof(int) * cnt, cudaMemcpyHostToDevice, h->stream));
    IterData<T> id = iter_data<T>(h);
    CheckData cd = check_data(h, 1.0);
    CU(launch_compact<T>(iter_bufs<T>(h), h->n, h->m, h->ld, h->mv, h->mv + h->ld, cnt, id.col, cd.col, h->stream));
    prof.compactions += 1;
    prof.kernels += 2;
    return LPB_OK;
}

// Runs checked intervals in precision T until the batch is done, max_iter is
// reached, or (FP32 with polish enabled) an LP stalls.  Returns with
// st.done = false only in the last case.
template <typename T>
lpb_err run_phase(lpb_ctx* h, SolveState& st, double tol, int64_t max_iter, lpb_batch* bt) {
    lpb_err rc;
    cudaStream_t s = h->stream;
    const int m = h->m, ld = h->ld;
    IterData<T> id = iter_data<T>(h);
    IterBufs<T> ib = iter_bufs<T>(h);
    CheckData cd = check_data(h, tol);
    const bool can_promote = sizeof(T) == sizeof(float) && polish_enabled(h);
    if (can_promote) cd.stall_checks = h->opt.polish_stall_checks;
    lpb_profile& prof = bt->prof;
    const bool profile = h->opt.profile != 0;
    const int ce = h->opt.check_every;
    const bool fp32 = sizeof(T) == sizeof(float);
    std::vector<int> fin;
    while (st.ncol > 0 && st.K < max_iter) {
        const int L = (int)std::min<int64_t>(ce, max_iter - st.K);
        for (int t = 0; t < L; ++t) {
            const bool chk = t == L - 1;
            CU(launch_iteration<T>(id, ib, ld, st.ncol, pick<T>(h->hal64, h->hal32), t, chk, s,
                                   profile ? &h->events[3 * t] : nullptr));
            prof.launches[0] += 1;
            prof.launches[1] += m > 0 ? 1 : 0;
            prof.kernels += m > 0 ? 2 : 1;
            prof.bytes[0] += step_bytes(fp32, h->nnz, m, h->n, true, chk, st.ncol);
            prof.bytes[1] += step_bytes(fp32, h->nnz, m, h->n, false, chk, st.ncol);
        }
        CU(launch_check<T>(cd, ib, ld, st.ncol, st.K + L - 1, L, st.K + L == max_iter, h->P, h->Q, h->partials,
                           h->colsum, h->rec, h->ctl, id.col, s, profile ? &h->events[3 * L] : nullptr));
        prof.launches[2] += m > 0 ? 2 : 1;
        prof.launches[3] += 1;
        prof.checks += 1;
        prof.kernels += (m > 0 ? 2 : 1) + (m > 0 ? 1 : 0) + 1 + 1 + 1 + (m > 0 ? 2 : 1);
        CU(cudaMemcpyAsync(h->rec_h, h->rec, sizeof(ColRecord) * st.ncol, cudaMemcpyDeviceToHost, s));
        CU(cudaMemcpyAsync(h->ctl_h, h->ctl, sizeof(Control), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        if (profile) {
            float ms = 0.f;
            for (int t = 0; t < L; ++t) {
                CU(cudaEventElapsedTime(&ms, h->events[3 * t], h->events[3 * t + 1]));
                prof.ms[0] += ms;
                CU(cudaEventElapsedTime(&ms, h->events[3 * t + 1], h->events[3 * t + 2]));
                prof.ms[1] += ms;
            }
            CU(cudaEventElapsedTime(&ms, h->events[3 * L], h->events[3 * L + 1]));
            prof.ms[2] += ms;
            CU(cudaEventElapsedTime(&ms, h->events[3 * L + 1], h->events[3 * L + 2]));
            prof.ms[3] += ms;
        }
        st.K += L;
        const int64_t restarts_before = h->ctl_h->restarts - h->ctl_h->restart;
        fin.clear();
        for (int j = 0; j < st.ncol; ++j) {
            int sj = h->rec_h[j].status;
            if (sj < 0 && st.K >= max_iter) sj = LPB_ITERATION_LIMIT;
            if (sj >= 0) {
                set_result(bt->res[st.colmap[j]], h->rec_h[j], sj, st.K, restarts_before);
                fin.push_back(j);
            }
        }
        if (!fin.empty()) {
            int* cols = h->mv_h + 2 * ld;
            int* lps = h->mv_h + 3 * ld;
            for (size_t q = 0; q < fin.size(); ++q) {
                cols[q] = fin[q];
                lps[q] = st.colmap[fin[q]];
            }
            const int cnt = (int)fin.size();
            CU(cudaMemcpyAsync(h->mv + 2 * ld, cols, sizeof(int) * cnt, cudaMemcpyHostToDevice, s));
            CU(cudaMemcpyAsync(h->mv + 3 * ld, lps, sizeof(int) * cnt, cudaMemcpyHostToDevice, s));
            CU(launch_extract<T>(cd, ib, ld, h->mv + 2 * ld, h->mv + 3 * ld, cnt, h->xl, h->xu, bt->x, bt->y, s));
            prof.kernels += 1;
            if ((rc = compact<T>(h, st, fin, prof)) != LPB_OK) return rc;
        }
        if (can_promote && h->ctl_h->stalled && st.ncol > 0 && st.K < max_iter) return LPB_OK;
    }
    st.done = true;
    return LPB_OK;
}

template <typename T>
lpb_err solve_impl(lpb_ctx* h, int num_lps, const lpb_lp_spec* specs_dev, double tol, int64_t max_iter,
                   const double* wx, const double* wy, lpb_batch* bt) {
    lpb_err rc;
    if ((rc = ensure_workspace(h, num_lps)) != LPB_OK) return rc;
    cudaStream_t s = h->stream;
    const int n = h->n, m = h->m, ld = h->ld;
    CU(cudaMalloc((void**)&bt->x, sizeof(double) * (size_t)n * (num_lps ? num_lps : 1)));
    CU(cudaMalloc((void**)&bt->y, sizeof(double) * (size_t)(m ? m : 1) * (num_lps ? num_lps : 1)));
    CU(cudaMemsetAsync(bt->x, 0, sizeof(double) * (size_t)n * num_lps, s));
    CU(cudaMemsetAsync(bt->y, 0, sizeof(double) * (size_t)m * num_lps, s));
    bt->res.assign(num_lps, lpb_lp_result{});
    lpb_profile& prof = bt->prof;
    prof.setup_ms = h->setup_ms;
    prof.fp64_switch_iter = -1;
    if (num_lps == 0) {
        CU(cudaStreamSynchronize(s));
        return LPB_OK;
    }
    const int ce = h->opt.check_every;
    if (h->opt.profile && (int)h->events.size() < 3 * ce + 3) {
        for (cudaEvent_t e : h->events) cudaEventDestroy(e);
        h->events.assign(3 * ce + 3, nullptr);
        for (auto& e : h->events) CU(cudaEventCreate(&e));
    }
    IterData<T> id = iter_data<T>(h);
    IterBufs<T> ib = iter_bufs<T>(h);
    CheckData cd = check_data(h, tol);
    CU(launch_init<T>(cd, id, ib, ld, num_lps, specs_dev, wx, wy, h->c_norm_base, h->b_norm, h->rec, h->ctl, s));
    prof.kernels += 3;
    CU(cudaMemcpyAsync(h->rec_h, h->rec, sizeof(ColRecord) * num_lps, cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(h->ctl_h, h->ctl, sizeof(Control), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (h->ctl_h->error) {
        const int code = h->ctl_h->error;
        return fail((lpb_err)code, code == LPB_ERR_BAD_INDEX ? "an override names a variable outside [0, n)"
                                                              : "an override record has an invalid kind or value");
    }
    SolveState st;
    st.colmap.resize(num_lps);
    for (int j = 0; j < num_lps; ++j) st.colmap[j] = j;
    st.ncol = num_lps;
    std::vector<int> fin;
    for (int j = 0; j < num_lps; ++j)
        if (h->rec_h[j].status >= 0) {
            set_result(bt->res[j], h->rec_h[j], h->rec_h[j].status, 0, 0);
            fin.push_back(j);
        }
    if ((rc = compact<T>(h, st, fin, prof)) != LPB_OK) return rc;
    if ((rc = run_phase<T>(h, st, tol, max_iter, bt)) != LPB_OK) return rc;
    if (!st.done) {
        // FP64 polish: the remaining batch continues from its FP32 state with
        // FP64 iterates; the batch state on the device (k, r0, w, ...) carries over
        CU(launch_promote(cd, iter_bufs<float>(h), iter_bufs<double>(h), iter_data<double>(h).col, ld, st.ncol, s));
        prof.kernels += 5;
        prof.fp64_switch_iter = st.K;
        if ((rc = run_phase<double>(h, st, tol, max_iter, bt)) != LPB_OK) return rc;
    }
    CU(cudaStreamSynchronize(s));
    return LPB_OK;
}

lpb_err solve_common(lpb_handle h, int32_t num_lps, const lpb_lp_spec* specs_dev, double tol, int64_t max_iter,
                     const double* wx, const double* wy, lpb_batch_t* out) {
    lpb_batch* bt = new (std::nothrow) lpb_batch();
    if (!bt) return fail(LPB_ERR_OOM, "host allocation failed");
    bt->device = h->device;
    bt->num_lps = num_lps;
    bt->m = h->m;
    bt->n = h->n;
    lpb_err rc = h->opt.precision == LPB_MIXED ? solve_impl<float>(h, num_lps, specs_dev, tol, max_iter, wx, wy, bt)
                                               : solve_impl<double>(h, num_lps, specs_dev, tol, max_iter, wx, wy, bt);
    if (rc != LPB_OK) {
        lpb_batch_free(bt);
        return rc;
    }
    *out = bt;
    return LPB_OK;
}

lpb_err check_solve_args(lpb_handle h, int32_t num_lps, const void* specs, double tol, int64_t max_iter,
                         lpb_batch_t* out) {
    if (!h || !out) return fail(LPB_ERR_INVALID_ARG, "null handle or output pointer");
    if (num_lps < 0) return fail(LPB_ERR_INVALID_ARG, "num_lps < 0");
    if (num_lps > 0 && !specs) return fail(LPB_ERR_INVALID_ARG, "specs is NULL");
    if (!(tol > 0.0) || !std::isfinite(tol)) return fail(LPB_ERR_INVALID_ARG, "tol must be positive and finite");
    if (max_iter < 1) return fail(LPB_ERR_INVALID_ARG, "max_iter must be >= 1");
    return LPB_OK;
}

}  // namespace

extern "C" {

void lpb_default_options(lpb_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = LPB_MIXED;
    o->check_every = 64;
    o->ruiz_iters = 10;
    o->pock_chambolle = 1;
    o->beta_s = 0.2;
    o->beta_n = 0.8;
    o->beta_a = 0.36;
    o->theta = 0.5;
    o->mnorm_sign = -1.0;
    o->restart_to_pdhg_output = 1;
    o->power_max_iter = 5000;
    o->power_tol = 1e-10;
    o->power_seed = 0x5eedULL;
    o->eps_infeas = -1.0;
    o->detect_infeasibility = 1;
    o->profile = 0;
    o->cuda_stream = nullptr;
    o->device = -1;
    o->fp64_polish = 1;
    o->polish_stall_checks = 32;
}

const char* lpb_last_error(void) { return g_err.c_str(); }

}  // extern "C"

void lpb::set_last_error(const char* msg) { g_err = msg ? msg : ""; }

extern "C" {

lpb_err lpb_create(int32_t m, int32_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
                   const double* vals, const double* c, const double* row_lo, const double* row_hi,
                   const double* var_lo, const double* var_hi, const lpb_options* opt, lpb_handle* out) {
    if (!out) return fail(LPB_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (m < 0 || n < 1) return fail(LPB_ERR_INVALID_ARG, "need m >= 0 and n >= 1");
    if (nnz < 0 || nnz >= (int64_t)INT32_MAX) return fail(LPB_ERR_INVALID_ARG, "nnz must be in [0, 2^31 - 1)");
    if (!row_ptr || (nnz > 0 && (!col_idx || !vals)) || !c || !var_lo || !var_hi || (m > 0 && (!row_lo || !row_hi)))
        return fail(LPB_ERR_INVALID_ARG, "a required pointer is NULL");
    lpb_options o;
    lpb_default_options(&o);
    if (opt) o = *opt;
    if (o.precision != LPB_FP64 && o.precision != LPB_MIXED) return fail(LPB_ERR_INVALID_ARG, "bad precision");
    if (o.check_every < 1 || o.ruiz_iters < 0 || o.power_max_iter < 1 || (o.fp64_polish && o.polish_stall_checks < 1) || !(o.power_tol >= 0.0) ||
        !(o.theta >= 0.0 && o.theta <= 1.0) || !(o.beta_s >= 0.0) || !(o.beta_n >= 0.0) || !(o.beta_a >= 0.0))
        return fail(LPB_ERR_INVALID_ARG, "bad option value");
    // host validation, O(nnz)
    if (row_ptr[0] != 0 || row_ptr[m] != nnz) return fail(LPB_ERR_INVALID_ARG, "row_ptr[0] != 0 or row_ptr[m] != nnz");
    for (int32_t i = 0; i < m; ++i)
        if (row_ptr[i + 1] < row_ptr[i]) return fail(LPB_ERR_INVALID_ARG, "row_ptr is not monotone");
    for (int64_t e = 0; e < nnz; ++e) {
        if (col_idx[e] < 0 || col_idx[e] >= n) return fail(LPB_ERR_INVALID_ARG, "column index out of range");
        if (!std::isfinite(vals[e])) return fail(LPB_ERR_INVALID_ARG, "non-finite matrix value");
    }
    for (int32_t j = 0; j < n; ++j) {
        if (!std::isfinite(c[j])) return fail(LPB_ERR_INVALID_ARG, "non-finite cost");
        if (std::isnan(var_lo[j]) || std::isnan(var_hi[j]) || var_lo[j] > var_hi[j] || var_lo[j] == HUGE_VAL ||
            var_hi[j] == -HUGE_VAL)
            return fail(LPB_ERR_INVALID_ARG, "bad variable bounds");
    }
    for (int32_t i = 0; i < m; ++i)
        if (std::isnan(row_lo[i]) || std::isnan(row_hi[i]) || row_lo[i] > row_hi[i] || row_lo[i] == HUGE_VAL ||
            row_hi[i] == -HUGE_VAL)
            return fail(LPB_ERR_INVALID_ARG, "bad row bounds");

    lpb_ctx* h = new (std::nothrow) lpb_ctx();
    if (!h) return fail(LPB_ERR_OOM, "host allocation failed");
    h->opt = o;
    h->m = m;
    h->n = n;
    h->nnz = (int)nnz;
    auto cleanup = [&](lpb_err code) {
        lpb_destroy(h);
        return code;
    };
    int dev = o.device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return cleanup(fail(LPB_ERR_CUDA, "no CUDA device"));
    h->device = dev;
    DeviceGuard guard(dev);
    struct TmpFree {
        std::vector<void*> v;
        ~TmpFree() { free_list(v); }
    } tmp;
    lpb_err rc = [&]() -> lpb_err {
        if (o.cuda_stream) {
            h->stream = (cudaStream_t)o.cuda_stream;
        } else {
            CU(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
            h->own_stream = true;
        }
        cudaStream_t s = h->stream;
        cudaEvent_t t0, t1;
        CU(cudaEventCreate(&t0));
        CU(cudaEventCreate(&t1));
        CU(cudaEventRecord(t0, s));
        auto& F = h->fixed_allocs;
        const size_t mm = m > 0 ? m : 1;
        // A (CSR) and raw values
        std::vector<int> rp32(m + 1);
        for (int32_t i = 0; i <= m; ++i) rp32[i] = (int)row_ptr[i];
        h->A.rows = m;
        h->A.cols = n;
        h->A.nnz = (int)nnz;
        CU(dmalloc(F, &h->A.rp, sizeof(int) * (m + 1)));
        CU(dmalloc(F, &h->A.ci, sizeof(int) * nnz));
        CU(dmalloc(F, &h->A.v64, sizeof(double) * nnz));
        double* raw = nullptr;
        CU(dmalloc(tmp.v, &raw, sizeof(double) * (nnz ? nnz : 1)));
        CU(cudaMemcpyAsync(h->A.rp, rp32.data(), sizeof(int) * (m + 1), cudaMemcpyHostToDevice, s));
        if (nnz) {
            CU(cudaMemcpyAsync(h->A.ci, col_idx, sizeof(int) * nnz, cudaMemcpyHostToDevice, s));
            CU(cudaMemcpyAsync(raw, vals, sizeof(double) * nnz, cudaMemcpyHostToDevice, s));
        }
        // vectors
        CU(dmalloc(F, &h->c, sizeof(double) * n));
        CU(dmalloc(F, &h->xl, sizeof(double) * n));
        CU(dmalloc(F, &h->xu, sizeof(double) * n));
        CU(dmalloc(F, &h->l, sizeof(double) * mm));
        CU(dmalloc(F, &h->u, sizeof(double) * mm));
        CU(cudaMemcpyAsync(h->c, c, sizeof(double) * n, cudaMemcpyHostToDevice, s));
        CU(cudaMemcpyAsync(h->xl, var_lo, sizeof(double) * n, cudaMemcpyHostToDevice, s));
        CU(cudaMemcpyAsync(h->xu, var_hi, sizeof(double) * n, cudaMemcpyHostToDevice, s));
        if (m) {
            CU(cudaMemcpyAsync(h->l, row_lo, sizeof(double) * m, cudaMemcpyHostToDevice, s));
            CU(cudaMemcpyAsync(h->u, row_hi, sizeof(double) * m, cudaMemcpyHostToDevice, s));
        }
        // transpose (A^T values land raw in At.v64)
        h->At.rows = n;
        h->At.cols = m;
        h->At.nnz = (int)nnz;
        CU(dmalloc(F, &h->At.rp, sizeof(int) * (n + 1)));
        CU(dmalloc(F, &h->At.ci, sizeof(int) * nnz));
        CU(dmalloc(F, &h->At.v64, sizeof(double) * nnz));
        int* perm = nullptr;
        CU(dmalloc(tmp.v, &perm, sizeof(int) * (nnz ? nnz : 1)));
        CU(transpose_csr(h->A, raw, h->At, perm, s));
        // equilibration
        CU(dmalloc(F, &h->d_r, sizeof(double) * mm));
        CU(dmalloc(F, &h->d_c, sizeof(double) * n));
        double *tr = nullptr, *tc = nullptr;
        CU(dmalloc(tmp.v, &tr, sizeof(double) * mm));
        CU(dmalloc(tmp.v, &tc, sizeof(double) * n));
        CU(ruiz_pock_chambolle(h->A, raw, h->At, h->At.v64, o.ruiz_iters, o.pock_chambolle, h->d_r, h->d_c, tr, tc, s));
        const bool mixed = o.precision == LPB_MIXED;
        if (mixed) {
            CU(dmalloc(F, &h->A.v32, sizeof(float) * nnz));
            CU(dmalloc(F, &h->At.v32, sizeof(float) * nnz));
        }
        CU(scale_values(h->A, raw, h->d_r, h->d_c, true, h->A.v64, h->A.v32, s));
        CU(scale_values(h->At, h->At.v64, h->d_r, h->d_c, false, h->At.v64, h->At.v32, s));
        CU(build_long_rows(h->A, s));
        CU(build_long_rows(h->At, s));
        if (h->A.long_rows) F.push_back(h->A.long_rows);
        if (h->At.long_rows) F.push_back(h->At.long_rows);
        // scaled vectors
        CU(dmalloc(F, &h->cs, sizeof(double) * n));
        CU(dmalloc(F, &h->xls, sizeof(double) * n));
        CU(dmalloc(F, &h->xus, sizeof(double) * n));
        CU(dmalloc(F, &h->ls, sizeof(double) * mm));
        CU(dmalloc(F, &h->us, sizeof(double) * mm));
        CU(scale_vectors(m, n, h->d_r, h->d_c, h->c, h->l, h->u, h->xl, h->xu, h->cs, h->ls, h->us, h->xls, h->xus, s));
        if (mixed) {
            CU(dmalloc(F, &h->cs32, sizeof(float) * n));
            CU(dmalloc(F, &h->xls32, sizeof(float) * n));
            CU(dmalloc(F, &h->xus32, sizeof(float) * n));
            CU(dmalloc(F, &h->ls32, sizeof(float) * mm));
            CU(dmalloc(F, &h->us32, sizeof(float) * mm));
            CU(convert_f32(h->cs, h->cs32, n, s));
            CU(convert_f32(h->xls, h->xls32, n, s));
            CU(convert_f32(h->xus, h->xus32, n, s));
            CU(convert_f32(h->ls, h->ls32, m, s));
            CU(convert_f32(h->us, h->us32, m, s));
            // double-float data of the FP32-iterate checks
            CU(dmalloc(F, &h->A.v32lo, sizeof(float) * nnz));
            CU(dmalloc(F, &h->At.v32lo, sizeof(float) * nnz));
            CU(split_lo(h->A.v64, h->A.v32, h->A.v32lo, (int)nnz, s));
            CU(split_lo(h->At.v64, h->At.v32, h->At.v32lo, (int)nnz, s));
            df** nv[] = {&h->f_dc, &h->f_idc, &h->f_c, &h->f_xl, &h->f_xu};
            for (df** p : nv) CU(dmalloc(F, p, sizeof(df) * n));
            df** mv[] = {&h->f_dr, &h->f_idr, &h->f_l, &h->f_u};
            for (df** p : mv) CU(dmalloc(F, p, sizeof(df) * mm));
            CU(split_df(h->d_c, h->f_dc, n, false, s));
            CU(split_df(h->d_c, h->f_idc, n, true, s));
            CU(split_df(h->c, h->f_c, n, false, s));
            CU(split_df(h->xl, h->f_xl, n, false, s));
            CU(split_df(h->xu, h->f_xu, n, false, s));
            CU(split_df(h->d_r, h->f_dr, m, false, s));
            CU(split_df(h->d_r, h->f_idr, m, true, s));
            CU(split_df(h->l, h->f_l, m, false, s));
            CU(split_df(h->u, h->f_u, m, false, s));
        }
        // ||c~||, ||b~|| (w0) and the power iteration (eta)
        double* scal = nullptr;
        CU(dmalloc(tmp.v, &scal, sizeof(double) * 2));
        CU(sq_norm(h->cs, n, scal, s));
        if (m) CU(rhs_norm2(h->ls, h->us, m, scal + 1, s));
        else CU(cudaMemsetAsync(scal + 1, 0, sizeof(double), s));
        double hs[2] = {0.0, 0.0};
        CU(cudaMemcpyAsync(hs, scal, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
        double* work = nullptr;
        const size_t wn = 2 * (size_t)n + mm + 3 + 2 * ((size_t)o.power_max_iter + 1) + 256;
        CU(dmalloc(tmp.v, &work, sizeof(double) * wn));
        double est = 0.0;
        int its = 0;
        CU(power_norm(h->A, h->At, o.power_max_iter, o.power_tol, o.power_seed, work, &est, &its, s));
        CU(cudaEventRecord(t1, s));
        CU(cudaStreamSynchronize(s));
        float ms = 0.f;
        CU(cudaEventElapsedTime(&ms, t0, t1));
        h->setup_ms = ms;
        cudaEventDestroy(t0);
        cudaEventDestroy(t1);
        h->c_norm_base = std::sqrt(hs[0]);
        h->b_norm = std::sqrt(hs[1]);
        h->norm_est = est;
        h->power_iters = its;
        h->eta = 0.998 / (est > 0.0 ? est : 1.0);
        return LPB_OK;
    }();
    if (rc != LPB_OK) return cleanup(rc);
    *out = h;
    return LPB_OK;
}

lpb_err lpb_solve(lpb_handle h, int32_t num_lps, const lpb_lp_spec* specs, double tol, int64_t max_iter,
                  const double* warm_x, const double* warm_y, lpb_batch_t* out) {
    lpb_err rc = check_solve_args(h, num_lps, specs, tol, max_iter, out);
    if (rc != LPB_OK) return rc;
    *out = nullptr;
    for (int32_t q = 0; q < num_lps; ++q) {
        const lpb_lp_spec& sp = specs[q];
        if (sp.kind < 0 || sp.kind > 2) return fail(LPB_ERR_INVALID_ARG, "override kind must be 0, 1 or 2");
        if (sp.kind != 0 && (sp.var < 0 || sp.var >= h->n))
            return fail(LPB_ERR_BAD_INDEX, "an override names a variable outside [0, n)");
        if (sp.kind == 1 && (std::isnan(sp.lo) || std::isnan(sp.hi)))
            return fail(LPB_ERR_INVALID_ARG, "NaN override bound");
        if (sp.kind == 2 && !std::isfinite(sp.sign)) return fail(LPB_ERR_INVALID_ARG, "non-finite objective sign");
    }
    DeviceGuard guard(h->device);
    if ((rc = ensure_workspace(h, num_lps)) != LPB_OK) return rc;
    cudaStream_t s = h->stream;
    double *wx = nullptr, *wy = nullptr;
    if (num_lps > 0) CU(cudaMemcpyAsync(h->specs_dev, specs, sizeof(lpb_lp_spec) * num_lps, cudaMemcpyHostToDevice, s));
    if (warm_x && num_lps > 0) {
        CU(cudaMallocAsync((void**)&wx, sizeof(double) * (size_t)h->n * num_lps, s));
        CU(cudaMemcpyAsync(wx, warm_x, sizeof(double) * (size_t)h->n * num_lps, cudaMemcpyHostToDevice, s));
    }
    if (warm_y && num_lps > 0 && h->m > 0) {
        CU(cudaMallocAsync((void**)&wy, sizeof(double) * (size_t)h->m * num_lps, s));
        CU(cudaMemcpyAsync(wy, warm_y, sizeof(double) * (size_t)h->m * num_lps, cudaMemcpyHostToDevice, s));
    }
    rc = solve_common(h, num_lps, h->specs_dev, tol, max_iter, wx, wy, out);
    if (wx) cudaFreeAsync(wx, s);
    if (wy) cudaFreeAsync(wy, s);
    return rc;
}

lpb_err lpb_solve_dev(lpb_handle h, int32_t num_lps, const lpb_lp_spec* specs_dev, double tol, int64_t max_iter,
                      const double* warm_x_dev, const double* warm_y_dev, lpb_batch_t* out) {
    lpb_err rc = check_solve_args(h, num_lps, specs_dev, tol, max_iter, out);
    if (rc != LPB_OK) return rc;
    *out = nullptr;
    DeviceGuard guard(h->device);
    return solve_common(h, num_lps, specs_dev, tol, max_iter, warm_x_dev, h->m > 0 ? warm_y_dev : nullptr, out);
}

lpb_err lpb_result(lpb_batch_t b, int32_t lp, lpb_lp_result* res, double* x, double* y) {
    if (!b) return fail(LPB_ERR_INVALID_ARG, "null batch");
    if (lp < 0 || lp >= b->num_lps) return fail(LPB_ERR_INVALID_ARG, "lp index out of range");
    if (res) *res = b->res[lp];
    if (x || y) {
        DeviceGuard guard(b->device);
        if (x) CU(cudaMemcpy(x, b->x + (size_t)lp * b->n, sizeof(double) * b->n, cudaMemcpyDeviceToHost));
        if (y && b->m > 0) CU(cudaMemcpy(y, b->y + (size_t)lp * b->m, sizeof(double) * b->m, cudaMemcpyDeviceToHost));
    }
    return LPB_OK;
}

lpb_err lpb_results(lpb_batch_t b, lpb_lp_result* res) {
    if (!b || (!res && b->num_lps > 0)) return fail(LPB_ERR_INVALID_ARG, "null argument");
    if (b->num_lps > 0) std::memcpy(res, b->res.data(), sizeof(lpb_lp_result) * b->num_lps);
    return LPB_OK;
}

lpb_err lpb_result_device(lpb_batch_t b, const double** x_dev, const double** y_dev) {
    if (!b) return fail(LPB_ERR_INVALID_ARG, "null batch");
    if (x_dev) *x_dev = b->x;
    if (y_dev) *y_dev = b->y;
    return LPB_OK;
}

lpb_err lpb_batch_profile(lpb_batch_t b, lpb_profile* p) {
    if (!b || !p) return fail(LPB_ERR_INVALID_ARG, "null argument");
    *p = b->prof;
    return LPB_OK;
}

lpb_err lpb_handle_info(lpb_handle h, double* eta, double* norm_est, int32_t* power_iters) {
    if (!h) return fail(LPB_ERR_INVALID_ARG, "null handle");
    if (eta) *eta = h->eta;
    if (norm_est) *norm_est = h->norm_est;
    if (power_iters) *power_iters = h->power_iters;
    return LPB_OK;
}

lpb_err lpb_scaling(lpb_handle h, double* d_row, double* d_col) {
    if (!h) return fail(LPB_ERR_INVALID_ARG, "null handle");
    DeviceGuard guard(h->device);
    if (d_row && h->m > 0) CU(cudaMemcpy(d_row, h->d_r, sizeof(double) * h->m, cudaMemcpyDeviceToHost));
    if (d_col) CU(cudaMemcpy(d_col, h->d_c, sizeof(double) * h->n, cudaMemcpyDeviceToHost));
    return LPB_OK;
}

void lpb_batch_free(lpb_batch_t b) {
    if (!b) return;
    DeviceGuard guard(b->device);
    if (b->x) cudaFree(b->x);
    if (b->y) cudaFree(b->y);
    delete b;
}

void lpb_destroy(lpb_handle h) {
    if (!h) return;
    DeviceGuard guard(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (cudaEvent_t e : h->events) cudaEventDestroy(e);
    free_workspace(h);
    free_list(h->fixed_allocs);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

}  // extern "C"
