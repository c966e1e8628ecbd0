// lpb_api.cu -- the C ABI (include/lpb.h): handle set-up, the batched solve
// loop, extraction of results.  Host code here only validates arguments,
// allocates, launches and moves O(N) per-LP records between checks; every
// step of the method runs in the kernels of lpb_setup.cu, lpb_iter.cu and
// lpb_check.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "lpb_engine.h"

using namespace lpb;

namespace {

thread_local std::string g_err;

#define CU(call) LPB_CU(call)

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

}  // namespace

struct lpb_batch {
    int device = 0;
    int num_lps = 0, m = 0, n = 0;
    std::vector<lpb_lp_result> res;
    double* x = nullptr;
    double* y = nullptr;
    lpb_profile prof{};
};

namespace {

template <typename T> constexpr int prec_of() {
    return std::is_same<T, float>::value ? kPrecF32 : std::is_same<T, double>::value ? kPrecF64 : kPrecDfl;
}

lpb_err ensure_events(lpb_ctx* h) {
    const int ce = h->opt.check_every;
    if (!h->opt.profile || (int)h->events.size() >= 3 * ce + 3) return LPB_OK;
    for (cudaEvent_t e : h->events) cudaEventDestroy(e);
    h->events.assign(3 * ce + 3, nullptr);
    for (auto& e : h->events) CU(cudaEventCreate(&e));
    return LPB_OK;
}

// Runs checked intervals of lane ln until group g is done or (with can_stall)
// it stalls; returns done = false only in the second case.
template <typename T>
lpb_err run_group(lpb_ctx* h, Lane& ln, GroupRun& g, std::vector<GroupRun*>& groups, bool can_stall, bool& done,
                  lpb_profile& prof) {
    cudaStream_t s = h->stream;
    const int ce = h->opt.check_every;
    const int stall_checks = can_stall ? h->opt.polish_stall_checks : 0;
    lpb_err rc;
    done = false;
    while (g.live > 0) {
        const int L = (int)std::min<int64_t>(ce, g.max_iter - g.K);
        if ((rc = lane_interval<T>(h, ln, L, stall_checks, s, &prof)) != LPB_OK) return rc;
        CU(cudaStreamSynchronize(s));
        add_interval_times(h, L, &prof);
        if ((rc = lane_collect<T>(h, ln, groups, s, &prof, true)) != LPB_OK) return rc;
        if (can_stall && g.live > 0 && g.stalled) return LPB_OK;
    }
    done = true;
    return LPB_OK;
}

// Polish: group g, stalled on the handle's FP32 lane ln, continues from its
// FP32 state in double-float (or FP64) iterates on the polish lane, with its
// restart state (k, r0, w, ...) carried over.
lpb_err polish_group(lpb_ctx* h, Lane& ln, GroupRun& g, std::vector<GroupRun*>& groups, lpb_profile& prof) {
    cudaStream_t s = h->stream;
    const int pp = polish_dfloat(h) ? kPrecDfl : kPrecF64;
    Lane& pl = h->lane[pp];
    std::vector<GroupRun*> pgroups(1, nullptr);
    prof.kernels += 5;
    prof.fp64_switch_iter = g.K;
    bool done = true;
    lpb_err rc = lane_reserve(h, pl, pp, ln.cap, 1);
    if (rc == LPB_OK) {
        if (pp == kPrecDfl) {
            if ((rc = lane_migrate<dfloat>(h, ln, pl, g, 0, 0, s, groups)) == LPB_OK) {
                pgroups[0] = &g;
                rc = run_group<dfloat>(h, pl, g, pgroups, false, done, prof);
            }
        } else {
            if ((rc = lane_migrate<double>(h, ln, pl, g, 0, 0, s, groups)) == LPB_OK) {
                pgroups[0] = &g;
                rc = run_group<double>(h, pl, g, pgroups, false, done, prof);
            }
        }
    }
    if (rc != LPB_OK) {
        pl.ncol = 0;
        cudaMemsetAsync(pl.ctl, 0, sizeof(Control) * pl.gcap, s);
    }
    return rc;
}

// A batched solve: the batch is one restart group on the handle's lane of
// its precision; with polish, a stalled batch moves to the polish lane.
template <typename T>
lpb_err solve_impl(lpb_ctx* h, int num_lps, const lpb_lp_spec* specs_dev, double tol, int64_t max_iter,
                   const double* wx, const double* wy, lpb_batch* bt) {
    lpb_err rc;
    cudaStream_t s = h->stream;
    const int n = h->n, m = h->m;
    Lane& ln = h->lane[prec_of<T>()];
    if ((rc = lane_reserve(h, ln, prec_of<T>(), num_lps, 1)) != LPB_OK) return rc;
    if ((rc = ensure_check_ws(h, ln.cap)) != LPB_OK) return rc;
    if ((rc = ensure_events(h)) != LPB_OK) return rc;
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
    GroupRun g;
    g.id = 0;
    g.count = num_lps;
    g.slot0 = 0;
    g.max_iter = max_iter;
    g.res = bt->res.data();
    g.x_dev = bt->x;
    g.y_dev = bt->y;
    std::vector<GroupRun*> groups(1, nullptr);
    prof.kernels += 3;
    rc = lane_admit<T>(h, ln, g, specs_dev, wx, wy, n, m, tol, s, groups);
    bool done = true;
    const bool can_stall = std::is_same<T, float>::value && polish_enabled(h);
    if (rc == LPB_OK && g.live > 0) rc = run_group<T>(h, ln, g, groups, can_stall, done, prof);
    if (rc == LPB_OK && !done) rc = polish_group(h, ln, g, groups, prof);
    if (rc != LPB_OK) {
        // leave the lane empty for the next solve
        ln.ncol = 0;
        std::fill(ln.slot_used.begin(), ln.slot_used.end(), 0);
        cudaMemsetAsync(ln.ctl, 0, sizeof(Control) * ln.gcap, s);
        cudaStreamSynchronize(s);
        return rc;
    }
    CU(cudaStreamSynchronize(s));
    return LPB_OK;
}

// Joint intervals over the lanes of precision prec of the handles idx, on
// stream s, until each of their groups is done or (can_stall) has stalled.
// Groups whose next interval has the same length share one joint interval;
// near the iteration cap, groups that reached it from different iteration
// counts need intervals of different lengths.  So every group runs the
// intervals it would run alone.
template <typename T>
lpb_err joint_loop(const std::vector<lpb_ctx*>& hs, int prec, std::vector<GroupRun>& g,
                   std::vector<std::vector<GroupRun*>>& groups, std::vector<lpb_batch*>& bts,
                   const std::vector<char>& can_stall, const std::vector<int>& idx, int64_t max_iter,
                   cudaStream_t s) {
    std::map<int, JointGraph> graphs;  // by interval length
    std::vector<int> act, len, lens;
    std::vector<lpb_ctx*> ah;
    std::vector<Lane*> al;
    std::vector<int> sc;
    std::vector<lpb_profile*> ap;
    lpb_err rc = LPB_OK;
    while (rc == LPB_OK) {
        act.clear();
        len.clear();
        for (int i : idx)
            if (g[i].live > 0 && !(can_stall[i] && g[i].stalled)) {
                act.push_back(i);
                len.push_back((int)std::min<int64_t>(hs[i]->opt.check_every, max_iter - g[i].K));
            }
        if (act.empty()) break;
        lens = len;
        std::sort(lens.begin(), lens.end());
        lens.erase(std::unique(lens.begin(), lens.end()), lens.end());
        for (int L : lens) {
            ah.clear();
            al.clear();
            sc.clear();
            ap.clear();
            for (size_t a = 0; a < act.size(); ++a)
                if (len[a] == L) {
                    const int i = act[a];
                    ah.push_back(hs[i]);
                    al.push_back(&hs[i]->lane[prec]);
                    sc.push_back(can_stall[i] ? hs[i]->opt.polish_stall_checks : 0);
                    ap.push_back(&bts[i]->prof);
                }
            if ((rc = joint_interval<T>(ah.data(), al.data(), sc.data(), (int)ah.size(), L, s, graphs[L], ap.data())) !=
                LPB_OK)
                break;
        }
        if (rc != LPB_OK) break;
        const cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "joint solve: interval");
            break;
        }
        for (int i : act)
            if ((rc = lane_collect<T>(hs[i], hs[i]->lane[prec], groups[i], s, &bts[i]->prof, true)) != LPB_OK) break;
    }
    for (auto& kv : graphs) joint_graph_free(kv.second);
    return rc;
}

// Joint polish: the groups idx, stalled on their handles' FP32 lanes, move to
// the polish lanes (iterate type TD) with their restart state (k, r0, w, ...)
// and continue together in joint intervals, as polish_group runs each alone.
template <typename TD>
lpb_err polish_joint(const std::vector<lpb_ctx*>& hs, std::vector<GroupRun>& g,
                     std::vector<std::vector<GroupRun*>>& groups, std::vector<lpb_batch*>& bts,
                     const std::vector<int>& idx, int64_t max_iter, cudaStream_t s) {
    constexpr int pp = std::is_same<TD, dfloat>::value ? kPrecDfl : kPrecF64;
    const int count = (int)hs.size();
    std::vector<std::vector<GroupRun*>> pg(count, std::vector<GroupRun*>(1, nullptr));
    const std::vector<char> no_stall(count, 0);
    std::vector<int> moved;
    lpb_err rc = LPB_OK;
    for (int i : idx) {
        lpb_ctx* h = hs[i];
        Lane& ln = h->lane[kPrecF32];
        Lane& pl = h->lane[pp];
        bts[i]->prof.kernels += 5;
        bts[i]->prof.fp64_switch_iter = g[i].K;
        if ((rc = lane_reserve(h, pl, pp, ln.cap, 1)) != LPB_OK) break;
        moved.push_back(i);
        if ((rc = lane_migrate<TD>(h, ln, pl, g[i], 0, 0, s, groups[i])) != LPB_OK) break;
        pg[i][0] = &g[i];
    }
    if (rc == LPB_OK) rc = joint_loop<TD>(hs, pp, g, pg, bts, no_stall, moved, max_iter, s);
    if (rc != LPB_OK)
        for (int i : moved) {
            Lane& pl = hs[i]->lane[pp];
            pl.ncol = 0;
            cudaMemsetAsync(pl.ctl, 0, sizeof(Control) * pl.gcap, s);
        }
    return rc;
}

// A joint solve: batch i is one restart group on the lane of handle hs[i]
// (specs_dev[i] on that handle's device memory).  The lanes step together,
// one joint interval after another on the first handle's stream, until
// every batch is done or has stalled at FP32 resolution; the stalled
// batches then polish together on their handles' polish lanes.
template <typename T>
lpb_err solve_joint_impl(const std::vector<lpb_ctx*>& hs, const int32_t* num_lps,
                         const std::vector<const lpb_lp_spec*>& specs_dev, double tol, int64_t max_iter,
                         std::vector<lpb_batch*>& bts) {
    const int count = (int)hs.size(), prec = prec_of<T>();
    cudaStream_t s = hs[0]->stream;
    std::vector<GroupRun> g(count);
    std::vector<std::vector<GroupRun*>> groups(count, std::vector<GroupRun*>(1, nullptr));
    std::vector<char> can_stall(count, 0), admitted(count, 0);
    lpb_err rc = LPB_OK;
    for (int i = 0; i < count && rc == LPB_OK; ++i) {
        lpb_ctx* h = hs[i];
        Lane& ln = h->lane[prec];
        lpb_batch* bt = bts[i];
        const int nl = num_lps[i], n = h->n, m = h->m;
        if ((rc = lane_reserve(h, ln, prec, nl, 1)) != LPB_OK) break;
        if ((rc = ensure_check_ws(h, ln.cap)) != LPB_OK) break;
        cudaError_t e = cudaMalloc((void**)&bt->x, sizeof(double) * (size_t)n * (nl ? nl : 1));
        if (e == cudaSuccess) e = cudaMalloc((void**)&bt->y, sizeof(double) * (size_t)(m ? m : 1) * (nl ? nl : 1));
        if (e == cudaSuccess) e = cudaMemsetAsync(bt->x, 0, sizeof(double) * (size_t)n * nl, h->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(bt->y, 0, sizeof(double) * (size_t)m * nl, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "joint solve: result buffers");
            break;
        }
        bt->res.assign(nl, lpb_lp_result{});
        bt->prof.setup_ms = h->setup_ms;
        bt->prof.fp64_switch_iter = -1;
        if (nl == 0) continue;
        GroupRun& gi = g[i];
        gi.id = 0;
        gi.count = nl;
        gi.slot0 = 0;
        gi.max_iter = max_iter;
        gi.res = bt->res.data();
        gi.x_dev = bt->x;
        gi.y_dev = bt->y;
        bt->prof.kernels += 3;
        admitted[i] = 1;
        rc = lane_admit<T>(h, ln, gi, specs_dev[i], nullptr, nullptr, n, m, tol, h->stream, groups[i]);
        can_stall[i] = std::is_same<T, float>::value && polish_enabled(h);
    }
    std::vector<int> all;
    for (int i = 0; i < count; ++i) all.push_back(i);
    if (rc == LPB_OK) rc = joint_loop<T>(hs, prec, g, groups, bts, can_stall, all, max_iter, s);
    if (rc == LPB_OK) {
        const cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_fail(e, "joint solve");
    }
    if (rc == LPB_OK && std::is_same<T, float>::value) {
        // the batches still live have stalled: polish, by polish arithmetic
        std::vector<int> dfl, f64;
        for (int i = 0; i < count; ++i)
            if (g[i].live > 0) (polish_dfloat(hs[i]) ? dfl : f64).push_back(i);
        if (!dfl.empty()) rc = polish_joint<dfloat>(hs, g, groups, bts, dfl, max_iter, s);
        if (rc == LPB_OK && !f64.empty()) rc = polish_joint<double>(hs, g, groups, bts, f64, max_iter, s);
    }
    for (int i = 0; i < count; ++i) {
        lpb_ctx* h = hs[i];
        Lane& ln = h->lane[prec];
        if (rc != LPB_OK && admitted[i]) {
            // leave the lane empty for the next solve
            ln.ncol = 0;
            std::fill(ln.slot_used.begin(), ln.slot_used.end(), 0);
            cudaMemsetAsync(ln.ctl, 0, sizeof(Control) * ln.gcap, h->stream);
        }
        const cudaError_t e = cudaStreamSynchronize(h->stream);
        if (rc == LPB_OK && e != cudaSuccess) rc = cuda_fail(e, "joint solve");
    }
    if (rc == LPB_OK) {
        const cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_fail(e, "joint solve");
    }
    return rc;
}

// Times R plain iterations (no check) of `count` copies of the base LP on the
// handle's lane of its precision: per-iteration microseconds of the primal and
// dual steps (medians over the iterations).
template <typename T>
lpb_err time_steps(lpb_ctx* h, int count, int R, double* us_primal, double* us_dual) {
    lpb_err rc;
    cudaStream_t s = h->stream;
    Lane& ln = h->lane[prec_of<T>()];
    if ((rc = lane_reserve(h, ln, prec_of<T>(), count, 1)) != LPB_OK) return rc;
    if ((rc = ensure_check_ws(h, ln.cap)) != LPB_OK) return rc;
    if ((rc = ensure_specs(h, count)) != LPB_OK) return rc;
    std::vector<lpb_lp_spec> sp(count);
    for (auto& q : sp) {
        q.kind = 0;
        q.var = -1;
        q.lo = -HUGE_VAL;
        q.hi = HUGE_VAL;
        q.sign = 1.0;
    }
    CU(cudaMemcpyAsync(h->specs_dev, sp.data(), sizeof(lpb_lp_spec) * count, cudaMemcpyHostToDevice, s));
    std::vector<lpb_lp_result> res(count);
    GroupRun g;
    g.id = 0;
    g.count = count;
    g.slot0 = 0;
    g.max_iter = 1 << 30;
    g.res = res.data();
    std::vector<GroupRun*> groups(1, nullptr);
    if ((rc = lane_admit<T>(h, ln, g, h->specs_dev, nullptr, nullptr, 0, 0, 1e-4, s, groups)) != LPB_OK) return rc;
    const IterData<T> id = lane_iter_data<T>(h, ln);
    const IterBufs<T> ib = lane_iter_bufs<T>(ln);
    const T* hal = lane_hal<T>(ln);
    cudaEvent_t ev[3];
    for (auto& e : ev) CU(cudaEventCreate(&e));
    std::vector<float> tp, td;
    cudaError_t ce = cudaSuccess;
    for (int t = 0; t < R + 2 && ce == cudaSuccess; ++t) {
        ce = launch_iteration<T>(id, ib, ln.cap, ln.ncol, hal, t % h->opt.check_every, h->opt.check_every, 0, false,
                                 false, s, ev);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
        float a = 0.f, b = 0.f;
        if (ce == cudaSuccess && t >= 2) {
            cudaEventElapsedTime(&a, ev[0], ev[1]);
            cudaEventElapsedTime(&b, ev[1], ev[2]);
            tp.push_back(a);
            td.push_back(b);
        }
    }
    for (auto& e : ev) cudaEventDestroy(e);
    // leave the lane empty
    ln.ncol = 0;
    std::fill(ln.slot_used.begin(), ln.slot_used.end(), 0);
    std::fill(ln.col_group.begin(), ln.col_group.end(), -1);
    cudaMemsetAsync(ln.ctl, 0, sizeof(Control) * ln.gcap, s);
    cudaStreamSynchronize(s);
    if (ce != cudaSuccess) return cuda_fail(ce, "timed steps");
    std::sort(tp.begin(), tp.end());
    std::sort(td.begin(), td.end());
    *us_primal = 1e3 * tp[tp.size() / 2];
    *us_dual = 1e3 * td[td.size() / 2];
    return LPB_OK;
}

lpb_err time_steps_any(lpb_ctx* h, int count, int R, double* up, double* ud) {
    return h->opt.precision == LPB_MIXED ? time_steps<float>(h, count, R, up, ud)
                                         : time_steps<double>(h, count, R, up, ud);
}

lpb_err apply_shape(lpb_ctx* h, Csr& c, int thr, int shift) {
    if (c.long_thr != thr) {
        c.long_thr = thr;
        CU(build_long_rows(c, h->stream));
        // the segment scratch follows the new long-row lists
        lpb_err rc = ensure_long_scratch(h, std::max(h->lr_cap, h->ws_cap), true);
        if (rc != LPB_OK) return rc;
    }
    c.g_shift = shift;
    h->ws_epoch += 1;  // captured intervals hold the old launch shapes
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

// host override records: kinds, variable indices, bounds and signs
lpb_err check_specs(const lpb_ctx* h, int32_t num_lps, const lpb_lp_spec* specs) {
    for (int32_t q = 0; q < num_lps; ++q) {
        const lpb_lp_spec& sp = specs[q];
        if (sp.kind < 0 || sp.kind > 2) return fail(LPB_ERR_INVALID_ARG, "override kind must be 0, 1 or 2");
        if (sp.kind != 0 && (sp.var < 0 || sp.var >= h->n))
            return fail(LPB_ERR_BAD_INDEX, "an override names a variable outside [0, n)");
        if (sp.kind == 1 && (std::isnan(sp.lo) || std::isnan(sp.hi)))
            return fail(LPB_ERR_INVALID_ARG, "NaN override bound");
        if (sp.kind == 2 && !std::isfinite(sp.sign)) return fail(LPB_ERR_INVALID_ARG, "non-finite objective sign");
    }
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
    o->polish_arith = LPB_POLISH_DFLOAT;
    o->eps_dual = -1.0;
    o->use_graphs = 1;
    o->use_pdl = 1;
    o->stream_priority = 0;
    o->reduced_cost = LPB_RC_BARRIER;
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
    if (o.check_every < 1 || o.ruiz_iters < 0 || o.power_max_iter < 1 || (o.fp64_polish && o.polish_stall_checks < 1) ||
        (o.polish_arith != LPB_POLISH_DFLOAT && o.polish_arith != LPB_POLISH_FP64) || !(o.power_tol >= 0.0) ||
        (o.reduced_cost != LPB_RC_BARRIER && o.reduced_cost != LPB_RC_ROBUST) ||
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
            int lo = 0, hi = 0;  // least and greatest priority
            CU(cudaDeviceGetStreamPriorityRange(&lo, &hi));
            const int pr = std::max(hi, std::min(lo, (int)o.stream_priority));
            CU(cudaStreamCreateWithPriority(&h->stream, cudaStreamNonBlocking, pr));
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
        if (polish_dfloat(h)) {
            // the scaled data as dfloat pairs for a double-float polish phase
            CU(dmalloc(F, &h->a_dfl, sizeof(dfloat) * nnz));
            CU(dmalloc(F, &h->at_dfl, sizeof(dfloat) * nnz));
            dfloat** nv[] = {&h->cs_dfl, &h->xls_dfl, &h->xus_dfl};
            for (dfloat** p : nv) CU(dmalloc(F, p, sizeof(dfloat) * n));
            dfloat** mv[] = {&h->ls_dfl, &h->us_dfl};
            for (dfloat** p : mv) CU(dmalloc(F, p, sizeof(dfloat) * mm));
            CU(split_df(h->A.v64, (df*)h->a_dfl, (int)nnz, false, s));
            CU(split_df(h->At.v64, (df*)h->at_dfl, (int)nnz, false, s));
            CU(split_df(h->cs, (df*)h->cs_dfl, n, false, s));
            CU(split_df(h->xls, (df*)h->xls_dfl, n, false, s));
            CU(split_df(h->xus, (df*)h->xus_dfl, n, false, s));
            CU(split_df(h->ls, (df*)h->ls_dfl, m, false, s));
            CU(split_df(h->us, (df*)h->us_dfl, m, false, s));
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
        const size_t wn = power_work_doubles(m, n, nnz, o.power_max_iter);
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
    if ((rc = check_specs(h, num_lps, specs)) != LPB_OK) return rc;
    DeviceGuard guard(h->device);
    if ((rc = ensure_specs(h, num_lps)) != LPB_OK) return rc;
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

lpb_err lpb_solve_multi(int32_t count, const lpb_handle* handles, const int32_t* num_lps,
                        const lpb_lp_spec* const* specs, double tol, int64_t max_iter, lpb_batch_t* out) {
    if (!handles || !num_lps || !specs || !out) return fail(LPB_ERR_INVALID_ARG, "null argument");
    if (count < 1 || count > LPB_MAX_JOINT) return fail(LPB_ERR_INVALID_ARG, "count must be in [1, LPB_MAX_JOINT]");
    for (int32_t i = 0; i < count; ++i) out[i] = nullptr;
    std::vector<lpb_ctx*> hs(count);
    lpb_err rc;
    for (int32_t i = 0; i < count; ++i) {
        if ((rc = check_solve_args(handles[i], num_lps[i], specs[i], tol, max_iter, out + i)) != LPB_OK) return rc;
        hs[i] = handles[i];
        for (int32_t j = 0; j < i; ++j)
            if (hs[j] == hs[i]) return fail(LPB_ERR_INVALID_ARG, "a handle appears twice in a joint solve");
        if (hs[i]->device != hs[0]->device) return fail(LPB_ERR_INVALID_ARG, "joint solve handles on different devices");
        if (hs[i]->opt.precision != hs[0]->opt.precision)
            return fail(LPB_ERR_INVALID_ARG, "joint solve handles with different precisions");
        if (hs[i]->opt.check_every != hs[0]->opt.check_every)
            return fail(LPB_ERR_INVALID_ARG, "joint solve handles with different check_every");
        if ((rc = check_specs(hs[i], num_lps[i], specs[i])) != LPB_OK) return rc;
    }
    DeviceGuard guard(hs[0]->device);
    std::vector<const lpb_lp_spec*> sd(count, nullptr);
    for (int32_t i = 0; i < count; ++i) {
        if ((rc = ensure_specs(hs[i], num_lps[i])) != LPB_OK) return rc;
        if (num_lps[i] > 0)
            CU(cudaMemcpyAsync(hs[i]->specs_dev, specs[i], sizeof(lpb_lp_spec) * num_lps[i], cudaMemcpyHostToDevice,
                               hs[i]->stream));
        sd[i] = hs[i]->specs_dev;
    }
    std::vector<lpb_batch*> bts(count, nullptr);
    for (int32_t i = 0; i < count; ++i) {
        bts[i] = new (std::nothrow) lpb_batch();
        if (!bts[i]) {
            for (lpb_batch* b : bts) lpb_batch_free(b);
            return fail(LPB_ERR_OOM, "host allocation failed");
        }
        bts[i]->device = hs[i]->device;
        bts[i]->num_lps = num_lps[i];
        bts[i]->m = hs[i]->m;
        bts[i]->n = hs[i]->n;
    }
    rc = hs[0]->opt.precision == LPB_MIXED ? solve_joint_impl<float>(hs, num_lps, sd, tol, max_iter, bts)
                                           : solve_joint_impl<double>(hs, num_lps, sd, tol, max_iter, bts);
    if (rc != LPB_OK) {
        for (lpb_batch* b : bts) lpb_batch_free(b);
        return rc;
    }
    for (int32_t i = 0; i < count; ++i) out[i] = bts[i];
    return LPB_OK;
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

lpb_err lpb_obbt_tighten(lpb_batch_t b, const lpb_lp_spec* specs, const double* var_lo, const double* var_hi,
                         double min_gain, double* new_lo, double* new_hi, int32_t* updated) {
    if (!b || !var_lo || !var_hi || !new_lo || !new_hi || (b->num_lps > 0 && !specs))
        return fail(LPB_ERR_INVALID_ARG, "null argument");
    if (!(min_gain >= 0.0)) return fail(LPB_ERR_INVALID_ARG, "min_gain must be >= 0");
    const int n = b->n;
    for (int j = 0; j < n; ++j) {
        new_lo[j] = var_lo[j];
        new_hi[j] = var_hi[j];
    }
    int32_t cnt = 0;
    for (int q = 0; q < b->num_lps; ++q) {
        const lpb_lp_spec& sp = specs[q];
        const lpb_lp_result& r = b->res[q];
        if (sp.kind != 2 || r.status != LPB_OPTIMAL || !std::isfinite(r.safe_bound)) continue;
        if (sp.var < 0 || sp.var >= n) return fail(LPB_ERR_BAD_INDEX, "an override names a variable outside [0, n)");
        const int j = sp.var;
        if (sp.sign > 0.0) {
            // min x_j >= safe_bound / sign
            const double cand = r.safe_bound / sp.sign;
            if (cand > new_lo[j] + min_gain && cand <= var_hi[j]) {
                new_lo[j] = cand;
                ++cnt;
            }
        } else if (sp.sign < 0.0) {
            // min sign x_j >= safe_bound, so x_j <= safe_bound / sign
            const double cand = r.safe_bound / sp.sign;
            if (cand < new_hi[j] - min_gain && cand >= var_lo[j]) {
                new_hi[j] = cand;
                ++cnt;
            }
        }
    }
    if (updated) *updated = cnt;
    return LPB_OK;
}

lpb_err lpb_get_tuning(lpb_handle h, lpb_tuning* t) {
    if (!h || !t) return fail(LPB_ERR_INVALID_ARG, "null argument");
    t->long_row_primal = h->At.long_thr;
    t->long_row_dual = h->A.long_thr;
    t->lane_shift_primal = h->At.g_shift;
    t->lane_shift_dual = h->A.g_shift;
    return LPB_OK;
}

lpb_err lpb_set_tuning(lpb_handle h, const lpb_tuning* t) {
    if (!h || !t) return fail(LPB_ERR_INVALID_ARG, "null argument");
    if (t->long_row_primal < 1 || t->long_row_dual < 1 || t->lane_shift_primal < 0 || t->lane_shift_primal > 5 ||
        t->lane_shift_dual < 0 || t->lane_shift_dual > 5)
        return fail(LPB_ERR_INVALID_ARG, "thresholds must be >= 1 and shifts in [0, 5]");
    DeviceGuard guard(h->device);
    lpb_err rc;
    if ((rc = apply_shape(h, h->At, t->long_row_primal, t->lane_shift_primal)) != LPB_OK) return rc;
    if ((rc = apply_shape(h, h->A, t->long_row_dual, t->lane_shift_dual)) != LPB_OK) return rc;
    CU(cudaStreamSynchronize(h->stream));
    return LPB_OK;
}

lpb_err lpb_autotune(lpb_handle h, int32_t num_lps, lpb_tuning* chosen) {
    if (!h) return fail(LPB_ERR_INVALID_ARG, "null handle");
    if (num_lps < 1 || num_lps > 65536) return fail(LPB_ERR_INVALID_ARG, "num_lps must be in [1, 65536]");
    DeviceGuard guard(h->device);
    const int thrs[] = {8, 16, 32, 64, 128, 256};
    double best_p = 1e300, best_d = 1e300;
    int bp_thr = h->At.long_thr, bp_sh = h->At.g_shift, bd_thr = h->A.long_thr, bd_sh = h->A.g_shift;
    lpb_err rc;
    for (int thr : thrs) {
        for (int sh = 0; sh <= 4; ++sh) {
            // both steps take the candidate; each step keeps its own best
            if ((rc = apply_shape(h, h->At, thr, sh)) != LPB_OK) return rc;
            if ((rc = apply_shape(h, h->A, thr, sh)) != LPB_OK) return rc;
            double up = 0.0, ud = 0.0;
            if ((rc = time_steps_any(h, num_lps, 9, &up, &ud)) != LPB_OK) return rc;
            if (up < best_p) {
                best_p = up;
                bp_thr = thr;
                bp_sh = sh;
            }
            if (ud < best_d) {
                best_d = ud;
                bd_thr = thr;
                bd_sh = sh;
            }
        }
    }
    lpb_tuning t{bp_thr, bd_thr, bp_sh, bd_sh};
    if ((rc = lpb_set_tuning(h, &t)) != LPB_OK) return rc;
    if (chosen) *chosen = t;
    return LPB_OK;
}

lpb_err lpb_tune_batch(lpb_handle h, const int32_t* widths, int32_t count, double* us_per_iter, int32_t* best) {
    if (!h || !widths || !us_per_iter || count < 1) return fail(LPB_ERR_INVALID_ARG, "null argument or count < 1");
    for (int32_t i = 0; i < count; ++i)
        if (widths[i] < 1 || widths[i] > 65536) return fail(LPB_ERR_INVALID_ARG, "widths must be in [1, 65536]");
    DeviceGuard guard(h->device);
    double best_rate = -1.0;
    for (int32_t i = 0; i < count; ++i) {
        double up = 0.0, ud = 0.0;
        lpb_err rc = time_steps_any(h, widths[i], 9, &up, &ud);
        if (rc != LPB_OK) return rc;
        us_per_iter[i] = up + ud;
        const double rate = widths[i] / (up + ud);
        if (rate > best_rate) {
            best_rate = rate;
            if (best) *best = i;
        }
    }
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
    for (auto& ln : h->lane) lane_free(ln);
    free_list(h->ws_allocs);
    if (h->specs_dev) cudaFree(h->specs_dev);
    free_list(h->fixed_allocs);
    free_long_rows(h->A);
    free_long_rows(h->At);
    free_long_scratch(h);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

}  // extern "C"
