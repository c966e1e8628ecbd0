// lpb_engine.h -- the host side of the batched solver, shared by the batch
// entry points (lpb_api.cu) and the serving loop (lpb_serve.cu).
//
// A handle (lpb_ctx) owns one sparse A with its scalings and base vectors.
// Its active LPs live in lanes: a lane is a set of batch columns with
// iterates in one precision (FP32, FP64 or double-float), laid out row-major
// and batch-contiguous with leading dimension cap.  The LPs of a lane are
// partitioned into restart groups (Control on the device): the LPs of one
// batched solve, or of one served request, form one group and share its
// averaged restart test and Halpern index.  Groups are independent, so a
// lane can take in new groups while others are running (continuous
// batching) and a group's trajectory does not depend on its neighbours.
//
// One interval = L iterations of every column of a lane followed by a check;
// between intervals the host reads O(columns + groups) records, extracts and
// compacts finished columns, admits new groups and moves stalled groups to a
// polish lane.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "lpb_internal.h"

namespace lpb {

enum LanePrec { kPrecF32 = 0, kPrecF64 = 1, kPrecDfl = 2 };

// Everything an interval's captured graph bakes into its kernel and copy
// nodes: the shape (active columns, the single group if there is one,
// interval length, stall setting, iterate size), the lane's leading dimension
// and buffers (identified by their base addresses), the check workspace
// generation, and each matrix's long-row list and launch shape.  A replay is
// valid only while every field holds; any difference re-captures.
struct GraphKey {
    int ncol = -1, uni = -1, L = -1, stall = -1, ws_epoch = -1, tsize = 0;
    int ld = -1;
    const void* X = nullptr;            // lane iterate blocks (all allocated together): Xbar
    const void* Y = nullptr;
    const void* rec = nullptr;          // per-column records and their pinned mirror
    const void* rec_h = nullptr;
    const int* long_a = nullptr;        // long-row lists of A~ and A~^T
    const int* long_at = nullptr;
    const void* part = nullptr;         // long-row segment scratch
    int n_long_a = -1, n_long_at = -1, thr_a = -1, thr_at = -1, shift_a = -1, shift_at = -1;
    bool operator==(const GraphKey& o) const {
        return ncol == o.ncol && uni == o.uni && L == o.L && stall == o.stall && ws_epoch == o.ws_epoch &&
               tsize == o.tsize && ld == o.ld && X == o.X && Y == o.Y && rec == o.rec && rec_h == o.rec_h &&
               long_a == o.long_a && long_at == o.long_at && part == o.part && n_long_a == o.n_long_a &&
               n_long_at == o.n_long_at &&
               thr_a == o.thr_a && thr_at == o.thr_at && shift_a == o.shift_a && shift_at == o.shift_at;
    }
};

struct Lane {
    int prec = kPrecF32;
    int cap = 0;    // columns (= leading dimension of the iterate blocks)
    int gcap = 0;   // restart groups
    // device: iterate blocks and per-column parameters in the lane's precision
    void *X = nullptr, *X0 = nullptr, *Xbar = nullptr, *Xh = nullptr, *DX = nullptr;
    void *Y = nullptr, *Y0 = nullptr, *Yh = nullptr, *DY = nullptr, *DYp = nullptr;
    void *clo = nullptr, *chi = nullptr, *cc = nullptr, *ctau = nullptr, *csigma = nullptr;
    // device: per-column check data, per-group state, scratch
    int *ckind = nullptr, *cvar = nullptr, *cgrp = nullptr, *cslot = nullptr, *k_stall = nullptr;
    double *k_lo = nullptr, *k_hi = nullptr, *k_c = nullptr, *k_w = nullptr, *k_best = nullptr;
    ColRecord* rec = nullptr;
    Control* ctl = nullptr;
    int* flags = nullptr;
    double* hal64 = nullptr;
    float* hal32 = nullptr;
    dfloat* haldf = nullptr;
    double* rscr = nullptr;
    int* rtag = nullptr;
    int* mv = nullptr;          // 4 * cap ints of column moves
    double** optr = nullptr;    // 2 * cap output pointers of an extraction
    // host mirrors (pinned)
    ColRecord* rec_h = nullptr;
    Control* ctl_h = nullptr;
    int* mv_h = nullptr;
    double** optr_h = nullptr;
    std::vector<void*> allocs;
    // the interval as an executable CUDA graph, for the shape gkey
    cudaGraphExec_t exec = nullptr;
    GraphKey gkey;
    // host bookkeeping
    int ncol = 0;
    std::vector<int> col_group;     // column -> group id
    std::vector<int> col_lp;        // column -> LP index within its group
    std::vector<char> slot_used;    // residual slots in use
};

// Where a group's results go and how far it is.
struct GroupRun {
    int id = -1;                 // index into the lane's Control array
    int count = 0;               // LPs of the group
    int slot0 = 0;
    int live = 0;                // columns still active
    int64_t max_iter = 0;
    int64_t K = 0;               // iterations run (mirror of Control::K)
    bool stalled = false;
    lpb_lp_result* res = nullptr;   // count results
    double* x_dev = nullptr;        // n * count results (LP-major), or null
    double* y_dev = nullptr;        // m * count results, or null
    int64_t iter_offset = 0;        // iterations run in an earlier lane (polish)
};

}  // namespace lpb

struct lpb_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    lpb_options opt{};
    int m = 0, n = 0, nnz = 0;
    lpb::Csr A, At;
    double *d_r = nullptr, *d_c = nullptr;
    double *c = nullptr, *l = nullptr, *u = nullptr, *xl = nullptr, *xu = nullptr;
    double *cs = nullptr, *ls = nullptr, *us = nullptr, *xls = nullptr, *xus = nullptr;
    float *cs32 = nullptr, *ls32 = nullptr, *us32 = nullptr, *xls32 = nullptr, *xus32 = nullptr;
    // double-float copies for the checks of FP32 and dfloat iterates
    lpb::df *f_dr = nullptr, *f_dc = nullptr, *f_idr = nullptr, *f_idc = nullptr, *f_c = nullptr;
    lpb::df *f_xl = nullptr, *f_xu = nullptr, *f_l = nullptr, *f_u = nullptr;
    // dfloat copies of the scaled data for a double-float polish phase
    lpb::dfloat *a_dfl = nullptr, *at_dfl = nullptr, *cs_dfl = nullptr, *xls_dfl = nullptr, *xus_dfl = nullptr;
    lpb::dfloat *ls_dfl = nullptr, *us_dfl = nullptr;
    double eta = 0.0, norm_est = 0.0, c_norm_base = 0.0, b_norm = 0.0, setup_ms = 0.0;
    int power_iters = 0;
    std::vector<void*> fixed_allocs;
    // lanes of the batch entry points: [kPrecF32], [kPrecF64], [kPrecDfl]
    lpb::Lane lane[3];
    // check workspace shared by the handle's lanes (they run on one stream)
    int ws_cap = 0;
    int ws_epoch = 0;
    double *P = nullptr, *Q = nullptr, *partials = nullptr, *colsum = nullptr;
    // long-row segment scratch of the step kernels (A~ and A~^T share it)
    int lr_cap = 0;
    void* lr_part = nullptr;
    unsigned* lr_ticket = nullptr;
    lpb_lp_spec* specs_dev = nullptr;
    int specs_cap = 0;
    std::vector<void*> ws_allocs;
    std::vector<cudaEvent_t> events;
};

namespace lpb {

// error reporting shared by the host files: sets lpb_last_error()
lpb_err fail(lpb_err code, const std::string& msg);
lpb_err cuda_fail(cudaError_t e, const char* what);

#define LPB_CU(call)                                              \
    do {                                                          \
        cudaError_t _e = (call);                                  \
        if (_e != cudaSuccess) return ::lpb::cuda_fail(_e, #call); \
    } while (0)

bool polish_enabled(const lpb_ctx* h);
bool polish_dfloat(const lpb_ctx* h);

// (Re)allocates a lane for at least cap columns and gcap groups; only an
// empty lane is reallocated.
lpb_err lane_reserve(lpb_ctx* h, Lane& ln, int prec, int cap, int gcap);
void lane_free(Lane& ln);
// check workspace for a lane of cap columns, and room for count spec records
lpb_err ensure_check_ws(lpb_ctx* h, int cap);
// the step kernels' long-row segment scratch for lanes of up to cap columns
// (force: reallocate after the long-row lists changed)
lpb_err ensure_long_scratch(lpb_ctx* h, int cap, bool force);
void free_long_scratch(lpb_ctx* h);
lpb_err ensure_specs(lpb_ctx* h, int count);
// first free run of count residual slots, or -1
int lane_find_slots(const Lane& ln, int count);
// a free group id, or -1
int lane_free_group(const Lane& ln, const std::vector<GroupRun*>& groups);

CheckData lane_check_data(const lpb_ctx* h, const Lane& ln, int stall_checks);
template <typename T> IterData<T> lane_iter_data(const lpb_ctx* h, const Lane& ln);
template <typename T> IterBufs<T> lane_iter_bufs(const Lane& ln);
template <typename T> const T* lane_hal(const Lane& ln);

// Admits a group of g.count LPs at columns [ln.ncol, ln.ncol + count); LPs
// that are infeasible from their overrides alone finish at once.  Synchronizes.
template <typename T>
lpb_err lane_admit(lpb_ctx* h, Lane& ln, GroupRun& g, const lpb_lp_spec* specs_dev, const double* wx,
                   const double* wy, int64_t wsx, int64_t wsy, double tol, cudaStream_t s,
                   std::vector<GroupRun*>& groups);

// Launches L iterations of every active column of the lane and the check,
// then queues the copies of the per-column and per-group records.
template <typename T>
lpb_err lane_interval(lpb_ctx* h, Lane& ln, int L, int stall_checks, cudaStream_t s, lpb_profile* prof);

// A joint interval's executable graph and the interval keys of its lanes,
// in order, and the keys of the last interval run; owned by the joint solve.
struct JointGraph {
    cudaGraphExec_t exec = nullptr;
    std::vector<GraphKey> keys, seen;
};
void joint_graph_free(JointGraph& jg);

// One interval of the lanes lns[0 .. count) of several handles at once (one
// iterate type, the same check interval), all on stream s: L iterations
// whose primal and dual steps each run as one launch over every lane
// (launch_iteration_multi), then each lane's check and record copies.  With
// the first handle's use_graphs it is one CUDA graph in jg, replayed while
// every lane's interval key holds (captured once a shape has held for one
// interval).  Each lane's results are those of lane_interval on its own.
template <typename T>
lpb_err joint_interval(lpb_ctx* const* hs, Lane* const* lns, const int* stall_checks, int count, int L,
                       cudaStream_t s, JointGraph& jg, lpb_profile* const* profs);

// After the interval's stream work is done: statuses of the checked
// columns, results and extraction of the finished ones, compaction, group
// progress (K, stalls).  groups[id] is the host record of group id.
// idle: s has been synchronized since the lane's last interval, so no copy
// queued earlier still reads its pinned lists (saves two waits).
template <typename T>
lpb_err lane_collect(lpb_ctx* h, Lane& ln, std::vector<GroupRun*>& groups, cudaStream_t s, lpb_profile* prof,
                     bool idle = false);

// Moves group g (all of its live columns) from the FP32 lane src to the
// polish lane dst (precision TD), into columns [dst.ncol, ...) as group
// id_dst with slots from slot0_dst.  The group keeps its restart state.
template <typename TD>
lpb_err lane_migrate(lpb_ctx* h, Lane& src, Lane& dst, GroupRun& g, int id_dst, int slot0_dst, cudaStream_t s,
                     std::vector<GroupRun*>& src_groups);

// event timing of the profiled intervals
void add_interval_times(lpb_ctx* h, int L, lpb_profile* prof);

double step_bytes(int prec, int nnz, int m, int n, bool primal, bool check, int ncol);

// The key of an interval of L iterations on lane ln (see GraphKey).
inline GraphKey interval_key(const lpb_ctx* h, const Lane& ln, int L, int stall_checks, int uni, int tsize) {
    GraphKey k;
    k.ncol = ln.ncol;
    k.uni = uni;
    k.L = L;
    k.stall = stall_checks;
    k.ws_epoch = h->ws_epoch;
    k.tsize = tsize;
    k.ld = ln.cap;
    k.X = ln.Xbar;
    k.Y = ln.Y;
    k.rec = ln.rec;
    k.rec_h = ln.rec_h;
    k.long_a = h->A.long_rows;
    k.long_at = h->At.long_rows;
    k.part = h->lr_part;
    k.n_long_a = h->A.n_long;
    k.n_long_at = h->At.n_long;
    k.thr_a = h->A.long_thr;
    k.thr_at = h->At.long_thr;
    k.shift_a = h->A.g_shift;
    k.shift_at = h->At.g_shift;
    return k;
}

}  // namespace lpb
