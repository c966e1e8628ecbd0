// lpb_internal.h -- device data layout and kernel launchers shared by the
// library's translation units (setup, iteration, check, C ABI).
//
// Layout in HBM (one handle):
//   A~ and A~^T as CSR with int32 row pointers and column indices; values in
//   FP64 (checks, FP64 path) and, for the mixed path, FP32.
//   Iterate blocks are row-major with the batch contiguous: element (i, j) of
//   an n x N block lives at i * ld + j, ld = capacity rounded up to 4, so a
//   row of the batch is one contiguous, 16-byte aligned vector that a CSR
//   gather reads with 128-bit loads.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lpb.h"
#include "lpb_df.h"

namespace lpb {

#ifndef LPB_BLOCK
#define LPB_BLOCK 128
#endif
#ifndef LPB_LONG_ROW
#define LPB_LONG_ROW 32
#endif
constexpr int kBlock = LPB_BLOCK;     // threads of every iteration / SpMM block
constexpr int kLongRow = LPB_LONG_ROW; // rows with more nonzeros get a whole block
constexpr int kReduceRows = 8;     // rows per step of a reduction block (blockDim.y)
#ifndef LPB_REDUCE_BLOCKS
#define LPB_REDUCE_BLOCKS 304
#endif
constexpr int kReduceBlocks = LPB_REDUCE_BLOCKS; // reduction blocks per column tile (fixed: the sum order)
constexpr int kNumStats = 18;      // per-column partial sums of a check

// per-column statistics produced by a check (indices into the stats arrays)
enum Stat {
    // from the m rows
    S_PRES2 = 0,  // ||Ax - Pi(Ax)||^2 (original space)
    S_AX2,        // ||Ax||^2
    S_PHY,        // phi_[l,u](y)
    S_DY2,        // ||y^ - y||^2 (scaled)
    S_CROSS,      // <y^ - y, A~ (x^ - x)> (scaled)
    S_DY02,       // ||y^ - y0||^2 (scaled)
    S_PHIDY,      // phi_[l,u](dy), dy = Pi_B(D_r (y^ - y))
    S_RA2,        // ||A dx - Pi_R(A dx)||^2
    // from the n rows
    S_DRES2,      // ||c + A^T y + r||^2
    S_C2,         // ||c||^2
    S_CTX,        // c^T x
    S_PHR,        // phi_[xlo,xhi](r)
    S_DX2,        // ||x^ - x||^2 (scaled)
    S_DX02,       // ||x^ - x0||^2 (scaled)
    S_PHIDR,      // phi_[xlo,xhi](dr)
    S_RES2,       // ||A^T dy + dr||^2
    S_CDX,        // c^T dx
    S_RX2         // ||dx - Pi_R(dx)||^2
};

struct Csr {
    int rows = 0, cols = 0, nnz = 0;
    int* rp = nullptr;          // rows + 1
    int* ci = nullptr;          // nnz
    double* v64 = nullptr;      // scaled values, FP64
    float* v32 = nullptr;       // scaled values, FP32 (mixed path)
    float* v32lo = nullptr;     // v64 - v32 rounded to FP32: (v32, v32lo) is v64 in double-float
    int* long_rows = nullptr;   // rows with > long_thr entries
    int n_long = 0;
    int long_thr = kLongRow;    // rows longer than this get a whole block (tunable)
    int g_shift = 0;            // step kernels use (lanes per row from the batch width) >> g_shift
    // Step kernels cut a long row into segments of at most kStepSeg entries,
    // one block each, listed segment-major (every row's segment 0, then every
    // row's segment 1, ...) so that the blocks running together gather from
    // the same range of columns.  lseg[2 b], lseg[2 b + 1]: the long row
    // (index into long_rows) and segment of block b; the segments of long row
    // i are lseg0[i] .. lseg0[i + 1] - 1 in the partial-sum scratch.
    int* lseg = nullptr;
    int* lseg0 = nullptr;
    int n_lblocks = 0;
    // partial sums of multi-segment rows, [segment][ld] in the iterate type,
    // and one completion ticket per (long row, column tile), tile stride ntix
    void* part = nullptr;
    unsigned* ticket = nullptr;
    int ntix = 0;
};

#ifndef LPB_LONG_SEG
#define LPB_LONG_SEG 1024
#endif
constexpr int kLongSeg = LPB_LONG_SEG;  // rows longer than this get a block in the power iteration
// Entries per segment of a long row in the step kernels.  Segments are
// listed segment-major, so the blocks resident together gather from a
// window of columns about (resident blocks / long rows) segments wide: with
// 256 entries that window of the gathered block fits in L2 on the large
// strong-branching batch (500 rows of 10k entries), where 1024-entry
// segments span twice the L2 (dual step 878 -> 844 ms per solve on GB300;
// 512: 858 ms; 128: 889 ms, more blocks and partial sums).
#ifndef LPB_STEP_SEG
#define LPB_STEP_SEG 256
#endif
constexpr int kStepSeg = LPB_STEP_SEG;

// Per-column parameters of the iteration kernels (structure of arrays,
// length >= ld, in the iterate precision T).
template <typename T>
struct ColParams {
    int* kind;   // override kind
    int* var;    // override variable (or -1)
    int* grp;    // restart group of the column (its Halpern weights)
    T* lo;       // kind 1: scaled box of var (intersected with the base box)
    T* hi;
    T* c;        // kind 2: scaled objective coefficient of var
    T* tau;      // primal step eta / w
    T* sigma;    // dual step eta * w
};

// Per-column data for the FP64 checks, original units.
struct ColCheck {
    int* kind;
    int* var;
    double* lo;   // kind 1: original box of var (intersected)
    double* hi;
    double* c;    // kind 2: sign
    double* w;    // primal weight
    int* grp;     // restart group of the column
    int* slot;    // the LP's slot in its group's range of the residual scratch
    double* best; // smallest KKT error seen since the last halving (stall test)
    int* stall;   // checks since the KKT error last halved
};

// One column's outcome of a check, copied to the host.
struct ColRecord {
    int status;   // -1 still active, else lpb_lp_status
    int pad;
    double r;     // fixed-point residual (scaled, M-norm)
    double obj, dual_obj, rel_primal, rel_dual, rel_gap;
    double safe;  // dual_obj - tol (1 + |obj| + |dual_obj|)
};

// State of one restart group on the device.  A group is the set of LPs
// solved as one batch in the sense of Sec. 5: they share the batch-averaged
// restart test and the Halpern index k.  A lane (the active columns of one
// handle in one iterate precision) holds any number of groups side by side;
// a plain batched solve is one group.
struct Control {
    int k;            // inner index of the group's next iteration
    int restart;      // 1 if the last check restarted the group
    int error;        // device-side admission flags (LPB_ERR_*)
    int stalled;      // 1 if an active LP of the group stalled at the last check
    double r0;        // residual at the start of the epoch (< 0: unset)
    double r_prev;    // residual at the previous check
    double r_avg;     // averaged residual of the last check
    int64_t restarts;
    int64_t K;        // iterations the group has run
    int64_t max_iter;
    double tol, eps_inf, tol_dual;
    int slot0, nslots;  // the group's LPs own residual slots [slot0, slot0 + nslots)
    int active;
    int pad;
};

// records the message lpb_last_error() returns on this thread (lpb_api.cu)
void set_last_error(const char* msg);

// ---------------------------------------------------------------------------
// setup (lpb_setup.cu)
// ---------------------------------------------------------------------------
cudaError_t transpose_csr(const Csr& a, const double* a_vals, Csr& at, int* perm_out, cudaStream_t s);
cudaError_t exclusive_scan_i32(const int* in, int* out, int count, int* total_dev, cudaStream_t s);
// (re)builds a.long_rows and the step kernels' segments for threshold
// a.long_thr (frees an old list); free_long_rows releases them
cudaError_t build_long_rows(Csr& a, cudaStream_t s);
void free_long_rows(Csr& a);
cudaError_t ruiz_pock_chambolle(const Csr& a, const double* a_vals, const Csr& at, const double* at_vals,
                                int ruiz_iters, int pock_chambolle, double* d_r, double* d_c,
                                double* tmp_r, double* tmp_c, cudaStream_t s);
cudaError_t scale_values(const Csr& a, const double* a_vals, const double* d_r, const double* d_c,
                         bool rows_are_constraints, double* out64, float* out32, cudaStream_t s);
// doubles of device work space power_norm needs for an m x n matrix of nnz entries
size_t power_work_doubles(int m, int n, long long nnz, int max_iter);
cudaError_t power_norm(const Csr& a, const Csr& at, int max_iter, double tol, uint64_t seed,
                       double* work, double* est_out, int* iters_out, cudaStream_t s);
cudaError_t scale_vectors(int m, int n, const double* d_r, const double* d_c, const double* c,
                          const double* l, const double* u, const double* xl, const double* xu,
                          double* cs, double* ls, double* us, double* xls, double* xus, cudaStream_t s);
cudaError_t sq_norm(const double* v, int count, double* out_dev, cudaStream_t s);
cudaError_t rhs_norm2(const double* ls, const double* us, int m, double* out_dev, cudaStream_t s);
cudaError_t convert_f32(const double* in, float* out, int count, cudaStream_t s);
// out[i] = in[i] (or 1 / in[i] when recip) as a double-float pair
cudaError_t split_df(const double* in, df* out, int count, bool recip, cudaStream_t s);
// lo[e] = v64[e] - (double)v32[e] rounded to FP32
cudaError_t split_lo(const double* v64, const float* v32, float* lo, int count, cudaStream_t s);

// ---------------------------------------------------------------------------
// iteration (lpb_iter.cu)
// ---------------------------------------------------------------------------
template <typename T>
struct IterBufs {
    T *X, *X0, *Xbar, *Y, *Y0;         // state
    T *Xh, *DX, *G, *Yh, *DY, *DYp;    // written on check iterations
};

template <typename T>
struct IterData {
    Csr A, At;                 // scaled CSRs (values in T taken from v64 / v32)
    const T* a_vals;
    const T* at_vals;
    const T *c, *xl, *xu;      // scaled base vectors (n)
    const T *l, *u;            // scaled row bounds (m)
    ColParams<T> col;
};

// One reflected-Halpern PDHG iteration on columns [0, ncol): primal step
// (A~^T Y fused with the box projection, reflection and Halpern update) then
// dual step (A~ Xbar fused with the row projection and Halpern update).
// hal[2 (g (ce + 1) + e)], hal[2 (g (ce + 1) + e) + 1] are the Halpern
// weights (k+1)/(k+2), 1/(k+2) of Eq. mainiter for k = k_start - 1 + e of
// restart group g (ce = check_every), written on the device by the checks;
// iteration t of the interval takes entry t + 1 and rebuilds its iterate
// from entry t.  uni >= 0 says that every active column belongs to group
// uni.  With pdl the step kernels after the interval's first are
// programmatic dependents of their predecessor (not with timing events,
// which sit between them).
template <typename T>
cudaError_t launch_iteration(const IterData<T>& d, const IterBufs<T>& b, int ld, int ncol,
                             const T* hal, int t, int ce, int uni, bool check, bool pdl, cudaStream_t s,
                             cudaEvent_t* ev /* 3 events or nullptr */);

// One matrix's share of a joint iteration: its operator and iterate blocks,
// the lane's leading dimension, active columns, check interval, single group
// (or -1) and Halpern table, as launch_iteration takes them.
template <typename T>
struct IterPart {
    IterData<T> d;
    IterBufs<T> b;
    int ld, ncol, ce, uni;
    const T* hal;
};

// Matrices per joint step launch.
constexpr int kMaxParts = 8;

// Iteration t of the intervals of several matrices at once: the primal steps
// of all parts in one launch, then their dual steps in one launch (one per
// row-group width among the parts, and per kMaxParts parts).  Each part gets
// exactly what launch_iteration gives it alone: its rows are taken by other
// blocks, but each row by one row group of the same width, summing in the
// same order.  With pdl, as in launch_iteration.
template <typename T>
cudaError_t launch_iteration_multi(const IterPart<T>* parts, int nparts, int t, bool check, bool pdl,
                                   cudaStream_t s);

// ---------------------------------------------------------------------------
// checks (lpb_check.cu)
// ---------------------------------------------------------------------------
struct CheckData {
    Csr A, At;                     // FP64 values in v64
    int m, n;
    const double *d_r, *d_c;
    const double *c, *xl, *xu;     // original base vectors (n)
    const double *l, *u;           // original row bounds (m)
    ColCheck col;                  // the lane's columns
    double eta, beta_s, beta_n, beta_a, theta, mnorm_sign;
    int detect_inf, restart_to_output;
    int robust_rc;                 // 1: the stopping test takes the reduced cost robust to large bounds
    int stall_checks;              // 0: no stall test
    int check_every;
    // the lane's restart groups
    Control* ctl;                  // gcap groups
    int gcap;
    double* hal64;                 // Halpern weights of each group's next interval,
    float* hal32;                  //   [gcap][check_every][2], in each iterate type
    dfloat* haldf;
    double* rscr;                  // per-LP residual slots of the averaged restart test
    int* rtag;                     // slot holds this check's value where rtag == the check's tag
    int* flags;                    // [0]: a group restarted at the last check; [1]: checks so far
    // double-float copies for the FP32-iterate checks: scalings, their
    // reciprocals, original c, xlo, xhi (n) and l, u (m)
    const df *f_dr, *f_dc, *f_idr, *f_idc, *f_c, *f_xl, *f_xu, *f_l, *f_u;
};

// The checks of an interval of interval_len iterations on columns [0, ncol):
// FP64-accurate KKT statistics, per-LP status, then each restart group's
// averaged restart test and primal-weight update and the anchor copies.
template <typename T>
cudaError_t launch_check(const CheckData& d, const IterBufs<T>& b, int ld, int ncol, int interval_len,
                         double* P, double* Q, double* partials, double* colsum, ColRecord* rec, ColParams<T> colp,
                         cudaStream_t s, cudaEvent_t* ev /* 3 events or nullptr */);

// Admits count LPs (specs_dev) into columns [c0, c0 + count) as restart
// group `group` with residual slots [slot0, slot0 + count): per-column data,
// the group's control record and Halpern table, and the starting iterates.
// LP q starts from warm_x + q * wsx, warm_y + q * wsy (device, original
// space; stride 0 gives every LP the same start), or from zero when null.
template <typename T>
cudaError_t launch_admit(const CheckData& d, const IterData<T>& it, const IterBufs<T>& b, int ld, int c0, int count,
                         int group, int slot0, const lpb_lp_spec* specs_dev, const double* warm_x,
                         const double* warm_y, int64_t wsx, int64_t wsy, double c_norm_base, double b_norm,
                         double tol, double eps_inf, double tol_dual, int64_t max_iter, ColRecord* rec,
                         cudaStream_t s);

// x, y of the finished columns cols_dev[f] in the original space, written to
// outp_dev[f] (n values) and outp_dev[count + f] (m values); null pointers skip.
template <typename T>
cudaError_t launch_extract(const CheckData& d, const IterBufs<T>& b, int ld, const int* cols_dev,
                           double* const* outp_dev, int count, const double* xl_base, const double* xu_base,
                           cudaStream_t s);

// Moves columns sc_dev[p] of an FP32 lane to columns dc_dev[p] of a polish
// lane in precision TD (double or dfloat): the iterates and anchors widened,
// the per-column data copied, the TD parameters rebuilt from the FP64
// originals; the columns join group group_dst with slots shifted by slot_shift.
template <typename TD>
cudaError_t launch_migrate(const CheckData& src, const IterBufs<float>& sb, int lds, const CheckData& dst,
                           const IterBufs<TD>& db, int ldd, ColParams<TD> dcolp, const int* sc_dev, const int* dc_dev,
                           int count, int group_dst, int slot_shift, cudaStream_t s);

// After the host copied a group's control record into dst.ctl[group]: its
// slots start at slot0 and its Halpern table is rewritten for its k.
cudaError_t launch_group_moved(const CheckData& dst, int group, int slot0, cudaStream_t s);

template <typename T>
cudaError_t launch_compact(const IterBufs<T>& b, int n, int m, int ld, const int* src_dev, const int* dst_dev,
                           int count, ColParams<T> colp, ColCheck colc, cudaStream_t s);

}  // namespace lpb
