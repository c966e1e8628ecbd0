// lpb_step.h -- device code of the step kernels (the fused CSR SpMM with
// its primal or dual epilogue, described in lpb_iter.cu) and the host
// helpers that shape their launches, shared by the launches of one matrix
// (lpb_iter.cu) and the joint launches over several matrices (lpb_multi.cu).
#pragma once

#include <atomic>
#include <climits>
#include <type_traits>

#include "lpb_internal.h"

// resident blocks per SM the step kernels are compiled for (register cap)
#ifndef LPB_STEP_MIN_BLOCKS
#define LPB_STEP_MIN_BLOCKS 5
#endif
// the same for the double-float instantiation, whose steps are bound by
// instruction latency rather than DRAM: more resident warps hide more of it
#ifndef LPB_STEP_MIN_BLOCKS_DF
#define LPB_STEP_MIN_BLOCKS_DF 7
#endif
// gathers a lane issues before it consumes them (loads in flight per lane)
#ifndef LPB_GATHER_BATCH
#define LPB_GATHER_BATCH 4
#endif

namespace lpb {

namespace {

template <typename T> struct Vec;
template <> struct Vec<float> { static constexpr int V = 4; };
template <> struct Vec<double> { static constexpr int V = 2; };
template <> struct Vec<dfloat> { static constexpr int V = 2; };

// the FP32 primal step streams several iterate blocks besides its gathers:
// on wide batches (row groups of 32 lanes, where 48 registers hold it
// without spilling) it gains from more resident warps, i.e. loads in flight
#ifndef LPB_STEP_MIN_BLOCKS_PRIMAL
#define LPB_STEP_MIN_BLOCKS_PRIMAL 10
#endif
template <typename T, int G, bool PRIMAL> struct MinBlocks { static constexpr int v = LPB_STEP_MIN_BLOCKS; };
template <int G> struct MinBlocks<float, G, true> {
    static constexpr int v = G >= 32 ? LPB_STEP_MIN_BLOCKS_PRIMAL : LPB_STEP_MIN_BLOCKS;
};
template <int G, bool PRIMAL> struct MinBlocks<dfloat, G, PRIMAL> { static constexpr int v = LPB_STEP_MIN_BLOCKS_DF; };

__device__ __forceinline__ void ldv(const float* p, float (&r)[4]) {
    float4 u = *reinterpret_cast<const float4*>(p);
    r[0] = u.x; r[1] = u.y; r[2] = u.z; r[3] = u.w;
}
__device__ __forceinline__ void ldv(const double* p, double (&r)[2]) {
    double2 u = *reinterpret_cast<const double2*>(p);
    r[0] = u.x; r[1] = u.y;
}
__device__ __forceinline__ void ldg_v(const float* p, float (&r)[4]) {
    float4 u = __ldg(reinterpret_cast<const float4*>(p));
    r[0] = u.x; r[1] = u.y; r[2] = u.z; r[3] = u.w;
}
__device__ __forceinline__ void ldg_v(const double* p, double (&r)[2]) {
    double2 u = __ldg(reinterpret_cast<const double2*>(p));
    r[0] = u.x; r[1] = u.y;
}
__device__ __forceinline__ void stv(float* p, const float (&r)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(r[0], r[1], r[2], r[3]);
}
__device__ __forceinline__ void stv(double* p, const double (&r)[2]) {
    *reinterpret_cast<double2*>(p) = make_double2(r[0], r[1]);
}
__device__ __forceinline__ void ldv(const dfloat* p, dfloat (&r)[2]) {
    float4 u = *reinterpret_cast<const float4*>(p);
    r[0] = dfloat(u.x, u.y); r[1] = dfloat(u.z, u.w);
}
__device__ __forceinline__ void ldg_v(const dfloat* p, dfloat (&r)[2]) {
    float4 u = __ldg(reinterpret_cast<const float4*>(p));
    r[0] = dfloat(u.x, u.y); r[1] = dfloat(u.z, u.w);
}
__device__ __forceinline__ void stv(dfloat* p, const dfloat (&r)[2]) {
    *reinterpret_cast<float4*>(p) = make_float4(r[0].hi, r[0].lo, r[1].hi, r[1].lo);
}

// The row-side operands of the epilogues (the iterate, anchor and reflected
// blocks, and the check outputs) are each read or written once per launch.
// When the gathered block is too large to stay in L2 anyway (StepArgs::
// stream), they take the streaming cache hint (evict first), so that L2
// keeps more of the gathered block, which is read once per nonzero.  When
// everything fits in L2 the hint would evict what the next step reads.
#ifndef LPB_STREAM_HINT
#define LPB_STREAM_HINT 1
#endif
template <typename T, int V>
__device__ __forceinline__ void lds(const T* p, T (&r)[V], bool stream) {
    static_assert(sizeof(T) * V == sizeof(float4), "one 16-byte vector per lane");
    if (LPB_STREAM_HINT && stream) {
        const float4 u = __ldcs(reinterpret_cast<const float4*>(p));
        memcpy(&r, &u, 16);
    } else {
        ldv(p, r);
    }
}
template <typename T, int V>
__device__ __forceinline__ void sts(T* p, const T (&r)[V], bool stream) {
    if (LPB_STREAM_HINT && stream) {
        float4 u;
        memcpy(&u, &r, 16);
        __stcs(reinterpret_cast<float4*>(p), u);
    } else {
        stv(p, r);
    }
}

// scalar read-only load, shuffle, multiply-add and infinity test for each
// iterate type
__device__ __forceinline__ float ldg1(const float* p) { return __ldg(p); }
__device__ __forceinline__ double ldg1(const double* p) { return __ldg(p); }
__device__ __forceinline__ dfloat ldg1(const dfloat* p) {
    const float2 u = __ldg(reinterpret_cast<const float2*>(p));
    return dfloat(u.x, u.y);
}
template <typename T>
__device__ __forceinline__ T shfl(unsigned mask, T v, int src, int width) {
    return __shfl_sync(mask, v, src, width);
}
__device__ __forceinline__ dfloat shfl(unsigned mask, dfloat v, int src, int width) {
    return dfloat(__shfl_sync(mask, v.hi, src, width), __shfl_sync(mask, v.lo, src, width));
}
__device__ __forceinline__ float mad(float a, float x, float acc) { return fmaf(a, x, acc); }
__device__ __forceinline__ double mad(double a, double x, double acc) { return fma(a, x, acc); }
// the SpMM's running sums: for dfloat the low part stays unnormalised until
// fin() (dfl_dot_acc), which shortens the dependent chain per nonzero
__device__ __forceinline__ dfloat mad(dfloat a, dfloat x, dfloat acc) { return dfl_fma(a, x, acc); }
__device__ __forceinline__ float dot_acc(float a, float x, float acc) { return fmaf(a, x, acc); }
__device__ __forceinline__ double dot_acc(double a, double x, double acc) { return fma(a, x, acc); }
__device__ __forceinline__ dfloat dot_acc(dfloat a, dfloat x, dfloat acc) { return dfl_dot_acc(a, x, acc); }
// 2 v, exact in every iterate type (for dfloat both parts scale)
__device__ __forceinline__ float twice(float v) { return 2.0f * v; }
__device__ __forceinline__ double twice(double v) { return 2.0 * v; }
__device__ __forceinline__ dfloat twice(dfloat v) { return dfloat(2.0f * v.hi, 2.0f * v.lo); }
// y / sigma: FP32 and FP64 divide; dfloat multiplies by the column's
// reciprocal 1/sigma (staged once per block), which a double-float division
// would recompute per element at several times the cost
__device__ __forceinline__ float over_sigma(float y, float sg, float) { return y / sg; }
__device__ __forceinline__ double over_sigma(double y, double sg, double) { return y / sg; }
__device__ __forceinline__ dfloat over_sigma(dfloat y, dfloat, dfloat isg) { return y * isg; }
template <int V> __device__ __forceinline__ void fin(float (&)[V]) {}
template <int V> __device__ __forceinline__ void fin(double (&)[V]) {}
template <int V> __device__ __forceinline__ void fin(dfloat (&acc)[V]) {
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = dfl_norm(acc[v]);
}
__device__ __forceinline__ bool is_inf(float v) { return isinf(v); }
__device__ __forceinline__ bool is_inf(double v) { return isinf(v); }
__device__ __forceinline__ bool is_inf(dfloat v) { return isinf(v.hi); }

// One round of a row's entries: the G lanes of the row group load up to
// R = G*K of the row's (col, value) pairs at once (K per lane, coalesced);
// narrow groups take rounds of 8 to bound the registers holding the entries.
template <typename T, int G>
struct Round {
    static constexpr int K = G >= 8 ? 1 : 8 / G;
    static constexpr int R = G * K;
};

template <typename T, int G>
__device__ __forceinline__ void load_round(const int* __restrict__ ci, const T* __restrict__ va, int e0, int end,
                                           int (&c)[Round<T, G>::K], T (&a)[Round<T, G>::K]) {
    constexpr int K = Round<T, G>::K;
    const int lane = threadIdx.x % G;
#pragma unroll
    for (int q = 0; q < K; ++q) {
        const int me = e0 + q * G + lane;
        c[q] = me < end ? __ldg(ci + me) : 0;
        a[q] = me < end ? ldg1(va + me) : T(0);
    }
}

// acc += sum over the round's cnt entries of a_e * src[col_e, colg .. colg+V):
// entries are broadcast by shuffle inside the row group (entry k sits in
// register slot k / G of lane k % G, compile-time after unrolling) and the
// gathers issued four at a time.  Entries past cnt get a = 0 and the round's
// first column, so every gather stays in bounds.  All lanes of the group
// must call it (lanes past the last LP pass the tile's first column).
template <typename T, int V, int G>
__device__ __forceinline__ void gather_round(const int (&c)[Round<T, G>::K], const T (&a)[Round<T, G>::K], int cnt,
                                             const T* __restrict__ src, int ld, int colg, unsigned gmask,
                                             T (&acc)[V]) {
    constexpr int R = Round<T, G>::R;
    constexpr int B = LPB_GATHER_BATCH < R ? LPB_GATHER_BATCH : R;
    static_assert(R % B == 0, "a round is a whole number of gather batches");
    const int cfirst = __shfl_sync(gmask, c[0], 0, G);
#pragma unroll
    for (int k0 = 0; k0 < R; k0 += B) {
        if (k0 >= cnt) break;
        int cc[B];
        T aa[B];
#pragma unroll
        for (int j = 0; j < B; ++j) {
            const int k = k0 + j;
            const int cs = __shfl_sync(gmask, c[k / G], k % G, G);
            const T as = shfl(gmask, a[k / G], k % G, G);
            cc[j] = k < cnt ? cs : cfirst;
            aa[j] = k < cnt ? as : T(0);
        }
        T xs[B][V];
#pragma unroll
        for (int j = 0; j < B; ++j) ldg_v(src + (size_t)cc[j] * ld + colg, xs[j]);
        // entries in order, so a column's sum does not depend on G
#pragma unroll
        for (int j = 0; j < B; ++j)
#pragma unroll
            for (int v = 0; v < V; ++v) acc[v] = dot_acc(aa[j], xs[j][v], acc[v]);
    }
}

template <typename T, int V, int G>
__device__ __forceinline__ void gather_range(const int* __restrict__ ci, const T* __restrict__ va,
                                             const T* __restrict__ src, int ld, int colg, int beg, int end,
                                             unsigned gmask, T (&acc)[V]) {
    constexpr int K = Round<T, G>::K, R = Round<T, G>::R;
#pragma unroll 1
    for (int e0 = beg; e0 < end; e0 += R) {
        int c[K];
        T a[K];
        load_round<T, G>(ci, va, e0, end, c, a);
        gather_round<T, V, G>(c, a, min(R, end - e0), src, ld, colg, gmask, acc);
    }
}

template <typename T>
struct StepArgs {
    // sparse operator (rows of A~^T for the primal step, of A~ for the dual step)
    int rows;
    const int* rp;
    const int* ci;
    const T* va;
    const int* long_rows;
    int n_long, long_thr;
    const int* lseg;  // long-row blocks: (long row, segment) of each, segment-major
    const int* lseg0; // first segment of each long row; segments of row i: lseg0[i + 1] - lseg0[i]
    int n_lblocks;
    T* part;          // partial sums of multi-segment rows, [segment][ld]
    unsigned* ticket; // completion count per (long row, column tile), tile stride ntix
    int ntix;
    const T* src;     // gathered block: Y^k (primal) or Xbar (dual)
    // row-side state
    T* Z;             // dual: Y^k -> Y^{k+1}, in place (unused by the primal step)
    const T* Z0;      // anchor
    T* Zbar;          // primal: Xbar of the previous iteration in, the new Xbar out (in place)
    T* Zh;            // check: x^ / y^
    T* DZ;            // check: x^ - X^k / y^ - Y^k
    T* Aux;           // check, dual: Pi_B(y^ - Y^k)
    const T* rc;      // primal: scaled c (n)
    const T* rlo;     // scaled lower bounds of the rows (xlo or l)
    const T* rhi;
    ColParams<T> col;
    int ld, ncol;
    const T* hal;     // per group g, entry e = 0 .. ce: (k+1)/(k+2), 1/(k+2) of Eq. mainiter
                      // for k = k_start - 1 + e at [2 (g (ce + 1) + e)]; iteration t of the
                      // interval uses entry t + 1, and entry t rebuilds its X^k
    int t, ce;
    int uni;          // the group of every active column, or -1 if they belong to several
    int pdl;          // launched as a programmatic dependent of the previous step kernel
    int stream;       // the gathered block exceeds half of L2: streaming hints on the row operands
};

// Reduce the row groups' partial sums of a long row through shared memory;
// on return only row group 0 holds the sum.  Every thread of the block calls it.
template <typename T, int V, int G>
__device__ __forceinline__ bool long_row_reduce(T (&acc)[V], T* red) {
    constexpr int GPB = kBlock / G;
    const int lane = threadIdx.x % G, grp = threadIdx.x / G;
#pragma unroll
    for (int v = 0; v < V; ++v) red[threadIdx.x * V + v] = acc[v];
    __syncthreads();
    if (grp != 0) return false;
    for (int g = 1; g < GPB; ++g)
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] += red[(g * G + lane) * V + v];
    return true;
}

template <typename T>
__device__ __forceinline__ T barrier(T v, T lo, T hi) {
    const bool li = is_inf(lo), hi_ = is_inf(hi);
    if (li && hi_) return T(0);
    if (li) return v > T(0) ? v : T(0);
    if (hi_) return v < T(0) ? v : T(0);
    return v;
}

// per-column parameters of the block's column tile, staged in shared memory;
// ca, cb are the Halpern weights of the column's restart group
template <typename T, int TN>
struct TileParams {
    T tau[TN], lo[TN], hi[TN], c[TN], sigma[TN], isigma[TN], ca[TN], cb[TN], pa[TN], pb[TN];
    int kind[TN], var[TN];
};

// primal epilogue for row `row`, lane columns col0 .. col0+V (q0 = their
// offset in the tile): the iterate rebuilt from the previous reflection,
// box projection, reflection (the Halpern update of Eq. mainiter is applied
// when the next step rebuilds its iterate)
template <typename T, int V, int TN, bool CHECK>
__device__ __forceinline__ void primal_epilogue(const StepArgs<T>& a, const TileParams<T, TN>& P, int row, int col0,
                                                int q0, const T (&acc)[V], T upa, T upb) {
    const size_t off = (size_t)row * a.ld + col0;
    T x[V], x0[V];
    lds(a.Zbar + off, x, a.stream);
    lds(a.Z0 + off, x0, a.stream);
    const T cr = a.rc[row], lor = a.rlo[row], hir = a.rhi[row];
    T xh[V], xb[V], dz[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const int q = q0 + v;
        const T pa = a.uni >= 0 ? upa : P.pa[q], pb = a.uni >= 0 ? upb : P.pb[q];
        x[v] = mad(pa, x[v], pb * x0[v]);  // X^k = k/(k+1) Xb + X^0/(k+1)
        const int kind = P.kind[q], var = P.var[q];
        T cj = cr, lo = lor, hi = hir;
        if (kind == 2) cj = var == row ? P.c[q] : T(0);
        else if (kind == 1 && var == row) { lo = P.lo[q]; hi = P.hi[q]; }
        const T step = P.tau[q] * (cj + acc[v]);
        T s = x[v] - step;
        const bool inside = s < hi && s > lo;
        s = s < hi ? s : hi;
        s = s > lo ? s : lo;
        xh[v] = s;
        xb[v] = twice(s) - x[v];
        // x^ - x: where the box is not active it is -tau (c + G) exactly,
        // which stays accurate when |x| is large (diverging iterates of an
        // infeasible LP); elsewhere the difference with the bound
        dz[v] = inside ? -step : s - x[v];
    }
    sts(a.Zbar + off, xb, a.stream);
    if (CHECK) {
        sts(a.Zh + off, xh, a.stream);
        sts(a.DZ + off, dz, a.stream);
    }
}

// dual epilogue: row projection and Halpern update
template <typename T, int V, int TN, bool CHECK>
__device__ __forceinline__ void dual_epilogue(const StepArgs<T>& a, const TileParams<T, TN>& P, int row, int col0,
                                              int q0, const T (&acc)[V], T uca, T ucb) {
    const size_t off = (size_t)row * a.ld + col0;
    T y[V], y0[V];
    lds(a.Z + off, y, a.stream);
    lds(a.Z0 + off, y0, a.stream);
    const T lr = a.rlo[row], ur = a.rhi[row];
    T yh[V], yn[V], dz[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const T sg = P.sigma[q0 + v];
        const T s = over_sigma(y[v], sg, P.isigma[q0 + v]) + acc[v];
        T p = s < ur ? s : ur;
        p = p > lr ? p : lr;
        yh[v] = sg * (s - p);
        const T ca = a.uni >= 0 ? uca : P.ca[q0 + v], cb = a.uni >= 0 ? ucb : P.cb[q0 + v];
        yn[v] = ca * (twice(yh[v]) - y[v]) + cb * y0[v];
        // y^ - y: y^ = 0 exactly where the row bound is not active; where it
        // is, y^ - y = sigma (A xb - Pi(v)) without the cancellation of y
        dz[v] = p == s ? -y[v] : sg * (acc[v] - p);
    }
    sts(a.Z + off, yn, a.stream);
    if (CHECK) {
        T dzp[V];
#pragma unroll
        for (int v = 0; v < V; ++v) dzp[v] = barrier(dz[v], lr, ur);
        sts(a.Zh + off, yh, a.stream);
        sts(a.DZ + off, dz, a.stream);
        sts(a.Aux + off, dzp, a.stream);
    }
}

__device__ __forceinline__ void stv_cg(float* p, const float (&r)[4]) {
    __stcg(reinterpret_cast<float4*>(p), make_float4(r[0], r[1], r[2], r[3]));
}
__device__ __forceinline__ void stv_cg(double* p, const double (&r)[2]) {
    __stcg(reinterpret_cast<double2*>(p), make_double2(r[0], r[1]));
}
__device__ __forceinline__ void stv_cg(dfloat* p, const dfloat (&r)[2]) {
    __stcg(reinterpret_cast<float4*>(p), make_float4(r[0].hi, r[0].lo, r[1].hi, r[1].lo));
}
__device__ __forceinline__ void ldv_cg(const float* p, float (&r)[4]) {
    const float4 u = __ldcg(reinterpret_cast<const float4*>(p));
    r[0] = u.x; r[1] = u.y; r[2] = u.z; r[3] = u.w;
}
__device__ __forceinline__ void ldv_cg(const double* p, double (&r)[2]) {
    const double2 u = __ldcg(reinterpret_cast<const double2*>(p));
    r[0] = u.x; r[1] = u.y;
}
__device__ __forceinline__ void ldv_cg(const dfloat* p, dfloat (&r)[2]) {
    const float4 u = __ldcg(reinterpret_cast<const float4*>(p));
    r[0] = dfloat(u.x, u.y); r[1] = dfloat(u.z, u.w);
}
__device__ __forceinline__ float add(float a, float b) { return a + b; }
__device__ __forceinline__ double add(double a, double b) { return a + b; }
__device__ __forceinline__ dfloat add(dfloat a, dfloat b) { return a + b; }

// One step (primal or dual) of the iteration on one column tile.
//   Blocks [0, n_lblocks): one segment of a long row each (at most kStepSeg
//   entries), split into contiguous pieces over the block's row groups and
//   reduced in shared memory.  A row of one segment is finished by its block;
//   for a row of several, each block stores its partial sums, and the block
//   that completes the row (the last to take the row's ticket; no block
//   waits) adds the partials in segment order and finishes the row, so the
//   result does not depend on which block ends last.
//   Blocks [n_lblocks, gx): persistent over the short rows, row group g
//   taking rows g, g + stride, ...; while it gathers and finishes a row, the
//   row pointers and the first index round of its next row are in flight.
//   (bx, by) is the block's place in the step's own grid (bx over the
//   long-row and persistent blocks, gx of them; by over the column tiles).
template <typename T, int G, bool CHECK, bool PRIMAL>
__device__ __forceinline__ void step_body(const StepArgs<T>& a, const int bx, const int by, const int gx) {
    constexpr int V = Vec<T>::V, GPB = kBlock / G, TN = G * V;
    constexpr int K = Round<T, G>::K, R = Round<T, G>::R;
    __shared__ T red[kBlock * V];
    __shared__ TileParams<T, TN> P;
    const int lane = threadIdx.x % G, grp = threadIdx.x / G;
    const int tile0 = by * TN;
    for (int q = threadIdx.x; q < TN; q += kBlock) {
        const int j = tile0 + q;
        const bool in = j < a.ncol;
        if (a.uni < 0) {
            // entry t + 1 of the column's group: this iteration's weights;
            // entry t: the previous iteration's, which rebuild X^k
            const int h = in ? 2 * (a.col.grp[j] * (a.ce + 1) + a.t + 1) : 2;
            if (PRIMAL) {
                P.pa[q] = in ? a.hal[h - 2] : T(0);
                P.pb[q] = in ? a.hal[h - 1] : T(0);
            } else {
                P.ca[q] = in ? a.hal[h] : T(0);
                P.cb[q] = in ? a.hal[h + 1] : T(0);
            }
        }
        if (PRIMAL) {
            P.kind[q] = in ? a.col.kind[j] : 0;
            P.var[q] = in ? a.col.var[j] : -1;
            P.tau[q] = in ? a.col.tau[j] : T(0);
            P.lo[q] = in ? a.col.lo[j] : T(0);
            P.hi[q] = in ? a.col.hi[j] : T(0);
            P.c[q] = in ? a.col.c[j] : T(0);
        } else {
            P.sigma[q] = in ? a.col.sigma[j] : T(1);
            if (std::is_same<T, dfloat>::value) P.isigma[q] = T(1) / P.sigma[q];
        }
    }
    __syncthreads();
    // Programmatic dependent launch: everything above reads only data that
    // the previous kernel does not write (per-column parameters, Halpern
    // weights).  That holds because only step kernels after an interval's
    // first are launched as programmatic dependents, and their predecessor
    // is a step kernel; the first primal step of an interval follows the
    // check, admission, extraction, compaction and migration kernels that do
    // write those parameters, and is launched without the attribute
    // (launch_iteration).  Wait for the predecessor to complete before
    // touching the iterates, then let the next step kernel start its own
    // prologue on the SMs this grid frees.
    if (a.pdl) {
        asm volatile("griddepcontrol.wait;" ::: "memory");
        asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    }
    // one restart group in the whole batch: its Halpern weights as scalars
    // (the primal step takes the previous iteration's, the dual step this one's)
    const int hu = a.uni >= 0 ? 2 * (a.uni * (a.ce + 1) + a.t + (PRIMAL ? 0 : 1)) : 0;
    const T uca = a.uni >= 0 ? a.hal[hu] : T(0), ucb = a.uni >= 0 ? a.hal[hu + 1] : T(0);
    const int col0 = tile0 + lane * V;
    const bool active = col0 < a.ncol;
    const int colg = active ? col0 : tile0;
    const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));

    if (bx < a.n_lblocks) {
        const int li = a.lseg[2 * bx], sg = a.lseg[2 * bx + 1];
        const int s0 = a.lseg0[li], ns = a.lseg0[li + 1] - s0;
        const int row = a.long_rows[li];
        const int rb0 = a.rp[row], re0 = a.rp[row + 1];
        const int sl = (re0 - rb0 + ns - 1) / ns;  // entries per segment
        const int rb = min(re0, rb0 + sg * sl), re = min(re0, rb + sl);
        const int piece = (re - rb + GPB - 1) / GPB;
        const int beg = min(re, rb + grp * piece), end = min(re, beg + piece);
        T acc[V];
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = T(0);
        gather_range<T, V, G>(a.ci, a.va, a.src, a.ld, colg, beg, end, gmask, acc);
        fin<V>(acc);
        if (!long_row_reduce<T, V, G>(acc, red)) return;
        // only row group 0 (lanes 0 .. G-1 of warp 0) continues
        if (ns > 1) {
            if (active) stv_cg(a.part + (size_t)(s0 + sg) * a.ld + col0, acc);
            __threadfence();
            __syncwarp(gmask);
            unsigned last = 0;
            if (lane == 0) {
                unsigned* t = a.ticket + (size_t)li * a.ntix + by;
                last = atomicAdd(t, 1u) == (unsigned)(ns - 1);
                if (last) *t = 0u;  // ready for the next launch
            }
            last = __shfl_sync(gmask, last, 0, G);
            if (!last) return;
            __threadfence();
            if (!active) return;
            T p[V];
            ldv_cg(a.part + (size_t)s0 * a.ld + col0, acc);
#pragma unroll 1
            for (int t = 1; t < ns; ++t) {
                ldv_cg(a.part + (size_t)(s0 + t) * a.ld + col0, p);
#pragma unroll
                for (int v = 0; v < V; ++v) acc[v] = add(acc[v], p[v]);
            }
        }
        if (!active) return;
        if (PRIMAL) primal_epilogue<T, V, TN, CHECK>(a, P, row, col0, lane * V, acc, uca, ucb);
        else dual_epilogue<T, V, TN, CHECK>(a, P, row, col0, lane * V, acc, uca, ucb);
        return;
    }

    const int stride = (gx - a.n_lblocks) * GPB;
    int r = (bx - a.n_lblocks) * GPB + grp;
    int beg = 0, end = 0;
    int c[K];
    T av[K];
    if (r < a.rows) {
        beg = a.rp[r];
        end = a.rp[r + 1];
        load_round<T, G>(a.ci, a.va, beg, end - beg <= a.long_thr ? end : beg, c, av);
    }
#pragma unroll 1
    while (r < a.rows) {
        const int rn = r + stride;
        int nbeg = 0, nend = 0;
        if (rn < a.rows) {
            nbeg = a.rp[rn];
            nend = a.rp[rn + 1];
        }
        const bool is_short = end - beg <= a.long_thr;
        T acc[V];
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = T(0);
        if (is_short) {
            gather_round<T, V, G>(c, av, min(R, end - beg), a.src, a.ld, colg, gmask, acc);
            if (end - beg > R)
                gather_range<T, V, G>(a.ci, a.va, a.src, a.ld, colg, beg + R, end, gmask, acc);
            fin<V>(acc);
        }
        // the next row's first index round, issued before this row's epilogue
        if (rn < a.rows) load_round<T, G>(a.ci, a.va, nbeg, nend - nbeg <= a.long_thr ? nend : nbeg, c, av);
        if (is_short && active) {
            if (PRIMAL) primal_epilogue<T, V, TN, CHECK>(a, P, r, col0, lane * V, acc, uca, ucb);
            else dual_epilogue<T, V, TN, CHECK>(a, P, r, col0, lane * V, acc, uca, ucb);
        }
        r = rn;
        beg = nbeg;
        end = nend;
    }
}

// Launch shapes are cached per device: SM count and resident blocks per SM
// packed into one int (sms * 64 + per_sm, 0 = not yet looked up), published
// with release / acquire so that every thread (the server runs one worker per
// matrix) reads both values of one lookup or does the lookup itself.
constexpr int kShapeDevices = 64;
inline int pack_shape(int sms, int per_sm) {
    sms = sms > 0 ? sms : 1;
    per_sm = per_sm > 0 ? (per_sm < 63 ? per_sm : 63) : 1;
    return sms * 64 + per_sm;
}

// SM count and resident blocks per SM of kernel f (kBlock threads) on the
// current device, through f's per-device cache `shape` (static storage)
template <typename F>
cudaError_t launch_shape(std::atomic<int>* shape, F f, int* sms, int* per_sm) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int packed = dev >= 0 && dev < kShapeDevices ? shape[dev].load(std::memory_order_acquire) : 0;
    if (packed == 0) {
        int b = 0, n = 0;
        if ((e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, f, kBlock, 0)) != cudaSuccess) return e;
        packed = pack_shape(n, b);
        if (dev >= 0 && dev < kShapeDevices) shape[dev].store(packed, std::memory_order_release);
    }
    *sms = packed / 64;
    *per_sm = packed % 64;
    return cudaSuccess;
}

// f<<<grid, kBlock, 0, s>>>(a), as a programmatic dependent of the previous
// kernel in s when pdl is set
template <typename A>
cudaError_t launch_with(void (*f)(A), dim3 grid, const A& a, bool pdl, cudaStream_t s) {
    if (!pdl) {
        f<<<grid, kBlock, 0, s>>>(a);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(kBlock);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, f, a);
}

// Lanes per row group for a batch of ncol columns (one vector of V columns
// per lane), halved g_shift times: narrower groups make more column tiles,
// each row's gathers split over more blocks.
template <typename T>
int row_group_lanes(int ncol, int g_shift) {
    constexpr int V = Vec<T>::V;
    int vecs = (ncol + V - 1) / V;
    for (int q = 0; q < g_shift && vecs > 1; ++q) vecs = (vecs + 1) / 2;
    return vecs <= 1 ? 1 : vecs <= 2 ? 2 : vecs <= 4 ? 4 : vecs <= 8 ? 8 : vecs <= 16 ? 16 : 32;
}

// L2 bytes of the current device, looked up once per device
inline cudaError_t l2_bytes(long long* out) {
    static std::atomic<long long> cache[kShapeDevices];  // static storage: starts at 0
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    long long v = dev >= 0 && dev < kShapeDevices ? cache[dev].load(std::memory_order_acquire) : 0;
    if (v == 0) {
        int b = 0;
        if ((e = cudaDeviceGetAttribute(&b, cudaDevAttrL2CacheSize, dev)) != cudaSuccess) return e;
        v = b > 0 ? b : 1;
        if (dev >= 0 && dev < kShapeDevices) cache[dev].store(v, std::memory_order_release);
    }
    *out = v;
    return cudaSuccess;
}

// The arguments of one matrix's primal step (rows of A~^T gathering Y) or
// dual step (rows of A~ gathering Xbar) at iteration t of its interval;
// pdl is left to the caller.  l2: the device's L2 bytes, which decide the
// streaming hints.
template <typename T>
StepArgs<T> step_args(bool primal, const IterData<T>& d, const IterBufs<T>& b, int ld, int ncol, const T* hal,
                      int t, int ce, int uni, long long l2) {
    const Csr& c = primal ? d.At : d.A;
    StepArgs<T> a{};
    a.rows = c.rows;
    a.rp = c.rp;
    a.ci = c.ci;
    a.va = primal ? d.at_vals : d.a_vals;
    a.long_rows = c.long_rows;
    a.n_long = c.n_long;
    a.long_thr = c.long_thr;
    a.lseg = c.lseg;
    a.lseg0 = c.lseg0;
    a.n_lblocks = c.n_lblocks;
    a.part = (T*)c.part;
    a.ticket = c.ticket;
    a.ntix = c.ntix;
    // the gathered block: Y (m x ld) for the primal step, Xbar (n x ld) for the dual step
    const long long gbytes = (long long)(primal ? d.A.rows : d.A.cols) * ld * (long long)sizeof(T);
    a.stream = 2 * gbytes > l2;
    if (primal) {
        a.src = b.Y;
        a.Z = nullptr;
        a.Z0 = b.X0;
        a.Zbar = b.Xbar;
        a.Zh = b.Xh;
        a.DZ = b.DX;
        a.Aux = nullptr;
        a.rc = d.c;
        a.rlo = d.xl;
        a.rhi = d.xu;
    } else {
        a.src = b.Xbar;
        a.Z = b.Y;
        a.Z0 = b.Y0;
        a.Zbar = nullptr;
        a.Zh = b.Yh;
        a.DZ = b.DY;
        a.Aux = b.DYp;
        a.rc = nullptr;
        a.rlo = d.l;
        a.rhi = d.u;
    }
    a.col = d.col;
    a.ld = ld;
    a.ncol = ncol;
    a.hal = hal;
    a.t = t;
    a.ce = ce;
    a.uni = uni;
    return a;
}

}  // namespace

}  // namespace lpb
