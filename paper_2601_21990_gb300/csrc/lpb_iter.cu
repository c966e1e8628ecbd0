// lpb_iter.cu -- the hot path: one reflected-Halpern PDHG iteration on the
// whole active batch (Sec. 5, Eq. batched_iter and main-iterate).
//
//   primal step  (rows of A~^T, one per variable i; G = A~^T Y^k):
//     x^  = Pi_[xlo_ij, xhi_ij](X^k_ij - tau_j (c_ij + G_ij))
//     xb  = 2 x^ - X^k_ij                     (the reflection, also A(2x - x^k))
//     X^{k+1}_ij = (k+1)/(k+2) xb + X^0_ij/(k+2)
//   dual step    (rows of A~, one per constraint i; H = A~ Xb):
//     v   = Y^k_ij / sigma_j + H_ij
//     y^  = sigma_j (v - Pi_[l_i,u_i](v))     (= Y + sigma H - sigma Pi(Y/sigma + H))
//     Y^{k+1}_ij = (k+1)/(k+2)(2 y^ - Y^k_ij) + Y^0_ij/(k+2)
//
// Both products are CSR SpMMs against a row-major, batch-contiguous dense
// block: a "row group" of G lanes owns one sparse row and a tile of G*V
// batch columns, each lane V consecutive columns loaded as one 16-byte
// vector per nonzero.  Rows longer than kLongRow get a whole block whose
// row groups split the nonzeros and reduce in shared memory; those blocks
// come first in the grid.  The projection, reflection and Halpern update
// run in the same kernel on the accumulator in registers, so H and A^T Y
// never touch memory.  Per-LP overrides (Sec. 5.1, 5.2) are applied by
// comparing the row index with each column's override variable; the
// matrices X_lo, X_hi and C are never formed.
#include "lpb_internal.h"

namespace lpb {

namespace {

template <typename T> struct Vec;
template <> struct Vec<float> { static constexpr int V = 4; };
template <> struct Vec<double> { static constexpr int V = 2; };

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
__device__ __forceinline__ void ldv_i(const int* p, int (&r)[4]) {
    int4 u = *reinterpret_cast<const int4*>(p);
    r[0] = u.x; r[1] = u.y; r[2] = u.z; r[3] = u.w;
}
__device__ __forceinline__ void ldv_i(const int* p, int (&r)[2]) {
    int2 u = *reinterpret_cast<const int2*>(p);
    r[0] = u.x; r[1] = u.y;
}

// acc += sum over the row's nonzeros e = beg+slot, beg+slot+nslot, ... of
// a_e * src[col_e, col0 .. col0+V)
template <typename T, int V>
__device__ __forceinline__ void gather_row(const int* __restrict__ rp, const int* __restrict__ ci,
                                           const T* __restrict__ va, const T* __restrict__ src, int ld, int col0,
                                           int row, int slot, int nslot, T (&acc)[V]) {
    const int end = rp[row + 1];
    int e = rp[row] + slot;
    for (; e + 3 * nslot < end; e += 4 * nslot) {
        const int c0 = ci[e], c1 = ci[e + nslot], c2 = ci[e + 2 * nslot], c3 = ci[e + 3 * nslot];
        const T a0 = va[e], a1 = va[e + nslot], a2 = va[e + 2 * nslot], a3 = va[e + 3 * nslot];
        T x0[V], x1[V], x2[V], x3[V];
        ldg_v(src + (size_t)c0 * ld + col0, x0);
        ldg_v(src + (size_t)c1 * ld + col0, x1);
        ldg_v(src + (size_t)c2 * ld + col0, x2);
        ldg_v(src + (size_t)c3 * ld + col0, x3);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            acc[v] = fma(a0, x0[v], acc[v]);
            acc[v] = fma(a1, x1[v], acc[v]);
            acc[v] = fma(a2, x2[v], acc[v]);
            acc[v] = fma(a3, x3[v], acc[v]);
        }
    }
    for (; e < end; e += nslot) {
        const int c0 = ci[e];
        const T a0 = va[e];
        T x0[V];
        ldg_v(src + (size_t)c0 * ld + col0, x0);
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = fma(a0, x0[v], acc[v]);
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
    int n_long;
    const T* src;     // gathered block: Y^k (primal) or Xbar (dual)
    // row-side state
    T* Z;             // X^k -> X^{k+1} (primal) / Y^k -> Y^{k+1} (dual), in place
    const T* Z0;      // anchor
    T* Zbar;          // primal: Xbar out
    T* Zh;            // check: x^ / y^
    T* DZ;            // check: x^ - X^k / y^ - Y^k
    T* Aux;           // check: G = A~^T Y^k (primal) / Pi_B(y^ - Y^k) (dual)
    const T* rc;      // primal: scaled c (n)
    const T* rlo;     // scaled lower bounds of the rows (xlo or l)
    const T* rhi;
    ColParams<T> col;
    int ld, ncol;
    const int* k_dev;
    int t;
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

template <typename T, int G, bool CHECK>
__global__ void __launch_bounds__(kBlock) k_primal(const StepArgs<T> a) {
    constexpr int V = Vec<T>::V, GPB = kBlock / G, TN = G * V;
    __shared__ T red[kBlock * V];
    const int lane = threadIdx.x % G, grp = threadIdx.x / G;
    const int col0 = blockIdx.y * TN + lane * V;
    const bool active = col0 < a.ncol;
    const bool is_long = (int)blockIdx.x < a.n_long;
    int row, slot = 0, nslot = 1;
    if (is_long) {
        row = a.long_rows[blockIdx.x];
        slot = grp;
        nslot = GPB;
    } else {
        row = ((int)blockIdx.x - a.n_long) * GPB + grp;
        if (row >= a.rows) return;
        if (a.rp[row + 1] - a.rp[row] > kLongRow) return;
    }
    T acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = T(0);
    if (active) gather_row<T, V>(a.rp, a.ci, a.va, a.src, a.ld, col0, row, slot, nslot, acc);
    if (is_long && !long_row_reduce<T, V, G>(acc, red)) return;
    if (!active) return;

    int kind[V], var[V];
    T tau[V], olo[V], ohi[V], oc[V];
    ldv_i(a.col.kind + col0, kind);
    ldv_i(a.col.var + col0, var);
    ldv(a.col.tau + col0, tau);
    ldv(a.col.lo + col0, olo);
    ldv(a.col.hi + col0, ohi);
    ldv(a.col.c + col0, oc);
    const int k = *a.k_dev + a.t;
    const T ca = (T)((double)(k + 1) / (double)(k + 2));
    const T cb = (T)(1.0 / (double)(k + 2));

    const size_t off = (size_t)row * a.ld + col0;
    T x[V], x0[V], xh[V], xb[V], xn[V], dz[V];
    ldv(a.Z + off, x);
    ldv(a.Z0 + off, x0);
    const T cr = a.rc[row], lor = a.rlo[row], hir = a.rhi[row];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        T cj = cr, lo = lor, hi = hir;
        if (kind[v] == 2) cj = var[v] == row ? oc[v] : T(0);
        else if (kind[v] == 1 && var[v] == row) { lo = olo[v]; hi = ohi[v]; }
        const T step = tau[v] * (cj + acc[v]);
        T s = x[v] - step;
        const bool inside = s < hi && s > lo;
        s = s < hi ? s : hi;
        s = s > lo ? s : lo;
        xh[v] = s;
        xb[v] = T(2) * s - x[v];
        xn[v] = ca * xb[v] + cb * x0[v];
        // x^ - x: where the box is not active it is -tau (c + G) exactly,
        // which stays accurate when |x| is large (diverging iterates of an
        // infeasible LP); elsewhere the difference with the bound
        dz[v] = inside ? -step : s - x[v];
    }
    stv(a.Zbar + off, xb);
    stv(a.Z + off, xn);
    if (CHECK) {
        stv(a.Zh + off, xh);
        stv(a.DZ + off, dz);
    }
}

template <typename T>
__device__ __forceinline__ T barrier(T v, T lo, T hi) {
    const bool li = isinf(lo), hi_ = isinf(hi);
    if (li && hi_) return T(0);
    if (li) return v > T(0) ? v : T(0);
    if (hi_) return v < T(0) ? v : T(0);
    return v;
}

template <typename T, int G, bool CHECK>
__global__ void __launch_bounds__(kBlock) k_dual(const StepArgs<T> a) {
    constexpr int V = Vec<T>::V, GPB = kBlock / G, TN = G * V;
    __shared__ T red[kBlock * V];
    const int lane = threadIdx.x % G, grp = threadIdx.x / G;
    const int col0 = blockIdx.y * TN + lane * V;
    const bool active = col0 < a.ncol;
    const bool is_long = (int)blockIdx.x < a.n_long;
    int row, slot = 0, nslot = 1;
    if (is_long) {
        row = a.long_rows[blockIdx.x];
        slot = grp;
        nslot = GPB;
    } else {
        row = ((int)blockIdx.x - a.n_long) * GPB + grp;
        if (row >= a.rows) return;
        if (a.rp[row + 1] - a.rp[row] > kLongRow) return;
    }
    T acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = T(0);
    if (active) gather_row<T, V>(a.rp, a.ci, a.va, a.src, a.ld, col0, row, slot, nslot, acc);
    if (is_long && !long_row_reduce<T, V, G>(acc, red)) return;
    if (!active) return;

    T sigma[V];
    ldv(a.col.sigma + col0, sigma);
    const int k = *a.k_dev + a.t;
    const T ca = (T)((double)(k + 1) / (double)(k + 2));
    const T cb = (T)(1.0 / (double)(k + 2));

    const size_t off = (size_t)row * a.ld + col0;
    T y[V], y0[V], yh[V], yn[V], dz[V];
    ldv(a.Z + off, y);
    ldv(a.Z0 + off, y0);
    const T lr = a.rlo[row], ur = a.rhi[row];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const T s = y[v] / sigma[v] + acc[v];
        T p = s < ur ? s : ur;
        p = p > lr ? p : lr;
        yh[v] = sigma[v] * (s - p);
        yn[v] = ca * (T(2) * yh[v] - y[v]) + cb * y0[v];
        // y^ - y: y^ = 0 exactly where the row bound is not active; where it
        // is, y^ - y = sigma (A xb - Pi(v)) without the cancellation of y
        dz[v] = p == s ? -y[v] : sigma[v] * (acc[v] - p);
    }
    stv(a.Z + off, yn);
    if (CHECK) {
        T dzp[V];
#pragma unroll
        for (int v = 0; v < V; ++v) dzp[v] = barrier(dz[v], lr, ur);
        stv(a.Zh + off, yh);
        stv(a.DZ + off, dz);
        stv(a.Aux + off, dzp);
    }
}

template <typename T, int G>
cudaError_t launch_step(bool primal, bool check, const StepArgs<T>& a, cudaStream_t s) {
    constexpr int V = Vec<T>::V, GPB = kBlock / G, TN = G * V;
    if (a.rows == 0 || a.ncol == 0) return cudaSuccess;
    dim3 grid(a.n_long + (a.rows + GPB - 1) / GPB, (a.ncol + TN - 1) / TN);
    if (primal) {
        if (check) k_primal<T, G, true><<<grid, kBlock, 0, s>>>(a);
        else k_primal<T, G, false><<<grid, kBlock, 0, s>>>(a);
    } else {
        if (check) k_dual<T, G, true><<<grid, kBlock, 0, s>>>(a);
        else k_dual<T, G, false><<<grid, kBlock, 0, s>>>(a);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t dispatch_step(bool primal, bool check, const StepArgs<T>& a, cudaStream_t s) {
    constexpr int V = Vec<T>::V;
    const int vecs = (a.ncol + V - 1) / V;
    if (vecs <= 1) return launch_step<T, 1>(primal, check, a, s);
    if (vecs <= 2) return launch_step<T, 2>(primal, check, a, s);
    if (vecs <= 4) return launch_step<T, 4>(primal, check, a, s);
    if (vecs <= 8) return launch_step<T, 8>(primal, check, a, s);
    if (vecs <= 16) return launch_step<T, 16>(primal, check, a, s);
    return launch_step<T, 32>(primal, check, a, s);
}

}  // namespace

template <typename T>
cudaError_t launch_iteration(const IterData<T>& d, const IterBufs<T>& b, int ld, int ncol, const int* k_dev, int t,
                             bool check, cudaStream_t s, cudaEvent_t* ev) {
    cudaError_t e;
    StepArgs<T> p{};
    p.rows = d.At.rows;
    p.rp = d.At.rp;
    p.ci = d.At.ci;
    p.va = d.at_vals;
    p.long_rows = d.At.long_rows;
    p.n_long = d.At.n_long;
    p.src = b.Y;
    p.Z = b.X;
    p.Z0 = b.X0;
    p.Zbar = b.Xbar;
    p.Zh = b.Xh;
    p.DZ = b.DX;
    p.Aux = b.G;
    p.rc = d.c;
    p.rlo = d.xl;
    p.rhi = d.xu;
    p.col = d.col;
    p.ld = ld;
    p.ncol = ncol;
    p.k_dev = k_dev;
    p.t = t;
    if (ev && (e = cudaEventRecord(ev[0], s)) != cudaSuccess) return e;
    if ((e = dispatch_step<T>(true, check, p, s)) != cudaSuccess) return e;
    if (ev && (e = cudaEventRecord(ev[1], s)) != cudaSuccess) return e;

    StepArgs<T> q{};
    q.rows = d.A.rows;
    q.rp = d.A.rp;
    q.ci = d.A.ci;
    q.va = d.a_vals;
    q.long_rows = d.A.long_rows;
    q.n_long = d.A.n_long;
    q.src = b.Xbar;
    q.Z = b.Y;
    q.Z0 = b.Y0;
    q.Zbar = nullptr;
    q.Zh = b.Yh;
    q.DZ = b.DY;
    q.Aux = b.DYp;
    q.rc = nullptr;
    q.rlo = d.l;
    q.rhi = d.u;
    q.col = d.col;
    q.ld = ld;
    q.ncol = ncol;
    q.k_dev = k_dev;
    q.t = t;
    if ((e = dispatch_step<T>(false, check, q, s)) != cudaSuccess) return e;
    if (ev && (e = cudaEventRecord(ev[2], s)) != cudaSuccess) return e;
    return cudaSuccess;
}

template cudaError_t launch_iteration<float>(const IterData<float>&, const IterBufs<float>&, int, int, const int*,
                                             int, bool, cudaStream_t, cudaEvent_t*);
template cudaError_t launch_iteration<double>(const IterData<double>&, const IterBufs<double>&, int, int,
                                              const int*, int, bool, cudaStream_t, cudaEvent_t*);

}  // namespace lpb
