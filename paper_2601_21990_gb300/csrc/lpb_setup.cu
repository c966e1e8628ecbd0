// lpb_setup.cu -- once-per-matrix device work of lpb_create:
//   transpose of A (A and A^T are both stored, Sec. 6 "Implementation details"),
//   Ruiz + Pock-Chambolle equilibration, scaled values and vectors,
//   power iteration for ||A~||_2 (eta = 0.998 / ||A~||_2, Sec. 4 "Step-size"),
//   lists of long rows for the SpMM kernels.
// Every kernel is deterministic: sums run in a fixed order, the transpose is
// sorted by the original entry index inside each row of A^T.
#include <algorithm>
#include <climits>
#include <cstdio>
#include <vector>

#include "lpb_internal.h"

namespace lpb {

namespace {

constexpr unsigned kFull = 0xffffffffu;


// ---------------------------------------------------------------------------
// exclusive scan of int32 (block = 1024 threads, 2 elements per thread)
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 1024;
constexpr int kScanTile = 2 * kScanThreads;

__global__ void k_scan_tile(const int* __restrict__ in, int* __restrict__ out, int count,
                            int* __restrict__ tile_sums) {
    __shared__ int warp_tot[kScanThreads / 32];
    const int base = blockIdx.x * kScanTile + 2 * threadIdx.x;
    int a0 = base < count ? in[base] : 0;
    int a1 = base + 1 < count ? in[base + 1] : 0;
    int local = a0 + a1;
    // inclusive warp scan of `local`
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int inc = local;
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int w = warp_tot[lane];
        int wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(kFull, wi, o);
            if (lane >= o) wi += t;
        }
        warp_tot[lane] = wi - w;  // exclusive prefix of warp totals
    }
    __syncthreads();
    int excl = inc - local + warp_tot[warp];
    if (base < count) out[base] = excl;
    if (base + 1 < count) out[base + 1] = excl + a0;
    if (threadIdx.x == kScanThreads - 1 && tile_sums) tile_sums[blockIdx.x] = excl + local;
}

__global__ void k_scan_add(int* __restrict__ out, int count, const int* __restrict__ tile_offs) {
    const int base = blockIdx.x * kScanTile + 2 * threadIdx.x;
    const int add = tile_offs[blockIdx.x];
    if (base < count) out[base] += add;
    if (base + 1 < count) out[base + 1] += add;
}

__global__ void k_copy_total(const int* in_last, const int* out_last, int* total) {
    *total = *in_last + *out_last;
}

// ---------------------------------------------------------------------------
// transpose
// ---------------------------------------------------------------------------
__global__ void k_count_cols(const int* __restrict__ ci, int nnz, int* __restrict__ cnt) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += gridDim.x * blockDim.x)
        atomicAdd(&cnt[ci[e]], 1);
}

// one warp per row of A: every entry takes a slot in its column's segment
__global__ void k_fill_slots(const int* __restrict__ rp, const int* __restrict__ ci, int rows,
                             const int* __restrict__ rp_t, int* __restrict__ cursor, int* __restrict__ key) {
    const int warps = gridDim.x * blockDim.x / 32;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) / 32; i < rows; i += warps) {
        for (int e = rp[i] + (threadIdx.x & 31); e < rp[i + 1]; e += 32) {
            int j = ci[e];
            int pos = rp_t[j] + atomicAdd(&cursor[j], 1);
            key[pos] = e;
        }
    }
}

// segments of <= 32 keys: one warp, bitonic network in registers
__global__ void k_segsort_warp(const int* __restrict__ seg, int nseg, int* __restrict__ key) {
    const int warps = gridDim.x * blockDim.x / 32;
    const int lane = threadIdx.x & 31;
    for (int s = (blockIdx.x * blockDim.x + threadIdx.x) / 32; s < nseg; s += warps) {
        const int beg = seg[s], len = seg[s + 1] - beg;
        if (len <= 1 || len > 32) continue;
        int v = lane < len ? key[beg + lane] : INT_MAX;
        for (int k = 2; k <= 32; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                int o = __shfl_xor_sync(kFull, v, j);
                bool asc = (lane & k) == 0, lower = (lane & j) == 0;
                v = (asc == lower) ? min(v, o) : max(v, o);
            }
        if (lane < len) key[beg + lane] = v;
    }
}

// segments of 33..2048 keys: one block, bitonic network in shared memory
constexpr int kSegBlock = 2048;
__global__ void k_segsort_block(const int* __restrict__ seg, int nseg, int* __restrict__ key) {
    __shared__ int buf[kSegBlock];
    for (int s = blockIdx.x; s < nseg; s += gridDim.x) {
        const int beg = seg[s], len = seg[s + 1] - beg;
        if (len <= 32 || len > kSegBlock) continue;
        int p = 64;
        while (p < len) p <<= 1;
        for (int i = threadIdx.x; i < p; i += blockDim.x) buf[i] = i < len ? key[beg + i] : INT_MAX;
        __syncthreads();
        for (int k = 2; k <= p; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = threadIdx.x; i < p; i += blockDim.x) {
                    int q = i ^ j;
                    if (q > i) {
                        bool asc = (i & k) == 0;
                        int a = buf[i], b = buf[q];
                        if ((a > b) == asc) { buf[i] = b; buf[q] = a; }
                    }
                }
                __syncthreads();
            }
        for (int i = threadIdx.x; i < len; i += blockDim.x) key[beg + i] = buf[i];
        __syncthreads();
    }
}

__device__ int lower_bound_i(const int* a, int n, int v) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// segments of > 2048 keys: one block, bottom-up merge sort through `tmp`
// (keys are distinct entry indices, so a key's rank in the other run fixes
// its output position)
__global__ void k_segsort_big(const int* __restrict__ seg, int nseg, int* __restrict__ key, int* __restrict__ tmp) {
    for (int s = blockIdx.x; s < nseg; s += gridDim.x) {
        const int beg = seg[s], len = seg[s + 1] - beg;
        if (len <= kSegBlock) continue;
        int* src = key + beg;
        int* dst = tmp + beg;
        for (int w = 1; w < len; w <<= 1) {
            for (int p = threadIdx.x; p < len; p += blockDim.x) {
                int lo = (p / (2 * w)) * (2 * w);
                int mid = min(lo + w, len), hi = min(lo + 2 * w, len);
                int v = src[p];
                int pos = p < mid ? (p - lo) + lower_bound_i(src + mid, hi - mid, v)
                                  : (p - mid) + lower_bound_i(src + lo, mid - lo, v);
                dst[lo + pos] = v;
            }
            __syncthreads();
            int* t = src; src = dst; dst = t;
        }
        if (src != key + beg)
            for (int p = threadIdx.x; p < len; p += blockDim.x) key[beg + p] = src[p];
        __syncthreads();
    }
}

// A^T entry at `pos` comes from A entry key[pos]: its column in A^T is the
// row of that entry in A (binary search in row_ptr), its value is A's value.
__global__ void k_finish_transpose(const int* __restrict__ rp, int rows, const int* __restrict__ key, int nnz,
                                   const double* __restrict__ vals, int* __restrict__ ci_t,
                                   double* __restrict__ vals_t) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += gridDim.x * blockDim.x) {
        int e = key[p];
        int lo = 0, hi = rows;  // last row with rp[row] <= e
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (rp[mid] <= e) lo = mid; else hi = mid;
        }
        ci_t[p] = lo;
        vals_t[p] = vals[e];
    }
}

// ---------------------------------------------------------------------------
// long-row lists
// ---------------------------------------------------------------------------
__global__ void k_long_flags(const int* __restrict__ rp, int rows, int thr, int* __restrict__ flag) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += gridDim.x * blockDim.x)
        flag[i] = (rp[i + 1] - rp[i]) > thr ? 1 : 0;
}

__global__ void k_long_lengths(const int* __restrict__ rp, const int* __restrict__ rows, int count,
                               int* __restrict__ len) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
        len[i] = rp[rows[i] + 1] - rp[rows[i]];
}

__global__ void k_long_scatter(const int* __restrict__ flag, const int* __restrict__ pos, int rows,
                               int* __restrict__ list) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += gridDim.x * blockDim.x)
        if (flag[i]) list[pos[i]] = i;
}

// ---------------------------------------------------------------------------
// equilibration
// ---------------------------------------------------------------------------
// One warp per CSR row: max or sum of |D_r[i] * a * D_c[j]| where, for the
// CSR of A^T, the row is a variable j and the column a constraint i (the
// product is always formed in the order D_r * a * D_c).
template <bool SUM>
__global__ void k_row_stat(const int* __restrict__ rp, const int* __restrict__ ci, const double* __restrict__ v,
                           int rows, const double* __restrict__ d_row, const double* __restrict__ d_col,
                           bool rows_are_constraints, double* __restrict__ out) {
    const int warps = gridDim.x * blockDim.x / 32;
    const int lane = threadIdx.x & 31;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) / 32; i < rows; i += warps) {
        double acc = 0.0;
        for (int e = rp[i] + lane; e < rp[i + 1]; e += 32) {
            int j = ci[e];
            double a = rows_are_constraints ? fabs(d_row[i] * v[e] * d_col[j]) : fabs(d_col[j] * v[e] * d_row[i]);
            acc = SUM ? acc + a : fmax(acc, a);
        }
        for (int o = 16; o > 0; o >>= 1) {
            double t = __shfl_down_sync(kFull, acc, o);
            acc = SUM ? acc + t : fmax(acc, t);
        }
        if (lane == 0) out[i] = acc;
    }
}

__global__ void k_apply_scale(double* __restrict__ d, const double* __restrict__ stat, int count) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
        if (stat[i] > 0.0) d[i] /= sqrt(stat[i]);
}

__global__ void k_fill_d(double* d, int count, double v) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) d[i] = v;
}

// scaled values: warp per row, D_r[i] * a * D_c[j] with i the constraint
__global__ void k_scale_vals(const int* __restrict__ rp, const int* __restrict__ ci, const double* __restrict__ v,
                             int rows, const double* __restrict__ d_r, const double* __restrict__ d_c,
                             bool rows_are_constraints, double* __restrict__ o64, float* __restrict__ o32) {
    const int warps = gridDim.x * blockDim.x / 32;
    const int lane = threadIdx.x & 31;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) / 32; i < rows; i += warps) {
        for (int e = rp[i] + lane; e < rp[i + 1]; e += 32) {
            int j = ci[e];
            double s = rows_are_constraints ? d_r[i] * v[e] * d_c[j] : d_r[j] * v[e] * d_c[i];
            o64[e] = s;
            if (o32) o32[e] = (float)s;
        }
    }
}

__global__ void k_scale_vectors(int m, int n, const double* __restrict__ d_r, const double* __restrict__ d_c,
                                const double* __restrict__ c, const double* __restrict__ l,
                                const double* __restrict__ u, const double* __restrict__ xl,
                                const double* __restrict__ xu, double* cs, double* ls, double* us, double* xls,
                                double* xus) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < max(m, n); i += gridDim.x * blockDim.x) {
        if (i < n) {
            cs[i] = d_c[i] * c[i];
            xls[i] = xl[i] / d_c[i];
            xus[i] = xu[i] / d_c[i];
        }
        if (i < m) {
            ls[i] = d_r[i] * l[i];
            us[i] = d_r[i] * u[i];
        }
    }
}

__global__ void k_to_f32(const double* __restrict__ in, float* __restrict__ out, int count) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) out[i] = (float)in[i];
}

// ---------------------------------------------------------------------------
// deterministic two-stage sums
// ---------------------------------------------------------------------------
constexpr int kSumBlocks = 256;
constexpr int kSumThreads = 256;

__device__ __forceinline__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (warp == 0) {
        t = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(kFull, t, o);
    }
    __syncthreads();
    return t;  // valid in thread 0
}

// mode 0: sum v^2; mode 1: sum over rows of b~_i^2 (finite bound of larger magnitude)
__global__ void k_sum_stage1(const double* __restrict__ a, const double* __restrict__ b, int count, int mode,
                             double* __restrict__ part) {
    __shared__ double sh[32];
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        if (mode == 0) {
            acc += a[i] * a[i];
        } else {
            double l = a[i], u = b[i], r = 0.0;
            bool fl = isfinite(l), fu = isfinite(u);
            if (fl && fu) r = fabs(l) > fabs(u) ? l : u;
            else if (fl) r = l;
            else if (fu) r = u;
            acc += r * r;
        }
    }
    double t = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void k_sum_stage2(const double* __restrict__ part, int count, double* __restrict__ out) {
    __shared__ double sh[32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) acc += part[i];
    double t = block_sum(acc, sh);
    if (threadIdx.x == 0) *out = t;
}

// ---------------------------------------------------------------------------
// power iteration
// ---------------------------------------------------------------------------
// SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): the index-th output of the
// generator whose state starts at `seed`.
__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t index) {
    uint64_t z = seed + (index + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_power_init(double* v, int n, uint64_t seed) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        v[j] = 2.0 * ((double)(splitmix64(seed, (uint64_t)j) >> 11) * 0x1.0p-53) - 1.0;
}

// One product of A~^T A~ takes two launches of k_power_spmv.  Each block
// leaves its share of the squared norm of the result as one partial; the
// last block to finish (an atomic ticket, no waiting) adds the partials in
// block order and writes the norm to a scalar the next launch reads.  The
// grid is fixed at kPowBlocks plus one block per long row, so the rows each
// block covers and the order of every sum are the same on every run.  The normalisation v = w / ||w|| is
// applied after the forward product, u = (A~ w) / ||w||, so no launch writes
// v and none only reduces.
//
// The short-row blocks of a launch: one per kPowRows rows, at least
// kPowBlocks and at most kPowBlocksMax (a function of the row count alone,
// so still the same on every run).  Each row group walks its rows one after
// another, a chain of dependent loads per row: on the 1M x 2M strong-
// branching matrix the fixed 512 blocks gave each row group 61 (A~) and
// 122 (A~^T) rows; matrices of up to 131k rows keep 512 blocks, the best of
// a sweep on the 20k-row and 100k-row matrices.
#ifndef LPB_POW_BLOCKS
#define LPB_POW_BLOCKS 512
#endif
#ifndef LPB_POW_BLOCKS_MAX
#define LPB_POW_BLOCKS_MAX 4096
#endif
#ifndef LPB_POW_ROWS
#define LPB_POW_ROWS 256
#endif
#ifndef LPB_POW_GROUP
#define LPB_POW_GROUP 8
#endif
constexpr int kPowBlocks = LPB_POW_BLOCKS;
constexpr int kPowBlocksMax = LPB_POW_BLOCKS_MAX;
constexpr int kPowRows = LPB_POW_ROWS;
constexpr int kPowThreads = 256;
static_assert(kPowBlocks <= kPowBlocksMax, "power grid bounds");
inline int pow_blocks(int rows) {
    const long long b = ((long long)rows + kPowRows - 1) / kPowRows;
    return (int)(b < kPowBlocks ? kPowBlocks : b > kPowBlocksMax ? kPowBlocksMax : b);
}
constexpr int kPowGroup = LPB_POW_GROUP;  // lanes per row
static_assert(kPowGroup >= 1 && kPowGroup <= 32 && (kPowGroup & (kPowGroup - 1)) == 0, "lanes per row: a power of 2");

// The last of the grid's blocks to call this (after writing part[blockIdx.x])
// sets *nrm = sqrt(sum of the partials in block order), records it at
// hist[slot] when hist is given, and rearms the ticket.
__device__ __forceinline__ void finish_norm(double* part, unsigned* __restrict__ ticket,
                                            double* __restrict__ nrm, double* __restrict__ hist, int slot,
                                            double* sh) {
    __shared__ bool last;
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double acc = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) acc += __ldcg(part + i);
    const double tot = block_sum(acc, sh);
    if (threadIdx.x == 0) {
        const double nr = sqrt(tot);
        *nrm = nr;
        if (hist) hist[slot] = nr;
        *ticket = 0u;
    }
}

// y = M x (divided by *nrm_x when nrm_x is given); *nrm_y = ||y|| (and
// hist[slot] = ||y|| when hist is given).  Blocks [0, n_long) take one of the
// rows longer than long_thr (a list of them) each, all threads striding over
// its entries; the other blocks take the remaining rows with kPowGroup lanes
// per row.
__global__ void __launch_bounds__(kPowThreads) k_power_spmv(const int* __restrict__ rp, const int* __restrict__ ci,
                                                            const double* __restrict__ v, int rows,
                                                            const int* __restrict__ long_rows, int n_long,
                                                            int long_thr, const double* __restrict__ x,
                                                            const double* __restrict__ nrm_x,
                                                            double* __restrict__ y, double* part,
                                                            unsigned* __restrict__ ticket, double* __restrict__ nrm_y,
                                                            double* __restrict__ hist, int slot) {
    __shared__ double sh[32];
    const double nx = nrm_x ? *nrm_x : 1.0;
    if ((int)blockIdx.x < n_long) {
        const int i = long_rows[blockIdx.x];
        double acc = 0.0;
        for (int e = rp[i] + threadIdx.x; e < rp[i + 1]; e += blockDim.x) acc += v[e] * x[ci[e]];
        const double t = block_sum(acc, sh);
        if (threadIdx.x == 0) {
            const double yi = !nrm_x ? t : (nx > 0.0 ? t / nx : 0.0);
            y[i] = yi;
            part[blockIdx.x] = yi * yi;
        }
        finish_norm(part, ticket, nrm_y, hist, slot, sh);
        return;
    }
    constexpr int kRowsPerWarp = 32 / kPowGroup;
    const int lane = threadIdx.x % kPowGroup, sub = (threadIdx.x & 31) / kPowGroup;
    const int warp = (((int)blockIdx.x - n_long) * blockDim.x + threadIdx.x) >> 5;
    const int warps = (((int)gridDim.x - n_long) * blockDim.x) >> 5;
    double sq = 0.0;  // the group's rows in order, in its first lane
    // the loop bound is the same for the whole warp, so every lane reaches the shuffles
    for (int base = warp * kRowsPerWarp; base < rows; base += warps * kRowsPerWarp) {
        const int i = base + sub;
        double acc = 0.0;
        const bool mine = i < rows && rp[i + 1] - rp[i] <= long_thr;
        if (mine)
            for (int e = rp[i] + lane; e < rp[i + 1]; e += kPowGroup) acc += v[e] * x[ci[e]];
        for (int o = kPowGroup / 2; o > 0; o >>= 1) acc += __shfl_down_sync(kFull, acc, o, kPowGroup);
        if (lane == 0 && mine) {
            const double yi = !nrm_x ? acc : (nx > 0.0 ? acc / nx : 0.0);
            y[i] = yi;
            sq += yi * yi;
        }
    }
    const double t = block_sum(sq, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
    finish_norm(part, ticket, nrm_y, hist, slot, sh);
}

// *nrm = ||x|| with the same two-level fixed-order sum
__global__ void __launch_bounds__(kPowThreads) k_power_norm(const double* __restrict__ x, int count,
                                                            double* part, unsigned* __restrict__ ticket,
                                                            double* __restrict__ nrm) {
    __shared__ double sh[32];
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) acc += x[i] * x[i];
    const double t = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
    finish_norm(part, ticket, nrm, nullptr, 0, sh);
}

// Blocks of the Ruiz and Pock-Chambolle row statistics (a warp per row, so
// the grid changes no result): up to 16384, about 8 rows per warp on a
// 1M-row matrix
constexpr int kStatCap = 16384;

inline int grid_for(long long work, int threads, int cap = 4096) {
    long long g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

}  // namespace

// ---------------------------------------------------------------------------
// host wrappers
// ---------------------------------------------------------------------------
cudaError_t exclusive_scan_i32(const int* in, int* out, int count, int* total_dev, cudaStream_t s) {
    if (count <= 0) {
        if (total_dev) return cudaMemsetAsync(total_dev, 0, sizeof(int), s);
        return cudaSuccess;
    }
    const int tiles = (count + kScanTile - 1) / kScanTile;
    int* sums = nullptr;
    int* offs = nullptr;
    cudaError_t e = cudaSuccess;
    if (tiles > 1) {
        if ((e = cudaMallocAsync((void**)&sums, sizeof(int) * tiles * 2, s)) != cudaSuccess) return e;
        offs = sums + tiles;
    }
    k_scan_tile<<<tiles, kScanThreads, 0, s>>>(in, out, count, sums);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (tiles > 1) {
        if ((e = exclusive_scan_i32(sums, offs, tiles, nullptr, s)) != cudaSuccess) return e;
        k_scan_add<<<tiles, kScanThreads, 0, s>>>(out, count, offs);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (total_dev) {
        k_copy_total<<<1, 1, 0, s>>>(in + count - 1, out + count - 1, total_dev);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (sums) e = cudaFreeAsync(sums, s);
    return e;
}

cudaError_t transpose_csr(const Csr& a, const double* a_vals, Csr& at, int* perm_out, cudaStream_t s) {
    // at.rp (cols + 1), at.ci (nnz) and perm_out-sized scratch are allocated by the caller;
    // perm_out receives the A^T slot -> A entry map, vals_t is written into at.v64.
    cudaError_t e;
    const int nnz = a.nnz, cols = a.cols;
    int *cnt = nullptr, *cursor = nullptr, *tmp = nullptr;
    if ((e = cudaMallocAsync((void**)&cnt, sizeof(int) * (size_t)(cols + 1) * 2, s)) != cudaSuccess) return e;
    cursor = cnt + cols + 1;
    if ((e = cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)(cols + 1) * 2, s)) != cudaSuccess) return e;
    if (nnz > 0) {
        k_count_cols<<<grid_for(nnz, 256), 256, 0, s>>>(a.ci, nnz, cnt);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((e = exclusive_scan_i32(cnt, at.rp, cols + 1, nullptr, s)) != cudaSuccess) return e;
    if (nnz > 0) {
        k_fill_slots<<<grid_for((long long)a.rows * 32, 256), 256, 0, s>>>(a.rp, a.ci, a.rows, at.rp, cursor, perm_out);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        k_segsort_warp<<<grid_for((long long)cols * 32, 256), 256, 0, s>>>(at.rp, cols, perm_out);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        k_segsort_block<<<grid_for(cols, 1, 1024), 1024, 0, s>>>(at.rp, cols, perm_out);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = cudaMallocAsync((void**)&tmp, sizeof(int) * (size_t)nnz, s)) != cudaSuccess) return e;
        k_segsort_big<<<grid_for(cols, 1, 256), 1024, 0, s>>>(at.rp, cols, perm_out, tmp);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        k_finish_transpose<<<grid_for(nnz, 256), 256, 0, s>>>(a.rp, a.rows, perm_out, nnz, a_vals, at.ci, at.v64);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = cudaFreeAsync(tmp, s)) != cudaSuccess) return e;
    }
    return cudaFreeAsync(cnt, s);
}

// Segments of the long rows for the step kernels: long row i (length len_i)
// gets ceil(len_i / kStepSeg) segments; blocks are listed segment-major.
static cudaError_t build_long_segments(Csr& a, cudaStream_t s) {
    cudaError_t e;
    if (a.n_long == 0) return cudaSuccess;
    std::vector<int> len(a.n_long);
    int* len_dev = nullptr;
    if ((e = cudaMallocAsync((void**)&len_dev, sizeof(int) * a.n_long, s)) != cudaSuccess) return e;
    k_long_lengths<<<grid_for(a.n_long, 256), 256, 0, s>>>(a.rp, a.long_rows, a.n_long, len_dev);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(len.data(), len_dev, sizeof(int) * a.n_long, cudaMemcpyDeviceToHost, s)) !=
        cudaSuccess)
        return e;
    if ((e = cudaFreeAsync(len_dev, s)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    std::vector<int> seg0(a.n_long + 1, 0);
    int max_ns = 0;
    for (int i = 0; i < a.n_long; ++i) {
        const int ns = std::max(1, (len[i] + kStepSeg - 1) / kStepSeg);
        seg0[i + 1] = seg0[i] + ns;
        max_ns = std::max(max_ns, ns);
    }
    std::vector<int> lseg;
    lseg.reserve(2 * (size_t)seg0[a.n_long]);
    for (int sg = 0; sg < max_ns; ++sg)
        for (int i = 0; i < a.n_long; ++i)
            if (sg < seg0[i + 1] - seg0[i]) {
                lseg.push_back(i);
                lseg.push_back(sg);
            }
    a.n_lblocks = seg0[a.n_long];
    if ((e = cudaMalloc((void**)&a.lseg, sizeof(int) * lseg.size())) != cudaSuccess) return e;
    if ((e = cudaMalloc((void**)&a.lseg0, sizeof(int) * seg0.size())) != cudaSuccess) return e;
    if ((e = cudaMemcpy(a.lseg, lseg.data(), sizeof(int) * lseg.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
        return e;
    return cudaMemcpy(a.lseg0, seg0.data(), sizeof(int) * seg0.size(), cudaMemcpyHostToDevice);
}

void free_long_rows(Csr& a) {
    if (a.long_rows) cudaFree(a.long_rows);
    if (a.lseg) cudaFree(a.lseg);
    if (a.lseg0) cudaFree(a.lseg0);
    a.long_rows = nullptr;
    a.lseg = a.lseg0 = nullptr;
    a.n_long = a.n_lblocks = 0;
}

cudaError_t build_long_rows(Csr& a, cudaStream_t s) {
    cudaError_t e;
    if (a.long_rows || a.lseg) {
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
        free_long_rows(a);
    }
    a.n_long = 0;
    a.n_lblocks = 0;
    if (a.rows == 0) return cudaSuccess;
    int *flag = nullptr, *total = nullptr;
    if ((e = cudaMallocAsync((void**)&flag, sizeof(int) * ((size_t)a.rows * 2 + 1), s)) != cudaSuccess) return e;
    int* pos = flag + a.rows;
    total = pos + a.rows;
    k_long_flags<<<grid_for(a.rows, 256), 256, 0, s>>>(a.rp, a.rows, a.long_thr, flag);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = exclusive_scan_i32(flag, pos, a.rows, total, s)) != cudaSuccess) return e;
    int h_total = 0;
    if ((e = cudaMemcpyAsync(&h_total, total, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    a.n_long = h_total;
    if (h_total > 0) {
        if ((e = cudaMalloc((void**)&a.long_rows, sizeof(int) * (size_t)h_total)) != cudaSuccess) return e;
        k_long_scatter<<<grid_for(a.rows, 256), 256, 0, s>>>(flag, pos, a.rows, a.long_rows);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((e = cudaFreeAsync(flag, s)) != cudaSuccess) return e;
    return build_long_segments(a, s);
}

cudaError_t ruiz_pock_chambolle(const Csr& a, const double* a_vals, const Csr& at, const double* at_vals,
                                int ruiz_iters, int pock_chambolle, double* d_r, double* d_c, double* tmp_r,
                                double* tmp_c, cudaStream_t s) {
    cudaError_t e;
    const int m = a.rows, n = a.cols;
    if (m > 0) k_fill_d<<<grid_for(m, 256), 256, 0, s>>>(d_r, m, 1.0);
    k_fill_d<<<grid_for(n, 256), 256, 0, s>>>(d_c, n, 1.0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    for (int it = 0; it < ruiz_iters + (pock_chambolle ? 1 : 0); ++it) {
        const bool pc = it >= ruiz_iters;
        // both statistics from the same A~, then both factors updated
        if (m > 0) {
            if (pc) k_row_stat<true><<<grid_for((long long)m * 32, 256, kStatCap), 256, 0, s>>>(a.rp, a.ci, a_vals, m, d_r, d_c, true, tmp_r);
            else k_row_stat<false><<<grid_for((long long)m * 32, 256, kStatCap), 256, 0, s>>>(a.rp, a.ci, a_vals, m, d_r, d_c, true, tmp_r);
        }
        if (pc) k_row_stat<true><<<grid_for((long long)n * 32, 256, kStatCap), 256, 0, s>>>(at.rp, at.ci, at_vals, n, d_c, d_r, false, tmp_c);
        else k_row_stat<false><<<grid_for((long long)n * 32, 256, kStatCap), 256, 0, s>>>(at.rp, at.ci, at_vals, n, d_c, d_r, false, tmp_c);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (m > 0) k_apply_scale<<<grid_for(m, 256), 256, 0, s>>>(d_r, tmp_r, m);
        k_apply_scale<<<grid_for(n, 256), 256, 0, s>>>(d_c, tmp_c, n);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t scale_values(const Csr& a, const double* a_vals, const double* d_r, const double* d_c,
                         bool rows_are_constraints, double* out64, float* out32, cudaStream_t s) {
    if (a.rows == 0 || a.nnz == 0) return cudaSuccess;
    k_scale_vals<<<grid_for((long long)a.rows * 32, 256), 256, 0, s>>>(a.rp, a.ci, a_vals, a.rows, d_r, d_c,
                                                                         rows_are_constraints, out64, out32);
    return cudaGetLastError();
}

cudaError_t scale_vectors(int m, int n, const double* d_r, const double* d_c, const double* c, const double* l,
                          const double* u, const double* xl, const double* xu, double* cs, double* ls, double* us,
                          double* xls, double* xus, cudaStream_t s) {
    k_scale_vectors<<<grid_for(m > n ? m : n, 256), 256, 0, s>>>(m, n, d_r, d_c, c, l, u, xl, xu, cs, ls, us, xls, xus);
    return cudaGetLastError();
}

cudaError_t convert_f32(const double* in, float* out, int count, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    k_to_f32<<<grid_for(count, 256), 256, 0, s>>>(in, out, count);
    return cudaGetLastError();
}

namespace {
// hi = value rounded to FP32, lo = the rounding error rounded to FP32; an
// infinite value is {+-inf, 0}
__global__ void k_split_df(const double* __restrict__ in, df* __restrict__ out, int count, bool recip) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const double v = recip ? 1.0 / in[i] : in[i];
        const float hi = (float)v;
        out[i] = df{hi, isfinite(v) && isfinite(hi) ? (float)(v - (double)hi) : 0.0f};
    }
}
__global__ void k_split_lo(const double* __restrict__ v64, const float* __restrict__ v32, float* __restrict__ lo,
                           int count) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
        lo[i] = (float)(v64[i] - (double)v32[i]);
}
}  // namespace

cudaError_t split_df(const double* in, df* out, int count, bool recip, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    k_split_df<<<grid_for(count, 256), 256, 0, s>>>(in, out, count, recip);
    return cudaGetLastError();
}

cudaError_t split_lo(const double* v64, const float* v32, float* lo, int count, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    k_split_lo<<<grid_for(count, 256), 256, 0, s>>>(v64, v32, lo, count);
    return cudaGetLastError();
}

static cudaError_t two_stage(const double* a, const double* b, int count, int mode, double* out_dev, double* part,
                             cudaStream_t s) {
    k_sum_stage1<<<kSumBlocks, kSumThreads, 0, s>>>(a, b, count, mode, part);
    k_sum_stage2<<<1, kSumThreads, 0, s>>>(part, kSumBlocks, out_dev);
    return cudaGetLastError();
}

cudaError_t sq_norm(const double* v, int count, double* out_dev, cudaStream_t s) {
    double* part = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&part, sizeof(double) * kSumBlocks, s);
    if (e != cudaSuccess) return e;
    if ((e = two_stage(v, nullptr, count, 0, out_dev, part, s)) != cudaSuccess) return e;
    return cudaFreeAsync(part, s);
}

cudaError_t rhs_norm2(const double* ls, const double* us, int m, double* out_dev, cudaStream_t s) {
    double* part = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&part, sizeof(double) * kSumBlocks, s);
    if (e != cudaSuccess) return e;
    if ((e = two_stage(ls, us, m, 1, out_dev, part, s)) != cudaSuccess) return e;
    return cudaFreeAsync(part, s);
}

// (at most nnz / kLongSeg rows have more than kLongSeg entries: one block
// and one norm partial each)
size_t power_work_doubles(int m, int n, long long nnz, int max_iter) {
    return (size_t)n + (size_t)(m > 0 ? m : 1) + (size_t)kPowBlocksMax + (size_t)(nnz / kLongSeg + 1) + 3 +
           2 * ((size_t)max_iter + 1);
}

// Power iteration on A~^T A~: sigma_est = ||A~ v|| for unit v.  Stops at the
// first product where the estimate moves by <= tol relative, or when
// ||A~^T A~ v|| = 0, or after max_iter products.  The host looks at the
// history every kChunk products; products past the stopping point change
// nothing that is returned.
static cudaError_t power_iterate(const Csr& a, const Csr& at, const Csr& va, const Csr& vat, int max_iter,
                                 double tol, uint64_t seed, double* part, double* nrm_u, double* nrm_w,
                                 unsigned* ticket, double* hist_est, double* hist_nw, double* w, double* u,
                                 double* est_out, int* iters_out, cudaStream_t s);

cudaError_t power_norm(const Csr& a, const Csr& at, int max_iter, double tol, uint64_t seed, double* work,
                       double* est_out, int* iters_out, cudaStream_t s) {
    const int m = a.rows, n = a.cols;
    // work layout (power_work_doubles): w (n), u (m), part (kPowBlocksMax + nnz / kLongSeg + 1),
    // ||u||, ||w||, the ticket, hist_est, hist_nw (max_iter + 1 each); w starts as the
    // unnormalised start vector
    double* w = work;
    double* u = w + n;
    double* part = u + (m > 0 ? m : 1);
    double* nrm_u = part + kPowBlocksMax + (size_t)a.nnz / kLongSeg + 1;
    double* nrm_w = nrm_u + 1;
    unsigned* ticket = reinterpret_cast<unsigned*>(nrm_w + 1);
    double* hist_est = nrm_w + 2;
    double* hist_nw = hist_est + (max_iter + 1);
    cudaError_t e;
    *est_out = 0.0;
    *iters_out = 0;
    if (m == 0 || a.nnz == 0) return cudaSuccess;
    // the rows of more than kLongSeg entries of A~ and A~^T, one block each
    Csr va = a, vat = at;
    for (Csr* c : {&va, &vat}) {
        c->long_rows = c->lseg = c->lseg0 = nullptr;
        c->long_thr = kLongSeg;
        if ((e = build_long_rows(*c, s)) != cudaSuccess) {
            free_long_rows(va);
            free_long_rows(vat);
            return e;
        }
    }
    e = power_iterate(a, at, va, vat, max_iter, tol, seed, part, nrm_u, nrm_w, ticket, hist_est, hist_nw, w, u,
                      est_out, iters_out, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    free_long_rows(va);
    free_long_rows(vat);
    return e;
}

// The products of power_norm; va and vat list the rows of more than kLongSeg
// entries of A~ and A~^T.
static cudaError_t power_iterate(const Csr& a, const Csr& at, const Csr& va, const Csr& vat, int max_iter,
                                 double tol, uint64_t seed, double* part, double* nrm_u, double* nrm_w,
                                 unsigned* ticket, double* hist_est, double* hist_nw, double* w, double* u,
                                 double* est_out, int* iters_out, cudaStream_t s) {
    const int m = a.rows, n = a.cols;
    cudaError_t e;
    if ((e = cudaMemsetAsync(ticket, 0, sizeof(unsigned), s)) != cudaSuccess) return e;
    k_power_init<<<grid_for(n, 256), 256, 0, s>>>(w, n, seed);
    k_power_norm<<<kPowBlocks, kPowThreads, 0, s>>>(w, n, part, ticket, nrm_w);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // products queued between two looks at the history (products past the
    // stopping point are wasted work)
    constexpr int kChunk = 16;
    std::vector<double> he(kChunk), hn(kChunk);
    double prev = -1.0;
    for (int base = 1; base <= max_iter; base += kChunk) {
        const int last = base + kChunk - 1 < max_iter ? base + kChunk - 1 : max_iter;
        for (int it = base; it <= last; ++it) {
            // u = A~ w / ||w|| (records ||u||), then w = A~^T u (records ||w||)
            // rows of more than kLongSeg entries get a whole block each
            k_power_spmv<<<va.n_long + pow_blocks(m), kPowThreads, 0, s>>>(a.rp, a.ci, a.v64, m, va.long_rows,
                                                                          va.n_long, kLongSeg, w, nrm_w, u, part,
                                                                          ticket, nrm_u, hist_est, it);
            k_power_spmv<<<vat.n_long + pow_blocks(n), kPowThreads, 0, s>>>(at.rp, at.ci, at.v64, n, vat.long_rows,
                                                                           vat.n_long, kLongSeg, u, nullptr, w, part,
                                                                           ticket, nrm_w, hist_nw, it);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        const int cnt = last - base + 1;
        if ((e = cudaMemcpyAsync(he.data(), hist_est + base, sizeof(double) * cnt, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
        if ((e = cudaMemcpyAsync(hn.data(), hist_nw + base, sizeof(double) * cnt, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
        for (int q = 0; q < cnt; ++q) {
            const int it = base + q;
            const double est = he[q];
            *est_out = est;
            *iters_out = it;
            if (!(hn[q] > 0.0)) return cudaSuccess;
            if (prev >= 0.0 && fabs(est - prev) <= tol * est) return cudaSuccess;
            prev = est;
        }
    }
    return cudaSuccess;
}

}  // namespace lpb
