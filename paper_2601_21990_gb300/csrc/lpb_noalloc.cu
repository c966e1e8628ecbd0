// lpb_noalloc.cu -- lpb_scaling_noalloc: the Ruiz + Pock-Chambolle
// equilibration factors of a CSR matrix already in device memory, computed
// without allocating anything.
//
// Its scratch (one statistic per row and per column) is the file-scope
// device array g_noalloc_scratch below, of kNoallocScratch doubles; every
// GPU that loads this library holds it until the process exits.  Host code
// cannot use the array's name as a device address, so the entry point looks
// the address up with cudaGetSymbolAddress once per device (on that device's
// first call) and passes it to the kernels.  All calls share the array: the
// kernels clear what they accumulate into, and calls that overlap on the GPU
// (two streams, two threads) race on it.
//
// The factors equal those lpb_create computes (the same passes and
// formulas); the column statistics here come from atomic updates over the
// rows instead of a transposed copy, so a Pock-Chambolle column sum may
// differ from lpb_create's in the last bits.
#include <mutex>
#include <string>

#include "lpb_internal.h"

namespace lpb {

namespace {

constexpr long long kNoallocScratch = 1ll << 21;  // doubles: m + n must not exceed this
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_noalloc_scratch[kNoallocScratch];

std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[kMaxDevices] = {};

__global__ void k_na_fill(double* d, int count, double v) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) d[i] = v;
}

// One warp per row of A: the row statistic (max or sum of |D_r a D_c|) in a
// fixed order, and the column statistics by atomics.  |.| >= 0, so the bit
// patterns of the doubles order like unsigned integers and atomicMax on
// them is the maximum.
template <bool SUM>
__global__ void k_na_stats(const int* __restrict__ rp, const int* __restrict__ ci, const double* __restrict__ v,
                           int rows, const double* __restrict__ d_r, const double* __restrict__ d_c,
                           double* __restrict__ row_stat, double* __restrict__ col_stat) {
    const int warps = gridDim.x * blockDim.x / 32;
    const int lane = threadIdx.x & 31;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) / 32; i < rows; i += warps) {
        double acc = 0.0;
        for (int e = rp[i] + lane; e < rp[i + 1]; e += 32) {
            const int j = ci[e];
            const double a = fabs(d_r[i] * v[e] * d_c[j]);
            acc = SUM ? acc + a : fmax(acc, a);
            if (SUM) atomicAdd(&col_stat[j], a);
            else atomicMax(reinterpret_cast<unsigned long long*>(&col_stat[j]), (unsigned long long)__double_as_longlong(a));
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double t = __shfl_down_sync(0xffffffffu, acc, o);
            acc = SUM ? acc + t : fmax(acc, t);
        }
        if (lane == 0) row_stat[i] = acc;
    }
}

__global__ void k_na_apply(double* __restrict__ d, const double* __restrict__ stat, int count) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
        if (stat[i] > 0.0) d[i] /= sqrt(stat[i]);
}

int blocks(long long work, int threads) {
    long long g = (work + threads - 1) / threads;
    return (int)(g < 1 ? 1 : (g > 4096 ? 4096 : g));
}

}  // namespace

}  // namespace lpb

using namespace lpb;

extern "C" lpb_err lpb_scaling_noalloc(int32_t m, int32_t n, int32_t nnz, const int32_t* row_ptr_dev,
                                       const int32_t* col_idx_dev, const double* vals_dev, int32_t ruiz_iters,
                                       int32_t pock_chambolle, double* d_row_dev, double* d_col_dev,
                                       void* cuda_stream) {
    if (m < 0 || n < 1 || nnz < 0 || ruiz_iters < 0) {
        set_last_error("lpb_scaling_noalloc: need m >= 0, n >= 1, nnz >= 0, ruiz_iters >= 0");
        return LPB_ERR_INVALID_ARG;
    }
    if ((long long)m + (long long)n > kNoallocScratch) {
        set_last_error("lpb_scaling_noalloc: m + n exceeds the 2097152 statistics its fixed scratch holds");
        return LPB_ERR_INVALID_ARG;
    }
    if (!row_ptr_dev || !d_col_dev || (m > 0 && !d_row_dev) || (nnz > 0 && (!col_idx_dev || !vals_dev))) {
        set_last_error("lpb_scaling_noalloc: a required device pointer is NULL");
        return LPB_ERR_INVALID_ARG;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        set_last_error("lpb_scaling_noalloc: no usable current CUDA device");
        return LPB_ERR_CUDA;
    }
    double* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_ptr[dev]) {
            // the device address of the file-scope array on this (current) device
            e = cudaGetSymbolAddress((void**)&g_noalloc_ptr[dev], g_noalloc_scratch);
            if (e != cudaSuccess) {
                g_noalloc_ptr[dev] = nullptr;
                set_last_error((std::string("lpb_scaling_noalloc: cudaGetSymbolAddress: ") +
                                     cudaGetErrorString(e)).c_str());
                return LPB_ERR_CUDA;
            }
        }
        scratch = g_noalloc_ptr[dev];
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    double* row_stat = scratch;
    double* col_stat = scratch + m;
    if (m > 0) k_na_fill<<<blocks(m, 256), 256, 0, s>>>(d_row_dev, m, 1.0);
    k_na_fill<<<blocks(n, 256), 256, 0, s>>>(d_col_dev, n, 1.0);
    // as lpb_create: ruiz_iters max-passes, then one sum-pass; both statistics
    // of a pass from the same scaled matrix, then both factors updated
    for (int it = 0; it < ruiz_iters + (pock_chambolle ? 1 : 0); ++it) {
        const bool pc = it >= ruiz_iters;
        k_na_fill<<<blocks(n, 256), 256, 0, s>>>(col_stat, n, 0.0);  // accumulated by atomics: clear first
        if (m > 0) {
            if (pc) k_na_stats<true><<<blocks((long long)m * 32, 256), 256, 0, s>>>(row_ptr_dev, col_idx_dev, vals_dev, m, d_row_dev, d_col_dev, row_stat, col_stat);
            else k_na_stats<false><<<blocks((long long)m * 32, 256), 256, 0, s>>>(row_ptr_dev, col_idx_dev, vals_dev, m, d_row_dev, d_col_dev, row_stat, col_stat);
            k_na_apply<<<blocks(m, 256), 256, 0, s>>>(d_row_dev, row_stat, m);
        }
        k_na_apply<<<blocks(n, 256), 256, 0, s>>>(d_col_dev, col_stat, n);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_error((std::string("lpb_scaling_noalloc: ") + cudaGetErrorString(e)).c_str());
        return LPB_ERR_CUDA;
    }
    return LPB_OK;
}
