// lpb_iter.cu -- the hot path: one reflected-Halpern PDHG iteration on the
// whole active batch (Sec. 5, Eq. batched_iter and main-iterate).
//
//   primal step  (rows of A~^T, one per variable i; G = A~^T Y^k):
//     X^k_ij = k/(k+1) Xb_ij + X^0_ij/(k+1)   (the previous Halpern update,
//                                              rebuilt from the stored Xb)
//     x^  = Pi_[xlo_ij, xhi_ij](X^k_ij - tau_j (c_ij + G_ij))
//     xb  = 2 x^ - X^k_ij                     (the reflection, also A(2x - x^k))
//     X^{k+1}_ij = (k+1)/(k+2) xb + X^0_ij/(k+2), not stored: the next
//     primal step rebuilds it from xb, which the dual step needs anyway
//     (at k = 0 the weights are 0 and 1, so X^0 itself)
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
//
// The per-column parameters of the block's column tile are staged in shared
// memory once per block.  No FP64 instruction runs in the FP32 kernels
// (GB300 executes FP64 at a small fraction of its FP32 rate); the Halpern
// weights come from a table written by the check kernels.  The kernels are
// instantiated for float (mixed path), double (FP64 path) and dfloat (the
// mixed path's polish phase: double-float values on the FP32 pipe).
#include "lpb_step.h"

namespace lpb {

namespace {

template <typename T, int G, bool CHECK, bool PRIMAL>
__global__ void __launch_bounds__(kBlock, (MinBlocks<T, G, PRIMAL>::v)) k_step(const __grid_constant__ StepArgs<T> a) {
    step_body<T, G, CHECK, PRIMAL>(a, (int)blockIdx.x, (int)blockIdx.y, (int)gridDim.x);
}

template <typename T, int G, bool CHECK, bool PRIMAL>
cudaError_t launch_k(const StepArgs<T>& a, cudaStream_t s) {
    constexpr int V = Vec<T>::V, GPB = kBlock / G, TN = G * V;
    static std::atomic<int> shape[kShapeDevices];  // static storage: starts at 0
    int sms = 0, per_sm = 0;
    const cudaError_t e = launch_shape(shape, k_step<T, G, CHECK, PRIMAL>, &sms, &per_sm);
    if (e != cudaSuccess) return e;
    const int need = (a.rows + GPB - 1) / GPB;
    const int persist = need < sms * per_sm ? need : sms * per_sm;
    const dim3 grid(a.n_lblocks + persist, (a.ncol + TN - 1) / TN);
    return launch_with(k_step<T, G, CHECK, PRIMAL>, grid, a, a.pdl != 0, s);
}

template <typename T, int G>
cudaError_t launch_step(bool primal, bool check, const StepArgs<T>& a, cudaStream_t s) {
    if (a.rows == 0 || a.ncol == 0) return cudaSuccess;
    if (primal) return check ? launch_k<T, G, true, true>(a, s) : launch_k<T, G, false, true>(a, s);
    return check ? launch_k<T, G, true, false>(a, s) : launch_k<T, G, false, false>(a, s);
}

template <typename T>
cudaError_t dispatch_step(bool primal, bool check, const StepArgs<T>& a, int g_shift, cudaStream_t s) {
    switch (row_group_lanes<T>(a.ncol, g_shift)) {
        case 1: return launch_step<T, 1>(primal, check, a, s);
        case 2: return launch_step<T, 2>(primal, check, a, s);
        case 4: return launch_step<T, 4>(primal, check, a, s);
        case 8: return launch_step<T, 8>(primal, check, a, s);
        case 16: return launch_step<T, 16>(primal, check, a, s);
        default: return launch_step<T, 32>(primal, check, a, s);
    }
}

}  // namespace

template <typename T>
cudaError_t launch_iteration(const IterData<T>& d, const IterBufs<T>& b, int ld, int ncol, const T* hal, int t,
                             int ce, int uni, bool check, bool pdl, cudaStream_t s, cudaEvent_t* ev) {
    cudaError_t e;
    long long l2 = 0;
    if ((e = l2_bytes(&l2)) != cudaSuccess) return e;
    StepArgs<T> p = step_args<T>(true, d, b, ld, ncol, hal, t, ce, uni, l2);
    // the first primal step of an interval follows the check's copies
    p.pdl = pdl && t > 0 && !ev;
    if (ev && (e = cudaEventRecord(ev[0], s)) != cudaSuccess) return e;
    if ((e = dispatch_step<T>(true, check, p, d.At.g_shift, s)) != cudaSuccess) return e;
    if (ev && (e = cudaEventRecord(ev[1], s)) != cudaSuccess) return e;
    StepArgs<T> q = step_args<T>(false, d, b, ld, ncol, hal, t, ce, uni, l2);
    q.pdl = pdl && !ev;
    if ((e = dispatch_step<T>(false, check, q, d.A.g_shift, s)) != cudaSuccess) return e;
    if (ev && (e = cudaEventRecord(ev[2], s)) != cudaSuccess) return e;
    return cudaSuccess;
}

template cudaError_t launch_iteration<float>(const IterData<float>&, const IterBufs<float>&, int, int, const float*,
                                             int, int, int, bool, bool, cudaStream_t, cudaEvent_t*);
template cudaError_t launch_iteration<double>(const IterData<double>&, const IterBufs<double>&, int, int,
                                              const double*, int, int, int, bool, bool, cudaStream_t, cudaEvent_t*);
template cudaError_t launch_iteration<dfloat>(const IterData<dfloat>&, const IterBufs<dfloat>&, int, int,
                                              const dfloat*, int, int, int, bool, bool, cudaStream_t, cudaEvent_t*);

}  // namespace lpb
