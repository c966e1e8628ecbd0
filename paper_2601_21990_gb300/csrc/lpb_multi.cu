// lpb_multi.cu -- joint step launches over several matrices.
//
// A joint solve (lpb_solve_multi) runs the batches of several handles, each
// with its own sparse A, iterate blocks, batch width and long-row segments,
// through one primal-step launch and one dual-step launch per iteration
// instead of one pair per handle: LPs of uneven size and iteration count in
// one persistent launch.  The kernel is the step of lpb_iter.cu (the same
// device code, lpb_step.h); a block locates its part in the flattened grid
// and runs that part's step at the place its own grid would give it.  Each
// row is still taken by one row group of the width its part would launch
// with alone and summed in the same order, so every part's iterates are
// bitwise those of its own launches.
#include <algorithm>
#include <vector>

#include "lpb_joint_grid.h"
#include "lpb_step.h"

// resident blocks per SM of the joint kernels with row groups of 8 or more
// lanes, FP32 and FP64 (see MultiMinBlocks)
#ifndef LPB_MULTI_MIN_BLOCKS_F32
#define LPB_MULTI_MIN_BLOCKS_F32 8
#endif
#ifndef LPB_MULTI_MIN_BLOCKS_F64
#define LPB_MULTI_MIN_BLOCKS_F64 7
#endif
// the double-float joint kernels (the joint polish phase): one block fewer
// than the single kernels, whose 72 registers the part lookup would overflow
#ifndef LPB_MULTI_MIN_BLOCKS_DF
#define LPB_MULTI_MIN_BLOCKS_DF 6
#endif

namespace lpb {

namespace {

// The parts of one joint launch.  Part p occupies blocks [block0[p],
// block0[p + 1]) of the flattened grid: its own grid of gx[p] long-row and
// persistent blocks per column tile, tile after tile, in the order in which
// k_step's blockIdx.x and blockIdx.y run.
template <typename T>
struct MultiStepArgs {
    int nparts;
    int block0[kMaxParts + 1];
    int gx[kMaxParts];
    StepArgs<T> part[kMaxParts];
};
// kernel parameters stay within the classic 4 KB limit
static_assert(sizeof(MultiStepArgs<double>) <= 4096, "joint step arguments exceed 4 KB");

// Resident blocks per SM of the joint kernels: those the single-matrix
// kernels reach with their register counts (the part lookup and the
// indexed arguments cost the joint kernels a few registers more).  Row
// groups of 4 lanes or fewer keep the single kernels' bound, where the
// tighter cap would spill.
template <typename T, int G, bool PRIMAL> struct MultiMinBlocks {
    static constexpr int cap = G <= 4 ? 5 : std::is_same<T, float>::value ? LPB_MULTI_MIN_BLOCKS_F32
                                                                           : LPB_MULTI_MIN_BLOCKS_F64;
    static constexpr int v = MinBlocks<T, G, PRIMAL>::v > cap ? MinBlocks<T, G, PRIMAL>::v : cap;
};
template <int G, bool PRIMAL> struct MultiMinBlocks<dfloat, G, PRIMAL> {
    static constexpr int v = LPB_MULTI_MIN_BLOCKS_DF;
};

template <typename T, int G, bool CHECK, bool PRIMAL>
__global__ void __launch_bounds__(kBlock, (MultiMinBlocks<T, G, PRIMAL>::v))
    k_step_multi(const __grid_constant__ MultiStepArgs<T> m) {
    const JointPlace q = joint_place((int)blockIdx.x, m.nparts, m.block0, m.gx);
    step_body<T, G, CHECK, PRIMAL>(m.part[q.part], q.bx, q.by, q.gx);
}

// Each part gets the grid k_step would get for it alone: its long-row
// blocks and up to one wave of persistent blocks per column tile.  Parts
// whose rows need less than a wave (small matrices, which alone leave most
// SMs idle) come first in the grid, so that their blocks run beside the
// first wave of the larger parts' blocks.  Which block takes a row does not
// change the row's arithmetic.
template <typename T, int G, bool CHECK, bool PRIMAL>
cudaError_t launch_multi_k(MultiStepArgs<T>& m, bool pdl, cudaStream_t s) {
    constexpr int V = Vec<T>::V, GPB = kBlock / G, TN = G * V;
    static std::atomic<int> shape[kShapeDevices];  // static storage: starts at 0
    int sms = 0, per_sm = 0;
    const cudaError_t e = launch_shape(shape, k_step_multi<T, G, CHECK, PRIMAL>, &sms, &per_sm);
    if (e != cudaSuccess) return e;
    int nlb[kMaxParts], need[kMaxParts], tiles[kMaxParts];
    for (int p = 0; p < m.nparts; ++p) {
        StepArgs<T>& a = m.part[p];
        a.pdl = pdl ? 1 : 0;
        nlb[p] = a.n_lblocks;
        need[p] = (a.rows + GPB - 1) / GPB;
        tiles[p] = (a.ncol + TN - 1) / TN;
    }
    const long long total = joint_layout(m.nparts, nlb, need, tiles, sms * per_sm, m.block0, m.gx);
    if (total < 0) return cudaErrorInvalidConfiguration;
    if (total == 0) return cudaSuccess;
    return launch_with(k_step_multi<T, G, CHECK, PRIMAL>, dim3((unsigned)total), m, pdl, s);
}

template <typename T, int G>
cudaError_t launch_multi_step(bool primal, bool check, MultiStepArgs<T>& m, bool pdl, cudaStream_t s) {
    if (primal) return check ? launch_multi_k<T, G, true, true>(m, pdl, s) : launch_multi_k<T, G, false, true>(m, pdl, s);
    return check ? launch_multi_k<T, G, true, false>(m, pdl, s) : launch_multi_k<T, G, false, false>(m, pdl, s);
}

template <typename T>
cudaError_t dispatch_multi(int lanes, bool primal, bool check, MultiStepArgs<T>& m, bool pdl, cudaStream_t s) {
    switch (lanes) {
        case 1: return launch_multi_step<T, 1>(primal, check, m, pdl, s);
        case 2: return launch_multi_step<T, 2>(primal, check, m, pdl, s);
        case 4: return launch_multi_step<T, 4>(primal, check, m, pdl, s);
        case 8: return launch_multi_step<T, 8>(primal, check, m, pdl, s);
        case 16: return launch_multi_step<T, 16>(primal, check, m, pdl, s);
        default: return launch_multi_step<T, 32>(primal, check, m, pdl, s);
    }
}

}  // namespace

template <typename T>
cudaError_t launch_iteration_multi(const IterPart<T>* parts, int nparts, int t, bool check, bool pdl,
                                   cudaStream_t s) {
    cudaError_t e;
    long long l2 = 0;
    if ((e = l2_bytes(&l2)) != cudaSuccess) return e;
    // the parts with work, by row-group width, then the fewer rows first
    struct Key {
        int lanes;
        long long rows;
        int part;
    };
    std::vector<Key> order;
    order.reserve(nparts);
    for (int step = 0; step < 2; ++step) {
        const bool primal = step == 0;
        order.clear();
        for (int i = 0; i < nparts; ++i) {
            const Csr& c = primal ? parts[i].d.At : parts[i].d.A;
            if (c.rows > 0 && parts[i].ncol > 0)
                order.push_back({row_group_lanes<T>(parts[i].ncol, c.g_shift), (long long)c.rows, i});
        }
        std::stable_sort(order.begin(), order.end(), [](const Key& x, const Key& y) {
            return x.lanes != y.lanes ? x.lanes < y.lanes : x.rows < y.rows;
        });
        bool first = true;
        for (size_t k = 0; k < order.size();) {
            const int lanes = order[k].lanes;
            MultiStepArgs<T> m{};
            m.nparts = 0;
            while (k < order.size() && order[k].lanes == lanes && m.nparts < kMaxParts) {
                const IterPart<T>& q = parts[order[k].part];
                m.part[m.nparts++] = step_args<T>(primal, q.d, q.b, q.ld, q.ncol, q.hal, t, q.ce, q.uni, l2);
                ++k;
            }
            // the interval's first primal launch follows the checks, which
            // write what its prologue reads: it is not a programmatic dependent
            const bool dep = pdl && !(primal && t == 0 && first);
            first = false;
            if ((e = dispatch_multi<T>(lanes, primal, check, m, dep, s)) != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

template cudaError_t launch_iteration_multi<float>(const IterPart<float>*, int, int, bool, bool, cudaStream_t);
template cudaError_t launch_iteration_multi<double>(const IterPart<double>*, int, int, bool, bool, cudaStream_t);
template cudaError_t launch_iteration_multi<dfloat>(const IterPart<dfloat>*, int, int, bool, bool, cudaStream_t);

}  // namespace lpb
