// lpb_joint_grid.h -- the flattened 1-D grid of a joint step launch
// (lpb_multi.cu): where each part's blocks sit, and which part and which
// place of that part's own grid a block takes.  Host and device code; the
// layout is checked on the host by tests/native/joint_grid_test.cu.
#pragma once

#include <climits>

#ifdef __CUDACC__
#define LPB_JG_HD __host__ __device__
#else
#define LPB_JG_HD
#endif

namespace lpb {

// Part p of nparts gets, per column tile, its n_lblocks[p] long-row blocks
// and min(need[p], wave) persistent blocks (gx[p] in all), and tiles[p]
// column tiles: blocks [block0[p], block0[p + 1]) of the flattened grid,
// tile after tile.  block0 has nparts + 1 entries.  Returns the number of
// blocks, or -1 when it exceeds INT_MAX.
inline long long joint_layout(int nparts, const int* n_lblocks, const int* need, const int* tiles, int wave,
                              int* block0, int* gx) {
    long long total = 0;
    for (int p = 0; p < nparts; ++p) {
        const int persist = need[p] < wave ? need[p] : wave;
        gx[p] = n_lblocks[p] + persist;
        block0[p] = (int)total;
        total += (long long)gx[p] * tiles[p];
        if (total > INT_MAX) return -1;
    }
    block0[nparts] = (int)total;
    return total;
}

// The part of flattened block b and its place (bx, by) in the part's own
// grid of gx blocks per tile: bx runs fastest, as blockIdx.x does in k_step.
struct JointPlace {
    int part, bx, by, gx;
};
LPB_JG_HD inline JointPlace joint_place(int b, int nparts, const int* block0, const int* gx) {
    int p = 0;
    while (p + 1 < nparts && b >= block0[p + 1]) ++p;
    const int local = b - block0[p], g = gx[p];
    return JointPlace{p, local % g, local / g, g};
}

}  // namespace lpb
