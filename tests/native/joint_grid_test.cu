// Host-side check of the flattened grid of a joint step launch
// (lpb_joint_grid.h): over seeded random mixes of parts, every block maps to
// one part and one (bx, by) inside that part's own grid, every place of every
// part is taken by exactly one block, and within a part bx runs fastest (the
// order of k_step's blockIdx.x, blockIdx.y).  Compiled by nvcc for the host;
// makes no CUDA call and needs no GPU.  Prints "ok" or the first failures.
#include <cstdio>
#include <vector>

#include "lpb_joint_grid.h"

static unsigned long long state = 0x9e3779b97f4a7c15ULL;
static int next_int(int lo, int hi) {  // SplitMix64, uniform-ish in [lo, hi]
    state += 0x9e3779b97f4a7c15ULL;
    unsigned long long z = state;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    z ^= z >> 31;
    return lo + (int)(z % (unsigned long long)(hi - lo + 1));
}

int main() {
    int fails = 0;
    for (int trial = 0; trial < 2000 && fails < 10; ++trial) {
        const int nparts = next_int(1, 8), wave = next_int(1, 1216);
        int nlb[8], need[8], tiles[8], block0[9], gx[8];
        for (int p = 0; p < nparts; ++p) {
            nlb[p] = next_int(0, 3) == 0 ? next_int(1, 300) : 0;
            need[p] = next_int(1, 3000);
            tiles[p] = next_int(1, 9);
        }
        const long long total = lpb::joint_layout(nparts, nlb, need, tiles, wave, block0, gx);
        if (total <= 0) {
            std::printf("trial %d: total %lld\n", trial, total);
            ++fails;
            continue;
        }
        std::vector<std::vector<char>> seen(nparts);
        for (int p = 0; p < nparts; ++p) {
            const int persist = need[p] < wave ? need[p] : wave;
            if (gx[p] != nlb[p] + persist) {
                std::printf("trial %d part %d: gx %d, expected %d\n", trial, p, gx[p], nlb[p] + persist);
                ++fails;
            }
            seen[p].assign((size_t)gx[p] * tiles[p], 0);
        }
        int prev_part = 0, prev_idx = -1;
        for (int b = 0; b < (int)total; ++b) {
            const lpb::JointPlace q = lpb::joint_place(b, nparts, block0, gx);
            if (q.part < 0 || q.part >= nparts || q.bx < 0 || q.bx >= gx[q.part] || q.by < 0 ||
                q.by >= tiles[q.part] || q.gx != gx[q.part]) {
                std::printf("trial %d block %d: part %d bx %d by %d out of range\n", trial, b, q.part, q.bx, q.by);
                ++fails;
                break;
            }
            const int idx = q.by * gx[q.part] + q.bx;  // k_step's order: bx fastest, then by
            if (q.part < prev_part || (q.part == prev_part && idx != prev_idx + 1) ||
                (q.part > prev_part && idx != 0)) {
                std::printf("trial %d block %d: out of order (part %d, place %d)\n", trial, b, q.part, idx);
                ++fails;
                break;
            }
            if (seen[q.part][idx]++) {
                std::printf("trial %d block %d: place taken twice\n", trial, b);
                ++fails;
                break;
            }
            prev_part = q.part;
            prev_idx = idx;
        }
        for (int p = 0; p < nparts; ++p)
            for (char c : seen[p])
                if (c != 1) {
                    std::printf("trial %d part %d: a place not taken exactly once\n", trial, p);
                    ++fails;
                    break;
                }
    }
    // a part whose blocks would exceed the 1-D grid's INT_MAX blocks
    int nlb[1] = {0}, need[1] = {1 << 30}, tiles[1] = {4}, block0[2], gx[1];
    if (lpb::joint_layout(1, nlb, need, tiles, 1 << 30, block0, gx) != -1) {
        std::printf("an oversized grid was not rejected\n");
        ++fails;
    }
    if (fails == 0) std::printf("ok\n");
    return fails == 0 ? 0 : 1;
}
