// Host-side check of the key under which an interval's CUDA graph is replayed
// (interval_key in lpb_engine.h): every input that a captured graph bakes into
// its nodes changes the key, so a stale graph is never replayed.  Compiled by
// nvcc for the host; makes no CUDA call and needs no GPU.  Prints "ok" or the
// first failures.
#include <cstdio>

#include "lpb_engine.h"

static int fails = 0;

template <typename F>
static void expect_change(const char* what, F mutate) {
    lpb_ctx h;
    lpb::Lane ln;
    auto setup = [](lpb_ctx& hh, lpb::Lane& l) {
        l.cap = 128;
        l.ncol = 100;
        l.Xbar = reinterpret_cast<void*>(0x1000);
        l.Y = reinterpret_cast<void*>(0x2000);
        l.rec = reinterpret_cast<lpb::ColRecord*>(0x3000);
        l.rec_h = reinterpret_cast<lpb::ColRecord*>(0x4000);
        hh.ws_epoch = 3;
        hh.A.long_rows = reinterpret_cast<int*>(0x5000);
        hh.At.long_rows = reinterpret_cast<int*>(0x6000);
        hh.A.n_long = 500;
        hh.At.n_long = 0;
        hh.A.long_thr = 32;
        hh.At.long_thr = 32;
        hh.A.g_shift = 0;
        hh.At.g_shift = 1;
    };
    setup(h, ln);
    const lpb::GraphKey k0 = lpb::interval_key(&h, ln, 64, 0, 0, 4);
    const lpb::GraphKey k1 = lpb::interval_key(&h, ln, 64, 0, 0, 4);
    if (!(k0 == k1)) {
        std::printf("identical inputs give different keys\n");
        ++fails;
    }
    mutate(h, ln);
    const lpb::GraphKey k2 = lpb::interval_key(&h, ln, 64, 0, 0, 4);
    if (k0 == k2) {
        std::printf("key unchanged when %s changes\n", what);
        ++fails;
    }
}

int main() {
    expect_change("the active column count", [](lpb_ctx&, lpb::Lane& l) { l.ncol = 99; });
    expect_change("the leading dimension", [](lpb_ctx&, lpb::Lane& l) { l.cap = 256; });
    expect_change("the primal buffers", [](lpb_ctx&, lpb::Lane& l) { l.Xbar = reinterpret_cast<void*>(0x7000); });
    expect_change("the dual buffers", [](lpb_ctx&, lpb::Lane& l) { l.Y = reinterpret_cast<void*>(0x7000); });
    expect_change("the record buffer", [](lpb_ctx&, lpb::Lane& l) {
        l.rec = reinterpret_cast<lpb::ColRecord*>(0x7000);
    });
    expect_change("the pinned record mirror", [](lpb_ctx&, lpb::Lane& l) {
        l.rec_h = reinterpret_cast<lpb::ColRecord*>(0x7000);
    });
    expect_change("the check workspace", [](lpb_ctx& h, lpb::Lane&) { h.ws_epoch += 1; });
    expect_change("A's long-row list", [](lpb_ctx& h, lpb::Lane&) { h.A.long_rows = reinterpret_cast<int*>(0x7000); });
    expect_change("A^T's long-row list", [](lpb_ctx& h, lpb::Lane&) {
        h.At.long_rows = reinterpret_cast<int*>(0x7000);
    });
    expect_change("A's long-row count", [](lpb_ctx& h, lpb::Lane&) { h.A.n_long = 400; });
    expect_change("A's long-row threshold", [](lpb_ctx& h, lpb::Lane&) { h.A.long_thr = 64; });
    expect_change("A^T's lane shift", [](lpb_ctx& h, lpb::Lane&) { h.At.g_shift = 2; });
    expect_change("the long-row scratch", [](lpb_ctx& h, lpb::Lane&) { h.lr_part = reinterpret_cast<void*>(0x7000); });
    {
        lpb_ctx h;
        lpb::Lane ln;
        ln.ncol = 10;
        const lpb::GraphKey a = lpb::interval_key(&h, ln, 64, 0, 0, 4);
        if (a == lpb::interval_key(&h, ln, 32, 0, 0, 4) || a == lpb::interval_key(&h, ln, 64, 1, 0, 4) ||
            a == lpb::interval_key(&h, ln, 64, 0, -1, 4) || a == lpb::interval_key(&h, ln, 64, 0, 0, 8)) {
            std::printf("key unchanged by the interval length, stall setting, group or iterate size\n");
            ++fails;
        }
    }
    if (fails == 0) std::printf("ok\n");
    return fails == 0 ? 0 : 1;
}
