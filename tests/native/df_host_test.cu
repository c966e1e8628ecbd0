// Host-side pins of the double-float helpers in lpb_df.h (compiled by nvcc
// for the host; no GPU).  Prints "ok" or the first failure.
#include <cmath>
#include <cstdio>
#include <random>

#include "lpb_df.h"

using lpb::df;

static int fails = 0;
#define CHECK(cond, ...)                 \
    do {                                 \
        if (!(cond)) {                   \
            std::printf(__VA_ARGS__);    \
            std::printf("\n");           \
            ++fails;                     \
        }                                \
    } while (0)

static double val(df a) { return (double)a.hi + (double)a.lo; }
static df from(double v) {
    const float hi = (float)v;
    return df{hi, (float)(v - (double)hi)};
}

int main() {
    std::mt19937_64 rng(7);
    std::uniform_real_distribution<double> u(-1.0, 1.0);
    for (int t = 0; t < 200000; ++t) {
        const float a = (float)(u(rng) * std::ldexp(1.0, (int)(rng() % 40) - 20));
        const float b = (float)(u(rng) * std::ldexp(1.0, (int)(rng() % 40) - 20));
        // error-free transformations are exact in FP64 (which holds the exact results here)
        const df s = lpb::two_sum(a, b);
        CHECK((double)s.hi + (double)s.lo == (double)a + (double)b, "two_sum %a %a", a, b);
        const df p = lpb::two_prod(a, b);
        CHECK((double)p.hi + (double)p.lo == (double)a * (double)b, "two_prod %a %a", a, b);
        // double-float arithmetic against FP64 on values with ~48-bit significands
        const double x = u(rng) * 1e3, y = u(rng) * 1e-2, z = u(rng);
        const df X = from(x), Y = from(y);
        const double ex = val(X), ey = val(Y);
        const double add = val(lpb::df_add(X, Y)), mul = val(lpb::df_mul(X, Y));
        CHECK(std::fabs(add - (ex + ey)) <= 1e-13 * (std::fabs(ex) + std::fabs(ey)), "df_add %g", add);
        CHECK(std::fabs(mul - ex * ey) <= 1e-13 * std::fabs(ex * ey), "df_mul %g", mul);
        const double mf = val(lpb::df_mulf(X, (float)z));
        CHECK(std::fabs(mf - ex * (double)(float)z) <= 1e-13 * std::fabs(ex * (double)(float)z) + 1e-300, "df_mulf");
    }
    // accumulation with cancellation: sum of a_e * x_e (a in df, x FP32) against FP64
    for (int t = 0; t < 200; ++t) {
        df acc = lpb::df_zero();
        double exact = 0.0, mag = 0.0;
        for (int e = 0; e < 5000; ++e) {
            const double a = u(rng) * 10.0;
            const float x = (float)(u(rng) * 100.0);
            const df A = from(a);
            lpb::df_fma_acc(acc, A, x);
            exact += val(A) * (double)x;
            mag += std::fabs(val(A) * (double)x);
        }
        acc = lpb::quick_two_sum(acc.hi, acc.lo);
        CHECK(std::fabs(val(acc) - exact) <= 1e-11 * mag, "df_fma_acc %g vs %g (mag %g)", val(acc), exact, mag);
    }
    // dfloat dot products with the low part left unnormalised until the end
    // (dfl_dot_acc + dfl_norm) against FP64 and against the renormalising
    // dfl_fma: both within the twice-working-precision bound of the sum of
    // the terms' magnitudes
    for (int t = 0; t < 2000; ++t) {
        const int len = 1 + (int)(rng() % 64);
        lpb::dfloat acc(0.0f), ref(0.0f);
        double exact = 0.0, mag = 0.0;
        for (int e = 0; e < len; ++e) {
            const lpb::dfloat a(u(rng) * 10.0), x(u(rng) * std::ldexp(1.0, (int)(rng() % 20) - 10));
            acc = lpb::dfl_dot_acc(a, x, acc);
            ref = lpb::dfl_fma(a, x, ref);
            const double ad = (double)a.hi + (double)a.lo, xd = (double)x.hi + (double)x.lo;
            exact += ad * xd;
            mag += std::fabs(ad * xd);
        }
        acc = lpb::dfl_norm(acc);
        const double got = (double)acc.hi + (double)acc.lo, want = (double)ref.hi + (double)ref.lo;
        CHECK(std::fabs(got - exact) <= 1e-13 * mag, "dfl_dot_acc %g vs %g (mag %g)", got, exact, mag);
        CHECK(std::fabs(want - exact) <= 1e-13 * mag, "dfl_fma %g vs %g (mag %g)", want, exact, mag);
        CHECK(std::fabs(acc.lo) <= std::ldexp(std::fabs(acc.hi), -23), "dfl_norm leaves |lo| <= ulp(hi)/2");
    }
    // infinite bounds: compared, never subtracted
    const float inf = INFINITY;
    const df pinf{inf, 0.f}, minf{-inf, 0.f}, one{1.f, 0.f}, two{2.f, 0.f};
    CHECK(val(lpb::df_clamp(from(5.0), minf, two)) == 2.0, "clamp hi");
    CHECK(val(lpb::df_clamp(from(-5.0), one, pinf)) == 1.0, "clamp lo");
    CHECK(val(lpb::df_clamp(from(0.5), minf, pinf)) == 0.5, "clamp free");
    CHECK(val(lpb::df_support(from(2.0), minf, two)) == 4.0, "support +");
    CHECK(val(lpb::df_support(from(-2.0), one, pinf)) == -2.0, "support -");
    CHECK(std::isinf(val(lpb::df_support(from(1.0), one, pinf))), "support outside cone");
    CHECK(val(lpb::df_support(lpb::df_zero(), minf, pinf)) == 0.0, "support 0*inf");
    CHECK(val(lpb::df_barrier(from(-3.0), minf, two)) == 0.0, "barrier a=-inf");
    CHECK(val(lpb::df_barrier(from(-3.0), one, pinf)) == -3.0, "barrier b=inf");
    CHECK(val(lpb::df_barrier(from(3.0), minf, pinf)) == 0.0, "barrier free var");
    df s = lpb::df_zero();
    lpb::df_acc(s, from(1.0));
    lpb::df_acc(s, pinf);
    lpb::df_acc(s, from(1.0));
    CHECK(std::isinf(s.hi) && s.hi > 0 && !std::isnan(s.lo), "sticky inf");
    if (fails == 0) std::printf("ok\n");
    return fails == 0 ? 0 : 1;
}
