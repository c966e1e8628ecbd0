// lpb_df.h -- double-float ("df") arithmetic: a value is the unevaluated sum
// hi + lo of two FP32 numbers, about 48 bits of significand.  Built from the
// error-free transformations TwoSum (Knuth, TAOCP vol. 2, 4.2.2) and TwoProd
// through a fused multiply-add.  GB300 executes FP64 at a small fraction of
// its FP32 rate, so the FP64-accurate quantities of a check (A x against its
// bounds, c + A^T y, the duality gap) are formed in df on the FP32 pipe.
// Infinite bounds are kept as {+-inf, 0} and only ever compared; the
// accumulator in df_acc keeps an infinite term sticky instead of producing
// NaN from inf - inf.
#pragma once

#include <cuda_runtime.h>

#include <cmath>

#define LPB_HD __host__ __device__ __forceinline__

namespace lpb {

struct df {
    float hi, lo;
};

LPB_HD df df_of(float a) { return df{a, 0.0f}; }

// a + b = s + e exactly
LPB_HD df two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return df{s, e};
}

// a + b = s + e exactly when |a| >= |b|
LPB_HD df quick_two_sum(float a, float b) {
    const float s = a + b;
    return df{s, b - (s - a)};
}

// a * b = p + e exactly (barring underflow)
LPB_HD df two_prod(float a, float b) {
    const float p = a * b;
    return df{p, fmaf(a, b, -p)};
}

LPB_HD df df_add(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    s.lo += a.lo + b.lo;
    return quick_two_sum(s.hi, s.lo);
}
LPB_HD df df_neg(df a) { return df{-a.hi, -a.lo}; }
LPB_HD df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

LPB_HD df df_mulf(df a, float b) {
    df p = two_prod(a.hi, b);
    p.lo = fmaf(a.lo, b, p.lo);
    return quick_two_sum(p.hi, p.lo);
}
LPB_HD df df_mul(df a, df b) {
    df p = two_prod(a.hi, b.hi);
    p.lo = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo));
    return quick_two_sum(p.hi, p.lo);
}

LPB_HD bool df_lt(df a, df b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
LPB_HD bool df_gt(df a, df b) { return df_lt(b, a); }
LPB_HD bool df_isinf(df a) { return std::isinf(a.hi); }
LPB_HD float df_f(df a) { return a.hi + a.lo; }
LPB_HD double df_d(df a) { return (double)a.hi + (double)a.lo; }
LPB_HD df df_zero() { return df{0.0f, 0.0f}; }

// Pi_[a,b](v) = max(min(v, b), a)
LPB_HD df df_clamp(df v, df a, df b) {
    df t = df_lt(v, b) ? v : b;
    return df_gt(t, a) ? t : a;
}

// s += t, with an infinite term or sum kept infinite (never NaN from inf - inf)
LPB_HD void df_acc(df& s, df t) {
    if (std::isinf(t.hi) || std::isinf(s.hi)) {
        s.hi += t.hi;
        s.lo = 0.0f;
    } else {
        s = df_add(s, t);
    }
}

// sum += a * x for a df constant and an FP32 x, accumulated without rounding
// the product: the two-term product joins (s, c) through TwoSum
LPB_HD void df_fma_acc(df& acc, df a, float x) {
    const df p = two_prod(a.hi, x);
    const df s = two_sum(acc.hi, p.hi);
    acc.hi = s.hi;
    acc.lo += s.lo + fmaf(a.lo, x, p.lo);
}

// v in the barrier cone B_[a,b] (Sec. 3)
LPB_HD df df_barrier(df v, df a, df b) {
    const bool li = std::isinf(a.hi), hi = std::isinf(b.hi);
    if (li && hi) return df_zero();
    if (li) return v.hi > 0.0f ? v : df_zero();
    if (hi) return v.hi < 0.0f ? v : df_zero();
    return v;
}

LPB_HD df df_abs(df a) { return a.hi < 0.0f ? df_neg(a) : a; }

// Reduced cost robust to large finite bounds (Sec. 4, stopping criteria;
// the variant of PDLP's Appendix A): v pairs with b when positive and with a
// when negative, and is kept only where that bound is finite and
// |x - bound| <= |x|; elsewhere it is 0 and stays in the dual residual.
LPB_HD df df_robust_rc(df v, df x, df a, df b) {
    if (v.hi > 0.0f) return !std::isinf(b.hi) && !df_gt(df_abs(df_sub(x, b)), df_abs(x)) ? v : df_zero();
    if (v.hi < 0.0f) return !std::isinf(a.hi) && !df_gt(df_abs(df_sub(x, a)), df_abs(x)) ? v : df_zero();
    return df_zero();
}

// one term b v_+ + a v_- of phi_[a,b](v), with 0 * inf = 0
LPB_HD df df_support(df v, df a, df b) {
    if (v.hi > 0.0f) return std::isinf(b.hi) ? df{b.hi, 0.0f} : df_mul(b, v);
    if (v.hi < 0.0f) return std::isinf(a.hi) ? df{-a.hi, 0.0f} : df_mul(a, v);
    return df_zero();
}

// ---------------------------------------------------------------------------
// dfloat: a double-float number used as an iterate type.  The mixed path's
// polish phase runs the iteration kernels in dfloat instead of FP64: the
// same 8 bytes per value, about 48 bits of significand, and only FP32
// instructions, so the step kernels stay bound by memory rather than by the
// FP64 pipe.  The exponent range is FP32's; values beyond it are infinite,
// as in the FP32 path.  Device operators follow the df routines above.
// ---------------------------------------------------------------------------
struct dfloat {
    float hi, lo;
    dfloat() = default;
    LPB_HD constexpr dfloat(int v) : hi((float)v), lo(0.0f) {}
    LPB_HD constexpr dfloat(float h) : hi(h), lo(0.0f) {}
    LPB_HD constexpr dfloat(float h, float l) : hi(h), lo(l) {}
    // nearest pair to v; an infinite or overflowing v keeps lo = 0
    LPB_HD explicit dfloat(double v) : hi((float)v), lo(0.0f) {
        if (std::isfinite(hi)) lo = (float)(v - (double)hi);
    }
    LPB_HD explicit operator double() const { return (double)hi + (double)lo; }
};

static_assert(sizeof(dfloat) == sizeof(df) && alignof(dfloat) == alignof(df), "dfloat and df share a layout");

LPB_HD df df_of(dfloat a) { return df{a.hi, a.lo}; }
LPB_HD dfloat dfl_of(df a) { return dfloat(a.hi, a.lo); }

LPB_HD dfloat operator+(dfloat a, dfloat b) { return dfl_of(df_add(df_of(a), df_of(b))); }
LPB_HD dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }
LPB_HD dfloat operator-(dfloat a, dfloat b) { return dfl_of(df_add(df_of(a), df{-b.hi, -b.lo})); }
LPB_HD dfloat operator*(dfloat a, dfloat b) { return dfl_of(df_mul(df_of(a), df_of(b))); }
// a / b: quotient of the leading parts, corrected once by the remainder
LPB_HD dfloat operator/(dfloat a, dfloat b) {
    const float q1 = a.hi / b.hi;
    const df r = df_sub(df_of(a), df_mulf(df_of(b), q1));
    const float q2 = r.hi / b.hi;
    return dfl_of(quick_two_sum(q1, q2));
}
LPB_HD dfloat& operator+=(dfloat& a, dfloat b) { return a = a + b; }
LPB_HD bool operator<(dfloat a, dfloat b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
LPB_HD bool operator>(dfloat a, dfloat b) { return b < a; }
LPB_HD bool operator==(dfloat a, dfloat b) { return a.hi == b.hi && a.lo == b.lo; }

// acc + a * x with the product kept to df accuracy (the inner product step
// of the dfloat SpMMs)
LPB_HD dfloat dfl_fma(dfloat a, dfloat x, dfloat acc) {
    const df p = two_prod(a.hi, x.hi);
    const df s = two_sum(acc.hi, p.hi);
    const float e = s.lo + acc.lo + fmaf(a.hi, x.lo, fmaf(a.lo, x.hi, p.lo));
    return dfl_of(quick_two_sum(s.hi, e));
}

// acc + a * x for a running dot product whose low part is left unnormalised
// (the dot product in twice the working precision of Ogita, Rump and Oishi,
// "Accurate sum and dot product", SIAM J. Sci. Comput. 26 (2005), with the
// low parts of a and x included): the high part follows the FP32 sum through
// TwoSum, every rounding error and the products' low parts collect in lo, and
// dfl_norm renormalises once at the end.  Its dependent chain per term is the
// TwoSum on the high part alone.
LPB_HD dfloat dfl_dot_acc(dfloat a, dfloat x, dfloat acc) {
    const df p = two_prod(a.hi, x.hi);
    const df s = two_sum(acc.hi, p.hi);
    return dfloat(s.hi, acc.lo + (s.lo + fmaf(a.hi, x.lo, fmaf(a.lo, x.hi, p.lo))));
}
LPB_HD dfloat dfl_norm(dfloat a) { return dfl_of(two_sum(a.hi, a.lo)); }

// acc += w * x for a df constant and a dfloat x (the check SpMMs)
LPB_HD void df_fma_acc(df& acc, df w, dfloat x) {
    const df p = two_prod(w.hi, x.hi);
    const df s = two_sum(acc.hi, p.hi);
    acc.hi = s.hi;
    acc.lo += s.lo + fmaf(w.hi, x.lo, fmaf(w.lo, x.hi, p.lo));
}

}  // namespace lpb
