// df64.cuh -- double-float arithmetic on the float32 pipe, for the
// float64-class form of the predictor (WT_FP64_DF).
//
// A value is carried as h + l with |l| <= ulp(h)/2: 48 significant bits,
// float64 accuracy to within a factor of 32, at float32 rates (the GB300's
// float64 pipe runs at a small fraction of its float32 rate). The building
// blocks are the two error-free transforms: Knuth's two-sum (a + b = s + e
// exactly) and the FMA product error (a b = p + e exactly, e = fma(a, b, -p)).
// Sums and products are renormalised with Dekker's fast two-sum; the sum
// drops the rounding error of the low parts' addition (absolute error below
// 2^-47 of the operands), the product drops l_a l_b (below 2^-48 of it).
#pragma once

#include "wt_internal.cuh"

namespace wt {

struct DF {
    float h, l;
};

__device__ __forceinline__ DF df_renorm(float s, float e)
{
    const float h = __fadd_rn(s, e);
    return DF{h, __fsub_rn(e, __fsub_rn(h, s))};
}

__device__ __forceinline__ DF df_add(DF a, DF b)
{
    float s, e;
    two_sum(a.h, b.h, s, e);
    return df_renorm(s, __fadd_rn(e, __fadd_rn(a.l, b.l)));
}

__device__ __forceinline__ DF df_add_f(DF a, float b)
{
    float s, e;
    two_sum(a.h, b, s, e);
    return df_renorm(s, __fadd_rn(e, a.l));
}

__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.h, -a.l}; }

__device__ __forceinline__ DF df_mul(DF a, DF b)
{
    const float p = __fmul_rn(a.h, b.h);
    const float e = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, __fmaf_rn(a.h, b.h, -p)));
    return df_renorm(p, e);
}

// times a power of two: exact
__device__ __forceinline__ DF df_scale(DF a, float pow2) { return DF{__fmul_rn(a.h, pow2), __fmul_rn(a.l, pow2)}; }

__device__ __forceinline__ double df_to_double(DF a) { return static_cast<double>(a.h) + static_cast<double>(a.l); }

__device__ __forceinline__ DF df_from_double(double x)
{
    const float h = __double2float_rn(x);
    return DF{h, __double2float_rn(x - static_cast<double>(h))};
}

// 2 pi and -1/6 as double-floats (the float32 rounding and its remainder)
constexpr float kTwoPiH = 6.2831854820251465f, kTwoPiL = -1.7484555314695172e-07f;
constexpr float kMinusSixthH = -0.1666666716337204f, kMinusSixthL = 4.967053879312289e-09f;

// exp(i 2 pi t) as double-floats for t = th + tl turns, |th| <= 1/2 and tl
// small (the phase of phase_turns_df). The table method of the float64 form
// (P. T. P. Tang, ACM TOMS 15(2), 1989) carried out in double-float:
// k = rint(256 th), f = (th - k/256) + tl (the difference exact, the sum
// error-free), x = 2 pi f (|x| <= 0.0123 plus the tail), then
//   sin x = x - x^3/6 + x^5/120 - x^7/5040,  cos x = 1 - x^2/2 + x^4/24 - x^6/720
// with the terms down to x^3 and x^2 in double-float and the rest, below
// 2.5e-12 and 1e-9, in float32 (their rounding stays below 1e-16), and
// finally the rotation by the table entry exp(i 2 pi k/256) = C + i S,
// tab[k + 128] = (C h, C l, S h, S l).
__device__ __forceinline__ void sincos_turns_df(float th, float tl, const float4* __restrict__ tab, DF& s, DF& c)
{
    const float k = rintf(__fmul_rn(th, 256.0f));
    float fh, fl;
    two_sum(__fmaf_rn(k, -0.00390625f, th), tl, fh, fl);
    const DF x = df_mul(DF{fh, fl}, DF{kTwoPiH, kTwoPiL});
    const DF x2 = df_mul(x, x);
    const DF x3 = df_mul(x2, x);
    const float q = x2.h;
    const float small_s = __fmul_rn(__fmul_rn(x3.h, q), __fmaf_rn(q, -1.9841269841269841e-4f, 8.3333333333333333e-3f));
    const float small_c = __fmul_rn(__fmul_rn(q, q), __fmaf_rn(q, -1.3888888888888889e-3f, 4.1666666666666667e-2f));
    const DF sx = df_add_f(df_add(x, df_mul(x3, DF{kMinusSixthH, kMinusSixthL})), small_s);
    const DF cx = df_add_f(df_add_f(df_neg(df_scale(x2, 0.5f)), 1.0f), small_c);
    const float4 e = tab[static_cast<int>(k) + 128];
    const DF C{e.x, e.y}, S{e.z, e.w};
    c = df_add(df_mul(C, cx), df_neg(df_mul(S, sx)));
    s = df_add(df_mul(S, cx), df_mul(C, sx));
}

constexpr int kDfTableEntries = 257;

// The table of exp(i 2 pi k/256), k = -128 .. 128, as double-floats, from
// the correctly rounded float64 table of the float64 form: 257 entries,
// written by the CTA's threads into shared memory.
__device__ __forceinline__ void load_sincos_table_df(float4* tab)
{
    for (int i = threadIdx.x; i < kDfTableEntries; i += blockDim.x) {
        const double2 e = kSinCos256[i];
        const DF c = df_from_double(e.x), s = df_from_double(e.y);
        tab[i] = make_float4(c.h, c.l, s.h, s.l);
    }
}

}  // namespace wt
