// wt_internal.cuh -- shared declarations of libwtvis (sm_103a).
//
// Device helpers used by more than one kernel file: PTX wrappers for the
// mbarrier / bulk-copy staging path, double-float arithmetic for the mixed
// precision forms, a float32 sin/cos of 2*pi*t written from the Taylor series,
// the per-device status word, and the host-side error plumbing.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/wtvis.h"

namespace wt {

// ---------------------------------------------------------------- constants
constexpr double kPi = 3.14159265358979323846;
constexpr int kMaxJ = 30;

// Upper bound on the polls of any bounded wait (mbarrier parity waits).
// A healthy wait finishes in microseconds; each failed poll may suspend the
// thread for a short hardware time slice, so this limit is of the order of
// a second.
constexpr uint32_t kSpinLimit = 1u << 20;

// ---------------------------------------------------------------- host side
// Thread-local error message + status helpers (wt_api.cu).
int set_error(int status, const char* fmt, ...);
int cuda_error(cudaError_t e, const char* what);
int* device_status_word();          // per-device int, zero-initialised
uint64_t current_context_id();      // unique ID of the current CUDA context, 0 if none

#define WT_CUDA_TRY(expr)                                             \
    do {                                                              \
        cudaError_t _e = (expr);                                      \
        if (_e != cudaSuccess) return ::wt::cuda_error(_e, #expr);    \
    } while (0)

// ---------------------------------------------------------------- device side
__device__ __forceinline__ void record_status(int* status, int code)
{
    atomicCAS(status, 0, code);
}

// ---- mbarrier + bulk copy (non-tensor TMA), one CTA, no multicast ----------
__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// Returns true once the phase with parity `parity` has completed; false if
// `limit` polls ran out.
__device__ __forceinline__ bool mbar_wait_parity(uint64_t* bar, uint32_t parity, uint32_t limit = kSpinLimit)
{
    const uint32_t a = smem_addr(bar);
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Bulk copy global -> shared of `bytes` (multiple of 16, both addresses
// 16-byte aligned), completion signalled on `bar` as transaction bytes.
__device__ __forceinline__ void bulk_copy_g2s(void* dst_smem, const void* src_gmem, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// ---- double-float helpers (mixed precision forms) --------------------------
// A float64 value x is carried as hi + lo, hi = fl32(x), lo = fl32(x - hi):
// 48 significant bits, enough for phases of many thousand turns.
struct F2 {
    float hi, lo;
};

__device__ __forceinline__ F2 split_f64(double x)
{
    F2 r;
    r.hi = __double2float_rn(x);
    r.lo = __double2float_rn(x - static_cast<double>(r.hi));
    return r;
}

// Error-free sum (Knuth): a + b = s + e exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    float bp = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

// Product of two double-floats x = xh + xl, y = yh + yl as an unevaluated
// sum p + t: p = fl(xh yh) and t = its exact rounding error (FMA) plus the
// cross terms xh yl + xl yh (xl yl is below 2^-48 of the product: dropped).
__device__ __forceinline__ void df_product(F2 x, F2 y, float& p, float& t)
{
    p = __fmul_rn(x.hi, y.hi);
    const float e = __fmaf_rn(x.hi, y.hi, -p);
    const float c = __fmaf_rn(x.hi, y.lo, __fmul_rn(x.lo, y.hi));
    t = __fadd_rn(e, c);
}

// Phase in turns of B.(s - P) = u*su + v*sv + w*sw1 modulo 1, returned as
// an unevaluated sum th + tl with th in [-1/2, 1/2] and tl small.
// Float64-accurate: the three head products are added with error-free sums
// (exact for any operands), so only their total needs reducing by its
// nearest integer (exact below 2^22 turns); all rounding errors, of size
// ulp(head), join the tail, whose own rounding (~1e-11 turns for heads of
// a thousand turns) is far below float32 resolution of th.
__device__ __forceinline__ void phase_turns_df(F2 u, F2 v, F2 w, F2 su, F2 sv, F2 sw1, float& th, float& tl)
{
    float p1, t1, p2, t2, p3, t3;
    df_product(u, su, p1, t1);
    df_product(v, sv, p2, t2);
    df_product(w, sw1, p3, t3);
    float s, e1, s2, e2;
    two_sum(p1, p2, s, e1);
    two_sum(s, p3, s2, e2);
    th = __fsub_rn(s2, rintf(s2));           // exact
    tl = __fadd_rn(__fadd_rn(__fadd_rn(t1, t2), __fadd_rn(t3, e1)), e2);
}

// sin and cos of 2*pi*(th + tl) for |th| <= 1/2 and small tl (turns),
// float32. Quadrant reduction q = rint(4 th), f = (4 th - q) + 4 tl, the
// first difference exact, so |f| <= 1/2 + 4|tl|; angle x = f * pi/2 (pi/2
// rounded to float32: relative error 3e-8, below the float32 result's own
// rounding); then the Taylor series of sin (to x^9) and cos (to x^10),
// whose truncation errors on |x| <= 0.8 (< 4e-9 and < 5e-10) are below
// float32 rounding.
__device__ __forceinline__ void sincos_turns_f32(float th, float tl, float& s, float& c)
{
    const float q = rintf(4.0f * th);
    const float f = __fmaf_rn(4.0f, tl, __fsub_rn(4.0f * th, q));
    const float x = __fmul_rn(f, 1.57079637050628662109375f);
    const float x2 = __fmul_rn(x, x);
    // sin x = x (1 - x^2/3! + x^4/5! - x^6/7! + x^8/9!)
    float ps = __fmaf_rn(x2, 2.7557319223985893e-6f, -1.9841269841269841e-4f);
    ps = __fmaf_rn(x2, ps, 8.3333333333333333e-3f);
    ps = __fmaf_rn(x2, ps, -1.6666666666666667e-1f);
    const float sx = __fmaf_rn(__fmul_rn(x, x2), ps, x);
    // cos x = 1 - x^2/2! + x^4/4! - x^6/6! + x^8/8! - x^10/10!
    float pc = __fmaf_rn(x2, -2.7557319223985891e-7f, 2.4801587301587302e-5f);
    pc = __fmaf_rn(x2, pc, -1.3888888888888889e-3f);
    pc = __fmaf_rn(x2, pc, 4.1666666666666667e-2f);
    pc = __fmaf_rn(x2, pc, -0.5f);
    const float cx = __fmaf_rn(x2, pc, 1.0f);
    const int qi = static_cast<int>(q) & 3;
    // angle = q * pi/2 + x
    const float ss = (qi & 1) ? cx : sx;
    const float cc = (qi & 1) ? sx : cx;
    s = (qi & 2) ? -ss : ss;
    c = ((qi + 1) & 2) ? -cc : cc;
}

// ---- float64 sin/cos of 2 pi t (t in turns, |t| < 2^40) ---------------------
// Table-driven reduction (the table-lookup method of P. T. P. Tang, ACM TOMS
// 15(2), 1989): k = rint(256 t), f = t - k/256 (exact, |f| <= 1/512), and
// exp(i 2 pi t) = exp(i 2 pi (k mod 256)/256) exp(i 2 pi f). The table holds
// the first factor correctly rounded (gen_sincos_table.py, entries for
// k = -128 .. 128, of which 0 .. 255 modulo 256 are used); the second comes
// from the Taylor series of sin (to x^7) and cos (to x^6) at x = 2 pi f,
// |x| <= 0.0123, whose truncation errors (< 2e-20 and < 8e-21) are far below
// float64 rounding. No separate reduction of t by its nearest integer is
// needed: k mod 256 absorbs the whole turns.
static __device__ const double2 kSinCos256[257] =
#include "sincos_table.inc"
    ;

__device__ __forceinline__ void sincos_turns_f64(double t, double& s, double& c)
{
    const double k = rint(t * 256.0);
    const double f = fma(k, -0.00390625, t);                       // t - k/256, exact
    const double x = f * 6.283185307179586476925286766559;          // 2 pi f
    const double x2 = x * x;
    const double ps = fma(x2, fma(x2, -1.9841269841269841e-4, 8.3333333333333333e-3), -1.6666666666666667e-1);
    const double sx = fma(x * x2, ps, x);
    const double pc = fma(x2, fma(x2, fma(x2, -1.3888888888888889e-3, 4.1666666666666667e-2), -0.5), 1.0);
    // entry j of the table is k = j - 128; k mod 256 in 0 .. 255 -> j = 128 + (k mod 256) - 256 * (k mod 256 >= 128)
    const int km = static_cast<int>(static_cast<long long>(k) & 255);
    const double2 tk = __ldg(&kSinCos256[(km < 128) ? km + 128 : km - 128]);
    c = fma(tk.x, pc, -tk.y * sx);
    s = fma(tk.y, pc, tk.x * sx);
}

// sin and cos of 2 pi (th + tl) from the special-function unit (the fast
// mixed form, WT_MIXED_FAST): the angle 2 pi th + 2 pi tl (|.| <= pi + small)
// goes to the hardware approximations (__sincosf; absolute error about
// 2^-21.4 on [-pi, pi] per the CUDA documentation), so one term carries at
// most ~7e-7 of its flux in error instead of ~1e-7; the phase itself stays
// float64-accurate.
__device__ __forceinline__ void sincos_turns_sfu(float th, float tl, float& s, float& c)
{
    const float twopi = 6.28318530717958648f;
    const float x = __fmaf_rn(twopi, th, __fmul_rn(twopi, tl));
    __sincosf(x, &s, &c);
}

template <bool FAST>
__device__ __forceinline__ void sincos_mixed(float th, float tl, float& s, float& c)
{
    if constexpr (FAST) sincos_turns_sfu(th, tl, s, c);
    else sincos_turns_f32(th, tl, s, c);
}

// ---- packed float32 pairs ---------------------------------------------------
// The sm_100 family issues two float32 adds, multiplies or FMAs per lane in
// one instruction (__fadd2_rn, __fmul2_rn, __ffma2_rn), each element rounded
// as the scalar operation rounds it; the FMA pipe's rate per element is
// unchanged, the issue slots halve. The mixed predictors are issue-bound, so
// they pair the real and imaginary parts of a complex value, or the same
// quantity of two visibilities. A difference is an FMA with -1: the exact
// difference rounded once, as a subtraction rounds it.
__device__ __forceinline__ float2 bcast2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Two double-floats side by side (element 0 one visibility, element 1
// another); nhi = -hi, kept so that the rounding error of a product comes
// out of one FMA without a negation.
struct DF2 {
    float2 hi, lo, nhi;
};

__device__ __forceinline__ DF2 df2_pack(F2 a, F2 b)
{
    DF2 r;
    r.hi = make_float2(a.hi, b.hi);
    r.lo = make_float2(a.lo, b.lo);
    r.nhi = make_float2(-a.hi, -b.hi);
    return r;
}

// Product of two double-floats for both elements of x against one
// double-float y, returned with its head negated: q = -fl(x.hi y.hi)
// (exact negation, from x.nhi), e = x.hi y.hi + q exactly (the rounding
// error of the head, one FMA), t = fl(x.hi y.lo + fl(x.lo y.hi + e)) (the
// tail; x.lo y.lo, below 2^-48 of the product, dropped). x y = t - q up to
// the tail's roundings, of the size of ulp(t).
__device__ __forceinline__ void df_product2n(const DF2& x, F2 y, float2& q, float2& t)
{
    const float2 yh = bcast2(y.hi);
    q = mul2(x.nhi, yh);
    const float2 e = fma2(x.hi, yh, q);
    t = fma2(x.hi, bcast2(y.lo), fma2(x.lo, yh, e));
}

__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2& s, float2& e)
{
    s = add2(a, b);
    const float2 bp = sub2(s, a);
    e = add2(sub2(a, sub2(s, bp)), sub2(b, bp));
}

// Phase in turns of B.(s - P) for two visibilities at once (u, v, w of
// visibility 0 in element 0, of visibility 1 in element 1), float64-
// accurate as phase_turns_df: the three negated heads are added with
// error-free sums and reduced by their nearest integer (exact), the
// rounding errors join the tail. Returns h = (sum of negated heads) -
// nearest integer, so that the phase is tl - h modulo 1, |h| <= 1/2.
__device__ __forceinline__ void phase_turns_df2(const DF2& u, const DF2& v, const DF2& w, F2 su, F2 sv, F2 sw1,
                                                float2& h, float2& tl)
{
    float2 q1, t1, q2, t2, q3, t3, a, ea, b, eb;
    df_product2n(u, su, q1, t1);
    df_product2n(v, sv, q2, t2);
    df_product2n(w, sw1, q3, t3);
    two_sum2(q1, q2, a, ea);
    two_sum2(a, q3, b, eb);
    h = sub2(b, make_float2(rintf(b.x), rintf(b.y)));
    tl = sub2(add2(add2(t1, t2), sub2(t3, ea)), eb);
}

// ---- phase with the heads on a common grid ----------------------------------
// The error-free sums of phase_turns_df2 exist to add the three head
// products without losing their low bits. When every head is first rounded
// onto one common grid G = 2^(k-23), with k chosen per visibility so that
// every product stays below 2^(k-1), the heads and their partial sums are
// multiples of G below 2^(k+1): 24 significant bits at most, so plain
// float32 additions are exact. A head is rounded onto the grid by one FMA
// against the constant C = 1.5 * 2^k (the sum x y + C stays in C's binade,
// where the spacing of floats is G) and recovered by one exact subtraction
// (Sterbenz); its remainder x y - (x y)_G, below G/2, goes to the tail with
// the cross terms. Per visibility and term this is 20 float32 operations
// against 29 for the error-free sums, with the same phase accuracy: the
// tail's roundings are of order 2^-24 G, the dropped x.lo y.lo below 2^-48
// of the product. Valid while k <= kGridMaxK, which keeps |tail| <= 2 G
// small enough for both sin/cos forms (sincos_turns_f32 then sees
// |x| <= 0.84); larger phases take phase_turns_df2 (the caller decides).
constexpr int kGridMinK = -8;    // finest grid used: 2^-31 turns
constexpr int kGridMaxK = 15;    // heads below 2^14 turns

// C = 1.5 * 2^k for the smallest k >= kGridMinK with bound < 2^(k-1); also
// returns k through kk. bound: an upper bound on the sum of |x.hi y.hi| over
// the three coordinates (a non-finite bound gives k > kGridMaxK).
__device__ __forceinline__ float grid_magic(float bound, int& kk)
{
    const int e = (__float_as_int(bound) >> 23) & 255;   // bound < 2^(e - 126) (e = 255: not finite)
    int k = e - 125;
    k = k < kGridMinK ? kGridMinK : k;
    kk = k;
    const int kc = k > kGridMaxK ? kGridMaxK : k;
    return __int_as_float(((kc + 127) << 23) | 0x400000);
}

// Head of x y on the grid of C, negated, and the tail, for both elements
// (element-wise C): nq = -(x.hi y.hi rounded to the grid), exactly;
// t = (x.hi y.hi + nq) + x.lo y.hi + x.hi y.lo, the first term exact.
__device__ __forceinline__ void grid_product2n(const DF2& x, F2 y, float2 C, float2& nq, float2& t)
{
    const float2 yh = bcast2(y.hi);
    nq = sub2(C, fma2(x.hi, yh, C));
    t = fma2(x.hi, bcast2(y.lo), fma2(x.lo, yh, fma2(x.hi, yh, nq)));
}

// phase_turns_df2 on the grid of C (per element): returns h and tl with the
// phase = tl - h modulo 1, |h| <= 1/2, |tl| <= 2^(k-22).
__device__ __forceinline__ void phase_turns_grid2(const DF2& u, const DF2& v, const DF2& w, F2 su, F2 sv, F2 sw1,
                                                  float2 C, float2& h, float2& tl)
{
    float2 q1, t1, q2, t2, q3, t3;
    grid_product2n(u, su, C, q1, t1);
    grid_product2n(v, sv, C, q2, t2);
    grid_product2n(w, sw1, C, q3, t3);
    const float2 b = add2(add2(q1, q2), q3);          // exact: multiples of the grid below 2^(k+1)
    h = sub2(b, make_float2(rintf(b.x), rintf(b.y)));
    tl = add2(add2(t1, t2), t3);
}

// The scalar form of phase_turns_grid2 (one visibility): the phase is
// th + tl modulo 1, |th| <= 1/2.
__device__ __forceinline__ void phase_turns_grid(F2 u, F2 v, F2 w, F2 su, F2 sv, F2 sw1, float C, float& th,
                                                 float& tl)
{
    const float p1 = __fsub_rn(__fmaf_rn(u.hi, su.hi, C), C);
    const float p2 = __fsub_rn(__fmaf_rn(v.hi, sv.hi, C), C);
    const float p3 = __fsub_rn(__fmaf_rn(w.hi, sw1.hi, C), C);
    const float t1 = __fmaf_rn(u.hi, su.lo, __fmaf_rn(u.lo, su.hi, __fmaf_rn(u.hi, su.hi, -p1)));
    const float t2 = __fmaf_rn(v.hi, sv.lo, __fmaf_rn(v.lo, sv.hi, __fmaf_rn(v.hi, sv.hi, -p2)));
    const float t3 = __fmaf_rn(w.hi, sw1.lo, __fmaf_rn(w.lo, sw1.hi, __fmaf_rn(w.hi, sw1.hi, -p3)));
    const float b = __fadd_rn(__fadd_rn(p1, p2), p3);
    th = __fsub_rn(b, rintf(b));
    tl = __fadd_rn(__fadd_rn(t1, t2), t3);
}

// Bound on sum_c |x_c.hi y_c.hi| for a visibility (u, v, w) against every
// leaf of a tree whose coordinates are bounded by smax (float32, rounded
// up): the float32 evaluation, raised by 2^-10 to cover its own roundings.
__device__ __forceinline__ float phase_bound(F2 u, F2 v, F2 w, const float* smax)
{
    const float b = __fmaf_rn(fabsf(u.hi), smax[0], __fmaf_rn(fabsf(v.hi), smax[1], fabsf(w.hi) * smax[2]));
    return b * 1.0009765625f;
}

// A predictor in a mixed form (the regrouped Eq. 17, the direct sum) is
// evaluated in two passes over the tiles. The grid pass takes every tile
// whose phases all fit the head grid (tile_grid_constants: all heads below
// 2^(kGridMaxK - 1) turns, which the coordinate bounds smax of the leaves or
// components and each visibility's |u|, |v|, |w| establish) and evaluates it
// with phase_turns_grid2; a tile that does not fit gets kDeferredMark in
// both parts of its first visibility and is left to the exact pass, which
// evaluates only tiles so marked, with error-free sums (phase_turns_df2).
// The two kernels are launched back to back on one stream; kept apart, each
// stays within its register budget.
constexpr uint32_t kDeferredMark = 0x7fc4b1d3u;   // a quiet NaN

// Grid constants of a thread's visibilities and the CTA's vote on whether
// every visibility of the tile fits; every thread of the CTA must call it.
template <int VPT>
__device__ __forceinline__ bool tile_grid_constants(const F2 (&u)[VPT], const F2 (&v)[VPT], const F2 (&w)[VPT],
                                                    const float* __restrict__ smax, float (&C)[VPT])
{
    const float sm[3] = {smax[0], smax[1], smax[2]};
    bool fits = true;
#pragma unroll
    for (int k = 0; k < VPT; ++k) {
        int kk;
        C[k] = grid_magic(phase_bound(u[k], v[k], w[k], sm), kk);
        fits = fits && kk <= kGridMaxK;
    }
    return __syncthreads_and(fits ? 1 : 0) != 0;
}

// The exact pass's test of a tile: whether its first visibility carries
// kDeferredMark (read by one thread, broadcast through shared memory);
// every thread of the CTA must call it.
__device__ __forceinline__ bool tile_deferred(const float2* first_vis)
{
    __shared__ int s_deferred;
    __syncthreads();
    if (threadIdx.x == 0) {
        const volatile float* x = reinterpret_cast<const volatile float*>(first_vis);
        s_deferred = __float_as_uint(x[0]) == kDeferredMark && __float_as_uint(x[1]) == kDeferredMark;
    }
    __syncthreads();
    return s_deferred != 0;
}

__device__ __forceinline__ void mark_deferred(float2* first_vis)
{
    if (threadIdx.x == 0) *first_vis = make_float2(__uint_as_float(kDeferredMark), __uint_as_float(kDeferredMark));
}

// sincos_turns_f32 of the phase tl - h (turns) of two visibilities, each
// result written as the pair (cos, sin) of its own visibility: e0 for
// element 0, e1 for element 1. Quadrant reduction and both polynomials on
// pairs (the same steps and roundings as sincos_turns_f32 on th = -h), the
// quadrant fix-up per element.
__device__ __forceinline__ void sincos_turns_f32x2(float2 h, float2 tl, float2& e0, float2& e1)
{
    const float2 t4 = mul2(bcast2(-4.0f), h);                      // 4 th, exact
    const float2 q = make_float2(rintf(t4.x), rintf(t4.y));
    const float2 f = fma2(bcast2(4.0f), tl, sub2(t4, q));
    const float2 x = mul2(f, bcast2(1.57079637050628662109375f));
    const float2 x2 = mul2(x, x);
    float2 ps = fma2(x2, bcast2(2.7557319223985893e-6f), bcast2(-1.9841269841269841e-4f));
    ps = fma2(x2, ps, bcast2(8.3333333333333333e-3f));
    ps = fma2(x2, ps, bcast2(-1.6666666666666667e-1f));
    const float2 sx = fma2(mul2(x, x2), ps, x);
    float2 pc = fma2(x2, bcast2(-2.7557319223985891e-7f), bcast2(2.4801587301587302e-5f));
    pc = fma2(x2, pc, bcast2(-1.3888888888888889e-3f));
    pc = fma2(x2, pc, bcast2(4.1666666666666667e-2f));
    pc = fma2(x2, pc, bcast2(-0.5f));
    const float2 cx = fma2(x2, pc, bcast2(1.0f));
    const int q0 = static_cast<int>(q.x) & 3, q1 = static_cast<int>(q.y) & 3;
    const float ss0 = (q0 & 1) ? cx.x : sx.x, cc0 = (q0 & 1) ? sx.x : cx.x;
    const float ss1 = (q1 & 1) ? cx.y : sx.y, cc1 = (q1 & 1) ? sx.y : cx.y;
    e0 = make_float2(((q0 + 1) & 2) ? -cc0 : cc0, (q0 & 2) ? -ss0 : ss0);
    e1 = make_float2(((q1 + 1) & 2) ? -cc1 : cc1, (q1 & 2) ? -ss1 : ss1);
}

// sincos_turns_sfu of the phase tl - h of two visibilities (the angle on
// pairs, the same roundings as 2 pi th + 2 pi tl), each result written as
// its visibility's (cos, sin) pair.
__device__ __forceinline__ void sincos_turns_sfu2(float2 h, float2 tl, float2& e0, float2& e1)
{
    const float2 x = fma2(bcast2(-6.28318530717958648f), h, mul2(bcast2(6.28318530717958648f), tl));
    __sincosf(x.x, &e0.y, &e0.x);
    __sincosf(x.y, &e1.y, &e1.x);
}

template <bool FAST>
__device__ __forceinline__ void sincos_mixed2(float2 h, float2 tl, float2& e0, float2& e1)
{
    if constexpr (FAST) sincos_turns_sfu2(h, tl, e0, e1);
    else sincos_turns_f32x2(h, tl, e0, e1);
}

// Blockwise compensated summation of the term-per-component sums (the
// direct sum, Eq. 12, and Eq. 16): the terms of up to kSumBlock consecutive
// records are added by plain FMAs into a partial sum (at most kSumBlock
// roundings, a relative error of at most 8 u of the block's sum of |terms|),
// and each partial enters the Kahan sum once.
constexpr int kSumBlock = 8;

// Kahan-compensated sum of pairs (each element as kahan_add).
__device__ __forceinline__ void kahan_add2(float2& sum, float2& comp, float2 x)
{
    const float2 y = sub2(x, comp);
    const float2 t = add2(sum, y);
    comp = sub2(sub2(t, sum), y);
    sum = t;
}

// Kahan-compensated float32 accumulation: sum + comp carries the total.
__device__ __forceinline__ void kahan_add(float& sum, float& comp, float x)
{
    const float y = __fsub_rn(x, comp);
    const float t = __fadd_rn(sum, y);
    comp = __fsub_rn(__fsub_rn(t, sum), y);
    sum = t;
}

// Component record of the direct sum's float forms (32 bytes): l, m and
// n - 1 as double-float pairs, C's high half (flux) and low half (flux_lo,
// the double-float form's).
struct CompF {
    float lh, ll, mh, ml, nh, nl, flux, flux_lo;
};
static_assert(sizeof(CompF) == 32, "component record layout");

// ---------------------------------------------------------------- tree handle
// Node records for the predictors, in post-order, pre-decoded at build time.
// A thread keeps one column of a shared-memory "stack" of 4 (J - 1) rows:
// row 4 (j - 2) + c holds the plane-wave coefficient eta of the open level-j
// node in child slot c (j = 2 .. J). meta bits:
//    0-6   store row: where this node's eta goes (unused at level 1)
//    7-13  child row: first of the node's four child rows, or, for a node
//          with a single child, that child's row
//   14-17  child mask (bit c: child 4k + c exists)
//   18     leaf (level J)
//   19     level 1 (adds A_1 lambda_1 eta_1, or Phi eta for a level-1 leaf)
//   20     single child
//   21-25  level j
constexpr uint32_t kRecLeaf = 1u << 18;
constexpr uint32_t kRecRoot = 1u << 19;
constexpr uint32_t kRecSingle = 1u << 20;
__host__ __device__ __forceinline__ uint32_t rec_store_row(uint32_t meta) { return meta & 127u; }
__host__ __device__ __forceinline__ uint32_t rec_child_row(uint32_t meta) { return (meta >> 7) & 127u; }
__host__ __device__ __forceinline__ uint32_t rec_mask(uint32_t meta) { return (meta >> 14) & 15u; }
__host__ __device__ __forceinline__ uint32_t rec_level(uint32_t meta) { return (meta >> 21) & 31u; }

// float64 record (48 bytes).
//   leaf:     a, b, c = s_u, s_v, s_w - 1 (pixel centre, uvw frame); d = Phi
//   internal: a, b, c = gamma^0, gamma^1, gamma^2 -- for a single-child node
//             each multiplied by that child's sign in the Hadamard row
//             (exact), so that gamma^m sigma^m = a_m (q eta_c);
//             d = q = sqrt(A_j) / 4; e = A_1 lambda_1 at level 1, else 0
struct RecD {
    uint32_t meta;
    uint32_t pad;
    double a, b, c, d, e;
};
static_assert(sizeof(RecD) == 48, "RecD layout");

// float32 record of the mixed form (32 bytes). The mixed predictors carry,
// per node, xi_j = 4^(J-j) eta_j: the plain sum of the children's xi (a
// leaf's xi is its eta), so the 1/4 of Eq. 9 disappears, and the factors
// q_j = sqrt(A_j)/4 and 4^-(J-j-1) that turn the children's xi into
// sigma^m are folded into gamma^m here, in float64, rounded once.
//   leaf:     (a, b), (c, d), (e, f) = s_u, s_v, s_w - 1 as double-float
//             pairs; g = Phi
//   internal: a, b, c = gamma^m q_j 4^-(J-j-1) (m = 0, 1, 2); for a
//             single-child node a = the sum of the three, each with that
//             child's Hadamard sign, and b = c = 0; d = 0;
//             g = A_1 lambda_1 4^-(J-1) at level 1, else 0
struct RecF {
    uint32_t meta;
    float a, b, c, d, e, f, g;
};
static_assert(sizeof(RecF) == 32, "RecF layout");

// Records of the regrouped Eq. 17 (WT_SUM_EQ17_REGROUPED). Per node n one
// weight w_n: for a node in child slot c of parent p at level j,
// w_n = q_j sum_m H_m[c] gamma^m_p (q_j = sqrt(A_j)/4, H the Eq. 10 sign
// rows), and w_n = A_1 lambda_1 at level 1; then, per visibility,
// V = sum_n w_n eta_n, the same sum as Eq. 17 with each node's
// sum_m gamma^m sigma^m distributed over its children
// (gamma^T (H eta) = (H^T gamma)^T eta). meta bits: 0-4 level, 5 leaf,
// 6 level 1, 7 first child of its parent (in post-order), 8 a leaf that
// takes its next record (its next sibling leaf) as a pair, 9 that second
// leaf of a pair, 10 a node at level J - 1 (its children are leaves),
// 11 a node at level J - 2, 12 the first leaf of a group: a run of sibling
// leaves whose parent (the next record after the run in post-order, a node
// at level J - 1) lies in the same staging chunk of kRecChunkW records, so
// that the run and its parent are taken in one step; bits 13-15 the run's
// length (1 to 4). The leaves of every run are paired greedily from its
// start, never across a staging chunk (in a group, from the group's start).
constexpr uint32_t kRwLeaf = 1u << 5;
constexpr uint32_t kRwRoot = 1u << 6;
constexpr uint32_t kRwFirst = 1u << 7;
constexpr uint32_t kRwPairFirst = 1u << 8;
constexpr uint32_t kRwPairSecond = 1u << 9;
constexpr uint32_t kRwLowSum = 1u << 10;
constexpr uint32_t kRwMidSum = 1u << 11;
constexpr uint32_t kRwGroup = 1u << 12;
constexpr int kRwGroupShift = 13;
constexpr int kRecChunkW = 128;   // records per staging buffer of the regrouped float32 form

// float64 (48 bytes): a, b, c = leaf pixel centre (s_u, s_v, s_w - 1); d = w.
struct RecWD {
    uint32_t meta;
    uint32_t pad;
    double a, b, c, d, e;
};
static_assert(sizeof(RecWD) == 48, "RecWD layout");

// float64-class double-float form (48 bytes): the fields of RecWD as
// double-floats: leaf pixel centre (s_u, s_v, s_w - 1) = (ah + al, bh + bl,
// ch + cl); weight w_n = wh + wl (every node); the leaf's merged flux
// Phi_k = fh + fl (Eq. 16; 0 for internal nodes).
struct RecWDF {
    uint32_t meta;
    float ah, al, bh, bl, ch, cl;
    float wh, wl;
    float fh, fl;
    float pad;
};
static_assert(sizeof(RecWDF) == 48, "RecWDF layout");

// mixed (32 bytes): leaf: (a, b), (c, d), (e, f) = pixel centre as
// double-float pairs; internal node: a, b = the stack rows of its own and
// its parent's xi sums (j - 1 and j - 2, 0 at level 1) as unsigned integers
// in the float fields; g = w_n 4^-(J-j), the weight of xi = 4^(J-j) eta.
struct RecWF {
    uint32_t meta;
    float a, b, c, d, e, f, g;
};
static_assert(sizeof(RecWF) == 32, "RecWF layout");

// Device-side header of a tree (written by the build kernels).
struct TreeHeader {
    int64_t n_leaves;
    int64_t n_nodes;
    int64_t per_level[kMaxJ + 1];   // [j] = nodes at level j (index 0 unused)
    int64_t rev_offset[kMaxJ + 2];  // start of level j in the level-J-first layout
    float smax[4];                  // max over the leaves of |s_u|, |s_v|, |s_w - 1| as the float32
                                    // heads of their records (0 for an empty tree); [3] unused
};

struct TreeDev {
    // capacity-sized arrays in "level J first" layout (level J, J-1, ..., 1)
    int64_t* key;
    double* lambda;
    double* gamma;        // [cap][3]
    int32_t* first_child; // index within the child level, -1 for leaves
    uint8_t* mask;
    int32_t* leaf_lo;     // first leaf index of the subtree
    int32_t* leaf_hi;     // one past the last leaf index
    int32_t* size;        // nodes in the subtree
    int32_t* parent;      // index of the parent within its level
    double* leaf_dir;     // [n_leaves cap][3]
    double* leaf_flux;    // [n_leaves cap]
    int64_t* anc_sum;     // per leaf: sum over levels of the ancestor's index
    int32_t* anc;         // per leaf: current ancestor index
    RecD* recd;           // post-order records [cap]
    RecF* recf;
    RecD* leafd;          // leaf records in key order [n_leaves cap] (Eq. 16)
    RecF* leaff;
    RecWD* recwd;         // post-order records of the regrouped Eq. 17 [cap]
    RecWF* recwf;
    RecWDF* recwdf;
    TreeHeader* hdr;
};

}  // namespace wt

// The opaque handle behind wt_tree.
struct wt_tree_s {
    uint64_t magic;
    int device;
    int J;
    double ra0, dec0;
    int64_t n_comp;
    int64_t cap_nodes;
    int64_t cap_leaves;
    cudaStream_t stream;          // stream of the build
    void* block;                  // single device allocation holding everything
    wt::TreeDev d;
    wt::TreeHeader* host_hdr;     // pinned copy of the header
    bool host_valid;
};

constexpr uint64_t kTreeMagic = 0x57545645455f3031ull;   // "WTVEE_01"

namespace wt {
// One wavelet-predictor launch, independent of the launch shape.
struct WaveletJob {
    const RecD* recd;        // post-order records (Eq. 17)
    const RecF* recf;
    const RecD* recd_leaf;   // leaf records (Eq. 16)
    const RecF* recf_leaf;
    const RecWD* recwd;      // regrouped Eq. 17
    const RecWF* recwf;
    const RecWDF* recwdf;    // regrouped Eq. 17, double-float
    const TreeHeader* hdr;
    const double* uvw;
    int64_t n_vis;
    void* vis;
    int mode, sign, which, J;
    int* status;
};

// tree_build.cu
// Where a tree's components come from: image-plane (l, m), or image pixels
// with their keys read from a cross-reference table (Sec. 3.5).
struct KeySource {
    const double* l = nullptr;
    const double* m = nullptr;
    const int64_t* table = nullptr;
    int64_t n_pix = 0;
    const int32_t* pix = nullptr;
    const int64_t* leaf_keys = nullptr;   // device: distinct level-J keys in ascending order (the fluxes
                                          // are the leaves' merged fluxes): no mapping, no sort
};
int build_tree(const KeySource& src, const double* flux, int64_t n_comp, double ra0, double dec0, int J, wt_tree t,
               cudaStream_t s);
int xref_table(int n, double dl, double ra0, double dec0, int J, int64_t* table, cudaStream_t s);
int tree_sync_header(wt_tree t);
// wavelet.cu
int predict_wavelet(wt_tree t, const double* uvw, int64_t n_vis, void* vis, int mode, int sign, int which,
                    cudaStream_t s);
extern const int kNumWaveletVariants;
int wavelet_variant_shape(int v, int* nt, int* vpt);
bool wavelet_variant_fits(int v, int mode, int which, int J);
size_t wavelet_variant_smem(int v, int mode, int which, int J);
int launch_wavelet(const WaveletJob& jb, int v, cudaStream_t s);
int default_wavelet_variant(int mode, int which, int J);
// autotune.cu
int choose_wavelet_variant(wt_tree t, const WaveletJob& jb, cudaStream_t s);
// batched.cu
int predict_batched(const wt_tree* trees, const double* freq_hz, int n_ch, const double* uvw_m, int64_t n_vis,
                    void* vis, int mode, int sign, cudaStream_t s);
void batch_forget_tree(wt_tree t);
// A device buffer of the current device holding at least `bytes` from p,
// p a multiple of `align` (the widest access the kernels make to it: 16 for
// complex128, 8 for float64 and complex64, 4 for int32 and float32); else
// WT_ERR_ARG with a message, before anything is launched.
int check_device_buffer(const void* p, size_t bytes, const char* fn, const char* name, size_t align);
// Alignment of a visibility buffer of `mode` (complex128 or complex64).
inline size_t vis_align(int mode) { return (mode == WT_FP64 || mode == WT_FP64_DF) ? 16 : 8; }
// dft_tc.cu: Eq. 16 over leaf records with the phase on the tensor cores
int eq16_tc_launch(const RecF* recs, const TreeHeader* hdr, int64_t cap, int64_t n_hint, const double* uvw,
                   int64_t n_vis, float2* vis, int sign, int* status, cudaStream_t s, const char* fn);
// dft.cu
int predict_dft(const double* l, const double* m, const double* flux, int64_t n_comp, const double* uvw,
                int64_t n_vis, void* vis, int mode, int sign, cudaStream_t s);
// subtract.cu
int subtract(const void* obs, const void* model, void* resid, int64_t n_vis, int mode, cudaStream_t s);
// utilities
int num_sms();
void rotation_matrix(double ra0, double dec0, double* R);
}  // namespace wt
