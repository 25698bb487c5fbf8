// wavelet_bodies.cuh -- per-record work of the wavelet predictors, shared by
// the single-tree kernels (wavelet.cu) and the batched kernel (batched.cu).
// Each body is called once per node record, in post-order, with the same
// record for every thread of the CTA; see wavelet.cu for the mapping.
#pragma once

#include "staging.cuh"
#include "wt_internal.cuh"

namespace wt {
namespace {

constexpr int kChunkD = 256;   // records per staging buffer (48 B each)
constexpr int kChunkF = 384;   // (32 B each)

__device__ __forceinline__ int clamp_row(uint32_t r, int maxrow) { return min(static_cast<int>(r), maxrow); }

// ---------------------------------------------------------------- float64
template <int NT, int VPT>
struct Eq17D {
    double u[VPT], v[VPT], w[VPT];
    double vr[VPT], vi[VPT];
    double sgn;
    double2* stk;   // shared stack + threadIdx.x; row stride VPT * NT
    int maxrow;     // 4 (J - 1) - 1

    __device__ __forceinline__ double2& slot(int row, int k) { return stk[(row * VPT + k) * NT]; }

    __device__ void operator()(const RecD& r)
    {
        const uint32_t meta = r.meta;
        const bool root = meta & kRecRoot;
        const int srow = clamp_row(rec_store_row(meta), maxrow);
        if (meta & kRecLeaf) {
#pragma unroll
            for (int k = 0; k < VPT; ++k) {
                double t = fma(w[k], r.c, fma(v[k], r.b, u[k] * r.a));
                double s, c;
                sincos_turns_f64(t, s, c);
                const double ei = s;
                if (root) {
                    vr[k] = fma(r.d, c, vr[k]);
                    vi[k] = fma(r.d, ei, vi[k]);
                } else {
                    slot(srow, k) = make_double2(c, ei);
                }
            }
        } else if (meta & kRecSingle) {
            const int crow = clamp_row(rec_child_row(meta), maxrow);
#pragma unroll
            for (int k = 0; k < VPT; ++k) {
                const double2 c = slot(crow, k);
                const double er = 0.25 * c.x, ei = 0.25 * c.y;
                const double sr = r.d * c.x, si = r.d * c.y;   // q eta_c; sigma^m = (sign) (sr, si)
                vr[k] = fma(r.a, sr, fma(r.b, sr, fma(r.c, sr, vr[k])));
                vi[k] = fma(r.a, si, fma(r.b, si, fma(r.c, si, vi[k])));
                if (root) {
                    vr[k] = fma(r.e, er, vr[k]);
                    vi[k] = fma(r.e, ei, vi[k]);
                } else {
                    slot(srow, k) = make_double2(er, ei);
                }
            }
        } else {
            const int crow = clamp_row(rec_child_row(meta), maxrow - 3);
            const uint32_t mask = rec_mask(meta);
#pragma unroll
            for (int k = 0; k < VPT; ++k) {
                double2 c0 = make_double2(0.0, 0.0), c1 = c0, c2 = c0, c3 = c0;
                if (mask & 1u) c0 = slot(crow, k);
                if (mask & 2u) c1 = slot(crow + 1, k);
                if (mask & 4u) c2 = slot(crow + 2, k);
                if (mask & 8u) c3 = slot(crow + 3, k);
                const double ar = c0.x + c1.x, ai = c0.y + c1.y;   // c0 + c1
                const double br = c0.x - c1.x, bi = c0.y - c1.y;   // c0 - c1
                const double cr = c2.x + c3.x, ci = c2.y + c3.y;   // c2 + c3
                const double dr = c2.x - c3.x, di = c2.y - c3.y;   // c2 - c3
                const double er = 0.25 * (ar + cr), ei = 0.25 * (ai + ci);   // Eq. 9 form
                const double q = r.d;                                        // Eq. 10 form:
                const double s0r = q * (br + dr), s0i = q * (bi + di);      //   + - + -
                const double s1r = q * (ar - cr), s1i = q * (ai - ci);      //   + + - -
                const double s2r = q * (br - dr), s2i = q * (bi - di);      //   + - - +
                vr[k] = fma(r.a, s0r, fma(r.b, s1r, fma(r.c, s2r, vr[k])));
                vi[k] = fma(r.a, s0i, fma(r.b, s1i, fma(r.c, s2i, vi[k])));
                if (root) {
                    vr[k] = fma(r.e, er, vr[k]);
                    vi[k] = fma(r.e, ei, vi[k]);
                } else {
                    slot(srow, k) = make_double2(er, ei);
                }
            }
        }
    }
};

template <int VPT>
struct Eq16D {
    double u[VPT], v[VPT], w[VPT];
    double vr[VPT], vi[VPT];
    double sgn;
    __device__ void operator()(const RecD& r)
    {
#pragma unroll
        for (int k = 0; k < VPT; ++k) {
            double t = fma(w[k], r.c, fma(v[k], r.b, u[k] * r.a));
            double s, c;
            sincos_turns_f64(t, s, c);
            vr[k] = fma(r.d, c, vr[k]);
            vi[k] = fma(r.d, s, vi[k]);
        }
    }
};

// ---------------------------------------------------------------- mixed
template <int NT, int VPT, bool FAST = false>
struct Eq17F {
    F2 u[VPT], v[VPT], w[VPT];
    float vr[VPT], vi[VPT], cr[VPT], ci[VPT];   // Kahan sums and compensations
    float sgn;
    float2* stk;
    int maxrow;

    __device__ __forceinline__ float2& slot(int row, int k) { return stk[(row * VPT + k) * NT]; }

    __device__ void operator()(const RecF& r)
    {
        const uint32_t meta = r.meta;
        const bool root = meta & kRecRoot;
        const int srow = clamp_row(rec_store_row(meta), maxrow);
        if (meta & kRecLeaf) {
            const F2 su{r.a, r.b}, sv{r.c, r.d}, sw{r.e, r.f};
#pragma unroll
            for (int k = 0; k < VPT; ++k) {
                float th, tl, s, c;
                phase_turns_df(u[k], v[k], w[k], su, sv, sw, th, tl);
                sincos_mixed<FAST>(th, tl, s, c);
                const float ei = s;
                if (root) {
                    kahan_add(vr[k], cr[k], r.g * c);
                    kahan_add(vi[k], ci[k], r.g * ei);
                } else {
                    slot(srow, k) = make_float2(c, ei);
                }
            }
        } else if (meta & kRecSingle) {
            const int crow = clamp_row(rec_child_row(meta), maxrow);
#pragma unroll
            for (int k = 0; k < VPT; ++k) {
                const float2 c = slot(crow, k);
                const float er = 0.25f * c.x, ei = 0.25f * c.y;
                const float sr = r.d * c.x, si = r.d * c.y;
                float xr = fmaf(r.a, sr, fmaf(r.b, sr, r.c * sr));
                float xi = fmaf(r.a, si, fmaf(r.b, si, r.c * si));
                if (root) {
                    xr = fmaf(r.g, er, xr);
                    xi = fmaf(r.g, ei, xi);
                } else {
                    slot(srow, k) = make_float2(er, ei);
                }
                kahan_add(vr[k], cr[k], xr);
                kahan_add(vi[k], ci[k], xi);
            }
        } else {
            const int crow = clamp_row(rec_child_row(meta), maxrow - 3);
            const uint32_t mask = rec_mask(meta);
#pragma unroll
            for (int k = 0; k < VPT; ++k) {
                float2 c0 = make_float2(0.f, 0.f), c1 = c0, c2 = c0, c3 = c0;
                if (mask & 1u) c0 = slot(crow, k);
                if (mask & 2u) c1 = slot(crow + 1, k);
                if (mask & 4u) c2 = slot(crow + 2, k);
                if (mask & 8u) c3 = slot(crow + 3, k);
                const float ar = c0.x + c1.x, ai = c0.y + c1.y;
                const float br = c0.x - c1.x, bi = c0.y - c1.y;
                const float cr_ = c2.x + c3.x, ci_ = c2.y + c3.y;
                const float dr = c2.x - c3.x, di = c2.y - c3.y;
                const float er = 0.25f * (ar + cr_), ei = 0.25f * (ai + ci_);
                const float q = r.d;
                const float s0r = q * (br + dr), s0i = q * (bi + di);
                const float s1r = q * (ar - cr_), s1i = q * (ai - ci_);
                const float s2r = q * (br - dr), s2i = q * (bi - di);
                float xr = fmaf(r.a, s0r, fmaf(r.b, s1r, r.c * s2r));
                float xi = fmaf(r.a, s0i, fmaf(r.b, s1i, r.c * s2i));
                if (root) {
                    xr = fmaf(r.g, er, xr);
                    xi = fmaf(r.g, ei, xi);
                } else {
                    slot(srow, k) = make_float2(er, ei);
                }
                kahan_add(vr[k], cr[k], xr);
                kahan_add(vi[k], ci[k], xi);
            }
        }
    }
};

template <int VPT, bool FAST = false>
struct Eq16F {
    F2 u[VPT], v[VPT], w[VPT];
    float vr[VPT], vi[VPT], cr[VPT], ci[VPT];
    float sgn;
    __device__ void operator()(const RecF& r)
    {
        const F2 su{r.a, r.b}, sv{r.c, r.d}, sw{r.e, r.f};
#pragma unroll
        for (int k = 0; k < VPT; ++k) {
            float th, tl, s, c;
            phase_turns_df(u[k], v[k], w[k], su, sv, sw, th, tl);
            sincos_mixed<FAST>(th, tl, s, c);
            kahan_add(vr[k], cr[k], r.g * c);
            kahan_add(vi[k], ci[k], r.g * s);
        }
    }
};

// ---------------------------------------------------------------- regrouped Eq. 17
// V = sum_n w_n eta_n (see RecWD in wt_internal.cuh). Per level j = 1 .. J-2
// a thread keeps two accumulators of the open level-j node in shared memory
// (row 2(j-1): sum of its children's eta; row 2(j-1)+1: sum of w_c eta_c);
// those of the open level-(J-1) node live in registers, so a leaf never
// touches shared memory. A node reads its own accumulators, forms
// eta = (1/4) sum (the Eq. 9 form), adds the children's weighted sum to V
// and passes eta and w eta up to its parent (the first child writes, the
// others add).
template <int NT, int VPT>
struct Eq17WD {
    double u[VPT], v[VPT], w[VPT];
    double vr[VPT], vi[VPT];
    double sr[VPT], si[VPT], xr[VPT], xi[VPT];
    double2* stk;   // shared stack + threadIdx.x; row stride VPT * NT
    int J;
    int maxrow;

    __device__ __forceinline__ double2& slot(int row, int k) { return stk[(row * VPT + k) * NT]; }

    __device__ void operator()(const RecWD& r)
    {
        const uint32_t meta = r.meta;
        const int lev = static_cast<int>(meta & 31u);
        const bool root = meta & kRwRoot, first = meta & kRwFirst;
        if (meta & kRwLeaf) {
#pragma unroll
            for (int k = 0; k < VPT; ++k) {
                const double t = fma(w[k], r.c, fma(v[k], r.b, u[k] * r.a));
                double s, c;
                sincos_turns_f64(t, s, c);
                if (root) {
                    vr[k] = fma(r.d, c, vr[k]);
                    vi[k] = fma(r.d, s, vi[k]);
                } else if (first) {
                    sr[k] = c;
                    si[k] = s;
                    xr[k] = r.d * c;
                    xi[k] = r.d * s;
                } else {
                    sr[k] += c;
                    si[k] += s;
                    xr[k] = fma(r.d, c, xr[k]);
                    xi[k] = fma(r.d, s, xi[k]);
                }
            }
            return;
        }
        const bool in_regs = (lev == J - 1);
        const int own = clamp_row(static_cast<uint32_t>(2 * (lev - 1)), maxrow - 1);
        const int par = clamp_row(static_cast<uint32_t>(2 * (lev > 1 ? lev - 2 : 0)), maxrow - 1);
#pragma unroll
        for (int k = 0; k < VPT; ++k) {
            double2 S, X;
            if (in_regs) {
                S = make_double2(sr[k], si[k]);
                X = make_double2(xr[k], xi[k]);
            } else {
                S = slot(own, k);
                X = slot(own + 1, k);
            }
            const double er = 0.25 * S.x, ei = 0.25 * S.y;   // Eq. 9 form
            vr[k] += X.x;
            vi[k] += X.y;
            if (root) {
                vr[k] = fma(r.d, er, vr[k]);
                vi[k] = fma(r.d, ei, vi[k]);
            } else if (first) {
                slot(par, k) = make_double2(er, ei);
                slot(par + 1, k) = make_double2(r.d * er, r.d * ei);
            } else {
                double2& ps = slot(par, k);
                double2& px = slot(par + 1, k);
                ps = make_double2(ps.x + er, ps.y + ei);
                px = make_double2(fma(r.d, er, px.x), fma(r.d, ei, px.y));
            }
        }
    }
};

template <int NT, int VPT, bool FAST = false>
struct Eq17WF {
    F2 u[VPT], v[VPT], w[VPT];
    float vr[VPT], vi[VPT], cr[VPT], ci[VPT];   // Kahan sums and compensations
    float sr[VPT], si[VPT], xr[VPT], xi[VPT];
    float2* stk;
    int J;
    int maxrow;

    __device__ __forceinline__ float2& slot(int row, int k) { return stk[(row * VPT + k) * NT]; }

    __device__ void operator()(const RecWF& r)
    {
        const uint32_t meta = r.meta;
        const int lev = static_cast<int>(meta & 31u);
        const bool root = meta & kRwRoot, first = meta & kRwFirst;
        if (meta & kRwLeaf) {
            const F2 su{r.a, r.b}, sv{r.c, r.d}, sw{r.e, r.f};
#pragma unroll
            for (int k = 0; k < VPT; ++k) {
                float th, tl, s, c;
                phase_turns_df(u[k], v[k], w[k], su, sv, sw, th, tl);
                sincos_mixed<FAST>(th, tl, s, c);
                if (root) {
                    kahan_add(vr[k], cr[k], r.g * c);
                    kahan_add(vi[k], ci[k], r.g * s);
                } else if (first) {
                    sr[k] = c;
                    si[k] = s;
                    xr[k] = r.g * c;
                    xi[k] = r.g * s;
                } else {
                    sr[k] += c;
                    si[k] += s;
                    xr[k] = fmaf(r.g, c, xr[k]);
                    xi[k] = fmaf(r.g, s, xi[k]);
                }
            }
            return;
        }
        const bool in_regs = (lev == J - 1);
        const int own = clamp_row(static_cast<uint32_t>(2 * (lev - 1)), maxrow - 1);
        const int par = clamp_row(static_cast<uint32_t>(2 * (lev > 1 ? lev - 2 : 0)), maxrow - 1);
#pragma unroll
        for (int k = 0; k < VPT; ++k) {
            float2 S, X;
            if (in_regs) {
                S = make_float2(sr[k], si[k]);
                X = make_float2(xr[k], xi[k]);
            } else {
                S = slot(own, k);
                X = slot(own + 1, k);
            }
            const float er = 0.25f * S.x, ei = 0.25f * S.y;
            kahan_add(vr[k], cr[k], X.x);
            kahan_add(vi[k], ci[k], X.y);
            if (root) {
                kahan_add(vr[k], cr[k], r.g * er);
                kahan_add(vi[k], ci[k], r.g * ei);
            } else if (first) {
                slot(par, k) = make_float2(er, ei);
                slot(par + 1, k) = make_float2(r.g * er, r.g * ei);
            } else {
                float2& ps = slot(par, k);
                float2& px = slot(par + 1, k);
                ps = make_float2(ps.x + er, ps.y + ei);
                px = make_float2(fmaf(r.g, er, px.x), fmaf(r.g, ei, px.y));
            }
        }
    }
};

}  // namespace
}  // namespace wt
