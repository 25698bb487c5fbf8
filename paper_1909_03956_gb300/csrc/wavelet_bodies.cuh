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
template <int NT, int VPT>
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
                sincos_turns_f32(th, tl, s, c);
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

template <int VPT>
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
            sincos_turns_f32(th, tl, s, c);
            kahan_add(vr[k], cr[k], r.g * c);
            kahan_add(vi[k], ci[k], r.g * s);
        }
    }
};

}  // namespace
}  // namespace wt
