// wavelet_bodies.cuh -- per-record work of the wavelet predictors, shared by
// the single-tree kernels (wavelet.cu) and the batched kernel (batched.cu).
// Each body is called once per node record, in post-order, with the same
// record for every thread of the CTA; see wavelet.cu for the mapping.
#pragma once

#include "df64.cuh"
#include "staging.cuh"
#include "wt_internal.cuh"

namespace wt {
namespace {

constexpr int kChunkD = 256;   // records per staging buffer (48 B each)
constexpr int kChunkDF = 128;  // double-float form (48 B each): smaller buffers, more CTAs per SM
constexpr int kChunkF = 384;   // (32 B each)
constexpr int kChunkW = kRecChunkW;   // regrouped float32 form (32 B each): its stack is small, so the
                               // staging buffers set how many CTAs fit on an SM

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
// Eq. 17 in the mixed forms, on packed float32 pairs. A thread's stack
// holds xi = 4^(J-j) eta (RecF): a node's xi is the plain sum of its
// children's, and gamma^m sigma^m = a_m (H_m xi_children) with the scale
// factors already in a_m. A complex value is one pair; the leaf phases of
// visibilities 2p and 2p + 1 are formed as one pair (VPT = 1 forms its one
// phase on scalars). Per visibility a four-child node costs 15 paired
// operations, Kahan included.
template <int NT, int VPT, bool FAST = false, bool GRID = false>
struct Eq17F {
    static constexpr int NP = VPT / 2;                // visibility pairs
    static constexpr bool ODD = (VPT & 1) != 0;       // a last, unpaired visibility
    F2 u[VPT], v[VPT], w[VPT];                        // set by the caller, then start()
    DF2 U[NP > 0 ? NP : 1], V[NP > 0 ? NP : 1], W[NP > 0 ? NP : 1];
    float2 Cg[NP > 0 ? NP : 1];                       // GRID: the grid constants of visibilities 2p, 2p + 1
    float Cs;                                         // GRID: that of the last, unpaired visibility
    float2 acc[VPT], comp[VPT];                       // Kahan sum of V and its compensation
    float2* stk;
    int maxrow;

    __device__ __forceinline__ float2& slot(int row, int k) { return stk[(row * VPT + k) * NT]; }

    __device__ __forceinline__ void start()
    {
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            U[p] = df2_pack(u[2 * p], u[2 * p + 1]);
            V[p] = df2_pack(v[2 * p], v[2 * p + 1]);
            W[p] = df2_pack(w[2 * p], w[2 * p + 1]);
        }
#pragma unroll
        for (int k = 0; k < VPT; ++k) {
            acc[k] = make_float2(0.f, 0.f);
            comp[k] = make_float2(0.f, 0.f);
        }
    }

    __device__ __forceinline__ float2 result(int k) const { return sub2(acc[k], comp[k]); }

    __device__ __forceinline__ void emit(int k, bool root, int srow, float g, float2 e)
    {
        if (root) kahan_add2(acc[k], comp[k], mul2(bcast2(g), e));
        else slot(srow, k) = e;
    }

    __device__ void operator()(const RecF& r)
    {
        const uint32_t meta = r.meta;
        const bool root = meta & kRecRoot;
        const int srow = clamp_row(rec_store_row(meta), maxrow);
        if (meta & kRecLeaf) {
            const F2 su{r.a, r.b}, sv{r.c, r.d}, sw{r.e, r.f};
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                float2 h, tl, e0, e1;
                if constexpr (GRID) phase_turns_grid2(U[p], V[p], W[p], su, sv, sw, Cg[p], h, tl);
                else phase_turns_df2(U[p], V[p], W[p], su, sv, sw, h, tl);
                sincos_mixed2<FAST>(h, tl, e0, e1);
                emit(2 * p, root, srow, r.g, e0);
                emit(2 * p + 1, root, srow, r.g, e1);
            }
            if constexpr (ODD) {
                constexpr int k = VPT - 1;
                float th, tl, s, c;
                if constexpr (GRID) phase_turns_grid(u[k], v[k], w[k], su, sv, sw, Cs, th, tl);
                else phase_turns_df(u[k], v[k], w[k], su, sv, sw, th, tl);
                sincos_mixed<FAST>(th, tl, s, c);
                emit(k, root, srow, r.g, make_float2(c, s));
            }
        } else if (meta & kRecSingle) {
            const int crow = clamp_row(rec_child_row(meta), maxrow);
            const float2 a = bcast2(r.a), g = bcast2(r.g);
#pragma unroll
            for (int k = 0; k < VPT; ++k) {
                const float2 xi = slot(crow, k);             // the node's xi is its child's
                float2 x = mul2(a, xi);
                if (root) x = fma2(g, xi, x);
                else slot(srow, k) = xi;
                kahan_add2(acc[k], comp[k], x);
            }
        } else {
            const int crow = clamp_row(rec_child_row(meta), maxrow - 3);
            const uint32_t mask = rec_mask(meta);
            const float2 ga = bcast2(r.a), gb = bcast2(r.b), gc = bcast2(r.c), g = bcast2(r.g);
#pragma unroll
            for (int k = 0; k < VPT; ++k) {
                float2 c0 = make_float2(0.f, 0.f), c1 = c0, c2 = c0, c3 = c0;
                if (mask & 1u) c0 = slot(crow, k);
                if (mask & 2u) c1 = slot(crow + 1, k);
                if (mask & 4u) c2 = slot(crow + 2, k);
                if (mask & 8u) c3 = slot(crow + 3, k);
                const float2 a = add2(c0, c1), b = sub2(c0, c1);   // c0 +- c1
                const float2 c = add2(c2, c3), d = sub2(c2, c3);   // c2 +- c3
                const float2 xi = add2(a, c);                      // Eq. 9 (times 4^(J-j))
                // Eq. 10 rows (+ - + -), (+ + - -), (+ - - +), weighted by gamma
                float2 x = fma2(ga, add2(b, d), fma2(gb, sub2(a, c), mul2(gc, sub2(b, d))));
                if (root) x = fma2(g, xi, x);
                else slot(srow, k) = xi;
                kahan_add2(acc[k], comp[k], x);
            }
        }
    }
};

// Eq. 16 in the mixed forms on packed pairs: a thread's visibilities taken
// two at a time (their phases against one leaf as one pair of double-floats,
// each visibility's (cos, sin) its own pair), an odd last visibility of the
// thread alone; the leaf records kSumBlock at a time (their terms added by
// FMAs into a partial per visibility, the partial then into its Kahan sum:
// blockwise compensated summation). GRID: the phases with their heads on each visibility's
// grid (constants Cg / Cs, set by the caller; phase_turns_grid2), else with
// error-free sums (phase_turns_df2).
template <int VPT, bool FAST, bool GRID>
struct Eq16F2 {
    static constexpr int NP = VPT / 2;
    static constexpr bool ODD = (VPT & 1) != 0;
    DF2 U[NP > 0 ? NP : 1], V[NP > 0 ? NP : 1], W[NP > 0 ? NP : 1];
    F2 us, vs, ws;                                    // the unpaired last visibility
    float2 Cg[NP > 0 ? NP : 1];
    float Cs;
    float2 acc[VPT], comp[VPT];

    __device__ __forceinline__ void start(const F2 (&u)[VPT], const F2 (&v)[VPT], const F2 (&w)[VPT],
                                          const float (&C)[VPT])
    {
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            U[p] = df2_pack(u[2 * p], u[2 * p + 1]);
            V[p] = df2_pack(v[2 * p], v[2 * p + 1]);
            W[p] = df2_pack(w[2 * p], w[2 * p + 1]);
            Cg[p] = make_float2(C[2 * p], C[2 * p + 1]);
        }
        us = u[VPT - 1];
        vs = v[VPT - 1];
        ws = w[VPT - 1];
        Cs = C[VPT - 1];
#pragma unroll
        for (int k = 0; k < VPT; ++k) {
            acc[k] = make_float2(0.f, 0.f);
            comp[k] = make_float2(0.f, 0.f);
        }
    }

    __device__ __forceinline__ float2 result(int k) const { return sub2(acc[k], comp[k]); }

    // One leaf's terms into the partials: p[k] += Phi exp(i 2 pi phase) of
    // visibility k.
    __device__ __forceinline__ void add_terms(const RecF& r, float2 (&x)[VPT]) const
    {
        const F2 su{r.a, r.b}, sv{r.c, r.d}, sw{r.e, r.f};
        const float2 fl = bcast2(r.g);
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            float2 h, tl, e0, e1;
            if constexpr (GRID) phase_turns_grid2(U[p], V[p], W[p], su, sv, sw, Cg[p], h, tl);
            else phase_turns_df2(U[p], V[p], W[p], su, sv, sw, h, tl);
            sincos_mixed2<FAST>(h, tl, e0, e1);
            x[2 * p] = fma2(fl, e0, x[2 * p]);
            x[2 * p + 1] = fma2(fl, e1, x[2 * p + 1]);
        }
        if constexpr (ODD) {
            float th, tl, sn, cs;
            if constexpr (GRID) phase_turns_grid(us, vs, ws, su, sv, sw, Cs, th, tl);
            else phase_turns_df(us, vs, ws, su, sv, sw, th, tl);
            sincos_mixed<FAST>(th, tl, sn, cs);
            x[VPT - 1] = fma2(fl, make_float2(cs, sn), x[VPT - 1]);
        }
    }

    // One block of leaves from record r on; returns how many it took
    // (kSumBlock, or what is left of a list's last chunk).
    __device__ __forceinline__ int at(const RecF* cb, int r, int n)
    {
        float2 x[VPT];
#pragma unroll
        for (int k = 0; k < VPT; ++k) x[k] = make_float2(0.f, 0.f);
        int taken;
        if (r + kSumBlock <= n) {
#pragma unroll 2
            for (int j = 0; j < kSumBlock; ++j) add_terms(cb[r + j], x);
            taken = kSumBlock;
        } else {
            for (int j = r; j < n; ++j) add_terms(cb[j], x);
            taken = n - r;
        }
#pragma unroll
        for (int k = 0; k < VPT; ++k) kahan_add2(acc[k], comp[k], x[k]);
        return taken;
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

// Eq. 16 in double-float (WT_FP64_DF, RecWDF): V = sum over the leaves of
// Phi_k times the plane wave at the pixel centre; internal records are
// passed over.
template <int VPT>
struct Eq16DF {
    F2 u[VPT], v[VPT], w[VPT];
    DF vr[VPT], vi[VPT];
    const float4* tab;
    __device__ void operator()(const RecWDF& r)
    {
        if (!(r.meta & kRwLeaf)) return;
        const F2 su{r.ah, r.al}, sv{r.bh, r.bl}, sw{r.ch, r.cl};
        const DF phi{r.fh, r.fl};
#pragma unroll
        for (int k = 0; k < VPT; ++k) {
            float th, tl;
            phase_turns_df(u[k], v[k], w[k], su, sv, sw, th, tl);
            DF s, c;
            sincos_turns_df(th, tl, tab, s, c);
            vr[k] = df_add(vr[k], df_mul(phi, c));
            vi[k] = df_add(vi[k], df_mul(phi, s));
        }
    }
};

// Regrouped Eq. 17 in double-float (WT_FP64_DF, RecWDF): V = sum_n w_n eta_n
// with every quantity a double-float on the float32 pipe. Each node adds
// its w eta to V as soon as its eta is known. Per visibility a thread keeps
// the sum of the children's eta of the open level-j node (j = 1 .. J-2) in
// shared-memory row j - 1 as (re h, re l, im h, im l); that of the open
// level-(J-1) node lives in registers, so a leaf never touches shared
// memory. A node's eta is a quarter of its children's sum (the Eq. 9 form;
// exact scaling), which it passes up to its parent (the first child
// writes, the others add).
template <int NT, int VPT>
struct Eq17DF {
    F2 u[VPT], v[VPT], w[VPT];
    DF vr[VPT], vi[VPT];   // V
    DF lr[VPT], li[VPT];   // children's eta sum of the open level-(J-1) node
    float4* stk;           // shared stack + threadIdx.x; row stride VPT * NT
    const float4* tab;     // exp(i 2 pi k/256), sincos_turns_df
    int J;
    int maxrow;

    __device__ __forceinline__ float4& slot(int row, int k) { return stk[(row * VPT + k) * NT]; }

    __device__ void operator()(const RecWDF& r)
    {
        const uint32_t meta = r.meta;
        const int lev = static_cast<int>(meta & 31u);
        const bool root = meta & kRwRoot, first = meta & kRwFirst;
        const DF wgt{r.wh, r.wl};
        if (meta & kRwLeaf) {
            const F2 su{r.ah, r.al}, sv{r.bh, r.bl}, sw{r.ch, r.cl};
#pragma unroll
            for (int k = 0; k < VPT; ++k) {
                float th, tl;
                phase_turns_df(u[k], v[k], w[k], su, sv, sw, th, tl);
                DF s, c;
                sincos_turns_df(th, tl, tab, s, c);
                vr[k] = df_add(vr[k], df_mul(wgt, c));
                vi[k] = df_add(vi[k], df_mul(wgt, s));
                if (root) continue;
                if (first) {
                    lr[k] = c;
                    li[k] = s;
                } else {
                    lr[k] = df_add(lr[k], c);
                    li[k] = df_add(li[k], s);
                }
            }
            return;
        }
        const bool in_regs = (lev == J - 1);
        const int own = clamp_row(static_cast<uint32_t>(lev > 1 ? lev - 1 : 0), maxrow);
        const int par = clamp_row(static_cast<uint32_t>(lev > 2 ? lev - 2 : 0), maxrow);
#pragma unroll
        for (int k = 0; k < VPT; ++k) {
            DF er, ei;
            if (in_regs) {
                er = df_scale(lr[k], 0.25f);
                ei = df_scale(li[k], 0.25f);
            } else {
                const float4 S = slot(own, k);
                er = DF{0.25f * S.x, 0.25f * S.y};
                ei = DF{0.25f * S.z, 0.25f * S.w};
            }
            vr[k] = df_add(vr[k], df_mul(wgt, er));
            vi[k] = df_add(vi[k], df_mul(wgt, ei));
            if (root) continue;
            float4& P = slot(par, k);
            if (first) {
                P = make_float4(er.h, er.l, ei.h, ei.l);
            } else {
                const DF pr = df_add(DF{P.x, P.y}, er), pi = df_add(DF{P.z, P.w}, ei);
                P = make_float4(pr.h, pr.l, pi.h, pi.l);
            }
        }
    }
};

// Regrouped Eq. 17 in the mixed forms: V = sum_n w_n xi_n over every node,
// xi = 4^(J-j) eta and w_n scaled to match by the build (RecWF). Per
// visibility a thread keeps one pair per level: the xi sum of the open
// level-j node (j = 1 .. J-3) in shared-memory row j - 1 (layout
// [row][thread][vis]: a thread's visibilities side by side, one 16-byte
// access per row at two visibilities per thread); those of the open
// level-(J-1) and level-(J-2) nodes live in registers, with the plain
// float32 sums of their children's terms (w xi, at most four each), so
// leaves and level-(J-1) nodes touch neither shared memory nor the
// compensated sum. Any other internal node reads its xi, adds w xi (plus,
// at level J-2, its children's terms) to V with compensation and passes xi
// up (the first child writes its parent's sum, the others add).
// Packed pairs as in Eq17F. GRID: the leaf phases with their heads on the
// common grid of each visibility's constant C (phase_turns_grid2; the
// caller sets Cg and Cs and guarantees that the grid is valid), else with
// error-free sums (phase_turns_df2). GROUPS: the fast form takes a group
// (a run of sibling leaves and their level-(J-1) parent) in one step of a
// variable-stride sweep, else every record in a fixed-stride sweep, the
// second leaf of a pair skipped (measured: groups faster in the single-tree
// predictor, slower in the batched one).
template <int NT, int VPT, bool FAST = false, bool GRID = false, bool GROUPS = true>
struct Eq17WF {
    static constexpr int NP = VPT / 2;
    static constexpr bool ODD = (VPT & 1) != 0;
    F2 u[VPT], v[VPT], w[VPT];                        // set by the caller, then start()
    DF2 U[NP > 0 ? NP : 1], V[NP > 0 ? NP : 1], W[NP > 0 ? NP : 1];
    float2 Cg[NP > 0 ? NP : 1];                       // GRID: the grid constants of visibilities 2p, 2p + 1
    float Cs;                                         // GRID: that of the last, unpaired visibility
    float2 acc[VPT], comp[VPT];                       // Kahan sum of V and its compensation
    float2 low[VPT];                                  // xi sum of the open level-(J-1) node
    float2 lowx[VPT];                                 // w xi sum of its leaves
    float2 mid[VPT];                                  // xi sum of the open level-(J-2) node
    float2 midx[VPT];                                 // plain sum of the terms of its children
                                                      // (at most 4)
    float2* stk;                                      // shared stack + threadIdx.x * VPT
    int J;
    int maxrow;

    __device__ __forceinline__ float2* row_ptr(int row) { return stk + row * (NT * VPT); }

    __device__ __forceinline__ void load_row(int row, float2 (&x)[VPT])
    {
        const float2* p = row_ptr(row);
        if constexpr (VPT % 2 == 0) {
#pragma unroll
            for (int k = 0; k < VPT; k += 2) {
                const float4 q = *reinterpret_cast<const float4*>(p + k);
                x[k] = make_float2(q.x, q.y);
                x[k + 1] = make_float2(q.z, q.w);
            }
        } else {
#pragma unroll
            for (int k = 0; k < VPT; ++k) x[k] = p[k];
        }
    }

    __device__ __forceinline__ void store_row(int row, const float2 (&x)[VPT])
    {
        float2* p = row_ptr(row);
        if constexpr (VPT % 2 == 0) {
#pragma unroll
            for (int k = 0; k < VPT; k += 2)
                *reinterpret_cast<float4*>(p + k) = make_float4(x[k].x, x[k].y, x[k + 1].x, x[k + 1].y);
        } else {
#pragma unroll
            for (int k = 0; k < VPT; ++k) p[k] = x[k];
        }
    }

    __device__ __forceinline__ void start()
    {
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            U[p] = df2_pack(u[2 * p], u[2 * p + 1]);
            V[p] = df2_pack(v[2 * p], v[2 * p + 1]);
            W[p] = df2_pack(w[2 * p], w[2 * p + 1]);
        }
#pragma unroll
        for (int k = 0; k < VPT; ++k) {
            acc[k] = make_float2(0.f, 0.f);
            comp[k] = make_float2(0.f, 0.f);
            low[k] = make_float2(0.f, 0.f);
            lowx[k] = make_float2(0.f, 0.f);
            mid[k] = make_float2(0.f, 0.f);
            midx[k] = make_float2(0.f, 0.f);
        }
    }

    __device__ __forceinline__ float2 result(int k) const { return sub2(acc[k], comp[k]); }

    __device__ __forceinline__ void phase2(int p, F2 su, F2 sv, F2 sw, float2& h, float2& tl) const
    {
        if constexpr (GRID) phase_turns_grid2(U[p], V[p], W[p], su, sv, sw, Cg[p], h, tl);
        else phase_turns_df2(U[p], V[p], W[p], su, sv, sw, h, tl);
    }

    __device__ __forceinline__ void phase1(F2 su, F2 sv, F2 sw, float& th, float& tl) const
    {
        constexpr int k = VPT - 1;
        if constexpr (GRID) phase_turns_grid(u[k], v[k], w[k], su, sv, sw, Cs, th, tl);
        else phase_turns_df(u[k], v[k], w[k], su, sv, sw, th, tl);
    }

    // A leaf's sums start from zero: its parent clears them after reading.
    __device__ __forceinline__ void leaf_up(int k, float2 xi, float2 wv, bool root)
    {
        if (root) {                                   // J = 1: the leaf is a level-1 pixel
            kahan_add2(acc[k], comp[k], mul2(wv, xi));
            return;
        }
        low[k] = add2(low[k], xi);
        lowx[k] = fma2(wv, xi, lowx[k]);
    }

    // Two sibling leaves together: four independent phase chains per thread
    // (two visibilities x two leaves), one dispatch.
    __device__ __forceinline__ void leaf_pair(const RecWF& a, const RecWF& b)
    {
        const F2 su0{a.a, a.b}, sv0{a.c, a.d}, sw0{a.e, a.f};
        const F2 su1{b.a, b.b}, sv1{b.c, b.d}, sw1{b.e, b.f};
        const float2 w0 = bcast2(a.g), w1 = bcast2(b.g);
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            float2 h0, tl0, h1, tl1, e00, e01, e10, e11;
            phase2(p, su0, sv0, sw0, h0, tl0);
            phase2(p, su1, sv1, sw1, h1, tl1);
            sincos_mixed2<FAST>(h0, tl0, e00, e01);
            sincos_mixed2<FAST>(h1, tl1, e10, e11);
            low[2 * p] = add2(low[2 * p], add2(e00, e10));
            low[2 * p + 1] = add2(low[2 * p + 1], add2(e01, e11));
            lowx[2 * p] = fma2(w1, e10, fma2(w0, e00, lowx[2 * p]));
            lowx[2 * p + 1] = fma2(w1, e11, fma2(w0, e01, lowx[2 * p + 1]));
        }
        if constexpr (ODD) {
            constexpr int k = VPT - 1;
            float th0, tl0, s0, c0, th1, tl1, s1, c1;
            phase1(su0, sv0, sw0, th0, tl0);
            phase1(su1, sv1, sw1, th1, tl1);
            sincos_mixed<FAST>(th0, tl0, s0, c0);
            sincos_mixed<FAST>(th1, tl1, s1, c1);
            const float2 e0 = make_float2(c0, s0), e1 = make_float2(c1, s1);
            low[k] = add2(low[k], add2(e0, e1));
            lowx[k] = fma2(w1, e1, fma2(w0, e0, lowx[k]));
        }
    }

    // One step of the fast form's grouped sweep; returns the records it took.
    // A group (in one chunk by construction) is one step: its leaves in
    // pairs, then the parent; a leaf marked as the first of a pair takes its
    // sibling with it.
    __device__ __forceinline__ int at_grouped(const RecWF* cb, int r, int n)
    {
        const RecWF& a = cb[r];
        const uint32_t meta = a.meta;
        if (meta & kRwGroup) {
            const int k = static_cast<int>((meta >> kRwGroupShift) & 7u);
            if (k >= 1 && k <= 4 && r + k < n) {
                group(cb + r, k);
                return k + 1;
            }
        } else if ((meta & kRwPairFirst) && r + 1 < n) {
            leaf_pair(a, cb[r + 1]);
            return 2;
        }
        (*this)(a);
        return 1;
    }

    // One record of a fixed-stride sweep: the fast form's first leaf of a
    // pair takes its sibling, the second is skipped. The polynomial form
    // takes every record alone: its four chains need more registers than the
    // pairing saves (measured 2 % slower).
    __device__ __forceinline__ void at_single(const RecWF* cb, int r, int n)
    {
        const RecWF& a = cb[r];
        if constexpr (FAST) {
            if (a.meta & (kRwPairFirst | kRwPairSecond)) {
                if (a.meta & kRwPairFirst) leaf_pair(a, cb[r + 1 < n ? r + 1 : r]);
                return;
            }
        }
        (*this)(a);
    }

    // The polynomial form takes every record alone: a fixed stride.
    __device__ __forceinline__ auto at(const RecWF* cb, int r, int n)
    {
        if constexpr (GROUPS && FAST) return at_grouped(cb, r, n);
        else at_single(cb, r, n);
    }

    // A group of k sibling leaves g[0 .. k-1] and their parent g[k].
    __device__ __forceinline__ void group(const RecWF* g, int k)
    {
        if (k >= 2) leaf_pair(g[0], g[1]);
        else leaf(g[0], false);
        if (k == 4) leaf_pair(g[2], g[3]);
        else if (k == 3) leaf(g[2], false);
        low_levels(g[k], g[k].meta);
    }

    // Parent's xi sum: the first child writes it, the others add (a select,
    // not a branch: internal nodes are most records of deep, sparse trees).
    __device__ __forceinline__ void pass_up(int par, bool first, const float2 (&xi)[VPT])
    {
        float2 ps[VPT];
        load_row(par, ps);
#pragma unroll
        for (int k = 0; k < VPT; ++k) ps[k] = first ? xi[k] : add2(ps[k], xi[k]);
        store_row(par, ps);
    }

    // Nodes at levels J - 1 and J - 2, whose sums are in registers.
    __device__ __forceinline__ void low_levels(const RecWF& r, uint32_t meta)
    {
        const bool root = meta & kRwRoot, first = meta & kRwFirst;
        const float2 wv = bcast2(r.g);
        float2 xi[VPT];
        if (meta & kRwLowSum) {                        // level J - 1: registers only
#pragma unroll
            for (int k = 0; k < VPT; ++k) {
                xi[k] = low[k];
                const float2 x = fma2(wv, xi[k], lowx[k]);
                low[k] = make_float2(0.f, 0.f);
                lowx[k] = make_float2(0.f, 0.f);
                if (root) {
                    kahan_add2(acc[k], comp[k], x);
                } else {                               // the parent (level J - 2) takes both
                    midx[k] = add2(midx[k], x);
                    mid[k] = add2(mid[k], xi[k]);
                }
            }
            return;
        }
#pragma unroll
        for (int k = 0; k < VPT; ++k) {                // level J - 2
            xi[k] = mid[k];
            kahan_add2(acc[k], comp[k], fma2(wv, xi[k], midx[k]));
            mid[k] = make_float2(0.f, 0.f);
            midx[k] = make_float2(0.f, 0.f);
        }
        if (!root) pass_up(clamp_row(__float_as_uint(r.b), maxrow), first, xi);
    }

    // One leaf alone (root: a level-1 pixel, J = 1).
    __device__ __forceinline__ void leaf(const RecWF& r, bool root)
    {
        const float2 wv = bcast2(r.g);
        const F2 su{r.a, r.b}, sv{r.c, r.d}, sw{r.e, r.f};
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            float2 h, tl, e0, e1;
            phase2(p, su, sv, sw, h, tl);
            sincos_mixed2<FAST>(h, tl, e0, e1);
            leaf_up(2 * p, e0, wv, root);
            leaf_up(2 * p + 1, e1, wv, root);
        }
        if constexpr (ODD) {
            constexpr int k = VPT - 1;
            float th, tl, s, c;
            phase1(su, sv, sw, th, tl);
            sincos_mixed<FAST>(th, tl, s, c);
            leaf_up(k, make_float2(c, s), wv, root);
        }
    }

    __device__ void operator()(const RecWF& r)
    {
        const uint32_t meta = r.meta;
        const float2 wv = bcast2(r.g);
        if (meta & kRwLeaf) {
            leaf(r, (meta & kRwRoot) != 0);
            return;
        }
        if (meta & (kRwLowSum | kRwMidSum)) {
            low_levels(r, meta);
            return;
        }
        // any other internal node (level <= J - 3): rows pre-decoded by the
        // build (own: lev - 1, parent's: lev - 2), clamped to the stack. A
        // level-1 node (a root, always a first child) writes its xi back into
        // its own row 0, which the next level-1 node's first child overwrites.
        const int own = clamp_row(__float_as_uint(r.a), maxrow);
        const int par = clamp_row(__float_as_uint(r.b), maxrow);
        float2 xi[VPT];
        load_row(own, xi);
#pragma unroll
        for (int k = 0; k < VPT; ++k) kahan_add2(acc[k], comp[k], mul2(wv, xi[k]));
        pass_up(par, (meta & kRwFirst) != 0, xi);
    }
};

// The regrouped Eq. 17 in a mixed form runs in a grid pass and an exact
// pass (the tile helpers in wt_internal.cuh: tile_grid_constants,
// tile_deferred, mark_deferred).

// One tile's sweep of the regrouped Eq. 17 (GRID: on the head grid of the
// constants C, else with error-free sums; GROUPS as Eq17WF). Returns false
// (CTA-wide) if a staging copy did not arrive; res receives V of each
// visibility.
template <int NT, int VPT, bool FAST, bool GRID, bool GROUPS = true>
__device__ __forceinline__ bool sweep_regrouped_mixed(Stager<RecWF>& st, const F2 (&u)[VPT], const F2 (&v)[VPT],
                                      const F2 (&w)[VPT], const float (&C)[VPT], float2* stk, int J, int maxrow,
                                      float2 (&res)[VPT])
{
    Eq17WF<NT, VPT, FAST, GRID, GROUPS> b;
#pragma unroll
    for (int k = 0; k < VPT; ++k) { b.u[k] = u[k]; b.v[k] = v[k]; b.w[k] = w[k]; }
    if constexpr (GRID) {
#pragma unroll
        for (int p = 0; p < VPT / 2; ++p) b.Cg[p] = make_float2(C[2 * p], C[2 * p + 1]);
        b.Cs = C[VPT - 1];
    }
    b.start();
    b.stk = stk;
    b.J = J;
    b.maxrow = maxrow;
    const bool good = st.sweep_at(b);
#pragma unroll
    for (int k = 0; k < VPT; ++k) res[k] = b.result(k);
    return good;
}


}  // namespace
}  // namespace wt
