// wavelet.cu -- wt_predict_vis: per-visibility plane-wave coefficients on
// the coefficient tree and the multiresolution sum (Sec. 3.3, Eqs. 14, 16,
// 17; per-visibility steps of Sec. 3.6.1).
//
// Mapping to the GPU. A thread owns VPT visibilities; a CTA owns a tile of
// NT * VPT visibilities and walks the whole tree for them. The tree is the
// same for every visibility, so the walk is uniform across the CTA: the node
// records (post-order, pre-decoded once per major cycle by the build) are
// streamed through shared memory by bulk copies and read as broadcasts; the
// record's fields are loaded once per thread and used for all VPT
// visibilities. Post-order visits every child before its parent, so each
// node's plane-wave coefficient eta_j,k is ready exactly when its parent
// needs it. A thread keeps, for levels j = 2..J, the four child slots of the
// open parent in shared-memory columns of its own (row-major
// [row][vis][thread]: conflict-free). Nothing per visibility is written to
// global memory except V.
//
// Per internal node the kernel forms eta (Eq. 9 form) and the three sigma
// (Eq. 10 form) explicitly and adds gamma^m sigma^m. A node with a single
// child needs no butterfly: its sigma^m are +-q eta_c, the sign folded into
// gamma^m by the build. The mixed forms carry xi = 4^(J-j) eta instead of
// eta, with the scale factors folded into gamma by the build, and do their
// float32 arithmetic on packed pairs (wavelet_bodies.cuh).
//
// Forms:
//   WT_FP64   float64 throughout; sin/cos by table-driven reduction
//             (sincos_turns_f64, wt_internal.cuh).
//   WT_MIXED  phase in double-float turns (float64-accurate), sin/cos of the
//             reduced phase in float32 (Taylor series, wt_internal.cuh),
//             recursion in float32, Kahan-compensated float32 V.
//   WT_MIXED_FAST  as WT_MIXED with sin/cos from the special-function unit.
//   WT_FP64_DF     float64-class: phase, sin/cos (table method) and every
//             sum in double-float arithmetic on the float32 pipe (df64.cuh);
//             the regrouped Eq. 17 and Eq. 16.
#include <type_traits>

#include "staging.cuh"
#include "wavelet_bodies.cuh"
#include "wt_internal.cuh"

namespace wt {
namespace {

// ---------------------------------------------------------------- kernels
// SUM: 0 = Eq. 17 with explicit sigma (RecD / RecF), 1 = Eq. 16 over the
// leaf records, 2 = regrouped Eq. 17 (RecWD / RecWF).
template <int NT, int VPT, int SUM, class Rec>
__global__ void __launch_bounds__(NT) k_wavelet_fp64(const Rec* __restrict__ recs, const TreeHeader* __restrict__ hdr,
                                                     const double* __restrict__ uvw, int64_t n_vis,
                                                     double2* __restrict__ vis, double sgn, int rows, int J,
                                                     int* status)
{
    extern __shared__ __align__(16) unsigned char smem[];
    Stager<Rec> st;
    const int64_t count = (SUM == 1) ? hdr->n_leaves : hdr->n_nodes;
    stager_setup(st, smem, recs, count, kChunkD);
    double2* stk = reinterpret_cast<double2*>(smem + stager_bytes<Rec>(kChunkD)) + threadIdx.x;
    const int64_t per_tile = static_cast<int64_t>(NT) * VPT;
    const int64_t ntiles = (n_vis + per_tile - 1) / per_tile;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t n0 = tile * per_tile + threadIdx.x;
        double U[VPT], V[VPT], W[VPT];
#pragma unroll
        for (int k = 0; k < VPT; ++k) {
            const int64_t n = n0 + static_cast<int64_t>(k) * NT;
            const bool ok = n < n_vis;
            U[k] = ok ? sgn * uvw[3 * n] : 0.0;       // sign folded in: exp(-i 2 pi t)
            V[k] = ok ? sgn * uvw[3 * n + 1] : 0.0;   // = exp(i 2 pi (-t)), exact
            W[k] = ok ? sgn * uvw[3 * n + 2] : 0.0;
        }
        bool good;
        double vr[VPT], vi[VPT];
        if constexpr (SUM == 1) {
            Eq16D<VPT> b;
#pragma unroll
            for (int k = 0; k < VPT; ++k) {
                b.u[k] = U[k]; b.v[k] = V[k]; b.w[k] = W[k]; b.vr[k] = 0.0; b.vi[k] = 0.0;
            }
            b.sgn = sgn;
            good = st.sweep(b);
#pragma unroll
            for (int k = 0; k < VPT; ++k) { vr[k] = b.vr[k]; vi[k] = b.vi[k]; }
        } else if constexpr (SUM == 0) {
            Eq17D<NT, VPT> b;
#pragma unroll
            for (int k = 0; k < VPT; ++k) {
                b.u[k] = U[k]; b.v[k] = V[k]; b.w[k] = W[k]; b.vr[k] = 0.0; b.vi[k] = 0.0;
            }
            b.sgn = sgn;
            b.stk = stk;
            b.maxrow = rows - 1;
            good = st.sweep(b);
#pragma unroll
            for (int k = 0; k < VPT; ++k) { vr[k] = b.vr[k]; vi[k] = b.vi[k]; }
        } else {
            Eq17WD<NT, VPT> b;
#pragma unroll
            for (int k = 0; k < VPT; ++k) {
                b.u[k] = U[k]; b.v[k] = V[k]; b.w[k] = W[k]; b.vr[k] = 0.0; b.vi[k] = 0.0;
                b.sr[k] = 0.0; b.si[k] = 0.0; b.xr[k] = 0.0; b.xi[k] = 0.0;
            }
            b.stk = stk;
            b.J = J;
            b.maxrow = rows - 1;
            good = st.sweep(b);
#pragma unroll
            for (int k = 0; k < VPT; ++k) { vr[k] = b.vr[k]; vi[k] = b.vi[k]; }
        }
        if (!good) {
            if (threadIdx.x == 0) record_status(status, WT_ERR_TIMEOUT);
            return;
        }
#pragma unroll
        for (int k = 0; k < VPT; ++k) {
            const int64_t n = n0 + static_cast<int64_t>(k) * NT;
            if (n < n_vis) vis[n] = make_double2(vr[k], vi[k]);
        }
    }
}

// The float64-class double-float form: regrouped Eq. 17 (Eq17DF) on the
// float32 pipe. Shared memory: the record staging, the 257-entry
// double-float sin/cos table, then the stack.
template <int NT, int VPT, int SUM>
__global__ void __launch_bounds__(NT) k_wavelet_df(const RecWDF* __restrict__ recs,
                                                   const TreeHeader* __restrict__ hdr,
                                                   const double* __restrict__ uvw, int64_t n_vis,
                                                   double2* __restrict__ vis, double sgn, int rows, int J,
                                                   int* status)
{
    extern __shared__ __align__(16) unsigned char smem[];
    Stager<RecWDF> st;
    stager_setup(st, smem, recs, hdr->n_nodes, kChunkDF);
    float4* tab = reinterpret_cast<float4*>(smem + stager_bytes<RecWDF>(kChunkDF));
    load_sincos_table_df(tab);
    float4* stk = tab + kDfTableEntries + threadIdx.x;
    __syncthreads();
    const int64_t per_tile = static_cast<int64_t>(NT) * VPT;
    const int64_t ntiles = (n_vis + per_tile - 1) / per_tile;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t n0 = tile * per_tile + threadIdx.x;
        using Body = typename std::conditional<SUM == 1, Eq16DF<VPT>, Eq17DF<NT, VPT>>::type;
        Body b;
#pragma unroll
        for (int k = 0; k < VPT; ++k) {
            const int64_t n = n0 + static_cast<int64_t>(k) * NT;
            const bool ok = n < n_vis;
            b.u[k] = split_f64(ok ? sgn * uvw[3 * n] : 0.0);   // sign folded in (exact)
            b.v[k] = split_f64(ok ? sgn * uvw[3 * n + 1] : 0.0);
            b.w[k] = split_f64(ok ? sgn * uvw[3 * n + 2] : 0.0);
            b.vr[k] = DF{0.f, 0.f};
            b.vi[k] = DF{0.f, 0.f};
        }
        b.tab = tab;
        if constexpr (SUM != 1) {
#pragma unroll
            for (int k = 0; k < VPT; ++k) b.lr[k] = b.li[k] = DF{0.f, 0.f};
            b.stk = stk;
            b.J = J;
            b.maxrow = rows - 1;
        }
        if (!st.sweep(b)) {
            if (threadIdx.x == 0) record_status(status, WT_ERR_TIMEOUT);
            return;
        }
#pragma unroll
        for (int k = 0; k < VPT; ++k) {
            const int64_t n = n0 + static_cast<int64_t>(k) * NT;
            if (n < n_vis) vis[n] = make_double2(df_to_double(b.vr[k]), df_to_double(b.vi[k]));
        }
    }
}

// SUM = 2 (the regrouped Eq. 17) runs as two passes (wavelet_bodies.cuh,
// sweep_regrouped_mixed): GRIDPASS = true evaluates the tiles whose phases
// fit the head grid and marks the others, GRIDPASS = false evaluates only the
// marked tiles, with error-free sums. GRIDPASS is unused for SUM = 0, 1.
// Register budgets of the regrouped form: 64 per thread at one or two
// visibilities per thread (1024 threads per SM; left free, the compiler gives
// the grid pass 80 and fits 6 CTAs of 128 threads per SM instead of 8), 128
// at four (512 threads per SM, the same 2048 visibilities in flight, with
// the per-record work -- loading, decoding and broadcasting a record --
// shared by twice as many visibilities).
template <int NT, int VPT, int SUM>
constexpr int mixed_min_blocks()
{
    return SUM != 2 ? 1 : VPT <= 2 ? 1024 / NT : VPT == 4 ? 512 / NT : 1;
}

template <int NT, int VPT, int SUM, class Rec, bool FAST, bool GRIDPASS = false>
__global__ void __launch_bounds__(NT, (mixed_min_blocks<NT, VPT, SUM>())) k_wavelet_mixed(const Rec* __restrict__ recs, const TreeHeader* __restrict__ hdr,
                                                      const double* __restrict__ uvw, int64_t n_vis,
                                                      float2* __restrict__ vis, float sgn, int rows, int J,
                                                      int* status)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int kChunk = (SUM == 2) ? kChunkW : kChunkF;
    Stager<Rec> st;
    const int64_t count = (SUM == 1) ? hdr->n_leaves : hdr->n_nodes;
    stager_setup(st, smem, recs, count, kChunk);
    float2* stk = reinterpret_cast<float2*>(smem + stager_bytes<Rec>(kChunk)) + threadIdx.x;
    const int64_t per_tile = static_cast<int64_t>(NT) * VPT;
    const int64_t ntiles = (n_vis + per_tile - 1) / per_tile;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        if constexpr (!GRIDPASS) {
            if (!tile_deferred(vis + tile * per_tile)) continue;   // done by the grid pass
        }
        const int64_t n0 = tile * per_tile + threadIdx.x;
        F2 U[VPT], V[VPT], W[VPT];
#pragma unroll
        for (int k = 0; k < VPT; ++k) {
            const int64_t n = n0 + static_cast<int64_t>(k) * NT;
            const bool ok = n < n_vis;
            const double sg = static_cast<double>(sgn);   // sign folded into B (exact)
            U[k] = split_f64(ok ? sg * uvw[3 * n] : 0.0);
            V[k] = split_f64(ok ? sg * uvw[3 * n + 1] : 0.0);
            W[k] = split_f64(ok ? sg * uvw[3 * n + 2] : 0.0);
        }
        bool good;
        bool defer = false;   // a tile the grid pass leaves marked for the exact pass
        float vr[VPT], vi[VPT];
        if constexpr (SUM == 1) {
            // grid pass / exact pass as for the regrouped sum below
            float C[VPT];
            if constexpr (GRIDPASS) {
                defer = !tile_grid_constants(U, V, W, hdr->smax, C);   // a CTA-wide decision
            } else {
#pragma unroll
                for (int k = 0; k < VPT; ++k) C[k] = 0.f;
            }
            Eq16F2<VPT, FAST, GRIDPASS> b;
            b.start(U, V, W, C);
            good = st.sweep_at(b);
#pragma unroll
            for (int k = 0; k < VPT; ++k) {
                const float2 r = b.result(k);
                vr[k] = r.x;
                vi[k] = r.y;
            }
        } else if constexpr (SUM == 0) {
            Eq17F<NT, VPT, FAST, GRIDPASS> b;
#pragma unroll
            for (int k = 0; k < VPT; ++k) { b.u[k] = U[k]; b.v[k] = V[k]; b.w[k] = W[k]; }
            if constexpr (GRIDPASS) {
                float C[VPT];
                defer = !tile_grid_constants(U, V, W, hdr->smax, C);   // a CTA-wide decision
#pragma unroll
                for (int p = 0; p < VPT / 2; ++p) b.Cg[p] = make_float2(C[2 * p], C[2 * p + 1]);
                b.Cs = C[VPT - 1];
            }
            b.start();
            b.stk = stk;
            b.maxrow = rows - 1;
            good = st.sweep(b);
#pragma unroll
            for (int k = 0; k < VPT; ++k) {
                const float2 r = b.result(k);
                vr[k] = r.x;
                vi[k] = r.y;
            }
        } else {
            float2 res[VPT];
            float C[VPT];
            float2* rstk = stk - threadIdx.x + threadIdx.x * VPT;   // [row][thread][vis] layout
            if constexpr (GRIDPASS) {
                // A tile that does not fit is swept too and its results are
                // discarded (marked for the exact pass instead): skipping the
                // sweep conditionally costs the kernel register spills, and
                // such tiles come only with phases of 2^14 turns or more.
                defer = !tile_grid_constants(U, V, W, hdr->smax, C);   // a CTA-wide decision
                good = sweep_regrouped_mixed<NT, VPT, FAST, true>(st, U, V, W, C, rstk, J, rows - 1, res);
            } else {
                good = sweep_regrouped_mixed<NT, VPT, FAST, false>(st, U, V, W, C, rstk, J, rows - 1, res);
            }
#pragma unroll
            for (int k = 0; k < VPT; ++k) {
                vr[k] = res[k].x;
                vi[k] = res[k].y;
            }
        }
        if (!good) {
            if (threadIdx.x == 0) record_status(status, WT_ERR_TIMEOUT);
            return;
        }
        if (defer) {
            mark_deferred(vis + tile * per_tile);
            continue;
        }
#pragma unroll
        for (int k = 0; k < VPT; ++k) {
            const int64_t n = n0 + static_cast<int64_t>(k) * NT;
            if (n < n_vis) vis[n] = make_float2(vr[k], vi[k]);
        }
    }
}

// ---------------------------------------------------------------- launch
struct Variant {
    int nt, vpt;
};

template <class K>
int prepare(K kernel, int nt, size_t smem, int64_t per_tile, int64_t n_vis, dim3& grid)
{
    WT_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
    int per_sm = 0;
    WT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, nt, smem));
    if (per_sm < 1) return set_error(WT_ERR_UNSUPPORTED, "wavelet kernel does not fit on an SM (smem %zu)", smem);
    // One CTA per tile, not a persistent grid: the hardware hands each SM a
    // new CTA as one of its own finishes, which balances the SMs to within
    // one tile. A grid of the resident CTAs striding over the tiles ran the
    // medium batch 11 % slower (SMs that finish their share early sit
    // idle); the two agree when the tiles fit in one wave. The kernels
    // still stride when the grid is capped.
    const int64_t ntiles = (n_vis + per_tile - 1) / per_tile;
    const int64_t g = ntiles < 0x7fffffff ? ntiles : 0x7fffffff;
    grid = dim3(static_cast<unsigned>(g));
    return WT_OK;
}

// Shared-memory stack rows a form needs for a tree of depth J.
int stack_rows(int mode, int which, int J)
{
    if (which == WT_SUM_EQ16) return 0;
    if (mode == WT_FP64_DF) return J > 3 ? J - 2 : 1;   // regrouped (Eq. 16 returned 0 above)
    if (which == WT_SUM_EQ17_REGROUPED) {
        if (mode == WT_FP64) return J > 3 ? 2 * (J - 2) : 2;
        return J > 4 ? J - 3 : 1;
    }
    return J > 1 ? 4 * (J - 1) : 4;
}

// Staging bytes of a form (two buffers of records plus the mbarriers).
size_t stage_bytes(int mode, int which)
{
    if (mode == WT_FP64) return stager_bytes<RecD>(kChunkD);
    if (mode == WT_FP64_DF) return stager_bytes<RecWDF>(kChunkDF) + kDfTableEntries * sizeof(float4);
    return (which == WT_SUM_EQ17_REGROUPED) ? stager_bytes<RecWF>(kChunkW) : stager_bytes<RecF>(kChunkF);
}

template <int NT, int VPT>
int run_fp64(const WaveletJob& jb, cudaStream_t s)
{
    const int rows = stack_rows(WT_FP64, jb.which, jb.J);
    const size_t stack = static_cast<size_t>(rows) * VPT * NT * sizeof(double2);
    const size_t smem = stage_bytes(WT_FP64, jb.which) + stack;
    dim3 grid;
    int rc;
    double2* out = static_cast<double2*>(jb.vis);
    const double sg = jb.sign;
    if (jb.which == WT_SUM_EQ16) {
        auto k = k_wavelet_fp64<NT, VPT, 1, RecD>;
        if ((rc = prepare(k, NT, smem, int64_t(NT) * VPT, jb.n_vis, grid))) return rc;
        k<<<grid, NT, smem, s>>>(jb.recd_leaf, jb.hdr, jb.uvw, jb.n_vis, out, sg, rows, jb.J, jb.status);
    } else if (jb.which == WT_SUM_EQ17) {
        auto k = k_wavelet_fp64<NT, VPT, 0, RecD>;
        if ((rc = prepare(k, NT, smem, int64_t(NT) * VPT, jb.n_vis, grid))) return rc;
        k<<<grid, NT, smem, s>>>(jb.recd, jb.hdr, jb.uvw, jb.n_vis, out, sg, rows, jb.J, jb.status);
    } else {
        auto k = k_wavelet_fp64<NT, VPT, 2, RecWD>;
        if ((rc = prepare(k, NT, smem, int64_t(NT) * VPT, jb.n_vis, grid))) return rc;
        k<<<grid, NT, smem, s>>>(jb.recwd, jb.hdr, jb.uvw, jb.n_vis, out, sg, rows, jb.J, jb.status);
    }
    WT_CUDA_TRY(cudaGetLastError());
    return WT_OK;
}

template <int NT, int VPT>
int run_df(const WaveletJob& jb, cudaStream_t s)
{
    const int rows = stack_rows(WT_FP64_DF, jb.which, jb.J);
    const size_t smem = stage_bytes(WT_FP64_DF, jb.which) + static_cast<size_t>(rows) * VPT * NT * sizeof(float4);
    dim3 grid;
    int rc;
    auto k = (jb.which == WT_SUM_EQ16) ? k_wavelet_df<NT, VPT, 1> : k_wavelet_df<NT, VPT, 2>;
    if ((rc = prepare(k, NT, smem, int64_t(NT) * VPT, jb.n_vis, grid))) return rc;
    k<<<grid, NT, smem, s>>>(jb.recwdf, jb.hdr, jb.uvw, jb.n_vis, static_cast<double2*>(jb.vis),
                             static_cast<double>(jb.sign), rows, jb.J, jb.status);
    WT_CUDA_TRY(cudaGetLastError());
    return WT_OK;
}

template <int NT, int VPT, bool FAST>
int run_mixed_form(const WaveletJob& jb, cudaStream_t s)
{
    const int rows = stack_rows(jb.mode, jb.which, jb.J);
    const size_t stack = static_cast<size_t>(rows) * VPT * NT * sizeof(float2);
    const size_t smem = stage_bytes(jb.mode, jb.which) + stack;
    dim3 grid;
    int rc;
    float2* out = static_cast<float2*>(jb.vis);
    const float sg = static_cast<float>(jb.sign);
    if (jb.which == WT_SUM_EQ16) {
        // the grid pass, then the exact pass over the tiles it left marked
        auto kg = k_wavelet_mixed<NT, VPT, 1, RecF, FAST, true>;
        auto ke = k_wavelet_mixed<NT, VPT, 1, RecF, FAST, false>;
        if ((rc = prepare(kg, NT, smem, int64_t(NT) * VPT, jb.n_vis, grid))) return rc;
        dim3 grid_e;
        if ((rc = prepare(ke, NT, smem, int64_t(NT) * VPT, jb.n_vis, grid_e))) return rc;
        kg<<<grid, NT, smem, s>>>(jb.recf_leaf, jb.hdr, jb.uvw, jb.n_vis, out, sg, rows, jb.J, jb.status);
        WT_CUDA_TRY(cudaGetLastError());
        ke<<<grid_e, NT, smem, s>>>(jb.recf_leaf, jb.hdr, jb.uvw, jb.n_vis, out, sg, rows, jb.J, jb.status);
    } else if (jb.which == WT_SUM_EQ17) {
        // the grid pass, then the exact pass over the tiles it left marked
        auto kg = k_wavelet_mixed<NT, VPT, 0, RecF, FAST, true>;
        auto ke = k_wavelet_mixed<NT, VPT, 0, RecF, FAST, false>;
        if ((rc = prepare(kg, NT, smem, int64_t(NT) * VPT, jb.n_vis, grid))) return rc;
        dim3 grid_e;
        if ((rc = prepare(ke, NT, smem, int64_t(NT) * VPT, jb.n_vis, grid_e))) return rc;
        kg<<<grid, NT, smem, s>>>(jb.recf, jb.hdr, jb.uvw, jb.n_vis, out, sg, rows, jb.J, jb.status);
        WT_CUDA_TRY(cudaGetLastError());
        ke<<<grid_e, NT, smem, s>>>(jb.recf, jb.hdr, jb.uvw, jb.n_vis, out, sg, rows, jb.J, jb.status);
    } else {
        // the grid pass, then the exact pass over the tiles it left marked
        auto kg = k_wavelet_mixed<NT, VPT, 2, RecWF, FAST, true>;
        auto ke = k_wavelet_mixed<NT, VPT, 2, RecWF, FAST, false>;
        if ((rc = prepare(kg, NT, smem, int64_t(NT) * VPT, jb.n_vis, grid))) return rc;
        dim3 grid_e;
        if ((rc = prepare(ke, NT, smem, int64_t(NT) * VPT, jb.n_vis, grid_e))) return rc;
        kg<<<grid, NT, smem, s>>>(jb.recwf, jb.hdr, jb.uvw, jb.n_vis, out, sg, rows, jb.J, jb.status);
        WT_CUDA_TRY(cudaGetLastError());
        ke<<<grid_e, NT, smem, s>>>(jb.recwf, jb.hdr, jb.uvw, jb.n_vis, out, sg, rows, jb.J, jb.status);
    }
    WT_CUDA_TRY(cudaGetLastError());
    return WT_OK;
}

template <int NT, int VPT>
int run_mixed(const WaveletJob& jb, cudaStream_t s)
{
    return (jb.mode == WT_MIXED_FAST) ? run_mixed_form<NT, VPT, true>(jb, s) : run_mixed_form<NT, VPT, false>(jb, s);
}

}  // namespace

// Launch-shape variants (threads per CTA, visibilities per thread). Which
// one runs is chosen per (form, sum, J, tree size) by the autotuner, or by
// stack_fits() when no tuning is available.
const int kNumWaveletVariants = 8;
static const Variant kVariants[kNumWaveletVariants] = {{256, 1}, {128, 1}, {128, 2}, {64, 2},
                                                       {64, 4},  {32, 4},  {32, 2},  {256, 2}};

int wavelet_variant_shape(int v, int* nt, int* vpt)
{
    if (v < 0 || v >= kNumWaveletVariants) return WT_ERR_ARG;
    *nt = kVariants[v].nt;
    *vpt = kVariants[v].vpt;
    return WT_OK;
}

// Shared memory a variant needs for a tree of depth J (stack only; the
// staging buffers add a fixed amount).
size_t wavelet_variant_smem(int v, int mode, int which, int J)
{
    if (v < 0 || v >= kNumWaveletVariants) return 0;
    const size_t cplx = (mode == WT_FP64 || mode == WT_FP64_DF) ? sizeof(double2) : sizeof(float2);
    const size_t stage = stage_bytes(mode, which);
    const size_t stack = static_cast<size_t>(stack_rows(mode, which, J)) * kVariants[v].nt * kVariants[v].vpt * cplx;
    return stage + stack;
}

bool wavelet_variant_fits(int v, int mode, int which, int J)
{
    if (v < 0 || v >= kNumWaveletVariants) return false;
    return wavelet_variant_smem(v, mode, which, J) <= 220 * 1024;
}

int launch_wavelet(const WaveletJob& jb, int v, cudaStream_t s)
{
    if (!wavelet_variant_fits(v, jb.mode, jb.which, jb.J))
        return set_error(WT_ERR_UNSUPPORTED, "wavelet variant %d does not fit for J = %d", v, jb.J);
    if (jb.mode == WT_FP64_DF) {
        switch (v) {
            case 0: return run_df<256, 1>(jb, s);
            case 1: return run_df<128, 1>(jb, s);
            case 2: return run_df<128, 2>(jb, s);
            case 3: return run_df<64, 2>(jb, s);
            case 4: return run_df<64, 4>(jb, s);
            case 5: return run_df<32, 4>(jb, s);
            case 6: return run_df<32, 2>(jb, s);
            default: return run_df<256, 2>(jb, s);
        }
    }
    if (jb.mode == WT_FP64) {
        switch (v) {
            case 0: return run_fp64<256, 1>(jb, s);
            case 1: return run_fp64<128, 1>(jb, s);
            case 2: return run_fp64<128, 2>(jb, s);
            case 3: return run_fp64<64, 2>(jb, s);
            case 4: return run_fp64<64, 4>(jb, s);
            case 5: return run_fp64<32, 4>(jb, s);
            case 6: return run_fp64<32, 2>(jb, s);
            default: return run_fp64<256, 2>(jb, s);
        }
    }
    switch (v) {
        case 0: return run_mixed<256, 1>(jb, s);
        case 1: return run_mixed<128, 1>(jb, s);
        case 2: return run_mixed<128, 2>(jb, s);
        case 3: return run_mixed<64, 2>(jb, s);
        case 4: return run_mixed<64, 4>(jb, s);
        case 5: return run_mixed<32, 4>(jb, s);
        case 6: return run_mixed<32, 2>(jb, s);
        default: return run_mixed<256, 2>(jb, s);
    }
}

// Default when nothing is tuned: the first variant that fits in a measured
// preference order.
int default_wavelet_variant(int mode, int which, int J)
{
    // measured on the medium and large workloads (J = 12): the explicit
    // mixed sum runs best at 256 x 1 (its stack limits the CTAs per SM), the
    // regrouped one, whose stack is small, at 64 x 4 (the per-record work
    // shared by four visibilities), then 128 x 2; Eq. 16 (no stack) on packed
    // pairs of visibilities at 128 x 2
    static const int order_mixed[kNumWaveletVariants] = {0, 2, 1, 3, 4, 5, 6, 7};
    static const int order_mixed16[kNumWaveletVariants] = {2, 7, 3, 4, 0, 1, 5, 6};
    static const int order_mixed_rg[kNumWaveletVariants] = {4, 2, 7, 6, 3, 5, 0, 1};
    static const int order_fp64[kNumWaveletVariants] = {1, 0, 2, 3, 4, 5, 6, 7};
    const int* order = (mode == WT_FP64 || mode == WT_FP64_DF) ? order_fp64
                       : (which == WT_SUM_EQ17_REGROUPED) ? order_mixed_rg
                       : (which == WT_SUM_EQ16)           ? order_mixed16
                                                          : order_mixed;
    for (int i = 0; i < kNumWaveletVariants; ++i)
        if (wavelet_variant_fits(order[i], mode, which, J)) return order[i];
    return kNumWaveletVariants - 1;
}

int predict_wavelet(wt_tree t, const double* uvw, int64_t n_vis, void* vis, int mode, int sign, int which,
                    cudaStream_t s)
{
    if (n_vis == 0) return WT_OK;
    if (mode == WT_MIXED_TC) {   // Eq. 16 as a direct sum over the leaves, the phase on the tensor cores
        if (which != WT_SUM_EQ16)
            return set_error(WT_ERR_UNSUPPORTED, "wt_predict_vis: WT_MIXED_TC is Eq. 16 only (WT_SUM_EQ16)");
        int* status = device_status_word();
        if (!status) return set_error(WT_ERR_CUDA, "wt_predict_vis: no device status word");
        const int64_t hint = tree_sync_header(t) == WT_OK ? t->host_hdr->n_leaves : -1;
        return eq16_tc_launch(t->d.leaff, t->d.hdr, t->cap_leaves, hint, uvw, n_vis, static_cast<float2*>(vis), sign,
                              status, s, "wt_predict_vis");
    }
    WaveletJob jb;
    jb.recd = t->d.recd;
    jb.recf = t->d.recf;
    jb.recd_leaf = t->d.leafd;
    jb.recf_leaf = t->d.leaff;
    jb.recwd = t->d.recwd;
    jb.recwf = t->d.recwf;
    jb.recwdf = t->d.recwdf;
    jb.hdr = t->d.hdr;
    jb.uvw = uvw;
    jb.n_vis = n_vis;
    jb.vis = vis;
    jb.mode = mode;
    jb.sign = sign;
    jb.which = which;
    jb.J = t->J;
    jb.status = device_status_word();
    if (!jb.status) return set_error(WT_ERR_CUDA, "wt_predict_vis: no device status word");
    const int v = choose_wavelet_variant(t, jb, s);
    return launch_wavelet(jb, v, s);
}

}  // namespace wt
