// batched.cu -- wt_predict_vis_batched: many frequency channels (or major
// cycles), each with its own coefficient tree, in one launch.
//
// Work items are (channel, tile of NT * VPT visibilities). Channels are
// ordered by decreasing tree size (largest work first), items numbered
// channel-major in that order, one CTA per item: the hardware hands each SM
// the next CTA as one of its own finishes, so channels of very uneven size
// keep every SM busy to the end (beyond 2^31 - 1 items, persistent CTAs take
// the next item from a device-wide atomic counter instead). Items depend on nothing but
// their own inputs: no CTA ever waits for another. A CTA re-targets its
// shared-memory record staging only when the channel changes. Baselines are
// shared in metres and scaled per channel, u_lambda = u_m f_c / c. The
// float64 form evaluates Eq. 17 explicitly (Eq17D), the mixed forms in the
// regrouped order (Eq17WF: one stack pair per level, so small CTAs fit many
// to an SM), the double-float form in the regrouped order too (Eq17DF).
//
// The memset of the counter plus the kernel are captured once into a CUDA
// graph per plan (tree set, frequencies, form, sign, buffers, launch shape)
// and replayed on the caller's stream; the launch shape is picked by timing
// the fitting shapes on the plan's first use (WT_AUTOTUNE=0: default shape).
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <map>
#include <memory>
#include <mutex>
#include <type_traits>
#include <vector>

#include "staging.cuh"
#include "wavelet_bodies.cuh"
#include "wt_internal.cuh"

namespace wt {
namespace {

constexpr double kLightSpeed = 299792458.0;   // m/s

struct BatchChan {
    const RecD* recd;
    const RecWF* recwf;
    const RecWDF* recwdf;
    const TreeHeader* hdr;
    double scale;          // f_c / c: metres -> wavelengths
    int64_t out_offset;    // channel * n_vis
    int64_t tile_base;     // first work item of this channel
    int32_t J;
    int32_t pad;
};
static_assert(sizeof(BatchChan) == 64, "BatchChan layout");

// The form a batched kernel evaluates: float64 explicit Eq. 17, regrouped
// Eq. 17 in the mixed forms, or regrouped Eq. 17 in double-float.
constexpr int kKindF64 = 0, kKindMixed = 1, kKindDF = 2;

__device__ __forceinline__ int find_channel(const BatchChan* __restrict__ ch, int n_ch, int64_t item)
{
    int a = 0, b = n_ch - 1;   // last channel whose tile_base <= item
    while (a < b) {
        const int mid = (a + b + 1) >> 1;
        if (__ldg(&ch[mid].tile_base) <= item) a = mid;
        else b = mid - 1;
    }
    return a;
}

// The mixed kind runs the regrouped Eq. 17 in two passes as the single-tree
// predictor does (wavelet_bodies.cuh, sweep_regrouped_mixed): GRIDPASS =
// true evaluates the items whose phases fit the head grid and marks the
// others, GRIDPASS = false evaluates only the marked items. GRIDPASS is
// unused for the other kinds.
template <int NT, int VPT, int KIND, bool FAST = false, bool GRIDPASS = false>
__global__ void __launch_bounds__(NT) k_batched(const BatchChan* __restrict__ chans, int n_ch, int64_t total_items,
                                                const double* __restrict__ uvw_m, int64_t n_vis, void* vis, double sgn,
                                                int rows_max, unsigned long long* queue, int* status)
{
    using Rec = typename std::conditional<KIND == kKindMixed, RecWF,
                                          typename std::conditional<KIND == kKindDF, RecWDF, RecD>::type>::type;
    constexpr int kChunk = KIND == kKindMixed ? kChunkW : (KIND == kKindDF ? kChunkDF : kChunkD);
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_item;
    Stager<Rec> st;
    stager_setup(st, smem, static_cast<const Rec*>(nullptr), 0, kChunk);
    unsigned char* stk_base = smem + stager_bytes<Rec>(kChunk);
    float4* tab = reinterpret_cast<float4*>(stk_base);   // double-float form: sin/cos table, then the stack
    if constexpr (KIND == kKindDF) {
        load_sincos_table_df(tab);
        stk_base += kDfTableEntries * sizeof(float4);
        __syncthreads();
    }
    int cur = -1;
    int maxrow = 0;
    constexpr int64_t per_tile = static_cast<int64_t>(NT) * VPT;
    for (int64_t step = 0;; ++step) {
        int64_t item;
        if (queue) {   // a persistent CTA takes the next item from the queue
            if (threadIdx.x == 0) s_item = static_cast<long long>(atomicAdd(queue, 1ull));
            __syncthreads();
            item = s_item;
            __syncthreads();
        } else {       // one CTA per item
            item = step == 0 ? static_cast<int64_t>(blockIdx.x) : total_items;
        }
        if (item >= total_items) break;
        const int c = find_channel(chans, n_ch, item);
        const BatchChan ch = chans[c];
        if (c != cur) {
            const Rec* recs;
            if constexpr (KIND == kKindMixed) recs = ch.recwf;
            else if constexpr (KIND == kKindDF) recs = ch.recwdf;
            else recs = ch.recd;
            st.retarget(recs, ch.hdr->n_nodes);
            cur = c;
            if constexpr (KIND == kKindMixed) maxrow = min(ch.J > 4 ? ch.J - 3 : 1, rows_max) - 1;
            else if constexpr (KIND == kKindDF) maxrow = min(ch.J > 3 ? ch.J - 2 : 1, rows_max) - 1;
            else maxrow = min(4 * (ch.J > 1 ? ch.J - 1 : 1), rows_max) - 1;
        }
        const int64_t n0 = (item - ch.tile_base) * per_tile + threadIdx.x;
        bool good;
        if constexpr (KIND == kKindDF) {
            Eq17DF<NT, VPT> b;
#pragma unroll
            for (int k = 0; k < VPT; ++k) {
                const int64_t n = n0 + static_cast<int64_t>(k) * NT;
                const bool ok = n < n_vis;
                const double s = sgn * ch.scale;   // sign folded into B (exact negation)
                b.u[k] = split_f64(ok ? uvw_m[3 * n] * s : 0.0);
                b.v[k] = split_f64(ok ? uvw_m[3 * n + 1] * s : 0.0);
                b.w[k] = split_f64(ok ? uvw_m[3 * n + 2] * s : 0.0);
                b.vr[k] = b.vi[k] = b.lr[k] = b.li[k] = DF{0.f, 0.f};
            }
            b.stk = reinterpret_cast<float4*>(stk_base) + threadIdx.x;
            b.tab = tab;
            b.J = ch.J;
            b.maxrow = maxrow;
            good = st.sweep(b);
            double2* out = static_cast<double2*>(vis) + ch.out_offset;
#pragma unroll
            for (int k = 0; k < VPT; ++k) {
                const int64_t n = n0 + static_cast<int64_t>(k) * NT;
                if (good && n < n_vis) out[n] = make_double2(df_to_double(b.vr[k]), df_to_double(b.vi[k]));
            }
        } else if constexpr (KIND == kKindMixed) {
            float2* out = static_cast<float2*>(vis) + ch.out_offset;
            float2* first_vis = out + (item - ch.tile_base) * per_tile;
            if constexpr (!GRIDPASS) {
                if (!tile_deferred(first_vis)) continue;   // done by the grid pass
            }
            F2 U[VPT], V[VPT], W[VPT];
#pragma unroll
            for (int k = 0; k < VPT; ++k) {
                const int64_t n = n0 + static_cast<int64_t>(k) * NT;
                const bool ok = n < n_vis;
                const double s = sgn * ch.scale;   // sign folded into B (exact negation)
                U[k] = split_f64(ok ? uvw_m[3 * n] * s : 0.0);
                V[k] = split_f64(ok ? uvw_m[3 * n + 1] * s : 0.0);
                W[k] = split_f64(ok ? uvw_m[3 * n + 2] * s : 0.0);
            }
            float2 res[VPT];
            float C[VPT];
            bool defer = false;
            float2* rstk = reinterpret_cast<float2*>(stk_base) + threadIdx.x * VPT;   // [row][thread][vis] layout
            if constexpr (GRIDPASS) {
                // an item that does not fit is swept too, its results discarded
                defer = !tile_grid_constants(U, V, W, ch.hdr->smax, C);   // a CTA-wide decision
                good = sweep_regrouped_mixed<NT, VPT, FAST, true, false>(st, U, V, W, C, rstk, ch.J, maxrow, res);
            } else {
                good = sweep_regrouped_mixed<NT, VPT, FAST, false, false>(st, U, V, W, C, rstk, ch.J, maxrow, res);
            }
            if (good && defer) mark_deferred(first_vis);
#pragma unroll
            for (int k = 0; k < VPT; ++k) {
                const int64_t n = n0 + static_cast<int64_t>(k) * NT;
                if (good && !defer && n < n_vis) out[n] = res[k];
            }
        } else {
            Eq17D<NT, VPT> b;
#pragma unroll
            for (int k = 0; k < VPT; ++k) {
                const int64_t n = n0 + static_cast<int64_t>(k) * NT;
                const bool ok = n < n_vis;
                const double s = sgn * ch.scale;
                b.u[k] = ok ? uvw_m[3 * n] * s : 0.0;
                b.v[k] = ok ? uvw_m[3 * n + 1] * s : 0.0;
                b.w[k] = ok ? uvw_m[3 * n + 2] * s : 0.0;
                b.vr[k] = 0.0; b.vi[k] = 0.0;
            }
            b.sgn = 1.0;
            b.stk = reinterpret_cast<double2*>(stk_base) + threadIdx.x;
            b.maxrow = maxrow;
            good = st.sweep(b);
            double2* out = static_cast<double2*>(vis) + ch.out_offset;
#pragma unroll
            for (int k = 0; k < VPT; ++k) {
                const int64_t n = n0 + static_cast<int64_t>(k) * NT;
                if (good && n < n_vis) out[n] = make_double2(b.vr[k], b.vi[k]);
            }
        }
        if (!good) {
            if (threadIdx.x == 0) record_status(status, WT_ERR_TIMEOUT);
            return;
        }
    }
}

// ---------------------------------------------------------------- host
struct Shape {
    int nt, vpt;
};
constexpr int kNumBatchShapes = 6;
const Shape kBatchShapes[kNumBatchShapes] = {{256, 1}, {128, 1}, {128, 2}, {64, 2}, {32, 1}, {32, 2}};

// Stack rows for the deepest tree of a plan: the explicit float64 sum keeps
// four child slots per level, the regrouped mixed sum one pair per level
// above J - 2, the double-float sum one entry per level above J - 1.
int batch_rows(int mode, int jmax)
{
    if (mode == WT_FP64) return jmax > 1 ? 4 * (jmax - 1) : 4;
    if (mode == WT_FP64_DF) return jmax > 3 ? jmax - 2 : 1;
    return jmax > 4 ? jmax - 3 : 1;
}

size_t batch_smem(int mode, int shape, int rows_max)
{
    const size_t cplx = (mode == WT_FP64 || mode == WT_FP64_DF) ? sizeof(double2) : sizeof(float2);
    const size_t stage = mode == WT_FP64      ? stager_bytes<RecD>(kChunkD)
                         : mode == WT_FP64_DF ? stager_bytes<RecWDF>(kChunkDF) + kDfTableEntries * sizeof(float4)
                                              : stager_bytes<RecWF>(kChunkW);
    return stage + static_cast<size_t>(rows_max) * kBatchShapes[shape].nt * kBatchShapes[shape].vpt * cplx;
}

bool batch_fits(int mode, int shape, int rows_max) { return batch_smem(mode, shape, rows_max) <= 220 * 1024; }

// Shape used without timing (WT_AUTOTUNE=0, or under stream capture): the
// first that fits in a measured preference order (the regrouped mixed sum
// runs best with two visibilities per thread).
int default_shape(int mode, int rows_max)
{
    static const int order_fp64[kNumBatchShapes] = {0, 1, 2, 3, 4, 5};
    static const int order_df[kNumBatchShapes] = {1, 0, 2, 3, 4, 5};
    static const int order_mixed[kNumBatchShapes] = {2, 3, 5, 0, 1, 4};
    const int* order = (mode == WT_FP64) ? order_fp64 : (mode == WT_FP64_DF) ? order_df : order_mixed;
    for (int i = 0; i < kNumBatchShapes; ++i)
        if (batch_fits(mode, order[i], rows_max)) return order[i];
    return -1;
}

// WT_BATCH_QUEUE=1 sends every batch through the persistent work queue
// (otherwise taken only beyond 2^31 - 1 items), so that tests reach it.
bool force_queue()
{
    const char* e = getenv("WT_BATCH_QUEUE");
    return e && e[0] == '1';
}

template <int NT, int VPT, int KIND, bool FAST = false, bool GRIDPASS = false>
int launch_pass(const BatchChan* chans, int n_ch, int64_t total, const double* uvw_m, int64_t n_vis, void* vis,
                int sign, int rows_max, unsigned long long* queue, int* status, size_t smem, cudaStream_t s)
{
    auto k = k_batched<NT, VPT, KIND, FAST, GRIDPASS>;
    int per_sm = 0;
    WT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NT, smem));
    if (per_sm < 1) return set_error(WT_ERR_UNSUPPORTED, "batched kernel does not fit on an SM");
    // One CTA per item: the hardware balances the SMs as CTAs finish, as for
    // the single-channel predictor. The queue serves batches of more items
    // than a grid holds (reset before each pass).
    const bool per_item = total <= 0x7fffffff && !force_queue();
    int64_t grid = per_item ? total : static_cast<int64_t>(num_sms()) * per_sm;
    if (grid < 1) grid = 1;
    if (!per_item) WT_CUDA_TRY(cudaMemsetAsync(queue, 0, sizeof(unsigned long long), s));
    k<<<static_cast<unsigned>(grid), NT, smem, s>>>(chans, n_ch, total, uvw_m, n_vis, vis, static_cast<double>(sign),
                                                    rows_max, per_item ? nullptr : queue, status);
    WT_CUDA_TRY(cudaGetLastError());
    return WT_OK;
}

// The mixed kind: the grid pass, then the exact pass over the items it left
// marked; the other kinds: one pass.
template <int NT, int VPT, int KIND, bool FAST = false>
int launch_shape(const BatchChan* chans, int n_ch, int64_t total, const double* uvw_m, int64_t n_vis, void* vis,
                 int sign, int rows_max, unsigned long long* queue, int* status, size_t smem, cudaStream_t s)
{
    if constexpr (KIND == kKindMixed) {
        const int rc = launch_pass<NT, VPT, KIND, FAST, true>(chans, n_ch, total, uvw_m, n_vis, vis, sign, rows_max,
                                                              queue, status, smem, s);
        if (rc) return rc;
        return launch_pass<NT, VPT, KIND, FAST, false>(chans, n_ch, total, uvw_m, n_vis, vis, sign, rows_max, queue,
                                                       status, smem, s);
    }
    return launch_pass<NT, VPT, KIND, FAST>(chans, n_ch, total, uvw_m, n_vis, vis, sign, rows_max, queue, status,
                                            smem, s);
}

template <int KIND, bool FAST = false, bool GRIDPASS = false>
int set_attr_pass(int shape, size_t smem)
{
    const void* fn;
    switch (shape) {
        case 0: fn = reinterpret_cast<const void*>(k_batched<256, 1, KIND, FAST, GRIDPASS>); break;
        case 1: fn = reinterpret_cast<const void*>(k_batched<128, 1, KIND, FAST, GRIDPASS>); break;
        case 2: fn = reinterpret_cast<const void*>(k_batched<128, 2, KIND, FAST, GRIDPASS>); break;
        case 3: fn = reinterpret_cast<const void*>(k_batched<64, 2, KIND, FAST, GRIDPASS>); break;
        case 4: fn = reinterpret_cast<const void*>(k_batched<32, 1, KIND, FAST, GRIDPASS>); break;
        default: fn = reinterpret_cast<const void*>(k_batched<32, 2, KIND, FAST, GRIDPASS>); break;
    }
    WT_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
    return WT_OK;
}

template <int KIND, bool FAST = false>
int set_attr(int shape, size_t smem)
{
    if constexpr (KIND == kKindMixed) {
        const int rc = set_attr_pass<KIND, FAST, true>(shape, smem);
        if (rc) return rc;
        return set_attr_pass<KIND, FAST, false>(shape, smem);
    }
    return set_attr_pass<KIND, FAST>(shape, smem);
}

template <int KIND, bool FAST = false>
int launch_kind(int shape, const BatchChan* chans, int n_ch, int64_t total, const double* uvw_m, int64_t n_vis,
                void* vis, int sign, int rows_max, unsigned long long* queue, int* status, size_t smem, cudaStream_t s)
{
    switch (shape) {
        case 0: return launch_shape<256, 1, KIND, FAST>(chans, n_ch, total, uvw_m, n_vis, vis, sign, rows_max, queue, status, smem, s);
        case 1: return launch_shape<128, 1, KIND, FAST>(chans, n_ch, total, uvw_m, n_vis, vis, sign, rows_max, queue, status, smem, s);
        case 2: return launch_shape<128, 2, KIND, FAST>(chans, n_ch, total, uvw_m, n_vis, vis, sign, rows_max, queue, status, smem, s);
        case 3: return launch_shape<64, 2, KIND, FAST>(chans, n_ch, total, uvw_m, n_vis, vis, sign, rows_max, queue, status, smem, s);
        case 4: return launch_shape<32, 1, KIND, FAST>(chans, n_ch, total, uvw_m, n_vis, vis, sign, rows_max, queue, status, smem, s);
        default: return launch_shape<32, 2, KIND, FAST>(chans, n_ch, total, uvw_m, n_vis, vis, sign, rows_max, queue, status, smem, s);
    }
}

int launch_batch(int mode, int shape, const BatchChan* chans, int n_ch, int64_t total, const double* uvw_m,
                 int64_t n_vis, void* vis, int sign, int rows_max, unsigned long long* queue, int* status,
                 cudaStream_t s)
{
    const size_t smem = batch_smem(mode, shape, rows_max);
    if (mode == WT_FP64)
        return launch_kind<kKindF64>(shape, chans, n_ch, total, uvw_m, n_vis, vis, sign, rows_max, queue, status, smem, s);
    if (mode == WT_FP64_DF)
        return launch_kind<kKindDF>(shape, chans, n_ch, total, uvw_m, n_vis, vis, sign, rows_max, queue, status, smem, s);
    if (mode == WT_MIXED_FAST)
        return launch_kind<kKindMixed, true>(shape, chans, n_ch, total, uvw_m, n_vis, vis, sign, rows_max, queue, status,
                                             smem, s);
    return launch_kind<kKindMixed>(shape, chans, n_ch, total, uvw_m, n_vis, vis, sign, rows_max, queue, status, smem, s);
}

// The shared-memory attribute of a shape's kernel in a plan's form.
int set_attr_mode(int mode, int shape, size_t smem)
{
    if (mode == WT_FP64) return set_attr<kKindF64>(shape, smem);
    if (mode == WT_FP64_DF) return set_attr<kKindDF>(shape, smem);
    if (mode == WT_MIXED_FAST) return set_attr<kKindMixed, true>(shape, smem);
    return set_attr<kKindMixed>(shape, smem);
}

// A plan: one set of trees and frequencies in one form, its device-side
// channel table and counter, its launch shape and its captured graph.
struct Plan {
    int device = 0, mode = 0, sign = 1, n_ch = 0;
    std::vector<wt_tree> trees;
    std::vector<double> freqs;
    std::vector<int> order;          // channels by decreasing node count
    std::vector<int64_t> nodes;
    int rows_max = 4;
    int shape = -1;
    void* dmem = nullptr;            // [n_ch] BatchChan + counter
    BatchChan* d_chan = nullptr;
    unsigned long long* d_queue = nullptr;
    int64_t table_nvis = -1;
    int table_shape = -1;
    int64_t total = 0;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec = nullptr;
    const double* g_uvw = nullptr;
    int64_t g_nvis = -1;
    void* g_vis = nullptr;
    int g_shape = -1;

    ~Plan()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (cap) cudaStreamDestroy(cap);
        if (dmem) cudaFree(dmem);
        cudaGetLastError();
    }
};

std::mutex g_mu;
std::vector<std::unique_ptr<Plan>> g_plans;

Plan* find_plan(const wt_tree* trees, const double* freqs, int n_ch, int mode, int sign, int dev)
{
    for (auto& p : g_plans) {
        if (p->device != dev || p->mode != mode || p->sign != sign || p->n_ch != n_ch) continue;
        bool same = true;
        for (int c = 0; c < n_ch && same; ++c) same = p->trees[c] == trees[c] && p->freqs[c] == freqs[c];
        if (same) return p.get();
    }
    return nullptr;
}

// Fill and upload the channel table for n_vis and the plan's shape.
int write_table(Plan& p, int64_t n_vis, int shape, cudaStream_t s)
{
    if (p.table_nvis == n_vis && p.table_shape == shape) return WT_OK;
    const int64_t per_tile = static_cast<int64_t>(kBatchShapes[shape].nt) * kBatchShapes[shape].vpt;
    const int64_t tiles = (n_vis + per_tile - 1) / per_tile;
    std::vector<BatchChan> h(p.n_ch);
    int64_t base = 0;
    for (int i = 0; i < p.n_ch; ++i) {
        const int c = p.order[i];
        wt_tree t = p.trees[c];
        BatchChan& b = h[i];
        b.recd = t->d.recd;
        b.recwf = t->d.recwf;
        b.recwdf = t->d.recwdf;
        b.hdr = t->d.hdr;
        b.scale = p.freqs[c] / kLightSpeed;
        b.out_offset = static_cast<int64_t>(c) * n_vis;
        b.tile_base = base;
        b.J = t->J;
        b.pad = 0;
        base += tiles;
    }
    // The table is read by kernels already enqueued on `s`; order the copy
    // after them and keep the host buffer alive until it is done.
    WT_CUDA_TRY(cudaMemcpyAsync(p.d_chan, h.data(), sizeof(BatchChan) * p.n_ch, cudaMemcpyHostToDevice, s));
    WT_CUDA_TRY(cudaStreamSynchronize(s));
    p.table_nvis = n_vis;
    p.table_shape = shape;
    p.total = base;
    return WT_OK;
}

int tune(Plan& p, const double* uvw_m, int64_t n_vis, void* vis, int* status, cudaStream_t s)
{
    const int first = default_shape(p.mode, p.rows_max);
    if (first < 0) return set_error(WT_ERR_UNSUPPORTED, "wt_predict_vis_batched: no launch shape fits J");
    const char* pin = getenv("WT_BATCH_SHAPE");   // pins shape k of kBatchShapes when it fits
    if (pin) {
        const int v = atoi(pin);
        if (v >= 0 && v < kNumBatchShapes && batch_fits(p.mode, v, p.rows_max)) return v;
    }
    const char* e = getenv("WT_AUTOTUNE");
    if (e && e[0] == '0') return first;
    // per channel: the mixed forms are timed on up to 131 072 visibilities
    // (with 64 channels, several waves of every shape), float64 on 16 384
    const int64_t cap = (p.mode == WT_FP64) ? 16384 : (p.mode == WT_FP64_DF) ? 32768 : 131072;
    const int64_t sample = n_vis < cap ? n_vis : cap;
    cudaEvent_t e0, e1;
    WT_CUDA_TRY(cudaEventCreate(&e0));
    WT_CUDA_TRY(cudaEventCreate(&e1));
    int best = first;
    float best_ms = 1e30f;
    for (int sh = 0; sh < kNumBatchShapes; ++sh) {
        if (!batch_fits(p.mode, sh, p.rows_max)) continue;
        const size_t sm = batch_smem(p.mode, sh, p.rows_max);
        int rc = set_attr_mode(p.mode, sh, sm);
        if (rc) continue;
        if (write_table(p, sample, sh, s)) continue;
        float ms_best_rep = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
            cudaMemsetAsync(p.d_queue, 0, sizeof(unsigned long long), s);
            cudaEventRecord(e0, s);
            rc = launch_batch(p.mode, sh, p.d_chan, p.n_ch, p.total, uvw_m, sample, vis, p.sign, p.rows_max,
                              p.d_queue, status, s);
            cudaEventRecord(e1, s);
            if (rc || cudaEventSynchronize(e1) != cudaSuccess) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < ms_best_rep) ms_best_rep = ms;
        }
        cudaGetLastError();
        const char* v = getenv("WT_AUTOTUNE_VERBOSE");
        if (v && v[0] == '1')
            fprintf(stderr, "[wt autotune] batched n_ch=%d mode%d shape %d (%d threads x %d vis): %.4f ms for %lld vis/ch\n",
                    p.n_ch, p.mode, sh, kBatchShapes[sh].nt, kBatchShapes[sh].vpt, ms_best_rep,
                    static_cast<long long>(sample));
        if (ms_best_rep < best_ms) {
            best_ms = ms_best_rep;
            best = sh;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}

}  // namespace

void batch_forget_tree(wt_tree t)
{
    std::lock_guard<std::mutex> lk(g_mu);
    for (size_t i = 0; i < g_plans.size();) {
        bool uses = false;
        for (wt_tree x : g_plans[i]->trees) uses = uses || x == t;
        if (uses) g_plans.erase(g_plans.begin() + static_cast<long>(i));
        else ++i;
    }
}

int predict_batched(const wt_tree* trees, const double* freq_hz, int n_ch, const double* uvw_m, int64_t n_vis,
                    void* vis, int mode, int sign, cudaStream_t s)
{
    int dev = 0;
    WT_CUDA_TRY(cudaGetDevice(&dev));
    int* status = device_status_word();
    if (!status) return set_error(WT_ERR_CUDA, "wt_predict_vis_batched: no device status word");
    std::lock_guard<std::mutex> lk(g_mu);
    Plan* p = find_plan(trees, freq_hz, n_ch, mode, sign, dev);
    if (!p) {
        std::unique_ptr<Plan> np(new Plan());
        np->device = dev;
        np->mode = mode;
        np->sign = sign;
        np->n_ch = n_ch;
        np->trees.assign(trees, trees + n_ch);
        np->freqs.assign(freq_hz, freq_hz + n_ch);
        np->nodes.resize(n_ch);
        int jmax = 1;
        for (int c = 0; c < n_ch; ++c) {
            int rc = tree_sync_header(trees[c]);
            if (rc) return rc;
            np->nodes[c] = trees[c]->host_hdr->n_nodes;
            if (trees[c]->J > jmax) jmax = trees[c]->J;
        }
        np->rows_max = batch_rows(mode, jmax);
        np->order.resize(n_ch);
        for (int c = 0; c < n_ch; ++c) np->order[c] = c;
        std::stable_sort(np->order.begin(), np->order.end(),
                         [&](int a, int b) { return np->nodes[a] > np->nodes[b]; });
        const size_t bytes = sizeof(BatchChan) * static_cast<size_t>(n_ch) + 256;
        cudaError_t e = cudaMalloc(&np->dmem, bytes);
        if (e != cudaSuccess) return cuda_error(e, "cudaMalloc (batch plan)");
        np->d_chan = static_cast<BatchChan*>(np->dmem);
        np->d_queue = reinterpret_cast<unsigned long long*>(static_cast<char*>(np->dmem) +
                                                            ((sizeof(BatchChan) * n_ch + 127) & ~size_t(127)));
        WT_CUDA_TRY(cudaStreamCreateWithFlags(&np->cap, cudaStreamNonBlocking));
        p = np.get();
        g_plans.push_back(std::move(np));
    }
    if (p->shape < 0) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        WT_CUDA_TRY(cudaStreamIsCapturing(s, &cs));
        if (cs != cudaStreamCaptureStatusNone) {
            p->shape = default_shape(mode, p->rows_max);
            if (p->shape < 0) return set_error(WT_ERR_UNSUPPORTED, "wt_predict_vis_batched: no launch shape fits J");
        } else {
            const int best = tune(*p, uvw_m, n_vis, vis, status, s);
            if (best < 0) return best;
            p->shape = best;
        }
    }
    const size_t smem = batch_smem(mode, p->shape, p->rows_max);
    int rc = set_attr_mode(mode, p->shape, smem);
    if (rc) return rc;
    if ((rc = write_table(*p, n_vis, p->shape, s))) return rc;
    if (!p->exec || p->g_uvw != uvw_m || p->g_nvis != n_vis || p->g_vis != vis || p->g_shape != p->shape) {
        // capture [counter reset, kernel] once for these buffers
        cudaGraph_t g = nullptr;
        WT_CUDA_TRY(cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal));
        cudaMemsetAsync(p->d_queue, 0, sizeof(unsigned long long), p->cap);
        rc = launch_batch(mode, p->shape, p->d_chan, n_ch, p->total, uvw_m, n_vis, vis, sign, p->rows_max,
                          p->d_queue, status, p->cap);
        cudaError_t e = cudaStreamEndCapture(p->cap, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture");
        if (p->exec) cudaGraphExecDestroy(p->exec);
        p->exec = nullptr;
        e = cudaGraphInstantiate(&p->exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_error(e, "cudaGraphInstantiate");
        p->g_uvw = uvw_m;
        p->g_nvis = n_vis;
        p->g_vis = vis;
        p->g_shape = p->shape;
    }
    WT_CUDA_TRY(cudaGraphLaunch(p->exec, s));
    return WT_OK;
}

}  // namespace wt

// ---------------------------------------------------------------------------
extern "C" int wt_predict_vis_batched(const wt_tree* trees, const double* freq_hz, int n_ch, const double* uvw_m,
                                      int64_t n_vis, void* vis_out, int mode, int sign, void* stream)
{
    using namespace wt;
    const char* fn = "wt_predict_vis_batched";
    if (!trees || !freq_hz) return set_error(WT_ERR_ARG, "%s: trees and freq_hz are host arrays, not NULL", fn);
    if (n_ch < 1 || n_ch > 65536) return set_error(WT_ERR_ARG, "%s: n_ch = %d outside 1..65536", fn, n_ch);
    if (n_vis < 0) return set_error(WT_ERR_ARG, "%s: n_vis < 0", fn);
    if (sign != 1 && sign != -1) return set_error(WT_ERR_ARG, "%s: sign must be +1 or -1", fn);
    if (mode != WT_FP64 && mode != WT_MIXED && mode != WT_MIXED_FAST && mode != WT_FP64_DF)
        return set_error(WT_ERR_ARG, "%s: bad mode %d", fn, mode);
    int dev = 0;
    WT_CUDA_TRY(cudaGetDevice(&dev));
    for (int c = 0; c < n_ch; ++c) {
        wt_tree t = trees[c];
        if (!t) return set_error(WT_ERR_ARG, "%s: tree %d is NULL", fn, c);
        if (t->magic != kTreeMagic) return set_error(WT_ERR_CORRUPT, "%s: tree %d is not a live handle", fn, c);
        if (t->device != dev) return set_error(WT_ERR_ARG, "%s: tree %d lives on another device", fn, c);
        if (!(freq_hz[c] > 0.0) || !isfinite(freq_hz[c]))
            return set_error(WT_ERR_RANGE, "%s: frequency %d must be positive and finite", fn, c);
    }
    const size_t ob = static_cast<size_t>(n_vis) * n_ch * ((mode == WT_FP64 || mode == WT_FP64_DF) ? 16 : 8);
    int rc;
    if ((rc = check_device_buffer(uvw_m, static_cast<size_t>(n_vis) * 24, fn, "uvw_m", 8)) ||
        (rc = check_device_buffer(vis_out, ob, fn, "vis_out", vis_align(mode))))
        return rc;
    if (n_vis == 0) return WT_OK;
    return predict_batched(trees, freq_hz, n_ch, uvw_m, n_vis, vis_out, mode, sign, static_cast<cudaStream_t>(stream));
}
