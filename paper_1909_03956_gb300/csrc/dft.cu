// dft.cu -- dft_predict_vis: the direct sum over the clean-component list
// (Sec. 3.3, Eq. 12; the "more accurate alternative" of Sec. 2.2):
//   V_n = sum_m C_m exp(sign i 2 pi [u_n l_m + v_n m_m + w_n (n_m - 1)]).
//
// A prologue kernel packs each component once into a 32-byte record in a
// scratch buffer: (l, m, n - 1, C) in float64 for WT_FP64, or double-float
// halves of l, m, n - 1 and C for the other forms (the mixed forms use C's
// high half only), and reduces the bounds max |l|, |m|, |n - 1| of the
// float32 heads into a 16-byte block after the records. The main kernel gives
// each thread one visibility (float64) or two (mixed, on packed float32
// pairs) and streams the records through shared memory (bulk copies,
// double-buffered, broadcast reads), like the wavelet kernels. The mixed
// forms run a grid pass and an exact pass, as the regrouped wavelet sum does
// (wt_internal.cuh): the phase heads on each visibility's common grid where
// the bounds allow, else error-free sums.
#include "df64.cuh"
#include "staging.cuh"
#include "wt_internal.cuh"

namespace wt {

// dft_tc.cu: the tensor-core form (WT_MIXED_TC)
size_t dft_tc_scratch_bytes(int64_t n_comp);
int dft_tc_launch(const double* l, const double* m, const double* flux, int64_t n_comp, const void* recs,
                  const uint32_t* bound, void* tc, const double* uvw, int64_t n_vis, float2* vis, int sign,
                  int* status, cudaStream_t s);

namespace {

constexpr int kChunk = 512;

struct CompD {
    double l, m, nm1, flux;
};
static_assert(sizeof(CompD) == 32, "component record layout");

// n - 1 = -(l^2 + m^2) / (1 + sqrt(1 - l^2 - m^2)), free of cancellation.
// bound (float records only; zeroed before the launch): the largest |l|,
// |m|, |n - 1| of the float32 heads as float bit patterns (non-negative
// floats order as their bits), reduced per warp, then by atomicMax; a
// component that fails the range check adds nothing.
__global__ void k_pack_components(const double* __restrict__ l, const double* __restrict__ m,
                                  const double* __restrict__ flux, int64_t n, CompD* __restrict__ outd,
                                  CompF* __restrict__ outf, uint32_t* __restrict__ bound, int* status)
{
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    uint32_t bl = 0, bm = 0, bn = 0;
    if (i < n) {
        const double li = l[i], mi = m[i], fi = flux[i];
        const double r2 = li * li + mi * mi;
        double nm1 = 0.0;
        const bool good = r2 < 1.0 && isfinite(li) && isfinite(mi) && isfinite(fi);
        if (!good) record_status(status, WT_ERR_RANGE);
        else nm1 = -r2 / (1.0 + sqrt(1.0 - r2));
        if (outd) outd[i] = CompD{li, mi, nm1, fi};
        if (outf) {
            const F2 a = split_f64(li), b = split_f64(mi), c = split_f64(nm1), f = split_f64(fi);
            outf[i] = CompF{a.hi, a.lo, b.hi, b.lo, c.hi, c.lo, f.hi, f.lo};
            if (good) {
                bl = __float_as_uint(fabsf(a.hi));
                bm = __float_as_uint(fabsf(b.hi));
                bn = __float_as_uint(fabsf(c.hi));
            }
        }
    }
    if (!bound) return;
    bl = __reduce_max_sync(0xffffffffu, bl);
    bm = __reduce_max_sync(0xffffffffu, bm);
    bn = __reduce_max_sync(0xffffffffu, bn);
    if ((threadIdx.x & 31) == 0) {
        if (bl) atomicMax(&bound[0], bl);
        if (bm) atomicMax(&bound[1], bm);
        if (bn) atomicMax(&bound[2], bn);
    }
}

struct BodyD {
    double u, v, w, sgn, vr, vi;
    __device__ void operator()(const CompD& c)
    {
        double t = fma(w, c.nm1, fma(v, c.m, u * c.l));
        double s, co;
        sincos_turns_f64(t, s, co);
        vr = fma(c.flux, co, vr);
        vi = fma(c.flux, s, vi);
    }
};

// Mixed forms on packed float32 pairs: a thread owns two visibilities
// (n and n + NT of its tile). The phases of the two visibilities against one
// component form one pair of double-floats; each visibility's (cos, sin)
// comes out as its own pair. The components are taken kSumBlock at a time:
// their terms added by FMAs into a partial per visibility, the partial then
// into its Kahan sum (blockwise compensated summation).
// GRID: the phases with their heads on the grids of Cg (phase_turns_grid2),
// else with error-free sums (phase_turns_df2).
template <bool FAST, bool GRID>
struct BodyF2 {
    DF2 U, V, W;
    float2 Cg;
    float2 acc[2], comp[2];

    // p0 += flux (cos, sin) of visibility 0, p1 of visibility 1
    __device__ __forceinline__ void add_term(const CompF& c, float2& p0, float2& p1) const
    {
        float2 h, tl, e0, e1;
        if constexpr (GRID) phase_turns_grid2(U, V, W, F2{c.lh, c.ll}, F2{c.mh, c.ml}, F2{c.nh, c.nl}, Cg, h, tl);
        else phase_turns_df2(U, V, W, F2{c.lh, c.ll}, F2{c.mh, c.ml}, F2{c.nh, c.nl}, h, tl);
        sincos_mixed2<FAST>(h, tl, e0, e1);
        const float2 f = bcast2(c.flux);
        p0 = fma2(f, e0, p0);
        p1 = fma2(f, e1, p1);
    }

    // One block of components from record r on; returns how many it took
    // (kSumBlock, or what is left of a list's last chunk).
    __device__ __forceinline__ int at(const CompF* cb, int r, int n)
    {
        float2 p0 = make_float2(0.f, 0.f), p1 = p0;
        int taken;
        if (r + kSumBlock <= n) {
#pragma unroll 2
            for (int j = 0; j < kSumBlock; ++j) add_term(cb[r + j], p0, p1);
            taken = kSumBlock;
        } else {
            for (int j = r; j < n; ++j) add_term(cb[j], p0, p1);
            taken = n - r;
        }
        kahan_add2(acc[0], comp[0], p0);
        kahan_add2(acc[1], comp[1], p1);
        return taken;
    }
};

// The float64-class double-float form: one visibility per thread, every
// step in double-float (df64.cuh).
struct BodyDF {
    F2 u, v, w;
    DF vr, vi;
    const float4* tab;
    __device__ void operator()(const CompF& c)
    {
        float th, tl;
        phase_turns_df(u, v, w, F2{c.lh, c.ll}, F2{c.mh, c.ml}, F2{c.nh, c.nl}, th, tl);
        DF s, co;
        sincos_turns_df(th, tl, tab, s, co);
        const DF f{c.flux, c.flux_lo};
        vr = df_add(vr, df_mul(f, co));
        vi = df_add(vi, df_mul(f, s));
    }
};

template <int NT>
__global__ void __launch_bounds__(NT) k_dft_df(const CompF* __restrict__ comps, int64_t n_comp,
                                               const double* __restrict__ uvw, int64_t n_vis,
                                               double2* __restrict__ vis, double sgn, int* status)
{
    extern __shared__ __align__(16) unsigned char smem[];
    Stager<CompF> st;
    stager_setup(st, smem, comps, n_comp, kChunk);
    float4* tab = reinterpret_cast<float4*>(smem + stager_bytes<CompF>(kChunk));
    load_sincos_table_df(tab);
    __syncthreads();
    const int64_t ntiles = (n_vis + NT - 1) / NT;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t n = tile * NT + threadIdx.x;
        const bool valid = n < n_vis;
        BodyDF b;
        b.u = split_f64(valid ? sgn * uvw[3 * n] : 0.0);   // sign folded into the baseline (exact)
        b.v = split_f64(valid ? sgn * uvw[3 * n + 1] : 0.0);
        b.w = split_f64(valid ? sgn * uvw[3 * n + 2] : 0.0);
        b.vr = DF{0.f, 0.f};
        b.vi = DF{0.f, 0.f};
        b.tab = tab;
        if (!st.sweep(b)) {
            if (threadIdx.x == 0) record_status(status, WT_ERR_TIMEOUT);
            return;
        }
        if (valid) vis[n] = make_double2(df_to_double(b.vr), df_to_double(b.vi));
    }
}

template <int NT>
__global__ void __launch_bounds__(NT) k_dft_fp64(const CompD* __restrict__ comps, int64_t n_comp,
                                                 const double* __restrict__ uvw, int64_t n_vis,
                                                 double2* __restrict__ vis, double sgn, int* status)
{
    extern __shared__ __align__(16) unsigned char smem[];
    Stager<CompD> st;
    stager_setup(st, smem, comps, n_comp, kChunk);
    const int64_t ntiles = (n_vis + NT - 1) / NT;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t n = tile * NT + threadIdx.x;
        const bool valid = n < n_vis;
        // the sign is folded into the baseline: exp(-i 2 pi t) = exp(i 2 pi (-t)), exact
        BodyD b{valid ? sgn * uvw[3 * n] : 0.0, valid ? sgn * uvw[3 * n + 1] : 0.0,
                valid ? sgn * uvw[3 * n + 2] : 0.0, sgn, 0.0, 0.0};
        if (!st.sweep(b)) {
            if (threadIdx.x == 0) record_status(status, WT_ERR_TIMEOUT);
            return;
        }
        if (valid) vis[n] = make_double2(b.vr, b.vi);
    }
}

// GRIDPASS: the grid pass (every tile; a tile whose phases do not all fit
// the head grid is swept too, its results discarded, and marked for the
// exact pass); else the exact pass (only the marked tiles). bound: the
// records' coordinate bounds (k_pack_components).
template <int NT, bool FAST, bool GRIDPASS>
__global__ void __launch_bounds__(NT) k_dft_mixed(const CompF* __restrict__ comps, int64_t n_comp,
                                                  const uint32_t* __restrict__ bound,
                                                  const double* __restrict__ uvw, int64_t n_vis,
                                                  float2* __restrict__ vis, float sgn, int* status)
{
    extern __shared__ __align__(16) unsigned char smem[];
    Stager<CompF> st;
    stager_setup(st, smem, comps, n_comp, kChunk);
    const int64_t ntiles = (n_vis + 2 * NT - 1) / (2 * NT);
    const double sg = static_cast<double>(sgn);       // sign folded into the baseline (exact)
    float smax[3] = {0.f, 0.f, 0.f};
    if constexpr (GRIDPASS) {
        smax[0] = __uint_as_float(bound[0]);
        smax[1] = __uint_as_float(bound[1]);
        smax[2] = __uint_as_float(bound[2]);
    }
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        float2* first_vis = vis + tile * 2 * NT;
        if constexpr (!GRIDPASS) {
            if (!tile_deferred(first_vis)) continue;   // done by the grid pass
        }
        const int64_t n0 = tile * 2 * NT + threadIdx.x, n1 = n0 + NT;
        const bool ok0 = n0 < n_vis, ok1 = n1 < n_vis;
        const F2 u[2] = {split_f64(ok0 ? sg * uvw[3 * n0] : 0.0), split_f64(ok1 ? sg * uvw[3 * n1] : 0.0)};
        const F2 v[2] = {split_f64(ok0 ? sg * uvw[3 * n0 + 1] : 0.0), split_f64(ok1 ? sg * uvw[3 * n1 + 1] : 0.0)};
        const F2 w[2] = {split_f64(ok0 ? sg * uvw[3 * n0 + 2] : 0.0), split_f64(ok1 ? sg * uvw[3 * n1 + 2] : 0.0)};
        BodyF2<FAST, GRIDPASS> b;
        bool defer = false;
        if constexpr (GRIDPASS) {
            float C[2];
            defer = !tile_grid_constants<2>(u, v, w, smax, C);   // a CTA-wide decision
            b.Cg = make_float2(C[0], C[1]);
        }
        b.U = df2_pack(u[0], u[1]);
        b.V = df2_pack(v[0], v[1]);
        b.W = df2_pack(w[0], w[1]);
        b.acc[0] = b.acc[1] = b.comp[0] = b.comp[1] = make_float2(0.f, 0.f);
        if (!st.sweep_at(b)) {
            if (threadIdx.x == 0) record_status(status, WT_ERR_TIMEOUT);
            return;
        }
        if (defer) {
            mark_deferred(first_vis);
            continue;
        }
        if (ok0) vis[n0] = sub2(b.acc[0], b.comp[0]);
        if (ok1) vis[n1] = sub2(b.acc[1], b.comp[1]);
    }
}

template <class K>
int grid_for(K kernel, int threads, int nt, size_t smem, int64_t n_vis, dim3& grid)
{
    WT_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
    int per_sm = 0;
    WT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem));
    if (per_sm < 1) return set_error(WT_ERR_UNSUPPORTED, "dft kernel does not fit on an SM");
    // one CTA per tile (nt visibilities), so that the hardware balances the
    // SMs as CTAs finish; the kernels stride only if the grid is capped
    const int64_t ntiles = (n_vis + nt - 1) / nt;
    grid = dim3(static_cast<unsigned>(ntiles < 0x7fffffff ? ntiles : 0x7fffffff));
    return WT_OK;
}

}  // namespace

// Launch the DFT on component records already packed in `scratch`
// (n_comp records of 32 bytes, 256-byte aligned) with their coordinate
// bounds at `bound` (mixed forms); errors go to `status`.
int dft_launch_packed(const void* scratch, const uint32_t* bound, int64_t n_comp, const double* uvw, int64_t n_vis,
                      void* vis, int mode, int sign, int* status, cudaStream_t s)
{
    dim3 grid;
    if (mode == WT_FP64) {
        constexpr int NT = 128;
        const size_t smem = static_cast<size_t>(stager_bytes<CompD>(kChunk));
        auto k = k_dft_fp64<NT>;
        int rc = grid_for(k, NT, NT, smem, n_vis, grid);
        if (rc) return rc;
        k<<<grid, NT, smem, s>>>(static_cast<const CompD*>(scratch), n_comp, uvw, n_vis, static_cast<double2*>(vis),
                                 static_cast<double>(sign), status);
    } else if (mode == WT_FP64_DF) {
        constexpr int NT = 128;
        const size_t smem = static_cast<size_t>(stager_bytes<CompF>(kChunk)) + kDfTableEntries * sizeof(float4);
        auto k = k_dft_df<NT>;
        int rc = grid_for(k, NT, NT, smem, n_vis, grid);
        if (rc) return rc;
        k<<<grid, NT, smem, s>>>(static_cast<const CompF*>(scratch), n_comp, uvw, n_vis, static_cast<double2*>(vis),
                                 static_cast<double>(sign), status);
    } else {
        // the grid pass, then the exact pass over the tiles it left marked
        constexpr int NT = 256;
        const size_t smem = static_cast<size_t>(stager_bytes<CompF>(kChunk));
        const bool fast = mode == WT_MIXED_FAST;
        auto kg = fast ? k_dft_mixed<NT, true, true> : k_dft_mixed<NT, false, true>;
        auto ke = fast ? k_dft_mixed<NT, true, false> : k_dft_mixed<NT, false, false>;
        dim3 grid_e;
        int rc = grid_for(kg, NT, 2 * NT, smem, n_vis, grid);   // two visibilities per thread
        if (!rc) rc = grid_for(ke, NT, 2 * NT, smem, n_vis, grid_e);
        if (rc) return rc;
        const CompF* recs = static_cast<const CompF*>(scratch);
        float2* out = static_cast<float2*>(vis);
        kg<<<grid, NT, smem, s>>>(recs, n_comp, bound, uvw, n_vis, out, static_cast<float>(sign), status);
        WT_CUDA_TRY(cudaGetLastError());
        ke<<<grid_e, NT, smem, s>>>(recs, n_comp, bound, uvw, n_vis, out, static_cast<float>(sign), status);
    }
    WT_CUDA_TRY(cudaGetLastError());
    return WT_OK;
}

// The exact pass of the mixed fast direct sum over 128-visibility tiles
// (64 threads, two visibilities each): only the tiles whose first
// visibility carries kDeferredMark are evaluated (the tensor-core form's
// tiles beyond its range).
int dft_exact_pass_128(const void* recs, const uint32_t* bound, int64_t n_comp, const double* uvw, int64_t n_vis,
                       float2* vis, int sign, int* status, cudaStream_t s)
{
    constexpr int NT = 64;
    const size_t smem = static_cast<size_t>(stager_bytes<CompF>(kChunk));
    auto ke = k_dft_mixed<NT, true, false>;
    dim3 grid;
    int rc = grid_for(ke, NT, 2 * NT, smem, n_vis, grid);
    if (rc) return rc;
    ke<<<grid, NT, smem, s>>>(static_cast<const CompF*>(recs), n_comp, bound, uvw, n_vis, vis,
                              static_cast<float>(sign), status);
    WT_CUDA_TRY(cudaGetLastError());
    return WT_OK;
}

// Pack the components into `scratch` and, for the float forms, zero and
// reduce their coordinate bounds at `bound` (16 bytes, 16-byte aligned).
int dft_pack(const double* l, const double* m, const double* flux, int64_t n_comp, void* scratch, uint32_t* bound,
             int mode, int* status, cudaStream_t s)
{
    const bool f64 = mode == WT_FP64;
    if (!f64) WT_CUDA_TRY(cudaMemsetAsync(bound, 0, 4 * sizeof(uint32_t), s));
    if (n_comp == 0) return WT_OK;
    const int tb = 256;
    k_pack_components<<<static_cast<unsigned>((n_comp + tb - 1) / tb), tb, 0, s>>>(
        l, m, flux, n_comp, f64 ? static_cast<CompD*>(scratch) : nullptr, f64 ? nullptr : static_cast<CompF*>(scratch),
        f64 ? nullptr : bound, status);
    WT_CUDA_TRY(cudaGetLastError());
    return WT_OK;
}

int predict_dft(const double* l, const double* m, const double* flux, int64_t n_comp, const double* uvw,
                int64_t n_vis, void* vis, int mode, int sign, cudaStream_t s)
{
    if (n_vis == 0) return WT_OK;
    // 32-byte records (a 16-byte multiple, as the bulk copies need), then
    // the 16-byte block of coordinate bounds; the tensor-core form's slices
    // after them
    const bool tc = mode == WT_MIXED_TC;
    const size_t rec_bytes = ((static_cast<size_t>(n_comp > 0 ? n_comp : 1) * 32 + 255) / 256) * 256;
    const size_t bytes = rec_bytes + 256 + (tc ? dft_tc_scratch_bytes(n_comp) : 0);
    void* scratch = nullptr;
    cudaError_t e = cudaMallocAsync(&scratch, bytes, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(WT_ERR_NOMEM, "dft_predict_vis: scratch allocation of %zu bytes failed: %s", bytes,
                         cudaGetErrorString(e));
    }
    uint32_t* bound = reinterpret_cast<uint32_t*>(static_cast<unsigned char*>(scratch) + rec_bytes);
    int* status = device_status_word();
    if (!status) {
        cudaFreeAsync(scratch, s);
        return set_error(WT_ERR_CUDA, "dft_predict_vis: no device status word");
    }
    int rc = dft_pack(l, m, flux, n_comp, scratch, bound, tc ? WT_MIXED_FAST : mode, status, s);
    if (rc == WT_OK) {
        if (tc)
            rc = dft_tc_launch(l, m, flux, n_comp, scratch, bound, static_cast<unsigned char*>(scratch) + rec_bytes + 256,
                               uvw, n_vis, static_cast<float2*>(vis), sign, status, s);
        else
            rc = dft_launch_packed(scratch, bound, n_comp, uvw, n_vis, vis, mode, sign, status, s);
    }
    cudaError_t ef = cudaFreeAsync(scratch, s);
    if (rc != WT_OK) return rc;
    if (ef != cudaSuccess) return cuda_error(ef, "cudaFreeAsync");
    return WT_OK;
}

}  // namespace wt

#include <mutex>

// ===========================================================================
// dft_predict_vis_noalloc -- the direct sum without any device allocation.
//
// For callers that must not allocate device memory once they are running:
// an application that reserves its whole device-memory budget up front and
// forbids allocation in its steady state (an allocation there could fail, or
// stall behind the allocator's synchronisation), or a host framework that
// owns every device allocation itself. dft_predict_vis allocates a scratch
// buffer for the packed component records on each call; this variant packs
// them instead into the fixed array below, which lives in the library's
// device image. The paper has no counterpart: it is plumbing, not method.
//
// Every GPU that loads the library holds the array (2 MiB) until the
// process exits. All calls on a device share it and it keeps the previous
// call's records, so two calls whose work overlaps on the GPU (different
// streams, no ordering between them) race on it and give wrong results.
// Nothing in it has to start at zero: each call overwrites the records it
// reads.
// ===========================================================================
namespace wt {
namespace {

constexpr int64_t kNoAllocMaxComponents = 65536;   // 32-byte records: 2 MiB
static_assert(sizeof(CompD) == 32 && sizeof(CompF) == 32, "record size assumed below");

static __device__ __align__(256) unsigned char g_noalloc_records[kNoAllocMaxComponents * 32];
// The records' coordinate bounds (the mixed forms' grid pass).
static __device__ __align__(16) uint32_t g_noalloc_bound[4];
// Where the kernels record errors when the caller passes no status word.
static __device__ int g_noalloc_status_sink;

std::mutex g_noalloc_mu;
void* g_noalloc_addr[64] = {nullptr};
uint32_t* g_noalloc_bnd[64] = {nullptr};
int* g_noalloc_sink[64] = {nullptr};
uint64_t g_noalloc_ctx[64] = {0};   // context ID the addresses belong to

// Device addresses of the three arrays above on the current device. The first
// call on a device looks them up (cudaGetSymbolAddress, with that device
// current), and so does the first call in a new context on it (after
// cudaDeviceReset, say: the module is loaded again and the arrays may move);
// in host code the names are only host-side stand-ins and must never be
// handed to a kernel.
int noalloc_addresses(void** records, uint32_t** bound, int** sink)
{
    int dev = 0;
    WT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return set_error(WT_ERR_CUDA, "device ordinal %d out of range", dev);
    const uint64_t ctx = current_context_id();
    if (ctx == 0) return set_error(WT_ERR_CUDA, "dft_predict_vis_noalloc: no current CUDA context");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev] || g_noalloc_ctx[dev] != ctx) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_records);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(g_noalloc_records)");
        void* q = nullptr;
        e = cudaGetSymbolAddress(&q, g_noalloc_status_sink);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(g_noalloc_status_sink)");
        void* b = nullptr;
        e = cudaGetSymbolAddress(&b, g_noalloc_bound);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(g_noalloc_bound)");
        if (!p || !q || !b) return set_error(WT_ERR_CUDA, "cudaGetSymbolAddress returned a null address");
        g_noalloc_addr[dev] = p;
        g_noalloc_bnd[dev] = static_cast<uint32_t*>(b);
        g_noalloc_sink[dev] = static_cast<int*>(q);
        g_noalloc_ctx[dev] = ctx;
    }
    *records = g_noalloc_addr[dev];
    *bound = g_noalloc_bnd[dev];
    *sink = g_noalloc_sink[dev];
    return WT_OK;
}

}  // namespace

}  // namespace wt

extern "C" int dft_predict_vis_noalloc(const double* l, const double* m, const double* flux, int64_t n_comp,
                                       const double* uvw, int64_t n_vis, void* vis_out, int mode, int sign,
                                       int* status, void* stream)
{
    using namespace wt;
    const char* fn = "dft_predict_vis_noalloc";
    if (n_comp < 0 || n_vis < 0) return set_error(WT_ERR_ARG, "%s: negative size", fn);
    if (n_comp > kNoAllocMaxComponents)
        return set_error(WT_ERR_RANGE, "%s: %lld components exceed the fixed capacity of %lld", fn,
                         static_cast<long long>(n_comp), static_cast<long long>(kNoAllocMaxComponents));
    if (sign != 1 && sign != -1) return set_error(WT_ERR_ARG, "%s: sign must be +1 or -1", fn);
    if (mode != WT_FP64 && mode != WT_FP64_DF && mode != WT_MIXED && mode != WT_MIXED_FAST)
        return set_error(WT_ERR_ARG, "%s: bad mode %d", fn, mode);
    const bool c128 = mode == WT_FP64 || mode == WT_FP64_DF;
    const size_t nb = static_cast<size_t>(n_comp) * 8;
    const size_t ob = static_cast<size_t>(n_vis) * (c128 ? 16 : 8);
    int rc;
    if ((rc = check_device_buffer(l, nb, fn, "l", 8)) || (rc = check_device_buffer(m, nb, fn, "m", 8)) ||
        (rc = check_device_buffer(flux, nb, fn, "flux", 8)) ||
        (rc = check_device_buffer(uvw, static_cast<size_t>(n_vis) * 24, fn, "uvw", 8)) ||
        (rc = check_device_buffer(vis_out, ob, fn, "vis_out", vis_align(mode))) ||
        (status && (rc = check_device_buffer(status, sizeof(int), fn, "status", 4))))
        return rc;
    void* records = nullptr;
    uint32_t* bound = nullptr;
    int* sink = nullptr;
    if ((rc = noalloc_addresses(&records, &bound, &sink))) return rc;
    if (!status) status = sink;
    if (n_vis == 0) return WT_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if ((rc = dft_pack(l, m, flux, n_comp, records, bound, mode, status, s))) return rc;
    return dft_launch_packed(records, bound, n_comp, uvw, n_vis, vis_out, mode, sign, status, s);
}

// ===========================================================================
// wt_selftest_context_reset -- the per-context caches across a context reset.
//
// One component of flux 3 at the phase centre (so that V = 3 exactly for
// every baseline in float64) through dft_predict_vis_noalloc with no status
// word (the library's sink) and a read of the device status word; then
// cudaDeviceReset, which ends this process's context on the device and with
// it every device allocation; then the same again in the new context, with
// buffers allocated afresh. Both rounds must give V = 3 + 0i and a clear
// status word, which they can only if the array addresses and the status
// word were looked up again for the new context.
// ===========================================================================
namespace wt {
namespace {

int noalloc_round(cudaStream_t s)
{
    // one allocation: l, m, flux at d[0..2], uvw at d[3..8], the two
    // complex128 outputs at d[10..13] (16-byte aligned, as the kernel's
    // stores need)
    const double l = 0.0, m = 0.0, flux = 3.0;
    const double uvw[6] = {1234.5, -987.25, 12.5, -3.0e4, 2.0e4, -150.0};
    double* d = nullptr;
    WT_CUDA_TRY(cudaMalloc(&d, sizeof(double) * 14));
    double out[4] = {0, 0, 0, 0};
    int rc = WT_OK;
    cudaError_t e = cudaMemcpy(d, &l, sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d + 1, &m, sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d + 2, &flux, sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d + 3, uvw, sizeof(uvw), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) rc = cuda_error(e, "wt_selftest_context_reset: upload");
    if (rc == WT_OK)
        rc = dft_predict_vis_noalloc(d, d + 1, d + 2, 1, d + 3, 2, d + 10, WT_FP64, 1, nullptr, s);
    if (rc == WT_OK) {
        e = cudaMemcpyAsync(out, d + 10, sizeof(out), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_error(e, "wt_selftest_context_reset: download");
    }
    cudaFree(d);
    if (rc != WT_OK) return rc;
    if (out[0] != 3.0 || out[1] != 0.0 || out[2] != 3.0 || out[3] != 0.0)
        return set_error(WT_ERR_CORRUPT, "wt_selftest_context_reset: V = (%g, %g), (%g, %g), expected (3, 0)", out[0],
                         out[1], out[2], out[3]);
    return wt_device_status(s);
}

}  // namespace
}  // namespace wt

extern "C" int wt_selftest_context_reset(void)
{
    using namespace wt;
    int rc = noalloc_round(nullptr);
    if (rc != WT_OK) return rc;
    WT_CUDA_TRY(cudaDeviceReset());
    return noalloc_round(nullptr);
}
