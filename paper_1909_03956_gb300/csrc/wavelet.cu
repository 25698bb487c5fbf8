// wavelet.cu -- wt_predict_vis: per-visibility plane-wave coefficients on
// the coefficient tree and the multiresolution sum (Sec. 3.3, Eqs. 14, 16,
// 17; per-visibility steps of Sec. 3.6.1).
//
// Mapping to the GPU. One thread owns one visibility; a CTA owns a tile of
// NT visibilities and walks the whole tree for them. The tree is the same
// for every visibility, so the walk is uniform across the CTA: the node
// records (post-order, built once per major cycle) are streamed through
// shared memory by bulk copies and read as broadcasts. Post-order visits
// every child before its parent, so each node's plane-wave coefficient
// eta_j,k is produced exactly when its parent needs it. A thread keeps, per
// level j = 2..J, the four child slots of the currently open parent in a
// shared-memory column of its own ([level][slot][thread]: conflict-free).
// Nothing per visibility is ever written to global memory except V.
//
// Forms:
//   WT_FP64   float64 throughout; sin/cos from sincospi.
//   WT_MIXED  phase in double-float turns (float64-accurate), sin/cos of the
//             reduced phase in float32 (Taylor series, wt_internal.cuh),
//             recursion in float32, Kahan-compensated float32 V.
#include "staging.cuh"
#include "wt_internal.cuh"

namespace wt {
namespace {

__constant__ double c_qd[kMaxJ + 1];   // sqrt(A_j) / 4
__constant__ float c_qf[kMaxJ + 1];

constexpr int kChunk = 256;

template <int NT>
__device__ __forceinline__ double2* stack_slot_d(double2* stk, int level, int slot)
{
    return stk + (static_cast<int64_t>(level - 2) * 4 + slot) * NT + threadIdx.x;
}

template <int NT>
__device__ __forceinline__ float2* stack_slot_f(float2* stk, int level, int slot)
{
    return stk + (static_cast<int64_t>(level - 2) * 4 + slot) * NT + threadIdx.x;
}

// ---------------------------------------------------------------- FP64 body
// A record whose level or leaf flag does not fit the tree's depth is
// skipped (and reported), so that no stack slot outside [2, J] is touched.
__device__ __forceinline__ bool record_fits(uint32_t meta, int J)
{
    const int lev = static_cast<int>(rec_level(meta));
    return lev >= 1 && lev <= J && (rec_leaf(meta) != 0) == (lev == J);
}

template <int NT>
struct BodyEq17D {
    double u, v, w;
    double sgn;
    double vr, vi;
    double2* stk;
    int J;
    int bad;
    __device__ void operator()(const RecD& r)
    {
        const uint32_t meta = r.meta;
        if (!record_fits(meta, J)) {
            bad = 1;
            return;
        }
        const int lev = static_cast<int>(rec_level(meta));
        double er, ei;
        if (rec_leaf(meta)) {
            // Eq. 14 at the pixel centre: t = u s_u + v s_v + w (s_w - 1) turns
            double t = fma(w, r.c, fma(v, r.b, u * r.a));
            t -= rint(t);
            double s, c;
            sincospi(2.0 * t, &s, &c);
            er = c;
            ei = sgn * s;
        } else {
            const uint32_t mask = rec_mask(meta);
            double2 c0 = make_double2(0.0, 0.0), c1 = c0, c2 = c0, c3 = c0;
            if (mask & 1u) c0 = *stack_slot_d<NT>(stk, lev + 1, 0);
            if (mask & 2u) c1 = *stack_slot_d<NT>(stk, lev + 1, 1);
            if (mask & 4u) c2 = *stack_slot_d<NT>(stk, lev + 1, 2);
            if (mask & 8u) c3 = *stack_slot_d<NT>(stk, lev + 1, 3);
            // Eq. 9 form for eta, Eq. 10 form for sigma (absent child = 0)
            const double ar = c0.x + c1.x, ai = c0.y + c1.y;   // c0 + c1
            const double br = c0.x - c1.x, bi = c0.y - c1.y;   // c0 - c1
            const double cr = c2.x + c3.x, ci = c2.y + c3.y;   // c2 + c3
            const double dr = c2.x - c3.x, di = c2.y - c3.y;   // c2 - c3
            er = 0.25 * (ar + cr);
            ei = 0.25 * (ai + ci);
            const double q = c_qd[lev];
            const double s0r = q * (br + dr), s0i = q * (bi + di);   // + - + -
            const double s1r = q * (ar - cr), s1i = q * (ai - ci);   // + + - -
            const double s2r = q * (br - dr), s2i = q * (bi - di);   // + - - +
            vr = fma(r.a, s0r, fma(r.b, s1r, fma(r.c, s2r, vr)));
            vi = fma(r.a, s0i, fma(r.b, s1i, fma(r.c, s2i, vi)));
        }
        if (lev == 1) {
            // A_1 lambda_1 eta_1 (internal) or Phi eta (a level-1 leaf, J = 1)
            vr = fma(r.d, er, vr);
            vi = fma(r.d, ei, vi);
        } else {
            *stack_slot_d<NT>(stk, lev, static_cast<int>(rec_slot(meta))) = make_double2(er, ei);
        }
    }
};

// Eq. 16: V = sum_k Phi_k eta_J,k over the leaf records.
struct BodyEq16D {
    double u, v, w;
    double sgn;
    double vr, vi;
    __device__ void operator()(const RecD& r)
    {
        double t = fma(w, r.c, fma(v, r.b, u * r.a));
        t -= rint(t);
        double s, c;
        sincospi(2.0 * t, &s, &c);
        vr = fma(r.d, c, vr);
        vi = fma(r.d, sgn * s, vi);
    }
};

// ---------------------------------------------------------------- mixed body
template <int NT>
struct BodyEq17F {
    F2 u, v, w;
    float sgn;
    float vr, vi, cr_, ci_;   // Kahan sums and compensations
    float2* stk;
    int J;
    int bad;
    __device__ void operator()(const RecF& r)
    {
        const uint32_t meta = r.meta;
        if (!record_fits(meta, J)) {
            bad = 1;
            return;
        }
        const int lev = static_cast<int>(rec_level(meta));
        float er, ei;
        float xr = 0.0f, xi = 0.0f;
        if (rec_leaf(meta)) {
            float th, tl;
            phase_turns_df(u, v, w, F2{r.a, r.b}, F2{r.c, r.d}, F2{r.e, r.f}, th, tl);
            float s, c;
            sincos_turns_f32(th, tl, s, c);
            er = c;
            ei = sgn * s;
        } else {
            const uint32_t mask = rec_mask(meta);
            float2 c0 = make_float2(0.f, 0.f), c1 = c0, c2 = c0, c3 = c0;
            if (mask & 1u) c0 = *stack_slot_f<NT>(stk, lev + 1, 0);
            if (mask & 2u) c1 = *stack_slot_f<NT>(stk, lev + 1, 1);
            if (mask & 4u) c2 = *stack_slot_f<NT>(stk, lev + 1, 2);
            if (mask & 8u) c3 = *stack_slot_f<NT>(stk, lev + 1, 3);
            const float ar = c0.x + c1.x, ai = c0.y + c1.y;
            const float br = c0.x - c1.x, bi = c0.y - c1.y;
            const float cr = c2.x + c3.x, ci = c2.y + c3.y;
            const float dr = c2.x - c3.x, di = c2.y - c3.y;
            er = 0.25f * (ar + cr);
            ei = 0.25f * (ai + ci);
            const float q = c_qf[lev];
            const float s0r = q * (br + dr), s0i = q * (bi + di);
            const float s1r = q * (ar - cr), s1i = q * (ai - ci);
            const float s2r = q * (br - dr), s2i = q * (bi - di);
            xr = fmaf(r.a, s0r, fmaf(r.b, s1r, r.c * s2r));
            xi = fmaf(r.a, s0i, fmaf(r.b, s1i, r.c * s2i));
        }
        if (lev == 1) {
            xr = fmaf(r.g, er, xr);
            xi = fmaf(r.g, ei, xi);
        } else {
            *stack_slot_f<NT>(stk, lev, static_cast<int>(rec_slot(meta))) = make_float2(er, ei);
        }
        if (!rec_leaf(meta) || lev == 1) {
            kahan_add(vr, cr_, xr);
            kahan_add(vi, ci_, xi);
        }
    }
};

struct BodyEq16F {
    F2 u, v, w;
    float sgn;
    float vr, vi, cr_, ci_;
    __device__ void operator()(const RecF& r)
    {
        float th, tl;
        phase_turns_df(u, v, w, F2{r.a, r.b}, F2{r.c, r.d}, F2{r.e, r.f}, th, tl);
        float s, c;
        sincos_turns_f32(th, tl, s, c);
        kahan_add(vr, cr_, r.g * c);
        kahan_add(vi, ci_, r.g * (sgn * s));
    }
};

// ---------------------------------------------------------------- kernels
template <int NT, bool EQ16>
__global__ void __launch_bounds__(NT) k_wavelet_fp64(const RecD* __restrict__ recs, const TreeHeader* __restrict__ hdr,
                                                     const double* __restrict__ uvw, int64_t n_vis,
                                                     double2* __restrict__ vis, double sgn, int J, int* status)
{
    extern __shared__ __align__(16) unsigned char smem[];
    Stager<RecD> st;
    const int64_t count = EQ16 ? hdr->n_leaves : hdr->n_nodes;
    stager_setup(st, smem, recs, count, kChunk);
    double2* stk = reinterpret_cast<double2*>(smem + stager_bytes<RecD>(kChunk));
    const int64_t ntiles = (n_vis + NT - 1) / NT;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t n = tile * NT + threadIdx.x;
        const bool valid = n < n_vis;
        const double u = valid ? uvw[3 * n] : 0.0, v = valid ? uvw[3 * n + 1] : 0.0, w = valid ? uvw[3 * n + 2] : 0.0;
        double vr, vi;
        bool ok;
        if (EQ16) {
            BodyEq16D body{u, v, w, sgn, 0.0, 0.0};
            ok = st.sweep(body);
            vr = body.vr;
            vi = body.vi;
        } else {
            BodyEq17D<NT> body{u, v, w, sgn, 0.0, 0.0, stk, J, 0};
            ok = st.sweep(body);
            vr = body.vr;
            vi = body.vi;
            if (body.bad) record_status(status, WT_ERR_CORRUPT);
        }
        if (!ok) {
            if (threadIdx.x == 0) record_status(status, WT_ERR_TIMEOUT);
            return;
        }
        if (valid) vis[n] = make_double2(vr, vi);
    }
}

template <int NT, bool EQ16>
__global__ void __launch_bounds__(NT) k_wavelet_mixed(const RecF* __restrict__ recs, const TreeHeader* __restrict__ hdr,
                                                      const double* __restrict__ uvw, int64_t n_vis,
                                                      float2* __restrict__ vis, float sgn, int J, int* status)
{
    extern __shared__ __align__(16) unsigned char smem[];
    Stager<RecF> st;
    const int64_t count = EQ16 ? hdr->n_leaves : hdr->n_nodes;
    stager_setup(st, smem, recs, count, kChunk);
    float2* stk = reinterpret_cast<float2*>(smem + stager_bytes<RecF>(kChunk));
    const int64_t ntiles = (n_vis + NT - 1) / NT;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t n = tile * NT + threadIdx.x;
        const bool valid = n < n_vis;
        const double u = valid ? uvw[3 * n] : 0.0, v = valid ? uvw[3 * n + 1] : 0.0, w = valid ? uvw[3 * n + 2] : 0.0;
        const F2 U = split_f64(u), V = split_f64(v), W = split_f64(w);
        float vr, vi, cr, ci;
        bool ok;
        if (EQ16) {
            BodyEq16F body{U, V, W, sgn, 0.f, 0.f, 0.f, 0.f};
            ok = st.sweep(body);
            vr = body.vr; vi = body.vi; cr = body.cr_; ci = body.ci_;
        } else {
            BodyEq17F<NT> body{U, V, W, sgn, 0.f, 0.f, 0.f, 0.f, stk, J, 0};
            ok = st.sweep(body);
            vr = body.vr; vi = body.vi; cr = body.cr_; ci = body.ci_;
            if (body.bad) record_status(status, WT_ERR_CORRUPT);
        }
        if (!ok) {
            if (threadIdx.x == 0) record_status(status, WT_ERR_TIMEOUT);
            return;
        }
        if (valid) vis[n] = make_float2(vr - cr, vi - ci);
    }
}

bool g_const_ready[64] = {false};

int ensure_constants()
{
    int dev = 0;
    WT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 64 && g_const_ready[dev]) return WT_OK;
    double qd[kMaxJ + 1];
    float qf[kMaxJ + 1];
    for (int j = 0; j <= kMaxJ; ++j) {
        qd[j] = (j == 0) ? 0.0 : ldexp(sqrt(kPi / 3.0), 1 - j) * 0.25;
        qf[j] = static_cast<float>(qd[j]);
    }
    WT_CUDA_TRY(cudaMemcpyToSymbol(c_qd, qd, sizeof(qd)));
    WT_CUDA_TRY(cudaMemcpyToSymbol(c_qf, qf, sizeof(qf)));
    if (dev < 64) g_const_ready[dev] = true;
    return WT_OK;
}

template <class K>
int launch_persistent(K kernel, int nt, size_t smem, int64_t n_vis, cudaStream_t s, dim3& grid_out)
{
    WT_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
    int per_sm = 0;
    WT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, nt, smem));
    if (per_sm < 1) return set_error(WT_ERR_UNSUPPORTED, "wavelet kernel does not fit on an SM (smem %zu)", smem);
    const int64_t ntiles = (n_vis + nt - 1) / nt;
    int64_t grid = static_cast<int64_t>(num_sms()) * per_sm;
    if (grid > ntiles) grid = ntiles;
    grid_out = dim3(static_cast<unsigned>(grid));
    return WT_OK;
}

template <int NT>
int run_fp64(wt_tree t, const double* uvw, int64_t n_vis, void* vis, int sign, int which, cudaStream_t s)
{
    const size_t stack = (which == WT_SUM_EQ16) ? 0 : static_cast<size_t>(t->J > 1 ? t->J - 1 : 1) * 4 * NT * sizeof(double2);
    const size_t smem = static_cast<size_t>(stager_bytes<RecD>(kChunk)) + stack;
    int* status = device_status_word();
    dim3 grid;
    if (which == WT_SUM_EQ16) {
        auto k = k_wavelet_fp64<NT, true>;
        int rc = launch_persistent(k, NT, smem, n_vis, s, grid);
        if (rc) return rc;
        k<<<grid, NT, smem, s>>>(t->d.leafd, t->d.hdr, uvw, n_vis, static_cast<double2*>(vis), sign, t->J, status);
    } else {
        auto k = k_wavelet_fp64<NT, false>;
        int rc = launch_persistent(k, NT, smem, n_vis, s, grid);
        if (rc) return rc;
        k<<<grid, NT, smem, s>>>(t->d.recd, t->d.hdr, uvw, n_vis, static_cast<double2*>(vis), sign, t->J, status);
    }
    WT_CUDA_TRY(cudaGetLastError());
    return WT_OK;
}

template <int NT>
int run_mixed(wt_tree t, const double* uvw, int64_t n_vis, void* vis, int sign, int which, cudaStream_t s)
{
    const size_t stack = (which == WT_SUM_EQ16) ? 0 : static_cast<size_t>(t->J > 1 ? t->J - 1 : 1) * 4 * NT * sizeof(float2);
    const size_t smem = static_cast<size_t>(stager_bytes<RecF>(kChunk)) + stack;
    int* status = device_status_word();
    dim3 grid;
    if (which == WT_SUM_EQ16) {
        auto k = k_wavelet_mixed<NT, true>;
        int rc = launch_persistent(k, NT, smem, n_vis, s, grid);
        if (rc) return rc;
        k<<<grid, NT, smem, s>>>(t->d.leaff, t->d.hdr, uvw, n_vis, static_cast<float2*>(vis), static_cast<float>(sign),
                                 t->J, status);
    } else {
        auto k = k_wavelet_mixed<NT, false>;
        int rc = launch_persistent(k, NT, smem, n_vis, s, grid);
        if (rc) return rc;
        k<<<grid, NT, smem, s>>>(t->d.recf, t->d.hdr, uvw, n_vis, static_cast<float2*>(vis), static_cast<float>(sign),
                                 t->J, status);
    }
    WT_CUDA_TRY(cudaGetLastError());
    return WT_OK;
}

}  // namespace

int predict_wavelet(wt_tree t, const double* uvw, int64_t n_vis, void* vis, int mode, int sign, int which,
                    cudaStream_t s)
{
    if (n_vis == 0) return WT_OK;
    int rc = ensure_constants();
    if (rc) return rc;
    const int levels = t->J > 1 ? t->J - 1 : 1;
    if (mode == WT_FP64) {
        // per-thread stack: levels * 4 * 16 bytes; keep it under ~160 KB per CTA
        const size_t per_thread = static_cast<size_t>(levels) * 4 * sizeof(double2);
        if (which == WT_SUM_EQ16 || per_thread * 128 <= 160 * 1024) return run_fp64<128>(t, uvw, n_vis, vis, sign, which, s);
        return run_fp64<64>(t, uvw, n_vis, vis, sign, which, s);
    }
    const size_t per_thread = static_cast<size_t>(levels) * 4 * sizeof(float2);
    if (which == WT_SUM_EQ16 || per_thread * 256 <= 160 * 1024) return run_mixed<256>(t, uvw, n_vis, vis, sign, which, s);
    if (per_thread * 128 <= 160 * 1024) return run_mixed<128>(t, uvw, n_vis, vis, sign, which, s);
    return run_mixed<64>(t, uvw, n_vis, vis, sign, which, s);
}

}  // namespace wt
