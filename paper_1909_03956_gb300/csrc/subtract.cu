// subtract.cu -- subtract_model: V_resid = V - V_M (Sec. 2.2, major-cycle
// step 2), element by element. Pure streaming: 16-byte vector loads and
// stores, a grid-stride loop sized to the SMs. HBM-bound by design.
#include "wt_internal.cuh"

namespace wt {
namespace {

// complex128: one double2 per visibility
__global__ void k_subtract_c128(const double2* a, const double2* __restrict__ b, double2* r, int64_t n)
{
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const double2 x = a[i], y = b[i];
        r[i] = make_double2(x.x - y.x, x.y - y.y);
    }
}

// complex64: two visibilities per float4, plus a scalar tail
__global__ void k_subtract_c64(const float4* a, const float4* __restrict__ b, float4* r, int64_t npairs,
                               const float2* a2, const float2* __restrict__ b2, float2* r2, int64_t n)
{
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < npairs;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const float4 x = a[i], y = b[i];
        r[i] = make_float4(x.x - y.x, x.y - y.y, x.z - y.z, x.w - y.w);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && (n & 1)) {
        const float2 x = a2[n - 1], y = b2[n - 1];
        r2[n - 1] = make_float2(x.x - y.x, x.y - y.y);
    }
}

// complex64 views without 16-byte alignment
__global__ void k_subtract_c64_scalar(const float2* a, const float2* __restrict__ b, float2* r, int64_t n)
{
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const float2 x = a[i], y = b[i];
        r[i] = make_float2(x.x - y.x, x.y - y.y);
    }
}

}  // namespace

int subtract(const void* obs, const void* model, void* resid, int64_t n_vis, int mode, cudaStream_t s)
{
    if (n_vis == 0) return WT_OK;
    const int tb = 256;
    const int64_t blocks_max = static_cast<int64_t>(num_sms()) * 8;
    if (mode == WT_FP64) {
        int64_t blocks = (n_vis + tb - 1) / tb;
        if (blocks > blocks_max) blocks = blocks_max;
        k_subtract_c128<<<static_cast<unsigned>(blocks), tb, 0, s>>>(static_cast<const double2*>(obs),
                                                                     static_cast<const double2*>(model),
                                                                     static_cast<double2*>(resid), n_vis);
    } else {
        const bool aligned = ((reinterpret_cast<uintptr_t>(obs) | reinterpret_cast<uintptr_t>(model) |
                               reinterpret_cast<uintptr_t>(resid)) & 15u) == 0;
        const int64_t npairs = aligned ? n_vis / 2 : 0;
        int64_t blocks = (npairs + tb - 1) / tb;
        if (blocks > blocks_max) blocks = blocks_max;
        if (blocks < 1) blocks = 1;
        if (aligned) {
            k_subtract_c64<<<static_cast<unsigned>(blocks), tb, 0, s>>>(
                static_cast<const float4*>(obs), static_cast<const float4*>(model), static_cast<float4*>(resid),
                npairs, static_cast<const float2*>(obs), static_cast<const float2*>(model),
                static_cast<float2*>(resid), n_vis);
        } else {
            int64_t b2 = (n_vis + tb - 1) / tb;
            if (b2 > blocks_max) b2 = blocks_max;
            k_subtract_c64_scalar<<<static_cast<unsigned>(b2), tb, 0, s>>>(
                static_cast<const float2*>(obs), static_cast<const float2*>(model), static_cast<float2*>(resid), n_vis);
        }
    }
    WT_CUDA_TRY(cudaGetLastError());
    return WT_OK;
}

}  // namespace wt
