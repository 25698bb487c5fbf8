// probe.cu -- wt_measure_pipe_rates: the issue rates of the arithmetic pipes
// the predictors run on, measured on the current device. They are the
// denominators of the predictors' rooflines: the float32 FMA pipe (scalar
// and packed-pair FMA), the float64 FMA pipe and the special-function unit
// (sine).
//
// One CTA of 512 threads per SM (a shared-memory request larger than half an
// SM's keeps every CTA alone on its SM), each thread running eight
// independent dependency chains of one operation, so that the pipe, not the
// chains' latency, sets the rate. Each CTA times its loop with its own SM's
// cycle counter (clock64); the rate per SM per clock is the operations
// (elements, for packed pairs) issued by the CTA over its cycles, and the
// median over the SMs is reported.
#include <algorithm>
#include <vector>

#include <cuda_bf16.h>

#include "wt_internal.cuh"

namespace wt {
namespace {

constexpr int kProbeThreads = 512;
constexpr int kProbeChains = 8;
constexpr size_t kProbeSmem = 150 * 1024;   // > half of an SM's shared memory: one CTA per SM

enum ProbeKind {
    kFfma = 0,
    kFfma2 = 1,
    kDfma = 2,
    kMufuSin = 3,
    kMufuTanh = 4,
    kMufuTanhBf16x2 = 5,
    kMufuEx2 = 6,
    kNumProbes = 7
};

template <int KIND>
__global__ void __launch_bounds__(kProbeThreads) k_pipe_probe(int iters, float b, float c, float* sink,
                                                              long long* cycles)
{
    extern __shared__ unsigned char keep_one_cta_per_sm[];
    (void)keep_one_cta_per_sm;
    const float x0 = 1e-3f * static_cast<float>(threadIdx.x & 63);
    float acc = 0.0f;
    __syncthreads();
    const long long t0 = clock64();
    if constexpr (KIND == kFfma) {
        float a[kProbeChains];
#pragma unroll
        for (int r = 0; r < kProbeChains; ++r) a[r] = x0 + r;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int r = 0; r < kProbeChains; ++r) a[r] = __fmaf_rn(a[r], b, c);
        }
#pragma unroll
        for (int r = 0; r < kProbeChains; ++r) acc += a[r];
    } else if constexpr (KIND == kFfma2) {
        float2 a[kProbeChains];
        const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
#pragma unroll
        for (int r = 0; r < kProbeChains; ++r) a[r] = make_float2(x0 + r, x0 - r);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int r = 0; r < kProbeChains; ++r) a[r] = __ffma2_rn(a[r], b2, c2);
        }
#pragma unroll
        for (int r = 0; r < kProbeChains; ++r) acc += a[r].x + a[r].y;
    } else if constexpr (KIND == kDfma) {
        double a[kProbeChains];
        const double bd = b, cd = c;
#pragma unroll
        for (int r = 0; r < kProbeChains; ++r) a[r] = x0 + r;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int r = 0; r < kProbeChains; ++r) a[r] = fma(a[r], bd, cd);
        }
#pragma unroll
        for (int r = 0; r < kProbeChains; ++r) acc += static_cast<float>(a[r]);
    } else if constexpr (KIND == kMufuSin) {
        float a[kProbeChains];
#pragma unroll
        for (int r = 0; r < kProbeChains; ++r) a[r] = x0 + 0.1f * r;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int r = 0; r < kProbeChains; ++r) a[r] = __sinf(a[r]);
        }
#pragma unroll
        for (int r = 0; r < kProbeChains; ++r) acc += a[r];
    } else if constexpr (KIND == kMufuTanh) {
        float a[kProbeChains];
#pragma unroll
        for (int r = 0; r < kProbeChains; ++r) a[r] = x0 + 0.1f * r;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int r = 0; r < kProbeChains; ++r) asm volatile("tanh.approx.f32 %0, %0;" : "+f"(a[r]));
        }
#pragma unroll
        for (int r = 0; r < kProbeChains; ++r) acc += a[r];
    } else if constexpr (KIND == kMufuTanhBf16x2) {
        uint32_t a[kProbeChains];
#pragma unroll
        for (int r = 0; r < kProbeChains; ++r) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(x0 + 0.1f * r, x0 - 0.1f * r);
            a[r] = *reinterpret_cast<const uint32_t*>(&h);
        }
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int r = 0; r < kProbeChains; ++r) asm volatile("tanh.approx.bf16x2 %0, %0;" : "+r"(a[r]));
        }
#pragma unroll
        for (int r = 0; r < kProbeChains; ++r) acc += __uint_as_float(a[r] << 16) + __uint_as_float(a[r] & 0xffff0000u);
    } else {
        float a[kProbeChains];
#pragma unroll
        for (int r = 0; r < kProbeChains; ++r) a[r] = -1e-3f * r;
        for (int i = 0; i < iters; ++i) {   // 2^x of a non-positive x stays in (0, 1]: no overflow
#pragma unroll
            for (int r = 0; r < kProbeChains; ++r) asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(a[r]));
#pragma unroll
            for (int r = 0; r < kProbeChains; ++r) a[r] = -a[r];
        }
#pragma unroll
        for (int r = 0; r < kProbeChains; ++r) acc += a[r];
    }
    __syncthreads();
    const long long t1 = clock64();
    sink[static_cast<int64_t>(blockIdx.x) * kProbeThreads + threadIdx.x] = acc;
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

template <int KIND>
int run_probe(int iters, int n_sm, float* sink, long long* cycles, cudaStream_t s)
{
    auto k = k_pipe_probe<KIND>;
    WT_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(kProbeSmem)));
    k<<<n_sm, kProbeThreads, kProbeSmem, s>>>(iters, 0.999f, 1e-3f, sink, cycles);
    WT_CUDA_TRY(cudaGetLastError());
    return WT_OK;
}

}  // namespace
}  // namespace wt

extern "C" int wt_measure_pipe_rates(double* per_clk_per_sm, void* stream)
{
    using namespace wt;
    if (!per_clk_per_sm) return set_error(WT_ERR_ARG, "wt_measure_pipe_rates: null output");
    const int n_sm = num_sms();
    if (n_sm <= 0) return set_error(WT_ERR_CUDA, "wt_measure_pipe_rates: no usable CUDA device");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float* sink = nullptr;
    long long* cyc = nullptr;
    WT_CUDA_TRY(cudaMallocAsync(&sink, sizeof(float) * kProbeThreads * n_sm, s));
    WT_CUDA_TRY(cudaMallocAsync(&cyc, sizeof(long long) * kNumProbes * n_sm, s));
    // iterations per kind: about a millisecond each at the expected rates
    const int iters[kNumProbes] = {40000, 20000, 1000, 5000, 5000, 5000, 5000};
    const double elems[kNumProbes] = {1.0, 2.0, 1.0, 1.0, 1.0, 2.0, 1.0};
    int rc = WT_OK;
    for (int rep = 0; rep < 2 && rc == WT_OK; ++rep) {   // the first pass warms the clocks up
        if (!rc) rc = run_probe<kFfma>(iters[kFfma], n_sm, sink, cyc + kFfma * n_sm, s);
        if (!rc) rc = run_probe<kFfma2>(iters[kFfma2], n_sm, sink, cyc + kFfma2 * n_sm, s);
        if (!rc) rc = run_probe<kDfma>(iters[kDfma], n_sm, sink, cyc + kDfma * n_sm, s);
        if (!rc) rc = run_probe<kMufuSin>(iters[kMufuSin], n_sm, sink, cyc + kMufuSin * n_sm, s);
        if (!rc) rc = run_probe<kMufuTanh>(iters[kMufuTanh], n_sm, sink, cyc + kMufuTanh * n_sm, s);
        if (!rc)
            rc = run_probe<kMufuTanhBf16x2>(iters[kMufuTanhBf16x2], n_sm, sink, cyc + kMufuTanhBf16x2 * n_sm, s);
        if (!rc) rc = run_probe<kMufuEx2>(iters[kMufuEx2], n_sm, sink, cyc + kMufuEx2 * n_sm, s);
    }
    std::vector<long long> h(static_cast<size_t>(kNumProbes) * n_sm);
    if (rc == WT_OK) {
        cudaError_t e = cudaMemcpyAsync(h.data(), cyc, h.size() * sizeof(long long), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_error(e, "wt_measure_pipe_rates: read cycles");
    }
    cudaFreeAsync(sink, s);
    cudaFreeAsync(cyc, s);
    if (rc != WT_OK) return rc;
    for (int k = 0; k < kNumProbes; ++k) {
        std::vector<double> r;
        for (int b = 0; b < n_sm; ++b) {
            const long long c = h[static_cast<size_t>(k) * n_sm + b];
            if (c > 0)
                r.push_back(static_cast<double>(kProbeThreads) * kProbeChains * iters[k] * elems[k] /
                            static_cast<double>(c));
        }
        if (r.empty()) return set_error(WT_ERR_CUDA, "wt_measure_pipe_rates: no cycles recorded");
        std::nth_element(r.begin(), r.begin() + r.size() / 2, r.end());
        per_clk_per_sm[k] = r[r.size() / 2];
    }
    return WT_OK;
}
