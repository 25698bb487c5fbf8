// imaging.cu -- the imaging half of the major cycle (Sec. 2.2, the Cotton-
// Schwab steps after Eq. 6) around the model prediction: gridding and FFT
// to a dirty image, Hogbom clean (Eqs. 4-6), and the loop of major cycles.
//
// Conventions (an n x n image, n even, pixel size dl radians):
//   pixel (ix, iy) at l = (ix - n/2) dl, m = (iy - n/2) dl, arrays [iy][ix];
//   uv cell (iu, iv) at u = (iu - n/2) du, v = (iv - n/2) du, du = 1/(n dl).
// Gridding is nearest-cell with unit weights: each visibility and its
// Hermitian conjugate at -B (a visibility whose cell falls outside the grid
// is left out); the w term is not used in imaging (the 2-D transform of
// Eq. 2). The dirty image is (1/W) Re sum_cells G(u, v) exp(-i 2 pi (ul + vm))
// with W the number of gridded entries, so that a unit point source at the
// phase centre images to 1; the dirty beam is the image of unit
// visibilities. Both index shifts of the transform (cell n/2 is u = 0,
// pixel n/2 is l = 0) are applied as (-1)^(iu+iv) on the grid and
// (-1)^(ix+iy) on the image, which is exact for even n.
//
// The 2-D FFT is cuFFT's, loaded at first use (a library call for a plain
// transform); everything else is in the kernels below.
//
// Hogbom clean takes "the pixel with the maximum value" literally (the
// largest value; ties to the first pixel in row-major order), subtracts
// g C times the beam centred there wherever it overlaps the image, and
// stops after max_iter components or when the maximum falls below the
// threshold. The arithmetic is float32 without contraction: fl(g C) and
// fl(I - fl(f B)). Two schedules, identical results:
//   persistent  the whole minor cycle in one cooperative launch: each CTA
//               keeps its rows of the image in shared memory for every
//               iteration, subtracts the pending component there (the beam
//               is read from global memory and stays in L2), and joins a
//               grid-wide maximum of the CTAs' (value, pixel) keys once per
//               iteration, which also serves as the iteration's barrier;
//   per launch  one launch per iteration when the rows do not fit in shared
//               memory: every CTA subtracts the previous component over its
//               pixels and finds its largest updated value; a 64-bit
//               atomicMax picks the winner and the last CTA to finish (an
//               atomic counter, no waiting) records the component for the
//               next launch.
#include <dlfcn.h>
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#include <string.h>

#include <cufft.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "wt_internal.cuh"

namespace wt {
namespace {

// ---------------------------------------------------------------- cuFFT
struct CufftApi {
    bool tried = false;
    void* so = nullptr;
    cufftResult (*plan2d)(cufftHandle*, int, int, cufftType) = nullptr;
    cufftResult (*set_stream)(cufftHandle, cudaStream_t) = nullptr;
    cufftResult (*exec_c2c)(cufftHandle, cufftComplex*, cufftComplex*, int) = nullptr;
    cufftResult (*destroy)(cufftHandle) = nullptr;
};

std::mutex g_fft_mu;
CufftApi g_fft;

struct FftPlan {
    int device, n;
    cufftHandle h;
};
std::vector<FftPlan> g_plans;

int fft_api()
{
    if (g_fft.so) return WT_OK;
    if (g_fft.tried) return set_error(WT_ERR_UNSUPPORTED, "cuFFT (libcufft.so) could not be loaded");
    g_fft.tried = true;
    const char* names[] = {"libcufft.so.12", "libcufft.so", "/usr/local/cuda/lib64/libcufft.so.12"};
    for (const char* nm : names)
        if ((g_fft.so = dlopen(nm, RTLD_NOW | RTLD_LOCAL))) break;
    if (!g_fft.so) return set_error(WT_ERR_UNSUPPORTED, "cuFFT (libcufft.so) could not be loaded");
    g_fft.plan2d = reinterpret_cast<decltype(g_fft.plan2d)>(dlsym(g_fft.so, "cufftPlan2d"));
    g_fft.set_stream = reinterpret_cast<decltype(g_fft.set_stream)>(dlsym(g_fft.so, "cufftSetStream"));
    g_fft.exec_c2c = reinterpret_cast<decltype(g_fft.exec_c2c)>(dlsym(g_fft.so, "cufftExecC2C"));
    g_fft.destroy = reinterpret_cast<decltype(g_fft.destroy)>(dlsym(g_fft.so, "cufftDestroy"));
    if (!g_fft.plan2d || !g_fft.set_stream || !g_fft.exec_c2c || !g_fft.destroy) {
        g_fft.so = nullptr;
        return set_error(WT_ERR_UNSUPPORTED, "cuFFT loaded without the expected entry points");
    }
    return WT_OK;
}

// In-place forward 2-D transform (sign -1) of an n x n complex64 array.
int fft2_forward(float2* data, int n, cudaStream_t s)
{
    std::lock_guard<std::mutex> lk(g_fft_mu);
    int rc = fft_api();
    if (rc) return rc;
    int dev = 0;
    WT_CUDA_TRY(cudaGetDevice(&dev));
    cufftHandle h = 0;
    bool found = false;
    for (const FftPlan& p : g_plans)
        if (p.device == dev && p.n == n) {
            h = p.h;
            found = true;
        }
    if (!found) {
        if (g_fft.plan2d(&h, n, n, CUFFT_C2C) != CUFFT_SUCCESS)
            return set_error(WT_ERR_CUDA, "cufftPlan2d(%d x %d) failed", n, n);
        g_plans.push_back(FftPlan{dev, n, h});
    }
    if (g_fft.set_stream(h, s) != CUFFT_SUCCESS) return set_error(WT_ERR_CUDA, "cufftSetStream failed");
    cufftComplex* d = reinterpret_cast<cufftComplex*>(data);
    if (g_fft.exec_c2c(h, d, d, CUFFT_FORWARD) != CUFFT_SUCCESS) return set_error(WT_ERR_CUDA, "cufftExecC2C failed");
    return WT_OK;
}

// ---------------------------------------------------------------- gridding
constexpr int kImgThreads = 256;

// Visibility n (unit value if vis is null) and its conjugate into their
// cells, times (-1)^(iu+iv) (the index shift); counts the entries.
__global__ void k_grid_nn(const double* __restrict__ uvw, const float2* __restrict__ vis, int64_t n_vis, int n,
                          double inv_du, float2* __restrict__ grid, unsigned long long* __restrict__ count)
{
    __shared__ unsigned int blk;
    if (threadIdx.x == 0) blk = 0;
    __syncthreads();
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n_vis) {
        const double ru = rint(uvw[3 * i] * inv_du), rv = rint(uvw[3 * i + 1] * inv_du);
        const double h = 0.5 * n;
        if (ru > -h && ru < h && rv > -h && rv < h) {
            const int iu = static_cast<int>(ru) + n / 2, iv = static_cast<int>(rv) + n / 2;
            const int ju = n - iu, jv = n - iv;               // the mirrored cell: n/2 - ru
            const float2 V = vis ? vis[i] : make_float2(1.0f, 0.0f);
            const float sg = ((iu + iv) & 1) ? -1.0f : 1.0f;   // (-1)^(ju+jv) is the same: n even
            float* a = reinterpret_cast<float*>(grid + static_cast<int64_t>(iv) * n + iu);
            float* b = reinterpret_cast<float*>(grid + static_cast<int64_t>(jv) * n + ju);
            atomicAdd(a, sg * V.x);
            atomicAdd(a + 1, sg * V.y);
            atomicAdd(b, sg * V.x);
            atomicAdd(b + 1, -sg * V.y);
            atomicAdd(&blk, 2u);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && blk) atomicAdd(count, static_cast<unsigned long long>(blk));
}

// Real part of the transformed grid, times (-1)^(ix+iy) / W.
__global__ void k_image_from_fft(const float2* __restrict__ f, int n, const unsigned long long* __restrict__ count,
                                 float* __restrict__ image)
{
    const unsigned long long W = *count;
    const float inv = W ? static_cast<float>(1.0 / static_cast<double>(W)) : 0.0f;
    for (int iy = blockIdx.x; iy < n; iy += gridDim.x) {            // a row per CTA step, no division
        const int64_t row = static_cast<int64_t>(iy) * n;
        for (int ix = threadIdx.x; ix < n; ix += blockDim.x) {
            const float sg = ((ix + iy) & 1) ? -1.0f : 1.0f;
            image[row + ix] = sg * f[row + ix].x * inv;
        }
    }
}

// ---------------------------------------------------------------- Hogbom
struct HogbomState {
    unsigned long long key;   // (ordered value << 32) | (0xffffffff - pixel) of the current maximum
    unsigned int done;        // CTAs finished in this launch
    int iter;                 // components recorded
    int stopped;              // 1 once the clean has ended
    int pend_pix;             // component to subtract at the next launch (-1: none)
    float pend_flux;
    int pad;
};

__device__ __forceinline__ unsigned int ordered(float v)
{
    const unsigned int b = __float_as_uint(v);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);   // monotone in v
}

__global__ void __launch_bounds__(kImgThreads) k_hogbom_step(float* __restrict__ img, const float* __restrict__ psf,
                                                             int n, float gain, float threshold, int max_iter,
                                                             HogbomState* __restrict__ st, int* __restrict__ comp_pix,
                                                             float* __restrict__ comp_flux, int* __restrict__ n_comp)
{
    __shared__ unsigned long long best[kImgThreads / 32];
    __shared__ bool last;
    if (st->stopped) return;
    const int p = st->pend_pix;
    const float f = st->pend_flux;
    const int py = p >= 0 ? p / n : 0, px = p >= 0 ? p % n : 0, c = n / 2;
    // this thread's largest value and its pixel: pixels are visited in
    // increasing order, so a strict comparison keeps the first of equals
    float bv = -INFINITY;
    unsigned int bq = 0xffffffffu;
    const bool vec4 = (n & 3) == 0 && (reinterpret_cast<uintptr_t>(img) & 15) == 0;
    for (int qy = blockIdx.x; qy < n; qy += gridDim.x) {            // a row per CTA step, no division
        const int by = qy - py + c;                                 // beam row under image row qy
        const bool row_hit = p >= 0 && by >= 0 && by < n;
        float* irow = img + static_cast<int64_t>(qy) * n;
        const float* brow = psf + static_cast<int64_t>(row_hit ? by : 0) * n;
        const unsigned int q0 = static_cast<unsigned int>(qy) * static_cast<unsigned int>(n);
        if (vec4) {                                                 // four pixels per step, 16-byte image accesses
            for (int qx = 4 * threadIdx.x; qx < n; qx += 4 * blockDim.x) {
                float4 v4 = *reinterpret_cast<const float4*>(irow + qx);
                float v[4] = {v4.x, v4.y, v4.z, v4.w};
                if (row_hit) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int bx = qx + j - px + c;             // beam column under qx + j
                        if (bx >= 0 && bx < n) v[j] = __fsub_rn(v[j], __fmul_rn(f, brow[bx]));
                    }
                    *reinterpret_cast<float4*>(irow + qx) = make_float4(v[0], v[1], v[2], v[3]);
                }
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (v[j] > bv) {
                        bv = v[j];
                        bq = q0 + static_cast<unsigned int>(qx + j);
                    }
            }
        } else {
            for (int qx = threadIdx.x; qx < n; qx += blockDim.x) {
                float v = irow[qx];
                const int bx = qx - px + c;
                if (row_hit && bx >= 0 && bx < n) {
                    v = __fsub_rn(v, __fmul_rn(f, brow[bx]));
                    irow[qx] = v;
                }
                if (v > bv) {
                    bv = v;
                    bq = q0 + static_cast<unsigned int>(qx);
                }
            }
        }
    }
    unsigned long long key =
        bq == 0xffffffffu ? 0ull : (static_cast<unsigned long long>(ordered(bv)) << 32) | (0xffffffffu - bq);
    __threadfence();   // this thread's image updates before the CTA's count below
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(0xffffffffu, key, o);
        if (other > key) key = other;
    }
    if ((threadIdx.x & 31) == 0) best[threadIdx.x >> 5] = key;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long b = best[0];
        for (int w = 1; w < kImgThreads / 32; ++w)
            if (best[w] > b) b = best[w];
        atomicMax(&st->key, b);
        __threadfence();   // the key before the count
        last = atomicAdd(&st->done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    // the last CTA: every other CTA's writes are visible after the fence
    __threadfence();
    const unsigned long long k = atomicAdd(&st->key, 0ull);
    // no comparable value anywhere (an all-NaN image): nothing to clean
    const int win = k ? static_cast<int>(0xffffffffu - static_cast<unsigned int>(k & 0xffffffffu)) : 0;
    const float peak = k ? __ldcg(img + win) : __int_as_float(0x7fc00000);
    const int it = st->iter;
    if (it >= max_iter || !(peak >= threshold)) {
        st->stopped = 1;
        st->pend_pix = -1;
    } else {
        const float flux = __fmul_rn(gain, peak);
        comp_pix[it] = win;
        comp_flux[it] = flux;
        st->iter = it + 1;
        st->pend_pix = win;
        st->pend_flux = flux;
    }
    *n_comp = st->iter;
    st->key = 0;
    st->done = 0;
    __threadfence();
}

__global__ void k_hogbom_reset(HogbomState* st, int* n_comp)
{
    st->key = 0;
    st->done = 0;
    st->iter = 0;
    st->stopped = 0;
    st->pend_pix = -1;
    st->pend_flux = 0.0f;
    st->pad = 0;
    *n_comp = 0;
}

// ---------------------------------------------------------------- persistent Hogbom
constexpr int kHogThreads = 512;
constexpr int kMaxHogCtas = 1024;   // grid cap of the persistent clean
constexpr int kRowsAhead = 4;   // rows whose beam values a thread loads before using them
// Polls of the grid barrier before a CTA gives up: each poll is an L2 load
// and a 40 ns sleep, so the limit is of the order of a second (a healthy
// barrier completes within microseconds).
constexpr uint32_t kGridSpinLimit = 1u << 20;

// Grid-wide maximum of one 64-bit key per CTA, once per iteration, in three
// rotating slots: iteration i uses slot i % 3.
struct HogSync {
    unsigned int count[3];        // CTAs arrived
    int abort;                    // 1 once a CTA gave up waiting
    unsigned long long key[3];    // running maximum of the arrived CTAs' keys
    unsigned long long result[3]; // the maximum, published by the last CTA to arrive (0: not yet)
};

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned int atom_add_acq_rel(unsigned int* p, unsigned int v)
{
    unsigned int old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ float unordered(unsigned int o)
{
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);   // inverse of ordered()
}

// Called by one thread of every CTA of a cooperative launch (all resident)
// with the CTA's key (nonzero); returns the grid's maximum in *out, or false
// when this CTA gave up waiting (WT_ERR_TIMEOUT recorded) or another CTA had.
// Each CTA folds its key into the slot's maximum and then counts itself in;
// the last to arrive reads the maximum and publishes it with a release
// store; the others poll for it with acquire loads, at most `limit` times.
// CTA 0 clears the slot of the previous iteration once this one's result is
// out: every CTA has read that slot's result before arriving here, and no
// CTA uses it again before CTA 0 arrives at the next iteration.
__device__ bool grid_max(HogSync* sy, int it, unsigned long long key, unsigned long long* out,
                         uint32_t limit = kGridSpinLimit)
{
    const int slot = it % 3;
    atomicMax(&sy->key[slot], key);
    unsigned long long r = 0;
    // release: the key, and this CTA's clearing of a slot, before its
    // arrival; acquire: for the last to arrive, every other CTA's key
    if (atom_add_acq_rel(&sy->count[slot], 1u) == gridDim.x - 1) {
        r = atomicAdd(&sy->key[slot], 0ull);   // every key is in
        st_release_u64(&sy->result[slot], r);
    } else {
        uint32_t polls = 0;
        while ((r = ld_acquire_u64(&sy->result[slot])) == 0) {
            if (*reinterpret_cast<volatile int*>(&sy->abort) || ++polls > limit) {
                atomicExch(&sy->abort, 1);
                return false;
            }
            __nanosleep(40);
        }
    }
    if (blockIdx.x == 0) {
        const int prev = (it + 2) % 3;
        sy->count[prev] = 0;
        sy->key[prev] = 0;
        sy->result[prev] = 0;
    }
    *out = r;
    return true;
}

// A grid maximum that never completes: the arrival count starts past the
// grid size.
__global__ void k_selftest_grid_barrier(HogSync* sy, uint32_t limit, int* status)
{
    unsigned long long r;
    if (threadIdx.x == 0 && !grid_max(sy, 0, 1ull, &r, limit)) record_status(status, WT_ERR_TIMEOUT);
}

// CTA b owns image rows b, b + G, b + 2G, ... (G = gridDim.x <= n), held in
// shared memory as local rows 0, 1, 2, ... for the whole clean. V4: n is a
// multiple of 4 and the image 16-byte aligned (four pixels per thread step).
template <bool V4>
__global__ void __launch_bounds__(kHogThreads) k_hogbom_persistent(float* __restrict__ img,
                                                                  const float* __restrict__ psf, int n, float gain,
                                                                  float threshold, int max_iter,
                                                                  HogSync* __restrict__ sy, int* __restrict__ comp_pix,
                                                                  float* __restrict__ comp_flux,
                                                                  int* __restrict__ n_comp, int* status)
{
    extern __shared__ __align__(16) float rows[];
    __shared__ unsigned long long wbest[kHogThreads / 32];
    __shared__ unsigned long long gbest;
    const int G = gridDim.x, b = blockIdx.x, c = n / 2;
    const int nloc = (n - 1 - b) / G + 1;
    constexpr int kStep = V4 ? 4 : 1;
    for (int r = 0; r < nloc; ++r) {
        const float* src = img + static_cast<int64_t>(b + r * G) * n;
        float* dst = rows + static_cast<int64_t>(r) * n;
        if constexpr (V4) {
            for (int x = 4 * threadIdx.x; x < n; x += 4 * kHogThreads)
                *reinterpret_cast<float4*>(dst + x) = __ldcg(reinterpret_cast<const float4*>(src + x));
        } else {
            for (int x = threadIdx.x; x < n; x += kHogThreads) dst[x] = __ldcg(src + x);
        }
    }
    __syncthreads();
    int pend = -1, it = 0;
    float pf = 0.0f;
    for (;;) {
        const int py = pend >= 0 ? pend / n : 0, px = pend >= 0 ? pend % n : 0;
        // this thread's largest value and its pixel (ties: the lower pixel)
        float bv = -INFINITY;
        unsigned int bq = 0xffffffffu;
        for (int qx = kStep * threadIdx.x; qx < n; qx += kStep * kHogThreads) {
            for (int r0 = 0; r0 < nloc; r0 += kRowsAhead) {
                // the beam values of kRowsAhead rows first: their loads overlap
                float bm[kRowsAhead][kStep];
                bool in[kRowsAhead][kStep];
#pragma unroll
                for (int i = 0; i < kRowsAhead; ++i) {
                    const int by = b + (r0 + i) * G - py + c;   // beam row under image row b + (r0 + i) G
                    const bool hit = pend >= 0 && r0 + i < nloc && by >= 0 && by < n;
                    const float* brow = psf + static_cast<int64_t>(hit ? by : 0) * n;
#pragma unroll
                    for (int j = 0; j < kStep; ++j) {
                        const int bx = qx + j - px + c;         // beam column under qx + j
                        in[i][j] = hit && bx >= 0 && bx < n;
                        bm[i][j] = in[i][j] ? __ldg(brow + bx) : 0.0f;
                    }
                }
#pragma unroll
                for (int i = 0; i < kRowsAhead; ++i) {
                    const int r = r0 + i;
                    if (r >= nloc) break;
                    float* row = rows + static_cast<int64_t>(r) * n;
                    float v[kStep];
                    if constexpr (V4) {
                        const float4 v4 = *reinterpret_cast<const float4*>(row + qx);
                        v[0] = v4.x; v[1] = v4.y; v[2] = v4.z; v[3] = v4.w;
                    } else {
                        v[0] = row[qx];
                    }
                    bool any = false;
#pragma unroll
                    for (int j = 0; j < kStep; ++j)
                        if (in[i][j]) {
                            v[j] = __fsub_rn(v[j], __fmul_rn(pf, bm[i][j]));
                            any = true;
                        }
                    if (any) {
                        if constexpr (V4) {
                            *reinterpret_cast<float4*>(row + qx) = make_float4(v[0], v[1], v[2], v[3]);
                        } else {
                            row[qx] = v[0];
                        }
                    }
                    const unsigned int q0 = static_cast<unsigned int>(b + r * G) * static_cast<unsigned int>(n);
#pragma unroll
                    for (int j = 0; j < kStep; ++j) {
                        const unsigned int q = q0 + static_cast<unsigned int>(qx + j);
                        if (v[j] > bv || (v[j] == bv && q < bq)) {
                            bv = v[j];
                            bq = q;
                        }
                    }
                }
            }
        }
        unsigned long long key =
            bq == 0xffffffffu ? 0ull : (static_cast<unsigned long long>(ordered(bv)) << 32) | (0xffffffffu - bq);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long other = __shfl_xor_sync(0xffffffffu, key, o);
            if (other > key) key = other;
        }
        if ((threadIdx.x & 31) == 0) wbest[threadIdx.x >> 5] = key;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long m = wbest[0];
            for (int w = 1; w < kHogThreads / 32; ++w)
                if (wbest[w] > m) m = wbest[w];
            // a CTA without a comparable value (all NaN) still takes part with
            // the smallest key, which decodes to NaN and stops the clean
            if (m == 0) m = 1;
            unsigned long long g = 0;
            if (!grid_max(sy, it, m, &g)) {
                record_status(status, WT_ERR_TIMEOUT);
                g = 0;
            }
            gbest = g;
        }
        __syncthreads();
        if (gbest == 0) return;   // gave up waiting: every CTA leaves
        const unsigned long long k = gbest;
        const float peak = unordered(static_cast<unsigned int>(k >> 32));
        if (it >= max_iter || !(peak >= threshold)) break;
        pend = static_cast<int>(0xffffffffu - static_cast<unsigned int>(k & 0xffffffffu));
        pf = __fmul_rn(gain, peak);
        if (b == 0 && threadIdx.x == 0) {
            comp_pix[it] = pend;
            comp_flux[it] = pf;
        }
        ++it;
    }
    for (int r = 0; r < nloc; ++r) {
        float* dst = img + static_cast<int64_t>(b + r * G) * n;
        const float* src = rows + static_cast<int64_t>(r) * n;
        if constexpr (V4) {
            for (int x = 4 * threadIdx.x; x < n; x += 4 * kHogThreads)
                *reinterpret_cast<float4*>(dst + x) = *reinterpret_cast<const float4*>(src + x);
        } else {
            for (int x = threadIdx.x; x < n; x += kHogThreads) dst[x] = src[x];
        }
    }
    if (b == 0 && threadIdx.x == 0) *n_comp = it;
}

// ---------------------------------------------------------------- components
// (l, m, flux) in float64 of recorded components [from, to).
__global__ void k_components_lm(const int* __restrict__ pix, const float* __restrict__ flux, int from, int to, int n,
                                double dl, double* __restrict__ l, double* __restrict__ m, double* __restrict__ f)
{
    const int i = from + static_cast<int>(blockIdx.x * blockDim.x + threadIdx.x);
    if (i >= to) return;
    const int p = pix[i];
    l[i] = static_cast<double>(p % n - n / 2) * dl;
    m[i] = static_cast<double>(p / n - n / 2) * dl;
    f[i] = static_cast<double>(flux[i]);
}

// CTAs for the row loops: one row per CTA step, at most 8 CTAs per SM.
int rows_blocks(int n)
{
    const int cap = num_sms() * 8;
    return n < cap ? n : cap;
}

}  // namespace

// Dirty image (or beam) into `image`, with `grid` (n x n complex64) as
// scratch and `count` (one unsigned long long) as the entry counter.
int dirty_image(const double* uvw, const float2* vis, int64_t n_vis, int n, double dl, float* image, float2* grid,
                unsigned long long* count, cudaStream_t s)
{
    const int64_t nn = static_cast<int64_t>(n) * n;
    WT_CUDA_TRY(cudaMemsetAsync(grid, 0, static_cast<size_t>(nn) * sizeof(float2), s));
    WT_CUDA_TRY(cudaMemsetAsync(count, 0, sizeof(unsigned long long), s));
    if (n_vis > 0) {
        const double inv_du = static_cast<double>(n) * dl;   // 1 / du
        k_grid_nn<<<static_cast<unsigned>((n_vis + kImgThreads - 1) / kImgThreads), kImgThreads, 0, s>>>(
            uvw, vis, n_vis, n, inv_du, grid, count);
        WT_CUDA_TRY(cudaGetLastError());
    }
    int rc = fft2_forward(grid, n, s);
    if (rc) return rc;
    k_image_from_fft<<<rows_blocks(n), kImgThreads, 0, s>>>(grid, n, count, image);
    WT_CUDA_TRY(cudaGetLastError());
    return WT_OK;
}

// Hogbom clean of `image` in place; components appended to comp_pix /
// comp_flux (device, capacity max_iter), their count in *n_comp (device).
// `state` is a device HogbomState, reset here.
namespace {

size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

// CTAs and shared-memory bytes of a persistent clean of an n x n image, or 0
// CTAs when the schedule does not apply (rows too large for shared memory,
// no cooperative launch, or WT_HOGBOM=launches in the environment).
template <bool V4>
int persistent_grid(int n, size_t* smem)
{
    const char* e = getenv("WT_HOGBOM");
    if (e && strcmp(e, "launches") == 0) return 0;
    int dev = 0, coop = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || !coop) {
        cudaGetLastError();
        return 0;
    }
    const int sms = num_sms();
    for (int per_sm = 2; per_sm >= 1; --per_sm) {
        const int G = std::min(std::min(n, per_sm * sms), kMaxHogCtas);
        const size_t bytes = static_cast<size_t>((n + G - 1) / G) * n * sizeof(float);
        if (bytes > static_cast<size_t>(optin) - 1024) continue;
        if (cudaFuncSetAttribute(k_hogbom_persistent<V4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(bytes)) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_hogbom_persistent<V4>, kHogThreads, bytes) !=
            cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (static_cast<int64_t>(occ) * sms >= G) {
            *smem = bytes;
            return G;
        }
    }
    return 0;
}

template <bool V4>
int launch_persistent(int G, size_t smem, float* image, const float* psf, int n, float gain, float threshold,
                      int max_iter, HogSync* sy, int* comp_pix, float* comp_flux, int* n_comp, cudaStream_t s)
{
    int* status = device_status_word();
    if (!status) return set_error(WT_ERR_CUDA, "wt_hogbom: no device status word");
    WT_CUDA_TRY(cudaMemsetAsync(sy, 0, sizeof(HogSync), s));
    void* args[] = {&image, &psf, &n, &gain, &threshold, &max_iter, &sy, &comp_pix, &comp_flux, &n_comp, &status};
    WT_CUDA_TRY(cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k_hogbom_persistent<V4>), dim3(G),
                                            dim3(kHogThreads), args, smem, s));
    return WT_OK;
}

}  // namespace

int hogbom(float* image, const float* psf, int n, float gain, float threshold, int max_iter, int* comp_pix,
           float* comp_flux, int* n_comp, void* state, cudaStream_t s)
{
    HogSync* sy = reinterpret_cast<HogSync*>(static_cast<char*>(state) + round256(sizeof(HogbomState)));
    const bool v4 = (n & 3) == 0 && (reinterpret_cast<uintptr_t>(image) & 15) == 0;
    size_t smem = 0;
    const int G = v4 ? persistent_grid<true>(n, &smem) : persistent_grid<false>(n, &smem);
    if (G > 0)
        return v4 ? launch_persistent<true>(G, smem, image, psf, n, gain, threshold, max_iter, sy, comp_pix,
                                            comp_flux, n_comp, s)
                  : launch_persistent<false>(G, smem, image, psf, n, gain, threshold, max_iter, sy, comp_pix,
                                             comp_flux, n_comp, s);
    k_hogbom_reset<<<1, 1, 0, s>>>(static_cast<HogbomState*>(state), n_comp);
    const int blocks = rows_blocks(n);
    // max_iter + 1 launches: the last subtracts the last component and stops
    for (int it = 0; it <= max_iter; ++it) {
        k_hogbom_step<<<blocks, kImgThreads, 0, s>>>(image, psf, n, gain, threshold, max_iter,
                                                     static_cast<HogbomState*>(state), comp_pix, comp_flux, n_comp);
    }
    WT_CUDA_TRY(cudaGetLastError());
    return WT_OK;
}

size_t hogbom_state_bytes() { return round256(sizeof(HogbomState)) + sizeof(HogSync); }

int components_lm(const int* pix, const float* flux, int from, int to, int n, double dl, double* l, double* m,
                  double* f, cudaStream_t s)
{
    if (to <= from) return WT_OK;
    const int cnt = to - from;
    k_components_lm<<<(cnt + 127) / 128, 128, 0, s>>>(pix, flux, from, to, n, dl, l, m, f);
    WT_CUDA_TRY(cudaGetLastError());
    return WT_OK;
}

}  // namespace wt

// ===========================================================================
// C entry points (declared in include/wtvis.h)
// ===========================================================================
namespace {

int check_image_args(const char* fn, int n, double dl)
{
    using namespace wt;
    if (n < 2 || n > 16384 || (n & 1)) return set_error(WT_ERR_ARG, "%s: n = %d must be even, 2..16384", fn, n);
    if (!(dl > 0.0) || !isfinite(dl)) return set_error(WT_ERR_RANGE, "%s: pixel size must be positive", fn);
    return WT_OK;
}

}  // namespace

extern "C" int wt_dirty_image(const double* uvw, const void* vis, int64_t n_vis, int n, double dl, float* image,
                              void* stream)
{
    using namespace wt;
    const char* fn = "wt_dirty_image";
    int rc = check_image_args(fn, n, dl);
    if (rc) return rc;
    if (n_vis < 0) return set_error(WT_ERR_ARG, "%s: n_vis < 0", fn);
    const size_t nn = static_cast<size_t>(n) * n;
    if ((rc = check_device_buffer(uvw, static_cast<size_t>(n_vis) * 24, fn, "uvw", 8)) ||
        (vis && (rc = check_device_buffer(vis, static_cast<size_t>(n_vis) * 8, fn, "vis", 8))) ||
        (rc = check_device_buffer(image, nn * 4, fn, "image", 4)))
        return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void* scratch = nullptr;
    const size_t bytes = nn * sizeof(float2) + 256;
    cudaError_t e = cudaMallocAsync(&scratch, bytes, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(WT_ERR_NOMEM, "%s: scratch allocation of %zu bytes failed", fn, bytes);
    }
    float2* grid = static_cast<float2*>(scratch);
    unsigned long long* count = reinterpret_cast<unsigned long long*>(static_cast<char*>(scratch) + nn * sizeof(float2));
    rc = dirty_image(uvw, static_cast<const float2*>(vis), n_vis, n, dl, image, grid, count, s);
    const cudaError_t ef = cudaFreeAsync(scratch, s);
    if (rc) return rc;
    if (ef != cudaSuccess) return cuda_error(ef, "cudaFreeAsync");
    return WT_OK;
}

extern "C" int wt_selftest_grid_barrier(uint32_t spin_limit, void* stream)
{
    using namespace wt;
    const char* fn = "wt_selftest_grid_barrier";
    if (spin_limit < 1 || spin_limit > 65536) return set_error(WT_ERR_ARG, "%s: spin_limit must be in 1..65536", fn);
    int dev = 0, coop = 0;
    WT_CUDA_TRY(cudaGetDevice(&dev));
    WT_CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    if (!coop) return set_error(WT_ERR_UNSUPPORTED, "%s: no cooperative launch on this device", fn);
    int* status = device_status_word();
    if (!status) return set_error(WT_ERR_CUDA, "%s: no device status word", fn);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    HogSync* sy = nullptr;
    WT_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&sy), sizeof(HogSync), s));
    int rc = WT_OK;
    cudaError_t e = cudaMemsetAsync(sy, 0, sizeof(HogSync), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(&sy->count[0], 0x02, sizeof(unsigned int), s);   // 0x02020202 arrivals
    if (e == cudaSuccess) {
        void* args[] = {&sy, &spin_limit, &status};
        e = cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k_selftest_grid_barrier), dim3(2), dim3(32),
                                        args, 0, s);
    }
    if (e != cudaSuccess) rc = cuda_error(e, fn);
    const cudaError_t ef = cudaFreeAsync(sy, s);
    if (!rc && ef != cudaSuccess) rc = cuda_error(ef, "cudaFreeAsync");
    return rc;
}

extern "C" int wt_hogbom(float* image, const float* psf, int n, float gain, float threshold, int max_iter,
                         int* comp_pix, float* comp_flux, int* n_comp, void* stream)
{
    using namespace wt;
    const char* fn = "wt_hogbom";
    if (n < 2 || n > 16384 || (n & 1)) return set_error(WT_ERR_ARG, "%s: n = %d must be even, 2..16384", fn, n);
    if (max_iter < 0 || max_iter > (1 << 24)) return set_error(WT_ERR_ARG, "%s: max_iter outside 0..2^24", fn);
    if (!(gain > 0.0f) || !(gain <= 1.0f)) return set_error(WT_ERR_RANGE, "%s: gain must be in (0, 1]", fn);
    if (!isfinite(threshold)) return set_error(WT_ERR_RANGE, "%s: threshold must be finite", fn);
    const size_t nn = static_cast<size_t>(n) * n;
    int rc;
    if ((rc = check_device_buffer(image, nn * 4, fn, "image", 4)) || (rc = check_device_buffer(psf, nn * 4, fn, "psf", 4)) ||
        (rc = check_device_buffer(n_comp, 4, fn, "n_comp", 4)) ||
        (max_iter > 0 && ((rc = check_device_buffer(comp_pix, static_cast<size_t>(max_iter) * 4, fn, "comp_pix", 4)) ||
                          (rc = check_device_buffer(comp_flux, static_cast<size_t>(max_iter) * 4, fn, "comp_flux", 4)))))
        return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void* state = nullptr;
    cudaError_t e = cudaMallocAsync(&state, hogbom_state_bytes(), s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(WT_ERR_NOMEM, "%s: state allocation failed", fn);
    }
    rc = hogbom(image, psf, n, gain, threshold, max_iter, comp_pix, comp_flux, n_comp, state, s);
    const cudaError_t ef = cudaFreeAsync(state, s);
    if (rc) return rc;
    if (ef != cudaSuccess) return cuda_error(ef, "cudaFreeAsync");
    return WT_OK;
}

extern "C" int wt_clean(const double* uvw, const void* vis_obs, int64_t n_vis, int n, double dl, double ra0,
                        double dec0, int J, int predictor, int mode, float gain, float threshold, int minor_iter,
                        int n_major, int* comp_pix, float* comp_flux, int* n_comp, void* vis_resid, float* image_resid,
                        void* stream)
{
    using namespace wt;
    const char* fn = "wt_clean";
    int rc = check_image_args(fn, n, dl);
    if (rc) return rc;
    if (n_vis < 0) return set_error(WT_ERR_ARG, "%s: n_vis < 0", fn);
    if (predictor != WT_PREDICT_TREE && predictor != WT_PREDICT_DIRECT)
        return set_error(WT_ERR_ARG, "%s: bad predictor %d", fn, predictor);
    if (mode != WT_MIXED && mode != WT_MIXED_FAST)
        return set_error(WT_ERR_ARG, "%s: mode must be WT_MIXED or WT_MIXED_FAST (complex64 visibilities)", fn);
    if (minor_iter < 0 || n_major < 0 || static_cast<int64_t>(minor_iter) * n_major > (1 << 24))
        return set_error(WT_ERR_ARG, "%s: minor_iter x n_major outside 0..2^24", fn);
    if (!(gain > 0.0f) || !(gain <= 1.0f)) return set_error(WT_ERR_RANGE, "%s: gain must be in (0, 1]", fn);
    if (!isfinite(threshold)) return set_error(WT_ERR_RANGE, "%s: threshold must be finite", fn);
    if (!n_comp) return set_error(WT_ERR_ARG, "%s: n_comp (host) is NULL", fn);
    const int cap = minor_iter * n_major;
    const size_t nn = static_cast<size_t>(n) * n;
    if ((rc = check_device_buffer(uvw, static_cast<size_t>(n_vis) * 24, fn, "uvw", 8)) ||
        (rc = check_device_buffer(vis_obs, static_cast<size_t>(n_vis) * 8, fn, "vis_obs", 8)) ||
        (rc = check_device_buffer(vis_resid, static_cast<size_t>(n_vis) * 8, fn, "vis_resid", 8)) ||
        (rc = check_device_buffer(image_resid, nn * 4, fn, "image_resid", 4)) ||
        (cap > 0 && ((rc = check_device_buffer(comp_pix, static_cast<size_t>(cap) * 4, fn, "comp_pix", 4)) ||
                     (rc = check_device_buffer(comp_flux, static_cast<size_t>(cap) * 4, fn, "comp_flux", 4)))))
        return rc;
    *n_comp = 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // scratch: grid, beam, model visibilities, component (l, m, flux), counters
    auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t c3 = static_cast<size_t>(cap > 0 ? cap : 1) * 8;
    const bool tree = predictor == WT_PREDICT_TREE;
    const size_t bytes = up(nn * 8) + up(nn * 4) + up(static_cast<size_t>(n_vis > 0 ? n_vis : 1) * 8) + 3 * up(c3) +
                         up(8) + up(hogbom_state_bytes()) + up(4) + (tree ? up(nn * 8) : 0);
    void* scratch = nullptr;
    cudaError_t e = cudaMallocAsync(&scratch, bytes, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(WT_ERR_NOMEM, "%s: scratch allocation of %zu bytes failed", fn, bytes);
    }
    char* q = static_cast<char*>(scratch);
    auto take = [&](size_t b) {
        char* r = q;
        q += up(b);
        return r;
    };
    float2* grid = reinterpret_cast<float2*>(take(nn * 8));
    float* beam = reinterpret_cast<float*>(take(nn * 4));
    float2* model = reinterpret_cast<float2*>(take(static_cast<size_t>(n_vis > 0 ? n_vis : 1) * 8));
    double* cl = reinterpret_cast<double*>(take(c3));
    double* cm = reinterpret_cast<double*>(take(c3));
    double* cf = reinterpret_cast<double*>(take(c3));
    unsigned long long* count = reinterpret_cast<unsigned long long*>(take(8));
    void* state = take(hogbom_state_bytes());
    int* d_found = reinterpret_cast<int*>(take(4));
    int64_t* xref = tree ? reinterpret_cast<int64_t*>(take(nn * 8)) : nullptr;

    int total = 0;
    // the tree predictor maps components through the cross-reference table
    // of the image pixels, built once (Sec. 3.5)
    rc = tree ? wt_xref_table(n, dl, ra0, dec0, J, xref, stream) : WT_OK;
    if (!rc) rc = dirty_image(uvw, nullptr, n_vis, n, dl, beam, grid, count, s);
    if (!rc && n_vis > 0) {
        e = cudaMemcpyAsync(vis_resid, vis_obs, static_cast<size_t>(n_vis) * 8, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) rc = cuda_error(e, "cudaMemcpyAsync");
    }
    for (int cycle = 0; cycle < n_major && !rc; ++cycle) {
        // 3. gridding and FFT of the residuals, then the minor cycles
        if ((rc = dirty_image(uvw, static_cast<const float2*>(vis_resid), n_vis, n, dl, image_resid, grid, count, s)))
            break;
        if ((rc = hogbom(image_resid, beam, n, gain, threshold, minor_iter, comp_pix + total, comp_flux + total, d_found,
                         state, s)))
            break;
        int found = 0;
        e = cudaMemcpyAsync(&found, d_found, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            rc = cuda_error(e, "reading the component count");
            break;
        }
        if (found == 0) break;
        if ((rc = components_lm(comp_pix, comp_flux, total, total + found, n, dl, cl, cm, cf, s))) break;
        total += found;
        // 1. model visibilities from every component so far, 2. subtraction
        if (predictor == WT_PREDICT_TREE) {
            wt_tree t = nullptr;
            if ((rc = wt_build_tree_xref(xref, n, comp_pix, cf, total, ra0, dec0, J, &t, stream))) break;
            rc = wt_predict_vis(t, uvw, n_vis, model, mode, 1, WT_SUM_EQ17_REGROUPED, stream);
            wt_free_tree(t);
        } else {
            rc = dft_predict_vis(cl, cm, cf, total, uvw, n_vis, model, mode, 1, stream);
        }
        if (!rc) rc = subtract_model(vis_obs, model, vis_resid, n_vis, mode, stream);
    }
    // the dirty image of the final residual visibilities
    if (!rc) rc = dirty_image(uvw, static_cast<const float2*>(vis_resid), n_vis, n, dl, image_resid, grid, count, s);
    *n_comp = total;
    const cudaError_t ef = cudaFreeAsync(scratch, s);
    if (rc) return rc;
    if (ef != cudaSuccess) return cuda_error(ef, "cudaFreeAsync");
    return WT_OK;
}
