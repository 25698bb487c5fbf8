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

// ---------------------------------------------------------------- w-projection
// The w-corrected dirty image (the wide-field imaging of Sec. 3.6.2, which
// grids with an anti-aliasing kernel and a w-kernel over w-planes):
//   I(l, m) = (1/W) Re sum_entries V exp(-i 2 pi (u l + v m + w (n(l, m) - 1))),
// approximated by convolutional gridding. In image units t = l / (n dl),
// s = m / (n dl) (the field is |t|, |s| < 1/2) and uv units of cells
// x = u / du, the kernel of a plane at w is
//   K_w(x, y) = int int c(t) c(s) exp(-i 2 pi w (n - 1)) exp(i 2 pi (x t + y s)) dt ds
// over the field, c the Fourier transform of a Kaiser-Bessel kernel of
// width kWpWidth cells (closed form, c(0) = 1); summed over all cells,
// sum_x K_w(x - x_k) exp(-i 2 pi x t) = c(t) exp(-i 2 pi w (n - 1)) exp(-i 2 pi x_k t)
// inside the field, so the transformed grid divided by c(t) c(s) is the
// image above. K_w is tabulated at kWpOversample points per cell over the
// support S = 2h + 1 cells (h from the largest chirp frequency of the field
// and the Kaiser-Bessel half-width) for planes uniformly spaced in |w|,
// from a midpoint sum over kWpSamples^2 points of the field (two complex
// matrix products per plane), and interpolated linearly in |w| between the
// two nearest planes; an entry at w < 0 takes conj(K_|w|(-x, -y)). Each
// entry is spread over the support its own |w| needs (the same rule at that
// |w|), not the table's.
constexpr int kWpWidth = 7;             // Kaiser-Bessel width (cells)
constexpr double kWpBeta = 16.25;       // its shape parameter
constexpr int kWpOversample = 8;        // table points per cell
constexpr int kWpSamples = 128;         // field samples per axis for the kernels
constexpr int kWpMaxHalf = 32;          // largest half-support h (cells)

// c(t) / c(0) for the Kaiser-Bessel kernel of width W and shape beta: the
// kernel's Fourier transform, sinh(sqrt(beta^2 - (pi W t)^2)) / sqrt(...),
// or sin(...) / ... past the zero of the root.
__host__ __device__ inline double kb_taper(double t)
{
    const double a = kWpBeta * kWpBeta - (kPi * kWpWidth * t) * (kPi * kWpWidth * t);
    const double c0 = sinh(kWpBeta) / kWpBeta;
    if (a > 0.0) {
        const double r = sqrt(a);
        return (sinh(r) / r) / c0;
    }
    if (a < 0.0) {
        const double r = sqrt(-a);
        return (sin(r) / r) / c0;
    }
    return 1.0 / c0;
}

struct WpPlan {
    int P;          // planes
    int h, S, T;    // half-support, support (cells), table points per axis (S * oversample + 1)
    double dw;      // plane spacing in |w|
    double ndl;     // n dl: the field width (radians)
    double xc_per_w;   // the field's largest chirp frequency (cells) per unit |w|
};

// f[p][q][r] = c(t_q) c(t_r) exp(-i 2 pi w_p (n - 1)) at the field's sample
// points t = (q + 1/2)/M - 1/2 (float64 phase reduced modulo 1).
__global__ void k_wp_field(WpPlan pl, float2* __restrict__ f)
{
    const int M = kWpSamples;
    const int64_t total = static_cast<int64_t>(pl.P) * M * M;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int r = static_cast<int>(i % M), q = static_cast<int>((i / M) % M), p = static_cast<int>(i / (M * M));
        const double tq = (q + 0.5) / M - 0.5, tr = (r + 0.5) / M - 0.5;
        const double l = tq * pl.ndl, m = tr * pl.ndl;
        const double r2 = l * l + m * m;
        const double nm1 = -r2 / (1.0 + sqrt(1.0 - r2));
        double ph = -(p * pl.dw) * nm1;                // turns
        ph -= rint(ph);
        double sn, cs;
        sincospi(2.0 * ph, &sn, &cs);
        const double c = kb_taper(tq) * kb_taper(tr);
        f[i] = make_float2(static_cast<float>(c * cs), static_cast<float>(c * sn));
    }
}

// tw[j][q] = exp(i 2 pi x_j t_q), x_j = j / oversample - (h + 1/2).
__global__ void k_wp_twiddles(WpPlan pl, float2* __restrict__ tw)
{
    const int M = kWpSamples;
    const int total = pl.T * M;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int q = i % M, j = i / M;
        const double x = static_cast<double>(j) / kWpOversample - (pl.h + 0.5);
        const double t = (q + 0.5) / M - 0.5;
        double ph = x * t;
        ph -= rint(ph);
        double sn, cs;
        sincospi(2.0 * ph, &sn, &cs);
        tw[i] = make_float2(static_cast<float>(cs), static_cast<float>(sn));
    }
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// a[p][q][j] = sum_r f[p][q][r] tw[j][r]: one CTA per (p, q), threads over j.
__global__ void k_wp_stage1(WpPlan pl, const float2* __restrict__ f, const float2* __restrict__ tw,
                            float2* __restrict__ a)
{
    const int M = kWpSamples;
    __shared__ float2 row[kWpSamples];
    const int64_t pq = blockIdx.x;
    for (int r = threadIdx.x; r < M; r += blockDim.x) row[r] = f[pq * M + r];
    __syncthreads();
    for (int j = threadIdx.x; j < pl.T; j += blockDim.x) {
        float2 acc = make_float2(0.f, 0.f);
        const float2* t = tw + static_cast<int64_t>(j) * M;
        for (int r = 0; r < M; ++r) {
            const float2 b = cmul(row[r], t[r]);
            acc.x += b.x;
            acc.y += b.y;
        }
        a[pq * pl.T + j] = acc;
    }
}

// K[p][i][j] = (1/M^2) sum_q tw[i][q] a[p][q][j]: one CTA per (p, i).
__global__ void k_wp_stage2(WpPlan pl, const float2* __restrict__ a, const float2* __restrict__ tw,
                            float2* __restrict__ K)
{
    const int M = kWpSamples;
    __shared__ float2 col[kWpSamples];
    const int p = blockIdx.x / pl.T, i = blockIdx.x % pl.T;
    for (int q = threadIdx.x; q < M; q += blockDim.x) col[q] = tw[static_cast<int64_t>(i) * M + q];
    __syncthreads();
    const float inv = 1.0f / (static_cast<float>(M) * static_cast<float>(M));
    for (int j = threadIdx.x; j < pl.T; j += blockDim.x) {
        float2 acc = make_float2(0.f, 0.f);
        const float2* ap = a + (static_cast<int64_t>(p) * M) * pl.T + j;
        for (int q = 0; q < M; ++q) {
            const float2 b = cmul(col[q], ap[static_cast<int64_t>(q) * pl.T]);
            acc.x += b.x;
            acc.y += b.y;
        }
        K[(static_cast<int64_t>(p) * pl.T + i) * pl.T + j] = make_float2(acc.x * inv, acc.y * inv);
    }
}

// One entry (V at x, y cells and w) into the grid by a warp, lanes over the
// S x S taps; false if its support leaves the grid (the entry is dropped).
__device__ __forceinline__ bool wp_entry(const WpPlan& pl, const float2* __restrict__ K, float2 V, double x,
                                         double y, double w, int n, float2* __restrict__ grid, int lane)
{
    const double icd = rint(x), jcd = rint(y);
    const int half = n / 2;
    const double lo = -half + pl.h + 1, hi = half - pl.h - 1;
    if (!(icd >= lo && icd <= hi && jcd >= lo && jcd <= hi && fabs(w) <= 1e30))   // false for NaN too
        return false;
    const int ic = static_cast<int>(icd), jc = static_cast<int>(jcd);
    const float fx = static_cast<float>(x - icd), fy = static_cast<float>(y - jcd);
    const bool neg = w < 0.0;
    double pw = fabs(w) / pl.dw;
    int p0 = static_cast<int>(floor(pw));
    if (p0 > pl.P - 2) p0 = pl.P - 2;
    if (p0 < 0) p0 = 0;
    const float a = static_cast<float>(fmin(fmax(pw - p0, 0.0), 1.0));
    const int last = pl.S * kWpOversample;                         // the table's last index
    const float2* K0 = K + static_cast<int64_t>(p0) * pl.T * pl.T;
    const float2* K1 = K0 + static_cast<int64_t>(pl.T) * pl.T;
    // this entry's own support: the Kaiser-Bessel half-width and the chirp
    // frequency of its |w| (the kernel is negligible beyond), within the table's
    int he = static_cast<int>(ceil(0.5 * kWpWidth + pl.xc_per_w * fabs(w))) + 1;
    he = he < pl.h ? he : pl.h;
    const int Se = 2 * he + 1;
    const int taps = Se * Se;
    for (int t = lane; t < taps; t += 32) {
        const int dx = t % Se - he, dy = t / Se - he;
        int ix = __float2int_rn((static_cast<float>(dx) - fx + pl.h + 0.5f) * kWpOversample);
        int iy = __float2int_rn((static_cast<float>(dy) - fy + pl.h + 0.5f) * kWpOversample);
        ix = min(max(ix, 0), last);
        iy = min(max(iy, 0), last);
        if (neg) {                                                 // conj(K_|w|(-x, -y))
            ix = last - ix;
            iy = last - iy;
        }
        const int64_t off = static_cast<int64_t>(ix) * pl.T + iy;  // table [x][y]
        const float2 k0 = K0[off], k1 = K1[off];
        float2 k = make_float2(fmaf(a, k1.x - k0.x, k0.x), fmaf(a, k1.y - k0.y, k0.y));
        if (neg) k.y = -k.y;
        const int iu = ic + dx + half, iv = jc + dy + half;
        const float sg = ((iu + iv) & 1) ? -1.0f : 1.0f;            // the index shift (-1)^(iu+iv)
        const float2 e = cmul(V, k);
        float* g = reinterpret_cast<float*>(grid + static_cast<int64_t>(iv) * n + iu);
        atomicAdd(g, sg * e.x);
        atomicAdd(g + 1, sg * e.y);
    }
    return true;
}

// A warp per visibility: the visibility (unit value if vis is null) and its
// conjugate at -B; counts the entries gridded.
__global__ void k_grid_wproj(WpPlan pl, const float2* __restrict__ K, const double* __restrict__ uvw,
                             const float2* __restrict__ vis, int64_t n_vis, int n, double inv_du,
                             float2* __restrict__ grid, unsigned long long* __restrict__ count)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x / 32);
    unsigned long long mine = 0;
    for (int64_t k = static_cast<int64_t>(blockIdx.x) * (blockDim.x / 32) + (threadIdx.x >> 5); k < n_vis;
         k += warps) {
        const double x = uvw[3 * k] * inv_du, y = uvw[3 * k + 1] * inv_du, w = uvw[3 * k + 2];
        const float2 V = vis ? vis[k] : make_float2(1.0f, 0.0f);
        const bool in = wp_entry(pl, K, V, x, y, w, n, grid, lane);
        if (in) wp_entry(pl, K, make_float2(V.x, -V.y), -x, -y, -w, n, grid, lane);
        if (in && lane == 0) mine += 2;
    }
    if (lane == 0 && mine) atomicAdd(count, mine);
}

// Real part of the transformed grid, times (-1)^(ix+iy) / (W c(t) c(s)).
__global__ void k_image_from_fft_wp(const float2* __restrict__ f, int n, const unsigned long long* __restrict__ count,
                                    float* __restrict__ image)
{
    const unsigned long long W = *count;
    const double inv = W ? 1.0 / static_cast<double>(W) : 0.0;
    for (int iy = blockIdx.x; iy < n; iy += gridDim.x) {
        const int64_t row = static_cast<int64_t>(iy) * n;
        const double cy = kb_taper(static_cast<double>(iy - n / 2) / n);
        for (int ix = threadIdx.x; ix < n; ix += blockDim.x) {
            const float sg = ((ix + iy) & 1) ? -1.0f : 1.0f;
            const double c = kb_taper(static_cast<double>(ix - n / 2) / n) * cy;
            image[row + ix] = static_cast<float>(sg * f[row + ix].x * inv / c);
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

namespace wt {
namespace {

// The largest |w| of the visibilities as float64 bits (non-negative doubles
// order as their bits); *out zeroed before the launch.
__global__ void k_max_abs_w(const double* __restrict__ uvw, int64_t n_vis, unsigned long long* __restrict__ out)
{
    unsigned long long m = 0;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n_vis;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const double w = fabs(uvw[3 * i + 2]);
        if (isfinite(w)) {
            const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(w));
            m = b > m ? b : m;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(0xffffffffu, m, o);
        m = other > m ? other : m;
    }
    if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

// The batch's largest finite |w| (1 if none is above 0); synchronises s.
int max_abs_w(const double* uvw, int64_t n_vis, cudaStream_t s, double* out)
{
    unsigned long long* d = nullptr;
    WT_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&d), sizeof(unsigned long long), s));
    unsigned long long h = 0;
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess && n_vis > 0) {
        int64_t b = (n_vis + 255) / 256;
        if (b > 4096) b = 4096;
        k_max_abs_w<<<static_cast<unsigned>(b), 256, 0, s>>>(uvw, n_vis, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFreeAsync(d, s);
    if (e != cudaSuccess) return cuda_error(e, "the largest |w|");
    double wm;
    memcpy(&wm, &h, sizeof(wm));
    *out = wm > 0.0 ? wm : 1.0;
    return WT_OK;
}

int dirty_image_w(const double* uvw, const float2* vis, int64_t n_vis, int n, double dl, int planes, double w_max,
                  float* image, cudaStream_t s)
{
    const char* fn = "wt_dirty_image_w";
    const double ndl = n * dl;
    if (!(ndl * ndl < 1.0)) return set_error(WT_ERR_RANGE, "%s: the field (n dl = %g) must lie inside l^2 + m^2 < 1", fn, ndl);
    const int64_t nn = static_cast<int64_t>(n) * n;
    if (w_max <= 0.0) {   // the batch's own largest |w|
        const int rc = max_abs_w(uvw, n_vis, s, &w_max);
        if (rc) return rc;
    }
    WpPlan pl;
    pl.P = planes;
    pl.dw = w_max / (planes - 1);
    pl.ndl = ndl;
    // the largest chirp frequency of the field in cells: w (n dl)^2 / (2 n) at its corner
    const double n_min = sqrt(1.0 - 0.5 * ndl * ndl);
    pl.xc_per_w = ndl * ndl / (2.0 * n_min);
    const double xc = w_max * pl.xc_per_w;
    pl.h = static_cast<int>(ceil(0.5 * kWpWidth + xc)) + 1;
    if (pl.h > kWpMaxHalf)
        return set_error(WT_ERR_RANGE, "%s: w up to %g needs a kernel half-width of %d cells (at most %d)", fn, w_max,
                         pl.h, kWpMaxHalf);
    if (2 * pl.h + 2 >= n / 2) return set_error(WT_ERR_RANGE, "%s: a %d-cell kernel does not fit an n = %d grid", fn,
                                                2 * pl.h + 1, n);
    pl.S = 2 * pl.h + 1;
    pl.T = pl.S * kWpOversample + 1;
    const int M = kWpSamples;
    auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t b_grid = up(nn * sizeof(float2)), b_cnt = 256;
    const size_t b_f = up(static_cast<size_t>(planes) * M * M * sizeof(float2));
    const size_t b_tw = up(static_cast<size_t>(pl.T) * M * sizeof(float2));
    const size_t b_a = up(static_cast<size_t>(planes) * M * pl.T * sizeof(float2));
    const size_t b_k = up(static_cast<size_t>(planes) * pl.T * pl.T * sizeof(float2));
    char* scratch = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&scratch), b_grid + b_cnt + b_f + b_tw + b_a + b_k, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(WT_ERR_NOMEM, "%s: scratch allocation failed: %s", fn, cudaGetErrorString(e));
    }
    float2* grid = reinterpret_cast<float2*>(scratch);
    unsigned long long* count = reinterpret_cast<unsigned long long*>(scratch + b_grid);
    float2* f = reinterpret_cast<float2*>(scratch + b_grid + b_cnt);
    float2* tw = reinterpret_cast<float2*>(scratch + b_grid + b_cnt + b_f);
    float2* a = reinterpret_cast<float2*>(scratch + b_grid + b_cnt + b_f + b_tw);
    float2* K = reinterpret_cast<float2*>(scratch + b_grid + b_cnt + b_f + b_tw + b_a);
    int rc = WT_OK;
    const int64_t nf = static_cast<int64_t>(planes) * M * M;
    k_wp_field<<<static_cast<unsigned>(std::min<int64_t>((nf + 255) / 256, 8192)), 256, 0, s>>>(pl, f);
    k_wp_twiddles<<<(pl.T * M + 255) / 256, 256, 0, s>>>(pl, tw);
    k_wp_stage1<<<static_cast<unsigned>(planes * M), 128, 0, s>>>(pl, f, tw, a);
    k_wp_stage2<<<static_cast<unsigned>(planes * pl.T), 128, 0, s>>>(pl, a, tw, K);
    if (cudaGetLastError() != cudaSuccess) rc = set_error(WT_ERR_CUDA, "%s: kernel tables", fn);
    if (rc == WT_OK && (cudaMemsetAsync(grid, 0, static_cast<size_t>(nn) * sizeof(float2), s) != cudaSuccess ||
                        cudaMemsetAsync(count, 0, sizeof(unsigned long long), s) != cudaSuccess))
        rc = set_error(WT_ERR_CUDA, "%s: clearing the grid", fn);
    if (rc == WT_OK && n_vis > 0) {
        int64_t b = (n_vis + 7) / 8;                   // 8 warps per CTA, a warp per visibility
        const int64_t cap = static_cast<int64_t>(num_sms()) * 32;
        if (b > cap) b = cap;
        k_grid_wproj<<<static_cast<unsigned>(b), 256, 0, s>>>(pl, K, uvw, vis, n_vis, n, ndl, grid, count);
        if (cudaGetLastError() != cudaSuccess) rc = set_error(WT_ERR_CUDA, "%s: gridding launch", fn);
    }
    if (rc == WT_OK) rc = fft2_forward(grid, n, s);
    if (rc == WT_OK) {
        k_image_from_fft_wp<<<rows_blocks(n), kImgThreads, 0, s>>>(grid, n, count, image);
        if (cudaGetLastError() != cudaSuccess) rc = set_error(WT_ERR_CUDA, "%s: image launch", fn);
    }
    const cudaError_t ef = cudaFreeAsync(scratch, s);
    if (rc) return rc;
    if (ef != cudaSuccess) return cuda_error(ef, "cudaFreeAsync");
    return WT_OK;
}

}  // namespace
}  // namespace wt

extern "C" int wt_dirty_image_w(const double* uvw, const void* vis, int64_t n_vis, int n, double dl, int w_planes,
                                double w_max, float* image, void* stream)
{
    using namespace wt;
    const char* fn = "wt_dirty_image_w";
    int rc = check_image_args(fn, n, dl);
    if (rc) return rc;
    if (n_vis < 0) return set_error(WT_ERR_ARG, "%s: n_vis < 0", fn);
    if (w_planes < 2 || w_planes > 1024) return set_error(WT_ERR_ARG, "%s: w_planes = %d must be 2..1024", fn, w_planes);
    if (!(w_max >= 0.0) || !isfinite(w_max)) return set_error(WT_ERR_ARG, "%s: w_max must be finite and >= 0", fn);
    const size_t nn = static_cast<size_t>(n) * n;
    if ((rc = check_device_buffer(uvw, static_cast<size_t>(n_vis) * 24, fn, "uvw", 8)) ||
        (vis && (rc = check_device_buffer(vis, static_cast<size_t>(n_vis) * 8, fn, "vis", 8))) ||
        (rc = check_device_buffer(image, nn * 4, fn, "image", 4)))
        return rc;
    return dirty_image_w(uvw, static_cast<const float2*>(vis), n_vis, n, dl, w_planes, w_max, image,
                         static_cast<cudaStream_t>(stream));
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
                        int n_major, int w_planes, int* comp_pix, float* comp_flux, int* n_comp, void* vis_resid,
                        float* image_resid, void* stream)
{
    using namespace wt;
    const char* fn = "wt_clean";
    int rc = check_image_args(fn, n, dl);
    if (rc) return rc;
    if (n_vis < 0) return set_error(WT_ERR_ARG, "%s: n_vis < 0", fn);
    if (predictor != WT_PREDICT_TREE && predictor != WT_PREDICT_DIRECT)
        return set_error(WT_ERR_ARG, "%s: bad predictor %d", fn, predictor);
    if (mode != WT_MIXED && mode != WT_MIXED_FAST && !(mode == WT_MIXED_TC && predictor == WT_PREDICT_DIRECT))
        return set_error(WT_ERR_ARG,
                         "%s: mode must be WT_MIXED or WT_MIXED_FAST (complex64 visibilities), or WT_MIXED_TC with "
                         "the direct-sum predictor", fn);
    if (minor_iter < 0 || n_major < 0 || static_cast<int64_t>(minor_iter) * n_major > (1 << 24))
        return set_error(WT_ERR_ARG, "%s: minor_iter x n_major outside 0..2^24", fn);
    if (!(gain > 0.0f) || !(gain <= 1.0f)) return set_error(WT_ERR_RANGE, "%s: gain must be in (0, 1]", fn);
    if (!isfinite(threshold)) return set_error(WT_ERR_RANGE, "%s: threshold must be finite", fn);
    if (w_planes != 0 && (w_planes < 2 || w_planes > 1024))
        return set_error(WT_ERR_ARG, "%s: w_planes = %d must be 0 or 2..1024", fn, w_planes);
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
    // the imaging: nearest-cell without w, or w-projection planned for the
    // batch's largest |w| (found once)
    double w_max = 0.0;
    auto image_of = [&](const float2* v, float* out) {
        return w_planes ? dirty_image_w(uvw, v, n_vis, n, dl, w_planes, w_max, out, s)
                        : dirty_image(uvw, v, n_vis, n, dl, out, grid, count, s);
    };
    rc = w_planes ? max_abs_w(uvw, n_vis, s, &w_max) : WT_OK;
    // the tree predictor maps components through the cross-reference table
    // of the image pixels, built once (Sec. 3.5)
    if (!rc && tree) rc = wt_xref_table(n, dl, ra0, dec0, J, xref, stream);
    if (!rc) rc = image_of(nullptr, beam);
    if (!rc && n_vis > 0) {
        e = cudaMemcpyAsync(vis_resid, vis_obs, static_cast<size_t>(n_vis) * 8, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) rc = cuda_error(e, "cudaMemcpyAsync");
    }
    for (int cycle = 0; cycle < n_major && !rc; ++cycle) {
        // 3. gridding and FFT of the residuals, then the minor cycles
        if ((rc = image_of(static_cast<const float2*>(vis_resid), image_resid))) break;
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
    if (!rc) rc = image_of(static_cast<const float2*>(vis_resid), image_resid);
    *n_comp = total;
    const cudaError_t ef = cudaFreeAsync(scratch, s);
    if (rc) return rc;
    if (ef != cudaSuccess) return cuda_error(ef, "cudaFreeAsync");
    return WT_OK;
}
