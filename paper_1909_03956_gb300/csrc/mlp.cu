// mlp.cu -- the learned per-level visibility response (an addition to the
// paper's method, not in arXiv:1909.03956).
//
// What is learned. For level j, let P_j be the level-j pixel holding the
// phase centre, c_j its centre and s_i its 4^D descendants D levels down.
// The pixel response R_j(B) = 4^-D sum_i exp(i 2 pi B.(s_i - c_j)) is the
// plane wave's level-j scaling coefficient on a fully populated sub-tree
// (the Eq. 9 recursion), demodulated by the plane wave at the centre. A
// pixel whose flux fills it uniformly contributes
// Phi exp(i 2 pi B.(c - P)) R_j(B) instead of the centre-snapped term of
// Eq. 16, so the learned form of the tree prediction is
//     V_learned(B) = R_j(B) sum_k Phi_k exp(i 2 pi B.(c_k - P))      (j = J).
// A network 3 -> 64 -> 64 -> 2 (SiLU) maps x = B Delta theta_j to
// (Re R, Im R). Outside |x|_inf <= x_max (the trained domain) the exact sum
// is evaluated instead: exact evaluation is the fallback and the yardstick.
//
// Kernels:
//   k_response_offsets  s_i - c_j for the 4^D sub-pixels (float64)
//   k_response_exact    R_j(B) by the exact sum (float64, table sin/cos)
//   k_mlp_apply         inference on the tensor cores: the 64 x 64 layer as
//                       tcgen05.mma BF16 x BF16 -> FP32 into tensor memory,
//                       128 samples per MMA tile, FP32 for the 3 -> 64 and
//                       64 -> 2 layers; writes R or multiplies visibilities
//                       by it in place
//   k_mlp_train_grad    forward + backward over a batch (FP32, with the
//                       hidden activations and W2 rounded to BF16 in the
//                       forward pass exactly as the inference kernel sees
//                       them), gradients reduced per CTA then atomically
//   k_mlp_adam          Adam update of the FP32 master parameters
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <cuda_bf16.h>

#include <algorithm>
#include <random>
#include <vector>

#include "sphere.cuh"
#include "tcgen05.cuh"
#include "wt_internal.cuh"

namespace wt {
namespace {

constexpr int kH = 64;                                   // hidden width
constexpr int kNumParams = kH * 3 + kH + kH * kH + kH + 2 * kH + 2;   // 4546
constexpr int kPartStride = ((kNumParams + 1 + 3) / 4) * 4;            // a CTA's partial gradient and loss
// offsets into the flat parameter vector (same order as the CPU oracle)
constexpr int oW1 = 0, ob1 = oW1 + kH * 3, oW2 = ob1 + kH, ob2 = oW2 + kH * kH, oW3 = ob2 + kH, ob3 = oW3 + 2 * kH;

__device__ __forceinline__ float silu_f(float z) { return z / (1.0f + __expf(-z)); }

// SiLU for inference: z sigma(z) = z/2 (1 + tanh(z/2)) with the hardware
// tanh (PTX tanh.approx.f32, one special-function op; its absolute error of
// about 2^-11 is below the bfloat16 rounding the hidden units get anyway).
// Training keeps silu_f, so that its gradients match the oracle's.
__device__ __forceinline__ float silu_fast(float z)
{
    const float hz = 0.5f * z;
    float t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(hz));
    return fmaf(hz, t, hz);
}
// silu_fast on a pair (the same roundings per element).
__device__ __forceinline__ float2 silu_fast2(float2 z)
{
    const float2 hz = mul2(make_float2(0.5f, 0.5f), z);
    float2 t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t.x) : "f"(hz.x));
    asm("tanh.approx.f32 %0, %1;" : "=f"(t.y) : "f"(hz.y));
    return fma2(hz, t, hz);
}
__device__ __forceinline__ float dsilu_f(float z)
{
    const float s = 1.0f / (1.0f + __expf(-z));
    return s * (1.0f + z * (1.0f - s));
}
__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}


struct Rot {
    double r[9];
};

// ---------------------------------------------------------------- exact response
// Unit vector of nested pixel `pix` at `level` in the uvw frame, (s_u, s_v, s_w - 1).
__device__ void pixel_dir(int level, int64_t pix, const Rot& R, double* d)
{
    double z, st, ph, sph, cph;
    pixel_centre(level - 1, pix, z, st, ph);
    sincos(ph, &sph, &cph);
    const double x = st * sph, y = z, zc = st * cph;
    const double su = R.r[0] * x + R.r[3] * y + R.r[6] * zc;
    const double sv = R.r[1] * x + R.r[4] * y + R.r[7] * zc;
    const double sw = R.r[2] * x + R.r[5] * y + R.r[8] * zc;
    d[0] = su;
    d[1] = sv;
    d[2] = (sw > 0.0) ? -(su * su + sv * sv) / (1.0 + sw) : sw - 1.0;
}

// Level-j pixel holding the phase centre: the image point l = m = 0, mapped
// exactly as the tree build maps a component.
__device__ int64_t phase_centre_pixel(int level, const Rot& R)
{
    double phi = atan2(R.r[2], R.r[8]);
    if (phi < 0.0) phi = __dadd_rn(phi, 2.0 * kPi);
    if (phi >= 2.0 * kPi) phi = __dsub_rn(phi, 2.0 * kPi);
    return pixel_of(level - 1, R.r[5], phi);
}

__global__ void k_response_offsets(int level, int depth, Rot R, double* __restrict__ offs)
{
    const int64_t nsub = int64_t(1) << (2 * depth);
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= nsub) return;
    const int64_t kref = phase_centre_pixel(level, R);
    double c[3], s[3];
    pixel_dir(level, kref, R, c);
    pixel_dir(level + depth, (kref << (2 * depth)) + i, R, s);
    offs[3 * i + 0] = s[0] - c[0];
    offs[3 * i + 1] = s[1] - c[1];
    offs[3 * i + 2] = s[2] - c[2];
}

__device__ double2 response_exact_one(double u, double v, double w, const double* __restrict__ offs, int n_off)
{
    double re = 0.0, im = 0.0;
    for (int i = 0; i < n_off; ++i) {
        double t = fma(w, __ldg(&offs[3 * i + 2]), fma(v, __ldg(&offs[3 * i + 1]), u * __ldg(&offs[3 * i])));
        double s, c;
        sincos_turns_f64(t, s, c);
        re += c;
        im += s;
    }
    const double inv = 1.0 / static_cast<double>(n_off);
    return make_double2(re * inv, im * inv);
}

__global__ void k_response_exact(const double* __restrict__ uvw, int64_t n, const double* __restrict__ offs, int n_off,
                                 double sgn, double2* __restrict__ out)
{
    for (int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; q < n;
         q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const double2 r = response_exact_one(uvw[3 * q], uvw[3 * q + 1], uvw[3 * q + 2], offs, n_off);
        out[q] = make_double2(r.x, sgn * r.y);
    }
}

// ---------------------------------------------------------------- inference
struct MlpDev {
    const float* params;        // FP32 master, oracle layout
    const uint32_t* w2_bf16x2;  // W2 as bf16 pairs, row n: W2[n][2p], W2[n][2p+1] -> [n * 32 + p]
};

// One sample per thread; a CTA's 128 samples are the M = 128 rows of one
// tcgen05 MMA tile (N = 64 hidden units, K = 64 inputs).
constexpr int kApplyThreads = 128;
constexpr uint32_t kTmemCols = 64;   // the 128 x 64 FP32 accumulator

// Instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator, BF16 A
// and B, both K-major, M = 128, N = 64.
constexpr uint32_t kMlpIdesc = idesc_f16(true, 128, 64);

// Inference of the 3 -> 64 -> 64 -> 2 network on the 5th-generation tensor
// cores. Per tile of 128 samples: every thread computes its sample's first
// layer in FP32 (SiLU, rounded to BF16) straight into the A operand in
// shared memory; one thread issues four tcgen05.mma (K = 16 each) against
// W2 (the B operand, staged once per CTA) into a 128 x 64 FP32 accumulator
// in tensor memory and commits to an mbarrier; every thread then reads its
// accumulator row (tcgen05.ld), adds b2, applies SiLU and the 64 -> 2 layer
// in FP32. Waits are bounded: a wait that runs out records WT_ERR_TIMEOUT,
// waits once more for the MMA in flight, frees the tensor memory and leaves.
// Eight CTAs per SM: 64 registers per thread (the accumulator row read in
// two halves of 32 columns) and 8 x 64 tensor-memory columns, all of an SM's.
template <bool APPLY>
__global__ void __launch_bounds__(kApplyThreads, 8) k_mlp_apply(MlpDev p, const double* __restrict__ uvw, int64_t n,
                                                             float2* __restrict__ io, float scale, int sign,
                                                             float x_max, const double* __restrict__ offs, int n_off,
                                                             int* status)
{
    __shared__ __align__(1024) unsigned char sA[128 * kH * 2];
    __shared__ __align__(1024) unsigned char sB[kH * kH * 2];
    // the small layers' parameters, laid out for one 16-byte load per two
    // packed pairs: for units (2q, 2q + 1) sL1a[q] = W1 columns 0 and 1,
    // sL1b[q] = W1 column 2 and b1; for units (c, c + 1) sW3q[c / 2] = W3's
    // two outputs of unit c, then of unit c + 1; sb2q[j] = b2 of units 4j .. 4j + 3
    __shared__ float4 sL1a[kH / 2], sL1b[kH / 2], sW3q[kH / 2], sb2q[kH / 4];
    __shared__ float sb3[2];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_base;
    const int t = threadIdx.x;
    for (int q = t; q < kH / 2; q += kApplyThreads) {
        const float* w1a = p.params + oW1 + 3 * (2 * q);   // W1 row of unit 2q, then of unit 2q + 1
        sL1a[q] = make_float4(w1a[0], w1a[3], w1a[1], w1a[4]);
        sL1b[q] = make_float4(w1a[2], w1a[5], p.params[ob1 + 2 * q], p.params[ob1 + 2 * q + 1]);
        sW3q[q] = make_float4(p.params[oW3 + 2 * q], p.params[oW3 + kH + 2 * q], p.params[oW3 + 2 * q + 1],
                              p.params[oW3 + kH + 2 * q + 1]);
    }
    for (int j = t; j < kH / 4; j += kApplyThreads)
        sb2q[j] = make_float4(p.params[ob2 + 4 * j], p.params[ob2 + 4 * j + 1], p.params[ob2 + 4 * j + 2],
                              p.params[ob2 + 4 * j + 3]);
    if (t < 2) sb3[t] = p.params[ob3 + t];
    for (int i = t; i < kH * kH / 2; i += kApplyThreads)   // W2 row n = output unit: K-major B
        *reinterpret_cast<uint32_t*>(sB + umma_off(i / 32, 2 * (i % 32))) = __ldg(&p.w2_bf16x2[i]);
    if (t == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    if (t < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tm = tmem_base;
    const uint32_t row_addr = tm + (static_cast<uint32_t>(t & ~31) << 16);   // this warp's lanes
    const uint32_t a_addr = smem_addr(sA), b_addr = smem_addr(sB);
    uint32_t phase = 0;
    const int64_t tiles = (n + 127) / 128;
    // the baselines of this thread's sample in the CTA's next tile, loaded
    // one tile ahead so that their latency overlaps the current tile's work
    double nu = 0.0, nv = 0.0, nw = 0.0;
    {
        const int64_t s0 = static_cast<int64_t>(blockIdx.x) * 128 + t;
        if (blockIdx.x < tiles && s0 < n) {
            nu = uvw[3 * s0];
            nv = uvw[3 * s0 + 1];
            nw = uvw[3 * s0 + 2];
        }
    }
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t s = tile * 128 + t;
        const bool live = s < n;
        const double bu = nu, bv = nv, bw = nw;
        float x[3] = {0.f, 0.f, 0.f};
        if (live) {
            x[0] = static_cast<float>(bu) * scale;
            x[1] = static_cast<float>(bv) * scale;
            x[2] = static_cast<float>(bw) * scale;
        }
        {
            const int64_t s1 = (tile + gridDim.x) * 128 + t;
            if (tile + gridDim.x < tiles && s1 < n) {
                nu = uvw[3 * s1];
                nv = uvw[3 * s1 + 1];
                nw = uvw[3 * s1 + 2];
            }
        }
        // layer 1 into row t of A, one 16-byte core-matrix row (8 units) at a
        // time, two units per packed operation (the scalar order of the FMAs)
        const float2 x0 = bcast2(x[0]), x1 = bcast2(x[1]), x2 = bcast2(x[2]);
#pragma unroll
        for (int kg = 0; kg < 8; ++kg) {
            uint32_t w[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int q = 4 * kg + e;                              // units 2q, 2q + 1
                const float4 a = sL1a[q], b = sL1b[q];
                const float2 z = fma2(make_float2(b.x, b.y), x2,
                                      fma2(make_float2(a.z, a.w), x1,
                                           fma2(make_float2(a.x, a.y), x0, make_float2(b.z, b.w))));
                const float2 h = silu_fast2(z);
                w[e] = pack_bf16x2(h.x, h.y);
            }
            *reinterpret_cast<uint4*>(sA + umma_off(t, 8 * kg)) = make_uint4(w[0], w[1], w[2], w[3]);
        }
        // the generic-proxy writes of A before the tensor cores read it
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (t == 0) {
#pragma unroll
            for (int kk = 0; kk < kH / 16; ++kk) {   // 16 columns = two core matrices = 256 bytes along K
                const uint64_t ad = umma_desc(a_addr + kk * 256), bd = umma_desc(b_addr + kk * 256);
                const uint32_t acc = kk > 0;
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tm),
                    "l"(ad), "l"(bd), "r"(kMlpIdesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_addr(&bar))
                         : "memory");
        }
        const bool done = mbar_wait_parity(&bar, phase);
        if (!__syncthreads_and(done)) {
            if (t == 0) record_status(status, WT_ERR_TIMEOUT);
            mbar_wait_parity(&bar, phase);   // once more for the MMA in flight
            break;
        }
        phase ^= 1u;
        tc_fence_after();
        // the accumulator row in two halves of 32 columns, each folded into
        // layer 3 at once (the same order of operations as one pass)
        float2 ro = make_float2(sb3[0], sb3[1]);                       // (real, imaginary) output
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            uint32_t r[32];
            tmem_ld32(row_addr + 32 * half, r);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int cc = 0; cc < 32; cc += 4) {
                const int c = 32 * half + cc;                          // units c .. c + 3
                const float4 b2 = sb2q[c / 4];
#pragma unroll
                for (int e = 0; e < 2; ++e) {                          // units c + 2e, c + 2e + 1
                    const float2 h = silu_fast2(
                        add2(make_float2(__uint_as_float(r[cc + 2 * e]), __uint_as_float(r[cc + 2 * e + 1])),
                             e ? make_float2(b2.z, b2.w) : make_float2(b2.x, b2.y)));
                    const float4 w3 = sW3q[c / 2 + e];
                    ro = fma2(make_float2(w3.x, w3.y), bcast2(h.x), ro);
                    ro = fma2(make_float2(w3.z, w3.w), bcast2(h.y), ro);
                }
            }
        }
        float rr = ro.x, ri = ro.y;
        if (live) {
            if (fmaxf(fabsf(x[0]), fmaxf(fabsf(x[1]), fabsf(x[2]))) > x_max) {
                const double2 e = response_exact_one(bu, bv, bw, offs, n_off);
                rr = static_cast<float>(e.x);
                ri = static_cast<float>(e.y);
            }
            if (sign < 0) ri = -ri;
            if (APPLY) {
                const float2 v = io[s];
                io[s] = make_float2(v.x * rr - v.y * ri, v.x * ri + v.y * rr);
            } else {
                io[s] = make_float2(rr, ri);
            }
        }
        tc_fence_before();   // this tile's accumulator reads before the next tile's MMA
    }
    __syncthreads();
    tc_fence_after();
    if (t < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(kTmemCols) : "memory");
}

__global__ void k_w2_to_bf16(const float* __restrict__ params, uint32_t* __restrict__ w2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;   // pair index
    if (i >= kH * kH / 2) return;
    const int nrow = i / 32, pcol = i % 32;
    w2[i] = pack_bf16x2(params[oW2 + nrow * kH + 2 * pcol], params[oW2 + nrow * kH + 2 * pcol + 1]);
}

// ---------------------------------------------------------------- training
constexpr int kTrainThreads = 256;
constexpr int kS = 64;   // samples per CTA tile

struct TrainSmem {
    float x[kS][3];
    float t[kS][2];
    float dy[kS][2];
    float valid[kS];
    float z1[kS][kH];    // pre-activation, later dz1
    float h1[kS][kH];    // bf16-rounded activation
    float z2[kS][kH];
    float h2[kS][kH];
    float dz2[kS][kH];
    float W2q[kH][kH];   // bf16-rounded W2
    float W1[kH * 3], b1[kH], b2[kH], W3[2 * kH], b3[2];
    float gW1[kH * 3], gb1[kH], gb2[kH], gW3[2 * kH], gb3[2];
    float e2[kS][2];     // squared errors of the current samples
    float loss;
};

__global__ void __launch_bounds__(kTrainThreads) k_mlp_train_grad(const float* __restrict__ params,
                                                                  const double* __restrict__ uvw,
                                                                  const float* __restrict__ target, int64_t first,
                                                                  int64_t count, int64_t n_total, int64_t n_data,
                                                                  float scale, float* __restrict__ part)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TrainSmem& sm = *reinterpret_cast<TrainSmem*>(smem_raw);
    const int tid = threadIdx.x;
    for (int i = tid; i < kH * kH; i += blockDim.x) sm.W2q[i / kH][i % kH] = bf16_round(params[oW2 + i]);
    for (int i = tid; i < kH * 3; i += blockDim.x) {
        sm.W1[i] = params[oW1 + i];
        sm.gW1[i] = 0.f;
    }
    for (int i = tid; i < kH; i += blockDim.x) {
        sm.b1[i] = params[ob1 + i];
        sm.b2[i] = params[ob2 + i];
        sm.gb1[i] = 0.f;
        sm.gb2[i] = 0.f;
    }
    for (int i = tid; i < 2 * kH; i += blockDim.x) {
        sm.W3[i] = params[oW3 + i];
        sm.gW3[i] = 0.f;
    }
    if (tid < 2) {
        sm.b3[tid] = params[ob3 + tid];
        sm.gb3[tid] = 0.f;
    }
    if (tid == 0) sm.loss = 0.f;
    float gW2[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) gW2[i] = 0.f;
    __syncthreads();
    const float inv_n = 1.0f / static_cast<float>(n_total);
    for (int64_t base = first + static_cast<int64_t>(blockIdx.x) * kS; base < first + count;
         base += static_cast<int64_t>(gridDim.x) * kS) {
        // samples wrap around the data set (minibatches are contiguous slices)
        if (tid < kS) {
            const int64_t q = base + tid;
            const bool ok = q < first + count;
            const int64_t qq = ok ? (q % n_data) : 0;
            for (int d = 0; d < 3; ++d) sm.x[tid][d] = ok ? static_cast<float>(uvw[3 * qq + d]) * scale : 0.f;
            sm.t[tid][0] = ok ? target[2 * qq] : 0.f;
            sm.t[tid][1] = ok ? target[2 * qq + 1] : 0.f;
            sm.valid[tid] = ok ? 1.f : 0.f;
        }
        __syncthreads();
        for (int e = tid; e < kS * kH; e += blockDim.x) {
            const int s = e / kH, k = e % kH;
            const float z = fmaf(sm.W1[3 * k + 2], sm.x[s][2], fmaf(sm.W1[3 * k + 1], sm.x[s][1],
                                                                    fmaf(sm.W1[3 * k], sm.x[s][0], sm.b1[k])));
            sm.z1[s][k] = z;
            sm.h1[s][k] = bf16_round(silu_f(z));
        }
        __syncthreads();
        for (int e = tid; e < kS * kH; e += blockDim.x) {
            const int s = e / kH, o = e % kH;
            float z = sm.b2[o];
#pragma unroll 16
            for (int k = 0; k < kH; ++k) z = fmaf(sm.W2q[o][k], sm.h1[s][k], z);
            sm.z2[s][o] = z;
            sm.h2[s][o] = silu_f(z);
        }
        __syncthreads();
        if (tid < 2 * kS) {
            const int s = tid >> 1, o = tid & 1;
            float y = sm.b3[o];
            for (int k = 0; k < kH; ++k) y = fmaf(sm.W3[o * kH + k], sm.h2[s][k], y);
            const float err = (sm.valid[s] != 0.f) ? y - sm.t[s][o] : 0.f;
            sm.e2[s][o] = err * err;
            sm.dy[s][o] = 2.f * err * inv_n;
        }
        __syncthreads();
        if (tid == 0) {   // in sample order: the same sum on every run
            for (int q = 0; q < kS; ++q) sm.loss += sm.e2[q][0] + sm.e2[q][1];
        }
        for (int e = tid; e < kS * kH; e += blockDim.x) {
            const int s = e / kH, o = e % kH;
            const float dh = sm.dy[s][0] * sm.W3[o] + sm.dy[s][1] * sm.W3[kH + o];
            sm.dz2[s][o] = dh * dsilu_f(sm.z2[s][o]);
        }
        if (tid < 2 * kH) {
            const int o2 = tid / kH, k = tid % kH;
            float a = 0.f;
            for (int s = 0; s < kS; ++s) a = fmaf(sm.dy[s][o2], sm.h2[s][k], a);
            sm.gW3[tid] += a;
        }
        if (tid < 2) {
            float a = 0.f;
            for (int s = 0; s < kS; ++s) a += sm.dy[s][tid];
            sm.gb3[tid] += a;
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int e = tid + kTrainThreads * i, o = e / kH, k = e % kH;
            float a = 0.f;
            for (int s = 0; s < kS; ++s) a = fmaf(sm.dz2[s][o], sm.h1[s][k], a);
            gW2[i] += a;
        }
        if (tid < kH) {
            float a = 0.f;
            for (int s = 0; s < kS; ++s) a += sm.dz2[s][tid];
            sm.gb2[tid] += a;
        }
        for (int e = tid; e < kS * kH; e += blockDim.x) {
            const int s = e / kH, k = e % kH;
            float dh = 0.f;
#pragma unroll 16
            for (int o = 0; o < kH; ++o) dh = fmaf(sm.dz2[s][o], sm.W2q[o][k], dh);
            sm.z1[s][k] = dh * dsilu_f(sm.z1[s][k]);   // dz1, in place
        }
        __syncthreads();
        if (tid < kH) {
            float a = 0.f;
            for (int s = 0; s < kS; ++s) a += sm.z1[s][tid];
            sm.gb1[tid] += a;
        }
        if (tid < kH * 3) {
            const int k = tid / 3, d = tid % 3;
            float a = 0.f;
            for (int s = 0; s < kS; ++s) a = fmaf(sm.z1[s][k], sm.x[s][d], a);
            sm.gW1[tid] += a;
        }
        __syncthreads();
    }
    // this CTA's partial gradient and loss: its own row of `part`, summed
    // over the rows in order by k_mlp_reduce (no atomics: every run of the
    // same steps gives the same parameters, bit for bit)
    float* row = part + static_cast<int64_t>(blockIdx.x) * kPartStride;
#pragma unroll
    for (int i = 0; i < 16; ++i) row[oW2 + tid + kTrainThreads * i] = gW2[i];
    for (int i = tid; i < kH * 3; i += blockDim.x) row[oW1 + i] = sm.gW1[i];
    for (int i = tid; i < kH; i += blockDim.x) {
        row[ob1 + i] = sm.gb1[i];
        row[ob2 + i] = sm.gb2[i];
    }
    for (int i = tid; i < 2 * kH; i += blockDim.x) row[oW3 + i] = sm.gW3[i];
    if (tid < 2) row[ob3 + tid] = sm.gb3[tid];
    if (tid == 0) row[kNumParams] = sm.loss * inv_n;
}

// grad[i] = sum over the rows r = 0 .. rows - 1 of part[r][i], in row
// order; the loss likewise.
__global__ void k_mlp_reduce(const float* __restrict__ part, int rows, float* __restrict__ grad,
                             float* __restrict__ loss)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > kNumParams) return;
    float a = 0.f;
    for (int r = 0; r < rows; ++r) a += part[static_cast<int64_t>(r) * kPartStride + i];
    if (i < kNumParams) grad[i] = a;
    else *loss = a;
}

__global__ void k_mlp_adam(float* __restrict__ params, float* __restrict__ m, float* __restrict__ v,
                           float* __restrict__ grad, float lr, float b1c, float b2c)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kNumParams) return;
    const float g = grad[i];
    const float mi = 0.9f * m[i] + 0.1f * g;
    const float vi = 0.999f * v[i] + 0.001f * g * g;
    m[i] = mi;
    v[i] = vi;
    params[i] -= lr * (mi / b1c) / (sqrtf(vi / b2c) + 1e-8f);
    grad[i] = 0.f;
}

}  // namespace
}  // namespace wt

// ===========================================================================
// Host side: the wt_mlp handle and the C entry points.
// ===========================================================================
struct wt_mlp_s {
    uint64_t magic;
    int device;
    int level, depth;
    float x_max;
    double ra0, dec0;
    void* block;                 // params, m, v, grad, loss, w2 bf16, offsets
    float* params;
    float* m;
    float* v;
    float* grad;
    float* loss;
    uint32_t* w2;
    double* offs;
    int n_off;
    int adam_t;
    float* part;                 // per-CTA partial gradients [part_rows][kPartStride]
    int part_rows;
};

namespace {
constexpr uint64_t kMlpMagic = 0x4d4c505f57543031ull;   // "MLP_WT01"

int check_mlp(wt_mlp m, const char* fn)
{
    using namespace wt;
    if (!m) return set_error(WT_ERR_ARG, "%s: mlp is NULL", fn);
    if (m->magic != kMlpMagic) return set_error(WT_ERR_CORRUPT, "%s: not a live mlp handle", fn);
    int dev = 0;
    WT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != m->device) return set_error(WT_ERR_ARG, "%s: mlp lives on device %d", fn, m->device);
    return WT_OK;
}

int refresh_bf16(wt_mlp m, cudaStream_t s)
{
    wt::k_w2_to_bf16<<<(wt::kH * wt::kH / 2 + 255) / 256, 256, 0, s>>>(m->params, m->w2);
    WT_CUDA_TRY(cudaGetLastError());
    return WT_OK;
}

int launch_apply(wt_mlp m, const double* uvw, int64_t n, void* io, int sign, bool apply, cudaStream_t s)
{
    using namespace wt;
    const float scale = static_cast<float>(ldexp(sqrt(kPi / 3.0), 1 - m->level));   // Delta theta_j
    MlpDev p{m->params, m->w2};
    int* status = device_status_word();
    if (!status) return set_error(WT_ERR_CUDA, "wt_mlp: no device status word");
    // CTAs of 128 samples, as many as the registers and shared memory let
    // reside on an SM (each holds 64 tensor-memory columns: at most 8 per SM)
    auto kern = apply ? k_mlp_apply<true> : k_mlp_apply<false>;
    cudaFuncAttributes fa;
    WT_CUDA_TRY(cudaFuncGetAttributes(&fa, kern));
    const int by_regs = fa.numRegs > 0 ? 65536 / (fa.numRegs * kApplyThreads) : 8;
    const int by_smem = static_cast<int>((227 * 1024) / (fa.sharedSizeBytes + 1024));
    int per_sm = std::min(std::min(by_regs, by_smem), 8);
    if (per_sm < 1) return set_error(WT_ERR_UNSUPPORTED, "wt_mlp: inference kernel does not fit on an SM");
    const int64_t tiles = (n + 127) / 128;
    int64_t blocks = static_cast<int64_t>(num_sms()) * per_sm;
    if (blocks > tiles) blocks = tiles;
    if (blocks < 1) blocks = 1;
    kern<<<static_cast<unsigned>(blocks), kApplyThreads, 0, s>>>(p, uvw, n, static_cast<float2*>(io), scale, sign,
                                                                 m->x_max, m->offs, m->n_off, status);
    WT_CUDA_TRY(cudaGetLastError());
    return WT_OK;
}

int run_grad(wt_mlp m, const double* uvw, const float* target, int64_t first, int64_t count, int64_t n_data,
             cudaStream_t s)
{
    using namespace wt;
    const size_t smem = sizeof(TrainSmem);
    WT_CUDA_TRY(cudaFuncSetAttribute(k_mlp_train_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(smem)));
    const float scale = static_cast<float>(ldexp(sqrt(kPi / 3.0), 1 - m->level));
    int64_t blocks = (count + kS - 1) / kS;
    const int64_t cap = static_cast<int64_t>(num_sms()) * 2;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    if (blocks > m->part_rows) blocks = m->part_rows;
    k_mlp_train_grad<<<static_cast<unsigned>(blocks), kTrainThreads, smem, s>>>(
        m->params, uvw, target, first, count, count, n_data, scale, m->part);
    k_mlp_reduce<<<(kNumParams + 1 + 255) / 256, 256, 0, s>>>(m->part, static_cast<int>(blocks), m->grad, m->loss);
    WT_CUDA_TRY(cudaGetLastError());
    return WT_OK;
}
}  // namespace

namespace wt {
namespace {
// ---------------------------------------------------------------- truncated tree
// The tree's level-`level` nodes as Eq. 16 leaf records (RecF): the pixel
// centre (s_u, s_v, s_w - 1) as double-float pairs and g = F_k =
// A_level lambda_level,k, the flux of the node's pixel (Eq. 9 averages the
// children, so A_j lambda_j,k is the merged flux below the node); and a
// header view whose n_leaves is their count, for the Eq. 16 kernel. The
// nodes of level j sit at rev_offset[j] .. + per_level[j] of the tree's
// level-J-first arrays, in key order.
__global__ void k_level_records(const int64_t* __restrict__ key, const double* __restrict__ lambda,
                                const TreeHeader* __restrict__ hdr, int level, Rot R, RecF* __restrict__ out,
                                TreeHeader* __restrict__ view, int64_t cap)
{
    int64_t n = hdr->per_level[level];
    n = n < cap ? n : cap;
    const int64_t base = hdr->rev_offset[level];
    const int64_t i0 = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i0 == 0) {
        view->n_leaves = n;
        view->n_nodes = n;
    }
    const double A = ldexp(kPi / 3.0, 2 * (1 - level));
    uint32_t bu = 0, bv = 0, bw = 0;
    for (int64_t i = i0; i < n; i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        double c[3];
        pixel_dir(level, key[base + i], R, c);
        const F2 a = split_f64(c[0]), b = split_f64(c[1]), e = split_f64(c[2]);
        RecF r;
        r.meta = kRecLeaf;
        r.a = a.hi;
        r.b = a.lo;
        r.c = b.hi;
        r.d = b.lo;
        r.e = e.hi;
        r.f = e.lo;
        r.g = static_cast<float>(A * lambda[base + i]);
        out[i] = r;
        bu = max(bu, __float_as_uint(fabsf(a.hi)));
        bv = max(bv, __float_as_uint(fabsf(b.hi)));
        bw = max(bw, __float_as_uint(fabsf(e.hi)));
    }
    // the records' coordinate bounds for the grid pass (view->smax zeroed
    // before the launch; non-negative floats order as their bits)
    bu = __reduce_max_sync(0xffffffffu, bu);
    bv = __reduce_max_sync(0xffffffffu, bv);
    bw = __reduce_max_sync(0xffffffffu, bw);
    if ((threadIdx.x & 31) == 0) {
        uint32_t* sm = reinterpret_cast<uint32_t*>(view->smax);
        if (bu) atomicMax(&sm[0], bu);
        if (bv) atomicMax(&sm[1], bv);
        if (bw) atomicMax(&sm[2], bw);
    }
}

// vis *= R, element by element (complex64 by complex128, formed in float64).
__global__ void k_mul_response(float2* __restrict__ vis, const double2* __restrict__ r, int64_t n)
{
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const float2 v = vis[i];
        const double2 q = r[i];
        const double vr = v.x, vi = v.y;
        vis[i] = make_float2(static_cast<float>(vr * q.x - vi * q.y), static_cast<float>(vr * q.y + vi * q.x));
    }
}

// ---------------------------------------------------------------- thresholded tree
// Exclusive prefix sum of one int per thread over a CTA of blockDim.x (a
// multiple of 32, at most 1024) threads; total receives the CTA's sum.
__device__ int cta_exclusive_scan(int x, int& total, int* warp_sums)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_sums[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int v = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        warp_sums[lane] = v;
    }
    __syncthreads();
    const int before = warp > 0 ? warp_sums[warp - 1] : 0;
    total = warp_sums[nw - 1];
    __syncthreads();
    return before + inc - x;
}

// Records of the kept details, level by level, in one CTA (deterministic:
// parents in key order, children in slot order). For each parent p at level
// j = j0 .. J-1 with at least one |gamma^m_p| >= tau, its four children at
// level j + 1 (present in the tree or not) get the records of their pixel
// centres with weights
//   w_c = (sqrt(A_j)/4) sum_{m kept} H_m[c] gamma^m_p,
// the kept coefficients' sum_m gamma^m sigma^m regrouped over the children
// (sigma^m = (sqrt(A_j)/4) H_m . eta_children, Eq. 10 form). The records of
// level L = j + 1 go to out + seg[L], its count into views[L - j0].
struct LevelSegs {
    int64_t off[kMaxJ + 2];   // first record of level L's segment
};

__global__ void __launch_bounds__(1024) k_threshold_records(const int64_t* __restrict__ key,
                                                            const double* __restrict__ gamma,
                                                            const TreeHeader* __restrict__ hdr, int j0, int J,
                                                            double tau, Rot R, RecF* __restrict__ out, LevelSegs seg,
                                                            TreeHeader* __restrict__ views)
{
    __shared__ int ws[32];
    __shared__ uint32_t wb[3][32];
    for (int j = j0; j < J; ++j) {
        const int64_t n = hdr->per_level[j];
        const int64_t base = hdr->rev_offset[j];
        RecF* dst = out + seg.off[j + 1];
        const double q = __dmul_rn(ldexp(__dsqrt_rn(kPi / 3.0), 1 - j), 0.25);
        int64_t carry = 0;
        uint32_t bu = 0, bv = 0, bw = 0;   // the level's coordinate bounds (float bits)
        for (int64_t start = 0; start < n; start += blockDim.x) {
            const int64_t i = start + threadIdx.x;
            double g[3] = {0.0, 0.0, 0.0};
            bool kept = false;
            if (i < n) {
#pragma unroll
                for (int mm = 0; mm < 3; ++mm) {
                    const double x = gamma[3 * (base + i) + mm];
                    if (fabs(x) >= tau) {
                        g[mm] = x;
                        kept = true;
                    }
                }
            }
            int total;
            const int pos = cta_exclusive_scan(kept ? 1 : 0, total, ws);
            if (kept) {
                const int64_t kp = key[base + i];
                for (int c = 0; c < 4; ++c) {
                    const double h0 = (c & 1) ? -1.0 : 1.0;                          // + - + -
                    const double h1 = (c & 2) ? -1.0 : 1.0;                          // + + - -
                    const double h2 = (((c & 1) ^ ((c >> 1) & 1)) != 0) ? -1.0 : 1.0;   // + - - +
                    double d[3];
                    pixel_dir(j + 1, 4 * kp + c, R, d);
                    const F2 a = split_f64(d[0]), b = split_f64(d[1]), e = split_f64(d[2]);
                    RecF r;
                    r.meta = kRecLeaf;
                    r.a = a.hi;
                    r.b = a.lo;
                    r.c = b.hi;
                    r.d = b.lo;
                    r.e = e.hi;
                    r.f = e.lo;
                    r.g = static_cast<float>(q * ((h0 * g[0] + h1 * g[1]) + h2 * g[2]));
                    dst[4 * (carry + pos) + c] = r;
                    bu = max(bu, __float_as_uint(fabsf(a.hi)));
                    bv = max(bv, __float_as_uint(fabsf(b.hi)));
                    bw = max(bw, __float_as_uint(fabsf(e.hi)));
                }
            }
            carry += total;
        }
        bu = __reduce_max_sync(0xffffffffu, bu);
        bv = __reduce_max_sync(0xffffffffu, bv);
        bw = __reduce_max_sync(0xffffffffu, bw);
        if ((threadIdx.x & 31) == 0) {
            wb[0][threadIdx.x >> 5] = bu;
            wb[1][threadIdx.x >> 5] = bv;
            wb[2][threadIdx.x >> 5] = bw;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            TreeHeader& vw = views[j + 1 - j0];
            vw.n_leaves = 4 * carry;
            vw.n_nodes = 4 * carry;
            uint32_t m[3] = {0, 0, 0};
            for (int k = 0; k < static_cast<int>(blockDim.x + 31) / 32; ++k)
                for (int c = 0; c < 3; ++c) m[c] = max(m[c], wb[c][k]);
            for (int c = 0; c < 3; ++c) vw.smax[c] = __uint_as_float(m[c]);
            vw.smax[3] = 0.f;
        }
        __syncthreads();
    }
}

// vis += x, element by element.
__global__ void k_accumulate(float2* __restrict__ vis, const float2* __restrict__ x, int64_t n)
{
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const float2 a = vis[i], b = x[i];
        vis[i] = make_float2(a.x + b.x, a.y + b.y);
    }
}

}  // namespace
}  // namespace wt

using namespace wt;

extern "C" {

int wt_predict_vis_truncated(wt_tree t, int level, int response, wt_mlp m, int depth, const double* uvw,
                             int64_t n_vis, void* vis_out, int sign, void* stream)
{
    const char* fn = "wt_predict_vis_truncated";
    if (!t || t->magic != kTreeMagic) return set_error(WT_ERR_ARG, "%s: bad tree handle", fn);
    if (level < 1 || level > t->J) return set_error(WT_ERR_RANGE, "%s: level %d outside 1..J = %d", fn, level, t->J);
    if (n_vis < 0 || (sign != 1 && sign != -1)) return set_error(WT_ERR_ARG, "%s: bad n_vis or sign", fn);
    int rc;
    if (response == WT_RESPONSE_LEARNED) {
        if ((rc = check_mlp(m, fn))) return rc;
        if (m->level != level)
            return set_error(WT_ERR_ARG, "%s: the network is for level %d, not %d", fn, m->level, level);
        if (t->ra0 != m->ra0 || t->dec0 != m->dec0)
            return set_error(WT_ERR_ARG, "%s: tree and network have different phase centres", fn);
    } else if (response == WT_RESPONSE_EXACT) {
        if (depth < 0 || depth > 8 || level + depth > kMaxJ)
            return set_error(WT_ERR_RANGE, "%s: need 0 <= depth <= 8 and level + depth <= %d", fn, kMaxJ);
    } else if (response != WT_RESPONSE_SNAPPED) {
        return set_error(WT_ERR_ARG, "%s: bad response %d", fn, response);
    }
    if ((rc = check_device_buffer(uvw, static_cast<size_t>(n_vis) * 24, fn, "uvw", 8)) ||
        (rc = check_device_buffer(vis_out, static_cast<size_t>(n_vis) * 8, fn, "vis_out", 8)))
        return rc;
    if (n_vis == 0) return WT_OK;
    int* status = device_status_word();
    if (!status) return set_error(WT_ERR_CUDA, "%s: no device status word", fn);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // scratch: the header view, the level's records, and for the exact
    // response the sub-pixel offsets and R(B) per visibility
    const int64_t cap = t->cap_leaves > 0 ? t->cap_leaves : 1;
    const int n_off = response == WT_RESPONSE_EXACT ? 1 << (2 * depth) : 0;
    const size_t rec_bytes = ((static_cast<size_t>(cap) * sizeof(RecF)) + 255) & ~size_t(255);
    const size_t off_bytes = ((sizeof(double) * 3 * static_cast<size_t>(n_off)) + 255) & ~size_t(255);
    const size_t r_bytes = response == WT_RESPONSE_EXACT ? sizeof(double2) * static_cast<size_t>(n_vis) : 0;
    const size_t hdr_bytes = (sizeof(TreeHeader) + 255) & ~size_t(255);
    char* scratch = nullptr;
    cudaError_t e =
        cudaMallocAsync(reinterpret_cast<void**>(&scratch), hdr_bytes + rec_bytes + off_bytes + r_bytes, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(WT_ERR_NOMEM, "%s: scratch allocation failed: %s", fn, cudaGetErrorString(e));
    }
    TreeHeader* view = reinterpret_cast<TreeHeader*>(scratch);
    RecF* recs = reinterpret_cast<RecF*>(scratch + hdr_bytes);
    double* offs = reinterpret_cast<double*>(scratch + hdr_bytes + rec_bytes);
    double2* resp = reinterpret_cast<double2*>(scratch + hdr_bytes + rec_bytes + off_bytes);
    Rot R;
    rotation_matrix(t->ra0, t->dec0, R.r);
    int64_t blocks = (cap + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (cudaMemsetAsync(view->smax, 0, sizeof(view->smax), s) != cudaSuccess) {
        cudaGetLastError();
        cudaFreeAsync(scratch, s);
        return set_error(WT_ERR_CUDA, "%s: clearing the bounds", fn);
    }
    k_level_records<<<static_cast<unsigned>(blocks), 256, 0, s>>>(t->d.key, t->d.lambda, t->d.hdr, level, R, recs,
                                                                  view, cap);
    rc = (cudaGetLastError() == cudaSuccess) ? WT_OK : set_error(WT_ERR_CUDA, "%s: level records launch", fn);
    // the level's size (the tree's header on the host): a large level's sum
    // runs with its phases on the tensor cores
    int64_t level_nodes = -1;
    if (rc == WT_OK && tree_sync_header(t) == WT_OK) level_nodes = t->host_hdr->per_level[level];
    if (rc == WT_OK && level_nodes >= WT_TRUNCATED_TC_MIN_NODES) {
        rc = eq16_tc_launch(recs, view, cap, level_nodes, uvw, n_vis, static_cast<float2*>(vis_out), sign, status, s,
                            fn);
    } else if (rc == WT_OK) {
        // Eq. 16 over the level's pixel centres, in the fast mixed form
        WaveletJob jb{};
        jb.recf_leaf = recs;
        jb.hdr = view;
        jb.uvw = uvw;
        jb.n_vis = n_vis;
        jb.vis = vis_out;
        jb.mode = WT_MIXED_FAST;
        jb.sign = sign;
        jb.which = WT_SUM_EQ16;
        jb.J = t->J;
        jb.status = status;
        rc = launch_wavelet(jb, default_wavelet_variant(WT_MIXED_FAST, WT_SUM_EQ16, t->J), s);
    }
    if (rc == WT_OK && response == WT_RESPONSE_LEARNED) rc = launch_apply(m, uvw, n_vis, vis_out, sign, true, s);
    if (rc == WT_OK && response == WT_RESPONSE_EXACT) {
        k_response_offsets<<<(n_off + 127) / 128, 128, 0, s>>>(level, depth, R, offs);
        int64_t b2 = (n_vis + 255) / 256;
        const int64_t bcap = static_cast<int64_t>(num_sms()) * 8;
        if (b2 > bcap) b2 = bcap;
        k_response_exact<<<static_cast<unsigned>(b2), 256, 0, s>>>(uvw, n_vis, offs, n_off, static_cast<double>(sign),
                                                                   resp);
        k_mul_response<<<static_cast<unsigned>(b2), 256, 0, s>>>(static_cast<float2*>(vis_out), resp, n_vis);
        if (cudaGetLastError() != cudaSuccess) rc = set_error(WT_ERR_CUDA, "%s: exact response launch", fn);
    }
    cudaFreeAsync(scratch, s);
    cudaGetLastError();
    return rc;
}

int wt_predict_vis_thresholded(wt_tree t, int j0, double tau, int response, const wt_mlp* mlps, int depth,
                               const double* uvw, int64_t n_vis, void* vis_out, int sign, void* stream)
{
    const char* fn = "wt_predict_vis_thresholded";
    if (!t || t->magic != kTreeMagic) return set_error(WT_ERR_ARG, "%s: bad tree handle", fn);
    const int J = t->J;
    if (j0 < 1 || j0 > J) return set_error(WT_ERR_RANGE, "%s: j0 %d outside 1..J = %d", fn, j0, J);
    if (!(tau >= 0.0)) return set_error(WT_ERR_ARG, "%s: tau must be >= 0", fn);
    if (n_vis < 0 || (sign != 1 && sign != -1)) return set_error(WT_ERR_ARG, "%s: bad n_vis or sign", fn);
    const int nl = J - j0 + 1;   // levels j0 .. J
    int rc;
    if (response == WT_RESPONSE_LEARNED) {
        if (!mlps) return set_error(WT_ERR_ARG, "%s: no networks", fn);
        for (int L = j0; L <= J; ++L) {
            wt_mlp m = mlps[L - j0];
            if ((rc = check_mlp(m, fn))) return rc;
            if (m->level != L) return set_error(WT_ERR_ARG, "%s: network %d is for level %d, not %d", fn, L - j0,
                                                m->level, L);
            if (t->ra0 != m->ra0 || t->dec0 != m->dec0)
                return set_error(WT_ERR_ARG, "%s: tree and network %d have different phase centres", fn, L - j0);
        }
    } else if (response == WT_RESPONSE_EXACT) {
        if (depth < J - j0 || depth > 8 || j0 + depth > kMaxJ)
            return set_error(WT_ERR_RANGE, "%s: need J - j0 <= depth <= 8 and j0 + depth <= %d", fn, kMaxJ);
    } else if (response != WT_RESPONSE_SNAPPED) {
        return set_error(WT_ERR_ARG, "%s: bad response %d", fn, response);
    }
    if ((rc = check_device_buffer(uvw, static_cast<size_t>(n_vis) * 24, fn, "uvw", 8)) ||
        (rc = check_device_buffer(vis_out, static_cast<size_t>(n_vis) * 8, fn, "vis_out", 8)))
        return rc;
    if (n_vis == 0) return WT_OK;
    int* status = device_status_word();
    if (!status) return set_error(WT_ERR_CUDA, "%s: no device status word", fn);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // scratch: a header view per level; the records, level by level, in
    // segments of the capacity bound (level j0: its nodes, at most the leaf
    // capacity; below it, four children per parent); a visibility buffer for
    // the levels below j0; for the exact response the sub-pixel offsets and
    // R(B) per visibility
    const int64_t capl = t->cap_leaves > 0 ? t->cap_leaves : 1;
    LevelSegs seg{};
    int64_t nrec = 0;
    for (int L = j0; L <= J; ++L) {
        seg.off[L] = nrec;
        nrec += (L == j0 ? 1 : 4) * capl;
    }
    auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
    const int n_off = response == WT_RESPONSE_EXACT ? 1 << (2 * depth) : 0;
    const size_t b_views = up(sizeof(TreeHeader) * static_cast<size_t>(nl));
    const size_t b_seg = 0;
    const size_t b_rec = up(sizeof(RecF) * static_cast<size_t>(nrec));
    const size_t b_tmp = up(sizeof(float2) * static_cast<size_t>(n_vis));
    const size_t b_off = up(sizeof(double) * 3 * static_cast<size_t>(n_off));
    const size_t b_r = response == WT_RESPONSE_EXACT ? sizeof(double2) * static_cast<size_t>(n_vis) : 0;
    char* scratch = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&scratch), b_views + b_seg + b_rec + b_tmp + b_off + b_r,
                                    s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(WT_ERR_NOMEM, "%s: scratch allocation failed: %s", fn, cudaGetErrorString(e));
    }
    TreeHeader* views = reinterpret_cast<TreeHeader*>(scratch);
    RecF* recs = reinterpret_cast<RecF*>(scratch + b_views + b_seg);
    float2* tmp = reinterpret_cast<float2*>(scratch + b_views + b_seg + b_rec);
    double* offs = reinterpret_cast<double*>(scratch + b_views + b_seg + b_rec + b_tmp);
    double2* resp = reinterpret_cast<double2*>(scratch + b_views + b_seg + b_rec + b_tmp + b_off);
    Rot R;
    rotation_matrix(t->ra0, t->dec0, R.r);
    rc = WT_OK;
    {
        int64_t blocks = (capl + 255) / 256;
        if (blocks > 4096) blocks = 4096;
        if (cudaMemsetAsync(views->smax, 0, sizeof(views->smax), s) != cudaSuccess) {
            cudaGetLastError();
            rc = set_error(WT_ERR_CUDA, "%s: clearing the bounds", fn);
        }
        k_level_records<<<static_cast<unsigned>(blocks), 256, 0, s>>>(t->d.key, t->d.lambda, t->d.hdr, j0, R,
                                                                      recs + seg.off[j0], views, capl);
        if (j0 < J)
            k_threshold_records<<<1, 1024, 0, s>>>(t->d.key, t->d.gamma, t->d.hdr, j0, J, tau, R, recs, seg, views);
        if (cudaGetLastError() != cudaSuccess) rc = set_error(WT_ERR_CUDA, "%s: record kernels", fn);
    }
    int64_t b2 = (n_vis + 255) / 256;
    const int64_t bcap = static_cast<int64_t>(num_sms()) * 8;
    if (b2 > bcap) b2 = bcap;
    // the size of level j0 (the tree's header on the host): a large one sums
    // with its phases on the tensor cores, as in the truncated predictor
    int64_t j0_nodes = -1;
    if (rc == WT_OK && tree_sync_header(t) == WT_OK) j0_nodes = t->host_hdr->per_level[j0];
    for (int L = j0; L <= J && rc == WT_OK; ++L) {
        float2* target = (L == j0) ? static_cast<float2*>(vis_out) : tmp;
        if (L == j0 && j0_nodes >= WT_TRUNCATED_TC_MIN_NODES) {
            rc = eq16_tc_launch(recs + seg.off[L], views, capl, j0_nodes, uvw, n_vis, target, sign, status, s, fn);
        } else {
            WaveletJob jb{};
            jb.recf_leaf = recs + seg.off[L];
            jb.hdr = views + (L - j0);
            jb.uvw = uvw;
            jb.n_vis = n_vis;
            jb.vis = target;
            jb.mode = WT_MIXED_FAST;
            jb.sign = sign;
            jb.which = WT_SUM_EQ16;
            jb.J = J;
            jb.status = status;
            rc = launch_wavelet(jb, default_wavelet_variant(WT_MIXED_FAST, WT_SUM_EQ16, J), s);
        }
        if (rc == WT_OK && response == WT_RESPONSE_LEARNED)
            rc = launch_apply(mlps[L - j0], uvw, n_vis, target, sign, true, s);
        if (rc == WT_OK && response == WT_RESPONSE_EXACT) {
            const int dL = depth - (L - j0);   // one common finest level, j0 + depth
            k_response_offsets<<<((1 << (2 * dL)) + 127) / 128, 128, 0, s>>>(L, dL, R, offs);
            k_response_exact<<<static_cast<unsigned>(b2), 256, 0, s>>>(uvw, n_vis, offs, 1 << (2 * dL),
                                                                       static_cast<double>(sign), resp);
            k_mul_response<<<static_cast<unsigned>(b2), 256, 0, s>>>(target, resp, n_vis);
        }
        if (rc == WT_OK && L > j0)
            k_accumulate<<<static_cast<unsigned>(b2), 256, 0, s>>>(static_cast<float2*>(vis_out), tmp, n_vis);
        if (rc == WT_OK && cudaGetLastError() != cudaSuccess) rc = set_error(WT_ERR_CUDA, "%s: level %d", fn, L);
    }
    cudaFreeAsync(scratch, s);
    cudaGetLastError();
    return rc;
}

int wt_mlp_create(int level, double ra0, double dec0, int depth, float x_max, uint64_t seed, wt_mlp* out)
{
    const char* fn = "wt_mlp_create";
    if (!out) return set_error(WT_ERR_ARG, "%s: out is NULL", fn);
    *out = nullptr;
    if (level < 1 || depth < 0 || depth > 8 || level + depth > kMaxJ)
        return set_error(WT_ERR_RANGE, "%s: need 1 <= level, 0 <= depth <= 8, level + depth <= %d", fn, kMaxJ);
    if (!(x_max >= 0.0f) || !isfinite(ra0) || !isfinite(dec0)) return set_error(WT_ERR_RANGE, "%s: bad x_max or centre", fn);
    int dev = 0;
    WT_CUDA_TRY(cudaGetDevice(&dev));
    wt_mlp m = new (std::nothrow) wt_mlp_s();
    if (!m) return set_error(WT_ERR_NOMEM, "%s: host allocation failed", fn);
    memset(static_cast<void*>(m), 0, sizeof(*m));
    m->device = dev;
    m->level = level;
    m->depth = depth;
    m->x_max = x_max;
    m->ra0 = ra0;
    m->dec0 = dec0;
    m->n_off = 1 << (2 * depth);
    const size_t fbytes = sizeof(float) * kNumParams;
    m->part_rows = 2 * num_sms();
    const size_t pbytes = sizeof(float) * kPartStride * static_cast<size_t>(m->part_rows);
    const size_t bytes = 4 * ((fbytes + 255) & ~size_t(255)) + 256 + (kH * kH / 2) * 4 + 256 +
                         sizeof(double) * 3 * static_cast<size_t>(m->n_off) + 256 + pbytes + 256;
    cudaError_t e = cudaMalloc(&m->block, bytes);
    if (e != cudaSuccess) {
        delete m;
        cudaGetLastError();
        return set_error(WT_ERR_NOMEM, "%s: device allocation failed", fn);
    }
    char* p = static_cast<char*>(m->block);
    auto take = [&](size_t b) {
        char* r = p;
        p += (b + 255) & ~size_t(255);
        return r;
    };
    m->params = reinterpret_cast<float*>(take(fbytes));
    m->m = reinterpret_cast<float*>(take(fbytes));
    m->v = reinterpret_cast<float*>(take(fbytes));
    m->grad = reinterpret_cast<float*>(take(fbytes));
    m->loss = reinterpret_cast<float*>(take(sizeof(float)));
    m->w2 = reinterpret_cast<uint32_t*>(take((kH * kH / 2) * 4));
    m->offs = reinterpret_cast<double*>(take(sizeof(double) * 3 * static_cast<size_t>(m->n_off)));
    m->part = reinterpret_cast<float*>(take(pbytes));
    // He-style initial weights, zero biases, from a seeded host generator
    std::vector<float> h(kNumParams, 0.0f);
    std::mt19937_64 rng(seed);
    std::normal_distribution<float> nd(0.0f, 1.0f);
    for (int i = 0; i < kH * 3; ++i) h[oW1 + i] = nd(rng) * 1.0f;
    for (int i = 0; i < kH * kH; ++i) h[oW2 + i] = nd(rng) * sqrtf(2.0f / kH);
    for (int i = 0; i < 2 * kH; ++i) h[oW3 + i] = nd(rng) * sqrtf(1.0f / kH);
    int rc = WT_OK;
    if (cudaMemcpy(m->params, h.data(), fbytes, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(m->m, 0, fbytes) != cudaSuccess || cudaMemset(m->v, 0, fbytes) != cudaSuccess ||
        cudaMemset(m->grad, 0, fbytes) != cudaSuccess || cudaMemset(m->loss, 0, sizeof(float)) != cudaSuccess)
        rc = cuda_error(cudaGetLastError(), "wt_mlp_create initialisation");
    if (rc == WT_OK) {
        Rot R;
        rotation_matrix(ra0, dec0, R.r);
        k_response_offsets<<<(m->n_off + 127) / 128, 128>>>(level, depth, R, m->offs);
        rc = refresh_bf16(m, nullptr);
        if (rc == WT_OK && cudaDeviceSynchronize() != cudaSuccess) rc = cuda_error(cudaGetLastError(), "wt_mlp_create");
    }
    if (rc != WT_OK) {
        cudaFree(m->block);
        delete m;
        return rc;
    }
    m->magic = kMlpMagic;
    *out = m;
    return WT_OK;
}

void wt_mlp_free(wt_mlp m)
{
    if (!m || m->magic != kMlpMagic) return;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != m->device) cudaSetDevice(m->device);
    cudaDeviceSynchronize();
    cudaFree(m->block);
    cudaGetLastError();
    if (prev >= 0 && prev != m->device) cudaSetDevice(prev);
    m->magic = 0;
    delete m;
}

int wt_mlp_get_params(wt_mlp m, float* host_params)
{
    int rc = check_mlp(m, "wt_mlp_get_params");
    if (rc) return rc;
    if (!host_params) return set_error(WT_ERR_ARG, "wt_mlp_get_params: NULL buffer");
    WT_CUDA_TRY(cudaDeviceSynchronize());
    WT_CUDA_TRY(cudaMemcpy(host_params, m->params, sizeof(float) * kNumParams, cudaMemcpyDeviceToHost));
    return WT_OK;
}

int wt_mlp_set_params(wt_mlp m, const float* host_params)
{
    int rc = check_mlp(m, "wt_mlp_set_params");
    if (rc) return rc;
    if (!host_params) return set_error(WT_ERR_ARG, "wt_mlp_set_params: NULL buffer");
    WT_CUDA_TRY(cudaDeviceSynchronize());
    WT_CUDA_TRY(cudaMemcpy(m->params, host_params, sizeof(float) * kNumParams, cudaMemcpyHostToDevice));
    WT_CUDA_TRY(cudaMemset(m->m, 0, sizeof(float) * kNumParams));
    WT_CUDA_TRY(cudaMemset(m->v, 0, sizeof(float) * kNumParams));
    m->adam_t = 0;
    if ((rc = refresh_bf16(m, nullptr))) return rc;
    WT_CUDA_TRY(cudaDeviceSynchronize());
    return WT_OK;
}

int wt_response_exact(int level, int depth, double ra0, double dec0, const double* uvw, int64_t n, int sign,
                      void* out, void* stream)
{
    const char* fn = "wt_response_exact";
    if (level < 1 || depth < 0 || depth > 8 || level + depth > kMaxJ)
        return set_error(WT_ERR_RANGE, "%s: need 1 <= level, 0 <= depth <= 8, level + depth <= %d", fn, kMaxJ);
    if (n < 0 || (sign != 1 && sign != -1)) return set_error(WT_ERR_ARG, "%s: bad n or sign", fn);
    int rc;
    if ((rc = check_device_buffer(uvw, static_cast<size_t>(n) * 24, fn, "uvw", 8)) ||
        (rc = check_device_buffer(out, static_cast<size_t>(n) * 16, fn, "out", 16)))
        return rc;
    if (n == 0) return WT_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int n_off = 1 << (2 * depth);
    double* offs = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&offs), sizeof(double) * 3 * n_off, s);
    if (e != cudaSuccess) return cuda_error(e, "cudaMallocAsync");
    Rot R;
    rotation_matrix(ra0, dec0, R.r);
    k_response_offsets<<<(n_off + 127) / 128, 128, 0, s>>>(level, depth, R, offs);
    int64_t blocks = (n + 255) / 256;
    const int64_t cap = static_cast<int64_t>(num_sms()) * 8;
    if (blocks > cap) blocks = cap;
    k_response_exact<<<static_cast<unsigned>(blocks), 256, 0, s>>>(uvw, n, offs, n_off, static_cast<double>(sign),
                                                                   static_cast<double2*>(out));
    cudaError_t le = cudaGetLastError();
    cudaFreeAsync(offs, s);
    if (le != cudaSuccess) return cuda_error(le, fn);
    return WT_OK;
}

int wt_mlp_loss_grad(wt_mlp m, const double* uvw, const float* target, int64_t n, float* loss, float* grad,
                     void* stream)
{
    const char* fn = "wt_mlp_loss_grad";
    int rc = check_mlp(m, fn);
    if (rc) return rc;
    if (n <= 0 || !loss || !grad) return set_error(WT_ERR_ARG, "%s: need n > 0 and host outputs", fn);
    if ((rc = check_device_buffer(uvw, static_cast<size_t>(n) * 24, fn, "uvw", 8)) ||
        (rc = check_device_buffer(target, static_cast<size_t>(n) * 8, fn, "target", 8)))
        return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    WT_CUDA_TRY(cudaMemsetAsync(m->grad, 0, sizeof(float) * kNumParams, s));
    WT_CUDA_TRY(cudaMemsetAsync(m->loss, 0, sizeof(float), s));
    if ((rc = run_grad(m, uvw, target, 0, n, n, s))) return rc;
    WT_CUDA_TRY(cudaMemcpyAsync(grad, m->grad, sizeof(float) * kNumParams, cudaMemcpyDeviceToHost, s));
    WT_CUDA_TRY(cudaMemcpyAsync(loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost, s));
    WT_CUDA_TRY(cudaStreamSynchronize(s));
    WT_CUDA_TRY(cudaMemsetAsync(m->grad, 0, sizeof(float) * kNumParams, s));
    return WT_OK;
}

int wt_mlp_train_range(wt_mlp m, const double* uvw, const float* target, int64_t n, int64_t step0, int steps,
                       int64_t total_steps, int batch, float lr, float* final_loss, void* stream)
{
    const char* fn = "wt_mlp_train_range";
    int rc = check_mlp(m, fn);
    if (rc) return rc;
    if (n <= 0 || steps < 0 || batch <= 0 || !(lr > 0.0f) || step0 < 0 || total_steps < step0 + steps)
        return set_error(WT_ERR_ARG, "%s: bad sizes, steps or lr", fn);
    if ((rc = check_device_buffer(uvw, static_cast<size_t>(n) * 24, fn, "uvw", 8)) ||
        (rc = check_device_buffer(target, static_cast<size_t>(n) * 8, fn, "target", 8)))
        return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    WT_CUDA_TRY(cudaMemsetAsync(m->grad, 0, sizeof(float) * kNumParams, s));
    // step i of the run takes the minibatch of samples i batch .. (i + 1) batch - 1 (mod n)
    int64_t first = static_cast<int64_t>((static_cast<unsigned __int128>(step0) * static_cast<uint64_t>(batch)) %
                                         static_cast<uint64_t>(n));
    for (int64_t it = step0; it < step0 + steps; ++it) {
        WT_CUDA_TRY(cudaMemsetAsync(m->loss, 0, sizeof(float), s));
        if ((rc = run_grad(m, uvw, target, first, batch, n, s))) return rc;
        m->adam_t += 1;
        // cosine decay of the learning rate over the run of total_steps
        const float lr_t = 0.5f * lr *
                           (1.0f + cosf(3.14159265f * static_cast<float>(it) / static_cast<float>(total_steps)));
        const float b1c = 1.0f - powf(0.9f, static_cast<float>(m->adam_t));
        const float b2c = 1.0f - powf(0.999f, static_cast<float>(m->adam_t));
        k_mlp_adam<<<(kNumParams + 255) / 256, 256, 0, s>>>(m->params, m->m, m->v, m->grad, lr_t, b1c, b2c);
        WT_CUDA_TRY(cudaGetLastError());
        first = (first + batch) % n;
    }
    if ((rc = refresh_bf16(m, s))) return rc;
    if (final_loss) {
        WT_CUDA_TRY(cudaMemcpyAsync(final_loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost, s));
        WT_CUDA_TRY(cudaStreamSynchronize(s));
    }
    return WT_OK;
}

int wt_mlp_train(wt_mlp m, const double* uvw, const float* target, int64_t n, int steps, int batch, float lr,
                 float* final_loss, void* stream)
{
    return wt_mlp_train_range(m, uvw, target, n, 0, steps, steps, batch, lr, final_loss, stream);
}

int wt_mlp_get_state(wt_mlp m, float* host_params, float* host_m, float* host_v, int64_t* step)
{
    int rc = check_mlp(m, "wt_mlp_get_state");
    if (rc) return rc;
    if (!host_params || !host_m || !host_v || !step) return set_error(WT_ERR_ARG, "wt_mlp_get_state: NULL output");
    WT_CUDA_TRY(cudaDeviceSynchronize());
    WT_CUDA_TRY(cudaMemcpy(host_params, m->params, sizeof(float) * kNumParams, cudaMemcpyDeviceToHost));
    WT_CUDA_TRY(cudaMemcpy(host_m, m->m, sizeof(float) * kNumParams, cudaMemcpyDeviceToHost));
    WT_CUDA_TRY(cudaMemcpy(host_v, m->v, sizeof(float) * kNumParams, cudaMemcpyDeviceToHost));
    *step = m->adam_t;
    return WT_OK;
}

int wt_mlp_set_state(wt_mlp m, const float* host_params, const float* host_m, const float* host_v, int64_t step)
{
    int rc = check_mlp(m, "wt_mlp_set_state");
    if (rc) return rc;
    if (!host_params || !host_m || !host_v || step < 0 || step > INT32_MAX)
        return set_error(WT_ERR_ARG, "wt_mlp_set_state: NULL input or bad step");
    WT_CUDA_TRY(cudaDeviceSynchronize());
    WT_CUDA_TRY(cudaMemcpy(m->params, host_params, sizeof(float) * kNumParams, cudaMemcpyHostToDevice));
    WT_CUDA_TRY(cudaMemcpy(m->m, host_m, sizeof(float) * kNumParams, cudaMemcpyHostToDevice));
    WT_CUDA_TRY(cudaMemcpy(m->v, host_v, sizeof(float) * kNumParams, cudaMemcpyHostToDevice));
    m->adam_t = static_cast<int>(step);
    if ((rc = refresh_bf16(m, nullptr))) return rc;
    WT_CUDA_TRY(cudaDeviceSynchronize());
    return WT_OK;
}

int wt_mlp_eval(wt_mlp m, const double* uvw, int64_t n, int sign, void* out, void* stream)
{
    const char* fn = "wt_mlp_eval";
    int rc = check_mlp(m, fn);
    if (rc) return rc;
    if (n < 0 || (sign != 1 && sign != -1)) return set_error(WT_ERR_ARG, "%s: bad n or sign", fn);
    if ((rc = check_device_buffer(uvw, static_cast<size_t>(n) * 24, fn, "uvw", 8)) ||
        (rc = check_device_buffer(out, static_cast<size_t>(n) * 8, fn, "out", 8)))
        return rc;
    if (n == 0) return WT_OK;
    return launch_apply(m, uvw, n, out, sign, false, static_cast<cudaStream_t>(stream));
}

int wt_predict_vis_learned(wt_tree t, wt_mlp m, const double* uvw, int64_t n_vis, void* vis_out, int sign,
                           void* stream)
{
    const char* fn = "wt_predict_vis_learned";
    int rc = check_mlp(m, fn);
    if (rc) return rc;
    if (!t || t->magic != kTreeMagic) return set_error(WT_ERR_ARG, "%s: bad tree handle", fn);
    if (t->J != m->level) return set_error(WT_ERR_ARG, "%s: the network is for level %d, the tree has J = %d", fn,
                                           m->level, t->J);
    if (t->ra0 != m->ra0 || t->dec0 != m->dec0)
        return set_error(WT_ERR_ARG, "%s: tree and network have different phase centres", fn);
    if ((rc = wt_predict_vis(t, uvw, n_vis, vis_out, WT_MIXED_FAST, sign, WT_SUM_EQ16, stream))) return rc;
    if (n_vis == 0) return WT_OK;
    return launch_apply(m, uvw, n_vis, vis_out, sign, true, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
