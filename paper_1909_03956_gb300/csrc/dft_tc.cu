// dft_tc.cu -- the direct sum (Sec. 3.3, Eq. 12) with its phase contraction
// on the 5th-generation tensor cores (mode WT_MIXED_TC).
//
// The phase of visibility n against component m is a contraction over the
// three coordinates, t = u l + v m + w (n - 1) turns: a matrix product of the
// n_vis x 3 baselines with the 3 x n_comp component coordinates. Only t
// modulo 1 matters, to about 2^-30 turns, while |t| reaches 2^14 turns, so
// float32 products cannot carry it. Here every coordinate is cut into exact
// 11-bit integer slices (float16 holds integers up to 2048 exactly), the
// products of slices are summed on the tensor cores (exact: each product is
// an integer below 2^20 and each sum stays below 2^24), and the three FP32
// accumulators are recombined modulo 1 in float32 with exact steps only.
//
// Slicing. For coordinate c, q_c is fixed per call by the components' bound
// (|s_c| < 1024 2^q_c). A component coordinate s = sum_j b_j 2^(q_c - 11 j),
// j = 0..3, with b_j = rint of the remainder (|b_j| <= 1024); a baseline
// coordinate x = sum_i a_i 2^(-q_c - 11 i), i = 0..4 (|a_0| <= 16 is the
// tile's condition, see below; |a_i| <= 1024). The product of slices a_i b_j
// carries the scale 2^(-11 (i + j)), so i + j = 0 is an integer and drops
// out modulo 1, and the rest is, per (visibility, component),
//   acc1 = sum_c (a0 b1 + a1 b0)                               (scale 2^-11)
//   acc2 = sum_c (a0 b2 + a1 b1 + a2 b0)                       (scale 2^-22)
//   acc3 = sum_c (a0 b3 + a1 b2 + a2 b1 + a3 b0)
//        + 2^-11 sum_c (a1 b3 + a2 b2 + a3 b1 + a4 b0)         (scale 2^-33)
// acc1 and acc2 are sums of at most 9 integer products below 2^20 x 1.01:
// exact in FP32 whatever the order of addition. acc3 is a small tail.
// Dropped: the slices' truncations (below 2^-30 turns for |a_0| <= 16) and
// i + j = 5 (below 2^-31 turns).
//
// Recombination (float32, exact until the last two roundings):
//   f1 = acc1 2^-11 - rint(acc1 2^-11)        (|acc1 2^-11| < 2^12: exact)
//   h  = acc2 2^-22 + f1                      (a multiple of 2^-22 below 2: exact)
//   t  = (h - rint(h)) + acc3 2^-33           (one rounding)
// rint by the 1.5 2^23 constant; sin/cos of 2 pi t from the special-function
// unit as in WT_MIXED_FAST.
//
// Layout. A tile is 128 visibilities (the MMA's M); each row of the A
// operand holds a visibility's 64 float16 slice products' left factors, in
// four K = 16 blocks (one MMA each): block 0 -> acc1, block 1 -> acc2,
// blocks 2 and 3 -> acc3. The components' B operand is built once per call
// by k_tc_slice_components in the same no-swizzle K-major layout, chunks of
// NC components (the MMA's N), and streamed through shared memory by bulk
// copies, two stages of 16 KB (with the components' fluxes). Per chunk one
// thread of a producer warp issues the four MMAs into one of two
// tensor-memory buffers (3 NC columns each) and commits to an mbarrier;
// while the tensor cores fill the next buffer, every epilogue thread reads
// its own row of the current one (tcgen05.ld), forms the terms
// C_m (cos, sin) and adds them, eight at a time, to its Kahan sum. The same
// kernel sums Eq. 16 over a tree's leaves (k_tc_slice_leaves builds the
// operand from the leaf records, the count read on the device).
//
// A tile whose baselines exceed the condition (|a_0| <= 16, i.e. phases
// below 2^14 turns per coordinate) or are not finite is marked and left to
// the exact pass of the double-float direct sum (dft.cu).
#include <cuda_fp16.h>

#include "tcgen05.cuh"
#include "wt_internal.cuh"

namespace wt {

// dft.cu: the exact pass of the mixed direct sum over 128-visibility tiles
// marked by mark_deferred.
int dft_exact_pass_128(const void* recs, const uint32_t* bound, int64_t n_comp, const double* uvw, int64_t n_vis,
                       float2* vis, int sign, int* status, cudaStream_t s);

namespace {

constexpr int kTcRows = 128;                // visibilities per tile (M of the MMA)
constexpr int kTcNC = 16;                   // components per chunk (N of the MMA)
constexpr int kTcStageBytes = 16384;        // B operand per stage
constexpr int kTcG = kTcStageBytes / (kTcNC * 128);   // chunks per stage
constexpr int kTcStageComps = kTcG * kTcNC;
// Tiles of 128 visibilities per CTA (one row of each per epilogue thread):
// a launch takes one, or two for a few hundred terms at most
// (kTcTwoTileMaxChunks chunks). Measured on the medium direct sum: one tile
// 1.64 T terms/s, two 1.45 (half the warps per SM at the same tensor
// memory); over 179 leaves (Eq. 16, the large workload at J = 10) two tiles
// took 2.38 ms against 2.82 for one (their set-up shared).
constexpr int kTcTwoTileMaxChunks = 16;
// tensor-memory columns per buffer (three accumulators of kTcNC per tile)
constexpr int tc_acc_cols(int tiles) { return 3 * kTcNC * tiles; }
// two buffers, rounded up to a power of two (at least 32 columns)
constexpr uint32_t tc_tmem_cols(int tiles)
{
    return 2 * tc_acc_cols(tiles) <= 32 ? 32 : 2 * tc_acc_cols(tiles) <= 64 ? 64 : 2 * tc_acc_cols(tiles) <= 128 ? 128
         : 2 * tc_acc_cols(tiles) <= 256 ? 256 : 512;
}
constexpr int kTcEmptyQ = -200;             // q of a coordinate that is zero for every component
constexpr float kTcMaxA0 = 16.0f;           // |a_0| bound of a tile on the tensor cores
static_assert(2 * tc_acc_cols(2) <= static_cast<int>(tc_tmem_cols(2)), "tensor memory of the two buffers");
static_assert(kTcG >= 1 && kTcG * kTcNC * 128 == kTcStageBytes, "stage layout");

constexpr uint32_t kTcIdesc = idesc_f16(false, kTcRows, kTcNC);

// q with |s| < 1024 2^q for every component coordinate s, from the bound of
// the float32 heads (raised by 2^-20 to cover their rounding).
__device__ __forceinline__ int tc_exponent(uint32_t bound_bits)
{
    const float b = __uint_as_float(bound_bits);
    if (!(b > 0.0f)) return kTcEmptyQ;
    return ilogb(static_cast<double>(b) * (1.0 + 0x1p-20)) - 9;
}

// n slices of y (float64): d_k = rint of the remainder, the remainder then
// scaled by 2^11. Every step is exact.
template <int N>
__device__ __forceinline__ void tc_slices(double y, float (&d)[N])
{
#pragma unroll
    for (int k = 0; k < N; ++k) {
        const double r = rint(y);
        d[k] = static_cast<float>(r);
        y = (y - r) * 2048.0;
    }
}

// The five slices of a baseline coordinate from its fixed-point value Y =
// rint(x 2^44) (|Y| <= 16 2^44): balanced base-2048 digits, least
// significant first (d = Y mod 2048 in [-1024, 1024), then Y = (Y - d) / 2048
// exactly), a[0] the rest (|a[0]| <= 16). The digits are the slices of x
// after rounding it to 2^-44, the precision of its five float64 slices.
// Integer steps and small-integer conversions by the 1.5 2^23 constant, so
// that no float64 or conversion-unit work is needed.
__device__ __forceinline__ float small_int_to_float(int d)
{
    return __int_as_float(0x4B400000 + d) - 12582912.0f;   // exact for |d| < 2^22
}

__device__ __forceinline__ void tc_slices5_int(long long Y, float (&a)[5])
{
#pragma unroll
    for (int k = 4; k >= 1; --k) {
        const int d = static_cast<int>((Y + 1024) & 2047) - 1024;
        a[k] = small_int_to_float(d);
        Y = (Y - d) >> 11;   // exact: Y - d is a multiple of 2048
    }
    a[0] = small_int_to_float(static_cast<int>(Y));
}

__device__ __forceinline__ uint32_t half2_bits(float lo, float hi)
{
    const __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&h);
}

// Row r of a 64-column float16 operand from v[64], in the umma_off layout
// at base (8 stores of 16 bytes).
__device__ __forceinline__ void tc_store_row(unsigned char* base, int r, const float (&v)[64])
{
#pragma unroll
    for (int g = 0; g < 8; ++g) {
        const uint4 q = make_uint4(half2_bits(v[8 * g], v[8 * g + 1]), half2_bits(v[8 * g + 2], v[8 * g + 3]),
                                   half2_bits(v[8 * g + 4], v[8 * g + 5]), half2_bits(v[8 * g + 6], v[8 * g + 7]));
        *reinterpret_cast<uint4*>(base + umma_off(r, 8 * g)) = q;
    }
}

// Row i of the B operand (component i as row i % NC of chunk i / NC;
// chunks of NC x 128 bytes, contiguous) from its coordinates s (float64)
// and the bounds' bits, and its flux as float32.
__device__ __forceinline__ void tc_write_b_row(int64_t i, const double (&s)[3], float f,
                                               const uint32_t* __restrict__ bound, unsigned char* __restrict__ bsl,
                                               float* __restrict__ bfl)
{
    float b[3][4];
#pragma unroll
    for (int c = 0; c < 3; ++c) tc_slices<4>(scalbn(s[c], -tc_exponent(bound[c])), b[c]);
    float v[64];
#pragma unroll
    for (int k = 0; k < 64; ++k) v[k] = 0.0f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        v[c] = b[c][1];            // block 0 (acc1): a0 b1, a1 b0
        v[3 + c] = b[c][0];
        v[16 + c] = b[c][2];       // block 1 (acc2): a0 b2, a1 b1, a2 b0
        v[19 + c] = b[c][1];
        v[22 + c] = b[c][0];
        v[32 + c] = b[c][3];       // block 2 (acc3): a0 b3, a1 b2, a2 b1, a3 b0, 2^-11 a4 b0
        v[35 + c] = b[c][2];
        v[38 + c] = b[c][1];
        v[41 + c] = b[c][0];
        v[44 + c] = b[c][0];
        v[48 + c] = b[c][3];       // block 3 (acc3): 2^-11 (a1 b3, a2 b2, a3 b1)
        v[51 + c] = b[c][2];
        v[54 + c] = b[c][1];
    }
    tc_store_row(bsl + (i / kTcNC) * (kTcNC * 128), static_cast<int>(i % kTcNC), v);
    bfl[i] = f;
}

// The B operand of the direct sum: component i of n_pad (zero beyond n).
// The coordinates are formed as k_pack_components forms them (a component
// that fails its range check there adds nothing here either).
__global__ void k_tc_slice_components(const double* __restrict__ l, const double* __restrict__ m,
                                      const double* __restrict__ flux, int64_t n, int64_t n_pad,
                                      const uint32_t* __restrict__ bound, unsigned char* __restrict__ bsl,
                                      float* __restrict__ bfl)
{
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n_pad) return;
    double s[3] = {0.0, 0.0, 0.0};
    float f = 0.0f;
    if (i < n) {
        const double li = l[i], mi = m[i], fi = flux[i];
        const double r2 = li * li + mi * mi;
        if (r2 < 1.0 && isfinite(li) && isfinite(mi) && isfinite(fi)) {
            s[0] = li;
            s[1] = mi;
            s[2] = -r2 / (1.0 + sqrt(1.0 - r2));
            f = static_cast<float>(fi);
        }
    }
    tc_write_b_row(i, s, f, bound, bsl, bfl);
}

// The B operand of Eq. 16 over a tree's leaf records (RecF: the pixel
// centre (s_u, s_v, s_w - 1) as double-float pairs, g = the merged flux
// Phi_k; their number in hdr->n_leaves, their bounds in hdr->smax): leaf i
// of cap_pad (zero beyond n_leaves). Also each leaf as a direct-sum record
// (CompF) for the exact pass of the tiles beyond the tensor-core range.
__global__ void k_tc_slice_leaves(const RecF* __restrict__ recs, const TreeHeader* __restrict__ hdr,
                                  int64_t cap_pad, unsigned char* __restrict__ bsl, float* __restrict__ bfl,
                                  CompF* __restrict__ exact)
{
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= cap_pad) return;
    double s[3] = {0.0, 0.0, 0.0};
    float f = 0.0f;
    CompF e{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (i < hdr->n_leaves) {
        const RecF r = recs[i];
        s[0] = static_cast<double>(r.a) + static_cast<double>(r.b);   // exact: a double-float pair
        s[1] = static_cast<double>(r.c) + static_cast<double>(r.d);
        s[2] = static_cast<double>(r.e) + static_cast<double>(r.f);
        f = r.g;
        e = CompF{r.a, r.b, r.c, r.d, r.e, r.f, r.g, 0.f};
    }
    tc_write_b_row(i, s, f, reinterpret_cast<const uint32_t*>(hdr->smax), bsl, bfl);
    exact[i] = e;
}

// One accumulator's NC columns of this thread's lane.
__device__ __forceinline__ void tmem_ld_cols(uint32_t taddr, uint32_t (&r)[kTcNC])
{
    if constexpr (kTcNC == 32) tmem_ld32(taddr, r);
    else if constexpr (kTcNC == 16) tmem_ld16(taddr, r);
    else {
        static_assert(kTcNC == 16 || kTcNC == 32, "chunks of 16 or 32 components");
    }
}

// Plain arrive on an mbarrier (one of its expected arrivals).
__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// The direct sum of kTcTiles tiles of 128 visibilities per CTA (see the top
// of the file), warp-specialised: warps 0-3 own kTcTiles visibilities per
// thread (TMEM lane = row = thread, one row of every tile) and form the
// terms; warp 4 (one lane) streams the B operand and issues the MMAs (four
// per tile and chunk, against the same B chunk). Two tensor-memory buffers:
// the producer fills buffer i & 1 with chunk i once the epilogue warps have
// read chunk i - 2 out of it (mbarrier `empty`, one arrival per warp, given
// as soon as a warp's tcgen05.ld of the accumulators completes and it has
// copied the chunk's fluxes), and commits to `full`. The B operand and its
// fluxes come in stages of kTcG chunks, two slots; the slot of stage s - 1
// is refilled with stage s + 1 once the MMAs that read it have completed
// (tcgen05.commit to `sdone` after a stage's last chunk) and the epilogue
// has released the stage's last chunk. Every wait is bounded; a wait that
// runs out records WT_ERR_TIMEOUT, the producer then waits once more
// (bounded) for its copies and MMAs in flight, and the CTA frees its tensor
// memory and leaves.
constexpr int kTcThreads = 160;

template <int kTcTiles>
__global__ void __launch_bounds__(kTcThreads) k_dft_tc(const unsigned char* __restrict__ bsl,
                                                      const float* __restrict__ bfl, int64_t n_chunks,
                                                      int64_t n_stages, const int64_t* __restrict__ n_dev,
                                                      const uint32_t* __restrict__ bound,
                                                      const double* __restrict__ uvw, int64_t n_vis,
                                                      float2* __restrict__ vis, float sgn, int* status)
{
    constexpr int kTcCtaVis = kTcRows * kTcTiles;                 // visibilities per CTA
    constexpr int kTcAcc = tc_acc_cols(kTcTiles);
    constexpr uint32_t kTcTmemCols = tc_tmem_cols(kTcTiles);
    if (n_dev) {   // the count on the device (a tree's leaves): the chunks it needs, at most those allocated
        const int64_t nd = *n_dev;
        const int64_t nc = nd > 0 ? (nd + kTcNC - 1) / kTcNC : 0;
        if (nc < n_chunks) n_chunks = nc;
        n_stages = (n_chunks + kTcG - 1) / kTcG;
    }
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar_full[2], bar_empty[2], bar_ld[2], bar_sdone[2];
    __shared__ uint32_t tmem_base;
    unsigned char* smem = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
    unsigned char* sA = smem;                                         // kTcTiles x 128 rows x 128 bytes
    unsigned char* sB = smem + kTcTiles * kTcRows * 128;
    float* sF = reinterpret_cast<float*>(sB + 2 * kTcStageBytes);   // the stages' fluxes

    const int t = threadIdx.x;
    const int warp = t >> 5, lane_id = t & 31;
    const bool epi = warp < 4;
    const int64_t tile = blockIdx.x;
    const double sg = static_cast<double>(sgn);       // the sign folded into the baseline (exact)
    bool fits = true;
    if (epi) {
#pragma unroll
        for (int q = 0; q < kTcTiles; ++q) {
            const int64_t n = tile * kTcCtaVis + q * kTcRows + t;
            double x[3] = {0.0, 0.0, 0.0};
            if (n < n_vis) {
                x[0] = sg * uvw[3 * n];
                x[1] = sg * uvw[3 * n + 1];
                x[2] = sg * uvw[3 * n + 2];
            }
            float a[3][5];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                // y = x 2^q in units of 2^-44: one exact scaling, one rounding
                const double y = x[c] * scalbn(1.0, tc_exponent(bound[c]) + 44);
                fits = fits && fabs(y) <= static_cast<double>(kTcMaxA0) * 0x1p44;   // false for a NaN
                tc_slices5_int(fits ? __double2ll_rn(y) : 0ll, a[c]);
            }
            float v[64];
#pragma unroll
            for (int k = 0; k < 64; ++k) v[k] = 0.0f;
            constexpr float s11 = 0x1p-11f;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                v[c] = a[c][0];
                v[3 + c] = a[c][1];
                v[16 + c] = a[c][0];
                v[19 + c] = a[c][1];
                v[22 + c] = a[c][2];
                v[32 + c] = a[c][0];
                v[35 + c] = a[c][1];
                v[38 + c] = a[c][2];
                v[41 + c] = a[c][3];
                v[44 + c] = a[c][4] * s11;
                v[48 + c] = a[c][1] * s11;
                v[51 + c] = a[c][2] * s11;
                v[54 + c] = a[c][3] * s11;
            }
            tc_store_row(sA + q * (kTcRows * 128), t, v);
        }
    }
    if (!__syncthreads_and(fits ? 1 : 0)) {
        // left to the exact pass, which takes tiles of 128 visibilities
        if (t == 0) {
#pragma unroll
            for (int q = 0; q < kTcTiles; ++q) {
                const int64_t first = tile * kTcCtaVis + q * kTcRows;
                if (first < n_vis)
                    vis[first] = make_float2(__uint_as_float(kDeferredMark), __uint_as_float(kDeferredMark));
            }
        }
        return;
    }
    if (t == 0) {
        for (int b = 0; b < 2; ++b) {
            mbar_init(&bar_full[b], 1);
            mbar_init(&bar_empty[b], 4);
            mbar_init(&bar_ld[b], 1);
            mbar_init(&bar_sdone[b], 1);
        }
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(&tmem_base, kTcTmemCols);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // A's generic writes before the MMAs read it
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tm = tmem_base;

    if (warp == 4) {
        // ------------------------------------------------------------ producer
        if (lane_id == 0 && n_chunks > 0) {
            const uint32_t a_addr = smem_addr(sA), b_addr = smem_addr(sB);
            int64_t st_issued = 0, mma_issued = 0;
            auto issue_stage = [&](int64_t s) {
                const int slot = static_cast<int>(s & 1);
                mbar_arrive_expect_tx(&bar_ld[slot], kTcStageBytes + kTcStageComps * 4);
                bulk_copy_g2s(sB + slot * kTcStageBytes, bsl + s * kTcStageBytes, kTcStageBytes, &bar_ld[slot]);
                bulk_copy_g2s(sF + slot * kTcStageComps, bfl + s * kTcStageComps, kTcStageComps * 4, &bar_ld[slot]);
                st_issued = s + 1;
            };
            issue_stage(0);
            if (n_stages > 1) issue_stage(1);
            bool ok = true;
            for (int64_t i = 0; i < n_chunks && ok; ++i) {
                const int b = static_cast<int>(i & 1);
                const int64_t s = i / kTcG;
                const int w = static_cast<int>(i % kTcG);
                if (i >= 2) ok = mbar_wait_parity(&bar_empty[b], static_cast<uint32_t>(((i >> 1) - 1) & 1));
                if (ok && w == 0) ok = mbar_wait_parity(&bar_ld[s & 1], static_cast<uint32_t>((s >> 1) & 1));
                if (ok && w == 1 && s >= 1 && s + 1 < n_stages) {
                    // stage s - 1's MMAs are done: its slot takes stage s + 1
                    ok = mbar_wait_parity(&bar_sdone[(s - 1) & 1], static_cast<uint32_t>(((s - 1) >> 1) & 1));
                    if (ok) issue_stage(s + 1);
                }
                if (!ok) break;
                tc_fence_after();
                const uint32_t bb = b_addr + static_cast<uint32_t>(s & 1) * kTcStageBytes + w * (kTcNC * 128);
                const uint32_t col = tm + static_cast<uint32_t>(b) * kTcAcc;
#pragma unroll
                for (int q = 0; q < kTcTiles; ++q) {
#pragma unroll
                    for (int kb = 0; kb < 4; ++kb) {
                        const uint32_t d = col + q * (3 * kTcNC) + (kb == 0 ? 0u : kb == 1 ? kTcNC : 2u * kTcNC);
                        tc_mma_f16(d, umma_desc(a_addr + q * (kTcRows * 128) + kb * 256), umma_desc(bb + kb * 256),
                                   kTcIdesc, kb == 3);
                    }
                }
                tc_commit(&bar_full[b]);
                if (w == kTcG - 1 || i + 1 == n_chunks) tc_commit(&bar_sdone[s & 1]);
                mma_issued = i + 1;
            }
            if (!ok) {
                record_status(status, WT_ERR_TIMEOUT);
                // once more, bounded, for what is in flight: the last two
                // chunks' MMAs and the stages issued (a completed phase
                // passes at once)
                for (int64_t c = mma_issued >= 2 ? mma_issued - 2 : 0; c < mma_issued; ++c)
                    mbar_wait_parity(&bar_full[c & 1], static_cast<uint32_t>((c >> 1) & 1));
                for (int64_t s = st_issued >= 2 ? st_issued - 2 : 0; s < st_issued; ++s)
                    mbar_wait_parity(&bar_ld[s & 1], static_cast<uint32_t>((s >> 1) & 1));
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const uint32_t lane = tm + (static_cast<uint32_t>(warp * 32) << 16);
        const float2 M2 = bcast2(12582912.0f);        // 1.5 2^23: x + M2 - M2 = rint(x) for |x| < 2^22
        const float2 s11 = bcast2(0x1p-11f), s22 = bcast2(0x1p-22f);
        const float2 twopi = bcast2(6.28318530717958648f), s33 = bcast2(6.28318530717958648f * 0x1p-33f);
        float2 acc[kTcTiles], cmp[kTcTiles];
#pragma unroll
        for (int q = 0; q < kTcTiles; ++q) acc[q] = cmp[q] = make_float2(0.f, 0.f);
        bool ok = true;
        for (int64_t i = 0; i < n_chunks; ++i) {
            const int b = static_cast<int>(i & 1);
            const int64_t st = i / kTcG;
            bool got = true;
            if (i % kTcG == 0)   // the stage's fluxes have landed (its phase stays complete until this
                                 // warp has released the stage's last chunk)
                got = mbar_wait_parity(&bar_ld[st & 1], static_cast<uint32_t>((st >> 1) & 1));
            got = got && mbar_wait_parity(&bar_full[b], static_cast<uint32_t>((i >> 1) & 1));
            ok = __all_sync(0xffffffffu, got);
            if (!ok) break;
            tc_fence_after();
            uint32_t r1[kTcTiles][kTcNC], r2[kTcTiles][kTcNC], r3[kTcTiles][kTcNC];
#pragma unroll
            for (int q = 0; q < kTcTiles; ++q) {
                const uint32_t col = lane + static_cast<uint32_t>(b) * kTcAcc + q * (3 * kTcNC);
                tmem_ld_cols(col, r1[q]);
                tmem_ld_cols(col + kTcNC, r2[q]);
                tmem_ld_cols(col + 2 * kTcNC, r3[q]);
            }
            // the chunk's fluxes into registers before its buffer and, with
            // the stage's last chunk, the stage's slot are given back
            float fx[kTcNC];
            {
                const float4* fl =
                    reinterpret_cast<const float4*>(sF + (st & 1) * kTcStageComps + (i % kTcG) * kTcNC);
#pragma unroll
                for (int k = 0; k < kTcNC / 4; ++k) {
                    const float4 f4 = fl[k];
                    fx[4 * k] = f4.x;
                    fx[4 * k + 1] = f4.y;
                    fx[4 * k + 2] = f4.z;
                    fx[4 * k + 3] = f4.w;
                }
            }
            tmem_wait_ld();
            tc_fence_before();
            __syncwarp();
            if (lane_id == 0) mbar_arrive(&bar_empty[b]);   // the buffer may be refilled
#pragma unroll
            for (int g = 0; g < kTcNC / 8; ++g) {
#pragma unroll
                for (int q = 0; q < kTcTiles; ++q) {
                    float2 p = make_float2(0.f, 0.f);
#pragma unroll
                    for (int j = 0; j < 8; j += 2) {
                        const int k = 8 * g + j;
                        const float2 A1 = make_float2(__uint_as_float(r1[q][k]), __uint_as_float(r1[q][k + 1]));
                        const float2 A2 = make_float2(__uint_as_float(r2[q][k]), __uint_as_float(r2[q][k + 1]));
                        const float2 A3 = make_float2(__uint_as_float(r3[q][k]), __uint_as_float(r3[q][k + 1]));
                        const float2 y = fma2(A1, s11, M2);
                        const float2 f1 = fma2(A1, s11, sub2(M2, y));         // acc1 2^-11 mod 1, exact
                        const float2 h = fma2(A2, s22, f1);                   // exact
                        const float2 hp = add2(h, sub2(M2, add2(h, M2)));     // h - rint(h), exact
                        const float2 xa = fma2(A3, s33, mul2(hp, twopi));     // 2 pi t
                        float s0, c0, s1, c1;
                        __sincosf(xa.x, &s0, &c0);
                        __sincosf(xa.y, &s1, &c1);
                        p = fma2(bcast2(fx[k]), make_float2(c0, s0), p);
                        p = fma2(bcast2(fx[k + 1]), make_float2(c1, s1), p);
                    }
                    kahan_add2(acc[q], cmp[q], p);
                }
            }
        }
        if (!ok && lane_id == 0) record_status(status, WT_ERR_TIMEOUT);
        __syncwarp();
        if (ok) {
#pragma unroll
            for (int q = 0; q < kTcTiles; ++q) {
                const int64_t n = tile * kTcCtaVis + q * kTcRows + t;
                if (n < n_vis) vis[n] = sub2(acc[q], cmp[q]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_free(tm, kTcTmemCols);
}

}  // namespace

// Bytes of the tensor-core form's component operand after the packed
// records: the float16 slices and the float32 fluxes of n_comp components
// padded to whole stages.
size_t dft_tc_scratch_bytes(int64_t n_comp)
{
    const int64_t stages = (n_comp + kTcStageComps - 1) / kTcStageComps;
    return static_cast<size_t>(stages) * (kTcStageBytes + kTcStageComps * 4);
}

namespace {

template <int TILES>
int tc_launch_tiles(const unsigned char* bsl, const float* bfl, int64_t n_chunks, int64_t stages,
                    const int64_t* n_dev, const uint32_t* bound, const double* uvw, int64_t n_vis, float2* vis,
                    int sign, int* status, cudaStream_t s, const char* fn)
{
    auto kernel = k_dft_tc<TILES>;
    // no more CTAs per SM than their tensor memory allows (a CTA beyond
    // that would wait in tcgen05.alloc)
    const size_t need = 1024 + TILES * kTcRows * 128 + 2 * kTcStageBytes + 2 * kTcStageComps * 4;
    size_t smem = need;
    int per_sm = 0;
    for (;;) {
        WT_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)));
        WT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kTcThreads, smem));
        if (per_sm < 1) return set_error(WT_ERR_UNSUPPORTED, "%s: tensor-core kernel does not fit on an SM", fn);
        if (per_sm * tc_tmem_cols(TILES) <= 512) break;
        smem += 8192;
    }
    const int64_t cta_vis = static_cast<int64_t>(kTcRows) * TILES;
    const int64_t tiles = (n_vis + cta_vis - 1) / cta_vis;
    if (tiles > 0x7fffffff) return set_error(WT_ERR_RANGE, "%s: too many visibilities for one launch", fn);
    kernel<<<static_cast<unsigned>(tiles), kTcThreads, smem, s>>>(bsl, bfl, n_chunks, stages, n_dev, bound, uvw, n_vis,
                                                                  vis, static_cast<float>(sign), status);
    WT_CUDA_TRY(cudaGetLastError());
    return WT_OK;
}

// Launch k_dft_tc over the tiles of n_vis visibilities: B operand bsl / bfl
// of `stages` stages, n_chunks chunks of it used (or those *n_dev items
// need, when n_dev is given); chunks_hint, the chunks the host expects,
// picks two tiles per CTA for a few hundred terms.
int tc_main_launch(const unsigned char* bsl, const float* bfl, int64_t n_chunks, int64_t stages, const int64_t* n_dev,
                   int64_t chunks_hint, const uint32_t* bound, const double* uvw, int64_t n_vis, float2* vis,
                   int sign, int* status, cudaStream_t s, const char* fn)
{
    if (chunks_hint <= kTcTwoTileMaxChunks)
        return tc_launch_tiles<2>(bsl, bfl, n_chunks, stages, n_dev, bound, uvw, n_vis, vis, sign, status, s, fn);
    return tc_launch_tiles<1>(bsl, bfl, n_chunks, stages, n_dev, bound, uvw, n_vis, vis, sign, status, s, fn);
}

}  // namespace

// The tensor-core direct sum on components already packed (recs, bound:
// k_pack_components in the mixed layout) with `tc` (dft_tc_scratch_bytes,
// 256-byte aligned) for the slices; then the exact pass over the tiles left
// to it.
int dft_tc_launch(const double* l, const double* m, const double* flux, int64_t n_comp, const void* recs,
                  const uint32_t* bound, void* tc, const double* uvw, int64_t n_vis, float2* vis, int sign,
                  int* status, cudaStream_t s)
{
    if (n_vis == 0) return WT_OK;
    const int64_t stages = (n_comp + kTcStageComps - 1) / kTcStageComps;
    const int64_t n_pad = stages * kTcStageComps;
    unsigned char* bsl = static_cast<unsigned char*>(tc);
    float* bfl = reinterpret_cast<float*>(bsl + stages * kTcStageBytes);
    if (n_pad > 0) {
        const int tb = 256;
        k_tc_slice_components<<<static_cast<unsigned>((n_pad + tb - 1) / tb), tb, 0, s>>>(l, m, flux, n_comp, n_pad,
                                                                                         bound, bsl, bfl);
        WT_CUDA_TRY(cudaGetLastError());
    }
    const int64_t chunks = (n_comp + kTcNC - 1) / kTcNC;
    int rc = tc_main_launch(bsl, bfl, chunks, stages, nullptr, chunks, bound, uvw, n_vis, vis, sign, status, s,
                            "dft_predict_vis");
    if (rc) return rc;
    return dft_exact_pass_128(recs, bound, n_comp, uvw, n_vis, vis, sign, status, s);
}

// Eq. 16 in the tensor-core form over leaf records (RecF, at most cap of
// them, their count and bounds in the device header hdr): V = sum_k Phi_k
// exp(sign i 2 pi B.(c_k - P)), the direct sum over the leaves' pixel
// centres with their merged fluxes; n_hint, their number as the host knows
// it (or -1), picks the launch shape. The scratch (the B operand and the
// exact pass's records) is allocated and released on the stream.
int eq16_tc_launch(const RecF* recs, const TreeHeader* hdr, int64_t cap, int64_t n_hint, const double* uvw,
                   int64_t n_vis, float2* vis, int sign, int* status, cudaStream_t s, const char* fn)
{
    if (n_hint < 0) n_hint = cap;
    if (n_vis == 0) return WT_OK;
    const int64_t stages = (cap + kTcStageComps - 1) / kTcStageComps;
    const int64_t cap_pad = stages * kTcStageComps;
    const size_t exact_bytes = static_cast<size_t>(cap_pad > 0 ? cap_pad : 1) * sizeof(CompF);
    const size_t bytes = ((exact_bytes + 255) / 256) * 256 + dft_tc_scratch_bytes(cap_pad);
    unsigned char* scratch = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&scratch), bytes, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(WT_ERR_NOMEM, "%s: scratch allocation of %zu bytes failed: %s", fn, bytes,
                         cudaGetErrorString(e));
    }
    CompF* exact = reinterpret_cast<CompF*>(scratch);
    unsigned char* bsl = scratch + ((exact_bytes + 255) / 256) * 256;
    float* bfl = reinterpret_cast<float*>(bsl + stages * kTcStageBytes);
    int rc = WT_OK;
    if (cap_pad > 0) {
        const int tb = 256;
        k_tc_slice_leaves<<<static_cast<unsigned>((cap_pad + tb - 1) / tb), tb, 0, s>>>(recs, hdr, cap_pad, bsl, bfl,
                                                                                       exact);
        if (cudaGetLastError() != cudaSuccess) rc = set_error(WT_ERR_CUDA, "%s: leaf slicing launch", fn);
    }
    const uint32_t* bound = reinterpret_cast<const uint32_t*>(hdr->smax);   // device address of the bounds
    if (rc == WT_OK)
        rc = tc_main_launch(bsl, bfl, stages * kTcG, stages, &hdr->n_leaves, (n_hint + kTcNC - 1) / kTcNC, bound, uvw,
                            n_vis, vis, sign, status, s, fn);
    // the exact pass over every capacity record (those beyond the count are zero)
    if (rc == WT_OK) rc = dft_exact_pass_128(exact, bound, cap_pad, uvw, n_vis, vis, sign, status, s);
    cudaError_t ef = cudaFreeAsync(scratch, s);
    if (rc != WT_OK) return rc;
    if (ef != cudaSuccess) return cuda_error(ef, "cudaFreeAsync");
    return WT_OK;
}

}  // namespace wt
