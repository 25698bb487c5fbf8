// tree_build.cu -- wt_build_tree: components -> sphere pixels -> coefficient
// tree (Sec. 3.3-3.5 and Eqs. 9, 10, 18 of arXiv:1909.03956).
//
// Device pipeline, all on the caller's stream:
//   k_map_components   one thread per component: SIN projection (Sec. 3.3),
//                      rotation into the xyz frame (Eq. 18), colatitude from
//                      the NCP and RA, nested pixel k_J (Sec. 3.2, 3.5);
//   or k_map_xref      for components found at image pixels: k_J read from
//                      the cross-reference table (Sec. 3.5) that
//                      k_xref_table fills with the same mapping.
//   radix sort         stable LSD sort of (k_J, component index), 8-bit
//                      digits, ceil((2J + 2) / 8) passes of three kernels.
//   k_gather_flux      fluxes in sorted order (contiguous for the sums).
//   k_tree_levels      one CTA: distinct leaves, merged fluxes Phi_k in input
//                      order, lambda_J = Phi / A_J, leaf pixel centres, then
//                      for j = J-1 .. 1 the distinct parents k >> 2, the
//                      topology and Eqs. 9/10 in the paper's order.
//   k_tree_records     one thread per node: post-order position and the
//                      packed records the predictors stream.
// Rounding: every float64 step that must match the CPU definition bit for bit
// uses the _rn intrinsics, which the compiler never contracts into FMAs.
#include <math.h>

#include "sphere.cuh"
#include "wt_internal.cuh"

namespace wt {
namespace {

constexpr int kSortThreads = 1024;
constexpr int kSortItems = 4;
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kLevelThreads = 1024;

struct Rot {
    double r[9];
};

// ---------------------------------------------------------------- K1: map
// k_J of the image point (l, m): SIN projection, rotation into the xyz frame,
// colatitude from the NCP and RA, nested pixel. False outside the unit disc
// or for a non-finite coordinate.
__device__ __forceinline__ bool map_lm(double li, double mi, const Rot& R, int J, uint64_t* key)
{
    const double r2 = __dadd_rn(__dmul_rn(li, li), __dmul_rn(mi, mi));
    if (!(r2 < 1.0) || !isfinite(li) || !isfinite(mi)) return false;
    const double ni = __dsqrt_rn(__dsub_rn(1.0, r2));
    const double x = __dadd_rn(__dadd_rn(__dmul_rn(R.r[0], li), __dmul_rn(R.r[1], mi)), __dmul_rn(R.r[2], ni));
    const double y = __dadd_rn(__dadd_rn(__dmul_rn(R.r[3], li), __dmul_rn(R.r[4], mi)), __dmul_rn(R.r[5], ni));
    const double zc = __dadd_rn(__dadd_rn(__dmul_rn(R.r[6], li), __dmul_rn(R.r[7], mi)), __dmul_rn(R.r[8], ni));
    double phi = atan2(x, zc);
    if (phi < 0.0) phi = __dadd_rn(phi, 2.0 * kPi);
    if (phi >= 2.0 * kPi) phi = __dsub_rn(phi, 2.0 * kPi);
    *key = static_cast<uint64_t>(pixel_of(J - 1, y, phi));
    return true;
}

__global__ void k_map_components(const double* __restrict__ l, const double* __restrict__ m,
                                 const double* __restrict__ flux, int64_t n, Rot R, int J,
                                 uint64_t* __restrict__ keys, uint32_t* __restrict__ idx, int* status)
{
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t key = 0;
    if (!isfinite(flux[i]) || !map_lm(l[i], m[i], R, J, &key)) {
        key = 0;
        record_status(status, WT_ERR_RANGE);
    }
    keys[i] = key;
    idx[i] = static_cast<uint32_t>(i);
}

// The cross-reference table of Sec. 3.5: k_J of every pixel of an n x n
// image, pixel (ix, iy) at l = (ix - n/2) dl, m = (iy - n/2) dl; -1 where
// the pixel lies outside the unit disc.
__global__ void k_xref_table(int n, double dl, Rot R, int J, int64_t* __restrict__ table)
{
    const int64_t nn = static_cast<int64_t>(n) * n;
    for (int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; q < nn;
         q += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int iy = static_cast<int>(q / n), ix = static_cast<int>(q - static_cast<int64_t>(iy) * n);
        const double li = static_cast<double>(ix - n / 2) * dl;
        const double mi = static_cast<double>(iy - n / 2) * dl;
        uint64_t key = 0;
        table[q] = map_lm(li, mi, R, J, &key) ? static_cast<int64_t>(key) : -1;
    }
}

// Keys of components found at image pixels, read from the table.
__global__ void k_map_xref(const int64_t* __restrict__ table, int64_t n_pix, const int32_t* __restrict__ pix,
                           const double* __restrict__ flux, int64_t n, uint64_t* __restrict__ keys,
                           uint32_t* __restrict__ idx, int* status)
{
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t p = pix[i];
    const int64_t k = (p >= 0 && p < n_pix) ? table[p] : -1;
    uint64_t key = 0;
    if (k < 0 || !isfinite(flux[i])) record_status(status, WT_ERR_RANGE);
    else key = static_cast<uint64_t>(k);
    keys[i] = key;
    idx[i] = static_cast<uint32_t>(i);
}

// ---------------------------------------------------------------- radix sort
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint64_t* __restrict__ keys, int64_t n,
                                                             int shift, uint32_t* __restrict__ hist, int nblk)
{
    __shared__ uint32_t h[256];
    for (int d = threadIdx.x; d < 256; d += blockDim.x) h[d] = 0;
    __syncthreads();
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kSortTile;
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const int64_t i = base + r * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[d * nblk + blockIdx.x] = h[d];
}

// Exclusive prefix sum of 1024 ints held one per thread; returns the block
// total in `total`.
__device__ __forceinline__ int block_exclusive_scan(int x, int& total, int* warp_sums)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    int incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int v = lane < nwarps ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        warp_sums[lane] = v;
    }
    __syncthreads();
    const int before = warp > 0 ? warp_sums[warp - 1] : 0;
    total = warp_sums[nwarps - 1];
    __syncthreads();
    return before + incl - x;
}

__global__ void __launch_bounds__(1024) k_radix_scan(uint32_t* __restrict__ hist, int count)
{
    __shared__ int ws[32];
    int carry = 0;
    for (int start = 0; start < count; start += blockDim.x) {
        const int i = start + threadIdx.x;
        const int x = i < count ? static_cast<int>(hist[i]) : 0;
        int total;
        const int ex = block_exclusive_scan(x, total, ws);
        if (i < count) hist[i] = static_cast<uint32_t>(ex + carry);
        carry += total;
    }
}

__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(const uint64_t* __restrict__ kin,
                                                                const uint32_t* __restrict__ vin,
                                                                uint64_t* __restrict__ kout,
                                                                uint32_t* __restrict__ vout, int64_t n, int shift,
                                                                const uint32_t* __restrict__ offs, int nblk)
{
    __shared__ uint32_t wcnt[32][257];
    __shared__ uint32_t base[256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int d = tid; d < 256; d += blockDim.x) base[d] = offs[d * nblk + blockIdx.x];
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int r = 0; r < kSortItems; ++r) {
        const int64_t i = static_cast<int64_t>(blockIdx.x) * kSortTile + r * kSortThreads + tid;
        const bool valid = i < n;
        const uint64_t key = valid ? kin[i] : 0ull;
        const uint32_t d = valid ? static_cast<uint32_t>((key >> shift) & 255u) : 256u;
        for (int k = lane; k < 256; k += 32) wcnt[warp][k] = 0;
        __syncwarp();
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int lrank = __popc(peers & lt_mask);
        if (valid && lrank == 0) wcnt[warp][d] = static_cast<uint32_t>(__popc(peers));
        __syncthreads();
        if (tid < 256) {
            uint32_t run = base[tid];
            for (int w = 0; w < 32; ++w) {
                const uint32_t c = wcnt[w][tid];
                wcnt[w][tid] = run;
                run += c;
            }
            base[tid] = run;
        }
        __syncthreads();
        if (valid) {
            const uint32_t pos = wcnt[warp][d] + static_cast<uint32_t>(lrank);
            kout[pos] = key;
            vout[pos] = vin[i];
        }
        __syncthreads();
    }
}

__global__ void k_gather_flux(const double* __restrict__ flux, const uint32_t* __restrict__ idx, int64_t n,
                              double* __restrict__ out)
{
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) out[i] = flux[idx[i]];
}

// ---------------------------------------------------------------- K2: levels
// A_j = (pi/3) 4^(1-j) and sqrt(A_j)/4 = sqrt(pi/3) 2^(1-j) / 4, formed the
// same way on every platform (one rounding for pi/3, one for the sqrt,
// exact power-of-two scalings).
__device__ __forceinline__ double area_level(int j) { return ldexp(kPi / 3.0, 2 * (1 - j)); }
__device__ __forceinline__ double quarter_sqrt_area(int j)
{
    return __dmul_rn(ldexp(__dsqrt_rn(kPi / 3.0), 1 - j), 0.25);
}

__global__ void __launch_bounds__(kLevelThreads) k_tree_levels(const uint64_t* __restrict__ skeys,
                                                               const double* __restrict__ sflux, int64_t n_comp,
                                                               int J, Rot R, TreeDev d)
{
    __shared__ int ws[32];
    __shared__ int64_t s_count[kMaxJ + 2];
    __shared__ int64_t s_roff[kMaxJ + 2];
    __shared__ unsigned s_smax[3];   // float bits of max |s_u|, |s_v|, |s_w - 1| (non-negative: ordered as integers)
    const int tid = threadIdx.x;
    const int nt = blockDim.x;
    if (tid < 3) s_smax[tid] = 0u;

    // ---- distinct level-J pixels (leaves) and their first sorted element
    int64_t carry = 0;
    for (int64_t start = 0; start < n_comp; start += nt) {
        const int64_t i = start + tid;
        const bool valid = i < n_comp;
        const uint64_t k = valid ? skeys[i] : 0ull;
        const int head = valid && (i == 0 || skeys[i - 1] != k);
        int total;
        const int ex = block_exclusive_scan(head, total, ws);
        if (head) {
            d.key[carry + ex] = static_cast<int64_t>(k);
            d.parent[carry + ex] = static_cast<int32_t>(i);   // first element (temporary)
        }
        carry += total;
    }
    const int64_t n_leaves = carry;
    if (tid == 0) {
        for (int j = 0; j <= kMaxJ + 1; ++j) {
            s_count[j] = 0;
            s_roff[j] = 0;
        }
        s_count[J] = n_leaves;
        s_roff[J] = 0;
    }
    __syncthreads();

    // ---- leaf values: Phi_k summed in input order, lambda_J, pixel centre
    const double AJ = area_level(J);
    for (int64_t leaf = tid; leaf < n_leaves; leaf += nt) {
        const int64_t e0 = d.parent[leaf];
        const int64_t e1 = (leaf + 1 < n_leaves) ? d.parent[leaf + 1] : n_comp;
        double phi_k = 0.0;
        for (int64_t e = e0; e < e1; ++e) phi_k = __dadd_rn(phi_k, sflux[e]);
        d.leaf_flux[leaf] = phi_k;
        d.lambda[leaf] = __ddiv_rn(phi_k, AJ);
        d.gamma[3 * leaf + 0] = 0.0;
        d.gamma[3 * leaf + 1] = 0.0;
        d.gamma[3 * leaf + 2] = 0.0;
        d.first_child[leaf] = -1;
        d.mask[leaf] = 0;
        d.leaf_lo[leaf] = static_cast<int32_t>(leaf);
        d.leaf_hi[leaf] = static_cast<int32_t>(leaf + 1);
        d.size[leaf] = 1;
        // pixel centre -> xyz (y to the NCP, x to RA 6h, z to RA 0h) -> uvw = R^T xyz
        double z, st, ph;
        pixel_centre(J - 1, d.key[leaf], z, st, ph);
        double sph, cph;
        sincos(ph, &sph, &cph);
        const double x = st * sph, y = z, zc = st * cph;
        const double su = R.r[0] * x + R.r[3] * y + R.r[6] * zc;
        const double sv = R.r[1] * x + R.r[4] * y + R.r[7] * zc;
        const double sw = R.r[2] * x + R.r[5] * y + R.r[8] * zc;
        const double sw1 = (sw > 0.0) ? -(su * su + sv * sv) / (1.0 + sw) : sw - 1.0;
        d.leaf_dir[3 * leaf + 0] = su;
        d.leaf_dir[3 * leaf + 1] = sv;
        d.leaf_dir[3 * leaf + 2] = sw1;
        // the float32 heads the records carry (split_f64), whose products
        // the grid pass bounds
        atomicMax(&s_smax[0], __float_as_uint(fabsf(split_f64(su).hi)));
        atomicMax(&s_smax[1], __float_as_uint(fabsf(split_f64(sv).hi)));
        atomicMax(&s_smax[2], __float_as_uint(fabsf(split_f64(sw1).hi)));
    }
    __syncthreads();

    // ---- levels J-1 .. 1
    for (int j = J - 1; j >= 1; --j) {
        const int64_t base_c = s_roff[j + 1];
        const int64_t n_c = s_count[j + 1];
        const int64_t base_p = base_c + n_c;
        carry = 0;
        for (int64_t start = 0; start < n_c; start += nt) {
            const int64_t c = start + tid;
            const bool valid = c < n_c;
            const int64_t kc = valid ? d.key[base_c + c] : 0;
            const int head = valid && (c == 0 || (d.key[base_c + c - 1] >> 2) != (kc >> 2));
            int total;
            const int ex = block_exclusive_scan(head, total, ws);
            if (head) {
                d.key[base_p + carry + ex] = kc >> 2;
                d.first_child[base_p + carry + ex] = static_cast<int32_t>(c);
            }
            if (valid) d.parent[base_c + c] = static_cast<int32_t>(carry + ex + head - 1);
            carry += total;
        }
        const int64_t n_p = carry;
        if (tid == 0) {
            s_count[j] = n_p;
            s_roff[j] = base_p;
        }
        const double q = quarter_sqrt_area(j);
        for (int64_t p = tid; p < n_p; p += nt) {
            const int64_t fc = d.first_child[base_p + p];
            const int64_t lc = (p + 1 < n_p) ? d.first_child[base_p + p + 1] : n_c;
            double ch[4] = {0.0, 0.0, 0.0, 0.0};
            uint32_t mask = 0;
            int32_t size = 1;
            for (int64_t c = fc; c < lc; ++c) {
                const int slot = static_cast<int>(d.key[base_c + c] & 3);
                ch[slot] = d.lambda[base_c + c];
                mask |= 1u << slot;
                size += d.size[base_c + c];
            }
            const int64_t P = base_p + p;
            d.mask[P] = static_cast<uint8_t>(mask);
            d.size[P] = size;
            d.leaf_lo[P] = d.leaf_lo[base_c + fc];
            d.leaf_hi[P] = d.leaf_hi[base_c + lc - 1];
            // Eq. 9 and Eq. 10, children added left to right in slot order
            d.lambda[P] = __dmul_rn(0.25, __dadd_rn(__dadd_rn(__dadd_rn(ch[0], ch[1]), ch[2]), ch[3]));
            d.gamma[3 * P + 0] = __dmul_rn(q, __dsub_rn(__dadd_rn(__dsub_rn(ch[0], ch[1]), ch[2]), ch[3]));
            d.gamma[3 * P + 1] = __dmul_rn(q, __dsub_rn(__dsub_rn(__dadd_rn(ch[0], ch[1]), ch[2]), ch[3]));
            d.gamma[3 * P + 2] = __dmul_rn(q, __dadd_rn(__dsub_rn(__dsub_rn(ch[0], ch[1]), ch[2]), ch[3]));
        }
        __syncthreads();
    }

    if (tid == 0) {
        int64_t total = 0;
        for (int j = 1; j <= J; ++j) {
            d.hdr->per_level[j] = s_count[j];
            d.hdr->rev_offset[j] = s_roff[j];
            total += s_count[j];
        }
        d.hdr->per_level[0] = 0;
        d.hdr->rev_offset[0] = total;
        d.hdr->n_leaves = n_leaves;
        d.hdr->n_nodes = total;
        for (int c = 0; c < 3; ++c) d.hdr->smax[c] = __uint_as_float(s_smax[c]);
        d.hdr->smax[3] = 0.0f;
    }
}

// ---------------------------------------------------------------- records
// Post-order position of a node n with leaf range [lo, hi) and subtree size
// S: the nodes entirely left of its range (at every level, those whose leaf
// range ends at or before lo) come first, then its S - 1 descendants.
__global__ void k_tree_records(TreeDev d, int J, int* status)
{
    const TreeHeader* h = d.hdr;
    const int64_t T = h->n_nodes;
    const double A1 = ldexp(kPi / 3.0, 0);
    for (int64_t n = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; n < T;
         n += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        // level of node n in the level-J-first layout
        int j = J;
        while (j > 1 && n >= h->rev_offset[j] + h->per_level[j]) --j;
        const int32_t lo = d.leaf_lo[n];
        int64_t before = 0;
        for (int jj = 1; jj <= J; ++jj) {
            // count level-jj nodes whose leaf range ends at or before lo
            const int32_t* hi = d.leaf_hi + h->rev_offset[jj];
            int64_t a = 0, b = h->per_level[jj];
            while (a < b) {
                const int64_t mid = (a + b) >> 1;
                if (hi[mid] <= lo) a = mid + 1;
                else b = mid;
            }
            before += a;
        }
        const int64_t post = before + d.size[n] - 1;
        if (post < 0 || post >= T) {
            record_status(status, WT_ERR_CORRUPT);
            continue;
        }
        const bool leaf = (j == J);
        const uint32_t mask = d.mask[n];
        const uint32_t slot = static_cast<uint32_t>(d.key[n] & 3);
        const bool single = !leaf && (__popc(mask) == 1);
        const uint32_t cslot = single ? static_cast<uint32_t>(__ffs(mask) - 1) : 0u;
        const uint32_t store_row = (j >= 2) ? static_cast<uint32_t>(4 * (j - 2)) + slot : 0u;
        const uint32_t child_row = leaf ? 0u : static_cast<uint32_t>(4 * (j - 1)) + cslot;
        const uint32_t meta = store_row | (child_row << 7) | (mask << 14) | (leaf ? kRecLeaf : 0u) |
                              (j == 1 ? kRecRoot : 0u) | (single ? kRecSingle : 0u) |
                              (static_cast<uint32_t>(j) << 21);
        RecD rd;
        RecF rf;
        rd.meta = meta;
        rd.pad = 0;
        rf.meta = meta;
        const int64_t li = n - h->rev_offset[J];   // leaf index (valid for leaves)
        if (leaf) {
            const double su = d.leaf_dir[3 * li], sv = d.leaf_dir[3 * li + 1], sw1 = d.leaf_dir[3 * li + 2];
            const double phi_k = d.leaf_flux[li];
            rd.a = su;
            rd.b = sv;
            rd.c = sw1;
            rd.d = phi_k;
            rd.e = 0.0;
            const F2 a = split_f64(su), b = split_f64(sv), c = split_f64(sw1);
            rf.a = a.hi;
            rf.b = a.lo;
            rf.c = b.hi;
            rf.d = b.lo;
            rf.e = c.hi;
            rf.f = c.lo;
            rf.g = static_cast<float>(phi_k);
            d.leafd[li] = rd;
            d.leaff[li] = rf;
        } else {
            double g0 = d.gamma[3 * n], g1 = d.gamma[3 * n + 1], g2 = d.gamma[3 * n + 2];
            if (single) {
                // Hadamard signs of the only child: rows (+-+-), (++--), (+--+)
                if (cslot & 1u) g0 = -g0;
                if (cslot & 2u) g1 = -g1;
                if (((cslot & 1u) ^ ((cslot >> 1) & 1u)) != 0u) g2 = -g2;
            }
            const double q = quarter_sqrt_area(j);
            const double root = (j == 1) ? A1 * d.lambda[n] : 0.0;
            rd.a = g0;
            rd.b = g1;
            rd.c = g2;
            rd.d = q;
            rd.e = root;
            // mixed forms: xi = 4^(J-j) eta, scale factors folded in (RecF)
            const double sc = ldexp(q, -2 * (J - j - 1));
            if (single) {
                rf.a = static_cast<float>(((g0 + g1) + g2) * sc);
                rf.b = 0.0f;
                rf.c = 0.0f;
            } else {
                rf.a = static_cast<float>(g0 * sc);
                rf.b = static_cast<float>(g1 * sc);
                rf.c = static_cast<float>(g2 * sc);
            }
            rf.d = 0.0f;
            rf.e = 0.0f;
            rf.f = 0.0f;
            rf.g = static_cast<float>(ldexp(root, -2 * (J - 1)));
        }
        d.recd[post] = rd;
        d.recf[post] = rf;
        // regrouped Eq. 17: the node's weight from its parent's gammas
        double wgt;
        bool first = true;
        bool pair_first = false, pair_second = false, group_first = false;
        uint32_t group_len = 0;
        if (j == 1) {
            wgt = A1 * d.lambda[n];
        } else {
            const int64_t P = h->rev_offset[j - 1] + d.parent[n];
            const double g0 = d.gamma[3 * P], g1 = d.gamma[3 * P + 1], g2 = d.gamma[3 * P + 2];
            const double h0 = (slot & 1u) ? -1.0 : 1.0;                          // + - + -
            const double h1 = (slot & 2u) ? -1.0 : 1.0;                          // + + - -
            const double h2 = (((slot & 1u) ^ ((slot >> 1) & 1u)) != 0u) ? -1.0 : 1.0;   // + - - +
            wgt = quarter_sqrt_area(j - 1) * ((h0 * g0 + h1 * g1) + h2 * g2);
            const uint32_t pmask = d.mask[P];
            first = slot == static_cast<uint32_t>(__ffs(pmask) - 1);
            if (leaf) {
                // sibling leaves are consecutive in post-order: this run
                // spans [post - sib_before, ... + nsib - 1]; pair it greedily
                // from the start of its part in this staging chunk
                const uint32_t sib_before = __popc(pmask & ((1u << slot) - 1u));
                const int64_t run_lo = post - sib_before;
                const int64_t run_hi = run_lo + __popc(pmask) - 1;
                const int64_t chunk_lo = post - post % kRecChunkW;
                const int64_t seg_lo = run_lo > chunk_lo ? run_lo : chunk_lo;
                const int64_t k = post - seg_lo;
                pair_second = (k & 1) != 0;
                pair_first = (k & 1) == 0 && post + 1 <= run_hi && (post + 1) % kRecChunkW != 0;
                if (run_lo / kRecChunkW == (run_hi + 1) / kRecChunkW) {
                    // the run and its parent (post-order: right after the
                    // run) in one chunk: a group, its pairs from its start
                    group_first = sib_before == 0;
                    group_len = static_cast<uint32_t>(__popc(pmask));
                }
            }
        }
        const uint32_t wmeta = static_cast<uint32_t>(j) | (leaf ? kRwLeaf : 0u) | (j == 1 ? kRwRoot : 0u) |
                               (first ? kRwFirst : 0u) | (pair_first ? kRwPairFirst : 0u) |
                               (pair_second ? kRwPairSecond : 0u) | ((!leaf && j == J - 1) ? kRwLowSum : 0u) |
                               ((!leaf && j == J - 2) ? kRwMidSum : 0u) |
                               (group_first ? (kRwGroup | (group_len << kRwGroupShift)) : 0u);
        RecWD wd;
        RecWF wf;
        wd.meta = wmeta;
        wd.pad = 0;
        wd.a = rd.a;
        wd.b = rd.b;
        wd.c = rd.c;
        wd.d = wgt;
        wd.e = 0.0;
        wf.meta = wmeta;
        // internal nodes: stack rows of the node's own xi sum and its parent's
        wf.a = leaf ? rf.a : __uint_as_float(static_cast<uint32_t>(j - 1));
        wf.b = leaf ? rf.b : __uint_as_float(static_cast<uint32_t>(j > 1 ? j - 2 : 0));
        wf.c = leaf ? rf.c : 0.f;
        wf.d = leaf ? rf.d : 0.f;
        wf.e = leaf ? rf.e : 0.f;
        wf.f = leaf ? rf.f : 0.f;
        wf.g = static_cast<float>(ldexp(wgt, -2 * (J - j)));   // weight of xi = 4^(J-j) eta
        if (!leaf) {
            wd.a = wd.b = wd.c = 0.0;
        }
        RecWDF wdf;
        auto split = [](double x, float& h, float& l) {
            h = __double2float_rn(x);
            l = __double2float_rn(x - static_cast<double>(h));
        };
        wdf.meta = wmeta;
        split(wd.a, wdf.ah, wdf.al);
        split(wd.b, wdf.bh, wdf.bl);
        split(wd.c, wdf.ch, wdf.cl);
        split(wgt, wdf.wh, wdf.wl);
        split(leaf ? d.leaf_flux[li] : 0.0, wdf.fh, wdf.fl);
        wdf.pad = 0.f;
        d.recwd[post] = wd;
        d.recwf[post] = wf;
        d.recwdf[post] = wdf;
    }
}

template <class T>
T* carve(char*& p, int64_t count)
{
    T* r = reinterpret_cast<T*>(p);
    const int64_t bytes = ((count * static_cast<int64_t>(sizeof(T))) + 255) & ~int64_t(255);
    p += bytes;
    return r;
}

int64_t carve_bytes(int64_t cap_nodes, int64_t cap_leaves)
{
    auto b = [](int64_t x) { return (x + 255) & ~int64_t(255); };
    return b(cap_nodes * 8) + b(cap_nodes * 8) + b(cap_nodes * 24) + b(cap_nodes * 4) + b(cap_nodes) +
           4 * b(cap_nodes * 4) + b(cap_leaves * 24) + b(cap_leaves * 8) + b(cap_leaves * 8) +
           b(cap_leaves * 4) + b(cap_nodes * int64_t(sizeof(RecD))) + b(cap_nodes * int64_t(sizeof(RecF))) +
           b(cap_leaves * int64_t(sizeof(RecD))) + b(cap_leaves * int64_t(sizeof(RecF))) +
           b(cap_nodes * int64_t(sizeof(RecWD))) + b(cap_nodes * int64_t(sizeof(RecWF))) +
           b(cap_nodes * int64_t(sizeof(RecWDF))) + b(sizeof(TreeHeader));
}

}  // namespace

void rotation_matrix(double ra0, double dec0, double* R)
{
    // R_uvw->xyz = R_y(ra0) R_x(-dec0) (Eq. 18), standard right-handed
    // rotations, written out entry by entry.
    const double ca = cos(ra0), sa = sin(ra0);
    const double cd = cos(-dec0), sd = sin(-dec0);
    R[0] = ca;
    R[1] = sa * sd;
    R[2] = sa * cd;
    R[3] = 0.0;
    R[4] = cd;
    R[5] = -sd;
    R[6] = -sa;
    R[7] = ca * sd;
    R[8] = ca * cd;
}

int build_tree(const KeySource& src, const double* flux, int64_t n_comp, double ra0, double dec0, int J, wt_tree t,
               cudaStream_t s)
{
    // Capacity: level j holds at most min(n_comp, N_j) nodes.
    int64_t cap_nodes = 0;
    for (int j = 1; j <= J; ++j) {
        const int64_t Nj = (j <= 16) ? 12 * (int64_t(1) << (2 * (j - 1))) : INT64_MAX / 4;
        cap_nodes += (n_comp < Nj) ? n_comp : Nj;
    }
    const int64_t cap_leaves = n_comp;
    if (cap_nodes > INT32_MAX / 2) return set_error(WT_ERR_RANGE, "wt_build_tree: too many nodes (%lld)", (long long)cap_nodes);
    const int64_t cap1 = cap_nodes > 0 ? cap_nodes : 1, capl = cap_leaves > 0 ? cap_leaves : 1;

    // scratch for the sort: keys x2, idx x2, histogram, sorted fluxes
    const int nblk = static_cast<int>((n_comp + kSortTile - 1) / kSortTile);
    auto b256 = [](int64_t x) { return (x + 255) & ~int64_t(255); };
    const int64_t scratch_bytes = 2 * b256(capl * 8) + 2 * b256(capl * 4) + b256(int64_t(256) * (nblk > 0 ? nblk : 1) * 4) +
                                  b256(capl * 8);
    const int64_t tree_bytes = carve_bytes(cap1, capl);

    char* block = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&block), tree_bytes, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(WT_ERR_NOMEM, "wt_build_tree: device allocation of %lld bytes failed: %s",
                         (long long)tree_bytes, cudaGetErrorString(e));
    }
    char* scratch = nullptr;
    e = cudaMallocAsync(reinterpret_cast<void**>(&scratch), scratch_bytes, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFreeAsync(block, s);
        return set_error(WT_ERR_NOMEM, "wt_build_tree: scratch allocation of %lld bytes failed: %s",
                         (long long)scratch_bytes, cudaGetErrorString(e));
    }
    t->block = block;
    t->cap_nodes = cap1;
    t->cap_leaves = capl;
    char* p = block;
    TreeDev& d = t->d;
    d.key = carve<int64_t>(p, cap1);
    d.lambda = carve<double>(p, cap1);
    d.gamma = carve<double>(p, 3 * cap1);
    d.first_child = carve<int32_t>(p, cap1);
    d.mask = carve<uint8_t>(p, cap1);
    d.leaf_lo = carve<int32_t>(p, cap1);
    d.leaf_hi = carve<int32_t>(p, cap1);
    d.size = carve<int32_t>(p, cap1);
    d.parent = carve<int32_t>(p, cap1);
    d.leaf_dir = carve<double>(p, 3 * capl);
    d.leaf_flux = carve<double>(p, capl);
    d.anc_sum = carve<int64_t>(p, capl);
    d.anc = carve<int32_t>(p, capl);
    d.recd = carve<RecD>(p, cap1);
    d.recf = carve<RecF>(p, cap1);
    d.leafd = carve<RecD>(p, capl);
    d.leaff = carve<RecF>(p, capl);
    d.recwd = carve<RecWD>(p, cap1);
    d.recwf = carve<RecWF>(p, cap1);
    d.recwdf = carve<RecWDF>(p, cap1);
    d.hdr = carve<TreeHeader>(p, 1);

    char* q = scratch;
    uint64_t* k0 = carve<uint64_t>(q, capl);
    uint64_t* k1 = carve<uint64_t>(q, capl);
    uint32_t* v0 = carve<uint32_t>(q, capl);
    uint32_t* v1 = carve<uint32_t>(q, capl);
    uint32_t* hist = carve<uint32_t>(q, int64_t(256) * (nblk > 0 ? nblk : 1));
    double* sflux = carve<double>(q, capl);

    Rot R;
    rotation_matrix(ra0, dec0, R.r);
    int* status = device_status_word();
    if (!status) return set_error(WT_ERR_CUDA, "wt_build_tree: no device status word");

    if (n_comp > 0 && src.leaf_keys) {
        // the leaves themselves (a tree re-imported from its export): one
        // component per distinct pixel, already in key order
        k_tree_levels<<<1, kLevelThreads, 0, s>>>(reinterpret_cast<const uint64_t*>(src.leaf_keys), flux, n_comp, J, R,
                                                  d);
        WT_CUDA_TRY(cudaGetLastError());
        k_tree_records<<<num_sms() * 4, 256, 0, s>>>(d, J, status);
        WT_CUDA_TRY(cudaGetLastError());
    } else if (n_comp > 0) {
        const int tb = 256;
        if (src.table)
            k_map_xref<<<static_cast<unsigned>((n_comp + tb - 1) / tb), tb, 0, s>>>(src.table, src.n_pix, src.pix,
                                                                                     flux, n_comp, k0, v0, status);
        else
            k_map_components<<<static_cast<unsigned>((n_comp + tb - 1) / tb), tb, 0, s>>>(src.l, src.m, flux, n_comp,
                                                                                            R, J, k0, v0, status);
        WT_CUDA_TRY(cudaGetLastError());
        const int bits = 2 * J + 2;
        const int passes = (bits + 7) / 8;
        uint64_t *kin = k0, *kout = k1;
        uint32_t *vin = v0, *vout = v1;
        for (int ps = 0; ps < passes; ++ps) {
            const int shift = 8 * ps;
            k_radix_hist<<<nblk, kSortThreads, 0, s>>>(kin, n_comp, shift, hist, nblk);
            k_radix_scan<<<1, 1024, 0, s>>>(hist, 256 * nblk);
            k_radix_scatter<<<nblk, kSortThreads, 0, s>>>(kin, vin, kout, vout, n_comp, shift, hist, nblk);
            WT_CUDA_TRY(cudaGetLastError());
            uint64_t* tk = kin;
            kin = kout;
            kout = tk;
            uint32_t* tv = vin;
            vin = vout;
            vout = tv;
        }
        k_gather_flux<<<static_cast<unsigned>((n_comp + tb - 1) / tb), tb, 0, s>>>(flux, vin, n_comp, sflux);
        WT_CUDA_TRY(cudaGetLastError());
        k_tree_levels<<<1, kLevelThreads, 0, s>>>(kin, sflux, n_comp, J, R, d);
        WT_CUDA_TRY(cudaGetLastError());
        const int nsm = num_sms();
        k_tree_records<<<nsm * 4, 256, 0, s>>>(d, J, status);
        WT_CUDA_TRY(cudaGetLastError());
    } else {
        WT_CUDA_TRY(cudaMemsetAsync(d.hdr, 0, sizeof(TreeHeader), s));
    }
    WT_CUDA_TRY(cudaMemcpyAsync(t->host_hdr, d.hdr, sizeof(TreeHeader), cudaMemcpyDeviceToHost, s));
    WT_CUDA_TRY(cudaFreeAsync(scratch, s));
    t->host_valid = false;
    return WT_OK;
}

int xref_table(int n, double dl, double ra0, double dec0, int J, int64_t* table, cudaStream_t s)
{
    Rot R;
    rotation_matrix(ra0, dec0, R.r);
    const int64_t nn = static_cast<int64_t>(n) * n;
    int64_t blocks = (nn + 255) / 256;
    const int64_t cap = static_cast<int64_t>(num_sms()) * 16;
    if (blocks > cap) blocks = cap;
    k_xref_table<<<static_cast<unsigned>(blocks > 0 ? blocks : 1), 256, 0, s>>>(n, dl, R, J, table);
    WT_CUDA_TRY(cudaGetLastError());
    return WT_OK;
}

int tree_sync_header(wt_tree t)
{
    if (!t->host_valid) {
        WT_CUDA_TRY(cudaStreamSynchronize(t->stream));
        t->host_valid = true;
    }
    return WT_OK;
}

}  // namespace wt
