// sphere.cuh -- device geometry of the nested sphere pixelisation
// (Sec. 3.2; HEALPix nested geometry of Gorski et al. 2005, read with the
// NCP as pole and the RA as longitude, Sec. 3.4), shared by the tree build
// and the learned-response kernels.
#pragma once

#include <math.h>

#include "wt_internal.cuh"

namespace wt {
namespace {

// ---------------------------------------------------------------- sphere
// Nested pixel of the point with z = cos(colatitude) and longitude phi in
// [0, 2 pi) at `order` (level order + 1). The equatorial belt |z| <= 2/3
// is cut by the lines Ns (1/2 + t) -/+ (3/4) Ns z = integer (t = phi/(pi/2));
// the polar caps by Ns sqrt(3 (1 - |z|)) t' = integer and
// Ns sqrt(3 (1 - |z|)) (1 - t') = integer (t' the longitude in the quarter).
__device__ __forceinline__ uint64_t interleave_bits(uint64_t x)
{
    // spread 32 bits into the even positions
    x &= 0xffffffffull;
    x = (x | (x << 16)) & 0x0000ffff0000ffffull;
    x = (x | (x << 8)) & 0x00ff00ff00ff00ffull;
    x = (x | (x << 4)) & 0x0f0f0f0f0f0f0f0full;
    x = (x | (x << 2)) & 0x3333333333333333ull;
    x = (x | (x << 1)) & 0x5555555555555555ull;
    return x;
}

__device__ __forceinline__ uint64_t compact_bits(uint64_t x)
{
    x &= 0x5555555555555555ull;
    x = (x | (x >> 1)) & 0x3333333333333333ull;
    x = (x | (x >> 2)) & 0x0f0f0f0f0f0f0f0full;
    x = (x | (x >> 4)) & 0x00ff00ff00ff00ffull;
    x = (x | (x >> 8)) & 0x0000ffff0000ffffull;
    x = (x | (x >> 16)) & 0x00000000ffffffffull;
    return x;
}

__device__ int64_t pixel_of(int order, double z, double phi)
{
    const int64_t ns = int64_t(1) << order;
    const double dns = static_cast<double>(ns);
    const double za = fabs(z);
    const double t = __ddiv_rn(phi, 0.5 * kPi);
    int64_t face, ix, iy;
    if (za <= 2.0 / 3.0) {
        const double a = __dmul_rn(dns, __dadd_rn(0.5, t));
        const double b = __dmul_rn(dns, __dmul_rn(z, 0.75));
        const int64_t up = static_cast<int64_t>(floor(__dsub_rn(a, b)));
        const int64_t dn = static_cast<int64_t>(floor(__dadd_rn(a, b)));
        const int64_t fu = up >> order, fd = dn >> order;
        face = (fu == fd) ? (fu & 3) + 4 : (fu < fd ? fu : fd + 8);
        ix = dn & (ns - 1);
        iy = ns - 1 - (up & (ns - 1));
    } else {
        int64_t q = static_cast<int64_t>(t);
        q = q > 3 ? 3 : q;
        const double tq = __dsub_rn(t, static_cast<double>(q));
        const double s = __dmul_rn(dns, __dsqrt_rn(__dmul_rn(3.0, __dsub_rn(1.0, za))));
        int64_t ja = static_cast<int64_t>(floor(__dmul_rn(tq, s)));
        int64_t jb = static_cast<int64_t>(floor(__dmul_rn(__dsub_rn(1.0, tq), s)));
        ja = ja < ns - 1 ? ja : ns - 1;
        jb = jb < ns - 1 ? jb : ns - 1;
        if (z > 0.0) {
            face = q;
            ix = ns - 1 - jb;
            iy = ns - 1 - ja;
        } else {
            face = q + 8;
            ix = ja;
            iy = jb;
        }
    }
    return face * ns * ns + static_cast<int64_t>(interleave_bits(ix) | (interleave_bits(iy) << 1));
}

// Centre of nested pixel `pix` at `order`: z, sin(colatitude), phi. The
// centre sits on iso-latitude ring r = (row + 2) Ns - ix - iy - 1.
__device__ void pixel_centre(int order, int64_t pix, double& z, double& st, double& phi)
{
    const int64_t ns = int64_t(1) << order;
    const int64_t npf = ns * ns;
    const int64_t face = pix >> (2 * order);
    const uint64_t in_face = static_cast<uint64_t>(pix & (npf - 1));
    const int64_t ix = static_cast<int64_t>(compact_bits(in_face));
    const int64_t iy = static_cast<int64_t>(compact_bits(in_face >> 1));
    const int64_t row = face >> 2, col = face & 3;
    const int64_t ring = (row + 2) * ns - ix - iy - 1;
    const int64_t lon_units = (row == 1) ? 2 * col : 2 * col + 1;   // face centre, in pi/4
    int64_t nr, shift;
    if (ring < ns) {
        nr = ring;
        const double d = static_cast<double>(nr * nr) / (3.0 * static_cast<double>(npf));
        z = 1.0 - d;
        st = sqrt(d * (2.0 - d));
        shift = 0;
    } else if (ring > 3 * ns) {
        nr = 4 * ns - ring;
        const double d = static_cast<double>(nr * nr) / (3.0 * static_cast<double>(npf));
        z = d - 1.0;
        st = sqrt(d * (2.0 - d));
        shift = 0;
    } else {
        nr = ns;
        z = static_cast<double>(2 * ns - ring) * 2.0 / (3.0 * static_cast<double>(ns));
        st = sqrt((1.0 - z) * (1.0 + z));
        shift = (ring - ns) & 1;
    }
    int64_t jpos = (lon_units * nr + ix - iy + 1 + shift) / 2;
    if (jpos > 4 * nr) jpos -= 4 * nr;
    if (jpos < 1) jpos += 4 * nr;
    phi = (static_cast<double>(jpos) - 0.5 * static_cast<double>(shift + 1)) * (0.5 * kPi) / static_cast<double>(nr);
}

}  // namespace
}  // namespace wt
