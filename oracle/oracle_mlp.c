/*
 * oracle_mlp.c -- plain FP64 oracle for the learned per-level visibility
 * response (an addition to arXiv:1909.03956, not in the paper): the exact
 * response the network learns, and the network's forward and backward pass.
 *
 * TEST INFRASTRUCTURE, like oracle.c: only tests, the smoke check and the CPU
 * legs of the benchmark load it; the CUDA library shares no code with it.
 *
 * Pixel response (reading R10). For level j, let P_j be the level-j pixel
 * that contains the phase centre, c_j its centre, and s_i (i < 4^D) the
 * centres of its descendants D levels down. The response is
 *     R_j(B) = 4^-D sum_i exp(sign i 2 pi B.(s_i - c_j)),
 * i.e. the plane wave's level-j scaling coefficient eta_j (the Eq. 9
 * recursion on the dense sub-tree of depth D), demodulated by the plane
 * wave at c_j. A pixel whose flux is spread uniformly over its area then
 * contributes Phi exp(sign i 2 pi B.(c - P)) R_j(B) to the visibility instead
 * of the centre-snapped Phi exp(sign i 2 pi B.(c - P)) of Eq. 16.
 * B.(s - c) = u (s_u - c_u) + v (s_v - c_v) + w ((s_w - 1) - (c_w - 1)).
 *
 * Network (reading R11): features x = (u, v, w) * Delta theta_j with
 * Delta theta_j = 2^(1-j) sqrt(pi/3) (Sec. 3.3); layers 3 -> 64 -> 64 -> 2,
 * SiLU after the first two, output (Re R, Im R). Parameters are one flat
 * float64 vector: W1[64][3], b1[64], W2[64][64], b2[64], W3[2][64], b3[2].
 * Loss: mean over samples of the squared error of both outputs.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846
#define H 64

/* Mutation testing of the pins, as in oracle.c: a test build may define
 * ORC_PLANT = k to plant the k-th known mistake (here k = 13 .. 16); the
 * normal build plants nothing. */
#ifndef ORC_PLANT
#define ORC_PLANT 0
#endif
#define PLANTED(k) (ORC_PLANT == (k))

/* Full-pixel response of pixel k at level j (reading R10 for any pixel):
 *     R_j,k(B) = 4^-D sum_i exp(sign i 2 pi B.(s_i - c_j,k))
 * over the centres s_i of the 4^D descendants of pixel k at level j + D
 * (nested numbering: keys k 4^D .. (k + 1) 4^D - 1, Sec. 3.5), c_j,k the
 * pixel's own centre. A flux spread uniformly over the pixel contributes
 * Phi exp(sign i 2 pi B.(c_j,k - P)) R_j,k(B) to the visibility. */
int orc_pixel_response_of(int j, int64_t k, int D, double ra0, double dec0, int64_t n, const double* uvw, int sign,
                          double* out /* [n][2] */)
{
    if (j < 1 || D < 0 || j + D > 30 || D > 10 || n < 0 || (sign != 1 && sign != -1)) return -1;
    if (k < 0 || k >= 12 * ((int64_t)1 << (2 * (j - 1)))) return -1;
    double c[3];
    orc_pixel_dir_uvw(j, k, ra0, dec0, c);
    const int64_t nsub = (int64_t)1 << (2 * D);
    double* d = (double*)malloc(sizeof(double) * 3 * (size_t)nsub);
    for (int64_t i = 0; i < nsub; ++i) {
        double s[3];
        orc_pixel_dir_uvw(j + D, (k << (2 * D)) + i, ra0, dec0, s);
        const double sg = PLANTED(13) ? -1.0 : 1.0;
        d[3 * i + 0] = sg * (s[0] - c[0]);
        d[3 * i + 1] = sg * (s[1] - c[1]);
        d[3 * i + 2] = sg * (s[2] - c[2]);
    }
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < n; ++q) {
        const double u = uvw[3 * q], v = uvw[3 * q + 1], w = uvw[3 * q + 2];
        double re = 0.0, im = 0.0;
        for (int64_t i = 0; i < nsub; ++i) {
            double t = u * d[3 * i] + v * d[3 * i + 1] + w * d[3 * i + 2];
            t = t - rint(t);
            re += cos(2.0 * ORC_PI * t);
            im += (double)sign * sin(2.0 * ORC_PI * t);
        }
        const double norm = PLANTED(14) ? (double)(nsub / 4 > 0 ? nsub / 4 : 1) : (double)nsub;
        out[2 * q] = re / norm;
        out[2 * q + 1] = im / norm;
    }
    free(d);
    return 0;
}

/* R_j(B) of the level-j pixel that holds the phase centre (reading R10). */
int orc_pixel_response(int j, int D, double ra0, double dec0, int64_t n, const double* uvw, int sign,
                       double* out /* [n][2] */)
{
    if (j < 1 || D < 0 || j + D > 30 || D > 10 || n < 0 || (sign != 1 && sign != -1)) return -1;
    const double zero = 0.0;
    int64_t kref;
    if (orc_map_components(1, &zero, &zero, ra0, dec0, j, &kref, NULL) != 0) return -2;
    return orc_pixel_response_of(j, kref, D, ra0, dec0, n, uvw, sign, out);
}

double orc_level_pixel_size(int j) { return ldexp(sqrt(ORC_PI / 3.0), 1 - j); }

int orc_mlp_n_params(void) { return H * 3 + H + H * H + H + 2 * H + 2; }

static double sigm(double z) { return 1.0 / (1.0 + exp(-z)); }
static double silu(double z) { return z * sigm(z); }
static double dsilu(double z)
{
    const double s = sigm(z);
    return PLANTED(15) ? s : s * (1.0 + z * (1.0 - s));
}

typedef struct {
    const double *W1, *b1, *W2, *b2, *W3, *b3;
} params_view;

static params_view view(const double* p)
{
    params_view v;
    v.W1 = p;
    v.b1 = v.W1 + H * 3;
    v.W2 = v.b1 + H;
    v.b2 = v.W2 + H * H;
    v.W3 = v.b2 + H;
    v.b3 = v.W3 + 2 * H;
    return v;
}

/* Features: x = B * Delta theta_j (reading R11). */
static void features(const double* B, double scale, double* x)
{
    x[0] = B[0] * scale;
    x[1] = B[1] * scale;
    x[2] = B[2] * scale;
}

static void forward_one(const params_view* P, const double* x, double* z1, double* h1, double* z2, double* h2,
                        double* y)
{
    for (int i = 0; i < H; ++i) {
        double s = P->b1[i];
        for (int d = 0; d < 3; ++d) s += P->W1[3 * i + d] * x[d];
        z1[i] = s;
        h1[i] = silu(s);
    }
    for (int o = 0; o < H; ++o) {
        double s = P->b2[o];
        for (int i = 0; i < H; ++i) s += (PLANTED(16) ? P->W2[H * i + o] : P->W2[H * o + i]) * h1[i];
        z2[o] = s;
        h2[o] = silu(s);
    }
    for (int o = 0; o < 2; ++o) {
        double s = P->b3[o];
        for (int i = 0; i < H; ++i) s += P->W3[H * o + i] * h2[i];
        y[o] = s;
    }
}

int orc_mlp_forward(const double* params, int level, int64_t n, const double* uvw, double* y /* [n][2] */)
{
    if (level < 1 || level > 30 || n < 0) return -1;
    const params_view P = view(params);
    const double scale = orc_level_pixel_size(level);
    double z1[H], h1[H], z2[H], h2[H], x[3];
    for (int64_t q = 0; q < n; ++q) {
        features(uvw + 3 * q, scale, x);
        forward_one(&P, x, z1, h1, z2, h2, y + 2 * q);
    }
    return 0;
}

/* Mean squared error over the batch and its gradient with respect to every
 * parameter (backpropagation, written out layer by layer). */
int orc_mlp_loss_grad(const double* params, int level, int64_t n, const double* uvw, const double* target,
                      double* loss, double* grad)
{
    if (level < 1 || level > 30 || n <= 0) return -1;
    const params_view P = view(params);
    const int np = orc_mlp_n_params();
    memset(grad, 0, sizeof(double) * (size_t)np);
    double* gW1 = grad;
    double* gb1 = gW1 + H * 3;
    double* gW2 = gb1 + H;
    double* gb2 = gW2 + H * H;
    double* gW3 = gb2 + H;
    double* gb3 = gW3 + 2 * H;
    const double scale = orc_level_pixel_size(level);
    double z1[H], h1[H], z2[H], h2[H], x[3], y[2], dy[2], dh2[H], dz2[H], dz1[H];
    double L = 0.0;
    for (int64_t q = 0; q < n; ++q) {
        features(uvw + 3 * q, scale, x);
        forward_one(&P, x, z1, h1, z2, h2, y);
        for (int o = 0; o < 2; ++o) {
            const double e = y[o] - target[2 * q + o];
            L += e * e;
            dy[o] = 2.0 * e / (double)n;
        }
        for (int o = 0; o < 2; ++o) {
            gb3[o] += dy[o];
            for (int i = 0; i < H; ++i) gW3[H * o + i] += dy[o] * h2[i];
        }
        for (int i = 0; i < H; ++i) {
            dh2[i] = dy[0] * P.W3[i] + dy[1] * P.W3[H + i];
            dz2[i] = dh2[i] * dsilu(z2[i]);
        }
        for (int o = 0; o < H; ++o) {
            gb2[o] += dz2[o];
            for (int i = 0; i < H; ++i) gW2[H * o + i] += dz2[o] * h1[i];
        }
        for (int i = 0; i < H; ++i) {
            double dh1 = 0.0;
            for (int o = 0; o < H; ++o) dh1 += dz2[o] * P.W2[H * o + i];
            dz1[i] = dh1 * dsilu(z1[i]);
        }
        for (int i = 0; i < H; ++i) {
            gb1[i] += dz1[i];
            for (int d = 0; d < 3; ++d) gW1[3 * i + d] += dz1[i] * x[d];
        }
    }
    *loss = L / (double)n;
    return 0;
}
