/*
 * oracle.c -- plain FP64 CPU oracle for arXiv:1909.03956 (Skipper, Scaife &
 * McEwen), "Cleaning radio interferometric images using a spherical wavelet
 * decomposition".
 *
 * TEST INFRASTRUCTURE. Only tests, the smoke check and the CPU-baseline leg
 * of the benchmark load this file's library. The CUDA library neither links
 * nor includes it; the two share no code.
 *
 * The code follows the paper's steps in its own order and notation and is
 * deliberately slow and plain: no blocking, no fusion, no reordering. Build
 * with -O2 -ffp-contract=off (every operation rounds once, as written).
 *
 * Readings of the paper that this file takes (the paper is silent or its
 * printed formulas do not fit together):
 *   R1  Sign: exp(+i 2 pi B.(s - P)) as printed in Eqs. 1, 12 and 14; the
 *       caller may pass sign = -1 for the conjugate convention.
 *   R2  n - 1 is evaluated as -(l^2 + m^2) / (1 + sqrt(1 - l^2 - m^2)), the
 *       same value as sqrt(1 - l^2 - m^2) - 1 without the cancellation.
 *   R3  The phase t = B.(C - P) is a number of turns; exp(i 2 pi t) is
 *       evaluated as exp(i 2 pi (t - rint t)), an identity.
 *   R4  Sphere pixels: HEALPix nested geometry (Sec. 3.2 says HEALPix-like
 *       with 12 base pixels and four children per pixel; Sec. 3.5 fixes the
 *       nested numbering k_j = k_J >> 2(J - j)). Level j is HEALPix order j-1.
 *       The HEALPix pole axis is the xyz frame's +y (the NCP) and the HEALPix
 *       longitude is the RA, phi = atan2(x, z) (Sec. 3.4).
 *   R5  Rotation matrices are the standard right-handed R_x, R_y, so that
 *       Eq. 18 takes P = [0,0,1] to RA alpha_P, Dec delta_P.
 *   R6  Normalisation. Eq. 15 integrates a sum of delta functions, so the
 *       level-J scaling coefficient is a flux density: lambda_J,k = Phi_k / A_J
 *       where Phi_k is the summed flux of the components in pixel k. The plane
 *       wave's level-J coefficient eta_J,k is the plane wave at the pixel
 *       centre. With Eqs. 9/10 as printed, the visibility is
 *           V = A_J sum_k lambda_J,k eta_J,k                       (Eq. 16)
 *             = A_1 sum_k lambda_1,k eta_1,k
 *               + sum_{j<J} sum_k sum_m gamma^m_j,k sigma^m_j,k   (Eq. 17)
 *       i.e. the printed Eqs. 16/17 with their area factors restored. The two
 *       forms agree because the Hadamard rows of Eq. 10 with (1,1,1,1) form
 *       an orthogonal 4x4 matrix.
 *   R7  A child pixel that holds no component has lambda = 0, and its eta is
 *       taken as 0 (Sec. 3.5: null branches are not computed). This changes
 *       no visibility: every term it touches is multiplied by lambda = 0.
 *   R8  A pixel is a node of the tree when at least one component maps to it,
 *       even if the fluxes there sum to zero.
 *   R9  Rounding order: Phi_k sums component fluxes in input order; Eq. 9 and
 *       Eq. 10 add the four children left to right in child order 0,1,2,3;
 *       A_j = (pi/3) 4^(1-j) and sqrt(A_j) = sqrt(pi/3) 2^(1-j).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

/* Mutation testing of the pins: a test build may define ORC_PLANT = k > 0
 * to plant the k-th known mistake (tests/test_oracle_planted.py checks that
 * a pin catches each one). The normal build plants nothing. */
#ifndef ORC_PLANT
#define ORC_PLANT 0
#endif
#define PLANTED(k) (ORC_PLANT == (k))

/* ========================================================================== */
/* Eq. 12 -- direct sum over the component list                              */
/* ========================================================================== */

/* n - 1 for a point at direction cosines (l, m): reading R2. */
static double n_minus_1(double l, double m)
{
    double r2 = l * l + m * m;
    return (PLANTED(1) ? 1.0 : -1.0) * r2 / (1.0 + sqrt(1.0 - r2));
}

/* V_n = sum_m C_m exp(sign * i 2 pi [u l_m + v m_m + w (n_m - 1)]), Eq. 12
 * with the dot product of Sec. 3.3 (P = [0, 0, 1]). Summed in input order. */
int orc_dft(int64_t n_comp, const double* l, const double* m, const double* flux,
            int64_t n_vis, const double* uvw, int sign, double* vis)
{
    if (n_comp < 0 || n_vis < 0 || (sign != 1 && sign != -1)) return -1;
    for (int64_t n = 0; n < n_vis; ++n) {
        const double u = uvw[3 * n], v = uvw[3 * n + 1], w = uvw[3 * n + 2];
        double re = 0.0, im = 0.0;
        for (int64_t c = 0; c < n_comp; ++c) {
            double t = u * l[c] + v * (PLANTED(2) ? l[c] : m[c]) + w * n_minus_1(l[c], m[c]);
            t = t - rint(t);                          /* R3 */
            const double phase = 2.0 * ORC_PI * t;
            re += flux[c] * cos(phase);
            im += flux[c] * ((double)sign * sin(phase));
        }
        vis[2 * n] = re;
        vis[2 * n + 1] = im;
    }
    return 0;
}

/* The same definition in long double: a higher-precision witness for the
 * FP64 evaluation on small inputs. */
int orc_dft_ld(int64_t n_comp, const double* l, const double* m, const double* flux,
               int64_t n_vis, const double* uvw, int sign, double* vis)
{
    if (n_comp < 0 || n_vis < 0 || (sign != 1 && sign != -1)) return -1;
    const long double pi = 3.141592653589793238462643383279502884L;
    for (int64_t n = 0; n < n_vis; ++n) {
        const long double u = uvw[3 * n], v = uvw[3 * n + 1], w = uvw[3 * n + 2];
        long double re = 0.0L, im = 0.0L;
        for (int64_t c = 0; c < n_comp; ++c) {
            const long double lc = l[c], mc = m[c];
            const long double r2 = lc * lc + mc * mc;
            const long double nm1 = -r2 / (1.0L + sqrtl(1.0L - r2));
            long double t = u * lc + v * mc + w * nm1;
            t = t - rintl(t);
            const long double phase = 2.0L * pi * t;
            re += (long double)flux[c] * cosl(phase);
            im += (long double)flux[c] * ((long double)sign * sinl(phase));
        }
        vis[2 * n] = (double)re;
        vis[2 * n + 1] = (double)im;
    }
    return 0;
}

/* ========================================================================== */
/* Sec. 3.4, Eq. 18 -- coordinate frames                                      */
/* ========================================================================== */

/* R_uvw->xyz(alpha, delta) = R_y(alpha) R_x(-delta), with (reading R5)
 *   R_x(a) = [[1,0,0],[0,cos a,-sin a],[0,sin a,cos a]]
 *   R_y(a) = [[cos a,0,sin a],[0,1,0],[-sin a,0,cos a]].
 * The product is written out one entry at a time. */
void orc_rotation(double ra0, double dec0, double* R)
{
    double Ry[9], Rx[9];
    const double ca = cos(ra0), sa = sin(ra0);
    const double cd = cos(PLANTED(3) ? dec0 : -dec0), sd = sin(PLANTED(3) ? dec0 : -dec0);
    Ry[0] = ca;   Ry[1] = 0.0; Ry[2] = sa;
    Ry[3] = 0.0;  Ry[4] = 1.0; Ry[5] = 0.0;
    Ry[6] = -sa;  Ry[7] = 0.0; Ry[8] = ca;
    Rx[0] = 1.0;  Rx[1] = 0.0; Rx[2] = 0.0;
    Rx[3] = 0.0;  Rx[4] = cd;  Rx[5] = -sd;
    Rx[6] = 0.0;  Rx[7] = sd;  Rx[8] = cd;
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += Ry[3 * r + k] * Rx[3 * k + c];
            R[3 * r + c] = s;
        }
}

/* ========================================================================== */
/* Sec. 3.2 -- nested pixelisation of the sphere (reading R4)                 */
/* ========================================================================== */
/*
 * The 12 base pixels of the HEALPix geometry (Gorski et al. 2005) are three
 * rows of four diamonds: a north row centred at z = 2/3, an equatorial row
 * centred at z = 0 and a south row centred at z = -2/3, with the north and
 * south rows at longitudes pi/4 + q pi/2 and the equatorial row at q pi/2.
 * Inside a base pixel the order-p sub-pixels form an Ns x Ns grid
 * (Ns = 2^p) with coordinates (ix, iy); the nested index is
 * face * Ns^2 + (bits of ix and iy interleaved, ix in the even bits), so the
 * four children of pixel k are 4k .. 4k + 3 (Eq. 9).
 *
 * In the equatorial belt |z| <= 2/3 the pixel edges are the straight lines
 * Ns (1/2 + t) -/+ (3/4) Ns z = integer in the (t = phi / (pi/2), z) plane.
 * In the polar caps the edges are the curves where
 * Ns sqrt(3 (1 - |z|)) times t' or (1 - t') is an integer, t' being the
 * longitude inside the quarter.
 */

static double dist_to_int(double x)
{
    double f = x - floor(x);
    return f < 1.0 - f ? f : 1.0 - f;
}

/* Spread the low 32 bits of x into the even bit positions. */
static uint64_t spread_bits(uint64_t x)
{
    uint64_t r = 0;
    for (int b = 0; b < 32; ++b) r |= ((x >> b) & 1ull) << (2 * b);
    return r;
}

static uint64_t gather_bits(uint64_t x)
{
    uint64_t r = 0;
    for (int b = 0; b < 32; ++b) r |= ((x >> (2 * b)) & 1ull) << b;
    return r;
}

int64_t orc_ang2pix_nest(int order, double z, double phi, double* margin)
{
    const int64_t ns = (int64_t)1 << order;
    const double za = fabs(z);
    const double t = phi / ((PLANTED(5) ? 1.0 : 0.5) * ORC_PI);   /* in [0, 4) */
    int64_t face, ix, iy;
    double marg;
    if (za <= 2.0 / 3.0) {
        const double a = (double)ns * (0.5 + t);
        const double b = (double)ns * (z * 0.75);
        const double x_asc = a - b;                    /* lines rising with z  */
        const double x_dsc = a + b;                    /* lines falling with z */
        const int64_t jp = (int64_t)floor(x_asc);
        const int64_t jm = (int64_t)floor(x_dsc);
        marg = fmin(dist_to_int(x_asc), dist_to_int(x_dsc));
        const int64_t fp = jp >> order, fm = jm >> order;   /* 0..4 */
        if (fp == fm) face = (fp % 4) + 4;             /* equatorial row */
        else if (fp < fm) face = fp;                   /* north row */
        else face = fm + 8;                            /* south row */
        ix = jm & (ns - 1);
        iy = ns - (jp & (ns - 1)) - (PLANTED(4) ? 0 : 1);
    } else {
        int64_t q = (int64_t)t;                        /* quarter 0..3 */
        if (q > 3) q = 3;
        const double tq = t - (double)q;               /* longitude inside quarter */
        const double s = (double)ns * sqrt(3.0 * (1.0 - za));
        const double xa = tq * s, xb = (1.0 - tq) * s;
        int64_t jp = (int64_t)floor(xa);
        int64_t jm = (int64_t)floor(xb);
        marg = fmin(dist_to_int(xa), dist_to_int(xb));
        if (jp > ns - 1) jp = ns - 1;
        if (jm > ns - 1) jm = ns - 1;
        if (z > 0.0) { face = q;     ix = ns - jm - 1; iy = ns - jp - 1; }
        else         { face = q + 8; ix = jp;          iy = jm; }
    }
    if (margin) *margin = marg;
    return face * ns * ns + (int64_t)(spread_bits((uint64_t)ix) | (spread_bits((uint64_t)iy) << 1));
}

/* Centre of nested pixel `pix` at `order`: z = cos(colatitude), its sine
 * (computed without cancellation near the poles) and phi. The centre lies on
 * iso-latitude ring r = (row + 2) Ns - ix - iy - 1 (r = 1 .. 4 Ns - 1, from
 * the north), at a longitude fixed by the position inside the ring. */
void orc_pix2ang_nest(int order, int64_t pix, double* z, double* sin_theta, double* phi)
{
    const int64_t ns = (int64_t)1 << order;
    const int64_t npface = ns * ns;
    const int64_t face = pix / npface;
    const int64_t ipf = pix % npface;
    const int64_t ix = (int64_t)gather_bits((uint64_t)ipf);
    const int64_t iy = (int64_t)gather_bits((uint64_t)ipf >> 1);
    const int64_t row = face / 4;                       /* 0 north, 1 equator, 2 south */
    const int64_t col = face % 4;
    const int64_t ring = (row + 2) * ns - ix - iy - 1;
    /* longitude offset of the face's centre in units of pi/4 */
    const int64_t face_lon = (row == 1) ? 2 * col : 2 * col + 1;
    int64_t nr, shift;
    double zz, st;
    if (ring < ns) {                                    /* north cap */
        nr = ring;
        const double d = (double)(nr * nr) / (3.0 * (double)npface);   /* 1 - z */
        zz = 1.0 - d;
        st = sqrt(d * (2.0 - d));
        shift = 0;
    } else if (ring > 3 * ns) {                         /* south cap */
        nr = 4 * ns - ring;
        const double d = (double)(nr * nr) / (3.0 * (double)npface);   /* 1 + z */
        zz = d - 1.0;
        st = sqrt(d * (2.0 - d));
        shift = 0;
    } else {                                            /* equatorial belt */
        nr = ns;
        zz = (double)(2 * ns - ring) * (PLANTED(10) ? 4.0 : 2.0) / (3.0 * (double)ns);
        st = sqrt((1.0 - zz) * (1.0 + zz));
        shift = (ring - ns) & 1;
    }
    int64_t jpos = (face_lon * nr + ix - iy + 1 + shift) / 2;  /* 1 .. 4 nr */
    if (jpos > 4 * nr) jpos -= 4 * nr;
    if (jpos < 1) jpos += 4 * nr;
    *z = zz;
    *sin_theta = st;
    *phi = ((double)jpos - 0.5 * (double)(shift + 1)) * (0.5 * ORC_PI) / (double)nr;
}

/* Unit vector towards the centre of level-J pixel k, in the uvw frame,
 * returned as (s_u, s_v, s_w - 1). xyz has y towards the NCP, x towards RA 6h
 * and z towards RA 0h (Sec. 3.4); uvw = R^T xyz (R orthogonal, Eq. 18). */
void orc_pixel_dir_uvw(int J, int64_t k, double ra0, double dec0, double* out3)
{
    double z, st, phi, R[9];
    orc_pix2ang_nest(J - 1, k, &z, &st, &phi);
    const double x = st * sin(phi), y = z, zc = st * cos(phi);
    orc_rotation(ra0, dec0, R);
    const double su = R[0] * x + R[3] * y + R[6] * zc;
    const double sv = R[1] * x + R[4] * y + R[7] * zc;
    const double sw = R[2] * x + R[5] * y + R[8] * zc;
    out3[0] = su;
    out3[1] = sv;
    /* s_w - 1 without cancellation when s_w > 0 (reading R2's identity) */
    out3[2] = (sw > 0.0) ? (PLANTED(11) ? 1.0 : -1.0) * (su * su + sv * sv) / (1.0 + sw) : sw - 1.0;
}

/* Sec. 3.5 cross-reference: image position [l, m] -> SIN projection onto the
 * sphere [l, m, sqrt(1 - l^2 - m^2)] (Sec. 3.3) -> xyz by Eq. 18 -> (z, RA)
 * -> level-J pixel. */
int orc_map_components(int64_t n, const double* l, const double* m, double ra0, double dec0,
                       int J, int64_t* kJ, double* margin)
{
    if (J < 1 || J > 30 || n < 0) return -1;
    double R[9];
    orc_rotation(ra0, dec0, R);
    for (int64_t i = 0; i < n; ++i) {
        const double r2 = l[i] * l[i] + m[i] * m[i];
        if (!(r2 < 1.0)) return -2;
        const double c[3] = {l[i], m[i], sqrt(1.0 - r2)};
        const double x = R[0] * c[0] + R[1] * c[1] + R[2] * c[2];
        const double y = R[3] * c[0] + R[4] * c[1] + R[5] * c[2];
        const double zc = R[6] * c[0] + R[7] * c[1] + R[8] * c[2];
        double phi = atan2(x, zc);                     /* RA */
        if (phi < 0.0) phi += 2.0 * ORC_PI;
        if (phi >= 2.0 * ORC_PI) phi -= 2.0 * ORC_PI;
        double mg;
        kJ[i] = orc_ang2pix_nest(J - 1, y, phi, &mg);
        if (margin) margin[i] = mg;
    }
    return 0;
}

/* ========================================================================== */
/* Sec. 3.2 / 3.5 -- the coefficient tree                                     */
/* ========================================================================== */

/* A_j = 4 pi / N_j = (pi/3) 4^(1-j) and sqrt(A_j) = sqrt(pi/3) 2^(1-j) (R9). */
static double area_of_level(int j) { return ldexp(ORC_PI / 3.0, 2 * (1 - j)); }
static double sqrt_area_of_level(int j) { return ldexp(sqrt(ORC_PI / 3.0), 1 - j); }

/* A node of the tree of Sec. 3.5: pixel k at level j, up to four children at
 * level j + 1 (null = the whole branch is zero), the image coefficients and,
 * at level J, the pixel centre and the summed flux. */
typedef struct orc_node {
    int64_t key;
    int level;
    struct orc_node* child[4];
    double lambda;
    double gamma[3];
    double flux;          /* Phi_k, level J only */
    double dir[3];        /* (s_u, s_v, s_w - 1), level J only */
    int64_t bfs;          /* index in the breadth-first export */
} orc_node;

struct orc_tree {
    int J;
    double ra0, dec0;
    orc_node* roots[12];
    int64_t n_nodes, n_leaves;
    int64_t per_level[31];
    orc_node** bfs;       /* nodes in (level, key) order */
};

static orc_node* new_node(int64_t key, int level)
{
    orc_node* nd = (orc_node*)calloc(1, sizeof(orc_node));
    nd->key = key;
    nd->level = level;
    return nd;
}

static void free_nodes(orc_node* nd)
{
    if (!nd) return;
    for (int c = 0; c < 4; ++c) free_nodes(nd->child[c]);
    free(nd);
}

/* Eqs. 9 and 10 at one node, after its children are final (R7, R9). */
static void image_coefficients(orc_node* nd, int J)
{
    if (nd->level == J) return;
    double c[4];
    for (int s = 0; s < 4; ++s) {
        if (nd->child[s]) {
            image_coefficients(nd->child[s], J);
            c[s] = nd->child[s]->lambda;
        } else {
            c[s] = 0.0;
        }
    }
    const double q = sqrt_area_of_level(nd->level) * 0.25;
    nd->lambda = (PLANTED(6) ? 0.5 : 0.25) * (((c[0] + c[1]) + c[2]) + c[3]);
    nd->gamma[0] = q * (((c[0] - c[1]) + c[2]) - c[3]);
    nd->gamma[1] = q * (((c[0] + c[1]) - c[2]) + (PLANTED(7) ? c[3] : -c[3]));
    nd->gamma[2] = q * (((c[0] - c[1]) - c[2]) + c[3]);
}

static int cmp_key(const void* a, const void* b)
{
    const orc_node* x = *(orc_node* const*)a;
    const orc_node* y = *(orc_node* const*)b;
    return (x->key > y->key) - (x->key < y->key);
}

static void collect(orc_node* nd, orc_node*** lists, int64_t* fill)
{
    if (!nd) return;
    lists[nd->level][fill[nd->level]++] = nd;
    for (int c = 0; c < 4; ++c) collect(nd->child[c], lists, fill);
}

orc_tree* orc_tree_build(int64_t n, const double* l, const double* m, const double* flux,
                         double ra0, double dec0, int J)
{
    if (J < 1 || J > 30 || n < 0) return NULL;
    int64_t* kJ = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (orc_map_components(n, l, m, ra0, dec0, J, kJ, NULL) != 0) { free(kJ); return NULL; }
    orc_tree* t = (orc_tree*)calloc(1, sizeof(orc_tree));
    t->J = J;
    t->ra0 = ra0;
    t->dec0 = dec0;
    /* Sec. 3.5: for each component, create nodes k_1 .. k_J along its path
     * (k_j = k_J >> 2(J - j)) if absent, linking parent to child; the leaf's
     * plane-wave position (pixel centre) is set when the leaf is created.
     * Fluxes landing in one pixel are summed in input order (Sec. 3.3). */
    for (int64_t i = 0; i < n; ++i) {
        const int64_t k1 = kJ[i] >> (2 * (J - 1));
        if (!t->roots[k1]) {
            t->roots[k1] = new_node(k1, 1);
            if (J == 1) orc_pixel_dir_uvw(J, k1, ra0, dec0, t->roots[k1]->dir);
        }
        orc_node* nd = t->roots[k1];
        for (int j = 2; j <= J; ++j) {
            const int64_t kj = kJ[i] >> (2 * (J - j));
            const int slot = (int)(kj & 3);
            if (!nd->child[slot]) {
                nd->child[slot] = new_node(kj, j);
                if (j == J) orc_pixel_dir_uvw(J, kj, ra0, dec0, nd->child[slot]->dir);
            }
            nd = nd->child[slot];
        }
        nd->flux = (PLANTED(9) ? 0.0 : nd->flux) + flux[i];
    }
    free(kJ);
    /* Breadth-first lists, sorted by key within each level. */
    orc_node** lists[31];
    int64_t count[31] = {0}, fill[31] = {0};
    int64_t total = 0;
    /* count nodes per level */
    {
        orc_node** stack = NULL;
        int64_t cap = 0, sp = 0;
        for (int r = 0; r < 12; ++r) {
            if (!t->roots[r]) continue;
            if (sp == cap) { cap = cap ? 2 * cap : 64; stack = (orc_node**)realloc(stack, sizeof(orc_node*) * (size_t)cap); }
            stack[sp++] = t->roots[r];
        }
        while (sp > 0) {
            orc_node* nd = stack[--sp];
            count[nd->level]++;
            total++;
            for (int c = 0; c < 4; ++c)
                if (nd->child[c]) {
                    if (sp == cap) { cap = 2 * cap; stack = (orc_node**)realloc(stack, sizeof(orc_node*) * (size_t)cap); }
                    stack[sp++] = nd->child[c];
                }
        }
        free(stack);
    }
    for (int j = 1; j <= J; ++j) lists[j] = (orc_node**)malloc(sizeof(orc_node*) * (size_t)(count[j] > 0 ? count[j] : 1));
    for (int r = 0; r < 12; ++r) collect(t->roots[r], lists, fill);
    t->bfs = (orc_node**)malloc(sizeof(orc_node*) * (size_t)(total > 0 ? total : 1));
    int64_t pos = 0;
    for (int j = 1; j <= J; ++j) {
        qsort(lists[j], (size_t)count[j], sizeof(orc_node*), cmp_key);
        for (int64_t i = 0; i < count[j]; ++i) {
            lists[j][i]->bfs = pos;
            t->bfs[pos++] = lists[j][i];
        }
        t->per_level[j] = count[j];
        free(lists[j]);
    }
    t->n_nodes = total;
    t->n_leaves = count[J];
    /* Level J coefficients (R6), then Eqs. 9/10 recursively. */
    const double AJ = area_of_level(J);
    for (int64_t i = total - count[J]; i < total; ++i) t->bfs[i]->lambda = t->bfs[i]->flux / AJ;
    for (int r = 0; r < 12; ++r)
        if (t->roots[r]) image_coefficients(t->roots[r], J);
    return t;
}

void orc_tree_free(orc_tree* t)
{
    if (!t) return;
    for (int r = 0; r < 12; ++r) free_nodes(t->roots[r]);
    free(t->bfs);
    free(t);
}

int orc_tree_sizes(const orc_tree* t, int64_t* n_leaves, int64_t* n_nodes, int64_t* per_level)
{
    if (!t) return -1;
    if (n_leaves) *n_leaves = t->n_leaves;
    if (n_nodes) *n_nodes = t->n_nodes;
    if (per_level)
        for (int j = 1; j <= t->J; ++j) per_level[j - 1] = t->per_level[j];
    return 0;
}

int orc_tree_export(const orc_tree* t, int64_t* key, uint8_t* child_mask, int32_t* first_child,
                    double* lambda, double* gamma, double* leaf_dir, double* leaf_flux)
{
    if (!t) return -1;
    const int64_t leaf0 = t->n_nodes - t->n_leaves;
    for (int64_t i = 0; i < t->n_nodes; ++i) {
        const orc_node* nd = t->bfs[i];
        uint8_t mask = 0;
        int64_t first = -1;
        for (int c = 0; c < 4; ++c)
            if (nd->child[c]) {
                mask |= (uint8_t)(1u << c);
                if (first < 0) first = nd->child[c]->bfs;
            }
        if (key) key[i] = nd->key;
        if (child_mask) child_mask[i] = mask;
        if (first_child) first_child[i] = (int32_t)first;
        if (lambda) lambda[i] = nd->lambda;
        if (gamma) for (int q = 0; q < 3; ++q) gamma[3 * i + q] = (nd->level < t->J) ? nd->gamma[q] : 0.0;
        if (i >= leaf0) {
            if (leaf_dir) for (int q = 0; q < 3; ++q) leaf_dir[3 * (i - leaf0) + q] = nd->dir[q];
            if (leaf_flux) leaf_flux[i - leaf0] = nd->flux;
        }
    }
    return 0;
}

/* Plane wave F^P at direction d (Eq. 14): exp(sign i 2 pi B.(s - P)). */
static void plane_wave(const double* B, const double* d, int sign, double* re, double* im)
{
    double t = B[0] * d[0] + B[1] * d[1] + B[2] * d[2];
    t = t - rint(t);
    const double phase = 2.0 * ORC_PI * t;
    *re = cos(phase);
    *im = (double)sign * sin(phase);
}

/* Per-visibility Eq. 17 (Sec. 3.3 and 3.6.1): (1) the plane wave at the
 * level-J nodes, (2) the plane-wave coefficients eta (Eq. 9 form) and sigma
 * (Eq. 10 form) for j = J-1 .. 1, (3) the multiresolution sum. */
int orc_tree_vis_eq17(const orc_tree* t, int64_t n_vis, const double* uvw, int sign, double* vis)
{
    if (!t || n_vis < 0 || (sign != 1 && sign != -1)) return -1;
    const int64_t T = t->n_nodes, leaf0 = T - t->n_leaves;
    double* eta = (double*)malloc(sizeof(double) * 2 * (size_t)(T > 0 ? T : 1));
    double* sig = (double*)malloc(sizeof(double) * 6 * (size_t)(T > 0 ? T : 1));
    for (int64_t n = 0; n < n_vis; ++n) {
        const double* B = uvw + 3 * n;
        /* (1) level J */
        for (int64_t i = leaf0; i < T; ++i)
            plane_wave(B, t->bfs[i]->dir, sign, &eta[2 * i], &eta[2 * i + 1]);
        /* (2) levels J-1 .. 1; a level's nodes precede the next level's */
        for (int64_t i = leaf0 - 1; i >= 0; --i) {
            const orc_node* nd = t->bfs[i];
            const double q = sqrt_area_of_level(nd->level) * 0.25;
            for (int part = 0; part < 2; ++part) {
                double c[4];
                for (int s = 0; s < 4; ++s)
                    c[s] = nd->child[s] ? eta[2 * nd->child[s]->bfs + part] : 0.0;
                eta[2 * i + part] = 0.25 * (((c[0] + c[1]) + c[2]) + c[3]);
                sig[6 * i + 0 + part] = q * (((c[0] - c[1]) + c[2]) + (PLANTED(12) ? c[3] : -c[3]));
                sig[6 * i + 2 + part] = q * (((c[0] + c[1]) - c[2]) - c[3]);
                sig[6 * i + 4 + part] = q * (((c[0] - c[1]) - c[2]) + c[3]);
            }
        }
        /* (3) V = A_1 sum_k lambda_1 eta_1 + sum_{j<J} sum_k sum_m gamma sigma */
        double re = 0.0, im = 0.0;
        const double A1 = area_of_level(1);
        const int64_t n1 = t->per_level[1];
        if (t->J == 1) {
            for (int64_t i = 0; i < n1; ++i) {
                re += (PLANTED(8) ? 1.0 : A1) * (t->bfs[i]->lambda * eta[2 * i]);
                im += (PLANTED(8) ? 1.0 : A1) * (t->bfs[i]->lambda * eta[2 * i + 1]);
            }
        } else {
            for (int64_t i = 0; i < n1; ++i) {
                re += (PLANTED(8) ? 1.0 : A1) * (t->bfs[i]->lambda * eta[2 * i]);
                im += (PLANTED(8) ? 1.0 : A1) * (t->bfs[i]->lambda * eta[2 * i + 1]);
            }
            for (int64_t i = 0; i < leaf0; ++i)
                for (int mm = 0; mm < 3; ++mm) {
                    re += t->bfs[i]->gamma[mm] * sig[6 * i + 2 * mm];
                    im += t->bfs[i]->gamma[mm] * sig[6 * i + 2 * mm + 1];
                }
        }
        vis[2 * n] = re;
        vis[2 * n + 1] = im;
    }
    free(eta);
    free(sig);
    return 0;
}

/* Eq. 17 as orc_tree_vis_eq17, with the visibilities split into n_threads
 * contiguous ranges evaluated side by side by OpenMP threads (the CPU
 * baseline on all host cores). Every visibility is independent of the
 * others (Sec. 3.6.1), so each range runs the single-threaded routine above
 * unchanged and the results are identical bit for bit. */
int orc_tree_vis_eq17_mt(const orc_tree* t, int64_t n_vis, const double* uvw, int sign, double* vis,
                         int n_threads)
{
    if (!t || n_vis < 0 || (sign != 1 && sign != -1) || n_threads < 1) return -1;
    int rc = 0;
#pragma omp parallel for schedule(static) num_threads(n_threads) reduction(| : rc)
    for (int r = 0; r < n_threads; ++r) {
        const int64_t a = n_vis * r / n_threads, b = n_vis * (r + 1) / n_threads;
        rc |= (b > a) ? orc_tree_vis_eq17(t, b - a, uvw + 3 * a, sign, vis + 2 * a) : 0;
    }
    return rc;
}

/* Eq. 12 as orc_dft, on n_threads OpenMP threads over contiguous ranges of
 * the visibilities (identical results). */
int orc_dft_mt(int64_t n_comp, const double* l, const double* m, const double* flux,
               int64_t n_vis, const double* uvw, int sign, double* vis, int n_threads)
{
    if (n_comp < 0 || n_vis < 0 || (sign != 1 && sign != -1) || n_threads < 1) return -1;
    int rc = 0;
#pragma omp parallel for schedule(static) num_threads(n_threads) reduction(| : rc)
    for (int r = 0; r < n_threads; ++r) {
        const int64_t a = n_vis * r / n_threads, b = n_vis * (r + 1) / n_threads;
        rc |= (b > a) ? orc_dft(n_comp, l, m, flux, b - a, uvw + 3 * a, sign, vis + 2 * a) : 0;
    }
    return rc;
}

/* Per-visibility Eq. 16: V = A_J sum_k lambda_J,k eta_J,k (R6). */
int orc_tree_vis_eq16(const orc_tree* t, int64_t n_vis, const double* uvw, int sign, double* vis)
{
    if (!t || n_vis < 0 || (sign != 1 && sign != -1)) return -1;
    const int64_t T = t->n_nodes, leaf0 = T - t->n_leaves;
    const double AJ = area_of_level(t->J);
    for (int64_t n = 0; n < n_vis; ++n) {
        double re = 0.0, im = 0.0;
        for (int64_t i = leaf0; i < T; ++i) {
            double er, ei;
            plane_wave(uvw + 3 * n, t->bfs[i]->dir, sign, &er, &ei);
            re += AJ * (t->bfs[i]->lambda * er);
            im += AJ * (t->bfs[i]->lambda * ei);
        }
        vis[2 * n] = re;
        vis[2 * n + 1] = im;
    }
    return 0;
}

/* Reading R12 (the use of the learned response, an addition to the paper):
 * the tree truncated at level jt keeps its level-jt nodes, each with the
 * flux of its pixel F_k = A_jt lambda_jt,k (Eq. 9 averages the children, so
 * A_j lambda_j,k is the merged flux below the node), and predicts
 *     V = sum_k F_k exp(sign i 2 pi B.(c_k - P)) R_k(B)
 * with c_k the pixel centre and R_k(B):
 *   kind 0: 1 -- centre-snapped: Eq. 16 read at level jt;
 *   kind 1: R_jt(B), the response of the level-jt pixel holding the phase
 *           centre, for every k (what the per-level network learns);
 *   kind 2: R_jt,k(B), each pixel's own response (its flux spread uniformly
 *           over its area),
 * the responses by dense quadrature D levels down. Summed over the nodes in
 * breadth-first (key) order. */
int orc_tree_vis_truncated(const orc_tree* t, int jt, int kind, int D, int64_t n_vis, const double* uvw, int sign,
                           double* vis)
{
    if (!t || jt < 1 || jt > t->J || kind < 0 || kind > 2 || n_vis < 0 || (sign != 1 && sign != -1)) return -1;
    if (kind > 0 && (D < 0 || jt + D > 30 || D > 10)) return -1;
    double* R = NULL;
    if (kind > 0) {
        R = (double*)malloc(sizeof(double) * 2 * (size_t)(n_vis > 0 ? n_vis : 1));
        if (kind == 1 && orc_pixel_response(jt, D, t->ra0, t->dec0, n_vis, uvw, sign, R) != 0) {
            free(R);
            return -2;
        }
    }
    for (int64_t q = 0; q < 2 * n_vis; ++q) vis[q] = 0.0;
    const double Aj = area_of_level(jt);
    for (int64_t i = 0; i < t->n_nodes; ++i) {
        const orc_node* nd = t->bfs[i];
        if (nd->level != jt) continue;
        const double F = PLANTED(17) ? nd->lambda : Aj * nd->lambda;
        double c[3];
        orc_pixel_dir_uvw(jt, nd->key, t->ra0, t->dec0, c);
        if (kind == 2 && orc_pixel_response_of(jt, nd->key, D, t->ra0, t->dec0, n_vis, uvw, sign, R) != 0) {
            free(R);
            return -2;
        }
        for (int64_t q = 0; q < n_vis; ++q) {
            double er, ei;
            plane_wave(uvw + 3 * q, c, sign, &er, &ei);
            if (kind > 0) {
                const double rr = R[2 * q], ri = PLANTED(18) ? -R[2 * q + 1] : R[2 * q + 1];
                const double xr = er * rr - ei * ri, xi = er * ri + ei * rr;
                er = xr;
                ei = xi;
            }
            vis[2 * q] += F * er;
            vis[2 * q + 1] += F * ei;
        }
    }
    free(R);
    return 0;
}

/* Eq. 11 on the tree: for each child c of a node at level j,
 *   lambda_c = lambda_j + (1 / sqrt(A_j)) sum_m H[m][c] gamma^m_j,
 * with H the sign rows of Eq. 10. Top-down from level 1. */
int orc_tree_synthesis(const orc_tree* t, double* lambda_J)
{
    if (!t) return -1;
    static const double H[3][4] = {{1, -1, 1, -1}, {1, 1, -1, -1}, {1, -1, -1, 1}};
    const int64_t T = t->n_nodes, leaf0 = T - t->n_leaves;
    double* rec = (double*)malloc(sizeof(double) * (size_t)(T > 0 ? T : 1));
    for (int64_t i = 0; i < t->per_level[1]; ++i) rec[i] = t->bfs[i]->lambda;
    for (int64_t i = 0; i < leaf0; ++i) {
        const orc_node* nd = t->bfs[i];
        const double inv = 1.0 / sqrt_area_of_level(nd->level);
        for (int c = 0; c < 4; ++c) {
            if (!nd->child[c]) continue;
            const double d = (H[0][c] * nd->gamma[0] + H[1][c] * nd->gamma[1]) + H[2][c] * nd->gamma[2];
            rec[nd->child[c]->bfs] = rec[i] + inv * d;
        }
    }
    for (int64_t i = leaf0; i < T; ++i) lambda_J[i - leaf0] = rec[i];
    free(rec);
    return 0;
}

/* ========================================================================== */
/* Brute force on the dense pixel grid                                        */
/* ========================================================================== */

static int64_t pixels_at_level(int j) { return 12 * ((int64_t)1 << (2 * (j - 1))); }

int orc_dense_coeffs(int J, int64_t n, const double* l, const double* m, const double* flux,
                     double ra0, double dec0, double* lambda_all, double* gamma_all)
{
    if (J < 1 || J > 12) return -1;
    int64_t* kJ = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (orc_map_components(n, l, m, ra0, dec0, J, kJ, NULL) != 0) { free(kJ); return -2; }
    int64_t off[32];
    off[1] = 0;
    for (int j = 1; j <= J; ++j) off[j + 1] = off[j] + pixels_at_level(j);
    const int64_t NJ = pixels_at_level(J);
    double* lamJ = lambda_all + off[J];
    for (int64_t k = 0; k < NJ; ++k) lamJ[k] = 0.0;
    for (int64_t i = 0; i < n; ++i) lamJ[kJ[i]] += flux[i];
    const double AJ = area_of_level(J);
    for (int64_t k = 0; k < NJ; ++k) lamJ[k] = lamJ[k] / AJ;
    free(kJ);
    int64_t goff = 0;
    int64_t goffs[32];
    for (int j = 1; j < J; ++j) { goffs[j] = goff; goff += pixels_at_level(j); }
    for (int j = J - 1; j >= 1; --j) {
        const double q = sqrt_area_of_level(j) * 0.25;
        const double* ch = lambda_all + off[j + 1];
        double* lam = lambda_all + off[j];
        double* gam = gamma_all + 3 * goffs[j];
        for (int64_t k = 0; k < pixels_at_level(j); ++k) {
            const double c0 = ch[4 * k], c1 = ch[4 * k + 1], c2 = ch[4 * k + 2], c3 = ch[4 * k + 3];
            lam[k] = 0.25 * (((c0 + c1) + c2) + c3);
            gam[3 * k + 0] = q * (((c0 - c1) + c2) - c3);
            gam[3 * k + 1] = q * (((c0 + c1) - c2) - c3);
            gam[3 * k + 2] = q * (((c0 - c1) - c2) + c3);
        }
    }
    return 0;
}

int orc_dense_vis_eq17(int J, int64_t n, const double* l, const double* m, const double* flux,
                       double ra0, double dec0, int64_t n_vis, const double* uvw, int sign,
                       double* vis)
{
    if (J < 1 || J > 8) return -1;
    int64_t total = 0, off[32];
    for (int j = 1; j <= J; ++j) { off[j] = total; total += pixels_at_level(j); }
    double* lam = (double*)malloc(sizeof(double) * (size_t)total);
    double* gam = (double*)malloc(sizeof(double) * 3 * (size_t)total);
    if (orc_dense_coeffs(J, n, l, m, flux, ra0, dec0, lam, gam) != 0) { free(lam); free(gam); return -2; }
    int64_t goff[32], g = 0;
    for (int j = 1; j < J; ++j) { goff[j] = g; g += pixels_at_level(j); }
    const int64_t NJ = pixels_at_level(J);
    double* dirs = (double*)malloc(sizeof(double) * 3 * (size_t)NJ);
    for (int64_t k = 0; k < NJ; ++k) orc_pixel_dir_uvw(J, k, ra0, dec0, dirs + 3 * k);
    double* eta = (double*)malloc(sizeof(double) * 2 * (size_t)total);
    double* sig = (double*)malloc(sizeof(double) * 6 * (size_t)total);
    for (int64_t nv = 0; nv < n_vis; ++nv) {
        const double* B = uvw + 3 * nv;
        for (int64_t k = 0; k < NJ; ++k)
            plane_wave(B, dirs + 3 * k, sign, &eta[2 * (off[J] + k)], &eta[2 * (off[J] + k) + 1]);
        for (int j = J - 1; j >= 1; --j) {
            const double q = sqrt_area_of_level(j) * 0.25;
            for (int64_t k = 0; k < pixels_at_level(j); ++k) {
                const int64_t p = off[j] + k;
                for (int part = 0; part < 2; ++part) {
                    double c[4];
                    for (int s = 0; s < 4; ++s) c[s] = eta[2 * (off[j + 1] + 4 * k + s) + part];
                    eta[2 * p + part] = 0.25 * (((c[0] + c[1]) + c[2]) + c[3]);
                    sig[6 * p + 0 + part] = q * (((c[0] - c[1]) + c[2]) - c[3]);
                    sig[6 * p + 2 + part] = q * (((c[0] + c[1]) - c[2]) - c[3]);
                    sig[6 * p + 4 + part] = q * (((c[0] - c[1]) - c[2]) + c[3]);
                }
            }
        }
        double re = 0.0, im = 0.0;
        const double A1 = area_of_level(1);
        for (int64_t k = 0; k < 12; ++k) {
            re += A1 * (lam[k] * eta[2 * k]);
            im += A1 * (lam[k] * eta[2 * k + 1]);
        }
        for (int j = 1; j < J; ++j)
            for (int64_t k = 0; k < pixels_at_level(j); ++k)
                for (int mm = 0; mm < 3; ++mm) {
                    const int64_t p = off[j] + k;
                    re += gam[3 * (goff[j] + k) + mm] * sig[6 * p + 2 * mm];
                    im += gam[3 * (goff[j] + k) + mm] * sig[6 * p + 2 * mm + 1];
                }
        vis[2 * nv] = re;
        vis[2 * nv + 1] = im;
    }
    free(lam); free(gam); free(dirs); free(eta); free(sig);
    return 0;
}

/* ========================================================================== */
/* Helpers                                                                    */
/* ========================================================================== */

/* Sec. 3.3: pixel size Delta theta_j = 2^(1-j) sqrt(pi/3); Table 1 picks the
 * smallest J whose pixel oversamples the dirty-image pixel by two. */
int orc_recommended_J(double dtheta_rad)
{
    if (!(dtheta_rad > 0.0)) return -1;
    for (int J = 1; J <= 30; ++J)
        if (ldexp(sqrt(ORC_PI / 3.0), 1 - J) <= 0.5 * dtheta_rad) return J;
    return -2;
}

int orc_subtract(int64_t n_vis, const double* obs, const double* model, double* resid)
{
    if (n_vis < 0) return -1;
    for (int64_t i = 0; i < 2 * n_vis; ++i) resid[i] = obs[i] - model[i];
    return 0;
}
