/*
 * oracle.h -- plain FP64 CPU oracle for the model-visibility prediction of
 * Skipper, Scaife & McEwen, "Cleaning radio interferometric images using a
 * spherical wavelet decomposition" (arXiv:1909.03956).
 *
 * TEST INFRASTRUCTURE. Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this code. The CUDA library never
 * links, includes or calls it, and it shares no code, header or table with
 * the CUDA library.
 *
 * Everything here is double precision, compiled with -ffp-contract=off so
 * that every operation rounds once, in the order written.
 *
 * Conventions shared by every function:
 *   - uvw is an array of n_vis baselines [u, v, w] in wavelengths (Sec. 2.1,
 *     Eq. 1: the exponent is dimensionless, so B is in units of wavelength).
 *   - vis is an array of n_vis complex values stored as [re, im] pairs.
 *   - sign is +1 for the paper's convention exp(+i 2 pi B.(s - P)) (Eq. 12,
 *     Eq. 14) and -1 for the conjugate convention.
 *   - Components are (flux C_i, image-plane direction cosines l_i, m_i) of the
 *     clean-component list (Sec. 2.2, Eq. 5).
 *   - J is the most detailed wavelet level (Sec. 3.2); level j has
 *     N_j = 12 * 4^(j-1) pixels, HEALPix nested order j-1.
 */
#ifndef WT_ORACLE_H
#define WT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- Eq. 12: direct sum over the component list --------------------------- */
int orc_dft(int64_t n_comp, const double* l, const double* m, const double* flux,
            int64_t n_vis, const double* uvw, int sign, double* vis);
/* Same definition evaluated in long double (extended or quad precision). */
int orc_dft_ld(int64_t n_comp, const double* l, const double* m, const double* flux,
               int64_t n_vis, const double* uvw, int sign, double* vis);

/* ---- Sec. 3.4, Eq. 18: uvw -> xyz rotation, row-major 3x3 ----------------- */
void orc_rotation(double ra0, double dec0, double* R);

/* ---- Sec. 3.2: nested sphere pixelisation (Gorski et al. 2005 geometry) --- */
/* z = cos(colatitude) measured from +y (the NCP), phi = RA in [0, 2 pi).
 * margin (may be NULL) receives the smallest distance, in pixel-grid units,
 * between a floor() argument and an integer: a measure of how close the point
 * lies to a pixel edge. */
int64_t orc_ang2pix_nest(int order, double z, double phi, double* margin);
void orc_pix2ang_nest(int order, int64_t pix, double* z, double* sin_theta, double* phi);
/* Unit vector of the centre of level-J pixel k in the uvw frame: (s_u, s_v, s_w - 1). */
void orc_pixel_dir_uvw(int J, int64_t k, double ra0, double dec0, double* out3);
/* Map components to level-J pixels (Sec. 3.5 cross-reference): SIN projection
 * (Sec. 3.3), rotation Eq. 18, then the level-J pixel index. */
int orc_map_components(int64_t n, const double* l, const double* m, double ra0, double dec0,
                       int J, int64_t* kJ, double* margin);

/* ---- Sec. 3.5: the coefficient tree --------------------------------------- */
typedef struct orc_tree orc_tree;
orc_tree* orc_tree_build(int64_t n, const double* l, const double* m, const double* flux,
                         double ra0, double dec0, int J);
void orc_tree_free(orc_tree* t);
int orc_tree_sizes(const orc_tree* t, int64_t* n_leaves, int64_t* n_nodes, int64_t* per_level);
/* Breadth-first export: nodes ordered by (level ascending, key ascending). */
int orc_tree_export(const orc_tree* t, int64_t* key, uint8_t* child_mask, int32_t* first_child,
                    double* lambda, double* gamma /* [n_nodes][3] */,
                    double* leaf_dir /* [n_leaves][3] */, double* leaf_flux);
/* Eq. 17 with the area factors (multiresolution sum). */
int orc_tree_vis_eq17(const orc_tree* t, int64_t n_vis, const double* uvw, int sign, double* vis);
/* Eq. 16 with the area factor (level-J sum). */
int orc_tree_vis_eq17_mt(const orc_tree* t, int64_t n_vis, const double* uvw, int sign, double* vis,
                         int n_threads);
int orc_dft_mt(int64_t n_comp, const double* l, const double* m, const double* flux,
               int64_t n_vis, const double* uvw, int sign, double* vis, int n_threads);
int orc_tree_vis_eq16(const orc_tree* t, int64_t n_vis, const double* uvw, int sign, double* vis);
/* Eq. 11 synthesis restricted to the tree: rebuild lambda_J from lambda_1 and
 * the gammas, top-down; out receives one value per leaf in BFS order. */
int orc_tree_synthesis(const orc_tree* t, double* lambda_J);

/* ---- Brute force on the dense pixel grid (small J only) ------------------- */
/* Dense lambda_j for every pixel of every level (levels concatenated, level 1
 * first) and gamma^m_j for levels 1..J-1 ([pixel][3], concatenated). */
int orc_dense_coeffs(int J, int64_t n, const double* l, const double* m, const double* flux,
                     double ra0, double dec0, double* lambda_all, double* gamma_all);
/* Eq. 17 over every pixel of every level (zero coefficients included). */
int orc_dense_vis_eq17(int J, int64_t n, const double* l, const double* m, const double* flux,
                       double ra0, double dec0, int64_t n_vis, const double* uvw, int sign,
                       double* vis);

/* ---- Learned response (oracle_mlp.c; an addition, not in the paper) -------- */
/* Exact per-level pixel response R_j(B) over the 4^D descendants of the
 * level-j pixel holding the phase centre (see oracle_mlp.c). out: [n][2]. */
int orc_pixel_response_of(int j, int64_t k, int D, double ra0, double dec0, int64_t n, const double* uvw, int sign,
                          double* out);
int orc_tree_vis_truncated(const orc_tree* t, int jt, int kind, int D, int64_t n_vis, const double* uvw, int sign,
                           double* vis);
int orc_pixel_response(int j, int D, double ra0, double dec0, int64_t n, const double* uvw, int sign,
                       double* out);
double orc_level_pixel_size(int j);
int orc_mlp_n_params(void);
int orc_mlp_forward(const double* params, int level, int64_t n, const double* uvw, double* y);
int orc_mlp_loss_grad(const double* params, int level, int64_t n, const double* uvw, const double* target,
                      double* loss, double* grad);

/* ---- Helpers ---------------------------------------------------------------- */
/* Sec. 3.3: smallest J with Delta theta_J <= dtheta / 2 (Table 1 rule). */
int orc_recommended_J(double dtheta_rad);
/* Sec. 2.2, major-cycle step 2: resid = obs - model, complex pairs. */
int orc_subtract(int64_t n_vis, const double* obs, const double* model, double* resid);

#ifdef __cplusplus
}
#endif
#endif
