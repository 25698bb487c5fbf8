/*
 * wtvis.h -- C ABI of libwtvis: GB300 (sm_103a) model-visibility prediction
 * for the major cycle of CLEAN, after Skipper, Scaife & McEwen,
 * "Cleaning radio interferometric images using a spherical wavelet
 * decomposition" (arXiv:1909.03956).
 *
 * Two routes compute the model visibilities of a clean-component list:
 *   - the direct sum over components (Sec. 3.3, Eq. 12): dft_predict_vis;
 *   - the spherical Haar wavelet route (Sec. 3.2-3.5, Eqs. 9, 10, 16, 17):
 *     wt_build_tree maps the components onto a nested pixelisation of the
 *     celestial sphere and keeps the nonzero scaling/wavelet coefficients in
 *     a tree; wt_predict_vis evaluates, per visibility, the plane wave's
 *     coefficients on that tree and the multiresolution sum.
 * The direct sum, and Eq. 16 over the tree's leaves, can form their phases
 * on the tensor cores (WT_MIXED_TC). subtract_model forms the residual
 * visibilities (Sec. 2.2, major-cycle step 2).
 *
 * Conventions (all entry points):
 *   - Pointers are DEVICE pointers unless the comment says host. The caller
 *     owns every input and output buffer; the library owns only wt_tree
 *     handles (and their device memory) and the scratch it allocates inside
 *     a call.
 *   - uvw is an array of n_vis baselines [u, v, w] in wavelengths, row-major
 *     (24 bytes per visibility), float64. The exponent of Eq. 1 is then
 *     dimensionless.
 *   - Components are (l, m, flux): float64 direction cosines relative to the
 *     phase centre (Sec. 2.2; l east, m north) and float64 fluxes.
 *   - Visibilities are interleaved complex: complex128 ([re, im] float64
 *     pairs) in the WT_FP64 and WT_FP64_DF modes, complex64 ([re, im]
 *     float32 pairs) in the others (WT_MIXED, WT_MIXED_FAST, WT_MIXED_TC).
 *   - sign = +1 evaluates exp(+i 2 pi B.(s - P)) as printed in Eqs. 1, 12
 *     and 14; sign = -1 the conjugate convention.
 *   - stream is a cudaStream_t (NULL = legacy default stream). Every call is
 *     asynchronous on that stream unless its comment says otherwise.
 *   - Return value: WT_OK or a negative wt_status. Argument errors are
 *     detected on the host and returned at once, before anything is
 *     enqueued. Errors found by a kernel (a component with l^2 + m^2 >= 1, a
 *     non-finite input, a wait that ran out of time) are recorded in a
 *     per-device status word that wt_device_status() reads and clears.
 *   - wt_last_error() gives a text message for the calling thread's last
 *     failing call.
 *   - There is no CPU fallback: without a usable CUDA device every compute
 *     entry point returns WT_ERR_CUDA.
 */
#ifndef WTVIS_H
#define WTVIS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wt_tree_s* wt_tree;     /* opaque, owned by the library */

typedef enum {
    WT_OK = 0,
    WT_ERR_ARG = -1,          /* null pointer, negative size, bad mode/sign */
    WT_ERR_RANGE = -2,        /* J outside 1..30, l^2 + m^2 >= 1, non-finite input */
    WT_ERR_CUDA = -3,         /* a CUDA call failed (message in wt_last_error) */
    WT_ERR_NOMEM = -4,        /* device allocation failed */
    WT_ERR_TIMEOUT = -5,      /* a bounded device-side wait ran out */
    WT_ERR_CORRUPT = -6,      /* a tree handle failed validation */
    WT_ERR_UNSUPPORTED = -7   /* mode not available for this entry point */
} wt_status;

typedef enum {
    WT_FP64 = 0,     /* float64 throughout, complex128 output */
    WT_MIXED = 1,    /* float64-accurate phase (double-float), float32 sincos and
                        compensated float32 accumulation, complex64 output */
    WT_LEARNED = 2,  /* wavelet route only: learned per-level response (MLP) */
    WT_MIXED_FAST = 3, /* as WT_MIXED, but sin/cos of the reduced phase from the
                         special-function unit: at most ~7e-7 of a term's flux in
                         error per term (measured against the oracle); complex64 */
    WT_FP64_DF = 4,   /* float64-class accuracy on the float32 pipe: phase, sin/cos
                         (table method) and every sum in double-float arithmetic
                         (48-bit significands: a term's phase error is a few times
                         2^-48 |B.s| turns, 32x float64's); complex128 output;
                         wt_predict_vis with WT_SUM_EQ17_REGROUPED or
                         WT_SUM_EQ16 */
    WT_MIXED_TC = 5   /* dft_predict_vis, and wt_predict_vis with WT_SUM_EQ16
                         (a direct sum over the leaves): WT_MIXED_FAST's sin/cos
                         and sums, with the phase contraction
                         u l + v m + w (n - 1) on the tensor cores from exact
                         11-bit float16 slices of the baselines and coordinates
                         (three FP32 accumulators, recombined modulo 1 in
                         float32; phase error below 2^-29 turns); tiles of 128
                         visibilities beyond 2^14 turns per coordinate fall
                         back to WT_MIXED_FAST's exact pass; faster than
                         WT_MIXED_FAST from about 150 terms on; complex64 */
} wt_mode;

typedef enum {
    WT_SUM_EQ17 = 0,          /* multiresolution sum over all tree nodes (Eq. 17):
                                 per node eta and sigma^m formed, gamma^m sigma^m added */
    WT_SUM_EQ16 = 1,          /* level-J sum over the leaves only (Eq. 16) */
    WT_SUM_EQ17_REGROUPED = 2 /* Eq. 17 with each node's sum_m gamma^m sigma^m
                                 distributed over its children: per node a weight
                                 w = (sqrt(A_j)/4) sum_m H_m[c] gamma^m_parent, fixed per
                                 major cycle, and V = sum_n w_n eta_n (same terms,
                                 regrouped; the eta recursion is unchanged) */
} wt_sum;

/* ---------------------------------------------------------------------------
 * wt_build_tree -- Sec. 3.5 (the algorithm) with Sec. 3.3 (SIN projection),
 * Sec. 3.4 / Eq. 18 (uvw -> xyz rotation) and Eqs. 9, 10 (coefficients).
 *
 * Maps the n_comp components to pixels of level J of the HEALPix-nested
 * pixelisation of Sec. 3.2 (N_j = 12 * 4^(j-1) pixels at level j; the pole
 * axis is the NCP and the longitude the RA), merges components that share a
 * level-J pixel (Phi_k = summed flux, in input order), builds every ancestor
 * k_j = k_J >> 2(J - j), and computes the image coefficients:
 *   lambda_J,k = Phi_k / A_J,   A_j = 4 pi / N_j,
 *   lambda_j,k = (1/4) sum of the four children (absent child = 0)   (Eq. 9)
 *   gamma^m_j,k = (sqrt(A_j)/4) (H_m . children)                      (Eq. 10)
 * in the same rounding order as the paper's formulas read left to right, so
 * that keys, topology and coefficients are reproducible bit for bit.
 *
 *   l, m, flux  device float64 [n_comp]; l^2 + m^2 < 1 required.
 *   n_comp      >= 0 (0 gives an empty tree whose visibilities are 0).
 *   ra0, dec0   phase centre (radians).
 *   J           level, 1 <= J <= 30.
 *   out         host pointer receiving the new handle (freed by wt_free_tree).
 * The call allocates the tree's device memory, enqueues the build on
 * `stream` and returns without waiting. Input buffers may be reused once
 * the stream has passed the build.
 * ------------------------------------------------------------------------- */
int wt_build_tree(const double* l, const double* m, const double* flux, int64_t n_comp,
                  double ra0, double dec0, int J, wt_tree* out, void* stream);

/* ---------------------------------------------------------------------------
 * wt_xref_table -- Sec. 3.5: the cross-reference table built before
 * cleaning, which maps every pixel of the dirty image to its pixel k_J on
 * the sphere at level J. Pixel (ix, iy) of an n x n image of pixel size dl
 * sits at l = (ix - n/2) dl, m = (iy - n/2) dl (the imaging convention
 * below) and is mapped exactly as wt_build_tree maps a component there.
 *   table   device int64 [n][n] (row-major, iy n + ix), written; -1 where
 *           l^2 + m^2 >= 1
 *   n       1..16384; dl > 0 radians; J 1..30
 * Asynchronous on `stream`.
 * ------------------------------------------------------------------------- */
int wt_xref_table(int n, double dl, double ra0, double dec0, int J, int64_t* table, void* stream);

/* wt_build_tree_xref -- Sec. 3.5: the tree of components found at image
 * pixels (the clean components of a minor cycle): component i at pixel
 * pix[i] (row-major iy n + ix) with flux[i], its k_J read from a table made
 * by wt_xref_table with the same n, dl, ra0, dec0 and J (the table carries
 * none of them: the caller keeps them consistent). Everything after the
 * mapping is wt_build_tree's, so the tree equals wt_build_tree of the pixel
 * centres' (l, m) bit for bit.
 *   table  device int64 [n][n]; pix device int32 [n_comp];
 *   flux   device float64 [n_comp]
 * A pixel index outside 0..n*n-1 or a pixel outside the unit disc, or a
 * non-finite flux, records WT_ERR_RANGE in the device status word. */
int wt_build_tree_xref(const int64_t* table, int n, const int32_t* pix, const double* flux, int64_t n_comp,
                       double ra0, double dec0, int J, wt_tree* out, void* stream);

/* Sizes of a built tree (host outputs; any may be NULL). Waits for the
 * build's stream. nodes_per_level has J entries, level 1 first. */
int wt_tree_info(wt_tree t, int* J, int64_t* n_leaves, int64_t* n_nodes, int64_t* nodes_per_level);

/* Copy a built tree to HOST buffers in breadth-first order: nodes sorted by
 * (level ascending, pixel key ascending). Waits for the build's stream.
 *   key [n_nodes]            nested pixel index k_j of each node
 *   child_mask [n_nodes]     bit c set when child 4k + c exists (0 for leaves)
 *   first_child [n_nodes]    breadth-first index of the first child, -1 for leaves
 *   lambda [n_nodes]         scaling coefficient (Eq. 9; level J: Phi / A_J)
 *   gamma [n_nodes][3]       wavelet coefficients (Eq. 10; 0 for leaves)
 *   leaf_dir [n_leaves][3]   pixel centre in the uvw frame as (s_u, s_v, s_w - 1)
 *   leaf_flux [n_leaves]     Phi_k, the merged flux of each leaf
 * Any pointer may be NULL to skip that array. */
int wt_tree_export(wt_tree t, int64_t* key, uint8_t* child_mask, int32_t* first_child,
                   double* lambda, double* gamma, double* leaf_dir, double* leaf_flux);

/* wt_tree_import -- the inverse of wt_tree_export, for checkpoint and resume
 * of a major cycle's tree (the paper has no counterpart). A tree is fully
 * determined by its leaves: their level-J keys and merged fluxes Phi_k, as
 * wt_tree_export returns them (the last n_leaves keys, and leaf_flux); every
 * other coefficient follows by Eqs. 9 and 10 in the same rounding order, so
 * the imported tree equals the exported one bit for bit (its keys, topology,
 * lambda, gamma, pixel centres and predictions).
 *   leaf_keys  HOST int64 [n_leaves]: distinct, ascending, 0 .. 12 4^(J-1) - 1
 *   leaf_flux  HOST float64 [n_leaves], finite
 *   ra0, dec0, J as for wt_build_tree; out receives the handle.
 * Argument errors (keys out of range or out of order) are returned before
 * anything is enqueued; the build is enqueued on `stream`. */
int wt_tree_import(const int64_t* leaf_keys, const double* leaf_flux, int64_t n_leaves, double ra0, double dec0,
                   int J, wt_tree* out, void* stream);

/* Release a tree handle and its device memory (synchronises with the
 * stream the tree was built on). NULL is ignored. */
void wt_free_tree(wt_tree t);

/* ---------------------------------------------------------------------------
 * wt_predict_vis -- Sec. 3.3 (Eqs. 13-17) and Sec. 3.6.1 (per-visibility
 * steps): for each baseline B_n,
 *   1. the plane wave F^P (Eq. 14) at every leaf pixel centre: eta_J,k;
 *   2. the plane wave's coefficients for j = J-1 .. 1, bottom-up:
 *      eta_j,k = (1/4) sum of children, sigma^m_j,k = (sqrt(A_j)/4) H_m . children
 *      (absent child = 0; Sec. 3.5: empty branches are skipped);
 *   3. the multiresolution sum (Eq. 17 with the area factor of level 1):
 *      V = A_1 sum_k lambda_1,k eta_1,k + sum_j sum_k sum_m gamma^m sigma^m.
 * With which = WT_SUM_EQ16 the level-J sum V = sum_k Phi_k eta_J,k (Eq. 16)
 * is evaluated instead, and with WT_SUM_EQ17_REGROUPED the regrouped Eq. 17
 * (see wt_sum); all three agree up to rounding.
 *
 *   t        a built tree (the build must precede this call in stream order)
 *   uvw      device float64 [n_vis][3], wavelengths
 *   vis_out  device complex128 [n_vis] (WT_FP64, WT_FP64_DF) or complex64 [n_vis] (WT_MIXED,
 *            WT_MIXED_FAST)
 *   mode     WT_FP64, WT_FP64_DF (regrouped Eq. 17 or Eq. 16), WT_MIXED or
 *            WT_MIXED_FAST (WT_LEARNED: see
 *            wt_predict_vis_learned)
 *   which    wt_sum
 * ------------------------------------------------------------------------- */
int wt_predict_vis(wt_tree t, const double* uvw, int64_t n_vis, void* vis_out,
                   int mode, int sign, int which, void* stream);

/* ---------------------------------------------------------------------------
 * wt_predict_vis_batched -- wt_predict_vis (Eq. 17) for many channels (or
 * major cycles) at once: channel c has its own tree trees[c] and frequency
 * freq_hz[c]; the baselines are shared, in metres, and scaled per channel to
 * wavelengths, u_lambda = u_m f_c / c (c = 299 792 458 m/s).
 *
 *   trees    HOST array [n_ch] of built trees (any mix of J and sizes)
 *   freq_hz  HOST array [n_ch], > 0
 *   uvw_m    device float64 [n_vis][3], metres
 *   vis_out  device [n_ch][n_vis], complex128 (WT_FP64, WT_FP64_DF) or complex64
 *            (WT_MIXED, WT_MIXED_FAST)
 *   mode     WT_FP64 (explicit Eq. 17), WT_FP64_DF, WT_MIXED or WT_MIXED_FAST
 *            (regrouped Eq. 17); sign +1 / -1
 * All channels run in one kernel of one CTA per (channel, tile) work item,
 * largest trees first. The first call for
 * a given (trees, freq_hz, mode, sign) builds a plan: it reads the trees'
 * sizes (waiting for their build streams), times the fitting launch shapes
 * on the caller's stream (skipped under WT_AUTOTUNE=0 or when the stream is
 * being captured) and captures [counter reset + kernel] into a CUDA graph;
 * later calls with the same buffers replay that graph. Freeing any of the
 * trees drops the plans that use it.
 * ------------------------------------------------------------------------- */
int wt_predict_vis_batched(const wt_tree* trees, const double* freq_hz, int n_ch, const double* uvw_m,
                           int64_t n_vis, void* vis_out, int mode, int sign, void* stream);

/* ---------------------------------------------------------------------------
 * dft_predict_vis -- Sec. 3.3, Eq. 12: the direct sum over the component list
 *   V_n = sum_m C_m exp(sign i 2 pi [u_n l_m + v_n m_m + w_n (n_m - 1)]),
 *   n_m = sqrt(1 - l_m^2 - m_m^2),
 * the "more accurate alternative" of Sec. 2.2. Components are staged through
 * a device scratch buffer the call allocates and releases on `stream`.
 *   l, m, flux  device float64 [n_comp]
 *   uvw         device float64 [n_vis][3]
 *   vis_out     device complex128 (WT_FP64, WT_FP64_DF) or complex64
 *               (WT_MIXED, WT_MIXED_FAST, WT_MIXED_TC) [n_vis]
 *   mode        WT_FP64, WT_FP64_DF, WT_MIXED, WT_MIXED_FAST or WT_MIXED_TC
 * ------------------------------------------------------------------------- */
int dft_predict_vis(const double* l, const double* m, const double* flux, int64_t n_comp,
                    const double* uvw, int64_t n_vis, void* vis_out, int mode, int sign,
                    void* stream);

/* ---------------------------------------------------------------------------
 * dft_predict_vis_noalloc -- the same direct sum as dft_predict_vis, for
 * callers that cannot allocate device memory while they run: an application
 * that reserves its whole device-memory budget at start-up and forbids
 * allocation afterwards (an allocation could fail, or stall behind the
 * allocator's synchronisation), or a host framework that owns every device
 * allocation. The paper has no counterpart; this is plumbing.
 *
 * Nothing is allocated: the packed component records go to a fixed array in
 * the library's device image, WT_NOALLOC_MAX_COMPONENTS records of 32 bytes
 * (2 MiB), and the mixed forms' coordinate bounds to a 16-byte one beside
 * it, which every GPU that loads the library holds until the process exits.
 * n_comp above that limit returns WT_ERR_RANGE before anything is enqueued.
 * The call enqueues the pack kernel and the direct-sum kernel (the mixed
 * forms: a memset of the bounds, then a grid pass and an exact pass, as
 * dft_predict_vis does).
 *   - The first call on a device looks up the arrays' device addresses with
 *     that device current, and so does the first call in a new context on
 *     that device (after cudaDeviceReset, say); make that first call before
 *     any stream capture.
 *   - mode: WT_FP64 or WT_FP64_DF (complex128 out), WT_MIXED or
 *     WT_MIXED_FAST (complex64 out), as for dft_predict_vis; WT_MIXED_TC,
 *     whose operand for the tensor cores needs more room than the fixed
 *     array, returns WT_ERR_ARG.
 *   - All calls on a device share the array and it keeps the last call's
 *     records. Calls whose work overlaps on the GPU (e.g. on two streams with
 *     no ordering between them) race on it and give wrong results; order
 *     them on one stream.
 *   - status: optional caller-owned device int; kernels record the first
 *     device-side error there (WT_ERR_RANGE for a component with
 *     l^2 + m^2 >= 1 or a non-finite input) and leave it untouched otherwise.
 *     With status = NULL such errors are not reported.
 * Arguments otherwise as dft_predict_vis.
 * ------------------------------------------------------------------------- */
#define WT_NOALLOC_MAX_COMPONENTS 65536
int dft_predict_vis_noalloc(const double* l, const double* m, const double* flux, int64_t n_comp,
                            const double* uvw, int64_t n_vis, void* vis_out, int mode, int sign,
                            int* status, void* stream);

/* ---------------------------------------------------------------------------
 * subtract_model -- Sec. 2.2, major-cycle step 2: V_resid = V - V_M,
 * element by element. vis_resid may alias vis_obs (in place).
 *   mode WT_FP64 or WT_FP64_DF: complex128 arrays; any other mode: complex64
 *   arrays.
 * ------------------------------------------------------------------------- */
int subtract_model(const void* vis_obs, const void* vis_model, void* vis_resid,
                   int64_t n_vis, int mode, void* stream);

/* ---------------------------------------------------------------------------
 * The imaging half of the major cycle (Sec. 2.2: Hogbom clean, Eqs. 4-6, and
 * the Cotton-Schwab steps after Eq. 6). Conventions: an n x n float32 image,
 * n even, pixel size dl radians, pixel (ix, iy) at l = (ix - n/2) dl,
 * m = (iy - n/2) dl, stored row-major [iy][ix]; visibilities complex64 with
 * uvw in wavelengths (device float64 [n_vis][3]). Gridding is nearest-cell
 * (cell size 1/(n dl)) with unit weights, each visibility with its Hermitian
 * conjugate at -B; a visibility whose cell falls outside the grid is left
 * out; w is not used in imaging (the 2-D transform of Eq. 2). The 2-D FFT is
 * cuFFT's, loaded at the first call (WT_ERR_UNSUPPORTED if libcufft.so.12
 * cannot be loaded).
 * ------------------------------------------------------------------------- */

/* wt_dirty_image -- major-cycle step 3: grid and transform to the dirty image
 *   I(l, m) = (1/W) Re sum_cells G(u, v) exp(-i 2 pi (ul + vm)),
 * W = the number of gridded entries, so a unit point source at the phase
 * centre images to 1. vis = NULL gives the dirty beam (the image of unit
 * visibilities, 1 at pixel (n/2, n/2)).
 *   vis    device complex64 [n_vis], or NULL
 *   image  device float32 [n][n], written
 * Allocates an n x n complex64 scratch grid on `stream` and releases it. */
int wt_dirty_image(const double* uvw, const void* vis, int64_t n_vis, int n, double dl, float* image,
                   void* stream);

/* wt_dirty_image_w -- the w-corrected dirty image (the wide-field imaging of
 * Sec. 3.6.2, which grids over w-planes with an anti-aliasing kernel and a
 * w-kernel):
 *   I(l, m) = (1/W) Re sum_entries V exp(-i 2 pi (u l + v m + w (n(l, m) - 1))),
 * n(l, m) = sqrt(1 - l^2 - m^2), over each visibility and its conjugate at
 * -B, W the number of entries gridded; the same geometry and normalisation
 * as wt_dirty_image, which it equals at w = 0 up to the gridding
 * approximation. Convolutional gridding: a Kaiser-Bessel kernel of width 7
 * cells (the image divided by its Fourier transform afterwards) convolved
 * with each plane's w-kernel, tabulated at 8 points per cell over a support
 * of 2h + 1 cells (h from the field's largest chirp frequency, at most 32),
 * for w_planes planes uniformly spaced in |w| over [0, w_max] and
 * interpolated linearly in |w|. A visibility whose kernel support would
 * leave the grid is left out (and not counted in W); |w| above w_max takes
 * the last plane's kernel (a w_max below the batch's largest |w| degrades
 * the image, it does not fail).
 *   w_planes  2 .. 1024
 *   w_max     the largest |w| to plan for; 0: the batch's own, found on the
 *             device (this synchronises `stream`)
 * WT_ERR_RANGE if the field n dl reaches beyond l^2 + m^2 < 1 or the kernel
 * would need h > 32 or would not fit the grid. Allocates scratch on
 * `stream` (the grid and the kernel tables, tens of MB) and releases it. */
int wt_dirty_image_w(const double* uvw, const void* vis, int64_t n_vis, int n, double dl, int w_planes,
                     double w_max, float* image, void* stream);

/* wt_hogbom -- Eqs. 4-5: Hogbom clean of `image` in place. Each iteration
 * takes the pixel with the largest value C (ties: the first in row-major
 * order), records the component g C there, and subtracts g C times the beam
 * centred on it wherever the shifted beam overlaps the image (float32,
 * fl(I - fl(f B))). Stops after max_iter components or when the largest
 * value falls below `threshold`.
 *   image      device float32 [n][n], cleaned in place (the residual)
 *   psf        device float32 [n][n], the beam with its centre at (n/2, n/2)
 *   comp_pix   device int32 [max_iter]: row-major pixel index iy n + ix
 *   comp_flux  device float32 [max_iter]: g C of each component
 *   n_comp     device int32: the number of components recorded
 * gain in (0, 1]. Asynchronous. When the image's rows fit in shared memory
 * across the GPU's CTAs (n up to about 2700 on 152 SMs) the whole clean is
 * one cooperative launch whose CTAs meet at a grid barrier per iteration
 * (bounded waits: WT_ERR_TIMEOUT in the device status word if one runs out,
 * the image and the components then undefined); otherwise one launch per
 * iteration. WT_HOGBOM=launches in the environment forces the latter. The
 * two give identical results. */
int wt_hogbom(float* image, const float* psf, int n, float gain, float threshold, int max_iter, int* comp_pix,
              float* comp_flux, int* n_comp, void* stream);

/* wt_clean -- Cotton-Schwab major cycles (Sec. 2.2) around the paper's
 * prediction: the dirty beam once; then per major cycle the dirty image of
 * the residual visibilities, up to minor_iter Hogbom iterations, model
 * visibilities from every component found so far (predictor
 * WT_PREDICT_TREE: the tree at level J, its components mapped through the
 * cross-reference table of the image pixels built once per call
 * (wt_xref_table, wt_build_tree_xref), and the regrouped Eq. 17;
 * WT_PREDICT_DIRECT: the direct sum, Eq. 12), and V_resid = V - V_M. Ends
 * after n_major cycles or a cycle that finds no component, and leaves the
 * dirty image of the final residual visibilities in image_resid.
 *   vis_obs     device complex64 [n_vis]
 *   mode        WT_MIXED or WT_MIXED_FAST (the prediction's form), or
 *               WT_MIXED_TC with WT_PREDICT_DIRECT (the direct sum with its
 *               phases on the tensor cores)
 *   w_planes    0: the images as wt_dirty_image (nearest cell, no w term);
 *               2 .. 1024: as wt_dirty_image_w with that many w-planes over
 *               the batch's largest |w| (found once: one more stream
 *               synchronisation), the beam included
 *   comp_pix, comp_flux  device [minor_iter * n_major], as wt_hogbom,
 *               every cycle's components in order
 *   n_comp      HOST int32: the number of components found
 *   vis_resid   device complex64 [n_vis], written
 *   image_resid device float32 [n][n], written
 * Components sit at pixel centres (l, m) of the image. Synchronises the
 * stream once per major cycle (to read the component count); allocates its
 * scratch on `stream` and releases it. */
#define WT_PREDICT_TREE 0
#define WT_PREDICT_DIRECT 1
int wt_clean(const double* uvw, const void* vis_obs, int64_t n_vis, int n, double dl, double ra0, double dec0,
             int J, int predictor, int mode, float gain, float threshold, int minor_iter, int n_major, int w_planes,
             int* comp_pix, float* comp_flux, int* n_comp, void* vis_resid, float* image_resid, void* stream);

/* ---------------------------------------------------------------------------
 * Learned response (an addition to the paper's method).
 *
 * For level j, R_j(B) = 4^-D sum_i exp(i 2 pi B.(s_i - c_j)) over the 4^D
 * descendants s_i, D levels down, of the level-j pixel c_j holding the phase
 * centre: the plane wave's level-j scaling coefficient on a fully populated
 * sub-tree (the Eq. 9 recursion), demodulated by the plane wave at c_j. A
 * per-level network 3 -> 64 -> 64 -> 2 (SiLU; BF16 weights, FP32
 * accumulation on the tensor cores) maps x = B Delta theta_j
 * (Delta theta_j = 2^(1-j) sqrt(pi/3), Sec. 3.3) to (Re R, Im R). Where
 * |x|_inf > x_max (outside the trained domain) the exact sum is used.
 * Parameters: 4546 float32 in the order W1[64][3], b1[64], W2[64][64],
 * b2[64], W3[2][64], b3[2]. All entry points below synchronise with the
 * device where they say so; uvw is device float64 [n][3] in wavelengths.
 * ------------------------------------------------------------------------- */
typedef struct wt_mlp_s* wt_mlp;

/* New network for `level`, seeded random weights; depth = D (0..8) of the
 * exact response used as fallback; x_max bounds the trained domain.
 * Synchronises the device. */
int wt_mlp_create(int level, double ra0, double dec0, int depth, float x_max, uint64_t seed, wt_mlp* out);
void wt_mlp_free(wt_mlp m);
/* Host copies of the 4546 float32 parameters (both synchronise). */
int wt_mlp_get_params(wt_mlp m, float* host_params);
int wt_mlp_set_params(wt_mlp m, const float* host_params);
/* Exact R_j(B) in float64 (the fallback and the yardstick); out: device
 * complex128 [n]. sign = -1 gives the conjugate. */
int wt_response_exact(int level, int depth, double ra0, double dec0, const double* uvw, int64_t n, int sign,
                      void* out, void* stream);
/* Mean squared error of both outputs against target (device float32
 * [n][2]) and its gradient (HOST float32 [4546]); synchronises `stream`.
 * The forward pass rounds W2 and the hidden activations to BF16 exactly as
 * inference does. */
int wt_mlp_loss_grad(wt_mlp m, const double* uvw, const float* target, int64_t n, float* loss, float* grad,
                     void* stream);
/* `steps` Adam steps (cosine-decayed rate from lr) on contiguous minibatches
 * of `batch` samples taken cyclically from (uvw, target); final_loss (host,
 * may be NULL) receives the last minibatch's loss (synchronises). */
int wt_mlp_train(wt_mlp m, const double* uvw, const float* target, int64_t n, int steps, int batch, float lr,
                 float* final_loss, void* stream);
/* Steps step0 .. step0 + steps - 1 of a training run of total_steps Adam
 * steps: the learning rate of step i is the run's cosine-decayed
 * 0.5 lr (1 + cos(pi i / total_steps)), its minibatch the samples
 * i batch .. (i + 1) batch - 1 (mod n). wt_mlp_train is the whole run
 * (step0 = 0, total_steps = steps). The gradient is reduced over the CTAs in
 * a fixed order, so a run cut into ranges -- with the optimiser state saved
 * by wt_mlp_get_state and restored by wt_mlp_set_state in between -- ends
 * with the same parameters, bit for bit, as the uninterrupted run. */
int wt_mlp_train_range(wt_mlp m, const double* uvw, const float* target, int64_t n, int64_t step0, int steps,
                       int64_t total_steps, int batch, float lr, float* final_loss, void* stream);
/* Checkpoint and resume of training: the parameters, Adam's first and
 * second moments (HOST float32 [4546] each, the parameter order above) and
 * its step count. Parameters and state travel only as host arrays: writing
 * them to a file, and reading them back, is the caller's. Both synchronise
 * the device. */
int wt_mlp_get_state(wt_mlp m, float* host_params, float* host_m, float* host_v, int64_t* step);
int wt_mlp_set_state(wt_mlp m, const float* host_params, const float* host_m, const float* host_v, int64_t step);
/* R(B) by the network (exact sum beyond x_max); out: device complex64 [n]. */
int wt_mlp_eval(wt_mlp m, const double* uvw, int64_t n, int sign, void* out, void* stream);
/* Learned form of the tree prediction: V = R_J(B) sum_k Phi_k exp(sign i 2 pi
 * B.(c_k - P)) -- the level-J sum (Eq. 16, fast mixed form) with each leaf's
 * centre-snapped plane wave replaced by the pixel's full response. The network's level must
 * equal the tree's J and the phase centres must match. Output complex64. */
int wt_predict_vis_learned(wt_tree t, wt_mlp m, const double* uvw, int64_t n_vis, void* vis_out, int sign,
                           void* stream);

/* ---------------------------------------------------------------------------
 * wt_predict_vis_truncated -- the tree truncated at one level, the use of
 * the per-level response (an addition to the paper's method). The level's
 * nodes stand for their pixels, each with its pixel's flux
 * F_k = A_level lambda_level,k (Eq. 9: the merged flux below the node):
 *   V = R(B) sum_k F_k exp(sign i 2 pi B.(c_k - P))
 * (c_k the pixel centres, the sum in the fast mixed form, or, for a level
 * of at least WT_TRUNCATED_TC_MIN_NODES nodes, in WT_MIXED_TC: the same
 * terms with the phases on the tensor cores, faster there; the call then
 * waits once for the tree's build stream to read the level's size), with
 *   response = WT_RESPONSE_SNAPPED: R = 1, each pixel's flux at its centre
 *              (Eq. 16 read at the truncation level);
 *              WT_RESPONSE_LEARNED: R = the network m of that level (exact
 *              sum beyond its x_max), the flux spread over each pixel;
 *              WT_RESPONSE_EXACT: R = the exact response of the level-`level`
 *              pixel holding the phase centre, `depth` levels of sub-pixels
 *              (float64; the learned form's yardstick).
 * All pixels of the level share one response: the change of pixel shape
 * across the field is neglected. level 1..J of the tree; m (LEARNED) must be
 * for that level and the tree's phase centre; depth (EXACT) 0..8. Output
 * device complex64 [n_vis]. Allocates scratch on `stream` and releases it.
 * ------------------------------------------------------------------------- */
#define WT_TRUNCATED_TC_MIN_NODES 160
#define WT_RESPONSE_SNAPPED 0
#define WT_RESPONSE_LEARNED 1
#define WT_RESPONSE_EXACT 2
int wt_predict_vis_truncated(wt_tree t, int level, int response, wt_mlp m, int depth, const double* uvw,
                             int64_t n_vis, void* vis_out, int sign, void* stream);

/* ---------------------------------------------------------------------------
 * wt_predict_vis_thresholded -- hard thresholding of the wavelet
 * coefficients with full-pixel responses (Sec. 1 recalls McEwen (2008),
 * which keeps only the largest coefficients; an addition to the paper's own
 * method). Every coefficient above level j0 is kept, so the coarse part is
 * the tree truncated at j0 (wt_predict_vis_truncated); of the coefficients
 * gamma^m_j,k of levels j0 .. J-1 only those with |gamma| >= tau are kept,
 * each through the responses of all four of its node's children (present
 * in the tree or not):
 *   V = R_j0(B) sum_k F_k exp(sign i 2 pi B.(c_k - P))
 *     + sum_{L = j0+1..J} R_L(B) sum_c w_c exp(sign i 2 pi B.(c_c - P)),
 *   w_c = (sqrt(A_j)/4) sum_{m kept} H_m[c] gamma^m_parent   (Eq. 10 form),
 * the c running over the children at level L of the parents with a kept
 * coefficient. The Haar wavelets are orthonormal on the sphere, so this is
 * the visibility of the best image of so many coefficients; tau = 0 keeps
 * all. R_L: 1 (WT_RESPONSE_SNAPPED); the networks mlps[L - j0] (HOST array
 * of J - j0 + 1, levels j0 .. J; WT_RESPONSE_LEARNED); or the exact response
 * of the phase-centre pixel with depth - (L - j0) levels of sub-pixels (one
 * common finest level j0 + depth; J - j0 <= depth <= 8; WT_RESPONSE_EXACT).
 * As in wt_predict_vis_truncated all pixels of a level share one response,
 * and level j0's sum runs on the tensor cores when that level has at least
 * WT_TRUNCATED_TC_MIN_NODES nodes (the finer levels' sums, whose sizes the
 * device decides, in the fast mixed form).
 * Output device complex64 [n_vis]; the selection runs on the device
 * (deterministic). Allocates scratch on `stream` and releases it.
 * ------------------------------------------------------------------------- */
int wt_predict_vis_thresholded(wt_tree t, int j0, double tau, int response, const wt_mlp* mlps, int depth,
                               const double* uvw, int64_t n_vis, void* vis_out, int sign, void* stream);

/* ---------------------------------------------------------------------------
 * Helpers
 * ------------------------------------------------------------------------- */

/* Sec. 3.3 and Table 1: the smallest J whose pixel size
 * Delta theta_J = 2^(1-J) sqrt(pi/3) is at most half of dtheta (radians),
 * i.e. the sphere oversamples the image pixel by two. Host only. Returns
 * WT_ERR_ARG for dtheta <= 0 and WT_ERR_RANGE when J would exceed 30. */
int wt_recommended_J(double dtheta_rad);

/* Read and clear the device status word of the current device after
 * synchronising `stream`: WT_OK, or the first error a kernel recorded.
 * WT_ERR_TIMEOUT means a bounded wait ran out: the results of that call are
 * undefined, and since a bulk copy that never arrived may still land later,
 * later results on the device are not to be trusted either. */
int wt_device_status(void* stream);

/* Failure-detection self-test: a one-CTA kernel waits, with at most
 * spin_limit (1..65536) polls, on an mbarrier phase that never completes, gives
 * up and records WT_ERR_TIMEOUT in the device status word -- the path every
 * bounded wait of the library takes when a copy does not arrive. The kernel
 * returns normally; read the outcome with wt_device_status(). */
int wt_selftest_bounded_wait(uint32_t spin_limit, void* stream);

/* Failure-detection self-test of the grid barrier of the persistent Hogbom
 * clean (wt_hogbom): a two-CTA cooperative launch meets at a barrier that
 * never opens (its arrival count starts past the grid size); each CTA gives
 * up after spin_limit (1..65536) polls and WT_ERR_TIMEOUT is recorded in the
 * device status word. The kernel returns normally; read the outcome with
 * wt_device_status(). WT_ERR_UNSUPPORTED without cooperative launches. */
int wt_selftest_grid_barrier(uint32_t spin_limit, void* stream);

/* wt_measure_pipe_rates -- the issue rates of the arithmetic pipes the
 * predictors run on, measured on the current device (the denominators of
 * their rooflines; the paper has no counterpart). One CTA of 512 threads per
 * SM runs eight independent dependency chains per thread of one operation,
 * timed by its SM's own cycle counter; the median over the SMs is returned.
 *   per_clk_per_sm  HOST double [7], written: operations per clock per SM of
 *                   [0] float32 FMA, [1] float32 packed-pair FMA (elements),
 *                   [2] float64 FMA, [3] special-function-unit sine,
 *                   [4] tanh (PTX tanh.approx.f32), [5] tanh on packed
 *                   BF16 pairs (tanh.approx.bf16x2, elements), [6] 2^x
 *                   (ex2.approx.ftz.f32)
 * Allocates a few KB of scratch on `stream`, runs about 10 ms of kernels and
 * synchronises `stream`. */
int wt_measure_pipe_rates(double* per_clk_per_sm, void* stream);

/* Self-test of the library's per-context state (the device status word and
 * the device address of dft_predict_vis_noalloc's fixed array; the paper has
 * no counterpart): one component of flux 3 at the phase centre through
 * dft_predict_vis_noalloc (V = 3 exactly), then cudaDeviceReset on the
 * current device, then the same again in the new context. Returns WT_OK when
 * both rounds give V = 3 and a clear status word. cudaDeviceReset ends this
 * process's context on the device: every device pointer, stream and tree
 * handle of the process on it becomes invalid, so call this only from a
 * process that holds nothing on the device. Synchronises. */
int wt_selftest_context_reset(void);

/* Text of the calling thread's last error (never NULL). */
const char* wt_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* WTVIS_H */
