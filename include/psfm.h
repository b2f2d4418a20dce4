/*
 * psfm.h -- C ABI of the GB300 PSF-matching library (libpsfm.so).
 *
 * The library implements the data-parallel hot path of the PSF-matching method of Price &
 * Magnier, "Pan-STARRS PSF-Matching for Subtraction and Stacking" (arXiv:1901.09999):
 *   - solving for a spatially varying convolution kernel K that matches the PSF of a
 *     reference image I1 to a science image I2 (Sec. 2, Eq. 2-6 with c_i = 0, p_i = 0),
 *     with the ISIS Gaussian x polynomial basis (Eq. 7), stamps chosen per subregion and
 *     discrepant stamps rejected over several iterations (Sec. 3.2-3.6);
 *   - applying K to the whole image (Eq. 12), propagating the variance map (Eq. 13), the
 *     covariance pseudo-matrix (Eq. 10-11, Sec. 4.3-4.4) and the mask (Sec. 3.4);
 *   - PSF-homogenised stacking of several inputs (Sec. 5.1).
 *
 * Conventions shared by every entry point
 *   Images are row-major, indexed [y][x] with x the fast axis, and share one row pitch
 *   (in elements, >= width) given in psfm_shape.  float images are IEEE binary32;
 *   masks are uint16 bit sets.  Unless a parameter says "host", every array pointer is
 *   DEVICE memory on the current CUDA device, owned by the caller; the library never
 *   frees or retains it.  Scratch memory comes from the caller's `workspace` (device,
 *   256-byte aligned, at least psfm_workspace_size() bytes); the library allocates no
 *   device memory on these paths.
 *   Work is enqueued on `stream` (0 = legacy default stream).  psfm_convolve is
 *   asynchronous; psfm_solve_kernel, psfm_subtract and psfm_stack synchronise `stream`
 *   before returning because they fill host-side results.
 *   Errors are returned as psfm_status; no exception or signal crosses the ABI.  Outputs
 *   are undefined unless the call returns PSFM_OK.  Invalid sizes or pointers are rejected
 *   with PSFM_ERR_BAD_ARG before any work is enqueued.
 *
 * Kernel convention (Eq. 12): O(x, y) = sum_{u,v} K_{x,y}(u, v) R(x-u, y-v) + d0, where
 *   R is I1 with masked pixels set to zero (Sec. 3.4), off-image pixels count as zero,
 *   and K_{x,y} = b0 delta + sum_k a_k(x, y) B_k with a_k(x, y) = sum_s a_{k,s} g_s(x, y),
 *   g_s = xt^l yt^m, xt = 2x/(W-1) - 1, yt = 2y/(H-1) - 1 (Sec. 2).
 * Basis (Eq. 7): for Gaussian g (width sigma_g, degree d_g) and p + q <= d_g,
 *   B'_k(u, v) = psi_k u^p v^q exp(-(u^2+v^2) / (2 sigma_g^2)), psi_k giving unit L2 norm,
 *   and B_k = B'_k - s_k delta with s_k = sum B'_k for p, q both even (else 0), so that
 *   every B_k has zero sum (Sec. 2).
 * Coefficient order ("canonical"): g ascending, then p = 0..d_g, then q = 0..d_g - p, then
 *   the spatial term (l, m) with l = 0..S, m = 0..S-l; index = k * N_s + s.
 */
#ifndef PSFM_H
#define PSFM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* psfm_stream; /* same handle as cudaStream_t */

typedef int32_t psfm_status;
#define PSFM_OK 0
#define PSFM_ERR_BAD_ARG 1        /* invalid size, pointer, alignment or option */
#define PSFM_ERR_TOO_FEW_STAMPS 2 /* fewer than 3 usable stamps (Sec. 3.7 quality cut) */
#define PSFM_ERR_SINGULAR 3       /* normal equations not solvable (Cholesky and LU fail) */
#define PSFM_ERR_NONFINITE 4      /* NaN or Inf in an unmasked input pixel used by the fit */
#define PSFM_ERR_CUDA 5           /* a CUDA runtime call or kernel launch failed */
#define PSFM_ERR_TIMEOUT 6        /* a bounded device-side wait ran out */
#define PSFM_ERR_WORKSPACE 8      /* workspace too small, or a fixed-capacity table overflowed */
#define PSFM_ERR_UNSUPPORTED 9    /* option combination this build does not implement */

#define PSFM_MAX_GAUSS 4
#define PSFM_MAX_DEGREE 8
#define PSFM_MAX_HALF_WIDTH 24
#define PSFM_MAX_SPATIAL_ORDER 3

/* Image geometry: width W (x), height H (y), row pitch in elements (>= W). */
typedef struct {
  int32_t width, height;
  int64_t pitch;
} psfm_shape;

/* Stamp centre pixel (Sec. 3.3). */
typedef struct {
  int32_t x, y;
} psfm_stamp;

/* ISIS kernel basis (Eq. 7): n_gauss Gaussians of width sigma[g] (pixels) carrying
 * polynomials of total degree degree[g]; kernel (2*half_width+1)^2; spatial polynomial
 * order spatial_order (Sec. 2).  bg_order must be 0 (constant differential background d0). */
typedef struct {
  int32_t n_gauss;
  double sigma[PSFM_MAX_GAUSS];
  int32_t degree[PSFM_MAX_GAUSS];
  int32_t half_width;
  int32_t spatial_order;
  int32_t bg_order;
} psfm_basis_spec;

#define PSFM_NORM_SEPARATE 0 /* b0, d0 first, unweighted footprint sums (Sec. 3.2) */
#define PSFM_NORM_JOINT 1    /* b0, d0 in the weighted fit with the kernel terms */

/* Arithmetic of the stamp design blocks and their Gram matrices (the normal equations are
 * always assembled and solved in FP64; the image, variance and mask passes are FP32). */
#define PSFM_PREC_FP64 0     /* design and Gram in FP64 (slow on this GPU's FP64 pipes) */
#define PSFM_PREC_FP32 1     /* FP32 design and products, FP64 sums over 32-pixel chunks */
#define PSFM_PREC_TF32 2     /* FP32 design; Gram on the tensor cores, TF32 products, FP32 sums */
#define PSFM_PREC_BF16X3 3   /* FP32 design; Gram on the tensor cores from a BF16 hi/lo split,
                                3 products (hi*hi + hi*lo + lo*hi), FP32 sums */
#define PSFM_PREC_F32X2 4    /* design and Gram in double-float (FP32 pairs, ~48 bits) */
#define PSFM_PREC_BF16X6 5   /* double-float design; Gram on the tensor cores as
                                (sqrt(w) C)^T (sqrt(w) C) from seven BF16 slices of the scaled
                                columns, exact per-level sums (>= 48 bits); a basis with more
                                than 64 augmented columns takes the double-float Gram */

/* Options; psfm_config_default() fills the defaults noted in brackets. */
typedef struct {
  int32_t grid_nx, grid_ny; /* stamp subregion grid [6, 5] (Sec. 3.3) */
  int32_t stamp_half;       /* s: stamps are (2s+1)^2 pixels; < 0 means s = half_width [-1] */
  int32_t max_cand;         /* candidates kept per subregion, 1..16 [8] */
  double thresh_nsigma;     /* detection threshold over background [5] (Sec. 3.3) */
  double reject_nsigma;     /* reject chi2 > mean + this * std [3] (Sec. 3.3) */
  double soften_alpha;      /* chi2 denominator V1 + V2 + alpha |I2| [0.1] (Sec. 3.6) */
  double bad_frac;          /* CONV.BAD radius: K^2 outside <= bad_frac of total [0.2] (Sec. 3.4) */
  int32_t max_iter;         /* solves of the rejection loop, 1..16 [5] */
  int32_t var_tile;         /* constant-kernel patch for variance, 8..256 [64] (Sec. 4.4) */
  int32_t cov_grid;         /* n x n kernels averaged for the pseudo-matrix, 1..8 [5] (Sec. 4.4) */
  int32_t norm_mode;        /* PSFM_NORM_* [SEPARATE] */
  int32_t precision;        /* PSFM_PREC_* [FP64] */
  uint16_t badmask;         /* input mask bits that mark a pixel unusable [0x00FF] */
  uint16_t conv_bad;        /* CONV.BAD output bit [1 << 14] */
  uint16_t conv_poor;       /* CONV.POOR output bit [1 << 15] */
  uint16_t nodata;          /* stack pixel with no contributing input [1 << 0] */
  int32_t dual;             /* 1: convolve both images, D = K2 (x) I2 - K1 (x) I1 - d0 with
                               K2 = delta - sum_i c_i g_i k_i (Eq. 2, c_i != 0); needs
                               precision F32X2, the science image and white inputs (no
                               cov_ref / cov_img); the solution holds 2 N_b N_s coefficients
                               (b terms, then c terms); the stacks and psfm_convolve_noalloc
                               return PSFM_ERR_UNSUPPORTED for it [0] */
  double penalty;           /* dual only: lambda of the penalty Phi p_i, p_i = sum (u^2+v^2)^2
                               k_i^2, Phi = lambda * sum M_ii / sum p_i over the kernel unknowns
                               (Sec. 2) [0.01] */
} psfm_config;

#define PSFM_CAND_UNUSED 0
#define PSFM_CAND_USED 1
#define PSFM_CAND_REJECTED 2

/* Result of a kernel solve.  All pointers are HOST memory owned by the caller; any of
 * coeff, cand, cand_status, chi2 may be NULL to skip that output.  Candidate tables are
 * laid out [region][rank], region = j * grid_nx + i (or one region per caller stamp). */
typedef struct {
  double b0;             /* normalisation (kernel sum), Sec. 3.2 */
  double d0;             /* differential background */
  double* coeff;         /* [n_coeff] canonical order a_{k,s} */
  int32_t n_coeff;       /* capacity of coeff; must be >= N_b * N_s when coeff != NULL */
  int32_t n_regions;     /* filled: number of regions */
  int32_t max_cand;      /* filled: candidates per region */
  int32_t cand_capacity; /* capacity of cand / cand_status / chi2 in entries */
  psfm_stamp* cand;      /* [n_regions * max_cand] candidate centres, (-1,-1) = empty */
  int32_t* cand_status;  /* PSFM_CAND_* */
  double* chi2;          /* last chi^2 of each candidate, NaN if never active */
  int32_t n_used;        /* stamps in the final solve */
  int32_t n_iter;        /* solves performed */
  int32_t r_bad;         /* CONV.BAD box radius (Sec. 3.4) */
  double chi2_mean;      /* mean chi^2 over the final stamps (Sec. 3.6) */
  double chi2_rms;       /* population std of chi^2 over the final stamps */
  float median;          /* background of the detection image I1 + I2 */
  /* Quality diagnostics (Sec. 3.7), from the kernel K realised at the image centre in FP64
   * (u, v the kernel offsets, sums over the (2h+1)^2 box): */
  double kernel_sum;     /* sum K */
  double mom_x, mom_y;   /* first moments sum u K / sum K, sum v K / sum K */
  double mom_xx, mom_yy, mom_xy;  /* central second moments, e.g. sum (u - mom_x)^2 K / sum K */
  double deconv_max;     /* max over r = 0..h of sum_{u^2+v^2 <= r^2} K / sum K (> 1: deconvolution) */
  int32_t quality_flags; /* PSFM_QUALITY_* bits: the paper's recommended cuts */
} psfm_solution;

/* Quality cuts recommended for flagging bad subtractions (Sec. 3.7).  The two deviation
 * cuts are applied to chi2_mean and chi2_rms as defined above (softened chi^2 with
 * sigma^2 = V1 + V2), the reading taken of the paper's normalised deviations. */
#define PSFM_QUALITY_FEW_STAMPS 1  /* n_used < 3 */
#define PSFM_QUALITY_MEAN_DEV 2    /* chi2_mean > 0.5 */
#define PSFM_QUALITY_RMS_DEV 4     /* chi2_rms > 0.3 */
#define PSFM_QUALITY_MOMENT1 8     /* |mom_x| > 0.5 or |mom_y| > 0.5 */
#define PSFM_QUALITY_MOMENT2 16    /* mom_xx < 0 or mom_yy < 0 */
#define PSFM_QUALITY_DECONV 32     /* deconv_max > 1.03 */

/* Fill `cfg` with the defaults listed in psfm_config. */
void psfm_config_default(psfm_config* cfg);

/* Human-readable name of a status code (static storage). */
const char* psfm_status_string(psfm_status s);

/* Number of basis terms N_b, spatial terms N_s and the width of the output covariance
 * pseudo-matrix for an input pseudo-matrix of width cov_in_w (1 for white noise) combined
 * with a science pseudo-matrix of width cov_img_w (0 if not subtracting): 2w + c - 2 with
 * w = 2h+1 (Sec. 4.3), at least cov_img_w.  Return -1 on an invalid basis. */
int32_t psfm_basis_size(const psfm_basis_spec* basis);
int32_t psfm_spatial_size(const psfm_basis_spec* basis);
int32_t psfm_cov_width(const psfm_basis_spec* basis, int32_t cov_in_w, int32_t cov_img_w);

#define PSFM_OP_SOLVE 1
#define PSFM_OP_CONVOLVE 2
#define PSFM_OP_SUBTRACT 3
#define PSFM_OP_STACK 4

/* Bytes of device workspace an operation needs for this geometry and options
 * (n_stamps: caller stamps, 0 to run the extractor; for PSFM_OP_STACK, the number of
 * sources of the largest input).  0 on invalid arguments. */
size_t psfm_workspace_size(int32_t op, psfm_shape shape, const psfm_basis_spec* basis,
                           const psfm_config* cfg, int32_t n_stamps);

/* Solve for the PSF-matching kernel (Sec. 2 Eq. 2-6 with c_i = p_i = 0; Sec. 3.2-3.6).
 *   img = I2 (science, target), ref = I1 (reference, to be convolved); var_* are their
 *   variance maps; mask_* their masks (pixels with any `badmask` bit are unusable).
 *   Weights in the fit are 1 / (V1 + V2) (Eq. 5-6).
 *   stamps / n_stamps: caller-chosen stamp centres (host), one region each, no
 *   replacement; n_stamps == 0 runs the extractor (grid_nx x grid_ny subregions, up to
 *   max_cand candidates each, replacement on rejection).
 *   out: host result (see psfm_solution).  Synchronises `stream`. */
psfm_status psfm_solve_kernel(const float* img, const float* ref, const float* var_img,
                              const float* var_ref, const uint16_t* mask_img,
                              const uint16_t* mask_ref, psfm_shape shape,
                              const psfm_stamp* stamps, int32_t n_stamps,
                              const psfm_basis_spec* basis, const psfm_config* cfg,
                              psfm_solution* out, void* workspace, size_t ws_bytes,
                              psfm_stream stream);

/* Apply a solved kernel (Eq. 12-13, Sec. 3.4, Sec. 4.3-4.4).
 *   ref, var_ref, mask_ref: I1 and its variance and mask (device).
 *   img, var_img, mask_img: I2 and its maps, or all NULL.  With img set the outputs are the
 *     difference D = I2 - (K (x) I1 + d0), its variance V2 + V' and mask m1 | m2 | flags;
 *     without, the convolved image K (x) I1 + d0, V' and m1 | flags.
 *   sol: host solution (b0, d0, coeff, r_bad are read).
 *   cov_ref (device, cov_ref_w^2 doubles, odd width, centre = zero lag) is the input
 *     pseudo-matrix of I1, NULL for white noise; cov_img likewise for I2 (difference only).
 *   out, out_var, out_mask: device outputs with the input pitch; out_var / out_mask may be
 *     NULL to skip them.  cov_out: device, cov_out_w^2 doubles, may be NULL; cov_out_w must
 *     equal psfm_cov_width(basis, cov_ref_w or 1, cov_img_w or (img ? 1 : 0)).
 *   V'(x, y) = f_t sum K_t(u,v)^2 V1(x-u, y-v) with K_t realised at the centre of the
 *     var_tile x var_tile patch t and f_t its covariance factor (Sec. 4.4).
 *   Asynchronous on `stream`. */
psfm_status psfm_convolve(const float* ref, const float* var_ref, const uint16_t* mask_ref,
                          const float* img, const float* var_img, const uint16_t* mask_img,
                          psfm_shape shape, const psfm_basis_spec* basis,
                          const psfm_config* cfg, const psfm_solution* sol,
                          const double* cov_ref, int32_t cov_ref_w, const double* cov_img,
                          int32_t cov_img_w, float* out, float* out_var, uint16_t* out_mask,
                          double* cov_out, int32_t cov_out_w, void* workspace,
                          size_t ws_bytes, psfm_stream stream);

/* psfm_solve_kernel followed by psfm_convolve in difference mode, with the solution kept
 * on the device between the two (one pass of the whole subtraction path).  `out` receives
 * the solution as in psfm_solve_kernel.  Synchronises `stream` once, at the end. */
psfm_status psfm_subtract(const float* img, const float* ref, const float* var_img,
                          const float* var_ref, const uint16_t* mask_img,
                          const uint16_t* mask_ref, psfm_shape shape,
                          const psfm_stamp* stamps, int32_t n_stamps,
                          const psfm_basis_spec* basis, const psfm_config* cfg,
                          const double* cov_ref, int32_t cov_ref_w, const double* cov_img,
                          int32_t cov_img_w, float* diff, float* diff_var,
                          uint16_t* diff_mask, double* cov_out, int32_t cov_out_w,
                          psfm_solution* out, void* workspace, size_t ws_bytes,
                          psfm_stream stream);

/* PSF-homogenised stack (Sec. 5.1-5.2).  For each of the n inputs (device image, variance,
 * mask, all with `shape`): render the fake target, a circular Gaussian of FWHM
 * target_fwhm at every source of src_xyf[i] (host, n_src[i] triples x, y, flux), solve for
 * the kernel matching the input to it (I1 = input, I2 = target, V2 = 0), convolve the
 * input, its variance and mask, and accumulate with weight w_i = 1 / mean(V'_i) over
 * pixels without badmask or CONV.BAD bits:
 *   out = sum w_i I'_i / sum w_i,  out_var = sum w_i^2 V'_i / (sum w_i)^2,
 *   out_count = number of contributing inputs, out_mask = nodata where none contributed,
 *   cov_out = pseudo-matrices averaged with weights w_i^2 mean(V'_i) (Sec. 4.4).
 * basis[i] is the basis of input i (host array of n specs).  sols (host, may be NULL)
 * receives the n solutions.  cov_out (device, may be NULL) has width
 * max_i psfm_cov_width(&basis[i], 1, 0) = cov_out_w.  Synchronises `stream`. */
psfm_status psfm_stack(int32_t n, const float* const* imgs, const float* const* vars,
                       const uint16_t* const* masks, psfm_shape shape,
                       const double* const* src_xyf, const int32_t* n_src, double target_fwhm,
                       const psfm_basis_spec* basis, const psfm_config* cfg, float* out,
                       float* out_var, uint16_t* out_mask, int32_t* out_count,
                       double* cov_out, int32_t cov_out_w, psfm_solution* sols,
                       void* workspace, size_t ws_bytes, psfm_stream stream);

/* Integer binning by b (Sec. 4.3: a convolution with a constant kernel followed by a change
 * of scale).  Output pixel (X, Y) covers the input block [bX, bX+b) x [bY, bY+b); partial
 * blocks at the far edges are dropped, so out_shape must be (width / b, height / b) with any
 * pitch >= its width.  out = sum of the block's pixels without `badmask` bits (flux kept),
 * out_mask = OR of the block's masks, out_var = f * sum of those pixels' variances with
 * f = (box * C * box)(0) / b^2 the covariance factor of the box (C = cov_in, the identity when
 * NULL; cov_in_w odd).  cov_out (device, may be NULL) receives the box pseudo-matrix
 * P(D) = sum_{|u| < b} (b - |u_x|)(b - |u_y|) C(D + u) sampled at lags that are multiples of b
 * and normalised to centre 1, width psfm_bin_cov_width(cov_in_w, b).  Planes are device
 * memory; workspace: PSFM_BIN_WORKSPACE bytes, 256-byte aligned.  Synchronises `stream` once
 * (to read the factor). */
#define PSFM_BIN_WORKSPACE 4096
int32_t psfm_bin_cov_width(int32_t cov_in_w, int32_t b);
psfm_status psfm_bin(const float* img, const float* var, const uint16_t* mask, psfm_shape shape,
                     int32_t b, uint16_t badmask, const double* cov_in, int32_t cov_in_w,
                     float* out, float* out_var, uint16_t* out_mask, psfm_shape out_shape,
                     double* cov_out, int32_t cov_out_w, void* workspace, size_t ws_bytes,
                     psfm_stream stream);

/* Pseudo-matrix of an image resampled by a non-integer scale (Sec. 4.4: the pseudo-matrix is
 * resampled by bilinear interpolation, and the total covariance excluding the variance is
 * kept).  scale s > 0 is the output pixel size in input pixels.  Output lag D (output pixels)
 * takes the bilinear interpolation of cov_in at the input lag s D (zero beyond cov_in's
 * extent); the entries off the centre are then multiplied by one factor so that their sum
 * equals cov_in's sum off the centre (left as interpolated when their sum is 0).  Readings: the
 * centre (the variance term) is cov_in's; the output radius is floor(r_in / s), the ratio
 * rounded to 1e-9.  cov_in: device [w_in][w_in] double, w_in odd, at most
 * PSFM_RESAMPLE_COV_MAX; cov_out: device [w][w], w = psfm_resample_cov_width(w_in, s).
 * Asynchronous on `stream`; errors: BAD_ARG (sizes, scale not positive and finite, NULL), CUDA. */
#define PSFM_RESAMPLE_COV_MAX 513
int32_t psfm_resample_cov_width(int32_t cov_in_w, double scale);
psfm_status psfm_resample_cov(const double* cov_in, int32_t cov_in_w, double scale,
                              double* cov_out, int32_t cov_out_w, psfm_stream stream);

/* PSF-homogenised stack with outlier rejection and the unconvolved companion stack (Sec. 5.1:
 * outliers are identified once the inputs share a PSF, carried back to the unconvolved inputs
 * by a matched filter, and the same rejection list serves a stack without convolution).
 * Inputs as for psfm_stack, at most PSFM_STACK_FULL_MAX of them.
 *   Pass 1: every input is matched to its target and convolved as in psfm_stack; the convolved
 *   image, variance and mask of all inputs are kept in the workspace.
 *   Outliers: at a pixel where at least 3 convolved inputs are usable (no badmask or CONV.BAD
 *   bit), input i is an outlier when |I'_i - m| > clip_nsigma * sqrt(V'_i + soften_alpha |m|),
 *   m the median of the usable convolved values there; n_rejected[i] (host, may be NULL)
 *   counts them; outliers (device [H][pitch] uint32, may be NULL) receives, per pixel, bit i
 *   set where input i is an outlier.
 *   Rejection: input pixels within the CONV.BAD radius r_bad of input i's kernel (Chebyshev
 *   distance) of one of its outliers get reject_bit (a bit outside badmask, conv_bad and
 *   conv_poor) and count as masked from then on.
 *   Pass 2: every input is convolved again with its pass-1 kernel and the rejected pixels
 *   masked, then accumulated as in psfm_stack into out, out_var, out_mask, out_count (and
 *   cov_out); the unconvolved inputs, without their badmask or rejected pixels, are
 *   accumulated with the same pass-1 weights into uout, uout_var, uout_mask, uout_count.
 * All output planes are device memory with `shape`.  Workspace:
 * psfm_stack_full_workspace_size(n, shape, basis, cfg, max n_src) bytes, 256-byte aligned
 * (it holds the n convolved inputs).  Synchronises `stream`. */
#define PSFM_STACK_FULL_MAX 32
size_t psfm_stack_full_workspace_size(int32_t n, psfm_shape shape, const psfm_basis_spec* basis,
                                      const psfm_config* cfg, int32_t n_src_max);
psfm_status psfm_stack_full(int32_t n, const float* const* imgs, const float* const* vars,
                            const uint16_t* const* masks, psfm_shape shape,
                            const double* const* src_xyf, const int32_t* n_src,
                            double target_fwhm, const psfm_basis_spec* basis,
                            const psfm_config* cfg, double clip_nsigma, uint16_t reject_bit,
                            float* out, float* out_var, uint16_t* out_mask, int32_t* out_count,
                            float* uout, float* uout_var, uint16_t* uout_mask,
                            int32_t* uout_count, int32_t* n_rejected, uint32_t* outliers,
                            double* cov_out, int32_t cov_out_w, psfm_solution* sols,
                            void* workspace, size_t ws_bytes, psfm_stream stream);

/* PSF model of one stack input for the envelope PSF: a flux-normalised mixture
 * (1 - moffat_frac) Gaussian + moffat_frac Moffat(beta), both components with the same FWHM
 * along the major and minor axes (pixels). */
typedef struct {
  double fwhm_major, fwhm_minor;
  double moffat_frac;  /* 0 .. 1 */
  double beta;         /* Moffat exponent, > 1 when moffat_frac > 0 */
} psfm_psf_model;

#define PSFM_ENVELOPE_MAX_RADIUS 64
#define PSFM_ENVELOPE_WORKSPACE 256

/* Envelope PSF of a stack's inputs (Sec. 5.1: each input's PSF realised as a circular profile
 * with a common peak flux, the maximum taken pixel by pixel, and a PSF model fitted to the
 * result).  Readings: the circular version of an input has FWHM sqrt(major * minor) and the
 * same profile mixture; the pixels are the offsets |u|, |v| <= R from the centre; the fitted
 * model is a circular Gaussian A exp(-r^2 / (2 s^2)), A and s by least squares, with s searched
 * between 0.2 of the narrowest and 4 times the widest input's Gaussian width.  Writes its FWHM
 * (2 sqrt(2 ln 2) s), the target_fwhm of psfm_stack and psfm_stack_full, to *fwhm (host).
 *   n: 1 .. PSFM_STACK_FULL_MAX models (host array);
 *   radius: R, 1 .. PSFM_ENVELOPE_MAX_RADIUS, or 0 for ceil(3 x the widest circular FWHM);
 *   workspace: PSFM_ENVELOPE_WORKSPACE bytes of 256-byte-aligned device memory.
 * Synchronises `stream`.  Errors: BAD_ARG (n, NULL pointers, a FWHM that is not positive and
 * finite, moffat_frac outside [0, 1], beta <= 1 with moffat_frac > 0, radius out of range or
 * an automatic radius above the maximum), WORKSPACE, CUDA. */
psfm_status psfm_envelope_fwhm(int32_t n, const psfm_psf_model* models, int32_t radius,
                               double* fwhm, void* workspace, size_t ws_bytes,
                               psfm_stream stream);

/* Batched subtraction (Sec. 3, Sec. 4 applied chip by chip; the batching itself has no
 * counterpart in the paper).  A batch is n chips, each with its own shape, basis (size, degrees,
 * spatial order) and buffers; the configuration is shared.  psfm_batch_create lays out one
 * caller workspace (psfm_batch_workspace_size bytes, 256-byte aligned) for all chips, uploads
 * their tables once and creates n_streams (1..32) pairs of CUDA streams on which chips run
 * concurrently: chip i is solved on the high-priority stream of pair i % n_streams and its
 * image, variance, mask and pseudo-matrix passes then run on that pair's low-priority stream.
 * The batch object is host memory owned by the library until psfm_batch_destroy.
 * psfm_batch_subtract enqueues every chip's psfm_subtract work (extractor, rejection loop,
 * image, variance, mask, pseudo-matrix of width 2w-1 when cov_outs[i] is set) without any host
 * synchronisation.  On a non-default stream the first call is captured into a CUDA graph and
 * later calls with the same buffer pointers replay it; on the legacy default stream the work
 * is enqueued directly.  Array arguments are host arrays of n device pointers; diff_vars,
 * diff_masks and cov_outs may be NULL.  Errors raised on the device are reported by
 * psfm_batch_solutions, which synchronises `stream` and fills n host solutions (sols may be
 * NULL) and returns the first chip's non-OK status.  Concurrent calls on one batch race. */
typedef struct psfm_batch psfm_batch;
size_t psfm_batch_workspace_size(int32_t n, const psfm_shape* shapes,
                                 const psfm_basis_spec* bases, const psfm_config* cfg);
psfm_status psfm_batch_create(int32_t n, const psfm_shape* shapes, const psfm_basis_spec* bases,
                              const psfm_config* cfg, int32_t n_streams, void* workspace,
                              size_t ws_bytes, psfm_batch** out);
psfm_status psfm_batch_subtract(psfm_batch* b, const float* const* imgs, const float* const* refs,
                                const float* const* var_imgs, const float* const* var_refs,
                                const uint16_t* const* mask_imgs,
                                const uint16_t* const* mask_refs, float* const* diffs,
                                float* const* diff_vars, uint16_t* const* diff_masks,
                                double* const* cov_outs, psfm_stream stream);
psfm_status psfm_batch_solutions(psfm_batch* b, psfm_solution* sols, psfm_stream stream);
/* Kernels one execution of the batch launches (counted when it was enqueued or captured). */
long long psfm_batch_kernel_count(const psfm_batch* b);
void psfm_batch_destroy(psfm_batch* b);

/* psfm_convolve without a workspace (no counterpart in the paper: this is an integration
 * aid).  For callers that cannot allocate device memory or hand over a workspace -- for
 * example a plugin loaded into a pipeline whose device memory pool is owned by the host
 * application, or a real-time scheduler that bans allocation after start-up.  Computes
 * the convolved (or difference) image, variance and mask exactly as psfm_convolve does with
 * cov_ref = cov_img = NULL and cov_out = NULL; it allocates nothing and calls no allocating
 * routine.  Its scratch is a fixed 6.1 MiB device array inside the library, present on every
 * GPU that loads the library until the process exits.
 *   Limits: width and height at most 4096 (PSFM_ERR_WORKSPACE otherwise).
 *   The first call on a device looks up the array's device address with that device
 *   current; make that first call before any stream capture.
 *   Each call uploads its coefficients and tables from host memory (cudaMemcpyAsync on
 *   `stream`).
 *   All calls share the array: calls that may overlap on the GPU (other streams, unordered
 *   host threads) race and give undefined results.  Calls on one stream are ordered.
 *   Asynchronous on `stream`; errors as for psfm_convolve. */
psfm_status psfm_convolve_noalloc(const float* ref, const float* var_ref,
                                  const uint16_t* mask_ref, const float* img,
                                  const float* var_img, const uint16_t* mask_img,
                                  psfm_shape shape, const psfm_basis_spec* basis,
                                  const psfm_config* cfg, const psfm_solution* sol, float* out,
                                  float* out_var, uint16_t* out_mask, psfm_stream stream);

/* Weighted Gram of column blocks: the normal-equation block C^T W C of one stamp (Eq. 5-6,
 * the Gram accumulation of Sec. 3.5), exposed on its own for the precision study.  For each
 * block b < n_blocks:
 *   gram[b][i][j] = sum_p weights[b][p] * cols[b][i][p] * cols[b][j][p].
 * cols: device [n_blocks][n_cols][n_pix] float; weights: device [n_blocks][n_pix] float;
 * gram: device [n_blocks][n_cols][n_cols] double, written symmetric.  precision:
 *   PSFM_PREC_FP64   FP64 products and sums (the reference; workspace unused, may be NULL);
 *   PSFM_PREC_TF32   tensor cores, TF32 products, FP32 accumulation, n_cols <= 128;
 *   PSFM_PREC_BF16X6 tensor cores, the Gram as (sqrt(w) C)^T (sqrt(w) C): seven BF16 slices
 *                    of each scaled column (scaled by a power of two), 28 slice products,
 *                    levels 0..4 summed exactly as integers over 224-pixel groups,
 *                    n_cols <= 64 (at least 48 bits, like double-float);
 *   PSFM_PREC_BF16X3 tensor cores, BF16 hi/lo split, three products, FP32 accumulation,
 *                    n_cols <= 128;
 * others return PSFM_ERR_UNSUPPORTED.  The tensor-core modes need PSFM_GRAM_WORKSPACE bytes of
 * 256-byte-aligned device workspace (a status word) and synchronise `stream` to report a
 * device-side PSFM_ERR_TIMEOUT; the FP64 mode is asynchronous. */
/* Poll limit of the tensor-core Gram's pipeline waits (no counterpart in the paper: a test
 * hook for the failure path).  Each wait for a shared-memory buffer's earlier MMAs gives up
 * after `polls` polls: the kernel then records PSFM_ERR_TIMEOUT, waits for the MMAs it has
 * issued (always with the default limit) and frees its tensor memory, so the context stays
 * usable and psfm_gram / the TF32 and BF16X3 solves return PSFM_ERR_TIMEOUT.  Applies to the
 * current device from the next launch; PSFM_WAIT_LIMIT_DEFAULT restores normal operation.
 * Errors: CUDA. */
#define PSFM_WAIT_LIMIT_DEFAULT (1u << 24)
psfm_status psfm_set_pipeline_wait_limit(uint32_t polls);

#define PSFM_GRAM_WORKSPACE 256
psfm_status psfm_gram(int32_t n_blocks, int32_t n_cols, int32_t n_pix, const float* cols,
                      const float* weights, int32_t precision, double* gram, void* workspace,
                      size_t ws_bytes, psfm_stream stream);

/* Instrumentation (no counterpart in the paper).  psfm_profile_enable(1) clears the stage
 * table and starts recording a CUDA event pair around every stage the library enqueues
 * (on the caller's stream); psfm_profile_enable(0) stops.  psfm_profile_entry(i, ...) reports
 * stage i: its name (NUL-terminated, truncated to name_cap), total device milliseconds
 * (synchronising on its events), kernels launched and times run; returns -1 if i is out of
 * range.  psfm_launch_count() is the number of kernels the library has launched so far in
 * this process, counted whether or not profiling is on. */
void psfm_profile_enable(int32_t on);
int32_t psfm_profile_count(void);
int32_t psfm_profile_entry(int32_t i, char* name, int32_t name_cap, double* ms,
                           long long* launches, long long* calls);
long long psfm_launch_count(void);

/* Autotuner of the image convolution's launch shape (no counterpart in the paper).  The
 * library keeps a table, per basis class (half width, spatial order, Gaussian count and degrees),
 * of the tile height the image convolution is launched with in psfm_convolve, psfm_subtract,
 * the batches and the stacks: 64 output rows (two CTAs of 8 warps per SM) or 128 (one CTA of
 * 16 warps); classes not in the table use 64.  Entries apply to launches enqueued (or
 * captured) after they are set.
 * psfm_tune_conv times both heights for `basis` on a synthetic width x height image (three
 * launches each, median, CUDA events on `stream`, which it synchronises; give the size of the
 * images the shape will serve: whether a tile's inputs come from L2 or from HBM changes which
 * shape is fastest), stores the faster in the table and, if `out` is not NULL, returns it
 * (ms = its median time).  Its workspace (psfm_tune_conv_workspace_size bytes, 256-byte
 * aligned device memory) holds the image, the output and the tables.  psfm_tune_get /
 * psfm_tune_set / psfm_tune_count / psfm_tune_clear read and write the table (for example to
 * persist it between processes).  The table is shared by every thread of the process.
 * Errors: BAD_ARG, WORKSPACE, UNSUPPORTED, CUDA. */
typedef struct {
  int32_t half_width, spatial_order, n_gauss;
  int32_t degree[PSFM_MAX_GAUSS];
  int32_t tile_rows;    /* 64 or 128 */
  int32_t plane_chunk;  /* horizontal planes per shared-memory chunk: 4 (0 reads as 4) */
  float ms;             /* measured median time of the tuning image, or 0 */
} psfm_tune_entry;
size_t psfm_tune_conv_workspace_size(int32_t width, int32_t height, const psfm_basis_spec* basis);
psfm_status psfm_tune_conv(int32_t width, int32_t height, const psfm_basis_spec* basis,
                           void* workspace, size_t ws_bytes, psfm_stream stream,
                           psfm_tune_entry* out);
int32_t psfm_tune_count(void);
psfm_status psfm_tune_get(int32_t i, psfm_tune_entry* out);
psfm_status psfm_tune_set(const psfm_tune_entry* e);
void psfm_tune_clear(void);

/* FP32 FMA throughput probe (no counterpart in the paper: it measures the FP32 peak that the
 * image and variance kernels are compared with).  Launches n_blocks blocks of 256 threads, each
 * thread running 8 independent FMA chains for iters x 8 steps, and writes one float per thread
 * to out (device, n_blocks * 256 floats).  *flops (host, may be NULL) receives the launch's
 * floating-point operations (2 per FMA); time the launch with CUDA events on `stream`.
 * Errors: BAD_ARG, CUDA. */
psfm_status psfm_fma_probe(int32_t n_blocks, int32_t iters, float* out, double* flops,
                           psfm_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* PSFM_H */
