// Kernel solve (Sec. 2 Eq. 2-6 with c_i = p_i = 0; Sec. 3.2-3.6) and stacking (Sec. 5.1)
// orchestration, shared between the C ABI and the device kernels.
#pragma once

#include "psfm_internal.h"

namespace psfm {

// Blocks that share one stamp's Gram (pixel chunks split between them).
constexpr int kGramSplit = 4;
// Blocks that share one stamp's chi^2 (pixel ranges).
constexpr int kChi2Split = 2;

struct SolveBuffers {
  // extractor (Sec. 3.3)
  uint32_t* hist;     // [3][2048] radix-select histograms of the detection image
  uint32_t* badbits;  // [H][nwords] bad bits of mask_ref | mask_img
  uint32_t* keys;     // [H][W] order-preserving keys of the detection image, 0 where masked
  int32_t* over;      // [over_capacity] pixels above the detection threshold (linear index)
  int32_t* n_over;    // their count
  float* bin_val;     // [nreg][kBinCap] detections per subregion
  int32_t* bin_idx;   // [nreg][kBinCap] their linear index y * W + x
  int32_t* bin_cnt;   // [nreg]
  // candidates
  int32_t* cand;       // [nreg][max_cand][2] (x, y), -1 = empty
  int32_t* cand_stat;  // [nreg][max_cand] PSFM_CAND_*
  double* cand_chi2;   // [nreg][max_cand]
  int32_t* ptr;        // [nreg] rank of the active candidate
  int32_t* have;       // [nreg] rank whose design block is cached, -1 none
  // per-region stamp data
  void* C;       // [nreg][Nb][P] basis-convolved masked reference at the stamp pixels (float or double)
  double* Gt;    // [nreg][Nc][Nc] weighted Gram of (zero-sum basis columns psi_k C_k - s_k X,
                 // R, 1, I2)
  double* Gpart;        // [nreg][kGramSplit][Nc][Nc] partial Grams over pixel chunks
  int32_t* gram_count;  // [nreg] partial Grams finished for the stamp being built
  double* foot;  // [nreg][4] footprint sums F1, F2, n, unused
  double* chi2;  // [nreg] chi^2 of the active stamp
  double* chi2_part;    // [nreg][kChi2Split][2] per-block chi^2 sums
  int32_t* chi2_count;  // [nreg] chi^2 blocks finished
  // normal equations
  double* M;  // [Nsys][Nsys]
  double* v;  // [Nsys]
  double* L;  // [Nsys][Nsys] factor
  float2* rinv;  // [Nsys/32][32][32] inverses of the diagonal blocks (double-float)
  float* Lh;     // [Nsys][Nsys] double-float working copy of M (lower triangle), high parts
  float* Ll;     // low parts
  float* Fh;     // [Nsys][Nsys] double-float Cholesky factor L by rows (lower), high parts
  float* Fl;     // low parts
  double* x;     // [Nsys] solution being refined
  double* pdiag; // [Nsys] penalty on the diagonal (dual kernel; zeros otherwise)
  double* y;  // [Nsys]
  int32_t* piv;  // [Nsys] LU pivots
  double* gv;    // [nreg][Ns] spatial factors at the stamp centres, 0 when inactive
  double* gp;    // [nreg][(Ns+1)^2] their pairwise products (index Ns stands for 1)
  int32_t* fresh;    // [nreg] Gram computed in this iteration
  int32_t* removed;  // [nreg] stamp rejected in this iteration
};

void carve_solve(const Plan& p, Workspace& ws, SolveBuffers& b);

// Pixels above the detection threshold the extractor can list: every pixel, so the list never
// overflows (the guard in the kernel stays).
inline int64_t over_capacity(const Plan& p) { return (int64_t)p.W * p.H; }

// Tensor-core weighted Gram of caller column blocks (TF32 mode 0, BF16 hi/lo mode 1):
// G[b] = cols[b] diag(w[b]) cols[b]^T, cols [n_blocks][n_cols][n_pix], n_cols <= 128; a wait
// that runs out writes PSFM_ERR_TIMEOUT to *status.
cudaError_t launch_gram_tc_plain(int mode, const float* cols, const float* w, int n_blocks,
                                 int n_cols, int n_pix, double* G, int32_t* status,
                                 cudaStream_t s);

// Enqueue the whole solve (extractor or caller stamps, rejection loop, r_bad).
psfm_status run_solve(const Plan& p, const DevTables& t, DevState* st, double* dsol,
                      const SolveBuffers& b, const float* img, const float* ref,
                      const float* var_img, const float* var_ref, const uint16_t* mask_img,
                      const uint16_t* mask_ref, const psfm_stamp* stamps, cudaStream_t s);

// Synchronise and copy the solution to the host structure.
psfm_status fetch_solution(const Plan& p, const DevState* st, const double* dsol,
                           const SolveBuffers& b, psfm_solution* out, cudaStream_t s);

// Synchronise and return the device error word.
psfm_status sync_status(const DevState* st, cudaStream_t s);

struct StackBuffers {
  float* target;     // [H][pitch] fake target image (Sec. 5.1)
  float* zero_var;   // [H][pitch] zero variance of the target
  uint16_t* zero_m;  // [H][pitch] empty target mask
  float* conv;       // [H][pitch] convolved input
  float* conv_var;   // [H][pitch] its variance
  uint16_t* conv_m;  // [H][pitch] its mask
  float* acc_w;      // [H][pitch] sum of weights of the contributing inputs
  double* src;       // [n_src_max][3] sources of the current input
  double* pm;        // [kMaxCovOut^2] pseudo-matrix of the current input
  double* pm_acc;    // [kMaxCovOut^2] weighted sum of pseudo-matrices
  double* wsum;      // [2] sum of pseudo-matrix weights, scratch
};

constexpr int kMaxCovOut = 2 * (2 * PSFM_MAX_HALF_WIDTH + 1) - 1;

void carve_stack(const Plan& p, Workspace& ws, StackBuffers& b, int n_src_max);

cudaError_t launch_render_target(const Plan& p, const double* src, int n_src, double fwhm,
                                 float* target, cudaStream_t s);
cudaError_t launch_stack_accum(const Plan& p, const float* conv, const float* conv_var,
                               const uint16_t* conv_m, const DevState* st, float* num,
                               float* var, float* wsum, int32_t* count, cudaStream_t s);
cudaError_t launch_stack_cov_accum(const double* pm, int n_pm, int n_acc, const DevState* st,
                                   double* pm_acc, double* wsum, cudaStream_t s);
cudaError_t launch_stack_final(const Plan& p, float* out, float* out_var, uint16_t* out_mask,
                               const float* wsum, const int32_t* count, const double* pm_acc,
                               const double* pw, double* cov_out, int cov_out_w,
                               cudaStream_t s);

}  // namespace psfm
