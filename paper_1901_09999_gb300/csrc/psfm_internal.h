// Internal declarations shared by the CUDA translation units of libpsfm.
//
// Notation follows Price & Magnier (arXiv:1901.09999), Sec. 2:
//   kernel half-width h (w = 2h+1), Gaussians g with width sigma_g and degree d_g,
//   basis terms k = (g, p, q), p + q <= d_g, N_b of them, spatial terms s = (l, m),
//   l + m <= S, N_s of them.  The 1-D factors f_{g,n}(t) = t^n exp(-t^2 / (2 sigma_g^2)),
//   t = -h..h, n = 0..d_g, make every basis term separable:
//   B'_k(u, v) = psi_k f_{g,p}(u) f_{g,q}(v).  A "plane" is one (g, n) pair; there are
//   N_H = sum_g (d_g + 1) planes.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/psfm.h"

namespace psfm {

constexpr int kMaxBasis = 4 * (PSFM_MAX_DEGREE + 1) * (PSFM_MAX_DEGREE + 2) / 2;  // 180
constexpr int kMaxSpatial = (PSFM_MAX_SPATIAL_ORDER + 1) * (PSFM_MAX_SPATIAL_ORDER + 2) / 2;
constexpr int kMaxPlanes = 4 * (PSFM_MAX_DEGREE + 1);
constexpr int kConvTX = 32;   // image-convolution tile width (one warp of columns)
constexpr int kConvTY = 64;   // image-convolution tile height
constexpr int kVarTile = 64;  // variance patch the fast variance kernel supports
constexpr int kBinCap = 512;  // detection candidates kept per subregion before ranking

// Device-side scalars kept in the workspace.
struct DevState {
  int32_t error;        // first psfm_status raised by a kernel (0 = OK)
  int32_t done;         // rejection loop finished
  int32_t iter;         // solves performed
  int32_t n_active;     // stamps in the current solve
  int32_t r_bad;        // CONV.BAD radius
  int32_t n_cand_total; // detections seen
  int32_t chol_fail;    // Cholesky met a non-positive pivot: LU fallback
  int32_t refined;      // the first refinement step's correction was small: skip the second
  double sum_var_conv;  // sum of V' over unmasked output pixels
  double sum_var_img;   // sum of V2 over unmasked output pixels
  double n_unmasked;    // count of unmasked output pixels
  double chi2_mean, chi2_rms, threshold;
  uint32_t median_key;  // order-preserving key of the detection-image median
  uint32_t sel_prefix;  // radix-select state
  int32_t sel_rank;
  int32_t sel_pad;
  // quality diagnostics of the solution (Sec. 3.7), kernel realised at the image centre
  int32_t q_flags;
  int32_t r_bad2;       // CONV.BAD radius of the dual kernel K2 applied to I2
  double q_ksum, q_mx, q_my, q_mxx, q_myy, q_mxy, q_deconv;
};

// Host-side plan: everything derived from (shape, basis, config).
struct Plan {
  int W = 0, H = 0;
  int64_t pitch = 0;
  int h = 0, w = 0, wpad = 0;
  int ng = 0;
  int deg[PSFM_MAX_GAUSS] = {0, 0, 0, 0};
  double sigma[PSFM_MAX_GAUSS] = {0, 0, 0, 0};
  int plane_base[PSFM_MAX_GAUSS] = {0, 0, 0, 0};
  int kbase[PSFM_MAX_GAUSS] = {0, 0, 0, 0};
  int S = 0, Ns = 0, Nb = 0, NH = 0, dmax = 0;
  int Nd = 0;     // design columns per stamp: Nb, or 2 Nb with the dual kernel (I1 then I2)
  int ncoef = 0;  // Nd * Ns
  // terms
  int tg[kMaxBasis], tp[kMaxBasis], tq[kMaxBasis];
  int sl[kMaxSpatial], sm[kMaxSpatial];
  double psi[kMaxBasis], sk[kMaxBasis], pen[kMaxBasis];
  std::vector<double> f1d;  // [NH][w]
  // configuration
  psfm_config cfg;
  int s = 0, P = 0, sw = 0, foot = 0;   // stamp half, pixels, side, footprint side
  int nreg = 0, max_cand = 0, n_stamps = 0;
  int Nsys = 0;  // unknowns of the kernel-term system (Nb*Ns [+2 for joint])
  int Nc = 0;    // columns of a stamp's augmented design block (Nd + 3: basis, R, 1, I2)
};

// Tables uploaded to the device at the start of a call (one blob in the workspace).
struct DevTables {
  float* f1d;       // [NH][wpad] FP32 1-D factors, zero padded
  double* f1d64;    // [NH][w]
  double* psi;      // [Nb]
  double* sk;       // [Nb]
  int32_t* term;    // [Nb] g | p << 8 | q << 16
  int32_t* spat;    // [Ns] l | m << 8
  double* pen;      // [Nb] penalty p_k of the dual kernel (Sec. 2)
};

// Basis geometry passed by value to kernels.
struct BasisDev {
  int h, w, wpad, ng, S, Ns, Nb, NH, dmax;
  int deg[PSFM_MAX_GAUSS];
  int plane_base[PSFM_MAX_GAUSS];
  int kbase[PSFM_MAX_GAUSS];
};

struct ImgGeom {
  int W, H;
  int64_t pitch;
};

// Workspace carving (device pointers inside the caller's buffer).
struct Workspace {
  char* base = nullptr;
  size_t size = 0, used = 0;
  bool measuring = false;  // only count bytes
  template <class T>
  T* take(size_t n) {
    size_t bytes = (n * sizeof(T) + 255) & ~size_t(255);
    T* p = measuring ? nullptr : reinterpret_cast<T*>(base + used);
    used += bytes;
    return p;
  }
};

// Everything the apply path needs on the device.
struct ApplyBuffers {
  DevTables tab;
  DevState* st;
  double* dsol;        // [2 + Nb*Ns]: b0, d0, coeff
  uint32_t* bits;      // [H][nwords] badmask bits of mask_ref
  uint32_t* hb_bad;    // horizontally dilated by r_bad
  uint32_t* hb_poor;   // horizontally dilated by h
  uint16_t* mask_tmp;  // output mask when the caller does not want one but needs statistics
  double* kern;        // [n_cov][w*w] sample kernels
  double* kern_t;      // [n_cov][(w+c-1)^2] K (x) C_in
  double* kern_s2;     // [n_cov] sum K^2
  float2* kern_f;      // the sample kernels as FP32 pairs
  float2* kern_tf;     // K (x) C_in as FP32 pairs
  double* cov_acc;     // [n_cov][n_out^2] per-sample partial pseudo-matrices
  double* cov_tmp;     // [(2w-1)^2] pseudo-matrix of the dual kernel's first part
  double* var_part;    // [variance patches][3] per-patch statistics for the combination weights
};

BasisDev basis_dev(const Plan& p);

#ifdef __CUDACC__
// Stage the rows x ld tile whose top-left image pixel is (gx0, gy0) into shared memory: the
// image value where the pixel is inside the image, in the first `cols` columns and not
// flagged in `badmask`, else 0.  Each thread keeps G elements' global loads in flight
// together, so the tile arrives in a few memory latencies instead of one per element.
template <int G>
__device__ __forceinline__ void stage_masked_tile(const float* img, const uint16_t* mask,
                                                  uint16_t badmask, int W, int H,
                                                  int64_t pitch, int gx0, int gy0, int rows,
                                                  int cols, int ld, float* dst, int tid,
                                                  int nthreads) {
  const int n = rows * ld;
  for (int i0 = tid; i0 < n; i0 += G * nthreads) {
    float v[G];
    uint16_t m[G];
    bool ok[G];
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int i = i0 + g * nthreads;
      const int r = i / ld, c = i - r * ld;
      const int gx = gx0 + c, gy = gy0 + r;
      ok[g] = i < n && c < cols && gx >= 0 && gx < W && gy >= 0 && gy < H;
      v[g] = 0.f;
      m[g] = 0;
      if (ok[g]) {
        const int64_t o = (int64_t)gy * pitch + gx;
        v[g] = img[o];
        m[g] = mask[o];
      }
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int i = i0 + g * nthreads;
      if (i < n) dst[i] = (ok[g] && !(m[g] & badmask)) ? v[g] : 0.f;
    }
  }
}
#endif

// Stage timing (CUDA events on the launching stream when profiling is on) and launch count.
void prof_begin(const char* name, cudaStream_t s);
void prof_end(const char* name, cudaStream_t s, int n_launches);
psfm_status make_plan(Plan& p, psfm_shape shape, const psfm_basis_spec* b, const psfm_config* c,
                      int n_stamps);
void pack_tables(const Plan& p, std::vector<char>& blob, size_t offs[7]);

// ---- launchers (return cudaError_t of the launch) ----
cudaError_t launch_conv_image(const Plan& p, const DevTables& t, const double* dsol,
                              const float* ref, const uint16_t* mref, const float* img,
                              float* out, cudaStream_t st);
cudaError_t launch_variance(const Plan& p, const DevTables& t, const double* dsol,
                            const float* var_ref, const uint16_t* mref, const float* var_img,
                            const double* cov_in, int cov_in_w, const uint16_t* omask,
                            float* out_var, DevState* ds, double* stats_part, cudaStream_t st);
// dual_pass 0: the single kernel; 1: the dual kernel's first pass (proximity flags of the
// reference's bad pixels only); 2: its second pass (the science image's bad pixels dilated by
// r_bad2, combined with the first pass's flags into the output mask)
cudaError_t launch_mask(const Plan& p, const ApplyBuffers& b, const uint16_t* mref,
                        const uint16_t* mimg, uint16_t* out, cudaStream_t st,
                        int dual_pass = 0);
cudaError_t launch_cov(const Plan& p, const ApplyBuffers& b, const double* cov_in,
                       int cov_in_w, const double* cov_img, int cov_img_w, double* cov_out,
                       int cov_out_w, cudaStream_t st);
cudaError_t launch_rbad(const Plan& p, const DevTables& t, const double* dsol, DevState* ds,
                        cudaStream_t st, bool second = false);

}  // namespace psfm
