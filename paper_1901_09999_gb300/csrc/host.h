// Host-side helpers shared by the C ABI entry points (workspace head, apply path).
#pragma once

#include <vector>

#include "psfm_internal.h"

namespace psfm {

constexpr int kMaxCovIn = 129;

// Layout of the head of the workspace: [DevState][dsol][tables], uploaded in one copy.
struct Head {
  DevState* st = nullptr;
  double* dsol = nullptr;
  double* dsol2 = nullptr;  // dual kernel: (0, 0, c) the terms applied to I2
  double* dsol3 = nullptr;  // dual kernel: (1, 0, -c) = K2, for its variance and pseudo-matrix
  char* tables = nullptr;
  size_t bytes = 0;
  size_t offs[7];
  std::vector<char> blob;
};

size_t head_layout(const Plan& p, Head& h);
void head_bind(Head& h, char* base, const Plan& p);
DevTables bind_tables(char* t, const size_t offs[7]);
void carve_apply(const Plan& p, Workspace& ws, ApplyBuffers& b);
bool aligned256(const void* p);
cudaError_t upload_head(const Plan& p, Head& h, const double* sol_vals, int r_bad,
                        cudaStream_t st);
psfm_status check_cov(const Plan& p, const double* cov_ref, int cov_ref_w, bool diff,
                      const double* cov_img, int cov_img_w, const double* cov_out, int cov_out_w,
                      int* c_ref, int* c_img);
psfm_status run_apply(const Plan& p, const Head& h, const ApplyBuffers& b, const float* ref,
                      const float* var_ref, const uint16_t* mask_ref, const float* img,
                      const float* var_img, const uint16_t* mask_img, const double* cov_ref,
                      int c_ref, const double* cov_img, int c_img, float* out, float* out_var,
                      uint16_t* out_mask, double* cov_out, int cov_out_w, bool stats,
                      cudaStream_t st);

}  // namespace psfm
