// PSF-homogenised stacking (Sec. 5.1-5.2): fake target rendering and the weighted coadd.
//
// The target of each input is a circular Gaussian of the stack FWHM at every source
// position, sampled at pixel centres within ceil(5 sigma) of the nearest pixel (the paper
// builds it from the envelope PSF and the known source positions).  Each convolved input
// contributes where its mask carries neither badmask nor CONV.BAD bits, with weight
// w_i = 1 / mean(V'_i) (the paper weights by the mean variance of the convolved image; the
// inverse is the reading used):
//   I = sum w_i I'_i / sum w_i,   V = sum w_i^2 V'_i / (sum w_i)^2.
// Pseudo-matrices are averaged with weights w_i^2 mean(V'_i) = w_i (Sec. 4.4).
#include "psfm_internal.h"
#include "solve.h"

namespace psfm {
namespace {

// One CTA per source: add its Gaussian to the target box.
__global__ void k_render_target(const double* src, int n_src, double sigma, int radius, int W,
                                int H, int64_t pitch, float* target) {
  const int i = blockIdx.x;
  if (i >= n_src) return;
  const double x0 = src[3 * i], y0 = src[3 * i + 1], f = src[3 * i + 2];
  const int xi = (int)rint(x0), yi = (int)rint(y0);
  const int n = 2 * radius + 1;
  const double norm = f / (2.0 * 3.14159265358979323846 * sigma * sigma);
  const double c = -1.0 / (2.0 * sigma * sigma);
  for (int j = threadIdx.x; j < n * n; j += blockDim.x) {
    const int x = xi - radius + j % n, y = yi - radius + j / n;
    if (x < 0 || x >= W || y < 0 || y >= H) continue;
    const double dx = x - x0, dy = y - y0;
    atomicAdd(&target[(int64_t)y * pitch + x], (float)(norm * exp(c * (dx * dx + dy * dy))));
  }
}

__global__ void k_stack_accum(int W, int H, int64_t pitch, uint16_t okmask, const float* conv,
                              const float* conv_var, const uint16_t* conv_m, const DevState* st,
                              float* num, float* var, float* wsum, int32_t* count) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= W) return;
  if (!(st->n_unmasked > 0.0) || !(st->sum_var_conv > 0.0)) return;
  const float w = (float)(st->n_unmasked / st->sum_var_conv);
  const int64_t o = (int64_t)y * pitch + x;
  if (conv_m[o] & okmask) return;
  num[o] += w * conv[o];
  var[o] += w * w * conv_var[o];
  wsum[o] += w;
  count[o] += 1;
}

__global__ void k_stack_cov_accum(const double* pm, int n_pm, int n_acc, const DevState* st,
                                  double* pm_acc, double* wsum) {
  if (!(st->n_unmasked > 0.0) || !(st->sum_var_conv > 0.0)) return;
  const double w = st->n_unmasked / st->sum_var_conv;
  const int o = (n_acc - n_pm) / 2;
  for (int j = threadIdx.x; j < n_pm * n_pm; j += blockDim.x) {
    const int y = j / n_pm, x = j - y * n_pm;
    pm_acc[(y + o) * n_acc + x + o] += w * pm[j];
  }
  if (threadIdx.x == 0) wsum[0] += w;
}

__global__ void k_stack_final(int W, int H, int64_t pitch, uint16_t nodata, float* out,
                              float* out_var, uint16_t* out_mask, const float* wsum,
                              const int32_t* count) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= W) return;
  const int64_t o = (int64_t)y * pitch + x;
  const float w = wsum[o];
  if (count[o] > 0 && w > 0.f) {
    out[o] = out[o] / w;
    out_var[o] = out_var[o] / (w * w);
    out_mask[o] = 0;
  } else {
    out[o] = 0.f;
    out_var[o] = 0.f;
    out_mask[o] = nodata;
  }
}

__global__ void k_stack_cov_final(const double* pm_acc, const double* wsum, int n,
                                  double* cov_out) {
  for (int j = threadIdx.x; j < n * n; j += blockDim.x)
    cov_out[j] = wsum[0] > 0.0 ? pm_acc[j] / wsum[0] : 0.0;
}

}  // namespace

void carve_stack(const Plan& p, Workspace& ws, StackBuffers& b, int n_src_max) {
  const size_t npx = (size_t)p.H * p.pitch;
  b.target = ws.take<float>(npx);
  b.zero_var = ws.take<float>(npx);
  b.zero_m = ws.take<uint16_t>(npx);
  b.conv = ws.take<float>(npx);
  b.conv_var = ws.take<float>(npx);
  b.conv_m = ws.take<uint16_t>(npx);
  b.acc_w = ws.take<float>(npx);
  b.src = ws.take<double>((size_t)(n_src_max > 0 ? n_src_max : 1) * 3);
  b.pm = ws.take<double>((size_t)kMaxCovOut * kMaxCovOut);
  b.pm_acc = ws.take<double>((size_t)kMaxCovOut * kMaxCovOut);
  b.wsum = ws.take<double>(2);
}

cudaError_t launch_render_target(const Plan& p, const double* src, int n_src, double fwhm,
                                 float* target, cudaStream_t s) {
  const double sigma = fwhm / (2.0 * sqrt(2.0 * log(2.0)));
  const int radius = (int)ceil(5.0 * sigma);
  if (n_src > 0)
    k_render_target<<<n_src, 256, 0, s>>>(src, n_src, sigma, radius, p.W, p.H, p.pitch, target);
  return cudaGetLastError();
}

cudaError_t launch_stack_accum(const Plan& p, const float* conv, const float* conv_var,
                               const uint16_t* conv_m, const DevState* st, float* num,
                               float* var, float* wsum, int32_t* count, cudaStream_t s) {
  k_stack_accum<<<dim3((p.W + 255) / 256, p.H), 256, 0, s>>>(
      p.W, p.H, p.pitch, (uint16_t)(p.cfg.badmask | p.cfg.conv_bad), conv, conv_var, conv_m, st,
      num, var, wsum, count);
  return cudaGetLastError();
}

cudaError_t launch_stack_cov_accum(const double* pm, int n_pm, int n_acc, const DevState* st,
                                   double* pm_acc, double* wsum, cudaStream_t s) {
  k_stack_cov_accum<<<1, 256, 0, s>>>(pm, n_pm, n_acc, st, pm_acc, wsum);
  return cudaGetLastError();
}

cudaError_t launch_stack_final(const Plan& p, float* out, float* out_var, uint16_t* out_mask,
                               const float* wsum, const int32_t* count, const double* pm_acc,
                               const double* pw, double* cov_out, int cov_out_w,
                               cudaStream_t s) {
  k_stack_final<<<dim3((p.W + 255) / 256, p.H), 256, 0, s>>>(p.W, p.H, p.pitch, p.cfg.nodata, out,
                                                             out_var, out_mask, wsum, count);
  if (cov_out) k_stack_cov_final<<<1, 256, 0, s>>>(pm_acc, pw, cov_out_w, cov_out);
  return cudaGetLastError();
}

}  // namespace psfm
