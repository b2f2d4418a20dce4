// Integer binning of an image with its variance, mask and covariance pseudo-matrix (Sec. 4.3:
// binning is a convolution with a constant kernel followed by a change of scale).
//
// Output pixel (X, Y) covers the input block [bX, bX + b) x [bY, bY + b): the sum of the
// block's unmasked pixels (flux kept), the OR of its masks, and the covariance factor of the
// box times the sum of its unmasked variances, f = (box * C * box)(0) / b^2 (as the per-patch
// factor of a convolution, Sec. 4.4).  The box pseudo-matrix is
//   P(D) = sum_u (b - |u_x|)(b - |u_y|) C(D + u),   |u_x|, |u_y| < b,
// (the autocorrelation of the box is the triangle), sampled at lags that are multiples of b
// and normalised to centre 1.  Partial blocks at the far edges are dropped.
#include <cmath>

#include "psfm_internal.h"

namespace psfm {
namespace {

__global__ void k_bin_planes(const float* img, const float* var, const uint16_t* mask, int64_t pitch,
                             int b, uint16_t badmask, int Wb, int Hb, float f, float* out,
                             float* out_var, uint16_t* out_mask, int64_t out_pitch) {
  const int X = blockIdx.x * blockDim.x + threadIdx.x, Y = blockIdx.y;
  if (X >= Wb) return;
  float s = 0.f, v = 0.f;
  uint16_t m = 0;
  for (int dy = 0; dy < b; ++dy) {
    const int64_t row = (int64_t)(Y * b + dy) * pitch + (int64_t)X * b;
    for (int dx = 0; dx < b; ++dx) {
      const uint16_t mm = mask[row + dx];
      m |= mm;
      if (!(mm & badmask)) {
        s += img[row + dx];
        v += var[row + dx];
      }
    }
  }
  const int64_t o = (int64_t)Y * out_pitch + X;
  out[o] = s;
  out_var[o] = f * v;
  out_mask[o] = m;
}

// One thread per output lag (and one for the central factor): FP64 sums over the triangle.
__global__ void k_bin_pm(const double* cin, int c, int b, int r, double* pm_out, double* factor) {
  const int w = 2 * r + 1;
  const int hc = (c - 1) / 2;
  auto box = [&](int Dy, int Dx) {
    double s = 0.0;
    for (int uy = -(b - 1); uy <= b - 1; ++uy)
      for (int ux = -(b - 1); ux <= b - 1; ++ux) {
        const int y = Dy + uy + hc, x = Dx + ux + hc;
        if (y < 0 || y >= c || x < 0 || x >= c) continue;
        s += (double)((b - abs(ux)) * (b - abs(uy))) * cin[y * c + x];
      }
    return s;
  };
  __shared__ double centre;
  if (threadIdx.x == 0) {
    centre = box(0, 0);
    *factor = centre / ((double)b * b);
  }
  __syncthreads();
  for (int q = threadIdx.x; q < w * w; q += blockDim.x) {
    const int Y = q / w - r, X = q % w - r;
    pm_out[q] = box(b * Y, b * X) / centre;
  }
}

}  // namespace
}  // namespace psfm

extern "C" {

int32_t psfm_bin_cov_width(int32_t cov_in_w, int32_t b) {
  if (cov_in_w < 1 || cov_in_w % 2 == 0 || b < 1) return -1;
  const int n = 2 * b + cov_in_w - 2;  // box pseudo-matrix width (odd)
  const int c = (n - 1) / 2;
  return 2 * (c / b) + 1;
}

psfm_status psfm_bin(const float* img, const float* var, const uint16_t* mask, psfm_shape shape,
                     int32_t b, uint16_t badmask, const double* cov_in, int32_t cov_in_w,
                     float* out, float* out_var, uint16_t* out_mask, psfm_shape out_shape,
                     double* cov_out, int32_t cov_out_w, void* workspace, size_t ws_bytes,
                     psfm_stream stream) {
  if (!img || !var || !mask || !out || !out_var || !out_mask || b < 1) return PSFM_ERR_BAD_ARG;
  if (shape.width < 1 || shape.height < 1 || shape.pitch < shape.width) return PSFM_ERR_BAD_ARG;
  const int Wb = shape.width / b, Hb = shape.height / b;
  if (out_shape.width != Wb || out_shape.height != Hb || out_shape.pitch < Wb || Wb < 1 || Hb < 1)
    return PSFM_ERR_BAD_ARG;
  const int c = cov_in ? cov_in_w : 1;
  const int wout = psfm_bin_cov_width(c, b);
  if (wout < 0 || (cov_out && cov_out_w != wout)) return PSFM_ERR_BAD_ARG;
  if (!workspace || ws_bytes < PSFM_BIN_WORKSPACE ||
      (reinterpret_cast<uintptr_t>(workspace) & 255) != 0)
    return PSFM_ERR_WORKSPACE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // scratch: the unit pseudo-matrix when none is given, the factor and a throwaway output
  double* one = static_cast<double*>(workspace);
  double* dfactor = one + 1;
  double* scratch = one + 2;  // [wout^2] when cov_out is NULL (wout is 1 then)
  const double* cin = cov_in;
  if (!cov_in) {
    const double v = 1.0;
    if (cudaMemcpyAsync(one, &v, sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess)
      return PSFM_ERR_CUDA;
    cin = one;
  }
  if (!cov_out && (size_t)(2 + wout * wout) * sizeof(double) > ws_bytes) return PSFM_ERR_WORKSPACE;
  psfm::k_bin_pm<<<1, 256, 0, s>>>(cin, c, b, (wout - 1) / 2, cov_out ? cov_out : scratch,
                                   dfactor);
  double f = 0.0;
  if (cudaMemcpyAsync(&f, dfactor, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return PSFM_ERR_CUDA;
  psfm::k_bin_planes<<<dim3((Wb + 127) / 128, Hb), 128, 0, s>>>(
      img, var, mask, shape.pitch, b, badmask, Wb, Hb, (float)f, out, out_var, out_mask,
      out_shape.pitch);
  return cudaGetLastError() == cudaSuccess ? PSFM_OK : PSFM_ERR_CUDA;
}

}  // extern "C"

// ---- Resampling of a pseudo-matrix by a non-integer scale (Sec. 4.4) ----
//
// Output lag D (in output pixels) samples the input pseudo-matrix at the input lag s D by
// bilinear interpolation (zero beyond the input's extent); the entries off the centre are then
// scaled so that their sum equals the input's sum off the centre (the total covariance
// excluding the variance is preserved; the centre, the variance term, is the interpolated
// centre, i.e. the input's).  One CTA; sums in FP64 in a fixed order.
namespace psfm {
namespace {

constexpr int kResThreads = 256;

__global__ void __launch_bounds__(kResThreads) k_resample_cov(const double* cin, int win,
                                                              double scale, double* cout,
                                                              int wout) {
  __shared__ double red[2][kResThreads / 32];
  const int tid = threadIdx.x, rin = (win - 1) / 2, rout = (wout - 1) / 2;
  double s_in = 0.0, s_out = 0.0;
  for (int i = tid; i < win * win; i += kResThreads)
    if (i != rin * win + rin) s_in += cin[i];
  for (int i = tid; i < wout * wout; i += kResThreads) {
    const int dy = i / wout - rout, dx = i % wout - rout;
    const double px = scale * dx + rin, py = scale * dy + rin;
    const double fx0 = floor(px), fy0 = floor(py);
    const int x0 = (int)fx0, y0 = (int)fy0;
    const double fx = px - fx0, fy = py - fy0;
    auto at = [&](int x, int y) {
      return (x >= 0 && x < win && y >= 0 && y < win) ? cin[y * win + x] : 0.0;
    };
    const double v = (1.0 - fy) * ((1.0 - fx) * at(x0, y0) + fx * at(x0 + 1, y0)) +
                     fy * ((1.0 - fx) * at(x0, y0 + 1) + fx * at(x0 + 1, y0 + 1));
    cout[i] = v;
    if (dx != 0 || dy != 0) s_out += v;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s_in += __shfl_xor_sync(0xffffffffu, s_in, o);
    s_out += __shfl_xor_sync(0xffffffffu, s_out, o);
  }
  if ((tid & 31) == 0) {
    red[0][tid >> 5] = s_in;
    red[1][tid >> 5] = s_out;
  }
  __syncthreads();
  double a = 0.0, b = 0.0;
  for (int w = 0; w < kResThreads / 32; ++w) {
    a += red[0][w];
    b += red[1][w];
  }
  const double f = b != 0.0 ? a / b : 1.0;
  for (int i = tid; i < wout * wout; i += kResThreads)
    if (i != rout * wout + rout) cout[i] *= f;
}

}  // namespace
}  // namespace psfm

extern "C" {

int32_t psfm_resample_cov_width(int32_t cov_in_w, double scale) {
  if (cov_in_w < 1 || cov_in_w % 2 == 0 || cov_in_w > PSFM_RESAMPLE_COV_MAX) return -1;
  if (!(scale > 0.0) || !std::isfinite(scale)) return -1;
  const int rin = (cov_in_w - 1) / 2;
  const double r = std::floor(rin / scale + 1e-9);
  return 2 * (int32_t)r + 1;
}

psfm_status psfm_resample_cov(const double* cov_in, int32_t cov_in_w, double scale,
                              double* cov_out, int32_t cov_out_w, psfm_stream stream) {
  using namespace psfm;
  const int32_t w = psfm_resample_cov_width(cov_in_w, scale);
  if (w < 0 || !cov_in || !cov_out || cov_out_w != w) return PSFM_ERR_BAD_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  prof_begin("resample_cov", st);
  k_resample_cov<<<1, kResThreads, 0, st>>>(cov_in, cov_in_w, scale, cov_out, cov_out_w);
  prof_end("resample_cov", st, 1);
  return cudaGetLastError() == cudaSuccess ? PSFM_OK : PSFM_ERR_CUDA;
}

}  // extern "C"
