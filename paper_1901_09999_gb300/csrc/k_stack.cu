// PSF-homogenised stacking (Sec. 5.1-5.2): fake target rendering and the weighted coadd.
//
// The target of each input is a circular Gaussian of the stack FWHM at every source
// position, sampled at pixel centres within ceil(5 sigma) of the nearest pixel (the paper
// builds it from the envelope PSF and the known source positions), summed over the sources
// in their given order in FP64 and rounded to FP32 once per pixel.  Each convolved input
// contributes where its mask carries neither badmask nor CONV.BAD bits, with weight
// w_i = 1 / mean(V'_i) (the paper weights by the mean variance of the convolved image; the
// inverse is the reading used):
//   I = sum w_i I'_i / sum w_i,   V = sum w_i^2 V'_i / (sum w_i)^2.
// Pseudo-matrices are averaged with weights w_i^2 mean(V'_i) = w_i (Sec. 4.4).
#include "psfm_internal.h"
#include "solve.h"

namespace psfm {
namespace {

// One CTA per 32 x 32 tile of the target.  The CTA lists, in source order, the sources whose
// box (radius `radius` around the nearest pixel) meets the tile, then every pixel adds the
// Gaussians of the listed sources that cover it in that order, in FP64, and is rounded to FP32
// once: the target does not depend on scheduling and equals the FP64 sum over sources in
// their given order.  The list is processed in batches of kRenderBatch sources.
constexpr int kRenderTile = 32;
constexpr int kRenderThreads = 256;
constexpr int kRenderBatch = 512;
constexpr int kRenderPix = kRenderTile * kRenderTile / kRenderThreads;  // pixels per thread

__global__ void __launch_bounds__(kRenderThreads) k_render_target(
    const double* src, int n_src, double sigma, int radius, int W, int H, int64_t pitch,
    float* target) {
  __shared__ double s_x[kRenderBatch], s_y[kRenderBatch], s_n[kRenderBatch];
  __shared__ int s_xi[kRenderBatch], s_yi[kRenderBatch];
  __shared__ int s_warp[kRenderThreads / 32];
  __shared__ int s_count;
  const int tx0 = blockIdx.x * kRenderTile, ty0 = blockIdx.y * kRenderTile;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double inv2s2 = 2.0 * sigma * sigma;
  const double area = 2.0 * 3.14159265358979323846 * sigma * sigma;
  double acc[kRenderPix];
#pragma unroll
  for (int k = 0; k < kRenderPix; ++k) acc[k] = 0.0;
  if (threadIdx.x == 0) s_count = 0;
  __syncthreads();
  for (int base = 0; base < n_src; base += kRenderThreads) {
    // list the sources of this chunk whose box meets the tile, keeping their order
    const int i = base + threadIdx.x;
    bool hit = false;
    double x0 = 0.0, y0 = 0.0, f = 0.0;
    int xi = 0, yi = 0;
    if (i < n_src) {
      x0 = src[3 * i];
      y0 = src[3 * i + 1];
      f = src[3 * i + 2];
      xi = (int)rint(x0);
      yi = (int)rint(y0);
      hit = xi + radius >= tx0 && xi - radius < tx0 + kRenderTile && yi + radius >= ty0 &&
            yi - radius < ty0 + kRenderTile;
    }
    const unsigned m = __ballot_sync(0xffffffffu, hit);
    if (lane == 0) s_warp[warp] = __popc(m);
    __syncthreads();
    int off = s_count, tot = 0;
    for (int w = 0; w < kRenderThreads / 32; ++w) {
      if (w < warp) off += s_warp[w];
      tot += s_warp[w];
    }
    // flush the list first when this chunk would overflow it
    if (s_count + tot > kRenderBatch) {
      const int nl = s_count;
#pragma unroll
      for (int k = 0; k < kRenderPix; ++k) {
        const int j = threadIdx.x + k * kRenderThreads;
        const int x = tx0 + (j % kRenderTile), y = ty0 + (j / kRenderTile);
        for (int l = 0; l < nl; ++l) {
          if (abs(x - s_xi[l]) > radius || abs(y - s_yi[l]) > radius) continue;
          const double dx = x - s_x[l], dy = y - s_y[l];
          acc[k] += s_n[l] * exp(-(dx * dx + dy * dy) / inv2s2) / area;
        }
      }
      off -= nl;
      __syncthreads();
    }
    if (hit) {
      const int o = off + __popc(m & ((1u << lane) - 1u));
      s_x[o] = x0;
      s_y[o] = y0;
      s_n[o] = f;
      s_xi[o] = xi;
      s_yi[o] = yi;
    }
    __syncthreads();
    if (threadIdx.x == 0) s_count = (s_count + tot > kRenderBatch ? 0 : s_count) + tot;
    __syncthreads();
  }
  const int nl = s_count;
#pragma unroll
  for (int k = 0; k < kRenderPix; ++k) {
    const int j = threadIdx.x + k * kRenderThreads;
    const int x = tx0 + (j % kRenderTile), y = ty0 + (j / kRenderTile);
    for (int l = 0; l < nl; ++l) {
      if (abs(x - s_xi[l]) > radius || abs(y - s_yi[l]) > radius) continue;
      const double dx = x - s_x[l], dy = y - s_y[l];
      acc[k] += s_n[l] * exp(-(dx * dx + dy * dy) / inv2s2) / area;
    }
    if (x < W && y < H) target[(int64_t)y * pitch + x] = (float)acc[k];
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
  const dim3 grid((p.W + kRenderTile - 1) / kRenderTile, (p.H + kRenderTile - 1) / kRenderTile);
  k_render_target<<<grid, kRenderThreads, 0, s>>>(src, n_src, sigma, radius, p.W, p.H, p.pitch,
                                                   target);
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
