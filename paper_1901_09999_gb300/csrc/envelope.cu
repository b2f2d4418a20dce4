// Envelope PSF of a stack's inputs (Sec. 5.1): each input's PSF model is realised as a circular
// profile with a common peak, the maximum is taken pixel by pixel, and a PSF model (a circular
// Gaussian, the profile the stack's target image is rendered with) is fitted to the result.
//
// The realised profiles depend on the pixel offset only through r^2 = u^2 + v^2, so the grid
// |u|, |v| <= R is held as the envelope value at every r^2 and the number of grid pixels with
// that r^2.  The least-squares fit of A exp(-r^2 / 2 s^2) eliminates A (A = sum E g / sum g^2),
// leaving h(s) = (sum E g)^2 / sum g^2 to maximise: a scan over 64 log-spaced s brackets the
// maximum, then bisection on the sign of dh/ds, which is the sign of
//   F(s) = (sum E g r^2)(sum g^2) - (sum E g)(sum g^2 r^2),
// locates it (a root of the derivative is located to rounding, a flat maximum of h is not).
// Profiles in FP32, sums in double-float (FP32 pairs), one CTA.
#include <cmath>

#include "psfm_internal.h"

namespace psfm {
namespace {

constexpr int kEnvThreads = 1024;
constexpr int kEnvScan = 64;
constexpr int kEnvBisect = 60;

struct EnvModels {
  float fwhm[PSFM_STACK_FULL_MAX];  // circular FWHM sqrt(major * minor)
  float frac[PSFM_STACK_FULL_MAX];  // Moffat fraction
  float beta[PSFM_STACK_FULL_MAX];
  int n;
};

struct dfe {
  float hi, lo;
};

__device__ __forceinline__ dfe dfe_add(dfe a, dfe b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  const float lo = __fadd_rn(__fadd_rn(a.lo, b.lo), err);
  const float h = __fadd_rn(s, lo);
  return dfe{h, __fsub_rn(lo, __fsub_rn(h, s))};
}

// a += x (x an FP32 value)
__device__ __forceinline__ void dfe_acc(dfe& a, float x) { a = dfe_add(a, dfe{x, 0.f}); }

// Peak-normalised circular profile: flux-normalised mixture (1 - a) Gaussian + a Moffat(beta)
// with a common FWHM, divided by its value at r = 0.
__device__ float profile(float r2, float fwhm, float a, float beta) {
  const float sig = fwhm / 2.35482004503f;
  const float g0 = 1.f / (6.28318530718f * sig * sig);
  const float g = g0 * expf(-0.5f * r2 / (sig * sig));
  float m = 0.f, m0 = 0.f;
  if (a > 0.f) {
    const float al2 = fwhm * fwhm / (4.f * (exp2f(1.f / beta) - 1.f));  // alpha^2
    m0 = (beta - 1.f) / (3.14159265359f * al2);
    m = m0 * powf(1.f + r2 / al2, -beta);
  }
  return ((1.f - a) * g + a * m) / ((1.f - a) * g0 + a * m0);
}

// Block sum of four double-float values; the result is valid in thread 0.
__device__ void block_sum4(dfe v[4], dfe (*sh)[4]) {
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const dfe u = {__shfl_xor_sync(0xffffffffu, v[k].hi, o),
                     __shfl_xor_sync(0xffffffffu, v[k].lo, o)};
      v[k] = dfe_add(v[k], u);
    }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0)
    for (int k = 0; k < 4; ++k) sh[w][k] = v[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k < 4; ++k) {
      dfe t = sh[0][k];
      for (int i = 1; i < kEnvThreads / 32; ++i) t = dfe_add(t, sh[i][k]);
      v[k] = t;
    }
  }
}

// S1 = sum c E g, S2 = sum c g^2, S3 = sum c E g r^2, S4 = sum c g^2 r^2 (thread 0).
__device__ void moments(const float* E, const float* cnt, int nr2, float sig, dfe v[4],
                        dfe (*sh)[4]) {
  for (int k = 0; k < 4; ++k) v[k] = dfe{0.f, 0.f};
  const float c2 = -0.5f / (sig * sig);
  for (int k = threadIdx.x; k < nr2; k += kEnvThreads) {
    const float c = cnt[k];
    if (c == 0.f) continue;
    const float r2 = (float)k;
    const float g = expf(c2 * r2);
    const float eg = c * E[k] * g, gg = c * g * g;
    dfe_acc(v[0], eg);
    dfe_acc(v[1], gg);
    dfe_acc(v[2], eg * r2);
    dfe_acc(v[3], gg * r2);
  }
  block_sum4(v, sh);
}

__global__ void __launch_bounds__(kEnvThreads) k_envelope(EnvModels M, int R, double* out) {
  extern __shared__ float env_sh[];
  const int nr2 = 2 * R * R + 1;
  float* E = env_sh;         // [nr2] envelope at r^2
  float* cnt = E + nr2;      // [nr2] grid pixels with that r^2
  __shared__ dfe sh[kEnvThreads / 32][4];
  __shared__ float s_sig[kEnvScan];
  __shared__ float s_h[kEnvScan];
  __shared__ float s_lo, s_hi;
  const int tid = threadIdx.x;
  for (int k = tid; k < nr2; k += kEnvThreads) cnt[k] = 0.f;
  __syncthreads();
  const int side = 2 * R + 1;
  for (int i = tid; i < side * side; i += kEnvThreads) {
    const int v = i / side - R, u = i % side - R;
    atomicAdd(&cnt[u * u + v * v], 1.f);
  }
  float fmin = 1e30f, fmax = 0.f;
  for (int i = 0; i < M.n; ++i) {
    fmin = fminf(fmin, M.fwhm[i]);
    fmax = fmaxf(fmax, M.fwhm[i]);
  }
  for (int k = tid; k < nr2; k += kEnvThreads) {
    float e = 0.f;
    for (int i = 0; i < M.n; ++i)
      e = fmaxf(e, profile((float)k, M.fwhm[i], M.frac[i], M.beta[i]));
    E[k] = e;
  }
  __syncthreads();
  // scan: s from 0.2 of the narrowest to 4 times the widest input's Gaussian width
  const float lo0 = 0.2f * fmin / 2.35482004503f, hi0 = 4.f * fmax / 2.35482004503f;
  dfe v[4];
  for (int j = 0; j < kEnvScan; ++j) {
    const float sig = lo0 * powf(hi0 / lo0, (float)j / (kEnvScan - 1));
    moments(E, cnt, nr2, sig, v, sh);
    if (tid == 0) {
      const double s1 = (double)v[0].hi + v[0].lo, s2 = (double)v[1].hi + v[1].lo;
      s_sig[j] = sig;
      s_h[j] = s2 > 0.0 ? (float)(s1 * s1 / s2) : 0.f;
    }
  }
  __syncthreads();
  if (tid == 0) {
    int jb = 0;
    for (int j = 1; j < kEnvScan; ++j)
      if (s_h[j] > s_h[jb]) jb = j;
    s_lo = s_sig[jb > 0 ? jb - 1 : 0];
    s_hi = s_sig[jb < kEnvScan - 1 ? jb + 1 : kEnvScan - 1];
  }
  __syncthreads();
  // bisection on the sign of F (positive where h still rises)
  for (int it = 0; it < kEnvBisect; ++it) {
    const float mid = 0.5f * (s_lo + s_hi);
    moments(E, cnt, nr2, mid, v, sh);
    if (tid == 0) {
      const double s1 = (double)v[0].hi + v[0].lo, s2 = (double)v[1].hi + v[1].lo;
      const double s3 = (double)v[2].hi + v[2].lo, s4 = (double)v[3].hi + v[3].lo;
      if (s3 * s2 - s1 * s4 > 0.0)
        s_lo = mid;
      else
        s_hi = mid;
    }
    __syncthreads();
  }
  if (tid == 0) *out = 2.3548200450309493 * 0.5 * ((double)s_lo + (double)s_hi);
}

}  // namespace
}  // namespace psfm

extern "C" psfm_status psfm_envelope_fwhm(int32_t n, const psfm_psf_model* models,
                                          int32_t radius, double* fwhm, void* workspace,
                                          size_t ws_bytes, psfm_stream stream) {
  using namespace psfm;
  if (n < 1 || n > PSFM_STACK_FULL_MAX || !models || !fwhm) return PSFM_ERR_BAD_ARG;
  if (!workspace || ws_bytes < PSFM_ENVELOPE_WORKSPACE) return PSFM_ERR_WORKSPACE;
  if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0) return PSFM_ERR_BAD_ARG;
  EnvModels M;
  M.n = n;
  double fmax = 0.0;
  for (int i = 0; i < n; ++i) {
    const psfm_psf_model& m = models[i];
    if (!(m.fwhm_major > 0.0) || !(m.fwhm_minor > 0.0) || !std::isfinite(m.fwhm_major) ||
        !std::isfinite(m.fwhm_minor))
      return PSFM_ERR_BAD_ARG;
    if (!(m.moffat_frac >= 0.0 && m.moffat_frac <= 1.0)) return PSFM_ERR_BAD_ARG;
    if (m.moffat_frac > 0.0 && !(m.beta > 1.0 && std::isfinite(m.beta))) return PSFM_ERR_BAD_ARG;
    const double f = std::sqrt(m.fwhm_major * m.fwhm_minor);
    M.fwhm[i] = (float)f;
    M.frac[i] = (float)m.moffat_frac;
    M.beta[i] = (float)(m.moffat_frac > 0.0 ? m.beta : 2.0);
    if (f > fmax) fmax = f;
  }
  int R = radius;
  if (R == 0) R = (int)std::ceil(3.0 * fmax);
  if (R < 1 || R > PSFM_ENVELOPE_MAX_RADIUS) return PSFM_ERR_BAD_ARG;
  const int nr2 = 2 * R * R + 1;
  const size_t smem = sizeof(float) * 2 * (size_t)nr2;
  if (cudaFuncSetAttribute(k_envelope, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess)
    return PSFM_ERR_CUDA;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  double* d_out = static_cast<double*>(workspace);
  prof_begin("envelope", st);
  k_envelope<<<1, kEnvThreads, smem, st>>>(M, R, d_out);
  prof_end("envelope", st, 1);
  if (cudaGetLastError() != cudaSuccess) return PSFM_ERR_CUDA;
  if (cudaMemcpyAsync(fwhm, d_out, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return PSFM_ERR_CUDA;
  return PSFM_OK;
}
