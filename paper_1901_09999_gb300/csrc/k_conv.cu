// Spatially varying PSF-matching convolution of the whole image (Eq. 12 with the kernel of
// Sec. 2): O(x, y) = b0 R + sum_k a_k(x, y) (B_k (x) R)(x, y) + d0, written as separable
// passes.  With B_k = psi_k f_{g,p}(u) f_{g,q}(v) - s_k delta:
//   H_{g,p}(x, y) = sum_u f_{g,p}(u) R(x-u, y)              (horizontal pass, one per plane)
//   V_k(x, y)     = sum_v f_{g,q}(v) H_{g,p}(x, y-v)        (vertical pass, one per term)
//   O(x, y)       = sum_k [a_k(x, y) psi_k] V_k + beta(x, y) R(x, y) + d0,
//   beta(x, y)    = b0 - sum_k a_k(x, y) s_k,
// where a_k(x, y) = sum_s a_{k,s} xt^l yt^m is evaluated per output pixel (Horner in xt, yt).
//
// One CTA computes a 32 (x) by 64 (y) output tile.  The masked reference with a halo of h
// pixels is staged in shared memory once; for each Gaussian the horizontal passes of a group of
// its degrees share each register window of the staged rows (the group is as many planes as
// keep two CTAs per SM: all degrees up to 6 at h = 15), and for each (g, p) plane every
// vertical tap read from shared memory feeds the 8 output rows a thread owns and all degrees q.
// Weights live in shared memory and are read as broadcast float4s.
#include "psfm_internal.h"

namespace psfm {
namespace {

struct ConvParams {
  BasisDev b;
  ImgGeom g;
  const float* ref;
  const uint16_t* mref;
  const float* img;
  float* out;
  const float* f1d;
  const double* psi;
  const double* sk;
  const double* dsol;
  float xscale, yscale;
  int pgroup;  // horizontal planes held in shared memory at a time
  uint16_t badmask;
};

template <int HW>
struct ConvShape {
  static constexpr int W = 2 * HW + 1;
  static constexpr int RS = kConvTX + ((2 * HW + 3) / 4) * 4;  // staged row stride (x4 floats)
  static constexpr int RR = kConvTY + 2 * HW;                   // staged rows
  static constexpr int NV4 = (4 + 2 * HW + 3) / 4;              // float4s per H window
};

__device__ __forceinline__ int spatial_index(int l, int m, int S) {
  // l = 0..S, m = 0..S-l  ->  sum_{l'<l} (S - l' + 1) + m
  return l * (S + 1) - (l * (l - 1)) / 2 + m;
}

// Adds c_k(x, y_i) acc[i] to out[i] for the 8 rows of a thread, with the term's coefficient
// polynomial c_k = sum_{l+m<=SS} a[m][l] xt^l yt^m evaluated by Horner (x first, then y).
template <int SS>
__device__ __forceinline__ void add_term(const float* a, float xt, const float yt[8],
                                         const float acc[8], float out[8]) {
  constexpr int S1 = SS + 1;
  float cm[SS + 1];
#pragma unroll
  for (int m = 0; m <= SS; ++m) {
    float t = 0.f;
#pragma unroll
    for (int l = SS - m; l >= 0; --l) t = fmaf(t, xt, a[m * S1 + l]);
    cm[m] = t;
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    float c = cm[SS];
#pragma unroll
    for (int m = SS - 1; m >= 0; --m) c = fmaf(c, yt[i], cm[m]);
    out[i] = fmaf(c, acc[i], out[i]);
  }
}

// The spatial order is uniform over the launch: one branch per term selects the unrolled
// polynomial of that order.
__device__ __forceinline__ void add_term_s(int S, const float* a, float xt, const float yt[8],
                                           const float acc[8], float out[8]) {
  switch (S) {
    case 0: add_term<0>(a, xt, yt, acc, out); break;
    case 1: add_term<1>(a, xt, yt, acc, out); break;
    case 2: add_term<2>(a, xt, yt, acc, out); break;
    default: add_term<3>(a, xt, yt, acc, out); break;
  }
}

template <int HW>
__global__ void __launch_bounds__(256, 2) k_conv_image(ConvParams P) {
  using CS = ConvShape<HW>;
  constexpr int TX = kConvTX, TY = kConvTY, W = CS::W, RS = CS::RS, RR = CS::RR;
  constexpr int NV4 = CS::NV4;
  extern __shared__ float4 smem4[];
  float* Rs = reinterpret_cast<float*>(smem4);
  float* Hs = Rs + RR * RS;
  const int S = P.b.S, S1 = S + 1;
  float* Ws = Hs + P.pgroup * RR * TX;
  float* alpha = Ws + P.b.NH * P.b.wpad;
  float* beta = alpha + P.b.Nb * S1 * S1;

  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;

  for (int i = tid; i < P.b.NH * P.b.wpad; i += 256) Ws[i] = P.f1d[i];
  for (int i = tid; i < P.b.Nb * S1 * S1; i += 256) {
    const int k = i / (S1 * S1), r = i - k * S1 * S1, m = r / S1, l = r - m * S1;
    float v = 0.f;
    if (l + m <= S) v = (float)(P.dsol[2 + k * P.b.Ns + spatial_index(l, m, S)] * P.psi[k]);
    alpha[i] = v;
  }
  if (tid < S1 * S1) {
    const int m = tid / S1, l = tid - m * S1;
    double v = 0.0;
    if (l + m <= S) {
      const int s = spatial_index(l, m, S);
      if (s == 0) v = P.dsol[0];
      for (int k = 0; k < P.b.Nb; ++k) v -= P.dsol[2 + k * P.b.Ns + s] * P.sk[k];
    }
    beta[tid] = (float)v;
  }
  // masked reference tile with halo; zero padding to the row stride
  stage_masked_tile<8>(P.ref, P.mref, P.badmask, P.g.W, P.g.H, P.g.pitch, x0 - HW, y0 - HW, RR,
                       TX + 2 * HW, RS, Rs, tid, 256);
  __syncthreads();

  const int lane = tid & 31, wi = tid >> 5;
  const int gx = x0 + lane;
  const float xt = (float)gx * P.xscale - 1.f;
  float yt[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) yt[i] = (float)(y0 + wi * 8 + i) * P.yscale - 1.f;
  float out[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) out[i] = 0.f;

  for (int g = 0; g < P.b.ng; ++g) {
    const int dg = P.b.deg[g];
    const int pb = P.b.plane_base[g];
    for (int p0 = 0; p0 <= dg; p0 += P.pgroup) {
    const int p1 = min(dg, p0 + P.pgroup - 1);
    // ---- horizontal passes of degrees p0..p1 of Gaussian g over the staged rows
    for (int item = tid; item < RR * 8; item += 256) {
      const int row = item >> 3, xg = item & 7;
      float rv[4 * NV4];
      const float4* src = reinterpret_cast<const float4*>(Rs + row * RS + xg * 4);
#pragma unroll
      for (int j = 0; j < NV4; ++j) {
        const float4 t = src[j];
        rv[4 * j] = t.x;
        rv[4 * j + 1] = t.y;
        rv[4 * j + 2] = t.z;
        rv[4 * j + 3] = t.w;
      }
      for (int n = p0; n <= p1; ++n) {
        const float4* wn = reinterpret_cast<const float4*>(Ws + (pb + n) * P.b.wpad);
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
        for (int t4 = 0; t4 < (W + 3) / 4; ++t4) {
          const float4 wv = wn[t4];
          const float wt[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int t = 4 * t4 + e;  // tap index, u = t - HW; R(x_j - u) = rv[j - t + 2HW]
            if (t < W) {
              a0 = fmaf(wt[e], rv[0 - t + 2 * HW], a0);
              a1 = fmaf(wt[e], rv[1 - t + 2 * HW], a1);
              a2 = fmaf(wt[e], rv[2 - t + 2 * HW], a2);
              a3 = fmaf(wt[e], rv[3 - t + 2 * HW], a3);
            }
          }
        }
        *reinterpret_cast<float4*>(Hs + ((n - p0) * RR + row) * TX + xg * 4) =
            make_float4(a0, a1, a2, a3);
      }
    }
    __syncthreads();
    // ---- vertical passes: each H value in registers serves 8 outputs and all q
    for (int p = p0; p <= p1; ++p) {
      float col[8 + 2 * HW];
      const float* hp = Hs + ((p - p0) * RR + wi * 8) * TX + lane;
#pragma unroll
      for (int t = 0; t < 8 + 2 * HW; ++t) col[t] = hp[t * TX];
      const int kgp = P.b.kbase[g] + p * (dg + 1) - (p * (p - 1)) / 2;
      for (int q = 0; q <= dg - p; ++q) {
        const float4* wq = reinterpret_cast<const float4*>(Ws + (pb + q) * P.b.wpad);
        float acc[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) acc[i] = 0.f;
#pragma unroll
        for (int t4 = 0; t4 < (W + 3) / 4; ++t4) {
          const float4 wv = wq[t4];
          const float wt[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int t = 4 * t4 + e;  // v = t - HW; H(y_i - v) = col[i - t + 2HW]
            if (t < W) {
#pragma unroll
              for (int i = 0; i < 8; ++i) acc[i] = fmaf(wt[e], col[i - t + 2 * HW], acc[i]);
            }
          }
        }
        add_term_s(S, alpha + (kgp + q) * S1 * S1, xt, yt, acc, out);
      }
    }
    __syncthreads();
    }
  }

  float rc[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) rc[i] = Rs[(wi * 8 + i + HW) * RS + lane + HW];
  add_term_s(S, beta, xt, yt, rc, out);
  const float d0 = (float)P.dsol[1];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int gy = y0 + wi * 8 + i;
    float o = out[i] + d0;
    if (gx < P.g.W && gy < P.g.H) {
      const int64_t off = (int64_t)gy * P.g.pitch + gx;
      if (P.img) o = P.img[off] - o;
      P.out[off] = o;
    }
  }
}

// Shared memory per CTA that leaves room for two resident CTAs per SM (228 KB per SM, 1 KB of
// it reserved per CTA).
constexpr size_t kConvSmemTwoCtas = 112 * 1024;

template <int HW>
cudaError_t launch_hw(ConvParams P, cudaStream_t st) {
  using CS = ConvShape<HW>;
  const int S1 = P.b.S + 1;
  const size_t fixed = sizeof(float) * ((size_t)CS::RR * CS::RS + (size_t)P.b.NH * P.b.wpad +
                                        (size_t)P.b.Nb * S1 * S1 + (size_t)S1 * S1);
  const size_t plane = sizeof(float) * (size_t)CS::RR * kConvTX;
  // as many horizontal planes per group as keep two CTAs per SM (at least one; a Gaussian's
  // degrees beyond that are processed in further groups)
  int pg = P.b.dmax + 1;
  if (fixed + pg * plane > kConvSmemTwoCtas)
    pg = fixed + plane < kConvSmemTwoCtas ? (int)((kConvSmemTwoCtas - fixed) / plane) : 1;
  P.pgroup = pg;
  const size_t smem = fixed + pg * plane;
  cudaError_t e = cudaFuncSetAttribute(k_conv_image<HW>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((P.g.W + kConvTX - 1) / kConvTX, (P.g.H + kConvTY - 1) / kConvTY);
  k_conv_image<HW><<<grid, 256, smem, st>>>(P);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_conv_image(const Plan& p, const DevTables& t, const double* dsol,
                              const float* ref, const uint16_t* mref, const float* img,
                              float* out, cudaStream_t st) {
  ConvParams P;
  P.b = basis_dev(p);
  P.g = ImgGeom{p.W, p.H, p.pitch};
  P.ref = ref;
  P.mref = mref;
  P.img = img;
  P.out = out;
  P.f1d = t.f1d;
  P.psi = t.psi;
  P.sk = t.sk;
  P.dsol = dsol;
  P.xscale = p.W > 1 ? (float)(2.0 / (p.W - 1)) : 0.f;
  P.yscale = p.H > 1 ? (float)(2.0 / (p.H - 1)) : 0.f;
  P.badmask = p.cfg.badmask;
  switch (p.h) {
#define PSFM_CASE(n) \
  case n:            \
    return launch_hw<n>(P, st);
    PSFM_CASE(1) PSFM_CASE(2) PSFM_CASE(3) PSFM_CASE(4) PSFM_CASE(5) PSFM_CASE(6)
    PSFM_CASE(7) PSFM_CASE(8) PSFM_CASE(9) PSFM_CASE(10) PSFM_CASE(11) PSFM_CASE(12)
    PSFM_CASE(13) PSFM_CASE(14) PSFM_CASE(15) PSFM_CASE(16) PSFM_CASE(17) PSFM_CASE(18)
    PSFM_CASE(19) PSFM_CASE(20) PSFM_CASE(21) PSFM_CASE(22) PSFM_CASE(23) PSFM_CASE(24)
#undef PSFM_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace psfm
