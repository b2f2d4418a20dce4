// Variance propagation through the PSF-matching convolution (Eq. 13, Sec. 4.4):
//   V'(x, y) = f_t sum_{u,v} K_t(u, v)^2 V1(x-u, y-v)
// with K_t the kernel realised at the centre of the 64 x 64 patch t that contains (x, y)
// (the paper applies a constant kernel per patch and puts that patch's covariance factor
// f_t into its variance), V1 with masked pixels set to zero and zero off the image.
// In difference mode V2 is added (variances of a difference sum, Sec. 4.4).  When asked, the
// kernel also accumulates sum V', sum V2 and the count over pixels the output mask marks
// usable, which weight the pseudo-matrix combination (Sec. 4.4).
//
// One CTA per patch: it realises K_t from the separable basis in FP32 (N_H w^2 FMAs per
// patch), stages the variance tile with its halo, and each thread convolves a 16-row column
// strip, one kernel column at a time, with the strip in registers.
#include "dfloat.cuh"
#include "psfm_internal.h"

namespace psfm {
namespace {

struct VarParams {
  BasisDev b;
  ImgGeom g;
  const float* var_ref;
  const uint16_t* mref;
  const float* var_img;
  float* out;
  const uint16_t* omask;
  const float* f1d;
  const double* psi;
  const double* sk;
  const double* dsol;
  const double* cov_in;
  int cov_in_w;
  double xscale, yscale;
  DevState* st;
  double* part;  // [patches][3] per-patch statistics, added in a fixed order afterwards
  uint16_t badmask, okmask;
  int want_stats;
};

__device__ __forceinline__ int sp_index(int l, int m, int S) {
  return l * (S + 1) - (l * (l - 1)) / 2 + m;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_sum_f(float x) {
  df v = {x, 0.f};
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const df u = {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
    v = df_add(v, u);
  }
  return df_to_d(v);
}

template <int HW>
__global__ void __launch_bounds__(256) k_variance(VarParams P) {
  constexpr int T = kVarTile, W = 2 * HW + 1, VR = T + 2 * HW, VS = VR;
  extern __shared__ float4 smem4[];
  float* Vs = reinterpret_cast<float*>(smem4);          // VR * VS
  float* K2 = Vs + VR * VS;                             // [u][v], W * wpad
  float* Kf = K2 + W * P.b.wpad;                        // K(v, u) row-major [v][u], W * W
  float* colgp = Kf + W * W;                            // [plane][v], NH * wpad
  float* akp = colgp + P.b.NH * P.b.wpad;               // [Nb]
  __shared__ double red[8][4];
  __shared__ float s_f, s_dc;

  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * T, y0 = blockIdx.y * T;
  const int x1 = min(x0 + T, P.g.W), y1 = min(y0 + T, P.g.H);
  const double xt = (0.5 * (x0 + x1 - 1)) * P.xscale - 1.0;
  const double yt = (0.5 * (y0 + y1 - 1)) * P.yscale - 1.0;
  const int S = P.b.S, Ns = P.b.Ns;

  // a_k at the patch centre (FP64), times psi_k; the delta coefficient b0 - sum a_k s_k
  double dpart = 0.0;
  for (int k = tid; k < P.b.Nb; k += 256) {
    double a = 0.0;
    double xp = 1.0;
    for (int l = 0; l <= S; ++l) {
      double yp = 1.0;
      for (int m = 0; m <= S - l; ++m) {
        a += P.dsol[2 + k * Ns + sp_index(l, m, S)] * xp * yp;
        yp *= yt;
      }
      xp *= xt;
    }
    akp[k] = (float)(a * P.psi[k]);
    dpart += a * P.sk[k];
  }
  dpart = warp_sum(dpart);
  if ((tid & 31) == 0) red[tid >> 5][0] = dpart;
  __syncthreads();
  if (tid == 0) {
    double d = 0.0;
    for (int i = 0; i < 8; ++i) d += red[i][0];
    s_dc = (float)(P.dsol[0] - d);
  }
  // column factors per plane (g, p): sum_q a_{gpq} psi f_{g,q}(v)
  for (int i = tid; i < P.b.NH * W; i += 256) {
    const int pl = i / W, v = i - pl * W;
    int g = 0;
    while (g + 1 < P.b.ng && pl >= P.b.plane_base[g + 1]) ++g;
    const int p = pl - P.b.plane_base[g], dg = P.b.deg[g];
    const int kgp = P.b.kbase[g] + p * (dg + 1) - (p * (p - 1)) / 2;
    float c = 0.f;
    for (int q = 0; q <= dg - p; ++q)
      c = fmaf(akp[kgp + q], P.f1d[(P.b.plane_base[g] + q) * P.b.wpad + v], c);
    colgp[pl * P.b.wpad + v] = c;
  }
  __syncthreads();
  for (int i = tid; i < W * W; i += 256) {
    const int v = i / W, u = i - v * W;
    float kv = 0.f;
    for (int pl = 0; pl < P.b.NH; ++pl)
      kv = fmaf(P.f1d[pl * P.b.wpad + u], colgp[pl * P.b.wpad + v], kv);
    if (u == HW && v == HW) kv += s_dc;
    Kf[i] = kv;
    K2[u * P.b.wpad + v] = kv * kv;
  }
  for (int i = tid; i < W * (P.b.wpad - W); i += 256) {
    const int u = i / (P.b.wpad - W), v = W + i % (P.b.wpad - W);
    K2[u * P.b.wpad + v] = 0.f;
  }
  // masked variance tile with halo
  stage_masked_tile<8>(P.var_ref, P.mref, P.badmask, P.g.W, P.g.H, P.g.pitch, x0 - HW, y0 - HW,
                       VR, VS, VS, Vs, tid, 256);
  __syncthreads();
  // covariance factor of K_t (Sec. 4.3): sum_d C(d) sum_a K(a) K(a-d) / sum K^2
  if (P.cov_in) {
    const int c = P.cov_in_w, hc = (c - 1) / 2;
    double num = 0.0, den = 0.0;
    for (int i = tid; i < W * W; i += 256) {
      const int v = i / W, u = i - v * W;
      const double ka = Kf[i];
      den += ka * ka;
      for (int dy = -hc; dy <= hc; ++dy) {
        const int vv = v - dy;
        if (vv < 0 || vv >= W) continue;
        for (int dx = -hc; dx <= hc; ++dx) {
          const int uu = u - dx;
          if (uu < 0 || uu >= W) continue;
          num += P.cov_in[(dy + hc) * c + dx + hc] * ka * (double)Kf[vv * W + uu];
        }
      }
    }
    num = warp_sum(num);
    den = warp_sum(den);
    if ((tid & 31) == 0) {
      red[tid >> 5][1] = num;
      red[tid >> 5][2] = den;
    }
    __syncthreads();
    if (tid == 0) {
      double n = 0.0, d = 0.0;
      for (int i = 0; i < 8; ++i) {
        n += red[i][1];
        d += red[i][2];
      }
      s_f = d > 0.0 ? (float)(n / d) : 1.f;
    }
  } else if (tid == 0) {
    s_f = 1.f;
  }
  __syncthreads();

  const int col = tid & 63, rg = tid >> 6;
  float acc[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) acc[i] = 0.f;
  for (int u = 0; u < W; ++u) {
    float cv[16 + 2 * HW];
    const float* src = Vs + (rg * 16) * VS + col + 2 * HW - u;
#pragma unroll
    for (int t = 0; t < 16 + 2 * HW; ++t) cv[t] = src[t * VS];
    const float4* kw = reinterpret_cast<const float4*>(K2 + u * P.b.wpad);
#pragma unroll
    for (int t4 = 0; t4 < (W + 3) / 4; ++t4) {
      const float4 wv = kw[t4];
      const float wt[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int v = 4 * t4 + e;  // tap v - HW; V(y_i - (v - HW)) = cv[i - v + 2HW]
        if (v < W) {
#pragma unroll
          for (int i = 0; i < 16; ++i) acc[i] = fmaf(wt[e], cv[i - v + 2 * HW], acc[i]);
        }
      }
    }
  }
  const float f = s_f;
  // per-thread partials of 16 pixels in FP32 (the FP64 pipe is 1/64 of the FP32 rate), then
  // warp and block sums in FP64
  float t_conv = 0.f, t_img = 0.f;
  int t_n = 0;
  const int gx = x0 + col;
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const int gy = y0 + rg * 16 + i;
    if (gx < P.g.W && gy < P.g.H) {
      const int64_t off = (int64_t)gy * P.g.pitch + gx;
      const float vp = f * acc[i];
      float o = vp;
      float v2 = 0.f;
      if (P.var_img) {
        v2 = P.var_img[off];
        o += v2;
      }
      if (P.out) P.out[off] = o;
      if (P.want_stats && !(P.omask[off] & P.okmask)) {
        t_conv += vp;
        t_img += v2;
        ++t_n;
      }
    }
  }
  if (P.want_stats) {
    // warp sums of the FP32 partials in double-float on the FP32 pipes (exact for these
    // 32-term sums, as FP64 would be, without the FP64 pipe's 1/64 rate), then FP64
    const double s_conv = warp_sum_f(t_conv);
    const double s_img = warp_sum_f(t_img);
    const double s_n = (double)__reduce_add_sync(0xffffffffu, (unsigned)t_n);
    if ((tid & 31) == 0) {
      red[tid >> 5][0] = s_conv;
      red[tid >> 5][1] = s_img;
      red[tid >> 5][2] = s_n;
    }
    __syncthreads();
    if (tid == 0) {
      double a = 0.0, b = 0.0, c = 0.0;
      for (int i = 0; i < 8; ++i) {
        a += red[i][0];
        b += red[i][1];
        c += red[i][2];
      }
      double* pp = P.part + 3 * ((int64_t)(y0 / T) * gridDim.x + x0 / T);
      pp[0] = a;
      pp[1] = b;
      pp[2] = c;
    }
  }
}

// The per-patch statistics added in a fixed order (strided per thread, then a fixed tree); one
// CTA of 1024 threads with four loads in flight per thread keeps this short.
constexpr int kStatThreads = 1024;

__global__ void __launch_bounds__(kStatThreads) k_var_stats(const double* part, int n,
                                                             DevState* st) {
  __shared__ double red[kStatThreads / 32][3];
  double a = 0.0, b = 0.0, c = 0.0;
#pragma unroll 4
  for (int i = threadIdx.x; i < n; i += kStatThreads) {
    a += part[3 * i];
    b += part[3 * i + 1];
    c += part[3 * i + 2];
  }
  a = warp_sum(a);
  b = warp_sum(b);
  c = warp_sum(c);
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5][0] = a;
    red[threadIdx.x >> 5][1] = b;
    red[threadIdx.x >> 5][2] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int w = 0; w < kStatThreads / 32; ++w) {
      s0 += red[w][0];
      s1 += red[w][1];
      s2 += red[w][2];
    }
    st->sum_var_conv = s0;
    st->sum_var_img = s1;
    st->n_unmasked = s2;
  }
}

template <int HW>
cudaError_t launch_hw(const VarParams& P, cudaStream_t st) {
  constexpr int W = 2 * HW + 1, VR = kVarTile + 2 * HW;
  const size_t smem = sizeof(float) * ((size_t)VR * VR + (size_t)W * P.b.wpad + (size_t)W * W +
                                       (size_t)P.b.NH * P.b.wpad + (size_t)P.b.Nb);
  cudaError_t e =
      cudaFuncSetAttribute(k_variance<HW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((P.g.W + kVarTile - 1) / kVarTile, (P.g.H + kVarTile - 1) / kVarTile);
  k_variance<HW><<<grid, 256, smem, st>>>(P);
  if (P.want_stats)
    k_var_stats<<<1, kStatThreads, 0, st>>>(P.part, (int)(grid.x * grid.y), P.st);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_variance(const Plan& p, const DevTables& t, const double* dsol,
                            const float* var_ref, const uint16_t* mref, const float* var_img,
                            const double* cov_in, int cov_in_w, const uint16_t* omask,
                            float* out_var, DevState* ds, double* stats_part, cudaStream_t st) {
  VarParams P;
  P.b = basis_dev(p);
  P.g = ImgGeom{p.W, p.H, p.pitch};
  P.var_ref = var_ref;
  P.mref = mref;
  P.var_img = var_img;
  P.out = out_var;
  P.omask = omask;
  P.f1d = t.f1d;
  P.psi = t.psi;
  P.sk = t.sk;
  P.dsol = dsol;
  P.cov_in = cov_in;
  P.cov_in_w = cov_in_w;
  P.xscale = p.W > 1 ? 2.0 / (p.W - 1) : 0.0;
  P.yscale = p.H > 1 ? 2.0 / (p.H - 1) : 0.0;
  P.st = ds;
  P.badmask = p.cfg.badmask;
  P.okmask = (uint16_t)(p.cfg.badmask | p.cfg.conv_bad);
  P.want_stats = omask != nullptr;
  P.part = stats_part;
  if (P.want_stats && !stats_part) return cudaErrorInvalidValue;
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
