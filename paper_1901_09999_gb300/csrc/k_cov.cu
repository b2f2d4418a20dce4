// Covariance pseudo-matrix of the convolved image (Eq. 10-11 written for a convolution,
// Sec. 4.3-4.4).  For a kernel K and input pseudo-matrix C_in the output pseudo-matrix is
//   C(D) = sum_a sum_b K(a) K(b) C_in(D + a - b)   (size 2w + c - 2),
// evaluated as T = K (x) C_in followed by C(D) = sum_a K(a) T(D + a).  The image's single
// pseudo-matrix is the mean of C / sum K^2 over an n x n grid of kernels realised at
// ((i + 1/2) W / n, (j + 1/2) H / n), divided by its centre value (the covariance factor
// has already gone into the variance map, patch by patch).  For a difference image it is
// averaged with the science image's pseudo-matrix, weighted by the two mean variances
// (Sec. 4.4).  Kernels and T in FP64, written also as FP32 pairs; the double sum over a and D
// (25 kernels of 31 x 31: about 50 M products) runs in double-float on the FP32 pipes (FP64
// runs at 1/64 of their rate here), one partial pseudo-matrix per sample kernel, and the
// samples are added in a fixed order.
#include "psfm_internal.h"

namespace psfm {
namespace {

__device__ __forceinline__ int sp_idx(int l, int m, int S) {
  return l * (S + 1) - (l * (l - 1)) / 2 + m;
}

// double-float (FP32 pair) helpers: exact products by FMA, sums by TwoSum
__device__ __forceinline__ float2 split2(double v) {
  const float hi = (float)v;
  return make_float2(hi, (float)(v - (double)hi));
}

// acc += a * b
__device__ __forceinline__ void fma2(float2& acc, float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  const float s = __fadd_rn(acc.x, p);
  const float bb = __fsub_rn(s, acc.x);
  const float err = __fadd_rn(__fsub_rn(acc.x, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  acc.x = s;
  acc.y = __fadd_rn(acc.y, __fadd_rn(err, e));
}

// One CTA per sample kernel: realise K_i (FP64), sum K_i^2, and T_i = K_i (x) C_in.
__global__ void k_cov_kernels(BasisDev b, ImgGeom g, int n, const double* f1d64,
                              const double* psi, const double* sk, const double* dsol,
                              const double* cov_in, int c, double* kern, double* kern_t,
                              double* kern_s2, float2* kern_f, float2* kern_tf) {
  extern __shared__ double sh[];
  const int W = b.w, h = b.h;
  double* ak = sh;                 // [Nb]
  double* colgp = ak + b.Nb;       // [NH][W]
  double* Kk = colgp + b.NH * W;   // [W*W]
  __shared__ double s_dc, s_red[32];
  const int tid = threadIdx.x, i = blockIdx.x;
  const double x = ((i % n) + 0.5) * g.W / n, y = ((i / n) + 0.5) * g.H / n;
  const double xt = g.W > 1 ? 2.0 * x / (g.W - 1) - 1.0 : 0.0;
  const double yt = g.H > 1 ? 2.0 * y / (g.H - 1) - 1.0 : 0.0;
  for (int k = tid; k < b.Nb; k += blockDim.x) {
    double a = 0.0, xp = 1.0;
    for (int l = 0; l <= b.S; ++l) {
      double yp = 1.0;
      for (int m = 0; m <= b.S - l; ++m) {
        a += dsol[2 + k * b.Ns + sp_idx(l, m, b.S)] * xp * yp;
        yp *= yt;
      }
      xp *= xt;
    }
    ak[k] = a;
  }
  __syncthreads();
  if (tid == 0) {
    double dc = dsol[0];
    for (int k = 0; k < b.Nb; ++k) dc -= ak[k] * sk[k];
    s_dc = dc;
  }
  for (int j = tid; j < b.NH * W; j += blockDim.x) {
    const int pl = j / W, v = j - pl * W;
    int gg = 0;
    while (gg + 1 < b.ng && pl >= b.plane_base[gg + 1]) ++gg;
    const int p = pl - b.plane_base[gg], dg = b.deg[gg];
    const int kgp = b.kbase[gg] + p * (dg + 1) - (p * (p - 1)) / 2;
    double cc = 0.0;
    for (int q = 0; q <= dg - p; ++q)
      cc += ak[kgp + q] * psi[kgp + q] * f1d64[(b.plane_base[gg] + q) * W + v];
    colgp[j] = cc;
  }
  __syncthreads();
  double s2 = 0.0;
  for (int j = tid; j < W * W; j += blockDim.x) {
    const int v = j / W, u = j - v * W;
    double kv = 0.0;
    for (int pl = 0; pl < b.NH; ++pl) kv += f1d64[pl * W + u] * colgp[pl * W + v];
    if (u == h && v == h) kv += s_dc;
    Kk[j] = kv;
    kern[(size_t)i * W * W + j] = kv;
    kern_f[(size_t)i * W * W + j] = split2(kv);
    s2 += kv * kv;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  if ((tid & 31) == 0) s_red[tid >> 5] = s2;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int j = 0; j < (int)(blockDim.x >> 5); ++j) t += s_red[j];
    kern_s2[i] = t;
  }
  // T = K (x) C_in, size (W + c - 1)^2; with white input (c = 1) T = K
  const int wt = W + c - 1;
  for (int j = tid; j < wt * wt; j += blockDim.x) {
    const int ty = j / wt, tx = j - ty * wt;
    double t = 0.0;
    if (cov_in) {
      for (int cy = 0; cy < c; ++cy) {
        const int ky = ty - cy;
        if (ky < 0 || ky >= W) continue;
        for (int cx = 0; cx < c; ++cx) {
          const int kx = tx - cx;
          if (kx < 0 || kx >= W) continue;
          t += Kk[ky * W + kx] * cov_in[cy * c + cx];
        }
      }
    } else {
      t = Kk[j];
    }
    kern_t[(size_t)i * wt * wt + j] = t;
    kern_tf[(size_t)i * wt * wt + j] = split2(t);
  }
}

// grid (n_samples, n_out): one CTA per output row of one sample; thread per output column.
// part[i](D) = sum_a K_i(a) T_i(D + a) / (sum K_i^2 * n_samples), in double-float.
__global__ void k_cov_rows(int W, int c, int nsamp, const float2* kern_f, const float2* kern_tf,
                           const double* kern_s2, double* part) {
  const int i = blockIdx.x, oy = blockIdx.y;
  const int wt = W + c - 1, nout = 2 * W + c - 2;
  const int ox = threadIdx.x;
  if (ox >= nout) return;
  // out index o <-> D = o - (nout-1)/2; T index t <-> e = t - (wt-1)/2; K index k <-> a = k - h
  // e = D + a  =>  t = o + k - (W - 1)
  const float2* K = kern_f + (size_t)i * W * W;
  const float2* T = kern_tf + (size_t)i * wt * wt;
  float2 s0 = make_float2(0.f, 0.f), s1 = s0, s2 = s0, s3 = s0;
  const int kx0 = max(0, (W - 1) - ox), kx1 = min(W, wt + (W - 1) - ox);
  for (int ky = 0; ky < W; ++ky) {
    const int ty = oy + ky - (W - 1);
    if (ty < 0 || ty >= wt) continue;
    const float2* Kr = K + ky * W + kx0;
    const float2* Tr = T + ty * wt + (ox + kx0 - (W - 1));  // tx = ox + kx - (W - 1) >= 0
    const int m = kx1 - kx0;
    int k = 0;
    for (; k + 3 < m; k += 4) {
      fma2(s0, Kr[k], Tr[k]);
      fma2(s1, Kr[k + 1], Tr[k + 1]);
      fma2(s2, Kr[k + 2], Tr[k + 2]);
      fma2(s3, Kr[k + 3], Tr[k + 3]);
    }
    for (; k < m; ++k) fma2(s0, Kr[k], Tr[k]);
  }
  const double v = (((double)s0.x + (double)s0.y) + ((double)s1.x + (double)s1.y)) +
                   (((double)s2.x + (double)s2.y) + ((double)s3.x + (double)s3.y));
  part[((size_t)i * nout + oy) * nout + ox] = v / (kern_s2[i] * nsamp);
}

// The samples' partial pseudo-matrices added in sample order, normalised to the centre, and
// combined with the science image's.
__global__ void k_cov_final(int nconv, int nsamp, const double* part, const double* cov_img,
                            int cimg, const DevState* st, double* out, int nout) {
  auto acc_at = [&](int q) {
    double v = 0.0;
    for (int i = 0; i < nsamp; ++i) v += part[(size_t)i * nconv * nconv + q];
    return v;
  };
  const double centre = acc_at((nconv / 2) * nconv + nconv / 2);
  double w1 = 1.0, w2 = 0.0;
  if (cimg > 0 && st->n_unmasked > 0.0) {
    w1 = st->sum_var_conv / st->n_unmasked;
    w2 = st->sum_var_img / st->n_unmasked;
  }
  if (w1 + w2 <= 0.0) {
    w1 = 1.0;
    w2 = 0.0;
  }
  const int oc = (nout - nconv) / 2, oi = (nout - cimg) / 2;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;  // one output entry per thread
  if (j < nout * nout) {
    const int y = j / nout, x = j - y * nout;
    double v = 0.0;
    if (y >= oc && y < oc + nconv && x >= oc && x < oc + nconv)
      v += w1 * acc_at((y - oc) * nconv + (x - oc)) / centre;
    if (cimg > 0 && y >= oi && y < oi + cimg && x >= oi && x < oi + cimg) {
      const double ci = cov_img ? cov_img[(y - oi) * cimg + (x - oi)] : 1.0;
      v += w2 * ci;
    }
    out[j] = v / (w1 + w2);
  }
}

}  // namespace

cudaError_t launch_cov(const Plan& p, const ApplyBuffers& b, const double* cov_in, int cov_in_w,
                       const double* cov_img, int cov_img_w, double* cov_out, int cov_out_w,
                       cudaStream_t st) {
  const int n = p.cfg.cov_grid, ns = n * n;
  const int c = cov_in ? cov_in_w : 1;
  const int nconv = 2 * p.w + c - 2;
  const size_t smem = sizeof(double) * ((size_t)p.Nb + (size_t)p.NH * p.w + (size_t)p.w * p.w);
  cudaError_t e = cudaFuncSetAttribute(k_cov_kernels, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_cov_kernels<<<ns, 256, smem, st>>>(basis_dev(p), ImgGeom{p.W, p.H, p.pitch}, n, b.tab.f1d64,
                                       b.tab.psi, b.tab.sk, b.dsol, cov_in, c, b.kern, b.kern_t,
                                       b.kern_s2, b.kern_f, b.kern_tf);
  k_cov_rows<<<dim3(ns, nconv), ((nconv + 31) / 32) * 32, 0, st>>>(p.w, c, ns, b.kern_f,
                                                                  b.kern_tf, b.kern_s2,
                                                                  b.cov_acc);
  // cov_img_w: 0 when not subtracting; a white science image is width 1 with no data
  k_cov_final<<<(cov_out_w * cov_out_w + 127) / 128 + 1, 128, 0, st>>>(
      nconv, ns, b.cov_acc, cov_img, cov_img_w, b.st, cov_out, cov_out_w);
  return cudaGetLastError();
}

}  // namespace psfm
