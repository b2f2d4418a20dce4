// Least-squares kernel solve on the device (Sec. 2 Eq. 3-6 with c_i = p_i = 0, Sec. 3.2-3.6).
//
// Per stamp (one CTA each; only stamps that became active since the last iteration):
//   design:  C[k][p] = (B'_k (x) R)(x_p, y_p) / psi_k at the (2s+1)^2 stamp pixels, by
//            separable passes over the staged footprint (FP32), i.e. the columns
//            g_i k_i (x) I1 of Eq. 4 before the spatial factor, psi and the delta term;
//   Gram:    G = A^T W A for A = (C columns, R, 1, I2), W = 1 / (V1 + V2) (Eq. 5-6),
//            FP32 products over 32-pixel chunks summed in FP64; cached across iterations
//            (Sec. 3.5: per-stamp matrices need not be recalculated).
// Per iteration (single small kernels):
//   norm:    b0, d0 from unweighted footprint sums (Sec. 3.2, SEPARATE), FP64;
//   assemble M = sum_stamps (g g^T) (x) G_basis and v (Eq. 5-6 with g_i at the stamp centre);
//   solve:   FP64 Cholesky, LU with partial pivoting as fallback (PSFM_ERR_SINGULAR if both
//            fail);
//   chi2:    per-stamp mean of residual^2 / (V1 + V2 + alpha |I2|) in FP64 (Sec. 3.6);
//   reject:  chi2 > mean + n sigma (population std) -> reject and replace from the same
//            subregion (Sec. 3.3); finish when nothing is rejected or after max_iter solves.
// The design block stores C without psi and without the delta: the Gram is accumulated on
// the raw separable convolutions and psi / s_k are applied when the system is assembled.
#include <cstring>
#include <vector>

#include "psfm_internal.h"
#include "solve.h"

namespace psfm {
namespace {

__device__ __forceinline__ void raise_error(DevState* st, int code) { atomicCAS(&st->error, 0, code); }

__device__ __forceinline__ bool region_active(const int32_t* ptr, const int32_t* cand, int r,
                                              int max_cand, int* cx, int* cy) {
  const int j = ptr[r];
  if (j >= max_cand) return false;
  const int64_t c = (int64_t)r * max_cand + j;
  *cx = cand[2 * c];
  *cy = cand[2 * c + 1];
  return *cx >= 0;
}

struct StampParams {
  BasisDev b;
  ImgGeom g;
  const float* i1;
  const float* i2;
  const float* v1;
  const float* v2;
  const uint16_t* m1;
  const uint16_t* m2;
  uint16_t badmask;
  int s, sw, P, foot, max_cand, Nc;
  const float* f1d;     // [NH][wpad]
  const double* f1d64;  // [NH][w]
  const double* psi;
  const double* sk;
  const int32_t* cand;
  const int32_t* ptr;
  int32_t* have;
  void* C;  // [nreg][Nb][P] of T (float or double, by precision mode)
  double* G;
  double* Gt;
  double* footsum;
  DevState* st;
};

template <typename T>
__device__ __forceinline__ T tap(const StampParams& P, int plane, int t) {
  if (sizeof(T) == 8) return (T)P.f1d64[plane * P.b.w + t];
  return (T)P.f1d[plane * P.b.wpad + t];
}

// grid (nreg, ng): basis-convolved footprint of one Gaussian's terms, in T arithmetic.
template <typename T>
__global__ void __launch_bounds__(256) k_stamp_design(StampParams P) {
  extern __shared__ __align__(16) unsigned char sh_raw[];
  T* sh = reinterpret_cast<T*>(sh_raw);
  const int r = blockIdx.x, g = blockIdx.y, tid = threadIdx.x;
  if (P.st->error || P.st->done) return;
  int cx, cy;
  if (!region_active(P.ptr, P.cand, r, P.max_cand, &cx, &cy)) return;
  if (P.have[r] == P.ptr[r]) return;
  const int h = P.b.h, W = P.b.w, foot = P.foot, sw = P.sw;
  T* F = sh;                  // foot x foot
  T* Hp = F + foot * foot;    // foot x sw
  const int x0 = cx - P.s - h, y0 = cy - P.s - h;
  double f1 = 0.0, f2 = 0.0, nf = 0.0;
  for (int i = tid; i < foot * foot; i += 256) {
    const int rr = i / foot, cc = i - rr * foot;
    const int gx = x0 + cc, gy = y0 + rr;
    T v = 0;
    if (gx >= 0 && gx < P.g.W && gy >= 0 && gy < P.g.H) {
      const int64_t o = (int64_t)gy * P.g.pitch + gx;
      const uint16_t a = P.m1[o] & P.badmask, b = P.m2[o] & P.badmask;
      if (!a) v = (T)P.i1[o];
      if (g == 0 && !a && !b) {
        f1 += v;
        f2 += P.i2[o];
        nf += 1.0;
      }
    }
    F[i] = v;
  }
  if (g == 0) {
    __shared__ double red[3][8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      f1 += __shfl_xor_sync(0xffffffffu, f1, o);
      f2 += __shfl_xor_sync(0xffffffffu, f2, o);
      nf += __shfl_xor_sync(0xffffffffu, nf, o);
    }
    if ((tid & 31) == 0) {
      red[0][tid >> 5] = f1;
      red[1][tid >> 5] = f2;
      red[2][tid >> 5] = nf;
    }
    __syncthreads();
    if (tid == 0) {
      double a = 0, b = 0, c = 0;
      for (int i = 0; i < 8; ++i) {
        a += red[0][i];
        b += red[1][i];
        c += red[2][i];
      }
      P.footsum[4 * r] = a;
      P.footsum[4 * r + 1] = b;
      P.footsum[4 * r + 2] = c;
    }
  }
  __syncthreads();
  const int dg = P.b.deg[g], pb = P.b.plane_base[g];
  for (int p = 0; p <= dg; ++p) {
    for (int i = tid; i < foot * sw; i += 256) {
      const int rr = i / sw, px = i - rr * sw;
      const T* src = F + rr * foot + px + 2 * h;
      T a = 0;
      for (int t = 0; t < W; ++t) a = fma(tap<T>(P, pb + p, t), src[-t], a);
      Hp[i] = a;
    }
    __syncthreads();
    const int kgp = P.b.kbase[g] + p * (dg + 1) - (p * (p - 1)) / 2;
    for (int q = 0; q <= dg - p; ++q) {
      T* out = reinterpret_cast<T*>(P.C) + ((int64_t)r * P.b.Nb + kgp + q) * P.P;
      for (int i = tid; i < P.P; i += 256) {
        const int py = i / sw, px = i - py * sw;
        const T* src = Hp + (py + 2 * h) * sw + px;
        T a = 0;
        for (int t = 0; t < W; ++t) a = fma(tap<T>(P, pb + q, t), src[-t * sw], a);
        out[i] = a;
      }
    }
    __syncthreads();
  }
}

// ---- Double-float ("FP32 pair") arithmetic: a value is hi + lo with |lo| <= ulp(hi) / 2.
// Products use the exact FMA residual, sums the error-free TwoSum, so each operation keeps
// about 48 significant bits while running on the FP32 pipes (FP64 on this GPU runs at 1/64
// of the FP32 rate).  Intrinsics keep the compiler from re-associating the compensations.
struct df {
  float hi, lo;
};

__device__ __forceinline__ df df_split(double v) {
  df r;
  r.hi = (float)v;
  r.lo = (float)(v - (double)r.hi);
  return r;
}

// acc += p + e where p is an FP32 value and e a small correction
__device__ __forceinline__ void df_acc(df& acc, float p, float e) {
  const float s = __fadd_rn(acc.hi, p);
  const float bb = __fsub_rn(s, acc.hi);
  const float err = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  acc.hi = s;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(err, e));
}

// acc += a * b for an FP32 a (exact) and a double-float b
__device__ __forceinline__ void df_fma_f(df& acc, float a, df b) {
  const float p = __fmul_rn(b.hi, a);
  float e = __fmaf_rn(b.hi, a, -p);
  e = __fmaf_rn(b.lo, a, e);
  df_acc(acc, p, e);
}

// acc += a * b for double-floats a and b (the lo * lo term is below the precision kept)
__device__ __forceinline__ void df_fma(df& acc, df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  df_acc(acc, p, e);
}

__device__ __forceinline__ df df_mul(df a, df b) {
  df r;
  r.hi = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -r.hi);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const float s = __fadd_rn(r.hi, e);
  r.lo = __fsub_rn(e, __fsub_rn(s, r.hi));
  r.hi = s;
  return r;
}

__device__ __forceinline__ df df_norm(df a) {
  df r;
  r.hi = __fadd_rn(a.hi, a.lo);
  r.lo = __fsub_rn(a.lo, __fsub_rn(r.hi, a.hi));
  return r;
}

__device__ __forceinline__ double df_to_d(df a) { return (double)a.hi + (double)a.lo; }

// grid (nreg, ng): basis-convolved footprint of one Gaussian's terms in double-float.  The
// reference pixels are exact FP32; the 1-D factors are split into FP32 pairs.
__global__ void __launch_bounds__(256) k_stamp_design_df(StampParams P) {
  extern __shared__ __align__(16) unsigned char sh_raw[];
  const int r = blockIdx.x, g = blockIdx.y, tid = threadIdx.x;
  if (P.st->error || P.st->done) return;
  int cx, cy;
  if (!region_active(P.ptr, P.cand, r, P.max_cand, &cx, &cy)) return;
  if (P.have[r] == P.ptr[r]) return;
  const int h = P.b.h, W = P.b.w, foot = P.foot, sw = P.sw;
  const int dg = P.b.deg[g], pb = P.b.plane_base[g];
  float* F = reinterpret_cast<float*>(sh_raw);   // foot x foot
  float* Hh = F + foot * foot;                    // foot x sw
  float* Hl = Hh + foot * sw;
  float* wh = Hl + foot * sw;                     // (dg+1) x W
  float* wl = wh + (dg + 1) * W;
  for (int i = tid; i < (dg + 1) * W; i += 256) {
    const int n = i / W, t = i - n * W;
    const df v = df_split(P.f1d64[(pb + n) * W + t]);
    wh[i] = v.hi;
    wl[i] = v.lo;
  }
  const int x0 = cx - P.s - h, y0 = cy - P.s - h;
  double f1 = 0.0, f2 = 0.0, nf = 0.0;
  for (int i = tid; i < foot * foot; i += 256) {
    const int rr = i / foot, cc = i - rr * foot;
    const int gx = x0 + cc, gy = y0 + rr;
    float v = 0.f;
    if (gx >= 0 && gx < P.g.W && gy >= 0 && gy < P.g.H) {
      const int64_t o = (int64_t)gy * P.g.pitch + gx;
      const uint16_t a = P.m1[o] & P.badmask, b = P.m2[o] & P.badmask;
      if (!a) v = P.i1[o];
      if (g == 0 && !a && !b) {
        f1 += v;
        f2 += P.i2[o];
        nf += 1.0;
      }
    }
    F[i] = v;
  }
  if (g == 0) {
    __shared__ double red[3][8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      f1 += __shfl_xor_sync(0xffffffffu, f1, o);
      f2 += __shfl_xor_sync(0xffffffffu, f2, o);
      nf += __shfl_xor_sync(0xffffffffu, nf, o);
    }
    if ((tid & 31) == 0) {
      red[0][tid >> 5] = f1;
      red[1][tid >> 5] = f2;
      red[2][tid >> 5] = nf;
    }
    __syncthreads();
    if (tid == 0) {
      double a = 0, b = 0, c = 0;
      for (int i = 0; i < 8; ++i) {
        a += red[0][i];
        b += red[1][i];
        c += red[2][i];
      }
      P.footsum[4 * r] = a;
      P.footsum[4 * r + 1] = b;
      P.footsum[4 * r + 2] = c;
    }
  }
  __syncthreads();
  for (int p = 0; p <= dg; ++p) {
    const float* ph = wh + p * W;
    const float* pl = wl + p * W;
    for (int i = tid; i < foot * sw; i += 256) {
      const int rr = i / sw, px = i - rr * sw;
      const float* src = F + rr * foot + px + 2 * h;
      df a = {0.f, 0.f};
      for (int t = 0; t < W; ++t) df_fma_f(a, src[-t], df{ph[t], pl[t]});
      a = df_norm(a);
      Hh[i] = a.hi;
      Hl[i] = a.lo;
    }
    __syncthreads();
    const int kgp = P.b.kbase[g] + p * (dg + 1) - (p * (p - 1)) / 2;
    for (int q = 0; q <= dg - p; ++q) {
      const float* qh = wh + q * W;
      const float* ql = wl + q * W;
      double* out = reinterpret_cast<double*>(P.C) + ((int64_t)r * P.b.Nb + kgp + q) * P.P;
      for (int i = tid; i < P.P; i += 256) {
        const int py = i / sw, px = i - py * sw;
        const int base = (py + 2 * h) * sw + px;
        df a = {0.f, 0.f};
        for (int t = 0; t < W; ++t)
          df_fma(a, df{Hh[base - t * sw], Hl[base - t * sw]}, df{qh[t], ql[t]});
        out[i] = df_to_d(a);
      }
    }
    __syncthreads();
  }
}

// grid (nreg): weighted Gram of the augmented block in double-float; chunk sums over 32
// pixels are accumulated in FP64, then transformed as in k_stamp_gram.
__global__ void __launch_bounds__(256) k_stamp_gram_df(StampParams P) {
  extern __shared__ double shd[];
  const int r = blockIdx.x, tid = threadIdx.x;
  if (P.st->error || P.st->done) return;
  int cx, cy;
  if (!region_active(P.ptr, P.cand, r, P.max_cand, &cx, &cy)) return;
  if (P.have[r] == P.ptr[r]) return;
  const int Nc = P.Nc, Nb = P.b.Nb;
  const int nblk = (Nc + 3) / 4, npair = nblk * (nblk + 1) / 2;
  double* acc = shd;                                            // [npair][16]
  float* Ah = reinterpret_cast<float*>(acc + (size_t)npair * 16);  // [nblk*4][32]
  float* Al = Ah + nblk * 4 * 32;
  float* wgh = Al + nblk * 4 * 32;                              // [32]
  float* wgl = wgh + 32;
  for (int i = tid; i < npair * 16; i += 256) acc[i] = 0.0;
  const double* Cr = reinterpret_cast<const double*>(P.C) + (int64_t)r * Nb * P.P;
  for (int base = 0; base < P.P; base += 32) {
    __syncthreads();
    for (int i = tid; i < nblk * 4 * 32; i += 256) {
      const int c = i >> 5, j = i & 31, pix = base + j;
      df v = {0.f, 0.f};
      if (pix < P.P && c < Nc) {
        const int py = pix / P.sw, px = pix - py * P.sw;
        const int gx = cx - P.s + px, gy = cy - P.s + py;
        const bool on = gx >= 0 && gx < P.g.W && gy >= 0 && gy < P.g.H;
        const int64_t o = (int64_t)gy * P.g.pitch + gx;
        if (c < Nb) {
          v = df_split(Cr[(int64_t)c * P.P + pix]);
        } else if (on) {
          const bool ok1 = !(P.m1[o] & P.badmask);
          if (c == Nb) v.hi = ok1 ? P.i1[o] : 0.f;
          else if (c == Nb + 1) v.hi = 1.f;
          else v.hi = P.i2[o];
        }
      }
      Ah[i] = v.hi;
      Al[i] = v.lo;
    }
    if (tid < 32) {
      const int pix = base + tid;
      df w = {0.f, 0.f};
      if (pix < P.P) {
        const int py = pix / P.sw, px = pix - py * P.sw;
        const int gx = cx - P.s + px, gy = cy - P.s + py;
        if (gx >= 0 && gx < P.g.W && gy >= 0 && gy < P.g.H) {
          const int64_t o = (int64_t)gy * P.g.pitch + gx;
          if (!((P.m1[o] | P.m2[o]) & P.badmask)) {
            const float a = P.i1[o], b = P.i2[o], vv = P.v1[o] + P.v2[o];
            if (!isfinite(a) || !isfinite(b) || !isfinite(vv)) raise_error(P.st, PSFM_ERR_NONFINITE);
            const double wd = 1.0 / ((double)P.v1[o] + (double)P.v2[o]);
            if (!isfinite(wd)) raise_error(P.st, PSFM_ERR_NONFINITE);
            w = df_split(wd);
          }
        }
      }
      wgh[tid] = w.hi;
      wgl[tid] = w.lo;
    }
    __syncthreads();
    for (int pr = tid; pr < npair; pr += 256) {
      int bi = 0, rem = pr;
      while (rem >= nblk - bi) {
        rem -= nblk - bi;
        ++bi;
      }
      const int bj = bi + rem;
      df s[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) s[e] = df{0.f, 0.f};
      for (int j = 0; j < 32; ++j) {
        const df w = {wgh[j], wgl[j]};
        df a[4], b[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          a[e] = df{Ah[(bi * 4 + e) * 32 + j], Al[(bi * 4 + e) * 32 + j]};
          b[e] = df_mul(w, df{Ah[(bj * 4 + e) * 32 + j], Al[(bj * 4 + e) * 32 + j]});
        }
#pragma unroll
        for (int e = 0; e < 4; ++e)
#pragma unroll
          for (int f = 0; f < 4; ++f) df_fma(s[e * 4 + f], a[e], b[f]);
      }
#pragma unroll
      for (int e = 0; e < 16; ++e) acc[pr * 16 + e] += df_to_d(s[e]);
    }
  }
  __syncthreads();
  double* Gr = P.G + (int64_t)r * Nc * Nc;
  for (int pr = tid; pr < npair; pr += 256) {
    int bi = 0, rem = pr;
    while (rem >= nblk - bi) {
      rem -= nblk - bi;
      ++bi;
    }
    const int bj = bi + rem;
    for (int e = 0; e < 4; ++e)
      for (int f = 0; f < 4; ++f) {
        const int i = bi * 4 + e, j = bj * 4 + f;
        if (i < Nc && j < Nc) {
          Gr[i * Nc + j] = acc[pr * 16 + e * 4 + f];
          Gr[j * Nc + i] = acc[pr * 16 + e * 4 + f];
        }
      }
  }
  __syncthreads();
  double* Gtr = P.Gt + (int64_t)r * Nc * Nc;
  const int cR = Nb;
  for (int q = tid; q < Nc * Nc; q += 256) {
    const int i = q / Nc, j = q - i * Nc;
    const double ai = i < Nb ? P.psi[i] : 1.0, bi = i < Nb ? P.sk[i] : 0.0;
    const double aj = j < Nb ? P.psi[j] : 1.0, bj = j < Nb ? P.sk[j] : 0.0;
    double e = ai * aj * Gr[i * Nc + j];
    if (bj != 0.0) e -= ai * bj * Gr[i * Nc + cR];
    if (bi != 0.0) e -= bi * aj * Gr[cR * Nc + j];
    if (bi != 0.0 && bj != 0.0) e += bi * bj * Gr[cR * Nc + cR];
    Gtr[q] = e;
  }
  __syncthreads();
  if (tid == 0) P.have[r] = P.ptr[r];
}

// grid (nreg): weighted Gram of the augmented design block of one stamp; products in T,
// sums over 32-pixel chunks in T, chunk sums accumulated in FP64.
template <typename T>
__global__ void __launch_bounds__(256) k_stamp_gram(StampParams P) {
  extern __shared__ double shd[];
  const int r = blockIdx.x, tid = threadIdx.x;
  if (P.st->error || P.st->done) return;
  int cx, cy;
  if (!region_active(P.ptr, P.cand, r, P.max_cand, &cx, &cy)) return;
  if (P.have[r] == P.ptr[r]) return;
  const int Nc = P.Nc, Nb = P.b.Nb;
  const int nblk = (Nc + 3) / 4, npair = nblk * (nblk + 1) / 2;
  double* acc = shd;                                        // [npair][16]
  T* A = reinterpret_cast<T*>(acc + (size_t)npair * 16);    // [nblk*4][32]
  T* wgt = A + nblk * 4 * 32;                               // [32]
  for (int i = tid; i < npair * 16; i += 256) acc[i] = 0.0;
  const T* Cr = reinterpret_cast<const T*>(P.C) + (int64_t)r * Nb * P.P;
  for (int base = 0; base < P.P; base += 32) {
    __syncthreads();
    for (int i = tid; i < nblk * 4 * 32; i += 256) {
      const int c = i >> 5, j = i & 31, pix = base + j;
      T v = 0;
      if (pix < P.P && c < Nc) {
        const int py = pix / P.sw, px = pix - py * P.sw;
        const int gx = cx - P.s + px, gy = cy - P.s + py;
        const bool on = gx >= 0 && gx < P.g.W && gy >= 0 && gy < P.g.H;
        const int64_t o = (int64_t)gy * P.g.pitch + gx;
        if (c < Nb) {
          v = Cr[(int64_t)c * P.P + pix];
        } else if (on) {
          const bool ok1 = !(P.m1[o] & P.badmask);
          if (c == Nb) v = ok1 ? (T)P.i1[o] : (T)0;
          else if (c == Nb + 1) v = 1;
          else v = (T)P.i2[o];
        }
      }
      A[i] = v;
    }
    if (tid < 32) {
      const int pix = base + tid;
      T w = 0;
      if (pix < P.P) {
        const int py = pix / P.sw, px = pix - py * P.sw;
        const int gx = cx - P.s + px, gy = cy - P.s + py;
        if (gx >= 0 && gx < P.g.W && gy >= 0 && gy < P.g.H) {
          const int64_t o = (int64_t)gy * P.g.pitch + gx;
          if (!((P.m1[o] | P.m2[o]) & P.badmask)) {
            const float a = P.i1[o], b = P.i2[o], vv = P.v1[o] + P.v2[o];
            if (!isfinite(a) || !isfinite(b) || !isfinite(vv)) raise_error(P.st, PSFM_ERR_NONFINITE);
            w = (T)(1.0 / ((double)P.v1[o] + (double)P.v2[o]));
            if (!isfinite(w)) raise_error(P.st, PSFM_ERR_NONFINITE);
          }
        }
      }
      wgt[tid] = w;
    }
    __syncthreads();
    for (int pr = tid; pr < npair; pr += 256) {
      // pair index -> (bi, bj), bi <= bj
      int bi = 0, rem = pr;
      while (rem >= nblk - bi) {
        rem -= nblk - bi;
        ++bi;
      }
      const int bj = bi + rem;
      T s[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) s[e] = 0;
      for (int j = 0; j < 32; ++j) {
        const T w = wgt[j];
        T a[4], b[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          a[e] = A[(bi * 4 + e) * 32 + j];
          b[e] = w * A[(bj * 4 + e) * 32 + j];
        }
#pragma unroll
        for (int e = 0; e < 4; ++e)
#pragma unroll
          for (int f = 0; f < 4; ++f) s[e * 4 + f] = fma(a[e], b[f], s[e * 4 + f]);
      }
#pragma unroll
      for (int e = 0; e < 16; ++e) acc[pr * 16 + e] += (double)s[e];
    }
  }
  __syncthreads();
  double* Gr = P.G + (int64_t)r * Nc * Nc;
  for (int pr = tid; pr < npair; pr += 256) {
    int bi = 0, rem = pr;
    while (rem >= nblk - bi) {
      rem -= nblk - bi;
      ++bi;
    }
    const int bj = bi + rem;
    for (int e = 0; e < 4; ++e)
      for (int f = 0; f < 4; ++f) {
        const int i = bi * 4 + e, j = bj * 4 + f;
        if (i < Nc && j < Nc) {
          Gr[i * Nc + j] = acc[pr * 16 + e * 4 + f];
          Gr[j * Nc + i] = acc[pr * 16 + e * 4 + f];
        }
      }
  }
  __syncthreads();
  // transformed Gram: basis column k becomes psi_k C_k - s_k R (the zero-sum term B_k of
  // Sec. 2 convolved with R); the R, 1 and I2 columns are unchanged
  double* Gtr = P.Gt + (int64_t)r * Nc * Nc;
  const int cR = Nb;
  for (int q = tid; q < Nc * Nc; q += 256) {
    const int i = q / Nc, j = q - i * Nc;
    const double ai = i < Nb ? P.psi[i] : 1.0, bi = i < Nb ? P.sk[i] : 0.0;
    const double aj = j < Nb ? P.psi[j] : 1.0, bj = j < Nb ? P.sk[j] : 0.0;
    double e = ai * aj * Gr[i * Nc + j];
    if (bj != 0.0) e -= ai * bj * Gr[i * Nc + cR];
    if (bi != 0.0) e -= bi * aj * Gr[cR * Nc + j];
    if (bi != 0.0 && bj != 0.0) e += bi * bj * Gr[cR * Nc + cR];
    Gtr[q] = e;
  }
  __syncthreads();
  if (tid == 0) P.have[r] = P.ptr[r];
}

struct SysParams {
  BasisDev b;
  ImgGeom g;
  int nreg, max_cand, Nc, Nsys, joint;
  const int32_t* cand;
  const int32_t* ptr;
  const double* Gt;
  const double* footsum;
  double* gv;      // [nreg][Ns] spatial factors at the stamp centre, 0 if inactive
  double* dsol;
  double* M;
  double* L;
  double* v;
  DevState* st;
};

// Fixed-order block sum (deterministic for a given launch shape).
__device__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < nw; ++i) t += sh[i];
  __syncthreads();
  return t;
}

// Active count, spatial factors, and (SEPARATE) b0, d0 from the unweighted regression of
// footprint sums (Sec. 3.2).  One CTA of 1024 threads.
__global__ void __launch_bounds__(1024) k_norm(SysParams P) {
  __shared__ double sh[32];
  if (P.st->error || P.st->done) return;
  double n = 0, s11 = 0, s12 = 0, s22 = 0, t1 = 0, t2 = 0;
  const double xs = P.g.W > 1 ? 2.0 / (P.g.W - 1) : 0.0, ys = P.g.H > 1 ? 2.0 / (P.g.H - 1) : 0.0;
  for (int r = threadIdx.x; r < P.nreg; r += blockDim.x) {
    int cx, cy;
    double* gr = P.gv + (int64_t)r * P.b.Ns;
    if (!region_active(P.ptr, P.cand, r, P.max_cand, &cx, &cy)) {
      for (int s = 0; s < P.b.Ns; ++s) gr[s] = 0.0;
      continue;
    }
    n += 1.0;
    const double xt = P.g.W > 1 ? cx * xs - 1.0 : 0.0;
    const double yt = P.g.H > 1 ? cy * ys - 1.0 : 0.0;
    int s = 0;
    double xp = 1.0;
    for (int l = 0; l <= P.b.S; ++l) {
      double yp = 1.0;
      for (int m = 0; m <= P.b.S - l; ++m) {
        gr[s++] = xp * yp;
        yp *= yt;
      }
      xp *= xt;
    }
    const double F1 = P.footsum[4 * r], F2 = P.footsum[4 * r + 1], nf = P.footsum[4 * r + 2];
    s11 += F1 * F1;
    s12 += F1 * nf;
    s22 += nf * nf;
    t1 += F1 * F2;
    t2 += nf * F2;
  }
  n = block_sum(n, sh);
  s11 = block_sum(s11, sh);
  s12 = block_sum(s12, sh);
  s22 = block_sum(s22, sh);
  t1 = block_sum(t1, sh);
  t2 = block_sum(t2, sh);
  if (threadIdx.x != 0) return;
  P.st->n_active = (int)n;
  P.st->chol_fail = 0;
  if (n < 3) {
    raise_error(P.st, PSFM_ERR_TOO_FEW_STAMPS);
    return;
  }
  if (!P.joint) {
    // 2 x 2 normal equations by Cholesky, Cramer's rule if not positive definite
    double b0, d0;
    const double l11 = sqrt(s11);
    const double l21 = s12 / l11;
    const double q = s22 - l21 * l21;
    if (s11 > 0.0 && q > 0.0) {
      const double l22 = sqrt(q);
      const double z1 = t1 / l11, z2 = (t2 - l21 * z1) / l22;
      d0 = z2 / l22;
      b0 = (z1 - l21 * d0) / l11;
    } else {
      const double det = s11 * s22 - s12 * s12;
      if (det == 0.0) {
        raise_error(P.st, PSFM_ERR_SINGULAR);
        return;
      }
      b0 = (t1 * s22 - s12 * t2) / det;
      d0 = (s11 * t2 - s12 * t1) / det;
    }
    P.dsol[0] = b0;
    P.dsol[1] = d0;
  }
}

// Unknown u -> (augmented-block column, spatial term or -1 for the JOINT b0 / d0 columns).
__device__ __forceinline__ void unknown_col(const SysParams& P, int u, int* a, int* s) {
  if (P.joint) {
    if (u == 0) {
      *a = P.b.Nb;  // R
      *s = -1;
      return;
    }
    if (u == P.Nsys - 1) {
      *a = P.b.Nb + 1;  // 1
      *s = -1;
      return;
    }
    u -= 1;
  }
  *a = u / P.b.Ns;
  *s = u - *a * P.b.Ns;
}

// M and v (Eq. 5-6 with g_i at the stamp centres): M_{(c,s),(c',s')} = sum_stamps g_s g_s'
// Gt[c][c'] with the transformed stamp Grams.  One thread per (u, u') entry; the spatial
// factors of a chunk of stamps are staged in shared memory.
constexpr int kAsmChunk = 512;
__global__ void __launch_bounds__(256) k_assemble(SysParams P) {
  __shared__ double gsh[kAsmChunk * kMaxSpatial];
  if (P.st->error || P.st->done) return;
  const int Ns = P.b.Ns, Nc = P.Nc, N = P.Nsys;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool mine = t < (int64_t)N * N;
  int ui = 0, uj = 0, ai = 0, aj = 0, si = -1, sj = -1;
  if (mine) {
    ui = (int)(t / N);
    uj = (int)(t - (int64_t)ui * N);
    unknown_col(P, ui, &ai, &si);
    unknown_col(P, uj, &aj, &sj);
  }
  const bool rhs = t < N;
  int av = 0, sv = -1;
  if (rhs) unknown_col(P, (int)t, &av, &sv);
  const int colR = P.b.Nb, col1 = P.b.Nb + 1, colI = P.b.Nb + 2;
  const double b0 = P.dsol[0], d0 = P.dsol[1];
  double acc = 0.0, accv = 0.0;
  for (int r0 = 0; r0 < P.nreg; r0 += kAsmChunk) {
    const int nr = min(kAsmChunk, P.nreg - r0);
    __syncthreads();
    for (int q = threadIdx.x; q < nr * Ns; q += blockDim.x) gsh[q] = P.gv[(int64_t)r0 * Ns + q];
    __syncthreads();
    for (int r = 0; r < nr; ++r) {
      const double* gr = gsh + r * Ns;
      if (gr[0] == 0.0) continue;  // inactive (the constant spatial term is 1)
      const double* Gr = P.Gt + (int64_t)(r0 + r) * Nc * Nc;
      if (mine) {
        const double gi = si < 0 ? 1.0 : gr[si], gj = sj < 0 ? 1.0 : gr[sj];
        acc += gi * gj * Gr[ai * Nc + aj];
      }
      if (rhs) {
        double e = Gr[av * Nc + colI];
        if (!P.joint) e -= b0 * Gr[av * Nc + colR] + d0 * Gr[av * Nc + col1];
        accv += (sv < 0 ? 1.0 : gr[sv]) * e;
      }
    }
  }
  if (mine) {
    P.M[t] = acc;
    P.L[t] = acc;
  }
  if (rhs) P.v[t] = accv;
}

// ---- Cholesky of the N x N system in FP64, right-looking by 32-column panels, spread over
// the GPU: the diagonal block is factored (and inverted) by one CTA, the panel below by
// 4-row CTAs, the trailing lower triangle by 16 x 16 tiles.  L holds M on entry.
constexpr int kNB = 32;

// Diagonal block: one warp, lane i holding row i of the 32 x 32 block in registers (rows
// beyond the matrix are padded with the identity), factored column by column with shuffles;
// then lane c builds column c of the block's inverse by forward substitution.
__global__ void __launch_bounds__(32) k_chol_diag(int n, int kb, double* L, double* Linv_all,
                                                  DevState* st) {
  if (st->error || st->done || st->chol_fail) return;
  const int k0 = kb * kNB, m = min(kNB, n - k0), lane = threadIdx.x;
  const unsigned full = 0xffffffffu;
  double a[kNB];
#pragma unroll
  for (int c = 0; c < kNB; ++c)
    a[c] = (lane < m && c <= lane) ? L[(int64_t)(k0 + lane) * n + k0 + c] : (lane == c ? 1.0 : 0.0);
  bool fail = false;
#pragma unroll
  for (int j = 0; j < kNB; ++j) {
    const double djj = __shfl_sync(full, a[j], j);
    if (!(djj > 0.0) || !isfinite(djj)) fail = true;
    const double ljj = sqrt(djj);
    const double rinv = 1.0 / ljj;
    if (lane == j)
      a[j] = ljj;
    else if (lane > j)
      a[j] *= rinv;
#pragma unroll
    for (int c = j + 1; c < kNB; ++c) {
      const double lcj = __shfl_sync(full, a[j], c);
      if (lane >= c) a[c] = fma(-a[j], lcj, a[c]);
    }
  }
  if (fail) {
    if (lane == 0) st->chol_fail = 1;
    return;
  }
  double x[kNB];  // x[i] = inv(L)[i][lane]
#pragma unroll
  for (int i = 0; i < kNB; ++i) {
    double sacc = lane == i ? 1.0 : 0.0;
#pragma unroll
    for (int t = 0; t < i; ++t) sacc = fma(-__shfl_sync(full, a[t], i), x[t], sacc);
    x[i] = sacc / __shfl_sync(full, a[i], i);
  }
  double* Linv = Linv_all + (int64_t)kb * kNB * kNB;
#pragma unroll
  for (int i = 0; i < kNB; ++i) Linv[i * kNB + lane] = x[i];
  if (lane < m) {
#pragma unroll
    for (int c = 0; c < kNB; ++c)
      if (c <= lane) L[(int64_t)(k0 + lane) * n + k0 + c] = a[c];
  }
}

// Rows below the diagonal block: L_ik = A_ik inv(L_kk)^T.  4 rows per CTA.
__global__ void __launch_bounds__(128) k_chol_trsm(int n, int kb, double* L,
                                                   const double* Linv_all, const DevState* st) {
  __shared__ double Li[kNB][kNB + 1];
  __shared__ double Ar[4][kNB];
  if (st->error || st->done || st->chol_fail) return;
  const int k0 = kb * kNB, m = min(kNB, n - k0);
  const int r0 = k0 + m + blockIdx.x * 4;
  const double* Linv = Linv_all + (int64_t)kb * kNB * kNB;
  for (int i = threadIdx.x; i < kNB * kNB; i += blockDim.x) Li[i / kNB][i % kNB] = Linv[i];
  const int rr = threadIdx.x / kNB, c = threadIdx.x % kNB;
  const int row = r0 + rr;
  Ar[rr][c] = (row < n && c < m) ? L[(int64_t)row * n + k0 + c] : 0.0;
  __syncthreads();
  if (row < n && c < m) {
    double sacc = 0.0;
    for (int t2 = 0; t2 <= c; ++t2) sacc += Ar[rr][t2] * Li[c][t2];
    L[(int64_t)row * n + k0 + c] = sacc;
  }
}

// Trailing update of the lower triangle: A_ij -= L_i,panel . L_j,panel, 16 x 16 tiles.
__global__ void __launch_bounds__(256) k_chol_update(int n, int kb, double* L,
                                                     const DevState* st) {
  __shared__ double Pi[16][kNB + 1];
  __shared__ double Pj[16][kNB + 1];
  if (st->error || st->done || st->chol_fail) return;
  const int k0 = kb * kNB, m = min(kNB, n - k0);
  const int base = k0 + m;
  const int nt = (n - base + 15) / 16;
  // tile index -> (ti, tj), tj <= ti
  int t = blockIdx.x, ti = 0;
  while (t >= ti + 1) {
    t -= ti + 1;
    ++ti;
  }
  const int tj = t;
  if (ti >= nt) return;
  const int r0 = base + ti * 16, c0 = base + tj * 16;
  for (int i = threadIdx.x; i < 16 * kNB; i += blockDim.x) {
    const int r = i / kNB, c = i % kNB;
    Pi[r][c] = (r0 + r < n && c < m) ? L[(int64_t)(r0 + r) * n + k0 + c] : 0.0;
    Pj[r][c] = (c0 + r < n && c < m) ? L[(int64_t)(c0 + r) * n + k0 + c] : 0.0;
  }
  __syncthreads();
  const int y = threadIdx.x / 16, x = threadIdx.x % 16;
  const int row = r0 + y, col = c0 + x;
  if (row < n && col < n && col <= row) {
    double sacc = 0.0;
    for (int c = 0; c < m; ++c) sacc += Pi[y][c] * Pj[x][c];
    L[(int64_t)row * n + col] -= sacc;
  }
}

// L z = v then L^T x = z with the factored blocks and their inverses; one CTA of 1024
// threads, blocked by panels.  Writes the solution into the device solution vector.
__global__ void __launch_bounds__(1024) k_chol_solve(int n, int joint, const double* L,
                                                     const double* Linv_all, const double* v,
                                                     double* dsol, DevState* st) {
  extern __shared__ double ys[];  // [n] + [32][33]
  double* part = ys + n;
  if (st->error || st->done || st->chol_fail) return;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  for (int i = tid; i < n; i += blockDim.x) ys[i] = v[i];
  __syncthreads();
  const int nb = (n + kNB - 1) / kNB;
  // forward: y_b = inv(L_bb) (v_b - L_b,<b y_<b)
  for (int b = 0; b < nb; ++b) {
    const int k0 = b * kNB, m = min(kNB, n - k0);
    // warp w: row k0 + w, lanes over previous columns
    double sacc = 0.0;
    if (w < m)
      for (int c = lane; c < k0; c += 32) sacc += L[(int64_t)(k0 + w) * n + c] * ys[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
    __syncthreads();
    if (w < m && lane == 0) part[w] = ys[k0 + w] - sacc;
    __syncthreads();
    const double* Li = Linv_all + (int64_t)b * kNB * kNB;
    if (w < m) {
      double t2 = 0.0;
      if (lane <= w) t2 = Li[w * kNB + lane] * part[lane];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t2 += __shfl_xor_sync(0xffffffffu, t2, o);
      if (lane == 0) ys[k0 + w] = t2;
    }
    __syncthreads();
  }
  // backward: x_b = inv(L_bb)^T (y_b - L_>b,b^T x_>b)
  for (int b = nb - 1; b >= 0; --b) {
    const int k0 = b * kNB, m = min(kNB, n - k0);
    // part[w][lane]: warp w sums rows i = k0 + m + w, +32, ... for column lane
    double sacc = 0.0;
    if (lane < m)
      for (int i = k0 + m + w; i < n; i += 32) sacc += L[(int64_t)i * n + k0 + lane] * ys[i];
    __syncthreads();
    double* pw = ys + n;  // [33][33]: per-warp partial sums, then z in row 32
    pw[w * 33 + lane] = sacc;
    __syncthreads();
    if (tid < m) {
      double z = ys[k0 + tid];
      for (int q = 0; q < 32; ++q) z -= pw[q * 33 + tid];
      pw[32 * 33 + tid] = z;
    }
    __syncthreads();
    const double* Li = Linv_all + (int64_t)b * kNB * kNB;
    if (w < m) {
      // x_w = sum_j inv(L)[j][w] z_j for j >= w
      double t2 = 0.0;
      if (lane >= w && lane < m) t2 = Li[lane * kNB + w] * pw[32 * 33 + lane];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t2 += __shfl_xor_sync(0xffffffffu, t2, o);
      if (lane == 0) ys[k0 + w] = t2;
    }
    __syncthreads();
  }
  for (int i = tid; i < n; i += blockDim.x) {
    const double x = ys[i];
    if (!isfinite(x)) raise_error(st, PSFM_ERR_SINGULAR);
    if (joint) {
      if (i == 0) dsol[0] = x;
      else if (i == n - 1) dsol[1] = x;
      else dsol[2 + (i - 1)] = x;
    } else {
      dsol[2 + i] = x;
    }
  }
}

// Fallback when the Cholesky factorisation meets a non-positive pivot: LU with partial
// pivoting in FP64, one CTA (rare path).
__global__ void __launch_bounds__(1024) k_lu_solve(int N, int joint, const double* M,
                                                   const double* v, double* L, double* y,
                                                   int32_t* piv, double* dsol, DevState* st) {
  const int tid = threadIdx.x, nt = blockDim.x;
  __shared__ int s_fail;
  if (st->error || st->done || !st->chol_fail) return;
  for (int64_t i = tid; i < (int64_t)N * N; i += nt) L[i] = M[i];
  for (int i = tid; i < N; i += nt) y[i] = v[i];
  if (tid == 0) s_fail = 0;
  __syncthreads();
  for (int j = 0; j < N; ++j) {
    if (tid == 0) {
      int pr = j;
      double best = fabs(L[(int64_t)j * N + j]);
      for (int i = j + 1; i < N; ++i) {
        const double a = fabs(L[(int64_t)i * N + j]);
        if (a > best) {
          best = a;
          pr = i;
        }
      }
      piv[j] = pr;
      if (!(best > 0.0)) s_fail = 2;
    }
    __syncthreads();
    if (s_fail == 2) break;
    const int pr = piv[j];
    if (pr != j) {
      for (int k = tid; k < N; k += nt) {
        const double a = L[(int64_t)j * N + k];
        L[(int64_t)j * N + k] = L[(int64_t)pr * N + k];
        L[(int64_t)pr * N + k] = a;
      }
      if (tid == 0) {
        const double a = y[j];
        y[j] = y[pr];
        y[pr] = a;
      }
    }
    __syncthreads();
    const double d = L[(int64_t)j * N + j];
    for (int i = j + 1 + tid; i < N; i += nt) {
      const double f = L[(int64_t)i * N + j] / d;
      L[(int64_t)i * N + j] = f;
      double* Li = L + (int64_t)i * N;
      const double* Lj = L + (int64_t)j * N;
      for (int k = j + 1; k < N; ++k) Li[k] -= f * Lj[k];
      y[i] -= f * y[j];
    }
    __syncthreads();
  }
  if (s_fail == 2) {
    if (tid == 0) raise_error(st, PSFM_ERR_SINGULAR);
    return;
  }
  for (int j = N - 1; j >= 0; --j) {
    if (tid == 0) y[j] /= L[(int64_t)j * N + j];
    __syncthreads();
    const double yj = y[j];
    for (int i = tid; i < j; i += nt) y[i] -= L[(int64_t)i * N + j] * yj;
    __syncthreads();
  }
  for (int i = tid; i < N; i += nt) {
    const double x = y[i];
    if (!isfinite(x)) raise_error(st, PSFM_ERR_SINGULAR);
    if (joint) {
      if (i == 0) dsol[0] = x;
      else if (i == N - 1) dsol[1] = x;
      else dsol[2 + (i - 1)] = x;
    } else {
      dsol[2 + i] = x;
    }
  }
}

struct Chi2Params {
  StampParams sp;
  const double* gv;
  const double* dsol;
  double alpha;
  double* chi2;
  double* cand_chi2;
};

// grid (nreg): chi^2 of the active stamp with the current solution (FP64).
template <typename T>
__global__ void __launch_bounds__(256) k_chi2(Chi2Params Q) {
  const StampParams& P = Q.sp;
  extern __shared__ double ak[];  // [Nb]: a_k(stamp) psi_k
  __shared__ double red[2][8];
  __shared__ double s_delta;
  const int r = blockIdx.x, tid = threadIdx.x;
  if (P.st->error || P.st->done) return;
  int cx, cy;
  if (!region_active(P.ptr, P.cand, r, P.max_cand, &cx, &cy)) return;
  const int Nb = P.b.Nb, Ns = P.b.Ns;
  const double* gr = Q.gv + (int64_t)r * Ns;
  for (int k = tid; k < Nb; k += 256) {
    double a = 0.0;
    for (int s = 0; s < Ns; ++s) a += Q.dsol[2 + k * Ns + s] * gr[s];
    ak[k] = a;
  }
  __syncthreads();
  if (tid == 0) {
    double d = Q.dsol[0];
    for (int k = 0; k < Nb; ++k) {
      d -= ak[k] * P.sk[k];
    }
    s_delta = d;
  }
  __syncthreads();
  for (int k = tid; k < Nb; k += 256) ak[k] *= P.psi[k];
  __syncthreads();
  const double delta = s_delta, d0 = Q.dsol[1];
  const T* Cr = reinterpret_cast<const T*>(P.C) + (int64_t)r * Nb * P.P;
  double q = 0.0, n = 0.0;
  for (int pix = tid; pix < P.P; pix += 256) {
    const int py = pix / P.sw, px = pix - py * P.sw;
    const int gx = cx - P.s + px, gy = cy - P.s + py;
    if (gx < 0 || gx >= P.g.W || gy < 0 || gy >= P.g.H) continue;
    const int64_t o = (int64_t)gy * P.g.pitch + gx;
    if ((P.m1[o] | P.m2[o]) & P.badmask) continue;
    const double R = P.i1[o], I2 = P.i2[o];
    double model = delta * R + d0;
    for (int k = 0; k < Nb; ++k) model += ak[k] * (double)Cr[(int64_t)k * P.P + pix];
    const double res = I2 - model;
    const double den = ((double)P.v1[o] + (double)P.v2[o]) + Q.alpha * fabs(I2);
    q += res * res / den;
    n += 1.0;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    q += __shfl_xor_sync(0xffffffffu, q, o);
    n += __shfl_xor_sync(0xffffffffu, n, o);
  }
  if ((tid & 31) == 0) {
    red[0][tid >> 5] = q;
    red[1][tid >> 5] = n;
  }
  __syncthreads();
  if (tid == 0) {
    double a = 0, b = 0;
    for (int i = 0; i < 8; ++i) {
      a += red[0][i];
      b += red[1][i];
    }
    const double c = a / (b > 1.0 ? b : 1.0);
    Q.chi2[r] = c;
    Q.cand_chi2[(int64_t)r * P.max_cand + P.ptr[r]] = c;
  }
}

// Rejection decision of Sec. 3.3 and loop control; one CTA of 1024 threads.
__global__ void __launch_bounds__(1024) k_reject(int nreg, int max_cand, int max_iter,
                                                 double nsig, const int32_t* cand, int32_t* ptr,
                                                 int32_t* cand_stat, const double* chi2,
                                                 DevState* st) {
  __shared__ double sh[32];
  __shared__ int s_finish;
  if (st->error || st->done) return;
  double n = 0.0, sum = 0.0;
  for (int r = threadIdx.x; r < nreg; r += blockDim.x) {
    int cx, cy;
    if (!region_active(ptr, cand, r, max_cand, &cx, &cy)) continue;
    sum += chi2[r];
    n += 1.0;
  }
  n = block_sum(n, sh);
  sum = block_sum(sum, sh);
  const double mu = sum / n;
  double ss = 0.0;
  for (int r = threadIdx.x; r < nreg; r += blockDim.x) {
    int cx, cy;
    if (!region_active(ptr, cand, r, max_cand, &cx, &cy)) continue;
    const double d = chi2[r] - mu;
    ss += d * d;
  }
  ss = block_sum(ss, sh);
  const double sd = sqrt(ss / n);
  const int it = st->iter;
  bool finish = it == max_iter - 1;
  double nrej = 0.0;
  if (!finish) {
    const double thr = mu + nsig * sd;
    for (int r = threadIdx.x; r < nreg; r += blockDim.x) {
      int cx, cy;
      if (!region_active(ptr, cand, r, max_cand, &cx, &cy)) continue;
      if (chi2[r] > thr) {
        cand_stat[(int64_t)r * max_cand + ptr[r]] = PSFM_CAND_REJECTED;
        ptr[r] += 1;
        nrej += 1.0;
      }
    }
    nrej = block_sum(nrej, sh);
    finish = nrej == 0.0;
    if (threadIdx.x == 0) st->threshold = thr;
  }
  if (threadIdx.x == 0) {
    st->chi2_mean = mu;
    st->chi2_rms = sd;
    st->iter = it + 1;
    s_finish = finish;
  }
  __syncthreads();
  if (s_finish) {
    double nu = 0.0;
    for (int r = threadIdx.x; r < nreg; r += blockDim.x) {
      int cx, cy;
      if (!region_active(ptr, cand, r, max_cand, &cx, &cy)) continue;
      cand_stat[(int64_t)r * max_cand + ptr[r]] = PSFM_CAND_USED;
      nu += 1.0;
    }
    nu = block_sum(nu, sh);
    if (threadIdx.x == 0) {
      st->n_active = (int)nu;
      st->done = 1;
    }
  }
}

}  // namespace

cudaError_t launch_extract(const Plan& p, DevState* st, const SolveBuffers& b, const float* img,
                           const float* ref, const float* var_img, const float* var_ref,
                           const uint16_t* mask_img, const uint16_t* mask_ref, cudaStream_t s);
cudaError_t launch_caller_stamps(const Plan& p, DevState* st, const SolveBuffers& b,
                                 const psfm_stamp* stamps, cudaStream_t s);

void carve_solve(const Plan& p, Workspace& ws, SolveBuffers& b) {
  const int nwords = (p.W + 31) / 32;
  b.hist = ws.take<uint32_t>(3 * 2048);
  b.badbits = ws.take<uint32_t>((size_t)p.H * nwords);
  b.bin_val = ws.take<float>((size_t)p.nreg * kBinCap);
  b.bin_idx = ws.take<int32_t>((size_t)p.nreg * kBinCap);
  b.bin_cnt = ws.take<int32_t>(p.nreg);
  b.cand = ws.take<int32_t>((size_t)p.nreg * p.max_cand * 2);
  b.cand_stat = ws.take<int32_t>((size_t)p.nreg * p.max_cand);
  b.cand_chi2 = ws.take<double>((size_t)p.nreg * p.max_cand);
  b.ptr = ws.take<int32_t>(p.nreg);
  b.have = ws.take<int32_t>(p.nreg);
  b.C = ws.take<double>((size_t)p.nreg * p.Nb * p.P);
  b.G = ws.take<double>((size_t)p.nreg * p.Nc * p.Nc);
  b.Gt = ws.take<double>((size_t)p.nreg * p.Nc * p.Nc);
  b.foot = ws.take<double>((size_t)p.nreg * 4);
  b.chi2 = ws.take<double>(p.nreg);
  b.M = ws.take<double>((size_t)p.Nsys * p.Nsys);
  b.v = ws.take<double>(p.Nsys);
  b.L = ws.take<double>((size_t)p.Nsys * p.Nsys);
  b.Linv = ws.take<double>((size_t)((p.Nsys + kNB - 1) / kNB) * kNB * kNB);
  b.y = ws.take<double>(p.Nsys);
  b.piv = ws.take<int32_t>(p.Nsys);
  b.gv = ws.take<double>((size_t)p.nreg * p.Ns);
}

psfm_status run_solve(const Plan& p, const DevTables& t, DevState* st, double* dsol,
                      const SolveBuffers& b, const float* img, const float* ref,
                      const float* var_img, const float* var_ref, const uint16_t* mask_img,
                      const uint16_t* mask_ref, const psfm_stamp* stamps, cudaStream_t s) {
  cudaError_t e;
  prof_begin("extract", s);
  if (p.n_stamps > 0)
    e = launch_caller_stamps(p, st, b, stamps, s);
  else
    e = launch_extract(p, st, b, img, ref, var_img, var_ref, mask_img, mask_ref, s);
  prof_end("extract", s, p.n_stamps > 0 ? 1 : 9);
  if (e != cudaSuccess) return PSFM_ERR_CUDA;

  StampParams sp;
  sp.b = basis_dev(p);
  sp.g = ImgGeom{p.W, p.H, p.pitch};
  sp.i1 = ref;
  sp.i2 = img;
  sp.v1 = var_ref;
  sp.v2 = var_img;
  sp.m1 = mask_ref;
  sp.m2 = mask_img;
  sp.badmask = p.cfg.badmask;
  sp.s = p.s;
  sp.sw = p.sw;
  sp.P = p.P;
  sp.foot = p.foot;
  sp.max_cand = p.max_cand;
  sp.Nc = p.Nc;
  sp.f1d = t.f1d;
  sp.f1d64 = t.f1d64;
  sp.psi = t.psi;
  sp.sk = t.sk;
  sp.cand = b.cand;
  sp.ptr = b.ptr;
  sp.have = b.have;
  sp.C = b.C;
  sp.G = b.G;
  sp.Gt = b.Gt;
  sp.footsum = b.foot;
  sp.st = st;

  SysParams sy;
  sy.b = sp.b;
  sy.g = sp.g;
  sy.nreg = p.nreg;
  sy.max_cand = p.max_cand;
  sy.Nc = p.Nc;
  sy.Nsys = p.Nsys;
  sy.joint = p.cfg.norm_mode == PSFM_NORM_JOINT;
  sy.cand = b.cand;
  sy.ptr = b.ptr;
  sy.Gt = b.Gt;
  sy.footsum = b.foot;
  sy.gv = b.gv;
  sy.dsol = dsol;
  sy.M = b.M;
  sy.L = b.L;
  sy.v = b.v;
  sy.st = st;

  Chi2Params cq;
  cq.sp = sp;
  cq.gv = sy.gv;
  cq.dsol = dsol;
  cq.alpha = p.cfg.soften_alpha;
  cq.chi2 = b.chi2;
  cq.cand_chi2 = b.cand_chi2;

  // design block storage is double for the FP64 and double-float modes, float for FP32
  const int prec = p.cfg.precision;
  const bool wide = prec != PSFM_PREC_FP32;
  const size_t esz = prec == PSFM_PREC_FP64 ? sizeof(double) : sizeof(float);
  size_t sm_design = esz * ((size_t)p.foot * p.foot + (size_t)p.foot * p.sw);
  const int nblk = (p.Nc + 3) / 4, npair = nblk * (nblk + 1) / 2;
  size_t sm_gram = sizeof(double) * npair * 16 + esz * (nblk * 4 * 32 + 32);
  if (prec == PSFM_PREC_F32X2) {
    sm_design = sizeof(float) * ((size_t)p.foot * p.foot + 2 * (size_t)p.foot * p.sw +
                                 2 * (size_t)(p.dmax + 1) * p.w);
    sm_gram = sizeof(double) * npair * 16 + sizeof(float) * (2 * nblk * 4 * 32 + 64);
  }
  if (sm_design > 200 * 1024 || sm_gram > 200 * 1024) return PSFM_ERR_UNSUPPORTED;
  auto design = prec == PSFM_PREC_FP64 ? k_stamp_design<double>
                : prec == PSFM_PREC_F32X2 ? k_stamp_design_df : k_stamp_design<float>;
  auto gram = prec == PSFM_PREC_FP64 ? k_stamp_gram<double>
              : prec == PSFM_PREC_F32X2 ? k_stamp_gram_df : k_stamp_gram<float>;
  auto chi2 = wide ? k_chi2<double> : k_chi2<float>;
  if (cudaFuncSetAttribute(design, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_design) !=
          cudaSuccess ||
      cudaFuncSetAttribute(gram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_gram) !=
          cudaSuccess)
    return PSFM_ERR_CUDA;
  const int N = p.Nsys;
  const int64_t nthr = (int64_t)N * N;
  const int npanel = (N + kNB - 1) / kNB;
  const size_t sm_solve = sizeof(double) * ((size_t)N + 33 * 33);
  if (sm_solve > 200 * 1024) return PSFM_ERR_UNSUPPORTED;
  if (cudaFuncSetAttribute(k_chol_solve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sm_solve) != cudaSuccess)
    return PSFM_ERR_CUDA;
  for (int it = 0; it < p.cfg.max_iter; ++it) {
    prof_begin("stamps", s);
    design<<<dim3(p.nreg, p.ng), 256, sm_design, s>>>(sp);
    gram<<<p.nreg, 256, sm_gram, s>>>(sp);
    prof_end("stamps", s, 2);
    prof_begin("system", s);
    k_norm<<<1, 1024, 0, s>>>(sy);
    k_assemble<<<(unsigned)((nthr + 255) / 256), 256, 0, s>>>(sy);
    prof_end("system", s, 2);
    prof_begin("cholesky", s);
    for (int kb = 0; kb < npanel; ++kb) {
      k_chol_diag<<<1, 32, 0, s>>>(N, kb, b.L, b.Linv, st);
      const int k0 = kb * kNB, m = (N - k0) < kNB ? N - k0 : kNB;
      const int rest = N - k0 - m;
      if (rest > 0) {
        k_chol_trsm<<<(rest + 3) / 4, 128, 0, s>>>(N, kb, b.L, b.Linv, st);
        const int nt = (rest + 15) / 16;
        k_chol_update<<<nt * (nt + 1) / 2, 256, 0, s>>>(N, kb, b.L, st);
      }
    }
    k_chol_solve<<<1, 1024, sm_solve, s>>>(N, sy.joint, b.L, b.Linv, b.v, dsol, st);
    k_lu_solve<<<1, 1024, 0, s>>>(N, sy.joint, b.M, b.v, b.L, b.y, b.piv, dsol, st);
    prof_end("cholesky", s, 3 * npanel + 2);
    prof_begin("chi2_reject", s);
    chi2<<<p.nreg, 256, sizeof(double) * p.Nb, s>>>(cq);
    k_reject<<<1, 1024, 0, s>>>(p.nreg, p.max_cand, p.cfg.max_iter, p.cfg.reject_nsigma, b.cand,
                                b.ptr, b.cand_stat, b.chi2, st);
    prof_end("chi2_reject", s, 2);
  }
  prof_begin("rbad", s);
  if (launch_rbad(p, t, dsol, st, s) != cudaSuccess) return PSFM_ERR_CUDA;
  prof_end("rbad", s, 1);
  return cudaGetLastError() == cudaSuccess ? PSFM_OK : PSFM_ERR_CUDA;
}

psfm_status sync_status(const DevState* st, cudaStream_t s) {
  int32_t err = 0;
  if (cudaMemcpyAsync(&err, &st->error, sizeof(err), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return PSFM_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return PSFM_ERR_CUDA;
  return err;
}

psfm_status fetch_solution(const Plan& p, const DevState* st, const double* dsol,
                           const SolveBuffers& b, psfm_solution* out, cudaStream_t s) {
  DevState h;
  std::vector<double> sol(2 + p.ncoef);
  const size_t nc = (size_t)p.nreg * p.max_cand;
  std::vector<int32_t> cand(2 * nc), stat(nc);
  std::vector<double> chi2(nc);
  if (cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(sol.data(), dsol, sizeof(double) * sol.size(), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(cand.data(), b.cand, sizeof(int32_t) * cand.size(), cudaMemcpyDeviceToHost,
                      s) != cudaSuccess ||
      cudaMemcpyAsync(stat.data(), b.cand_stat, sizeof(int32_t) * nc, cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(chi2.data(), b.cand_chi2, sizeof(double) * nc, cudaMemcpyDeviceToHost, s) !=
          cudaSuccess)
    return PSFM_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return PSFM_ERR_CUDA;
  out->n_regions = p.nreg;
  out->max_cand = p.max_cand;
  if (h.error) return h.error;
  out->b0 = sol[0];
  out->d0 = sol[1];
  if (out->coeff) {
    if (out->n_coeff < p.ncoef) return PSFM_ERR_BAD_ARG;
    for (int i = 0; i < p.ncoef; ++i) out->coeff[i] = sol[2 + i];
  }
  if (out->cand || out->cand_status || out->chi2) {
    if (out->cand_capacity < (int32_t)nc) return PSFM_ERR_BAD_ARG;
    for (size_t i = 0; i < nc; ++i) {
      if (out->cand) {
        out->cand[i].x = cand[2 * i];
        out->cand[i].y = cand[2 * i + 1];
      }
      if (out->cand_status) out->cand_status[i] = stat[i];
      if (out->chi2) out->chi2[i] = chi2[i];
    }
  }
  out->n_used = h.n_active;
  out->n_iter = h.iter;
  out->r_bad = h.r_bad;
  out->chi2_mean = h.chi2_mean;
  out->chi2_rms = h.chi2_rms;
  {
    const uint32_t k = h.median_key;
    const uint32_t u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
    float f;
    std::memcpy(&f, &u, sizeof(f));
    out->median = p.n_stamps > 0 ? 0.f : f;
  }
  return PSFM_OK;
}

}  // namespace psfm
