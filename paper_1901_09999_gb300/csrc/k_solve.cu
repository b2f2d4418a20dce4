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
#include <algorithm>
#include <cstring>
#include <type_traits>
#include <vector>

#include "dfloat.cuh"
#include "psfm_internal.h"
#include "solve.h"
#include "stamp.h"

namespace psfm {

cudaError_t launch_gram_tc(int mode, const StampParams& sp, int nreg, cudaStream_t s);
cudaError_t launch_gram_oz(const StampParams& sp, int nreg, int nsplit, cudaStream_t s);
size_t design_df_smem(int foot, int sw, int h, int dmax);
cudaError_t launch_design_df(int h, dim3 grid, size_t smem, const StampParams& sp,
                             cudaStream_t s);

namespace {

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
  if (block_skip(P.st)) return;
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

// grid (nreg, kGramSplit), 384 threads, two blocks per SM: weighted Gram of the augmented
// block in double-float.  Block (r, j) takes the 64-pixel chunks j, j + kGramSplit, ... of
// stamp r.  Each thread owns a 4 x 4 block of the Gram and one of `nsl` interleaved pixel
// slices of every chunk (nsl a power of two, the slices of a block in adjacent lanes); its 16
// double-float sums stay in registers over all chunks, the slices are combined by shuffles,
// and each block writes its FP64 partial Gram.  The basis columns are staged as the zero-sum
// design columns psi_k C_k - s_k X (X the image the term convolves) per pixel, so the
// cancellation of the delta term happens once per pixel in double-float (as in the definition
// of Eq. 4) and not between large Gram entries; the weighted columns w * A are formed once per
// chunk in shared memory.  The last block of a stamp to finish (counted with an atomic) adds
// the partials in split order, so the result does not depend on which block finishes last.
constexpr int kGramChunk = 64;
// row stride of the staged columns: one float of padding puts the rows that the threads of a
// warp read (different columns, same pixel) in different shared-memory banks
constexpr int kGramLd = kGramChunk + 1;
constexpr int kGramThreads = 384;
constexpr int kGramBatch = 4;

__host__ __device__ constexpr int gram_slices(int npair) {
  int nsl = 1;
  while (nsl < 16 && 2 * nsl * npair <= kGramThreads) nsl *= 2;
  return nsl;
}

__global__ void __launch_bounds__(kGramThreads, 2) k_stamp_gram_df(StampParams P) {
  extern __shared__ double shd[];
  __shared__ int s_last;
  const int r = blockIdx.x, split = blockIdx.y, tid = threadIdx.x;
  if (block_skip(P.st)) return;
  int cx, cy;
  if (!region_active(P.ptr, P.cand, r, P.max_cand, &cx, &cy)) return;
  if (P.have[r] == P.ptr[r]) return;
  // design columns: N_d (the basis applied to R, then to I2 with the dual kernel), then R, 1, I2
  const int Nc = P.Nc, Nb = P.Nd;
  const int nblk = (Nc + 3) / 4, npair = nblk * (nblk + 1) / 2;
  const int nsl = gram_slices(npair);
  const int ncr = nblk * 4;  // padded column count
  float* Ah = reinterpret_cast<float*>(shd);  // [ncr][chunk]
  float* Al = Ah + ncr * kGramLd;
  float* Bh = Al + ncr * kGramLd;  // w * A
  float* Bl = Bh + ncr * kGramLd;
  // weights of every pixel this block takes, all computed up front: [chunk t][64]
  const int nchunk = (P.P + kGramChunk - 1) / kGramChunk;
  const int nsplit = kGramSplit;  // gridDim.y
  const int nch = (nchunk - split + nsplit - 1) / nsplit;
  float* wh = Bl + ncr * kGramLd;
  float* wl = wh + nch * kGramChunk;
  // and the pixel values of the images the zero-sum delta terms use (masked R; I2 for the
  // dual kernel's columns), [chunk t][64] each; the masks do not gate the pixel loads, so all
  // of a pixel's loads are in flight together
  float* xr = wl + nch * kGramChunk;
  float* xi = xr + nch * kGramChunk;
  for (int i = tid; i < nch * kGramChunk; i += kGramThreads) {
    const int t = i / kGramChunk;
    const int pix = (split + t * nsplit) * kGramChunk + (i - t * kGramChunk);
    df wv = {0.f, 0.f};
    float vr = 0.f, vi = 0.f;
    if (pix < P.P) {
      const int py = pix / P.sw, px = pix - py * P.sw;
      const int gx = cx - P.s + px, gy = cy - P.s + py;
      if (gx >= 0 && gx < P.g.W && gy >= 0 && gy < P.g.H) {
        const int64_t o = (int64_t)gy * P.g.pitch + gx;
        const uint16_t m1 = P.m1[o], m2 = P.m2[o];
        const float a = P.i1[o], b = P.i2[o], v1 = P.v1[o], v2 = P.v2[o];
        vr = (m1 & P.badmask) ? 0.f : a;
        vi = b;
        if (!((m1 | m2) & P.badmask)) {
          const float vv = v1 + v2;
          const double wd = 1.0 / ((double)v1 + (double)v2);
          if (!isfinite(a) || !isfinite(b) || !isfinite(vv) || !isfinite(wd))
            raise_error(P.st, PSFM_ERR_NONFINITE);
          wv = df_split(wd);
        }
      }
    }
    wh[i] = wv.hi;
    wl[i] = wv.lo;
    xr[i] = vr;
    xi[i] = vi;
  }
  const float2* Cr = reinterpret_cast<const float2*>(P.C) + (int64_t)r * Nb * P.P;
  double* Gp = P.Gpart + ((int64_t)r * kGramSplit + split) * Nc * Nc;
  // psi_k and s_k of every design column as double-floats
  float* psh = xi + nch * kGramChunk;
  float* psl = psh + Nb;
  float* skh = psl + Nb;
  float* skl = skh + Nb;
  const int nbk = P.b.Nb;
  for (int c = tid; c < Nb; c += kGramThreads) {
    const int k = c < nbk ? c : c - nbk;
    const df a = df_split(P.psi[k]), b = df_split(P.sk[k]);
    psh[c] = a.hi;
    psl[c] = a.lo;
    skh[c] = b.hi;
    skl[c] = b.lo;
  }
  const int nass = npair * nsl, rounds = (nass + kGramThreads - 1) / kGramThreads;
  for (int rd = 0; rd < rounds; ++rd) {
    const int pp = rd * kGramThreads + tid;
    const bool act = pp < nass;
    const int pr = act ? pp / nsl : 0, sl = pp - (pp / nsl) * nsl;
    int bi = 0, rem = pr;
    while (rem >= nblk - bi) {
      rem -= nblk - bi;
      ++bi;
    }
    const int bj = bi + rem;
    df s[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) s[e] = df{0.f, 0.f};
    for (int t = 0; t < nch; ++t) {
      const int base = (split + t * nsplit) * kGramChunk;
      const float* wht = wh + t * kGramChunk;
      const float* wlt = wl + t * kGramChunk;
      __syncthreads();
      const float* xrt = xr + t * kGramChunk;
      const float* xit = xi + t * kGramChunk;
      // the design values of kGramBatch elements per thread are loaded before any is used,
      // so that their global loads are in flight together
      for (int i0 = tid; i0 < ncr * kGramChunk; i0 += kGramBatch * kGramThreads) {
        float2 cv[kGramBatch];
#pragma unroll
        for (int e = 0; e < kGramBatch; ++e) {
          const int i = i0 + e * kGramThreads;
          const int c = i / kGramChunk, pix = base + (i - c * kGramChunk);
          cv[e] = make_float2(0.f, 0.f);
          if (i < ncr * kGramChunk && c < Nb && pix < P.P) cv[e] = Cr[(int64_t)c * P.P + pix];
        }
#pragma unroll
        for (int e = 0; e < kGramBatch; ++e) {
          const int i = i0 + e * kGramThreads;
          if (i >= ncr * kGramChunk) break;
          const int c = i / kGramChunk, j = i - c * kGramChunk, pix = base + j;
          df v = {0.f, 0.f};
          if (pix < P.P) {
            if (c < Nb) {
              v = df_mul(df{psh[c], psl[c]}, df{cv[e].x, cv[e].y});
              if (skh[c] != 0.f) {
                const float x = c < nbk ? xrt[j] : xit[j];
                v = df_add(v, df_neg(df_mul(df{skh[c], skl[c]}, df{x, 0.f})));
              }
            } else if (c < Nc) {
              v.hi = c == Nb ? xrt[j] : (c == Nb + 1 ? 1.f : xit[j]);
            }
          }
          const df b = df_mul(df{wht[j], wlt[j]}, v);
          Ah[c * kGramLd + j] = v.hi;
          Al[c * kGramLd + j] = v.lo;
          Bh[c * kGramLd + j] = b.hi;
          Bl[c * kGramLd + j] = b.lo;
        }
      }
      __syncthreads();
      if (act) {
        const int jmax = min(kGramChunk, P.P - base);  // the last chunk of a stamp is ragged
        for (int j = sl; j < jmax; j += nsl) {
          df a[4], b[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            a[e] = df{Ah[(bi * 4 + e) * kGramLd + j], Al[(bi * 4 + e) * kGramLd + j]};
            b[e] = df{Bh[(bj * 4 + e) * kGramLd + j], Bl[(bj * 4 + e) * kGramLd + j]};
          }
#pragma unroll
          for (int e = 0; e < 4; ++e)
#pragma unroll
            for (int f = 0; f < 4; ++f) df_fma(s[e * 4 + f], a[e], b[f]);
        }
      }
    }
    // combine the slices (adjacent lanes), in a fixed order
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      df v = df_norm(s[e]);
      for (int o = 1; o < nsl; o <<= 1) {
        const df u = {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
        v = (sl & o) ? df_add(u, v) : df_add(v, u);
      }
      const int i = bi * 4 + e / 4, j = bj * 4 + e % 4;
      if (act && sl == 0 && i < Nc && j < Nc) {
        const double g = (double)v.hi + (double)v.lo;
        Gp[i * Nc + j] = g;
        Gp[j * Nc + i] = g;
      }
    }
  }
  // publish the partial, then let the last block of this stamp combine them
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = atomicAdd(&P.gram_count[r], 1) == nsplit - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // the Gram of the zero-sum columns is the transformed Gram the system is assembled from
  double* Gr = P.Gt + (int64_t)r * Nc * Nc;
  const double* Gp0 = P.Gpart + (int64_t)r * kGramSplit * Nc * Nc;
  for (int q = tid; q < Nc * Nc; q += kGramThreads) {
    double v = 0.0;
    for (int k = 0; k < nsplit; ++k) v += __ldcg(Gp0 + (int64_t)k * Nc * Nc + q);
    Gr[q] = v;
  }
  __syncthreads();
  if (tid == 0) {
    P.gram_count[r] = 0;
    P.have[r] = P.ptr[r];
    P.fresh[r] = 1;
  }
}

// grid (nreg): weighted Gram of the augmented design block of one stamp (zero-sum basis
// columns psi_k C_k - s_k R formed per pixel, then R, 1, I2); products in T, sums over 32-pixel
// chunks in T, chunk sums accumulated in FP64.
template <typename T>
__global__ void __launch_bounds__(256) k_stamp_gram(StampParams P) {
  extern __shared__ double shd[];
  const int r = blockIdx.x, tid = threadIdx.x;
  if (block_skip(P.st)) return;
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
        const T xr = (on && !(P.m1[o] & P.badmask)) ? (T)P.i1[o] : (T)0;
        if (c < Nb) {
          // zero-sum design column psi_k C_k - s_k R, formed per pixel
          v = (T)P.psi[c] * Cr[(int64_t)c * P.P + pix];
          if (P.sk[c] != 0.0) v -= (T)P.sk[c] * xr;
        } else if (on) {
          if (c == Nb) v = xr;
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
  // the Gram of the zero-sum columns is the transformed Gram the system is assembled from
  double* Gr = P.Gt + (int64_t)r * Nc * Nc;
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
  if (tid == 0) {
    P.have[r] = P.ptr[r];
    P.fresh[r] = 1;
  }
}

struct SysParams {
  BasisDev b;
  ImgGeom g;
  int nreg, max_cand, Nc, Nsys, joint;
  int Nd;              // design columns (N_b, or 2 N_b with the dual kernel)
  double lambda;       // dual kernel: penalty scale; 0 without penalty
  const double* pen;   // [N_b] p_k
  double* pdiag;       // [Nsys] Phi p_i added to the diagonal (dual kernel), else zeros
  const int32_t* cand;
  const int32_t* ptr;
  const double* Gt;
  const double* footsum;
  double* gv;      // [nreg][Ns] spatial factors at the stamp centre, 0 if inactive
  double* gp;      // [nreg][(Ns+1)^2] products g_s g_s' (index Ns stands for 1), 0 if inactive
  const int32_t* fresh;    // [nreg] stamps whose Gram joins M in this iteration
  const int32_t* removed;  // [nreg] stamps rejected in this iteration (leave M)
  double* dsol;
  double* M;
  float* Lh;  // df working copy of M for the factorisation
  float* Ll;
  double* v;
  DevState* st;
};

// Fixed-order block sum (deterministic for a given launch shape): warp trees, then a tree
// over the warp partials (FP64 chains are long on this GPU, so no sequential loop).
__device__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    double t = lane < nw ? sh[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) sh[32] = t;
  }
  __syncthreads();
  return sh[32];
}

// K block sums at once, in a fixed order for a given launch shape: warp trees, then warp 0
// adds the warp partials; one pair of barriers for all K (FP64 is slow on this GPU, so few
// FP64 operations and few barriers).  sh: at least 33 * K doubles.  Every thread gets the sums.
template <int K>
__device__ void block_sums(double (&v)[K], double* sh) {
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) sh[k * 32 + w] = v[k];
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double t = lane < nw ? sh[k * 32 + lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) sh[32 * K + k] = t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = sh[32 * K + k];
}

// Active count, spatial factors, and (SEPARATE) b0, d0 from the unweighted regression of
// footprint sums (Sec. 3.2).  One CTA of 1024 threads.
__global__ void __launch_bounds__(1024) k_norm(SysParams P) {
  __shared__ double sh[33 * 6];
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
  __syncthreads();
  // pairwise products, one per thread (index Ns stands for 1; zero for an inactive region)
  {
    const int N1 = P.b.Ns + 1;
    for (int q = threadIdx.x; q < P.nreg * N1 * N1; q += blockDim.x) {
      const int r = q / (N1 * N1), e = q - r * N1 * N1, a = e / N1, c = e - a * N1;
      int cx, cy;
      double g = 0.0;
      if (region_active(P.ptr, P.cand, r, P.max_cand, &cx, &cy)) {
        const double* gr = P.gv + (int64_t)r * P.b.Ns;
        g = (a < P.b.Ns ? gr[a] : 1.0) * (c < P.b.Ns ? gr[c] : 1.0);
      }
      P.gp[q] = g;
    }
  }
  double sums[6] = {n, s11, s12, s22, t1, t2};
  block_sums<6>(sums, sh);
  n = sums[0];
  s11 = sums[1];
  s12 = sums[2];
  s22 = sums[3];
  t1 = sums[4];
  t2 = sums[5];
  if (threadIdx.x != 0) return;
  P.st->n_active = (int)n;
  P.st->chol_fail = 0;
  P.st->refined = 0;
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
      *a = P.Nd;  // R
      *s = -1;
      return;
    }
    if (u == P.Nsys - 1) {
      *a = P.Nd + 1;  // 1
      *s = -1;
      return;
    }
    u -= 1;
  }
  *a = u / P.b.Ns;
  *s = u - *a * P.b.Ns;
}

// M (Eq. 5-6 with g_i at the stamp centres): M_{(c,s),(c',s')} = sum_stamps g_s g_s'
// Gt[c][c'] with the transformed stamp Grams.  M is kept across the rejection iterations and
// updated by the stamps that change (Sec. 3.5: per-stamp matrices need not be recalculated):
// mode 0 adds the stamps whose Gram was computed in this iteration and refreshes the
// double-float copy for the factorisation; mode 1 subtracts the stamps just rejected.  One
// thread per entry of the upper triangle (mirrored); spatial products staged in shared memory.
__global__ void __launch_bounds__(256) k_system_delta(SysParams P, int mode, int chunk) {
  extern __shared__ double gsh[];  // [chunk][(Ns+1)^2]
  if (P.st->error || P.st->done) return;
  const int Ns = P.b.Ns, N1 = Ns + 1, Nc = P.Nc, N = P.Nsys;
  const int32_t* flag = mode == 0 ? P.fresh : P.removed;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  // one thread per entry of the upper triangle (uj >= ui), row by row: row i starts at
  // i N - i (i - 1) / 2
  int ui = 0, uj = 0, ai = 0, aj = 0, si = -1, sj = -1;
  const bool mine = t < (int64_t)N * (N + 1) / 2;
  if (mine) {
    const float b = 2.f * N + 1.f;
    int i = (int)((b - sqrtf(fmaxf(b * b - 8.f * (float)t, 0.f))) * 0.5f);
    i = max(0, min(N - 1, i));
    auto start = [&](int k) { return (int64_t)k * N - (int64_t)k * (k - 1) / 2; };
    while (i > 0 && start(i) > t) --i;
    while (i + 1 < N && start(i + 1) <= t) ++i;
    ui = i;
    uj = ui + (int)(t - start(i));
    unknown_col(P, ui, &ai, &si);
    unknown_col(P, uj, &aj, &sj);
  }
  const int pidx = (si < 0 ? Ns : si) * N1 + (sj < 0 ? Ns : sj);
  double acc = 0.0;
  const int64_t gij = (int64_t)ai * Nc + aj;
  int* list = reinterpret_cast<int*>(gsh + (size_t)chunk * N1 * N1);  // [chunk]
  __shared__ int s_nf;
  for (int r0 = 0; r0 < P.nreg; r0 += chunk) {
    const int nr = min(chunk, P.nreg - r0);
    __syncthreads();
    // warp 0 lists the flagged regions of this chunk in ascending order
    if (threadIdx.x < 32) {
      int base = 0;
      for (int j0 = 0; j0 < nr; j0 += 32) {
        const int j = j0 + threadIdx.x;
        const bool f = j < nr && flag[r0 + j];
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        if (f) list[base + __popc(bal & ((1u << threadIdx.x) - 1u))] = j;
        base += __popc(bal);
      }
      if (threadIdx.x == 0) s_nf = base;
    }
    __syncthreads();
    const int nf = s_nf;
    for (int q = threadIdx.x; q < nf * N1 * N1; q += blockDim.x) {
      const int f = q / (N1 * N1);
      gsh[q] = P.gp[(int64_t)(r0 + list[f]) * N1 * N1 + (q - f * N1 * N1)];
    }
    __syncthreads();
    if (mine) {
      // eight independent partial sums keep eight Gram loads in flight (fixed order)
      const double* Gr = P.Gt + (int64_t)r0 * Nc * Nc + gij;
      const double* gq = gsh + pidx;
      const int64_t gs = (int64_t)Nc * Nc;
      const int ps = N1 * N1;
      double a[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) a[k] = 0.0;
      int f = 0;
      for (; f + 7 < nf; f += 8) {
        double g[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) g[k] = Gr[list[f + k] * gs];
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = fma(gq[(f + k) * ps], g[k], a[k]);
      }
      for (; f < nf; ++f) a[0] = fma(gq[f * ps], Gr[list[f] * gs], a[0]);
      acc += ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
    }
  }
  if (!mine) return;
  const int64_t a = (int64_t)ui * N + uj, b = (int64_t)uj * N + ui;
  const double m = mode == 0 ? P.M[a] + acc : P.M[a] - acc;
  P.M[a] = m;
  P.M[b] = m;
  if (mode == 0) {
    const df d = df_split(m);
    P.Lh[a] = d.hi;
    P.Ll[a] = d.lo;
    P.Lh[b] = d.hi;
    P.Ll[b] = d.lo;
  }
}

// Right-hand side v (Eq. 6): target I2 (JOINT) or I2 - b0 R - d0 (SEPARATE), all stamps.
// One warp per unknown, lanes over the stamps, fixed-order warp reduction.
__global__ void __launch_bounds__(256) k_rhs(SysParams P) {
  if (P.st->error || P.st->done) return;
  const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (t >= P.Nsys) return;
  const int Ns = P.b.Ns, N1 = Ns + 1, Nc = P.Nc;
  int av = 0, sv = -1;
  unknown_col(P, t, &av, &sv);
  const int colR = P.Nd, col1 = P.Nd + 1, colI = P.Nd + 2;
  const double b0 = P.dsol[0], d0 = P.dsol[1];
  double accv = 0.0;
  for (int r = lane; r < P.nreg; r += 32) {
    const double gg = P.gp[(int64_t)r * N1 * N1 + (sv < 0 ? Ns : sv) * N1 + Ns];
    if (gg == 0.0) continue;
    const double* Gr = P.Gt + (int64_t)r * Nc * Nc;
    double e = Gr[av * Nc + colI];
    if (!P.joint) e -= b0 * Gr[av * Nc + colR] + d0 * Gr[av * Nc + col1];
    accv = fma(gg, e, accv);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) accv += __shfl_xor_sync(0xffffffffu, accv, o);
  if (lane == 0) P.v[t] = accv;
}

// Dual kernel (Sec. 2): Phi = lambda * sum M_ii / sum p_i over the kernel unknowns, and
// Phi p_i added to the diagonal of the double-float working copy of M (M itself stays the
// plain normal matrix, updated incrementally); the FP64 residuals of the refinement add
// pdiag * x.  One CTA of 1024 threads.
__global__ void __launch_bounds__(1024) k_penalty(SysParams P) {
  __shared__ double sh[33];
  if (P.st->error || P.st->done) return;
  const int N = P.Nsys, nbk = P.b.Nb;
  double tm = 0.0, tp = 0.0;
  for (int u = threadIdx.x; u < N; u += blockDim.x) {
    int a, sidx;
    unknown_col(P, u, &a, &sidx);
    if (sidx < 0) continue;  // b0, d0 of the joint fit
    tm += P.M[(int64_t)u * N + u];
    tp += P.pen[a < nbk ? a : a - nbk];
  }
  tm = block_sum(tm, sh);
  tp = block_sum(tp, sh);
  const double phi = tp > 0.0 ? P.lambda * tm / tp : 0.0;
  for (int u = threadIdx.x; u < N; u += blockDim.x) {
    int a, sidx;
    unknown_col(P, u, &a, &sidx);
    const double pd = sidx < 0 ? 0.0 : phi * P.pen[a < nbk ? a : a - nbk];
    P.pdiag[u] = pd;
    const int64_t o = (int64_t)u * N + u;
    const df d = df_split(P.M[o] + pd);
    P.Lh[o] = d.hi;
    P.Ll[o] = d.lo;
  }
}

constexpr int kNB = 32;

// ---- Cholesky of the N x N normal equations in double-float (FP32 pairs on the FP32 pipes;
// FP64 chains on this GPU are slow), right-looking by 32-column panels spread over the GPU,
// followed by iterative refinement with FP64 residuals of the exact FP64 matrix, which brings
// the solution to FP64 accuracy (the factor only preconditions the correction).


// Panel pipeline: one launch per 32-column panel.  Launch kb applies panel kb to the whole
// trailing matrix and, in its block 0, finishes the next diagonal block (its update by panel
// kb, factor and inverse), so the sequential chain per panel is one block's work inside one
// launch.  The working matrix A (Lh/Ll, lower triangle) is only ever read in the panel's own
// column block and written beyond it; the factor goes to F (Fh/Fl), so no block reads a value
// another block of the same launch writes.
// Panel rows L_ik = A_ik inv(L_kk)^T are recomputed by every block that needs them from the
// panel's block inverse (a few hundred double-float FMAs per thread) instead of a launch.

constexpr int kCholThreads = 512;
constexpr int kTileLd = kNB + 1;

__device__ __forceinline__ float2 f2(df a) { return make_float2(a.hi, a.lo); }
__device__ __forceinline__ df dfv(float2 a) { return df{a.x, a.y}; }

// out[y][c] = sum_t a[y][t] inv[c][t] for y < rows (inv lower triangular with exact zeros
// above the diagonal, so every dot product runs over all 32 terms without predicates).
__device__ __forceinline__ void panel_rows(const float2 (*a)[kTileLd], const float2 (*inv)[kTileLd],
                                           float2 (*out)[kTileLd], int rows) {
  const int c = threadIdx.x & 31;
  for (int y = threadIdx.x >> 5; y < rows; y += kCholThreads / 32) {
    df s0 = {0.f, 0.f}, s1 = {0.f, 0.f};
#pragma unroll 8
    for (int t = 0; t < kNB; t += 2) {
      df_fma(s0, dfv(a[y][t]), dfv(inv[c][t]));
      df_fma(s1, dfv(a[y][t + 1]), dfv(inv[c][t + 1]));
    }
    out[y][c] = f2(df_add(df_norm(s0), df_norm(s1)));
  }
}

// 1 / sqrt(d) for the pivots: the FP32 estimate r0 and one Newton step r0 + r0 (1 - d r0^2) / 2,
// with the residual 1 - d r0^2 formed from exact FMA products (1 - p is exact for p near 1).
__device__ __forceinline__ df df_rsqrt_pivot(df d) {
  const float r0 = rsqrtf(d.hi);
  const float a = __fmul_rn(d.hi, r0);
  const float a_err = __fmaf_rn(d.hi, r0, -a);
  const float p = __fmul_rn(a, r0);
  const float p_err = __fmaf_rn(a, r0, -p);
  const float tail = __fmaf_rn(__fmaf_rn(d.lo, r0, a_err), r0, p_err);
  const float e = __fsub_rn(__fsub_rn(1.0f, p), tail);
  const float corr = __fmul_rn(__fmul_rn(0.5f, r0), e);
  const float s = __fadd_rn(r0, corr);
  return df{s, __fsub_rn(corr, __fsub_rn(s, r0))};
}

// Numerical singularity (reading of "regular matrix methods", Eq. 5-6): a pivot whose size
// relative to its row's original diagonal, |d_j| / (M_jj + penalty_j), is at most
// kPivotSingular leaves column j a linear combination of the earlier columns to within the
// working precision of the factorisation (double-float, ~2^-48 per operation, a few 1e-13 over
// a few hundred columns), so the normal equations are singular (PSFM_ERR_SINGULAR).  A pivot
// below -kPivotSingular times its diagonal means the matrix is indefinite by rounding: the LU
// fallback takes it.  Full-rank systems have relative pivots of at least 1 / cond of the
// unit-diagonal matrix (1e-8 for the full-chip basis).
constexpr float kPivotSingular = 1e-11f;

// Loads the original diagonal M_jj + penalty_j of rows r0 .. r0 + 31 (1 past n) into dg.
__device__ __forceinline__ void load_ref_diag(const double* M, const double* pdiag, int n,
                                              int r0, float* dg) {
  if (threadIdx.x < kNB) {
    const int r = r0 + threadIdx.x;
    dg[threadIdx.x] = r < n ? (float)(M[(int64_t)r * n + r] + pdiag[r]) : 1.f;
  }
}

// Cholesky factor and inverse of the 32 x 32 block T (lower triangle; rows and columns past
// the block's size padded with the identity).  Factor: one barrier per column; thread = (row
// i, column group g) updating columns g and g + 16; column j is scaled on the fly by the pivot
// 1 / sqrt(T_jj), which the thread that completes T_jj (in step j - 1) computes at once, so the
// sequential chain per column is one update plus one reciprocal square root.  Inverse: from
// the diagonal 1 / L_ii up by doubling, [A 0; B C]^-1 = [A^-1 0; -C^-1 B A^-1 C^-1], two
// products per level, five levels.  Lo receives L, Xf inv(L) (zeros above the diagonal), W is
// scratch.  dg holds the rows' original diagonals.  Returns (uniformly) 0, or 1 when a pivot is
// negative beyond the singularity band or not finite (indefinite: LU fallback), or 2 when a
// pivot lies within the band (singular).
__device__ int tile_factor_inverse(float2 (*T)[kTileLd], float2 (*Lo)[kTileLd],
                                   float2 (*W)[kTileLd], float2 (*Xf)[kTileLd], float2* rp,
                                   const float* dg) {
  const int tid = threadIdx.x, i = tid >> 4, g = tid & 15;
  for (int q = tid; q < kNB * kNB; q += kCholThreads) {
    const int r = q >> 5, c = q & 31;
    Lo[r][c] = make_float2(0.f, 0.f);
    Xf[r][c] = make_float2(0.f, 0.f);
  }
  if (tid == 0) rp[0] = f2(df_rsqrt_pivot(dfv(T[0][0])));
  __syncthreads();
  for (int j = 0; j < kNB; ++j) {
    const df d = dfv(T[j][j]);  // the same d for every thread
    if (!isfinite(d.hi)) return 1;
    if (fabsf(d.hi) <= kPivotSingular * dg[j]) return 2;
    if (!(d.hi > 0.f)) return 1;
    const df r = dfv(rp[j]);
    if (i >= j) {
      const df lij = i == j ? df_mul(d, r) : df_mul(dfv(T[i][j]), r);
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int c = g + 16 * q;
        if (c > j && c <= i) {
          df a = dfv(T[i][c]);
          df_fma(a, df_neg(lij), df_mul(dfv(T[c][j]), r));
          a = df_norm(a);
          T[i][c] = f2(a);
          if (c == i && i == j + 1) rp[i] = f2(df_rsqrt_pivot(a));
        }
      }
      if (g == 0) Lo[i][j] = f2(lij);
    }
    __syncthreads();
  }
  if (tid < kNB) Xf[tid][tid] = rp[tid];
  __syncthreads();
  for (int b = 1; b < kNB; b *= 2) {
    // W = B A^-1 for each pair of diagonal blocks of size b (A at p0, C at p0 + b)
    const int nout = (kNB / (2 * b)) * b * b;
    int p0 = 0, rr = 0, cc = 0;
    if (tid < nout) {
      const int pair = tid / (b * b), rem = tid - pair * b * b;
      p0 = pair * 2 * b;
      rr = rem / b;
      cc = rem - rr * b;
      df s = {0.f, 0.f};
      for (int t = cc; t < b; ++t)
        df_fma(s, dfv(Lo[p0 + b + rr][p0 + t]), dfv(Xf[p0 + t][p0 + cc]));
      W[p0 + b + rr][p0 + cc] = f2(df_norm(s));
    }
    __syncthreads();
    if (tid < nout) {
      df s = {0.f, 0.f};
      for (int t = 0; t <= rr; ++t)
        df_fma(s, dfv(Xf[p0 + b + rr][p0 + b + t]), dfv(W[p0 + b + t][p0 + cc]));
      Xf[p0 + b + rr][p0 + cc] = f2(df_neg(df_norm(s)));
    }
    __syncthreads();
  }
  return 0;
}

// The first diagonal block.
__global__ void __launch_bounds__(kCholThreads) k_chol_first(int n, const float* Lh,
                                                             const float* Ll, float* Fh, float* Fl,
                                                             float2* Linv_all, const double* M,
                                                             const double* pdiag, DevState* st) {
  __shared__ float2 S[4][kNB][kTileLd];
  __shared__ float2 rp[kNB];
  __shared__ float dg[kNB];
  if (st->error || st->done || st->chol_fail) return;
  load_ref_diag(M, pdiag, n, 0, dg);
  const int m = min(kNB, n);
  for (int q = threadIdx.x; q < kNB * kNB; q += kCholThreads) {
    const int r = q >> 5, c = q & 31;
    float2 v = make_float2(r == c ? 1.f : 0.f, 0.f);
    if (r < m && c < m) v = c <= r ? make_float2(Lh[(int64_t)r * n + c], Ll[(int64_t)r * n + c])
                                   : make_float2(0.f, 0.f);
    S[0][r][c] = v;
  }
  __syncthreads();
  const int f = tile_factor_inverse(S[0], S[1], S[2], S[3], rp, dg);
  if (f) {
    if (threadIdx.x == 0) {
      if (f == 2) raise_error(st, PSFM_ERR_SINGULAR);
      else st->chol_fail = 1;
    }
    return;
  }
  for (int q = threadIdx.x; q < kNB * kNB; q += kCholThreads) {
    const int r = q >> 5, c = q & 31;
    Linv_all[q] = S[3][r][c];
    if (r < m && c <= r) {
      Fh[(int64_t)r * n + c] = S[1][r][c].x;
      Fl[(int64_t)r * n + c] = S[1][r][c].y;
    }
  }
}

// Launch kb (panel kb full, kb + 1 < number of panels).  Block 0: rows of block kb + 1 of the
// panel, their update of diagonal block kb + 1, its factor and inverse.  Blocks 1..: one 16 x 16
// tile (ti, tj) of the trailing lower triangle past block kb + 1's own 32 x 32 block; diagonal
// tiles also store their 16 panel rows into F.
__global__ void __launch_bounds__(kCholThreads) k_chol_panel(int n, int kb, float* Lh, float* Ll,
                                                             float* Fh, float* Fl,
                                                             float2* Linv_all, const double* M,
                                                             const double* pdiag, DevState* st) {
  __shared__ float2 S[5][kNB][kTileLd];
  __shared__ float2 rp[kNB];
  __shared__ float dg[kNB];
  if (st->error || st->done || st->chol_fail) return;
  const int tid = threadIdx.x;
  const int k0 = kb * kNB, base = k0 + kNB;
  const float2* Linv = Linv_all + (int64_t)kb * kNB * kNB;
  float2(*Li)[kTileLd] = S[0];
  for (int q = tid; q < kNB * kNB; q += kCholThreads) Li[q >> 5][q & 31] = Linv[q];
  if (blockIdx.x == 0) {
    const int mb = min(kNB, n - base);
    load_ref_diag(M, pdiag, n, base, dg);
    float2(*Ar)[kTileLd] = S[4];
    float2(*Pn)[kTileLd] = S[1];
    float2(*T)[kTileLd] = S[2];
    for (int q = tid; q < kNB * kNB; q += kCholThreads) {
      const int r = q >> 5, c = q & 31;
      float2 a = make_float2(0.f, 0.f), tv = make_float2(r == c ? 1.f : 0.f, 0.f);
      if (r < mb) {
        const int64_t o = (int64_t)(base + r) * n;
        a = make_float2(Lh[o + k0 + c], Ll[o + k0 + c]);
        if (c < mb) tv = c <= r ? make_float2(Lh[o + base + c], Ll[o + base + c])
                                : make_float2(0.f, 0.f);
      }
      Ar[r][c] = a;
      T[r][c] = tv;
    }
    __syncthreads();
    panel_rows(Ar, Li, Pn, kNB);
    __syncthreads();
    // panel rows of block kb + 1 into F; T -= Pn Pn^T on the lower triangle
    for (int q = tid; q < kNB * kNB; q += kCholThreads) {
      const int r = q >> 5, c = q & 31;
      if (r < mb) {
        const int64_t o = (int64_t)(base + r) * n + k0 + c;
        Fh[o] = Pn[r][c].x;
        Fl[o] = Pn[r][c].y;
      }
    }
    {
      const int r = tid >> 4, cg = tid & 15;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int c = cg + 16 * q;
        if (c <= r && r < mb) {
          df s0 = {0.f, 0.f}, s1 = {0.f, 0.f};
#pragma unroll 8
          for (int t = 0; t < kNB; t += 2) {
            df_fma(s0, dfv(Pn[r][t]), dfv(Pn[c][t]));
            df_fma(s1, dfv(Pn[r][t + 1]), dfv(Pn[c][t + 1]));
          }
          T[r][c] = f2(df_add(dfv(T[r][c]), df_neg(df_add(df_norm(s0), df_norm(s1)))));
        }
      }
    }
    __syncthreads();
    // Li and Ar are free from here: Xf and W reuse them
    const int f = tile_factor_inverse(T, S[3], S[4], S[0], rp, dg);
    if (f) {
      if (tid == 0) {
        if (f == 2) raise_error(st, PSFM_ERR_SINGULAR);
        else st->chol_fail = 1;
      }
      return;
    }
    float2* Lnext = Linv_all + (int64_t)(kb + 1) * kNB * kNB;
    for (int q = tid; q < kNB * kNB; q += kCholThreads) {
      const int r = q >> 5, c = q & 31;
      Lnext[q] = S[0][r][c];
      if (r < mb && c <= r) {
        const int64_t o = (int64_t)(base + r) * n + base + c;
        Fh[o] = S[3][r][c].x;
        Fl[o] = S[3][r][c].y;
      }
    }
    return;
  }
  // trailing tile
  const int nt = (n - base + 15) / 16;
  int t = blockIdx.x - 1, ti = 0;
  while (t >= ti + 1) {
    t -= ti + 1;
    ++ti;
  }
  const int tj = t;
  if (ti >= nt || (ti < 2 && tj < 2)) return;  // the 32 x 32 diagonal block is block 0's
  const int r0 = base + ti * 16, c0 = base + tj * 16;
  const bool diag = ti == tj;
  float2(*Ar)[kTileLd] = S[1];  // rows 0..15: tile rows, 16..31: tile columns
  float2(*Pn)[kTileLd] = S[2];
  for (int q = tid; q < kNB * kNB; q += kCholThreads) {
    const int r = q >> 5, c = q & 31;
    const int row = r < 16 ? r0 + r : c0 + r - 16;
    float2 a = make_float2(0.f, 0.f);
    if (row < n && (r < 16 || !diag)) {
      const int64_t o = (int64_t)row * n + k0 + c;
      a = make_float2(Lh[o], Ll[o]);
    }
    Ar[r][c] = a;
  }
  __syncthreads();
  panel_rows(Ar, Li, Pn, diag ? 16 : kNB);
  __syncthreads();
  const int y = (tid >> 4) & 15, x = tid & 15;
  const int row = r0 + y, col = c0 + x;
  const int xc = diag ? x : 16 + x;  // the column's panel row in Pn
  if (tid < 256 && row < n && col < n && col <= row) {
    df s0 = {0.f, 0.f}, s1 = {0.f, 0.f};
#pragma unroll 8
    for (int c = 0; c < kNB; c += 2) {
      df_fma(s0, dfv(Pn[y][c]), dfv(Pn[xc][c]));
      df_fma(s1, dfv(Pn[y][c + 1]), dfv(Pn[xc][c + 1]));
    }
    const int64_t o = (int64_t)row * n + col;
    const df a = df_add(df{Lh[o], Ll[o]}, df_neg(df_add(df_norm(s0), df_norm(s1))));
    Lh[o] = a.hi;
    Ll[o] = a.lo;
  }
  if (diag) {
    for (int q = tid; q < 16 * kNB; q += kCholThreads) {
      const int r = q >> 5, c = q & 31;
      if (r0 + r < n) {
        const int64_t o = (int64_t)(r0 + r) * n + k0 + c;
        Fh[o] = Pn[r][c].x;
        Fl[o] = Pn[r][c].y;
      }
    }
  }
}

__device__ __forceinline__ df warp_sum_df(df v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const df u = {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
    v = df_add(v, u);
  }
  return v;
}

// L z = b then L^T y = z in double-float with the block inverses: per 32-row block a
// dot-product phase (warp per row over the solved part) and a 32 x 32 inverse application
// (warp per row), one CTA; x_out = x_in + y.  Each block's inverse entries are loaded before
// its dot products so that their latency overlaps; the backward phase combines the 32 warps'
// column partials with a shuffle tree.
//
// Refinement: the factor's relative error e0 (about cond(M) times the double-float rounding)
// is also the contraction of each refinement step, so after a step whose correction is y the
// error left is about (|y| / |x|) |y|.  mode 1 (the first step) records whether |y| <= 1e-5 |x|
// (error left below about 1e-10 |x|, under the FP64 residual's own floor for these systems);
// mode 2 (the second step) is skipped when it did.
constexpr int kSolveThreads = 1024;

__global__ void __launch_bounds__(kSolveThreads) k_chol_solve(int n, const float* Lh,
                                                              const float* Ll,
                                                              const float2* Linv_all,
                                                              const double* b, const double* x_in,
                                                              double* x_out, DevState* st,
                                                              int mode) {
  extern __shared__ float2 ys[];  // [n] + [32][33] + [32]
  float2* pw = ys + n;
  float2* zb = pw + 32 * 33;
  if (st->error || st->done || st->chol_fail || (mode == 2 && st->refined)) return;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  for (int i = tid; i < n; i += blockDim.x) ys[i] = f2(df_split(b[i]));
  __syncthreads();
  const int nb = (n + kNB - 1) / kNB;
  for (int bk = 0; bk < nb; ++bk) {
    const int k0 = bk * kNB, m = min(kNB, n - k0);
    const float2* Li = Linv_all + (int64_t)bk * kNB * kNB;
    const float2 li = (w < m && lane <= w) ? Li[w * kNB + lane] : make_float2(0.f, 0.f);
    df sacc = {0.f, 0.f};
    if (w < m)
      for (int c = lane; c < k0; c += 32) {
        const int64_t o = (int64_t)(k0 + w) * n + c;
        df_fma(sacc, df{Lh[o], Ll[o]}, dfv(ys[c]));
      }
    sacc = warp_sum_df(df_norm(sacc));
    if (w < m && lane == 0) zb[w] = f2(df_add(dfv(ys[k0 + w]), df_neg(sacc)));
    __syncthreads();
    if (w < m) {
      df t2 = {0.f, 0.f};
      if (lane < m) df_fma(t2, dfv(li), dfv(zb[lane]));
      t2 = warp_sum_df(df_norm(t2));
      if (lane == 0) ys[k0 + w] = f2(t2);
    }
    __syncthreads();
  }
  for (int bk = nb - 1; bk >= 0; --bk) {
    const int k0 = bk * kNB, m = min(kNB, n - k0);
    const float2* Li = Linv_all + (int64_t)bk * kNB * kNB;
    const float2 li = (w < m && lane >= w && lane < m) ? Li[lane * kNB + w]
                                                       : make_float2(0.f, 0.f);
    df sacc = {0.f, 0.f};
    if (lane < m)
      for (int i = k0 + m + w; i < n; i += 32) {
        const int64_t o = (int64_t)i * n + k0 + lane;
        df_fma(sacc, df{Lh[o], Ll[o]}, dfv(ys[i]));
      }
    pw[w * 33 + lane] = f2(df_norm(sacc));
    __syncthreads();
    if (w < m) {
      // column w: the partials of the 32 warps, one per lane, summed by a shuffle tree
      const df z = warp_sum_df(dfv(pw[lane * 33 + w]));
      if (lane == 0) zb[w] = f2(df_add(dfv(ys[k0 + w]), df_neg(z)));
    }
    __syncthreads();
    if (w < m) {
      // x_w = sum_j inv(L)[j][w] z_j, j >= w
      df t2 = {0.f, 0.f};
      if (lane < m) df_fma(t2, dfv(li), dfv(zb[lane]));
      t2 = warp_sum_df(df_norm(t2));
      if (lane == 0) ys[k0 + w] = f2(t2);
    }
    __syncthreads();
  }
  float ymax = 0.f, xmax = 0.f;
  for (int i = tid; i < n; i += blockDim.x) {
    const double y = (double)ys[i].x + (double)ys[i].y;
    const double x = x_in ? x_in[i] + y : y;
    x_out[i] = x;
    ymax = fmaxf(ymax, (float)fabs(y));
    xmax = fmaxf(xmax, (float)fabs(x));
  }
  if (mode != 1) return;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ymax = fmaxf(ymax, __shfl_xor_sync(0xffffffffu, ymax, o));
    xmax = fmaxf(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
  }
  __syncthreads();  // pw is reused
  if (lane == 0) pw[w] = make_float2(ymax, xmax);
  __syncthreads();
  if (w == 0) {
    float2 v = lane < (int)(blockDim.x >> 5) ? pw[lane] : make_float2(0.f, 0.f);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      v.x = fmaxf(v.x, __shfl_xor_sync(0xffffffffu, v.x, o));
      v.y = fmaxf(v.y, __shfl_xor_sync(0xffffffffu, v.y, o));
    }
    // NaN compares false: not converged
    if (lane == 0) st->refined = v.x <= 1e-5f * v.y ? 1 : 0;
  }
}

// r = b - M x in FP64 (one warp per row).
__global__ void __launch_bounds__(256) k_residual(int n, const double* M, const double* pdiag,
                                                  const double* b, const double* x, double* r,
                                                  const DevState* st, int mode) {
  if (st->error || st->done || st->chol_fail || (mode == 2 && st->refined)) return;
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (row >= n) return;
  double s = 0.0;
  for (int c = lane; c < n; c += 32) s = fma(M[(int64_t)row * n + c], x[c], s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) r[row] = b[row] - s - pdiag[row] * x[row];
}

// Scatter the solution vector into the device solution (b0, d0, a_{k,s}).
__global__ void k_store_solution(int n, int joint, const double* x, double* dsol,
                                 DevState* st) {
  if (st->error || st->done || st->chol_fail) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double v = x[i];
    if (!isfinite(v)) atomicCAS(&st->error, 0, PSFM_ERR_SINGULAR);
    if (joint) {
      if (i == 0) dsol[0] = v;
      else if (i == n - 1) dsol[1] = v;
      else dsol[2 + (i - 1)] = v;
    } else {
      dsol[2 + i] = v;
    }
  }
}

// Fallback when the Cholesky factorisation meets a non-positive pivot: LU with partial
// pivoting in FP64, one CTA (rare path).
__global__ void __launch_bounds__(1024) k_lu_solve(int N, int joint, const double* M,
                                                   const double* pdiag, const double* v,
                                                   double* L, double* y, int32_t* piv,
                                                   double* dsol, DevState* st) {
  const int tid = threadIdx.x, nt = blockDim.x;
  __shared__ int s_fail;
  if (st->error || st->done || !st->chol_fail) return;
  for (int64_t i = tid; i < (int64_t)N * N; i += nt)
    L[i] = M[i] + (i / N == i % N ? pdiag[i / N] : 0.0);
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

// sum_k a_k psi_k C_k(pix) at NPX stamp pixels at once (independent loads and accumulators;
// each pixel still sums its terms in order k = 0..Nb-1): FP64 products for FP32 / FP64 design
// blocks, double-float products on the FP32 pipes for double-float blocks.  pix < 0 marks an
// unused slot.
template <int NPX>
__device__ __forceinline__ void basis_model(const double* ak, const float2*, const float* C,
                                            int Nb, int P, const int* pix, double* m) {
  double acc[NPX];
#pragma unroll
  for (int j = 0; j < NPX; ++j) acc[j] = 0.0;
  for (int k = 0; k < Nb; ++k) {
    const double a = ak[k];
#pragma unroll
    for (int j = 0; j < NPX; ++j)
      if (pix[j] >= 0) acc[j] += a * (double)C[(int64_t)k * P + pix[j]];
  }
#pragma unroll
  for (int j = 0; j < NPX; ++j) m[j] = acc[j];
}
template <int NPX>
__device__ __forceinline__ void basis_model(const double* ak, const float2*, const double* C,
                                            int Nb, int P, const int* pix, double* m) {
  double acc[NPX];
#pragma unroll
  for (int j = 0; j < NPX; ++j) acc[j] = 0.0;
  for (int k = 0; k < Nb; ++k) {
    const double a = ak[k];
#pragma unroll
    for (int j = 0; j < NPX; ++j)
      if (pix[j] >= 0) acc[j] += a * C[(int64_t)k * P + pix[j]];
  }
#pragma unroll
  for (int j = 0; j < NPX; ++j) m[j] = acc[j];
}
template <int NPX>
__device__ __forceinline__ void basis_model(const double*, const float2* akf, const float2* C,
                                            int Nb, int P, const int* pix, double* m) {
  df acc[NPX];
#pragma unroll
  for (int j = 0; j < NPX; ++j) acc[j] = df{0.f, 0.f};
  // unrolled so that the loads of several terms are in flight together
#pragma unroll 8
  for (int k = 0; k < Nb; ++k) {
    const df a = {akf[k].x, akf[k].y};
    float2 c[NPX];
#pragma unroll
    for (int j = 0; j < NPX; ++j)
      c[j] = pix[j] >= 0 ? C[(int64_t)k * P + pix[j]] : make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < NPX; ++j) df_fma(acc[j], a, df{c[j].x, c[j].y});
  }
#pragma unroll
  for (int j = 0; j < NPX; ++j) m[j] = df_to_d(df_norm(acc[j]));
}

// The double-float model sum_k a_k psi_k C_k at NPX pixels, left as a double-float.
template <int NPX>
__device__ __forceinline__ void basis_model_df(const float2* akf, const float2* C, int Nb, int P,
                                               const int* pix, df* m) {
#pragma unroll
  for (int j = 0; j < NPX; ++j) m[j] = df{0.f, 0.f};
#pragma unroll 8
  for (int k = 0; k < Nb; ++k) {
    const df a = {akf[k].x, akf[k].y};
    float2 c[NPX];
#pragma unroll
    for (int j = 0; j < NPX; ++j)
      c[j] = pix[j] >= 0 ? C[(int64_t)k * P + pix[j]] : make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < NPX; ++j) df_fma(m[j], a, df{c[j].x, c[j].y});
  }
}

struct Chi2Params {
  StampParams sp;
  const double* gv;
  const double* dsol;
  double alpha;
  double* chi2;
  double* cand_chi2;
  double* part;    // [nreg][kChi2Split][2] per-block sums (chi^2 terms, pixels)
  int32_t* count;  // [nreg] blocks finished, reset by the block that combines them
};

// grid (nreg, kChi2Split): chi^2 of the active stamp with the current solution (FP64).  Each
// block takes one pixel range of the stamp, kChi2Px pixels per thread; the design-column loads
// of a pixel depend only on the stamp geometry (the masks are applied afterwards), so they are
// in flight together with the mask and image loads.  The last block of a stamp to finish
// (counted with an atomic) adds the block sums in range order, so the value does not depend on
// which block finishes last.
constexpr int kChi2Threads = 256;
constexpr int kChi2Px = 2;
template <typename T>
__global__ void __launch_bounds__(kChi2Threads, 4) k_chi2(Chi2Params Q) {
  const StampParams& P = Q.sp;
  extern __shared__ double ak[];  // [Nd]: a_k(stamp) psi_k (then c_k psi_k, dual kernel)
  __shared__ double red[2][kChi2Threads / 32];
  __shared__ double s_delta, s_delta2;
  __shared__ int s_last;
  const int r = blockIdx.x, split = blockIdx.y, tid = threadIdx.x;
  if (block_skip(P.st)) return;
  int cx, cy;
  if (!region_active(P.ptr, P.cand, r, P.max_cand, &cx, &cy)) return;
  const int Nb = P.b.Nb, Nd = P.Nd, Ns = P.b.Ns;
  const double* gr = Q.gv + (int64_t)r * Ns;
  // a_k at the stamp centre, times psi_k, and the delta parts of the zero-sum terms (on R for
  // the first N_b columns, on I2 for the dual kernel's), reduced over the block
  double dd = 0.0, dd2 = 0.0;
  for (int k = tid; k < Nd; k += kChi2Threads) {
    double a = 0.0;
    for (int s = 0; s < Ns; ++s) a += Q.dsol[2 + k * Ns + s] * gr[s];
    const int kb = k < Nb ? k : k - Nb;
    if (k < Nb)
      dd += a * P.sk[kb];
    else
      dd2 += a * P.sk[kb];
    ak[k] = a * P.psi[kb];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    dd += __shfl_xor_sync(0xffffffffu, dd, o);
    dd2 += __shfl_xor_sync(0xffffffffu, dd2, o);
  }
  if ((tid & 31) == 0) {
    red[0][tid >> 5] = dd;
    red[1][tid >> 5] = dd2;
  }
  __syncthreads();
  if (tid == 0) {
    double d = 0.0, d2 = 0.0;
    for (int i = 0; i < kChi2Threads / 32; ++i) {
      d += red[0][i];
      d2 += red[1][i];
    }
    s_delta = Q.dsol[0] - d;
    s_delta2 = -d2;
  }
  float2* akf = reinterpret_cast<float2*>(ak + Nd);  // the same split into FP32 pairs
  for (int k = tid; k < Nd; k += kChi2Threads) {
    const df d = df_split(ak[k]);
    akf[k] = make_float2(d.hi, d.lo);
  }
  __syncthreads();
  const double delta = s_delta, delta2 = s_delta2, d0 = Q.dsol[1];
  const df dl = df_split(delta), dl2 = df_split(delta2), dd0 = df_split(d0);
  const float alpha_f = (float)Q.alpha;
  const T* Cr = reinterpret_cast<const T*>(P.C) + (int64_t)r * Nd * P.P;
  double q = 0.0, n = 0.0;
  // double-float blocks: each thread's few terms (at most kChi2Px per pass over the stamp)
  // summed in FP32 and counted as an integer, FP64 from the warp sums on
  float qf = 0.f;
  int ni = 0;
  constexpr int kStride = kChi2Split * kChi2Threads * kChi2Px;
  for (int base = split * kChi2Threads * kChi2Px + tid; base < P.P; base += kStride) {
    int pix[kChi2Px];
    int64_t off[kChi2Px];
    uint16_t mk[kChi2Px];
#pragma unroll
    for (int j = 0; j < kChi2Px; ++j) {
      pix[j] = -1;
      off[j] = 0;
      const int pp = base + kChi2Threads * j;
      if (pp >= P.P) continue;
      const int py = pp / P.sw, px = pp - py * P.sw;
      const int gx = cx - P.s + px, gy = cy - P.s + py;
      if (gx < 0 || gx >= P.g.W || gy < 0 || gy >= P.g.H) continue;
      pix[j] = pp;
      off[j] = (int64_t)gy * P.g.pitch + gx;
    }
#pragma unroll
    for (int j = 0; j < kChi2Px; ++j)
      mk[j] = pix[j] >= 0 ? (uint16_t)((P.m1[off[j]] | P.m2[off[j]]) & P.badmask) : (uint16_t)1;
    if constexpr (std::is_same<T, float2>::value) {
      // double-float blocks: the model and the residual in double-float on the FP32 pipes
      // (the cancellation I2 - model is exact there), the residual's square over the softened
      // variance in FP32 (one rounding per term); the pixel loads go out with the design loads
      float R[kChi2Px], I2v[kChi2Px], Vs[kChi2Px];
#pragma unroll
      for (int j = 0; j < kChi2Px; ++j) {
        R[j] = 0.f;
        I2v[j] = 0.f;
        Vs[j] = 1.f;
        if (pix[j] >= 0) {
          R[j] = P.i1[off[j]];
          I2v[j] = P.i2[off[j]];
          Vs[j] = __fadd_rn(P.v1[off[j]], P.v2[off[j]]);
        }
      }
      df mdf[kChi2Px];
      basis_model_df<kChi2Px>(akf, Cr, Nd, P.P, pix, mdf);
#pragma unroll
      for (int j = 0; j < kChi2Px; ++j) {
        if (mk[j]) continue;
        df m = mdf[j];
        df_fma_f(m, R[j], dl);
        if (Nd > Nb) df_fma_f(m, I2v[j], dl2);
        m = df_add(m, dd0);
        const df res = df_add(df{I2v[j], 0.f}, df_neg(m));
        const float r = __fadd_rn(res.hi, res.lo);
        const float den = __fadd_rn(Vs[j], __fmul_rn(alpha_f, fabsf(I2v[j])));
        qf = __fadd_rn(qf, __fdiv_rn(__fmul_rn(r, r), den));
        ++ni;
      }
    } else {
      double mod[kChi2Px];
      basis_model<kChi2Px>(ak, akf, Cr, Nd, P.P, pix, mod);
#pragma unroll
      for (int j = 0; j < kChi2Px; ++j) {
        if (mk[j]) continue;
        const int64_t o = off[j];
        const double R = P.i1[o], I2 = P.i2[o];
        const double model = delta * R + delta2 * (Nd > Nb ? I2 : 0.0) + d0 + mod[j];
        const double res = I2 - model;
        const double den = ((double)P.v1[o] + (double)P.v2[o]) + Q.alpha * fabs(I2);
        q += res * res / den;
        n += 1.0;
      }
    }
  }
  q += (double)qf;
  n += (double)ni;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    q += __shfl_xor_sync(0xffffffffu, q, o);
    n += __shfl_xor_sync(0xffffffffu, n, o);
  }
  __syncthreads();  // red is reused
  if ((tid & 31) == 0) {
    red[0][tid >> 5] = q;
    red[1][tid >> 5] = n;
  }
  __syncthreads();
  if (tid == 0) {
    double a = 0, b = 0;
    for (int i = 0; i < kChi2Threads / 32; ++i) {
      a += red[0][i];
      b += red[1][i];
    }
    double* pr = Q.part + ((int64_t)r * kChi2Split + split) * 2;
    pr[0] = a;
    pr[1] = b;
    __threadfence();
    s_last = atomicAdd(&Q.count[r], 1) == kChi2Split - 1;
  }
  __syncthreads();
  if (!s_last || tid != 0) return;
  __threadfence();
  double a = 0, b = 0;
  for (int k = 0; k < kChi2Split; ++k) {
    a += __ldcg(Q.part + ((int64_t)r * kChi2Split + k) * 2);
    b += __ldcg(Q.part + ((int64_t)r * kChi2Split + k) * 2 + 1);
  }
  const double c = a / (b > 1.0 ? b : 1.0);
  Q.chi2[r] = c;
  Q.cand_chi2[(int64_t)r * P.max_cand + P.ptr[r]] = c;
  Q.count[r] = 0;
}

// Rejection decision of Sec. 3.3 and loop control; one CTA of 1024 threads.
__global__ void __launch_bounds__(1024) k_reject(int nreg, int max_cand, int max_iter,
                                                 double nsig, const int32_t* cand, int32_t* ptr,
                                                 int32_t* cand_stat, const double* chi2,
                                                 int32_t* fresh, int32_t* removed, DevState* st) {
  __shared__ double sh[33 * 2];
  __shared__ int s_finish;
  if (st->error || st->done) return;
  // every thread reads the iteration count before the first barrier; thread 0 advances it
  // after the last one
  const int it = st->iter;
  double n = 0.0, sum = 0.0;
  for (int r = threadIdx.x; r < nreg; r += blockDim.x) {
    fresh[r] = 0;
    removed[r] = 0;
    int cx, cy;
    if (!region_active(ptr, cand, r, max_cand, &cx, &cy)) continue;
    sum += chi2[r];
    n += 1.0;
  }
  double ns[2] = {n, sum};
  block_sums<2>(ns, sh);
  n = ns[0];
  sum = ns[1];
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
        removed[r] = 1;
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
  b.keys = ws.take<uint32_t>((size_t)p.H * p.W);
  b.over = ws.take<int32_t>((size_t)over_capacity(p));
  b.n_over = ws.take<int32_t>(1);
  b.bin_val = ws.take<float>((size_t)p.nreg * kBinCap);
  b.bin_idx = ws.take<int32_t>((size_t)p.nreg * kBinCap);
  b.bin_cnt = ws.take<int32_t>(p.nreg);
  b.cand = ws.take<int32_t>((size_t)p.nreg * p.max_cand * 2);
  b.cand_stat = ws.take<int32_t>((size_t)p.nreg * p.max_cand);
  b.cand_chi2 = ws.take<double>((size_t)p.nreg * p.max_cand);
  b.ptr = ws.take<int32_t>(p.nreg);
  b.have = ws.take<int32_t>(p.nreg);
  b.C = ws.take<double>((size_t)p.nreg * p.Nd * p.P);
  b.Gt = ws.take<double>((size_t)p.nreg * p.Nc * p.Nc);
  b.Gpart = ws.take<double>((size_t)p.nreg * kGramSplit * p.Nc * p.Nc);
  b.gram_count = ws.take<int32_t>(p.nreg);
  b.foot = ws.take<double>((size_t)p.nreg * 4);
  b.chi2 = ws.take<double>(p.nreg);
  b.chi2_part = ws.take<double>((size_t)p.nreg * kChi2Split * 2);
  b.chi2_count = ws.take<int32_t>(p.nreg);
  b.M = ws.take<double>((size_t)p.Nsys * p.Nsys);
  b.v = ws.take<double>(p.Nsys);
  b.L = ws.take<double>((size_t)p.Nsys * p.Nsys);
  b.rinv = ws.take<float2>((size_t)((p.Nsys + kNB - 1) / kNB) * kNB * kNB);
  b.Lh = ws.take<float>((size_t)p.Nsys * p.Nsys);
  b.Ll = ws.take<float>((size_t)p.Nsys * p.Nsys);
  b.Fh = ws.take<float>((size_t)p.Nsys * p.Nsys);
  b.Fl = ws.take<float>((size_t)p.Nsys * p.Nsys);
  b.x = ws.take<double>(p.Nsys);
  b.pdiag = ws.take<double>(p.Nsys);
  b.y = ws.take<double>(p.Nsys);
  b.piv = ws.take<int32_t>(p.Nsys);
  b.gv = ws.take<double>((size_t)p.nreg * p.Ns);
  b.gp = ws.take<double>((size_t)p.nreg * (p.Ns + 1) * (p.Ns + 1));
  b.fresh = ws.take<int32_t>(p.nreg);
  b.removed = ws.take<int32_t>(p.nreg);
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
  sp.Nd = p.Nd;
  sp.f1d = t.f1d;
  sp.f1d64 = t.f1d64;
  sp.psi = t.psi;
  sp.sk = t.sk;
  sp.cand = b.cand;
  sp.ptr = b.ptr;
  sp.have = b.have;
  sp.fresh = b.fresh;
  sp.C = b.C;
  sp.Gt = b.Gt;
  sp.Gpart = b.Gpart;
  sp.gram_count = b.gram_count;
  sp.footsum = b.foot;
  sp.st = st;

  SysParams sy;
  sy.b = sp.b;
  sy.g = sp.g;
  sy.nreg = p.nreg;
  sy.max_cand = p.max_cand;
  sy.Nc = p.Nc;
  sy.Nd = p.Nd;
  sy.lambda = p.cfg.dual ? p.cfg.penalty : 0.0;
  sy.pen = t.pen;
  sy.pdiag = b.pdiag;
  sy.Nsys = p.Nsys;
  sy.joint = p.cfg.norm_mode == PSFM_NORM_JOINT;
  sy.cand = b.cand;
  sy.ptr = b.ptr;
  sy.Gt = b.Gt;
  sy.footsum = b.foot;
  sy.gv = b.gv;
  sy.gp = b.gp;
  sy.fresh = b.fresh;
  sy.removed = b.removed;
  sy.dsol = dsol;
  sy.M = b.M;
  sy.Lh = b.Lh;
  sy.Ll = b.Ll;
  sy.v = b.v;
  sy.st = st;

  Chi2Params cq;
  cq.sp = sp;
  cq.gv = sy.gv;
  cq.dsol = dsol;
  cq.alpha = p.cfg.soften_alpha;
  cq.chi2 = b.chi2;
  cq.cand_chi2 = b.cand_chi2;
  cq.part = b.chi2_part;
  cq.count = b.chi2_count;

  // design block storage is double for the FP64 and double-float modes, float for FP32
  const int prec = p.cfg.precision;
  const size_t esz = prec == PSFM_PREC_FP64 ? sizeof(double) : sizeof(float);
  size_t sm_design = esz * ((size_t)p.foot * p.foot + (size_t)p.foot * p.sw);
  const int nblk = (p.Nc + 3) / 4, npair = nblk * (nblk + 1) / 2;
  size_t sm_gram = sizeof(double) * npair * 16 + esz * (nblk * 4 * 32 + 32);
  if (prec == PSFM_PREC_F32X2 || prec == PSFM_PREC_BF16X6) {
    sm_design = design_df_smem(p.foot, p.sw, p.h, p.dmax);
    const int maxch = ((p.P + kGramChunk - 1) / kGramChunk + kGramSplit - 1) / kGramSplit;
    sm_gram = sizeof(float) * (4 * nblk * 4 * kGramLd + 4 * maxch * kGramChunk + 4 * p.Nd);
  }
  if (sm_design > 200 * 1024 || sm_gram > 200 * 1024) return PSFM_ERR_UNSUPPORTED;
  // TF32 / BF16X3: FP32 design blocks, the Gram on the tensor cores (k_gram_tc.cu)
  // BF16X6: double-float design blocks, the Gram on the tensor cores from exact split products
  const bool tcm = prec == PSFM_PREC_TF32 || prec == PSFM_PREC_BF16X3;
  // the split-product tensor-core Gram takes up to 64 augmented columns (one N = 64 tile);
  // wider BF16X6 bases use the double-float Gram
  const bool ozm = prec == PSFM_PREC_BF16X6 && p.Nc <= 64;
  const bool dfm = prec == PSFM_PREC_F32X2 || prec == PSFM_PREC_BF16X6;  // double-float design
  auto design = prec == PSFM_PREC_FP64 ? k_stamp_design<double> : k_stamp_design<float>;
  auto gram = prec == PSFM_PREC_FP64 ? k_stamp_gram<double>
              : dfm ? k_stamp_gram_df : k_stamp_gram<float>;
  auto chi2 = prec == PSFM_PREC_FP64 ? k_chi2<double> : dfm ? k_chi2<float2> : k_chi2<float>;
  if (cudaFuncSetAttribute(design, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_design) !=
          cudaSuccess ||
      cudaFuncSetAttribute(gram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_gram) !=
          cudaSuccess)
    return PSFM_ERR_CUDA;
  const int N = p.Nsys;
  const int64_t nthr = (int64_t)N * (N + 1) / 2;  // the assembly's upper-triangle entries
  const int N1 = p.Ns + 1;
  const int asm_chunk = (40 * 1024) / (N1 * N1 * (int)sizeof(double));
  // the rejection kernel works per region: one thread each (FP64 reductions over idle warps
  // cost as much as useful ones here)
  const int reject_threads = std::min(1024, std::max(32, (p.nreg + 31) / 32 * 32));
  const size_t sm_asm = (sizeof(double) * N1 * N1 + sizeof(int)) * (size_t)asm_chunk;
  const int npanel = (N + kNB - 1) / kNB;
  const size_t sm_solve = sizeof(float2) * ((size_t)N + 32 * 33 + 32);
  if (sm_solve > 200 * 1024) return PSFM_ERR_UNSUPPORTED;
  if (cudaFuncSetAttribute(k_chol_solve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sm_solve) != cudaSuccess)
    return PSFM_ERR_CUDA;
  // Gram blocks of regions that never hold a stamp stay zero (they are weighted by zero); M
  // starts empty and is updated by the stamps that join or leave it
  if (cudaMemsetAsync(b.Gt, 0, sizeof(double) * (size_t)p.nreg * p.Nc * p.Nc, s) != cudaSuccess ||
      cudaMemsetAsync(b.M, 0, sizeof(double) * (size_t)p.Nsys * p.Nsys, s) != cudaSuccess ||
      cudaMemsetAsync(b.fresh, 0, sizeof(int32_t) * p.nreg, s) != cudaSuccess ||
      cudaMemsetAsync(b.removed, 0, sizeof(int32_t) * p.nreg, s) != cudaSuccess ||
      cudaMemsetAsync(b.gram_count, 0, sizeof(int32_t) * p.nreg, s) != cudaSuccess ||
      cudaMemsetAsync(b.chi2_count, 0, sizeof(int32_t) * p.nreg, s) != cudaSuccess ||
      cudaMemsetAsync(b.pdiag, 0, sizeof(double) * p.Nsys, s) != cudaSuccess)
    return PSFM_ERR_CUDA;
  for (int it = 0; it < p.cfg.max_iter; ++it) {
    prof_begin("stamps", s);
    if (dfm) {
      if (launch_design_df(p.h, dim3(p.nreg, p.NH * (p.cfg.dual ? 2 : 1)), sm_design, sp, s) !=
          cudaSuccess)
        return PSFM_ERR_CUDA;
    } else {
      design<<<dim3(p.nreg, p.ng), 256, sm_design, s>>>(sp);
    }
    if (tcm) {
      if (launch_gram_tc(prec == PSFM_PREC_TF32 ? 0 : 1, sp, p.nreg, s) != cudaSuccess)
        return PSFM_ERR_CUDA;
    } else if (ozm) {
      // the first iteration's Grams fill the GPU one stamp per CTA; the few stamps replaced in
      // later iterations split over kGramSplit CTAs each, which shortens the solve's chain
      if (launch_gram_oz(sp, p.nreg, it == 0 ? 1 : kGramSplit, s) != cudaSuccess)
        return PSFM_ERR_CUDA;
    } else {
      gram<<<dim3(p.nreg, dfm ? kGramSplit : 1), dfm ? kGramThreads : 256, sm_gram, s>>>(sp);
    }
    prof_end("stamps", s, 2);
    prof_begin("system", s);
    k_norm<<<1, 1024, 0, s>>>(sy);
    k_system_delta<<<(unsigned)((nthr + 255) / 256), 256, sm_asm, s>>>(sy, 0, asm_chunk);
    if (p.cfg.dual) k_penalty<<<1, 1024, 0, s>>>(sy);
    k_rhs<<<(N * 32 + 255) / 256, 256, 0, s>>>(sy);
    prof_end("system", s, p.cfg.dual ? 4 : 3);
    prof_begin("cholesky", s);
    k_chol_first<<<1, kCholThreads, 0, s>>>(N, b.Lh, b.Ll, b.Fh, b.Fl, b.rinv, b.M, b.pdiag,
                                            st);
    for (int kb = 0; kb + 1 < npanel; ++kb) {
      const int nt = (N - (kb + 1) * kNB + 15) / 16;
      k_chol_panel<<<1 + nt * (nt + 1) / 2, kCholThreads, 0, s>>>(N, kb, b.Lh, b.Ll, b.Fh, b.Fl,
                                                                   b.rinv, b.M, b.pdiag, st);
    }
    k_chol_solve<<<1, kSolveThreads, sm_solve, s>>>(N, b.Fh, b.Fl, b.rinv, b.v, nullptr, b.x,
                                                    st, 0);
    for (int mode = 1; mode <= 2; ++mode) {
      k_residual<<<(N * 32 + 255) / 256, 256, 0, s>>>(N, b.M, b.pdiag, b.v, b.x, b.y, st, mode);
      k_chol_solve<<<1, kSolveThreads, sm_solve, s>>>(N, b.Fh, b.Fl, b.rinv, b.y, b.x, b.x,
                                                      st, mode);
    }
    k_store_solution<<<(N + 255) / 256, 256, 0, s>>>(N, sy.joint, b.x, dsol, st);
    k_lu_solve<<<1, 1024, 0, s>>>(N, sy.joint, b.M, b.pdiag, b.v, b.L, b.y, b.piv, dsol, st);
    prof_end("cholesky", s, npanel + 7);
    prof_begin("chi2_reject", s);
    chi2<<<dim3(p.nreg, kChi2Split), kChi2Threads, (sizeof(double) + sizeof(float2)) * p.Nd + 16,
           s>>>(cq);
    k_reject<<<1, reject_threads, 0, s>>>(p.nreg, p.max_cand, p.cfg.max_iter, p.cfg.reject_nsigma, b.cand,
                                b.ptr, b.cand_stat, b.chi2, b.fresh, b.removed, st);
    k_system_delta<<<(unsigned)((nthr + 255) / 256), 256, sm_asm, s>>>(sy, 1, asm_chunk);
    prof_end("chi2_reject", s, 3);
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
  out->kernel_sum = h.q_ksum;
  out->mom_x = h.q_mx;
  out->mom_y = h.q_my;
  out->mom_xx = h.q_mxx;
  out->mom_yy = h.q_myy;
  out->mom_xy = h.q_mxy;
  out->deconv_max = h.q_deconv;
  out->quality_flags = h.q_flags;
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
