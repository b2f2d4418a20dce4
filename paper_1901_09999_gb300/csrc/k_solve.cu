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
  if (tid == 0) P.have[r] = P.ptr[r];
}

struct SysParams {
  BasisDev b;
  ImgGeom g;
  int nreg, max_cand, Nc, Nsys, joint;
  const int32_t* cand;
  const int32_t* ptr;
  const double* G;
  const double* footsum;
  const double* psi;
  const double* sk;
  double* gv;      // [nreg][Ns] spatial factors at the stamp centre, 0 if inactive
  double* dsol;
  double* M;
  double* v;
  DevState* st;
};

// One thread: active count, spatial factors, and (SEPARATE) b0, d0 from footprint sums.
__global__ void k_norm(SysParams P) {
  if (threadIdx.x != 0) return;
  if (P.st->error || P.st->done) return;
  int n = 0;
  double s11 = 0, s12 = 0, s22 = 0, t1 = 0, t2 = 0;
  const double xs = P.g.W > 1 ? 2.0 / (P.g.W - 1) : 0.0, ys = P.g.H > 1 ? 2.0 / (P.g.H - 1) : 0.0;
  for (int r = 0; r < P.nreg; ++r) {
    int cx, cy;
    double* gr = P.gv + (int64_t)r * P.b.Ns;
    if (!region_active(P.ptr, P.cand, r, P.max_cand, &cx, &cy)) {
      for (int s = 0; s < P.b.Ns; ++s) gr[s] = 0.0;
      continue;
    }
    ++n;
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
  P.st->n_active = n;
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

// Unknown index -> (column of the augmented block, spatial term or -1).
__device__ __forceinline__ void unknown_col(const SysParams& P, int i, int* col, int* s) {
  if (P.joint) {
    if (i == 0) {
      *col = P.b.Nb;  // R
      *s = -1;
      return;
    }
    if (i == P.Nsys - 1) {
      *col = P.b.Nb + 1;  // 1
      *s = -1;
      return;
    }
    i -= 1;
  }
  *col = i / P.b.Ns;
  *s = i - *col * P.b.Ns;
}

// M_ij and v_i (Eq. 5-6), one thread per (i, j) with j >= i.  Basis columns carry psi_k and
// the delta term: the design column of term k is psi_k C_k - s_k R.
__global__ void k_assemble(SysParams P) {
  if (P.st->error || P.st->done) return;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int N = P.Nsys;
  const int Nb = P.b.Nb, Nc = P.Nc;
  const int colR = Nb, col1 = Nb + 1, colI = Nb + 2;
  if (t < (int64_t)N * N) {
    const int i = (int)(t / N), j = (int)(t - (int64_t)i * N);
    if (j < i) return;
    int ci, si, cj, sj;
    unknown_col(P, i, &ci, &si);
    unknown_col(P, j, &cj, &sj);
    const double pi = ci < Nb ? P.psi[ci] : 1.0, ki = ci < Nb ? P.sk[ci] : 0.0;
    const double pj = cj < Nb ? P.psi[cj] : 1.0, kj = cj < Nb ? P.sk[cj] : 0.0;
    double acc = 0.0;
    for (int r = 0; r < P.nreg; ++r) {
      const double* gr = P.gv + (int64_t)r * P.b.Ns;
      const double gi = si < 0 ? 1.0 : gr[si], gj = sj < 0 ? 1.0 : gr[sj];
      if (gr[0] == 0.0) continue;  // inactive region (the constant spatial term is 1)
      const double* Gr = P.G + (int64_t)r * Nc * Nc;
      // (pi C_i - ki R) . W (pj C_j - kj R), with C_R = R for the R column (pi = 1, ki = 0)
      double e = pi * pj * Gr[ci * Nc + cj];
      if (kj != 0.0) e -= pi * kj * Gr[ci * Nc + colR];
      if (ki != 0.0) e -= ki * pj * Gr[colR * Nc + cj];
      if (ki != 0.0 && kj != 0.0) e += ki * kj * Gr[colR * Nc + colR];
      acc += gi * gj * e;
    }
    P.M[(int64_t)i * N + j] = acc;
    P.M[(int64_t)j * N + i] = acc;
  }
  if (t < N) {
    const int i = (int)t;
    int ci, si;
    unknown_col(P, i, &ci, &si);
    const double pi = ci < Nb ? P.psi[ci] : 1.0, ki = ci < Nb ? P.sk[ci] : 0.0;
    const double b0 = P.dsol[0], d0 = P.dsol[1];
    double acc = 0.0;
    for (int r = 0; r < P.nreg; ++r) {
      const double* gr = P.gv + (int64_t)r * P.b.Ns;
      if (gr[0] == 0.0) continue;
      const double gi = si < 0 ? 1.0 : gr[si];
      const double* Gr = P.G + (int64_t)r * Nc * Nc;
      // target: I2 (joint) or I2 - b0 R - d0 (separate)
      double e = pi * Gr[ci * Nc + colI] - ki * Gr[colR * Nc + colI];
      if (!P.joint) {
        e -= b0 * (pi * Gr[ci * Nc + colR] - ki * Gr[colR * Nc + colR]);
        e -= d0 * (pi * Gr[ci * Nc + col1] - ki * Gr[colR * Nc + col1]);
      }
      acc += gi * e;
    }
    P.v[i] = acc;
  }
}

// Cholesky (then LU with partial pivoting) of the N x N system in FP64, one CTA.
__global__ void __launch_bounds__(1024) k_solve_system(int N, int joint, int ncoef,
                                                       const double* M, const double* v,
                                                       double* L, double* y, int32_t* piv,
                                                       double* dsol, DevState* st) {
  const int tid = threadIdx.x, nt = blockDim.x;
  __shared__ int s_fail;
  __shared__ double s_d;
  if (st->error || st->done) return;
  for (int64_t i = tid; i < (int64_t)N * N; i += nt) L[i] = M[i];
  for (int i = tid; i < N; i += nt) y[i] = v[i];
  if (tid == 0) s_fail = 0;
  __syncthreads();
  // right-looking Cholesky on the lower triangle
  for (int j = 0; j < N; ++j) {
    if (tid == 0) {
      const double d = L[(int64_t)j * N + j];
      if (!(d > 0.0) || !isfinite(d)) s_fail = 1;
      else {
        s_d = sqrt(d);
        L[(int64_t)j * N + j] = s_d;
      }
    }
    __syncthreads();
    if (s_fail) break;
    const double dj = s_d;
    for (int i = j + 1 + tid; i < N; i += nt) L[(int64_t)i * N + j] /= dj;
    __syncthreads();
    for (int i = j + 1 + tid; i < N; i += nt) {
      const double lij = L[(int64_t)i * N + j];
      double* Li = L + (int64_t)i * N;
      for (int k = j + 1; k <= i; ++k) Li[k] -= lij * L[(int64_t)k * N + j];
    }
    __syncthreads();
  }
  if (!s_fail) {
    // L z = v (column sweep), then L^T x = z
    for (int j = 0; j < N; ++j) {
      if (tid == 0) y[j] /= L[(int64_t)j * N + j];
      __syncthreads();
      const double yj = y[j];
      for (int i = j + 1 + tid; i < N; i += nt) y[i] -= L[(int64_t)i * N + j] * yj;
      __syncthreads();
    }
    for (int j = N - 1; j >= 0; --j) {
      if (tid == 0) y[j] /= L[(int64_t)j * N + j];
      __syncthreads();
      const double yj = y[j];
      for (int i = tid; i < j; i += nt) y[i] -= L[(int64_t)j * N + i] * yj;
      __syncthreads();
    }
  } else {
    // LU with partial pivoting on a fresh copy
    for (int64_t i = tid; i < (int64_t)N * N; i += nt) L[i] = M[i];
    for (int i = tid; i < N; i += nt) y[i] = v[i];
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
  (void)ncoef;
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

// One thread: rejection decision of Sec. 3.3 and loop control.
__global__ void k_reject(int nreg, int max_cand, int max_iter, double nsig, const int32_t* cand,
                         int32_t* ptr, int32_t* cand_stat, const double* chi2, DevState* st) {
  if (threadIdx.x != 0) return;
  if (st->error || st->done) return;
  int n = 0;
  double sum = 0.0;
  for (int r = 0; r < nreg; ++r) {
    int cx, cy;
    if (!region_active(ptr, cand, r, max_cand, &cx, &cy)) continue;
    sum += chi2[r];
    ++n;
  }
  const double mu = sum / n;
  double ss = 0.0;
  for (int r = 0; r < nreg; ++r) {
    int cx, cy;
    if (!region_active(ptr, cand, r, max_cand, &cx, &cy)) continue;
    const double d = chi2[r] - mu;
    ss += d * d;
  }
  const double sd = sqrt(ss / n);
  st->chi2_mean = mu;
  st->chi2_rms = sd;
  const int it = st->iter;
  st->iter = it + 1;
  bool finish = it == max_iter - 1;
  if (!finish) {
    const double thr = mu + nsig * sd;
    st->threshold = thr;
    int nrej = 0;
    for (int r = 0; r < nreg; ++r) {
      int cx, cy;
      if (!region_active(ptr, cand, r, max_cand, &cx, &cy)) continue;
      if (chi2[r] > thr) {
        cand_stat[(int64_t)r * max_cand + ptr[r]] = PSFM_CAND_REJECTED;
        ptr[r] += 1;
        ++nrej;
      }
    }
    finish = nrej == 0;
  }
  if (finish) {
    int nu = 0;
    for (int r = 0; r < nreg; ++r) {
      int cx, cy;
      if (!region_active(ptr, cand, r, max_cand, &cx, &cy)) continue;
      cand_stat[(int64_t)r * max_cand + ptr[r]] = PSFM_CAND_USED;
      ++nu;
    }
    st->n_active = nu;
    st->done = 1;
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
  b.foot = ws.take<double>((size_t)p.nreg * 4);
  b.chi2 = ws.take<double>(p.nreg);
  b.M = ws.take<double>((size_t)p.Nsys * p.Nsys);
  b.v = ws.take<double>(p.Nsys);
  b.L = ws.take<double>((size_t)p.Nsys * p.Nsys);
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
  sy.G = b.G;
  sy.footsum = b.foot;
  sy.psi = t.psi;
  sy.sk = t.sk;
  sy.gv = b.gv;
  sy.dsol = dsol;
  sy.M = b.M;
  sy.v = b.v;
  sy.st = st;

  Chi2Params cq;
  cq.sp = sp;
  cq.gv = sy.gv;
  cq.dsol = dsol;
  cq.alpha = p.cfg.soften_alpha;
  cq.chi2 = b.chi2;
  cq.cand_chi2 = b.cand_chi2;

  const bool fp64 = p.cfg.precision == PSFM_PREC_FP64;
  const size_t esz = fp64 ? sizeof(double) : sizeof(float);
  const size_t sm_design = esz * ((size_t)p.foot * p.foot + (size_t)p.foot * p.sw);
  const int nblk = (p.Nc + 3) / 4, npair = nblk * (nblk + 1) / 2;
  const size_t sm_gram = sizeof(double) * npair * 16 + esz * (nblk * 4 * 32 + 32);
  if (sm_design > 200 * 1024 || sm_gram > 200 * 1024) return PSFM_ERR_UNSUPPORTED;
  auto design = fp64 ? k_stamp_design<double> : k_stamp_design<float>;
  auto gram = fp64 ? k_stamp_gram<double> : k_stamp_gram<float>;
  auto chi2 = fp64 ? k_chi2<double> : k_chi2<float>;
  if (cudaFuncSetAttribute(design, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_design) !=
          cudaSuccess ||
      cudaFuncSetAttribute(gram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_gram) !=
          cudaSuccess)
    return PSFM_ERR_CUDA;
  const int64_t nn = (int64_t)p.Nsys * p.Nsys;
  for (int it = 0; it < p.cfg.max_iter; ++it) {
    prof_begin("stamps", s);
    design<<<dim3(p.nreg, p.ng), 256, sm_design, s>>>(sp);
    gram<<<p.nreg, 256, sm_gram, s>>>(sp);
    prof_end("stamps", s, 2);
    prof_begin("system", s);
    k_norm<<<1, 32, 0, s>>>(sy);
    k_assemble<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(sy);
    prof_end("system", s, 2);
    prof_begin("cholesky", s);
    k_solve_system<<<1, 1024, 0, s>>>(p.Nsys, sy.joint, p.ncoef, b.M, b.v, b.L, b.y, b.piv, dsol,
                                      st);
    prof_end("cholesky", s, 1);
    prof_begin("chi2_reject", s);
    chi2<<<p.nreg, 256, sizeof(double) * p.Nb, s>>>(cq);
    k_reject<<<1, 32, 0, s>>>(p.nreg, p.max_cand, p.cfg.max_iter, p.cfg.reject_nsigma, b.cand,
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
