// Stamp design columns in double-float (Sec. 2, Eq. 4; Sec. 3.5): for every active stamp and
// every horizontal plane (g, p) of the basis, the terms B_{g,p,q} (x) X for q = 0..d_g - p
// over the (2s+1)^2 stamp pixels, X the masked reference (or, for the dual kernel of Eq. 2,
// the masked science image).  The 1-D factors f_{g,n}(u) = u^n exp(-u^2 / 2 sigma_g^2) have
// parity (-1)^n, so each pass folds its taps: with the mirrored sums and differences
// S_u = X(c - u) + X(c + u) and D_u = X(c - u) - X(c + u) an output is
//   f_n(0) X(c) + sum_{u=1..h} f_n(u) (n even ? S_u : D_u),
// half the products of the plain sum, and the sums are shared by every output of the same
// parity.  The pixels are exact FP32, the factors FP32 pairs, the mirrored sums of pixels
// exact (TwoSum), the sums of double-float rows unnormalised pairs; every product and
// accumulation keeps about 48 bits (the error stays at 2^-48 of the sum of |terms|).
//
// grid (nreg, N_H x sets): one block per (stamp, plane), so a handful of replaced stamps in a
// later rejection iteration still spread over many SMs.  The kernel is specialised on the
// kernel half width, so the tap loops unroll and the pixel windows stay in registers.
#include "dfloat.cuh"
#include "stamp.h"

namespace psfm {
namespace {

constexpr int kDesignThreads = 256;
// vertical outputs of one plane formed together from one set of mirrored sums (planes with
// more q take several groups, each forming its sums again: smaller code, measured faster than
// eight at a time, which outgrew the instruction cache)
constexpr int kVq = 4;
// footprint elements staged per thread per round
constexpr int kStageBatch = 8;
// neighbouring outputs of one row per thread in the horizontal pass, and neighbouring columns
// per thread in the vertical passes (kVc / 2 16-byte loads per row and side)
constexpr int kHo = 4;
constexpr int kVc = 2;

__host__ __device__ __forceinline__ int round4(int x) { return (x + 3) & ~3; }
// row strides: F holds the kHo - 1 columns a thread group reads past the footprint, H a
// multiple of kVc columns
__host__ __device__ __forceinline__ int f_stride(int foot) { return foot + kHo; }
__host__ __device__ __forceinline__ int h_stride(int sw) { return (sw + kVc - 1) / kVc * kVc; }

// horizontal pass of plane p (parity ODD): H(rr, x) for the foot rows and the sw columns of
// the stamp; F has row stride fs >= foot + kHo - 1, H row stride sw2
template <int HW, bool ODD>
__device__ __forceinline__ void hpass(const float* F, int fs, int foot, int sw, int sw2,
                                      const float2* wp, float2* H, int tid) {
  const int ng = (sw + kHo - 1) / kHo;
  for (int it = tid; it < foot * ng; it += kDesignThreads) {
    const int rr = it / ng, x0 = (it - rr * ng) * kHo;
    // xv[i] = F(rr, x0 + i): the taps of the outputs x0 .. x0 + kHo - 1 (centre x + HW)
    const float* row = F + rr * fs + x0;
    float xv[2 * HW + kHo];
#pragma unroll
    for (int i = 0; i < 2 * HW + kHo; ++i) xv[i] = row[i];
    df acc[kHo];
#pragma unroll
    for (int j = 0; j < kHo; ++j) acc[j] = df{0.f, 0.f};
    if (!ODD) {  // f_p(0) = 0 for odd p
      const df w0 = {wp[0].x, wp[0].y};
#pragma unroll
      for (int j = 0; j < kHo; ++j) df_fma_f(acc[j], xv[j + HW], w0);
    }
#pragma unroll
    for (int u = 1; u <= HW; ++u) {
      const float2 wv = wp[u];
      const df w = {wv.x, wv.y};
#pragma unroll
      for (int j = 0; j < kHo; ++j) {
        const float b = xv[j + HW + u];
        df_fma(acc[j], two_sum(xv[j + HW - u], ODD ? -b : b), w);
      }
    }
#pragma unroll
    for (int j = 0; j < kHo; ++j)
      if (x0 + j < sw) {
        const df o = df_norm(acc[j]);
        H[rr * sw2 + x0 + j] = make_float2(o.hi, o.lo);
      }
  }
}

// vertical passes of one plane: out[q][y * sw + x] = sum_v f_q(v) H(y + HW - v, x) for
// q = 0..nq-1, kVc neighbouring columns per thread
template <int HW>
__device__ __forceinline__ void vpass(const float2* H, int sw, int sw2, const float2* wq,
                                      int nq, float2* out, int P, int tid) {
  constexpr int NV = kVc / 2;  // 16-byte loads per row
  const int ncg = sw2 / kVc;
  for (int it = tid; it < sw * ncg; it += kDesignThreads) {
    const int y = it / ncg, x0 = kVc * (it - y * ncg);
    const float4* col = reinterpret_cast<const float4*>(H + y * sw2 + x0);
    const int rs = sw2 / 2;  // row stride in float4
    for (int q0 = 0; q0 < nq; q0 += kVq) {
      df acc[kVq][kVc];
      {
        df c[kVc];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const float4 t = col[HW * rs + v];
          c[2 * v] = df{t.x, t.y};
          c[2 * v + 1] = df{t.z, t.w};
        }
#pragma unroll
        for (int qi = 0; qi < kVq; ++qi) {
#pragma unroll
          for (int j = 0; j < kVc; ++j) acc[qi][j] = df{0.f, 0.f};
          if ((qi & 1) == 0 && q0 + qi < nq) {  // q0 is even: q has the parity of qi
            const float2 wv = wq[(q0 + qi) * (HW + 1)];
            const df w = {wv.x, wv.y};
#pragma unroll
            for (int j = 0; j < kVc; ++j) df_fma(acc[qi][j], c[j], w);
          }
        }
      }
      const bool any_odd = nq - q0 > 1;
      // partly unrolled: the fully unrolled passes of every q outgrow the instruction cache
#pragma unroll 5
      for (int u = 1; u <= HW; ++u) {
        df sm[kVc], df_[kVc];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const float4 a = col[(HW - u) * rs + v];
          const float4 b = col[(HW + u) * rs + v];
          const df a0 = {a.x, a.y}, a1 = {a.z, a.w}, b0 = {b.x, b.y}, b1 = {b.z, b.w};
          sm[2 * v] = df_sum_raw(a0, b0);
          sm[2 * v + 1] = df_sum_raw(a1, b1);
          df_[2 * v] = df{0.f, 0.f};
          df_[2 * v + 1] = df{0.f, 0.f};
          if (any_odd) {
            df_[2 * v] = df_sum_raw(a0, df_neg(b0));
            df_[2 * v + 1] = df_sum_raw(a1, df_neg(b1));
          }
        }
#pragma unroll
        for (int qi = 0; qi < kVq; ++qi)
          if (q0 + qi < nq) {
            const float2 wv = wq[(q0 + qi) * (HW + 1) + u];
            const df w = {wv.x, wv.y};
#pragma unroll
            for (int j = 0; j < kVc; ++j) df_fma(acc[qi][j], (qi & 1) ? df_[j] : sm[j], w);
          }
      }
#pragma unroll
      for (int qi = 0; qi < kVq; ++qi)
        if (q0 + qi < nq) {
          float2* o = out + (int64_t)(q0 + qi) * P + y * sw + x0;
#pragma unroll
          for (int j = 0; j < kVc; ++j)
            if (x0 + j < sw) {
              const df rv = df_norm(acc[qi][j]);
              o[j] = make_float2(rv.hi, rv.lo);
            }
        }
    }
  }
}

// Footprint staging: kStageBatch elements per thread per round, all of their loads (masks and
// pixels, independent of each other) issued before any is used.  SUMS: also the unweighted
// footprint sums of the normalisation (Sec. 3.2) in FP64, only in the one block per stamp that
// forms them (the FP64 adds of every element would otherwise be issued, predicated off, by all
// blocks).
template <bool SUMS>
__device__ __forceinline__ void stage_footprint(const StampParams& P, int set, float* F, int fs,
                                                int foot, int x0, int y0, int tid, double* f1,
                                                double* f2, double* nf) {
  const int nst = foot * fs;
  for (int i0 = tid; i0 < nst; i0 += kStageBatch * kDesignThreads) {
    int64_t off[kStageBatch];
    bool in[kStageBatch];
#pragma unroll
    for (int e = 0; e < kStageBatch; ++e) {
      const int i = i0 + e * kDesignThreads;
      const int rr = i / fs, cc = i - rr * fs;
      const int gx = x0 + cc, gy = y0 + rr;
      in[e] = i < nst && cc < foot && gx >= 0 && gx < P.g.W && gy >= 0 && gy < P.g.H;
      off[e] = in[e] ? (int64_t)gy * P.g.pitch + gx : 0;
    }
    uint16_t ma[kStageBatch], mb[kStageBatch];
    float va[kStageBatch], vb[kStageBatch];
#pragma unroll
    for (int e = 0; e < kStageBatch; ++e) {
      ma[e] = in[e] ? P.m1[off[e]] : (uint16_t)0;
      mb[e] = in[e] ? P.m2[off[e]] : (uint16_t)0;
      va[e] = in[e] ? (set == 0 ? P.i1[off[e]] : P.i2[off[e]]) : 0.f;
      vb[e] = (SUMS && in[e]) ? P.i2[off[e]] : 0.f;
    }
#pragma unroll
    for (int e = 0; e < kStageBatch; ++e) {
      const int i = i0 + e * kDesignThreads;
      if (i >= nst) break;
      const bool a = (ma[e] & P.badmask) != 0, b = (mb[e] & P.badmask) != 0;
      F[i] = (set == 0 ? a : b) ? 0.f : va[e];
      if (SUMS && in[e] && !a && !b) {
        *f1 += va[e];
        *f2 += vb[e];
        *nf += 1.0;
      }
    }
  }
}

template <int HW>
__global__ void __launch_bounds__(kDesignThreads, 3) k_stamp_design_df(StampParams P) {
  constexpr int W = 2 * HW + 1;
  extern __shared__ __align__(16) unsigned char sh_raw[];
  // blockIdx.y = set * N_H + plane: set 0 convolves the masked reference, set 1 (dual kernel,
  // Eq. 2) the science image with its own mask, into design columns N_b..2 N_b - 1
  const int r = blockIdx.x, set = blockIdx.y / P.b.NH, pl = blockIdx.y - set * P.b.NH;
  const int tid = threadIdx.x;
  if (block_skip(P.st)) return;
  int cx, cy;
  if (!region_active(P.ptr, P.cand, r, P.max_cand, &cx, &cy)) return;
  if (P.have[r] == P.ptr[r]) return;
  int g = 0;
  while (g + 1 < P.b.ng && pl >= P.b.plane_base[g + 1]) ++g;
  const int foot = P.foot, sw = P.sw;
  const int dg = P.b.deg[g], pb = P.b.plane_base[g], p = pl - pb;
  const int fs = f_stride(foot), sw2 = h_stride(sw);
  float* F = reinterpret_cast<float*>(sh_raw);                  // foot x fs
  float2* H = reinterpret_cast<float2*>(F + round4(foot * fs));  // foot x sw2
  float2* wq = H + foot * sw2;                                  // (dg + 1) x (HW + 1)
  for (int i = tid; i < (dg + 1) * (HW + 1); i += kDesignThreads) {
    const int n = i / (HW + 1), u = i - n * (HW + 1);
    const df v = df_split(P.f1d64[(pb + n) * W + HW + u]);
    wq[i] = make_float2(v.hi, v.lo);
  }
  for (int i = tid; i < foot * (sw2 - sw); i += kDesignThreads) {
    const int rr = i / (sw2 - sw);
    H[rr * sw2 + sw + (i - rr * (sw2 - sw))] = make_float2(0.f, 0.f);
  }
  const int x0 = cx - P.s - HW, y0 = cy - P.s - HW;
  const bool sums = set == 0 && pl == 0;
  double f1 = 0.0, f2 = 0.0, nf = 0.0;
  if (sums)
    stage_footprint<true>(P, set, F, fs, foot, x0, y0, tid, &f1, &f2, &nf);
  else
    stage_footprint<false>(P, set, F, fs, foot, x0, y0, tid, &f1, &f2, &nf);
  if (sums) {
    // unweighted footprint sums for the normalisation (Sec. 3.2)
    __shared__ double red[3][kDesignThreads / 32];
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
      for (int i = 0; i < kDesignThreads / 32; ++i) {
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
  if (p & 1)
    hpass<HW, true>(F, fs, foot, sw, sw2, wq + p * (HW + 1), H, tid);
  else
    hpass<HW, false>(F, fs, foot, sw, sw2, wq + p * (HW + 1), H, tid);
  __syncthreads();
  const int kgp = P.b.kbase[g] + p * (dg + 1) - (p * (p - 1)) / 2;
  float2* out = reinterpret_cast<float2*>(P.C) + ((int64_t)r * P.Nd + set * P.b.Nb + kgp) * P.P;
  vpass<HW>(H, sw, sw2, wq, dg - p + 1, out, P.P, tid);
}

template <int HW>
cudaError_t launch_hw(dim3 grid, size_t smem, const StampParams& sp, cudaStream_t s) {
  if (cudaFuncSetAttribute(k_stamp_design_df<HW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess)
    return cudaGetLastError();
  k_stamp_design_df<HW><<<grid, kDesignThreads, smem, s>>>(sp);
  return cudaGetLastError();
}

}  // namespace

size_t design_df_smem(int foot, int sw, int h, int dmax) {
  const int fs = f_stride(foot), sw2 = h_stride(sw);
  return sizeof(float) * (size_t)round4(foot * fs) + sizeof(float2) * (size_t)foot * sw2 +
         sizeof(float2) * (size_t)(dmax + 1) * (h + 1);
}

cudaError_t launch_design_df(int h, dim3 grid, size_t smem, const StampParams& sp,
                             cudaStream_t s) {
  switch (h) {
#define PSFM_DESIGN_CASE(n) \
  case n:                   \
    return launch_hw<n>(grid, smem, sp, s);
    PSFM_DESIGN_CASE(1) PSFM_DESIGN_CASE(2) PSFM_DESIGN_CASE(3) PSFM_DESIGN_CASE(4)
    PSFM_DESIGN_CASE(5) PSFM_DESIGN_CASE(6) PSFM_DESIGN_CASE(7) PSFM_DESIGN_CASE(8)
    PSFM_DESIGN_CASE(9) PSFM_DESIGN_CASE(10) PSFM_DESIGN_CASE(11) PSFM_DESIGN_CASE(12)
    PSFM_DESIGN_CASE(13) PSFM_DESIGN_CASE(14) PSFM_DESIGN_CASE(15) PSFM_DESIGN_CASE(16)
    PSFM_DESIGN_CASE(17) PSFM_DESIGN_CASE(18) PSFM_DESIGN_CASE(19) PSFM_DESIGN_CASE(20)
    PSFM_DESIGN_CASE(21) PSFM_DESIGN_CASE(22) PSFM_DESIGN_CASE(23) PSFM_DESIGN_CASE(24)
#undef PSFM_DESIGN_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace psfm
