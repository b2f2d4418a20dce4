// Spatially varying PSF-matching convolution of the whole image (Eq. 12 with the kernel of
// Sec. 2): O(x, y) = b0 R + sum_k a_k(x, y) (B_k (x) R)(x, y) + d0, written as separable
// passes.  With B_k = psi_k f_{g,p}(u) f_{g,q}(v) - s_k delta:
//   H_{g,p}(x, y) = sum_u f_{g,p}(u) R(x-u, y)              (horizontal pass, one per plane)
//   V_k(x, y)     = sum_v f_{g,q}(v) H_{g,p}(x, y-v)        (vertical pass, one per term)
//   O(x, y)       = sum_k [a_k(x, y) psi_k] V_k + beta(x, y) R(x, y) + d0,
//   beta(x, y)    = b0 - sum_k a_k(x, y) s_k,
// where a_k(x, y) = sum_s a_{k,s} xt^l yt^m is evaluated per output pixel (Horner in xt, yt).
//
// Folded taps: f_{g,n}(t) = t^n exp(-t^2 / 2 sigma_g^2) has f_{g,n}(-t) = (-1)^n f_{g,n}(t), so
// a pass of parity n is f(0) X(0) + sum_{t>0} f(t) (X(-t) + (-1)^n X(t)).  The sums (even n) or
// differences (odd n) of the mirrored samples are formed once and shared by every plane (in
// the horizontal passes) or term (in the vertical passes) of that parity: each then costs h + 1
// (even) or h (odd) FMAs per output instead of 2h + 1.
//
// One CTA computes a 32 (x) by TY (y) output tile, TY = 64 (default) or 128 rows (8 per warp).  The masked reference with a halo of h
// pixels is staged in shared memory once.  For each Gaussian and parity, up to four horizontal
// planes at a time are computed over the staged rows (each thread takes a row and 4 columns
// and forms the mirrored sums once for all planes of the chunk) into shared memory; then for
// each of those planes p every thread takes 8 output rows of one column and runs the vertical
// passes of all terms q of the plane, even q from the mirrored sums of the column window, odd
// q from its differences.  The folded weights of a Gaussian are stored by (t, parity slot) so
// that one broadcast float4 read gives a tap of four planes or terms.
#pragma once

#include "psfm_internal.h"

namespace psfm {
namespace conv {

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
  int ty;      // tile rows: 8 per warp of the CTA (64 or 128)
  int nslots;  // horizontal planes held in shared memory at once (4..8)
  uint16_t badmask;
};

// Folded weight table of the vertical passes: per Gaussian g and tap t = 0..h a row of kFoldLd
// slots, even degrees n at slot n / 2 (0..4), odd degrees at slot 8 + (n - 1) / 2 (8..11),
// unused slots zero.  Every pass of up to four terms starts at degree 0, 8 (even) or 1 (odd),
// that is at slot 0, 4 or 8: its weights are one aligned float4 read.
constexpr int kFoldLd = 12;
constexpr int kMaxChunk = 4;

__host__ __device__ __forceinline__ int fold_slot(int n) { return (n & 1) ? 8 + (n >> 1) : n >> 1; }

template <int HW>
struct ConvShape {
  static constexpr int RS = kConvTX + ((2 * HW + 3) / 4) * 4;  // staged row stride (x4 floats)
  static constexpr int NV4 = (4 + 2 * HW + 3) / 4;              // float4s per H window
  // terms of one parity per vertical pass
  static constexpr int MAXNE = 4;
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

// Horizontal passes of NC planes of parity PAR for one item (a staged row, 4 columns): rv holds
// the row window (rv[j + HW] is the item's column j), wf the folded weights of the chunk's
// first plane (slot), hs the item's place in the first plane of the chunk.
template <int HW, int PAR, int NC>
__device__ __forceinline__ void hfold(const float* rv, const float* wf, float* hs, int pstride) {
  float a[NC][4];
  if (PAR == 0) {
    const float4 w0 = *reinterpret_cast<const float4*>(wf);
    const float wc[4] = {w0.x, w0.y, w0.z, w0.w};
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
      for (int j = 0; j < 4; ++j) a[c][j] = wc[c] * rv[j + HW];
  } else {
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
      for (int j = 0; j < 4; ++j) a[c][j] = 0.f;
  }
#pragma unroll
  for (int u = 1; u <= HW; ++u) {
    const float4 wv = *reinterpret_cast<const float4*>(wf + u * kFoldLd);
    const float wc[4] = {wv.x, wv.y, wv.z, wv.w};
    if (NC == 1) {  // one plane: the mirrored taps directly (as many FMAs, no sums)
      const float wm = PAR == 0 ? wc[0] : -wc[0];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        a[0][j] = fmaf(wc[0], rv[j + HW - u], a[0][j]);
        a[0][j] = fmaf(wm, rv[j + HW + u], a[0][j]);
      }
    } else {
      // each mirrored sum is used at once by every plane (formed column by column, which keeps
      // the compiler from holding all of them live)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float sd =
            PAR == 0 ? rv[j + HW - u] + rv[j + HW + u] : rv[j + HW - u] - rv[j + HW + u];
#pragma unroll
        for (int c = 0; c < NC; ++c) a[c][j] = fmaf(wc[c], sd, a[c][j]);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < NC; ++c)
    *reinterpret_cast<float4*>(hs + c * pstride) = make_float4(a[c][0], a[c][1], a[c][2], a[c][3]);
}

// Vertical passes of NE terms of parity PAR (q = q0, q0 + 2, ...) of one plane for the 8 rows of
// a thread: col holds the column window (col[i + HW] is output row i), wf the folded weights of
// the first term (slot), al the coefficient polynomial of the first term (terms 2 apart are
// 2 S1^2 floats apart).  Each term's result is weighted by its polynomial and added to out.
template <int HW, int SS, int PAR, int NE>
__device__ __forceinline__ void vfold(const float* col, const float* wf, const float* al,
                                      float xt, const float yt[8], float out[8]) {
  constexpr int S1 = SS + 1;
  float acc[NE][8];
  if (PAR == 0) {
    const float4 w0 = *reinterpret_cast<const float4*>(wf);
    const float wc[4] = {w0.x, w0.y, w0.z, w0.w};
#pragma unroll
    for (int e = 0; e < NE; ++e)
#pragma unroll
      for (int i = 0; i < 8; ++i) acc[e][i] = wc[e] * col[i + HW];
  } else {
#pragma unroll
    for (int e = 0; e < NE; ++e)
#pragma unroll
      for (int i = 0; i < 8; ++i) acc[e][i] = 0.f;
  }
#pragma unroll
  for (int v = 1; v <= HW; ++v) {
    const float4 wv = *reinterpret_cast<const float4*>(wf + v * kFoldLd);
    const float wc[4] = {wv.x, wv.y, wv.z, wv.w};
    if (NE == 1) {
      const float wm = PAR == 0 ? wc[0] : -wc[0];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        acc[0][i] = fmaf(wc[0], col[i + HW - v], acc[0][i]);
        acc[0][i] = fmaf(wm, col[i + HW + v], acc[0][i]);
      }
    } else {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float sd =
            PAR == 0 ? col[i + HW - v] + col[i + HW + v] : col[i + HW - v] - col[i + HW + v];
#pragma unroll
        for (int e = 0; e < NE; ++e) acc[e][i] = fmaf(wc[e], sd, acc[e][i]);
      }
    }
  }
#pragma unroll
  for (int e = 0; e < NE; ++e) add_term<SS>(al + 2 * e * S1 * S1, xt, yt, acc[e], out);
}

template <int HW, int PAR>
__device__ __forceinline__ void hfold_n(int nc, const float* rv, const float* wf, float* hs,
                                        int pstride) {
  switch (nc) {
    case 1: hfold<HW, PAR, 1>(rv, wf, hs, pstride); break;
    case 2: hfold<HW, PAR, 2>(rv, wf, hs, pstride); break;
    case 3: hfold<HW, PAR, 3>(rv, wf, hs, pstride); break;
    default: hfold<HW, PAR, 4>(rv, wf, hs, pstride); break;
  }
}

template <int HW, int SS, int PAR>
__device__ __forceinline__ void vfold_n(int ne, const float* col, const float* wf,
                                        const float* al, float xt, const float yt[8],
                                        float out[8]) {
  switch (ne) {
    case 1: vfold<HW, SS, PAR, 1>(col, wf, al, xt, yt, out); break;
    case 2: vfold<HW, SS, PAR, 2>(col, wf, al, xt, yt, out); break;
    case 3: vfold<HW, SS, PAR, 3>(col, wf, al, xt, yt, out); break;
    default: vfold<HW, SS, PAR, 4>(col, wf, al, xt, yt, out); break;
  }
}

// One CTA of 32 x TY outputs, TY = 8 x (warps of the CTA): 64 rows (two CTAs of 256 threads
// per SM) or 128 rows (one CTA of 512 threads); at most 128 registers a thread either way.
template <int HW, int SS, int TY>
__global__ void __launch_bounds__(4 * TY, TY == 64 ? 2 : 1) k_conv_image(ConvParams P) {
  using CS = ConvShape<HW>;
  constexpr int TX = kConvTX, RS = CS::RS;
  constexpr int NV4 = CS::NV4, MAXNE = CS::MAXNE;
  constexpr int NT = 4 * TY, RR = TY + 2 * HW;
  constexpr int FG = (HW + 1) * kFoldLd;  // folded weights per Gaussian
  extern __shared__ float4 smem4[];
  float* Rs = reinterpret_cast<float*>(smem4);
  float* Hs = Rs + RR * RS;
  constexpr int S = SS, S1 = SS + 1;
  float* Wf = Hs + P.nslots * RR * TX;
  float* alpha = Wf + P.b.ng * FG;
  float* beta = alpha + P.b.Nb * S1 * S1;

  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;

  for (int i = tid; i < P.b.ng * FG; i += NT) {
    const int g = i / FG, r = i - g * FG, t = r / kFoldLd, sl = r - t * kFoldLd;
    const int n = sl < 5 ? 2 * sl : (sl >= 8 ? 2 * (sl - 8) + 1 : -1);
    Wf[i] = (n >= 0 && n <= P.b.deg[g])
                ? P.f1d[(P.b.plane_base[g] + n) * P.b.wpad + HW + t] : 0.f;
  }

  for (int i = tid; i < P.b.Nb * S1 * S1; i += NT) {
    const int k = i / (S1 * S1), r = i - k * S1 * S1, m = r / S1, l = r - m * S1;
    float v = 0.f;
    if (l + m <= S) v = (float)(P.dsol[2 + k * P.b.Ns + spatial_index(l, m, S)] * P.psi[k]);
    alpha[i] = v;
  }
  // beta's polynomial: warp w forms the coefficients (m, l) = w, w + NT / 32, ..., each lane
  // summing the terms k = lane, lane + 32, ... and the warp adding the lanes' sums by shuffles
  // (no serial FP64 chain in the CTA's prologue)
  for (int c = tid >> 5; c < S1 * S1; c += NT / 32) {
    const int m = c / S1, l = c - m * S1, lane = tid & 31;
    double v = 0.0;
    if (l + m <= S) {
      const int s = spatial_index(l, m, S);
      for (int k = lane; k < P.b.Nb; k += 32) v += P.dsol[2 + k * P.b.Ns + s] * P.sk[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      v = (s == 0 ? P.dsol[0] : 0.0) - v;
    }
    if (lane == 0) beta[c] = (float)v;
  }
  // masked reference tile with halo; zero padding to the row stride
  stage_masked_tile<8>(P.ref, P.mref, P.badmask, P.g.W, P.g.H, P.g.pitch, x0 - HW, y0 - HW, RR,
                       TX + 2 * HW, RS, Rs, tid, NT);
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

  // One pass over the staged rows and one over the columns per group of planes: all planes of
  // a Gaussian when they fit the plane slots (even degrees first, then odd), otherwise the
  // planes of one parity four at a time.
  for (int g = 0; g < P.b.ng; ++g) {
    const int dg = P.b.deg[g];
    const float* wfg = Wf + g * FG;
    const int ne_g = dg / 2 + 1, no_g = (dg + 1) / 2;  // planes of even / odd degree
    const bool whole = ne_g + no_g <= P.nslots && ne_g <= kMaxChunk && no_g <= kMaxChunk;
    for (int grp = 0; grp < (whole ? 1 : 2 * ((ne_g + kMaxChunk - 1) / kMaxChunk)); ++grp) {
      // planes of this group: ce of even degree from e0, co of odd degree from o0
      int ce, co, e0, o0;
      if (whole) {
        ce = ne_g;
        co = no_g;
        e0 = 0;
        o0 = 1;
      } else {
        const int par = grp & 1, c0 = (grp >> 1) * kMaxChunk;
        const int np = par == 0 ? ne_g : no_g;
        const int nc = c0 < np ? min(kMaxChunk, np - c0) : 0;
        ce = par == 0 ? nc : 0;
        co = par == 1 ? nc : 0;
        e0 = 2 * c0;
        o0 = 1 + 2 * c0;
      }
      if (ce + co == 0) continue;  // uniform over the CTA
      // ---- horizontal passes of the group's planes over the staged rows; chunks start at
      // degree 0 or 8 (even) or 1 (odd): slot 0, 4 or 8, an aligned float4
      for (int item = tid; item < RR * 8; item += NT) {
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
        float* hs = Hs + row * TX + xg * 4;
        if (ce) hfold_n<HW, 0>(ce, rv, wfg + fold_slot(e0), hs, RR * TX);
        if (co) hfold_n<HW, 1>(co, rv, wfg + fold_slot(o0), hs + ce * RR * TX, RR * TX);
      }
      __syncthreads();
      // ---- vertical passes: each H value in registers serves 8 outputs and all q
      for (int c = 0; c < ce + co; ++c) {
        const int p = c < ce ? e0 + 2 * c : o0 + 2 * (c - ce);
        float col[8 + 2 * HW];
        const float* hp = Hs + (c * RR + wi * 8) * TX + lane;
#pragma unroll
        for (int t = 0; t < 8 + 2 * HW; ++t) col[t] = hp[t * TX];
        const int kgp = P.b.kbase[g] + p * (dg + 1) - (p * (p - 1)) / 2;  // term (g, p, 0)
        const int nq = dg - p + 1;
        for (int q0 = 0; q0 < nq; q0 += 2 * MAXNE) {  // even q
          const int ne = min(MAXNE, (nq - q0 + 1) / 2);
          vfold_n<HW, SS, 0>(ne, col, wfg + fold_slot(q0), alpha + (kgp + q0) * S1 * S1, xt, yt,
                             out);
        }
        for (int q0 = 1; q0 < nq; q0 += 2 * MAXNE) {  // odd q
          const int ne = min(MAXNE, (nq - q0 + 1) / 2);
          vfold_n<HW, SS, 1>(ne, col, wfg + fold_slot(q0), alpha + (kgp + q0) * S1 * S1, xt, yt,
                             out);
        }
      }
      __syncthreads();
    }
  }

  float rc[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) rc[i] = Rs[(wi * 8 + i + HW) * RS + lane + HW];
  add_term<SS>(beta, xt, yt, rc, out);
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
// it reserved per CTA), and the most one CTA may take.
constexpr size_t kConvSmemTwoCtas = 112 * 1024;
constexpr size_t kConvSmemMax = 227 * 1024;

// Shared memory of a CTA with tile height ty and ns plane slots.
template <int HW>
size_t conv_smem(const ConvParams& P, int ty, int ns) {
  using CS = ConvShape<HW>;
  const int S1 = P.b.S + 1, RR = ty + 2 * HW;
  return sizeof(float) * ((size_t)RR * CS::RS + (size_t)P.b.ng * (HW + 1) * kFoldLd +
                          (size_t)P.b.Nb * S1 * S1 + (size_t)S1 * S1 + (size_t)ns * RR * kConvTX);
}

template <int HW, int TY>
cudaError_t launch_ty(const ConvParams& P, size_t smem, cudaStream_t st) {
  dim3 grid((P.g.W + kConvTX - 1) / kConvTX, (P.g.H + TY - 1) / TY);
  switch (P.b.S) {
#define PSFM_SCASE(n)                                                                         \
  case n: {                                                                                  \
    cudaError_t e = cudaFuncSetAttribute(k_conv_image<HW, n, TY>,                            \
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,        \
                                         (int)smem);                                         \
    if (e != cudaSuccess) return e;                                                          \
    k_conv_image<HW, n, TY><<<grid, 4 * TY, smem, st>>>(P);                                  \
    break;                                                                                   \
  }
    PSFM_SCASE(0) PSFM_SCASE(1) PSFM_SCASE(2) PSFM_SCASE(3)
#undef PSFM_SCASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Launch with P.ty = 64 or 128 output rows per CTA and as many plane slots (up to all planes
// of the widest Gaussian, at least four) as keep the CTAs of that height resident together.
template <int HW>
cudaError_t launch_hw(ConvParams P, cudaStream_t st) {
  if (P.ty != 64 && P.ty != 128) return cudaErrorInvalidValue;
  const size_t budget = P.ty == 64 ? kConvSmemTwoCtas : kConvSmemMax;
  int want = kMaxChunk;
  for (int g = 0; g < P.b.ng; ++g) want = max(want, P.b.deg[g] + 1);
  want = min(want, 2 * kMaxChunk);
  int ns = want;
  while (ns > kMaxChunk && conv_smem<HW>(P, P.ty, ns) > budget) --ns;
  P.nslots = ns;
  const size_t smem = conv_smem<HW>(P, P.ty, ns);
  if (smem > budget) return cudaErrorInvalidValue;
  if (P.ty == 64) return launch_ty<HW, 64>(P, smem, st);
  return launch_ty<HW, 128>(P, smem, st);
}

// Launches the convolution for half widths in [lo, hi] (one translation unit per range, so that
// the instantiations compile in parallel); cudaErrorInvalidValue outside it.
cudaError_t launch_range_1_6(int h, const ConvParams& P, cudaStream_t st);
cudaError_t launch_range_7_10(int h, const ConvParams& P, cudaStream_t st);
cudaError_t launch_range_11_13(int h, const ConvParams& P, cudaStream_t st);
cudaError_t launch_range_14_15(int h, const ConvParams& P, cudaStream_t st);
cudaError_t launch_range_16_17(int h, const ConvParams& P, cudaStream_t st);
cudaError_t launch_range_18_19(int h, const ConvParams& P, cudaStream_t st);
cudaError_t launch_range_20_21(int h, const ConvParams& P, cudaStream_t st);
cudaError_t launch_range_22_24(int h, const ConvParams& P, cudaStream_t st);

}  // namespace conv
}  // namespace psfm
