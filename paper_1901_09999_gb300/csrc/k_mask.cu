// Mask propagation through the convolution (Sec. 3.4) and the CONV.BAD radius.
//
// A masked input pixel (or the image edge) within Chebyshev distance r_bad of an output pixel
// flags it CONV.BAD; one within h but none within r_bad flags CONV.POOR.  r_bad is the
// smallest box radius outside which the squared kernel, realised at the image centre, holds
// at most bad_frac of its total (Sec. 3.4).
//
// The dilation runs on bit planes: one 32-bit word per 32 pixels of a row, built with warp
// ballots, dilated horizontally with funnel shifts, then vertically by OR-ing rows while the
// output mask is written.
#include "psfm_internal.h"

namespace psfm {
namespace {

// Tiles of 256 pixels x kTileRows rows: a CTA walks its rows, one pixel per thread.
constexpr int kTileRows = 32;
constexpr int kTileWords = 8;  // 256 pixels

// Each thread loads kBitsBatch rows of its column before the first ballot, so that a CTA keeps
// enough bytes in flight to stream the 2-byte mask at HBM rate.
constexpr int kBitsBatch = 8;

__global__ void __launch_bounds__(256) k_mask_bits(const uint16_t* m1, const uint16_t* m2, int W,
                                                   int H, int64_t pitch, int nwords,
                                                   uint16_t badmask, uint32_t* bits) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y0 = blockIdx.y * kTileRows;
  const int wx = x >> 5;
  const int rows = min(kTileRows, H - y0);
  for (int r0 = 0; r0 < rows; r0 += kBitsBatch) {
    uint16_t m[kBitsBatch];
#pragma unroll
    for (int q = 0; q < kBitsBatch; ++q) {
      m[q] = 0;
      if (x < W && r0 + q < rows) {
        const int64_t o = (int64_t)(y0 + r0 + q) * pitch + x;
        m[q] = m1[o];
        if (m2) m[q] |= m2[o];
      }
    }
#pragma unroll
    for (int q = 0; q < kBitsBatch; ++q) {
      if (r0 + q >= rows) break;  // uniform over the CTA
      const uint32_t word = __ballot_sync(0xffffffffu, (m[q] & badmask) != 0);
      if ((threadIdx.x & 31) == 0 && wx < nwords)
        bits[(int64_t)(y0 + r0 + q) * nwords + wx] = word;
    }
  }
}

// Bits beyond the row end count as masked (off-image).
__device__ __forceinline__ uint32_t word_at(const uint32_t* row, int wx, int nwords, int W) {
  if (wx < 0 || wx >= nwords) return 0xffffffffu;
  uint32_t v = row[wx];
  const int valid = W - wx * 32;
  if (valid < 32) v |= ~((1u << valid) - 1u);
  return v;
}

__device__ __forceinline__ uint32_t hdilate(uint32_t prev, uint32_t cur, uint32_t next, int r) {
  const uint64_t lo = ((uint64_t)cur << 32) | prev;
  const uint64_t hi = ((uint64_t)next << 32) | cur;
  uint32_t out = cur;
  for (int d = 1; d <= r; ++d) {
    out |= (uint32_t)(lo >> (32 - d));  // neighbour at -d
    out |= (uint32_t)(hi >> d);         // neighbour at +d
  }
  return out;
}

__global__ void k_mask_hdilate(const uint32_t* bits, int W, int H, int nwords, int r_fixed,
                               const DevState* st, int h, uint32_t* hb_bad, uint32_t* hb_poor) {
  const int y = blockIdx.y;
  const int wx = blockIdx.x * blockDim.x + threadIdx.x;
  if (wx >= nwords) return;
  const uint32_t* row = bits + (int64_t)y * nwords;
  const uint32_t p = word_at(row, wx - 1, nwords, W);
  const uint32_t c = word_at(row, wx, nwords, W);
  const uint32_t n = word_at(row, wx + 1, nwords, W);
  const int rb = r_fixed >= 0 ? r_fixed : (r_fixed == -2 ? st->r_bad2 : st->r_bad);
  hb_bad[(int64_t)y * nwords + wx] = hdilate(p, c, n, rb);
  hb_poor[(int64_t)y * nwords + wx] = hdilate(p, c, n, h);
}

// Vertical dilation and output, one CTA per tile of 256 pixels x kTileRows rows: the tile's
// horizontally dilated words and the h rows above and below go to shared memory, each thread
// ORs one word's column window (r_bad rows for CONV.BAD, h for CONV.POOR), then the CTA writes
// the tile's pixels a row at a time (one pixel per thread, consecutive addresses).
// mode 0: out = m1 | m2 with CONV.BAD near a bad pixel, else CONV.POOR;
// mode 1 (first pass of the dual kernel): out holds only the two proximity flags;
// mode 2 (second pass): the flags already in out are ORed with this pass's, then mode 0's rule.
__global__ void __launch_bounds__(256) k_mask_out(const uint32_t* hb_bad, const uint32_t* hb_poor,
                                                  const uint16_t* m1, const uint16_t* m2, int W,
                                                  int H, int64_t pitch, int nwords, int r_fixed,
                                                  const DevState* st, int h, uint16_t conv_bad,
                                                  uint16_t conv_poor, int mode, uint16_t* out) {
  __shared__ uint32_t sb[kTileRows + 2 * PSFM_MAX_HALF_WIDTH][kTileWords];
  __shared__ uint32_t sp[kTileRows + 2 * PSFM_MAX_HALF_WIDTH][kTileWords];
  __shared__ uint32_t vbs[kTileRows][kTileWords], vps[kTileRows][kTileWords];
  const int tid = threadIdx.x;
  const int wx0 = blockIdx.x * kTileWords, y0 = blockIdx.y * kTileRows;
  const int rb = r_fixed >= 0 ? r_fixed : (r_fixed == -2 ? st->r_bad2 : st->r_bad);
  const int nr = kTileRows + 2 * h;
  for (int q = tid; q < nr * kTileWords; q += blockDim.x) {
    const int r = q / kTileWords, c = q - r * kTileWords;
    const int yy = y0 - h + r, wx = wx0 + c;
    uint32_t wb = 0xffffffffu, wp = 0xffffffffu;  // rows off the image count as masked
    if (yy >= 0 && yy < H) {
      wb = wx < nwords ? hb_bad[(int64_t)yy * nwords + wx] : 0u;
      wp = wx < nwords ? hb_poor[(int64_t)yy * nwords + wx] : 0u;
    }
    sb[r][c] = wb;
    sp[r][c] = wp;
  }
  __syncthreads();
  {
    const int r = tid / kTileWords, c = tid - r * kTileWords;
    uint32_t vb = 0, vp = 0;
    for (int d = -h; d <= h; ++d) {
      if ((d < 0 ? -d : d) <= rb) vb |= sb[r + h + d][c];
      vp |= sp[r + h + d][c];
    }
    vbs[r][c] = vb;
    vps[r][c] = vp;
  }
  __syncthreads();
  const int x = wx0 * 32 + tid;
  if (x >= W) return;
  const uint32_t bit = 1u << (tid & 31);
  const int wc = tid >> 5;
  const int rows = min(kTileRows, H - y0);
  // kBitsBatch rows at a time, their mask (and previous output) loads issued first
  for (int r0 = 0; r0 < rows; r0 += kBitsBatch) {
    uint16_t mv[kBitsBatch], pv[kBitsBatch];
#pragma unroll
    for (int q = 0; q < kBitsBatch; ++q) {
      mv[q] = 0;
      pv[q] = 0;
      if (r0 + q < rows && mode != 1) {
        const int64_t o = (int64_t)(y0 + r0 + q) * pitch + x;
        mv[q] = m1[o];
        if (m2) mv[q] |= m2[o];
        if (mode == 2) pv[q] = out[o];
      }
    }
#pragma unroll
    for (int q = 0; q < kBitsBatch; ++q) {
      const int r = r0 + q;
      if (r >= rows) break;
      const int64_t o = (int64_t)(y0 + r) * pitch + x;
      bool nb = (vbs[r][wc] & bit) != 0, np = (vps[r][wc] & bit) != 0;
      if (mode == 1) {
        out[o] = (uint16_t)((nb ? conv_bad : 0) | (np ? conv_poor : 0));
        continue;
      }
      if (mode == 2) {
        nb = nb || (pv[q] & conv_bad);
        np = np || (pv[q] & conv_poor);
      }
      uint16_t m = mv[q];
      if (nb)
        m |= conv_bad;
      else if (np)
        m |= conv_poor;
      out[o] = m;
    }
  }
}

// r_bad from the kernel at the image centre (xt = yt = 0, so only the constant spatial term
// survives), in FP64: K_c(u, v) = sum_k a_{k,0} psi_k f_{g,p}(u) f_{g,q}(v) + delta (b0 -
// sum_k a_{k,0} s_k).  One CTA.
__global__ void k_rbad(BasisDev b, const double* f1d64, const double* psi, const double* sk,
                       const double* dsol, double bad_frac, int second, DevState* st) {
  extern __shared__ double sh[];
  const int W = b.w, h = b.h;
  double* colgp = sh;            // [NH][W]
  double* K2 = colgp + b.NH * W; // [W*W]
  double* part = K2 + W * W;     // [h+2]
  double* Kc = part + 2 * h + 3; // [W*W] the kernel itself (after the [h+1] ring sums)
  double* encl = Kc + W * W;     // [h+1] kernel sum within radius r
  const int tid = threadIdx.x;
  if (st->error) return;
  for (int i = tid; i < b.NH * W; i += blockDim.x) {
    const int pl = i / W, v = i - pl * W;
    int g = 0;
    while (g + 1 < b.ng && pl >= b.plane_base[g + 1]) ++g;
    const int p = pl - b.plane_base[g], dg = b.deg[g];
    const int kgp = b.kbase[g] + p * (dg + 1) - (p * (p - 1)) / 2;
    double c = 0.0;
    for (int q = 0; q <= dg - p; ++q)
      c += dsol[2 + (kgp + q) * b.Ns] * psi[kgp + q] * f1d64[(b.plane_base[g] + q) * W + v];
    colgp[i] = c;
  }
  __syncthreads();
  if (tid == 0) {
    double dc = dsol[0];
    for (int k = 0; k < b.Nb; ++k) dc -= dsol[2 + k * b.Ns] * sk[k];
    part[h + 1] = dc;
  }
  __syncthreads();
  for (int i = tid; i < W * W; i += blockDim.x) {
    const int v = i / W, u = i - v * W;
    double kv = 0.0;
    for (int pl = 0; pl < b.NH; ++pl) kv += f1d64[pl * W + u] * colgp[pl * W + v];
    if (u == h && v == h) kv += part[h + 1];
    K2[i] = kv * kv;
    Kc[i] = kv;
  }
  __syncthreads();
  // energy per Chebyshev ring (thread c walks ring c in a fixed order, so the result does not
  // depend on scheduling), then outside(r) = sum of the rings beyond r
  double* ring = part + h + 2;  // [h+1]
  for (int c = tid; c <= h; c += blockDim.x) {
    double e = 0.0;
    if (c == 0) {
      e = K2[h * W + h];
    } else {
      for (int t = -c; t <= c; ++t) {
        e += K2[(h - c) * W + h + t];  // top row
        e += K2[(h + c) * W + h + t];  // bottom row
      }
      for (int t = -c + 1; t <= c - 1; ++t) {
        e += K2[(h + t) * W + h - c];  // left column
        e += K2[(h + t) * W + h + c];  // right column
      }
    }
    ring[c] = e;
  }
  __syncthreads();
  if (tid == 0) {
    // suffix sums from the outermost ring inwards: part[c] = sum_{c' >= c} ring[c']
    double acc = 0.0;
    for (int c = h; c >= 0; --c) {
      acc += ring[c];
      part[c] = acc;
    }
    const double tot = part[0];
    int rb = h;
    for (int r = 0; r < h; ++r)
      if (part[r + 1] <= bad_frac * tot) {
        rb = r;
        break;
      }
    if (second) st->r_bad2 = rb;
    else st->r_bad = rb;
  }
  if (second) return;
  // quality diagnostics (Sec. 3.7): moments and enclosed kernel sums; every sum is taken in a
  // fixed order (per-thread strided partials, xor-shuffle trees, warps in order)
  __shared__ double wpart[8][6];
  double m[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};  // K, uK, vK, uuK, vvK, uvK
  for (int i = tid; i < W * W; i += blockDim.x) {
    const double v = (double)(i / W - h), u = (double)(i % W - h), k = Kc[i];
    m[0] += k;
    m[1] += u * k;
    m[2] += v * k;
    m[3] += u * u * k;
    m[4] += v * v * k;
    m[5] += u * v * k;
  }
  const int lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    for (int o = 16; o > 0; o >>= 1) m[j] += __shfl_xor_sync(0xffffffffu, m[j], o);
    if (lane == 0) wpart[wid][j] = m[j];
  }
  // enclosed sums: warp w takes radii r = w, w + nw, ...
  for (int r = wid; r <= h; r += nw) {
    double e = 0.0;
    for (int i = lane; i < W * W; i += 32) {
      const int v = i / W - h, u = i % W - h;
      if (u * u + v * v <= r * r) e += Kc[i];
    }
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if (lane == 0) encl[r] = e;
  }
  __syncthreads();
  if (tid == 0) {
    double t[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int w = 0; w < nw; ++w)
      for (int j = 0; j < 6; ++j) t[j] += wpart[w][j];
    const double ks = t[0];
    const double mx = t[1] / ks, my = t[2] / ks;
    const double mxx = t[3] / ks - mx * mx, myy = t[4] / ks - my * my, mxy = t[5] / ks - mx * my;
    double dmax = -INFINITY;
    for (int r = 0; r <= h; ++r) dmax = fmax(dmax, encl[r] / ks);
    st->q_ksum = ks;
    st->q_mx = mx;
    st->q_my = my;
    st->q_mxx = mxx;
    st->q_myy = myy;
    st->q_mxy = mxy;
    st->q_deconv = dmax;
    int f = 0;
    if (st->n_active < 3) f |= PSFM_QUALITY_FEW_STAMPS;
    if (st->chi2_mean > 0.5) f |= PSFM_QUALITY_MEAN_DEV;
    if (st->chi2_rms > 0.3) f |= PSFM_QUALITY_RMS_DEV;
    if (fabs(mx) > 0.5 || fabs(my) > 0.5) f |= PSFM_QUALITY_MOMENT1;
    if (mxx < 0.0 || myy < 0.0) f |= PSFM_QUALITY_MOMENT2;
    if (dmax > 1.03) f |= PSFM_QUALITY_DECONV;
    st->q_flags = f;
  }
}

}  // namespace

cudaError_t launch_mask(const Plan& p, const ApplyBuffers& b, const uint16_t* mref,
                        const uint16_t* mimg, uint16_t* out, cudaStream_t st, int dual_pass) {
  const int nwords = (p.W + 31) / 32;
  const int rsel = dual_pass == 2 ? -2 : -1;
  // the dilated bad pixels: of the reference, or of the science image in the dual kernel's
  // second pass (both input masks still form the output bits)
  const uint16_t* src = dual_pass == 2 ? mimg : mref;
  dim3 blk(256);
  const dim3 tiles((p.W + 255) / 256, (p.H + kTileRows - 1) / kTileRows);
  k_mask_bits<<<tiles, blk, 0, st>>>(src, nullptr, p.W, p.H, p.pitch, nwords, p.cfg.badmask,
                                     b.bits);
  k_mask_hdilate<<<dim3((nwords + 127) / 128, p.H), 128, 0, st>>>(
      b.bits, p.W, p.H, nwords, rsel, b.st, p.h, b.hb_bad, b.hb_poor);
  k_mask_out<<<tiles, blk, 0, st>>>(b.hb_bad, b.hb_poor, mref, mimg, p.W, p.H, p.pitch, nwords,
                                    rsel, b.st, p.h, p.cfg.conv_bad, p.cfg.conv_poor, dual_pass,
                                    out);
  return cudaGetLastError();
}

cudaError_t launch_rbad(const Plan& p, const DevTables& t, const double* dsol, DevState* ds,
                        cudaStream_t st, bool second) {
  const size_t smem =
      sizeof(double) * ((size_t)p.NH * p.w + 2 * (size_t)p.w * p.w + 3 * (size_t)p.h + 4);
  cudaError_t e = cudaFuncSetAttribute(k_rbad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_rbad<<<1, 256, smem, st>>>(basis_dev(p), t.f1d64, t.psi, t.sk, dsol, p.cfg.bad_frac,
                               second ? 1 : 0, ds);
  return cudaGetLastError();
}

}  // namespace psfm
