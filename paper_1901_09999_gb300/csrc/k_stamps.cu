// Stamp candidates (Sec. 3.3): per subregion, the brightest peaks of the detection image
// S = I1 + I2 over a threshold of thresh_nsigma * sqrt(V1 + V2) above the background, with
// no masked pixel in the footprint that the kernel fit reads.
//
//   background: lower median of S over pixels unmasked in both images, found exactly by a
//               three-pass radix select on order-preserving 32-bit keys (11 + 11 + 10 bits);
//   peak:       S beats its 8 neighbours under the order (value, -linear index);
//   footprint:  no bad bit within Chebyshev radius s + h, read from a 1-bit-per-pixel plane;
//   ranking:    detections go to per-subregion bins, then each subregion keeps its
//               max_cand best under (value descending, index ascending), so the result does
//               not depend on the order in which threads found them.
// Every decision is taken in the same arithmetic as the definition (float32 sum, float64
// threshold), so the candidate table is bit-exact.
#include "psfm_internal.h"
#include "solve.h"

namespace psfm {
namespace {

__device__ __forceinline__ uint32_t fkey(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float fkey_inv(uint32_t k) {
  const uint32_t u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
  return __uint_as_float(u);
}

__device__ __forceinline__ void raise_error(DevState* st, int code) { atomicCAS(&st->error, 0, code); }

struct HistParams {
  const float* i1;
  const float* i2;
  const uint16_t* m1;
  const uint16_t* m2;
  int W, H;
  int64_t pitch;
  uint16_t badmask;
  int pass;
  uint32_t* hist;
  DevState* st;
};

__global__ void k_median_hist(HistParams P) {
  __shared__ uint32_t h[2048];
  for (int i = threadIdx.x; i < 2048; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const uint32_t prefix = P.st->sel_prefix;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  // rows strided over the grid; warp-uniform trip count so that the warp-wide match below
  // sees every lane
  for (int y = blockIdx.y; y < P.H; y += gridDim.y) {
    bool valid = false;
    uint32_t bin = 0;
    if (x < P.W) {
      const int64_t o = (int64_t)y * P.pitch + x;
      if (!((P.m1[o] | P.m2[o]) & P.badmask)) {
        const float s = P.i1[o] + P.i2[o];
        if (!isfinite(s)) {
          raise_error(P.st, PSFM_ERR_NONFINITE);
        } else {
          const uint32_t k = fkey(s);
          if (P.pass == 0) {
            bin = k >> 21;
            valid = true;
          } else if (P.pass == 1) {
            bin = (k >> 10) & 2047u;
            valid = (k >> 21) == prefix;
          } else {
            bin = k & 1023u;
            valid = (k >> 10) == prefix;
          }
        }
      }
    }
    // sky pixels crowd into a few bins: one shared-memory atomic per distinct bin per warp
    const unsigned act = __ballot_sync(0xffffffffu, valid);
    if (valid) {
      const unsigned same = __match_any_sync(act, bin);
      if ((int)(threadIdx.x & 31) == __ffs(same) - 1) atomicAdd(&h[bin], (uint32_t)__popc(same));
    }
  }
  __syncthreads();
  uint32_t* g = P.hist + P.pass * 2048;
  for (int i = threadIdx.x; i < 2048; i += blockDim.x)
    if (h[i]) atomicAdd(&g[i], h[i]);
}

// Pick the bin holding the rank-th key and narrow the prefix: a 1024-thread scan over the
// histogram (two bins per thread).
__global__ void __launch_bounds__(1024) k_median_select(const uint32_t* hist, int pass,
                                                        DevState* st) {
  __shared__ long long wsum[32];
  __shared__ long long s_rank;
  const uint32_t* g = hist + pass * 2048;
  const int nb = pass == 2 ? 1024 : 2048;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int b0 = 2 * tid;
  const long long c0 = b0 < nb ? g[b0] : 0, c1 = b0 + 1 < nb ? g[b0 + 1] : 0;
  long long incl = c0 + c1;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) wsum[w] = incl;
  if (tid == 0) s_rank = pass == 0 ? -1 : st->sel_rank;
  __syncthreads();
  if (w == 0) {
    long long v = wsum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long t = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += t;
    }
    wsum[lane] = v;
  }
  __syncthreads();
  if (w > 0) incl += wsum[w - 1];
  const long long tot = wsum[31];
  const long long excl = incl - (c0 + c1);
  long long rank = s_rank;
  if (pass == 0) {
    if (tot == 0) {
      if (tid == 0) {
        raise_error(st, PSFM_ERR_TOO_FEW_STAMPS);
        st->sel_prefix = 0;
      }
      return;
    }
    rank = (tot - 1) / 2;  // lower median
  }
  if (excl <= rank && rank < incl) {
    int b;
    long long rem;
    if (rank < excl + c0) {
      b = b0;
      rem = rank - excl;
    } else {
      b = b0 + 1;
      rem = rank - excl - c0;
    }
    st->sel_rank = (int32_t)rem;
    if (pass == 0)
      st->sel_prefix = (uint32_t)b;
    else if (pass == 1)
      st->sel_prefix = (st->sel_prefix << 11) | (uint32_t)b;
    else
      st->median_key = (st->sel_prefix << 10) | (uint32_t)b;
  }
}

__device__ __forceinline__ bool row_clean(const uint32_t* row, int xa, int xb) {
  // no set bit in [xa, xb] (inclusive, within the row)
  const int wa = xa >> 5, wb = xb >> 5;
  for (int w = wa; w <= wb; ++w) {
    uint32_t v = row[w];
    if (w == wa) v &= 0xffffffffu << (xa & 31);
    if (w == wb) v &= 0xffffffffu >> (31 - (xb & 31));
    if (v) return false;
  }
  return true;
}

struct DetectParams {
  const float* i1;
  const float* i2;
  const float* v1;
  const float* v2;
  const uint32_t* bits;
  int W, H, nwords;
  int64_t pitch;
  int R;  // s + h
  int nx, ny;
  double thresh;
  float* bin_val;
  int32_t* bin_idx;
  int32_t* bin_cnt;
  DevState* st;
};

__global__ void k_detect(DetectParams P) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (P.st->error) return;
  if (x < P.R || x >= P.W - P.R || y < P.R || y >= P.H - P.R) return;
  const int64_t o = (int64_t)y * P.pitch + x;
  const float s = P.i1[o] + P.i2[o];
  const float medf = fkey_inv(P.st->median_key);
  const float v1 = P.v1[o], v2 = P.v2[o];
  // FP32 pre-test with a margin far above FP32 rounding: pixels well below the threshold
  // skip the FP64 test (FP64 runs at 1/64 of the FP32 rate here); the decision itself is
  // always the FP64 one
  const float t32 = (float)P.thresh * sqrtf(v1 + v2);
  if (isfinite(t32) && isfinite(s) && s - medf < 0.999f * t32) return;
  const double med = (double)medf;
  const double thr = P.thresh * sqrt((double)v1 + (double)v2);
  if (!((double)s - med > thr)) return;
  const int64_t idx = (int64_t)y * P.W + x;
  for (int dy = -1; dy <= 1; ++dy)
    for (int dx = -1; dx <= 1; ++dx) {
      if (dx == 0 && dy == 0) continue;
      const int64_t on = o + (int64_t)dy * P.pitch + dx;
      const float sn = P.i1[on] + P.i2[on];
      const int64_t nidx = idx + (int64_t)dy * P.W + dx;
      if (!(s > sn || (s == sn && idx < nidx))) return;
    }
  for (int yy = y - P.R; yy <= y + P.R; ++yy)
    if (!row_clean(P.bits + (int64_t)yy * P.nwords, x - P.R, x + P.R)) return;
  int rx = (int)(((int64_t)x * P.nx) / P.W);
  rx = min(P.nx - 1, max(0, rx));
  while (rx > 0 && x < (int)(((int64_t)rx * P.W) / P.nx)) --rx;
  while (rx < P.nx - 1 && x >= (int)(((int64_t)(rx + 1) * P.W) / P.nx)) ++rx;
  int ry = (int)(((int64_t)y * P.ny) / P.H);
  ry = min(P.ny - 1, max(0, ry));
  while (ry > 0 && y < (int)(((int64_t)ry * P.H) / P.ny)) --ry;
  while (ry < P.ny - 1 && y >= (int)(((int64_t)(ry + 1) * P.H) / P.ny)) ++ry;
  const int r = ry * P.nx + rx;
  const int slot = atomicAdd(&P.bin_cnt[r], 1);
  if (slot < kBinCap) {
    P.bin_val[(int64_t)r * kBinCap + slot] = s;
    P.bin_idx[(int64_t)r * kBinCap + slot] = (int32_t)idx;
  } else {
    raise_error(P.st, PSFM_ERR_WORKSPACE);
  }
}

// One CTA per subregion: keep the max_cand best detections, ordered.
__global__ void k_rank_candidates(const float* bin_val, const int32_t* bin_idx,
                                  const int32_t* bin_cnt, int W, int max_cand, int32_t* cand,
                                  int32_t* cand_stat, double* cand_chi2, int32_t* ptr,
                                  int32_t* have) {
  __shared__ float v[kBinCap];
  __shared__ int32_t id[kBinCap];
  __shared__ float bv[32];
  __shared__ int32_t bi[32];
  const int r = blockIdx.x, tid = threadIdx.x;
  const int n = min(bin_cnt[r], kBinCap);
  for (int i = tid; i < n; i += blockDim.x) {
    v[i] = bin_val[(int64_t)r * kBinCap + i];
    id[i] = bin_idx[(int64_t)r * kBinCap + i];
  }
  __syncthreads();
  for (int j = 0; j < max_cand; ++j) {
    float best = -INFINITY;
    int32_t bidx = 0x7fffffff;
    for (int i = tid; i < n; i += blockDim.x) {
      if (id[i] < 0) continue;
      if (v[i] > best || (v[i] == best && id[i] < bidx)) {
        best = v[i];
        bidx = id[i];
      }
    }
    for (int off = 16; off > 0; off >>= 1) {
      const float ov = __shfl_xor_sync(0xffffffffu, best, off);
      const int32_t oi = __shfl_xor_sync(0xffffffffu, bidx, off);
      if (ov > best || (ov == best && oi < bidx)) {
        best = ov;
        bidx = oi;
      }
    }
    if ((tid & 31) == 0) {
      bv[tid >> 5] = best;
      bi[tid >> 5] = bidx;
    }
    __syncthreads();
    if (tid == 0) {
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
        if (bv[w] > bv[0] || (bv[w] == bv[0] && bi[w] < bi[0])) {
          bv[0] = bv[w];
          bi[0] = bi[w];
        }
      const int64_t c = (int64_t)r * max_cand + j;
      if (bi[0] != 0x7fffffff) {
        cand[2 * c] = bi[0] % W;
        cand[2 * c + 1] = bi[0] / W;
      } else {
        cand[2 * c] = -1;
        cand[2 * c + 1] = -1;
      }
      cand_stat[c] = PSFM_CAND_UNUSED;
      cand_chi2[c] = __longlong_as_double(0x7ff8000000000000ll);
    }
    __syncthreads();
    const int32_t taken = bi[0];
    for (int i = tid; i < n; i += blockDim.x)
      if (id[i] == taken) id[i] = -1;
    __syncthreads();
  }
  if (tid == 0) {
    ptr[r] = 0;
    have[r] = -1;
  }
}

__global__ void k_init_caller_stamps(int nreg, int W, int H, int32_t* cand, int32_t* cand_stat,
                                     double* cand_chi2, int32_t* ptr, int32_t* have,
                                     DevState* st) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nreg) return;
  const int x = cand[2 * r], y = cand[2 * r + 1];
  if (x < 0 || x >= W || y < 0 || y >= H) raise_error(st, PSFM_ERR_BAD_ARG);
  cand_stat[r] = PSFM_CAND_UNUSED;
  cand_chi2[r] = __longlong_as_double(0x7ff8000000000000ll);
  ptr[r] = 0;
  have[r] = -1;
}

__global__ void k_bad_bits2(const uint16_t* m1, const uint16_t* m2, int W, int64_t pitch,
                            int nwords, uint16_t badmask, uint32_t* bits) {
  const int y = blockIdx.y;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  bool bad = false;
  if (x < W) {
    const int64_t o = (int64_t)y * pitch + x;
    bad = ((m1[o] | m2[o]) & badmask) != 0;
  }
  const uint32_t word = __ballot_sync(0xffffffffu, bad);
  const int wx = x >> 5;
  if ((threadIdx.x & 31) == 0 && wx < nwords) bits[(int64_t)y * nwords + wx] = word;
}

}  // namespace

cudaError_t launch_extract(const Plan& p, DevState* st, const SolveBuffers& b, const float* img,
                           const float* ref, const float* var_img, const float* var_ref,
                           const uint16_t* mask_img, const uint16_t* mask_ref, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(b.hist, 0, sizeof(uint32_t) * 3 * 2048, s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(b.bin_cnt, 0, sizeof(int32_t) * p.nreg, s);
  if (e != cudaSuccess) return e;
  HistParams hp{ref, img, mask_ref, mask_img, p.W, p.H, p.pitch, p.cfg.badmask, 0, b.hist, st};
  for (int pass = 0; pass < 3; ++pass) {
    hp.pass = pass;
    k_median_hist<<<dim3((p.W + 255) / 256, p.H < 256 ? p.H : 256), 256, 0, s>>>(hp);
    k_median_select<<<1, 1024, 0, s>>>(b.hist, pass, st);
  }
  const int nwords = (p.W + 31) / 32;
  k_bad_bits2<<<dim3((p.W + 255) / 256, p.H), 256, 0, s>>>(mask_ref, mask_img, p.W, p.pitch,
                                                          nwords, p.cfg.badmask, b.badbits);
  DetectParams dp;
  dp.i1 = ref;
  dp.i2 = img;
  dp.v1 = var_ref;
  dp.v2 = var_img;
  dp.bits = b.badbits;
  dp.W = p.W;
  dp.H = p.H;
  dp.nwords = nwords;
  dp.pitch = p.pitch;
  dp.R = p.s + p.h;
  dp.nx = p.cfg.grid_nx;
  dp.ny = p.cfg.grid_ny;
  dp.thresh = p.cfg.thresh_nsigma;
  dp.bin_val = b.bin_val;
  dp.bin_idx = b.bin_idx;
  dp.bin_cnt = b.bin_cnt;
  dp.st = st;
  k_detect<<<dim3((p.W + 31) / 32, (p.H + 7) / 8), dim3(32, 8), 0, s>>>(dp);
  k_rank_candidates<<<p.nreg, 256, 0, s>>>(b.bin_val, b.bin_idx, b.bin_cnt, p.W, p.max_cand,
                                          b.cand, b.cand_stat, b.cand_chi2, b.ptr, b.have);
  return cudaGetLastError();
}

cudaError_t launch_caller_stamps(const Plan& p, DevState* st, const SolveBuffers& b,
                                 const psfm_stamp* stamps, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(b.cand, stamps, sizeof(psfm_stamp) * p.nreg,
                                  cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  k_init_caller_stamps<<<(p.nreg + 127) / 128, 128, 0, s>>>(p.nreg, p.W, p.H, b.cand, b.cand_stat,
                                                           b.cand_chi2, b.ptr, b.have, st);
  return cudaGetLastError();
}

}  // namespace psfm
