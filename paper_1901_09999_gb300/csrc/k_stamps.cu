// Stamp candidates (Sec. 3.3): per subregion, the brightest peaks of the detection image
// S = I1 + I2 over a threshold of thresh_nsigma * sqrt(V1 + V2) above the background, with
// no masked pixel in the footprint that the kernel fit reads.
//
//   background: lower median of S over pixels unmasked in both images, found exactly by a
//               three-pass radix select on order-preserving 32-bit keys (11 + 11 + 10 bits):
//               the first pass reads the images and masks once and writes every pixel's key
//               (0 for a masked pixel, a value no finite S takes) and the bad-bit plane, the
//               other two passes and the detection read the 4-byte keys;
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
  int W, H, nwords;
  int64_t pitch;
  uint16_t badmask;
  uint32_t* keys;  // [H][W]
  uint32_t* bits;  // [H][nwords] bad bits of m1 | m2
  uint32_t* hist;
  DevState* st;
};

// Adds a warp's bins to the block histogram: sky pixels crowd into a few bins, so one
// shared-memory atomic per distinct bin per warp.
__device__ __forceinline__ void warp_hist(uint32_t* h, bool valid, uint32_t bin) {
  const unsigned act = __ballot_sync(0xffffffffu, valid);
  if (valid) {
    const unsigned same = __match_any_sync(act, bin);
    if ((int)(threadIdx.x & 31) == __ffs(same) - 1) atomicAdd(&h[bin], (uint32_t)__popc(same));
  }
}

// First pass: keys, bad bits and the histogram of the top 11 key bits.  Rows strided over the
// grid, kKeyRows rows per step with all their loads issued first, one pixel per thread
// (warp-uniform trip count for the warp-wide votes).
constexpr int kKeyRows = 2;
__global__ void __launch_bounds__(256) k_median_keys(HistParams P) {
  __shared__ uint32_t h[2048];
  for (int i = threadIdx.x; i < 2048; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int wx = x >> 5;
  for (int y = blockIdx.y; y < P.H; y += kKeyRows * gridDim.y) {
    int yr[kKeyRows];
    float a[kKeyRows], b[kKeyRows];
    uint16_t m[kKeyRows];
#pragma unroll
    for (int q = 0; q < kKeyRows; ++q) {
      yr[q] = y + q * (int)gridDim.y;
      a[q] = 0.f;
      b[q] = 0.f;
      m[q] = 0;
    }
#pragma unroll
    for (int q = 0; q < kKeyRows; ++q) {
      if (x < P.W && yr[q] < P.H) {
        const int64_t o = (int64_t)yr[q] * P.pitch + x;
        m[q] = P.m1[o] | P.m2[o];
        a[q] = P.i1[o];
        b[q] = P.i2[o];
      }
    }
#pragma unroll
    for (int q = 0; q < kKeyRows; ++q) {
      if (yr[q] >= P.H) break;  // uniform over the block
      bool valid = false, bad = false;
      uint32_t k = 0;
      if (x < P.W) {
        bad = (m[q] & P.badmask) != 0;
        if (!bad) {
          const float sv = a[q] + b[q];
          if (!isfinite(sv)) {
            raise_error(P.st, PSFM_ERR_NONFINITE);
          } else {
            k = fkey(sv);
            valid = true;
          }
        }
        P.keys[(int64_t)yr[q] * P.W + x] = k;
      }
      const uint32_t word = __ballot_sync(0xffffffffu, bad);
      if ((threadIdx.x & 31) == 0 && wx < P.nwords)
        P.bits[(int64_t)yr[q] * P.nwords + wx] = word;
      warp_hist(h, valid, k >> 21);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 2048; i += blockDim.x)
    if (h[i]) atomicAdd(&P.hist[i], h[i]);
}

// Passes 1 and 2 over the key image (4 keys per thread per step, grid-stride).
__global__ void __launch_bounds__(256) k_median_key_hist(const uint32_t* keys, int64_t n,
                                                         int pass, uint32_t* hist,
                                                         const DevState* st) {
  __shared__ uint32_t h[2048];
  for (int i = threadIdx.x; i < 2048; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const uint32_t prefix = st->sel_prefix;
  const int64_t n4 = n >> 2;
  const uint4* k4 = reinterpret_cast<const uint4*>(keys);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // warp-uniform trip count
  const int64_t steps = (n4 + stride - 1) / stride;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint4 nxt = make_uint4(0u, 0u, 0u, 0u);
  if (steps > 0 && i < n4) nxt = k4[i];
  for (int64_t it = 0; it <= steps; ++it, i += stride) {
    uint32_t kv[4] = {0u, 0u, 0u, 0u};
    if (it < steps) {
      kv[0] = nxt.x;
      kv[1] = nxt.y;
      kv[2] = nxt.z;
      kv[3] = nxt.w;
      // the next step's keys are requested before this step's votes
      nxt = make_uint4(0u, 0u, 0u, 0u);
      if (it + 1 < steps && i + stride < n4) nxt = k4[i + stride];
    } else {
      // the last n % 4 keys, one per thread of the first block
      const int64_t j = 4 * n4 + threadIdx.x;
      if (blockIdx.x == 0 && j < n) kv[0] = keys[j];
    }
    // keys that share the selected prefix spread over many bins of the next digit, so each
    // counts with its own shared-memory atomic (no warp-wide grouping)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t k = kv[q];
      const bool valid = k != 0u && (pass == 1 ? (k >> 21) == prefix : (k >> 10) == prefix);
      if (valid) atomicAdd(&h[pass == 1 ? (k >> 10) & 2047u : k & 1023u], 1u);
    }
  }
  __syncthreads();
  uint32_t* g = hist + pass * 2048;
  for (int i2 = threadIdx.x; i2 < 2048; i2 += blockDim.x)
    if (h[i2]) atomicAdd(&g[i2], h[i2]);
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
  const uint32_t* keys;  // [H][W] order-preserving keys of S, 0 where masked
  const float* v1;
  const float* v2;
  const uint32_t* bits;
  int W, H, nwords;
  int64_t pitch;
  int R;  // s + h
  int nx, ny;
  double thresh;
  float thresh32;     // thresh rounded to FP32 (the pre-test only; FP64 is slow here)
  int thresh_nonneg;  // thresh >= 0
  float* bin_val;
  int32_t* bin_idx;
  int32_t* bin_cnt;
  int32_t* over;      // [cap] linear indices of the pixels above the threshold
  int32_t* n_over;    // their count
  int64_t over_cap;
  DevState* st;
};

// Phase 1 of the detection: the threshold test of one pixel given its key and variances,
// loaded by the caller; true when the pixel goes on to the peak and footprint tests.
__device__ __forceinline__ bool above_threshold(const DetectParams& P, int x, int y,
                                                uint32_t key, float v1, float v2, float medf) {
  if (x < P.R || x >= P.W - P.R || y < P.R || y >= P.H - P.R) return false;
  if (key == 0u) return false;  // a masked centre fails its own footprint test
  const float s = fkey_inv(key);  // the same FP32 value as I1 + I2
  // with thresh >= 0 the threshold is >= 0 (or NaN, which fails too): at or below the median
  // never passes
  if (P.thresh_nonneg && !(s > medf)) return false;
  // FP32 pre-test with a margin far above FP32 rounding: pixels well below the threshold
  // skip the FP64 test (FP64 runs at 1/64 of the FP32 rate here); the decision itself is
  // always the FP64 one
  const float t32 = P.thresh32 * sqrtf(v1 + v2);
  if (isfinite(t32) && isfinite(s) && s - medf < 0.999f * t32) return false;
  const double thr = P.thresh * sqrt((double)v1 + (double)v2);
  return (double)s - (double)medf > thr;
}

// Block 32 x 8 threads covering 32 x (8 kDetRows) pixels: each thread tests rows y, y + 8, ...
// (all loads issued first); the pixels that pass are appended to the candidate list, one
// atomic per warp.
constexpr int kDetRows = 4;
__global__ void __launch_bounds__(256) k_detect(DetectParams P) {
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y0 = blockIdx.y * (8 * kDetRows) + threadIdx.y;
  if (P.st->error) return;
  const float medf = fkey_inv(P.st->median_key);
  uint32_t key[kDetRows];
  float v1[kDetRows], v2[kDetRows];
#pragma unroll
  for (int q = 0; q < kDetRows; ++q) {
    key[q] = 0u;
    v1[q] = 0.f;
    v2[q] = 0.f;
  }
#pragma unroll
  for (int q = 0; q < kDetRows; ++q) {
    const int y = y0 + 8 * q;
    if (x < P.W && y < P.H) {
      const int64_t o = (int64_t)y * P.pitch + x;
      key[q] = P.keys[(int64_t)y * P.W + x];
      v1[q] = P.v1[o];
      v2[q] = P.v2[o];
    }
  }
  const int lane = threadIdx.x;
#pragma unroll
  for (int q = 0; q < kDetRows; ++q) {
    const int y = y0 + 8 * q;
    const bool pass = above_threshold(P, x, y, key[q], v1[q], v2[q], medf);
    const unsigned bal = __ballot_sync(0xffffffffu, pass);
    if (!bal) continue;
    int base = 0;
    if (lane == 0) base = atomicAdd(P.n_over, __popc(bal));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (pass) {
      const int64_t slot = base + __popc(bal & ((1u << lane) - 1u));
      if (slot < P.over_cap)
        P.over[slot] = y * P.W + x;
      else
        raise_error(P.st, PSFM_ERR_WORKSPACE);
    }
  }
}

// Phase 2: one warp per candidate.  Lanes 0..7 compare the 8 neighbours (strict peak under
// (value, -index)), all lanes check rows of the footprint for bad bits, and lane 0 puts a
// peak with a clean footprint in its subregion's bin.
__global__ void __launch_bounds__(256) k_detect_peaks(DetectParams P) {
  if (P.st->error) return;
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int n = min((int64_t)*P.n_over, P.over_cap);
  for (int64_t c = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < n; c += nw) {
    const int idx = P.over[c];
    const int y = idx / P.W, x = idx - y * P.W;
    const int64_t o = (int64_t)y * P.pitch + x;
    const float s = P.i1[o] + P.i2[o];
    bool ok = true;
    if (lane < 8) {
      const int d = lane < 4 ? lane : lane + 1;  // skip the centre of the 3 x 3
      const int dy = d / 3 - 1, dx = d % 3 - 1;
      const int64_t on = o + (int64_t)dy * P.pitch + dx;
      const float sn = P.i1[on] + P.i2[on];
      const int64_t nidx = (int64_t)idx + (int64_t)dy * P.W + dx;
      ok = s > sn || (s == sn && idx < nidx);
    }
    for (int yy = y - P.R + lane; yy <= y + P.R; yy += 32)
      ok = ok && row_clean(P.bits + (int64_t)yy * P.nwords, x - P.R, x + P.R);
    if (!__all_sync(0xffffffffu, ok) || lane != 0) continue;
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
      P.bin_idx[(int64_t)r * kBinCap + slot] = idx;
    } else {
      raise_error(P.st, PSFM_ERR_WORKSPACE);
    }
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

}  // namespace

cudaError_t launch_extract(const Plan& p, DevState* st, const SolveBuffers& b, const float* img,
                           const float* ref, const float* var_img, const float* var_ref,
                           const uint16_t* mask_img, const uint16_t* mask_ref, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(b.hist, 0, sizeof(uint32_t) * 3 * 2048, s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(b.bin_cnt, 0, sizeof(int32_t) * p.nreg, s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(b.n_over, 0, sizeof(int32_t), s);
  if (e != cudaSuccess) return e;
  const int nwords = (p.W + 31) / 32;
  HistParams hp;
  hp.i1 = ref;
  hp.i2 = img;
  hp.m1 = mask_ref;
  hp.m2 = mask_img;
  hp.W = p.W;
  hp.H = p.H;
  hp.nwords = nwords;
  hp.pitch = p.pitch;
  hp.badmask = p.cfg.badmask;
  hp.keys = b.keys;
  hp.bits = b.badbits;
  hp.hist = b.hist;
  hp.st = st;
  k_median_keys<<<dim3((p.W + 255) / 256, p.H < 256 ? p.H : 256), 256, 0, s>>>(hp);
  k_median_select<<<1, 1024, 0, s>>>(b.hist, 0, st);
  const int64_t npx = (int64_t)p.W * p.H;
  const int64_t blocks = ((npx >> 2) + 255) / 256;
  const unsigned grid = (unsigned)(blocks < 1 ? 1 : (blocks > 1216 ? 1216 : blocks));
  for (int pass = 1; pass < 3; ++pass) {
    k_median_key_hist<<<grid, 256, 0, s>>>(b.keys, npx, pass, b.hist, st);
    k_median_select<<<1, 1024, 0, s>>>(b.hist, pass, st);
  }
  DetectParams dp;
  dp.i1 = ref;
  dp.i2 = img;
  dp.keys = b.keys;
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
  dp.thresh32 = (float)p.cfg.thresh_nsigma;
  dp.thresh_nonneg = p.cfg.thresh_nsigma >= 0.0;
  dp.bin_val = b.bin_val;
  dp.bin_idx = b.bin_idx;
  dp.bin_cnt = b.bin_cnt;
  dp.st = st;
  dp.over = b.over;
  dp.n_over = b.n_over;
  dp.over_cap = over_capacity(p);
  k_detect<<<dim3((p.W + 31) / 32, (p.H + 8 * kDetRows - 1) / (8 * kDetRows)), dim3(32, 8), 0, s>>>(
      dp);
  k_detect_peaks<<<1216, 256, 0, s>>>(dp);
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
