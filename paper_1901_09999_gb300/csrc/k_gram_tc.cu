// Weighted Gram of the stamp design blocks on the 5th-generation tensor cores (Eq. 5-6:
// M_s = C_s^T W_s C_s over the stamp pixels, W = 1 / (V1 + V2)), in the two reduced-precision
// forms of the precision study: TF32 products, and BF16 products of a hi/lo split
// (a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi), both accumulated in FP32 in tensor memory.
//
// One CTA of 128 threads per stamp.  The augmented columns (basis columns C_k, the masked
// reference R, the constant 1 and I2) form A (M = 128 rows, Nc of them used, K = pixels) and
// the weighted columns W A form B (N = 64 or 128 rows); D = A B^T is the Gram.  Pixels are
// staged 32 at a time into a double-buffered shared-memory tile in the canonical K-major
// layout without swizzle (8-row x 16-byte core matrices), one thread issues the MMAs, and
// tcgen05.commit arrives on the buffer's mbarrier when they have consumed it.  Every wait is
// bounded: a wait that runs out records PSFM_ERR_TIMEOUT and the CTA still frees its tensor
// memory before it returns.
#include <algorithm>

#include <cuda_bf16.h>

#include "psfm_internal.h"
#include "solve.h"
#include "stamp.h"

namespace psfm {
namespace {

constexpr int kTcThreads = 128;
constexpr int kTcM = 128;   // rows of A (TMEM lanes)
constexpr int kTcKC = 32;   // pixels per staged chunk
constexpr uint32_t kTcSpinLimit = PSFM_WAIT_LIMIT_DEFAULT;

// Poll limit of the pipeline waits (a buffer's previous MMAs done before it is refilled).  The
// final drain wait always uses kTcSpinLimit, so that every MMA issued has completed before the
// tensor memory is freed, whatever this is set to.
__device__ uint32_t g_pipe_wait_limit = kTcSpinLimit;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: start address, leading (K-direction) and stride
// (M/N-direction) byte offsets between core matrices, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) |
         ((uint64_t)(sbo >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor: FP32 accumulator, A/B format, both K-major, N, M.
__device__ __forceinline__ uint32_t instr_desc(uint32_t ab_format, int n, int m) {
  return (1u << 4) | (ab_format << 7) | (ab_format << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

// Bounded wait (at most `limit` polls) for the phase with the given parity; false if it ran
// out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          uint32_t limit = kTcSpinLimit) {
  const uint32_t a = smem_u32(bar);
  for (uint32_t it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

template <int KIND>  // 0: kind::tf32, 1: kind::f16 (BF16 operands)
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                       uint32_t idesc, uint32_t accumulate) {
  if (KIND == 0)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// 16 consecutive FP32 columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 8 consecutive FP32 columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tc_ld8(uint32_t taddr, float v[8]) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// Byte offset of element (row, k) of a K-major operand tile with kTcKC columns, built from
// 8-row x 16-byte core matrices stored row group by row group: LBO = 128 B (next core matrix
// along K), SBO = (kTcKC * esz / 16) * 128 B (next group of 8 rows).
template <int ESZ>
__device__ __forceinline__ uint32_t tile_off(int row, int k) {
  constexpr int per = 16 / ESZ;  // elements per core-matrix row
  return (uint32_t)(((row >> 3) * (kTcKC / per) + k / per) * 128 + (row & 7) * 16 + (k % per) * ESZ);
}

__device__ __forceinline__ uint16_t bf16_bits(float x) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}

// Column source of the stamp Grams inside the solve: zero-sum basis columns psi_k C_k - s_k R
// from the FP32 design block, then R (masked), 1 and I2 read from the images at the stamp
// pixels, weights 1 / (V1 + V2) (0 at masked or off-image pixels).  After the Gram it marks
// the stamp's block as cached.
struct StampSource {
  StampParams P;
  int r, cx, cy;
  __device__ bool open(int blk) {
    r = blk;
    if (P.st->error || P.st->done) return false;
    if (!region_active(P.ptr, P.cand, r, P.max_cand, &cx, &cy)) return false;
    return P.have[r] != P.ptr[r];
  }
  __device__ int ncols() const { return P.Nc; }
  __device__ int npix() const { return P.P; }
  __device__ bool pixel(int pix, int64_t* o) const {
    const int py = pix / P.sw, px = pix - py * P.sw;
    const int gx = cx - P.s + px, gy = cy - P.s + py;
    if (gx < 0 || gx >= P.g.W || gy < 0 || gy >= P.g.H) return false;
    *o = (int64_t)gy * P.g.pitch + gx;
    return true;
  }
  __device__ float weight(int pix) const {
    int64_t o;
    if (pix >= P.P || !pixel(pix, &o) || ((P.m1[o] | P.m2[o]) & P.badmask)) return 0.f;
    const float a = P.i1[o], b = P.i2[o];
    const double wd = 1.0 / ((double)P.v1[o] + (double)P.v2[o]);
    if (!isfinite(a) || !isfinite(b) || !isfinite(wd)) raise_error(P.st, PSFM_ERR_NONFINITE);
    return (float)wd;
  }
  __device__ float value(int c, int pix) const {
    if (pix >= P.P) return 0.f;
    const int Nb = P.b.Nb;
    int64_t o;
    const bool on = pixel(pix, &o);
    const float xr = (on && !(P.m1[o] & P.badmask)) ? P.i1[o] : 0.f;
    if (c < Nb) {  // zero-sum design column psi_k C_k - s_k R, formed per pixel
      const float cv = reinterpret_cast<const float*>(P.C)[((int64_t)r * Nb + c) * P.P + pix];
      return (float)P.psi[c] * cv - (float)P.sk[c] * xr;
    }
    if (!on) return 0.f;
    if (c == Nb) return xr;
    if (c == Nb + 1) return 1.f;
    return P.i2[o];
  }
  // the Gram of the zero-sum columns is the transformed Gram the system is assembled from
  __device__ double* gram() const { return P.Gt + (int64_t)r * P.Nc * P.Nc; }
  __device__ void fail(int code) const { atomicCAS(&P.st->error, 0, code); }
  __device__ void finish(int tid, int nthreads) const {
    if (tid == 0) {
      P.have[r] = P.ptr[r];
      P.fresh[r] = 1;
    }
  }
};

// Column source of psfm_gram: caller blocks cols [blk][c][pix] and weights [blk][pix].
struct PlainSource {
  const float* cols;
  const float* w;
  double* G;
  int32_t* status;
  int n_cols, n_pix, r;
  __device__ bool open(int blk) {
    r = blk;
    return true;
  }
  __device__ int ncols() const { return n_cols; }
  __device__ int npix() const { return n_pix; }
  __device__ float weight(int pix) const {
    return pix < n_pix ? w[(int64_t)r * n_pix + pix] : 0.f;
  }
  __device__ float value(int c, int pix) const {
    return pix < n_pix ? cols[((int64_t)r * n_cols + c) * n_pix + pix] : 0.f;
  }
  __device__ double* gram() const { return G + (int64_t)r * n_cols * n_cols; }
  __device__ void fail(int code) const { atomicCAS(status, 0, code); }
  __device__ void finish(int, int) const {}
};

// MODE 0: TF32; MODE 1: BF16 hi/lo split with three products.  One block of 128 threads per
// column block (stamp).
template <int MODE, class Src>
__global__ void __launch_bounds__(kTcThreads) k_gram_tc(Src src, int n_tile) {
  constexpr int ESZ = MODE == 0 ? 4 : 2;
  constexpr int NOPS = MODE == 0 ? 1 : 2;  // operand planes: value, or hi and lo
  extern __shared__ __align__(1024) unsigned char tc_sh[];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ uint32_t s_tmem;
  __shared__ float wsm[kTcKC];
  __shared__ int s_ok, s_last, s_open;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // block-uniform early exit (finished loop, error, inactive region or cached Gram)
  if (tid == 0) s_open = src.open(blockIdx.x) ? 1 : 0;
  __syncthreads();
  if (!s_open) return;
  if (tid != 0) src.open(blockIdx.x);
  const int Nc = src.ncols(), npix = src.npix();
  const uint32_t a_bytes = kTcM * kTcKC * ESZ, b_bytes = (uint32_t)n_tile * kTcKC * ESZ;
  const uint32_t stage_bytes = NOPS * (a_bytes + b_bytes);
  // stage s: [A planes][B planes]
  auto a_plane = [&](int s, int o) { return tc_sh + s * stage_bytes + o * a_bytes; };
  auto b_plane = [&](int s, int o) {
    return tc_sh + s * stage_bytes + NOPS * a_bytes + o * b_bytes;
  };
  // rows >= Nc stay zero for the whole kernel
  for (uint32_t i = tid; i < 2 * stage_bytes / 4; i += kTcThreads)
    reinterpret_cast<uint32_t*>(tc_sh)[i] = 0u;
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_ok = 1;
    s_last = -1;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&s_tmem)),
                 "r"(n_tile)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  const uint32_t idesc = instr_desc(MODE == 0 ? 2u : 1u, n_tile, kTcM);
  const uint32_t sbo = (kTcKC * ESZ / 16) * 128;
  const int kstep = MODE == 0 ? 8 : 16;  // K of one MMA
  const int nchunk = (npix + kTcKC - 1) / kTcKC;
  const uint32_t pipe_limit = g_pipe_wait_limit;
  for (int ch = 0; ch < nchunk; ++ch) {
    const int s = ch & 1;
    // the MMAs that read this buffer two chunks ago must be done before it is rewritten
    if (ch >= 2 && !mbar_wait(&bars[s], ((ch - 2) >> 1) & 1, pipe_limit) && tid == 0) s_ok = 0;
    __syncthreads();
    if (!s_ok) break;
    const int base = ch * kTcKC;
    if (tid < kTcKC) wsm[tid] = src.weight(base + tid);
    __syncthreads();
    for (int i = tid; i < Nc * kTcKC; i += kTcThreads) {
      const int c = i / kTcKC, j = i - c * kTcKC;
      const float v = src.value(c, base + j);
      const float b = wsm[j] * v;
      const uint32_t oa = tile_off<ESZ>(c, j);
      if (MODE == 0) {
        *reinterpret_cast<float*>(a_plane(s, 0) + oa) = v;
        *reinterpret_cast<float*>(b_plane(s, 0) + oa) = b;
      } else {
        const float vh = __bfloat162float(__float2bfloat16_rn(v));
        const float bh = __bfloat162float(__float2bfloat16_rn(b));
        *reinterpret_cast<uint16_t*>(a_plane(s, 0) + oa) = bf16_bits(vh);
        *reinterpret_cast<uint16_t*>(a_plane(s, 1) + oa) = bf16_bits(v - vh);
        *reinterpret_cast<uint16_t*>(b_plane(s, 0) + oa) = bf16_bits(bh);
        *reinterpret_cast<uint16_t*>(b_plane(s, 1) + oa) = bf16_bits(b - bh);
      }
    }
    // make the generic-proxy stores visible to the tensor cores' reads
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      for (int k0 = 0; k0 < kTcKC; k0 += kstep) {
        const uint32_t koff = (uint32_t)(k0 / (16 / ESZ)) * 128;
        const uint64_t ah = smem_desc(smem_u32(a_plane(s, 0)) + koff, 128, sbo);
        const uint64_t bh = smem_desc(smem_u32(b_plane(s, 0)) + koff, 128, sbo);
        tc_mma<MODE>(tmem, ah, bh, idesc, (ch > 0 || k0 > 0) ? 1u : 0u);
        if (MODE == 1) {
          const uint64_t al = smem_desc(smem_u32(a_plane(s, 1)) + koff, 128, sbo);
          const uint64_t bl = smem_desc(smem_u32(b_plane(s, 1)) + koff, 128, sbo);
          tc_mma<MODE>(tmem, ah, bl, idesc, 1u);
          tc_mma<MODE>(tmem, al, bh, idesc, 1u);
        }
      }
      tc_commit(&bars[s]);
      s_last = ch;
    }
  }
  __syncthreads();
  // the last commit covers every MMA issued before it; after a timeout this still waits
  // (bounded) for the MMAs in flight before the tensor memory is freed
  const int last = s_last;
  const bool drained = last < 0 || mbar_wait(&bars[last & 1], (last >> 1) & 1);
  __syncthreads();
  if (!drained && tid == 0) s_ok = 0;
  __syncthreads();
  tc_fence_after();
  const bool ok = s_ok != 0 && last == nchunk - 1;
  double* Gr = src.gram();
  if (ok) {
    const int row = warp * 32 + lane;  // TMEM lane = row of D
    for (int c0 = 0; c0 < n_tile; c0 += 16) {
      float v[16];
      tc_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const int col = c0 + e;
        if (row < Nc && col <= row) {
          Gr[row * Nc + col] = (double)v[e];
          Gr[col * Nc + row] = (double)v[e];
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(n_tile)
                 : "memory");
  if (!ok) {
    if (tid == 0) src.fail(PSFM_ERR_TIMEOUT);
    return;
  }
  __syncthreads();
  src.finish(tid, kTcThreads);
}

// ---- Tensor-core Gram with error-free split products (precision mode BF16X6) ----
//
// The Gram A^T W A is formed as (sqrt(w) A)^T (sqrt(w) A): each augmented column c of the stamp
// (the zero-sum design columns in double-float, R, 1, I2) times sqrt(w) per pixel is scaled by a
// power of two so that its largest value is below 1/4 and written as seven signed base-256
// digits, x = sum_k d_k 2^(-8(k+1)), |d_k| <= 129, each digit times its weight held exactly by a
// BF16 slice: 56 bits below the column's largest value, enough for the 48 bits of a
// double-float value a hundred times smaller.  The product of slices i and j is exact in the
// tensor cores and has the weight 2^(-8(i+j+2)) of its level L = i + j; the B operand of each
// MMA is the first 64 rows of a slice of the same operand.  Levels 0..4 are accumulated in
// their own tensor-memory tiles over groups of 224 pixels, where every partial sum is an
// integer below 2^24 units of the level (|d_0| <= 64, |d_k| <= 129: at most 66435 units a pixel
// on level 4) and so exact in FP32; after each group they are read back and added, as integers,
// into a 64-bit accumulator per Gram entry.  Levels 5 and 6 (weights 2^-56, 2^-64) share one FP32
// tile over the whole stamp (with only four exact levels, the FP32 rounding of the shared tile
// was the largest error of this symmetric form, 3e-14 of the sum of |terms| in an emulation on
// full-chip stamps; with five it is 1.7e-15).  The Gram entry is the integer sum
// plus the small levels, times the two column scales: it carries the bits of its double-float
// inputs while the products run on the tensor cores.  One CTA of 32 warps per stamp: warp 0
// issues the MMAs of a 32-pixel chunk while the other 31 stage the next chunk's slices (triple
// buffered); all 32 read the accumulators back (a thread: 8 columns of one accumulator lane);
// at most 64 columns (one N = 64 tile).
constexpr int kOzSlices = 7;
constexpr int kOzExact = 5;  // levels summed exactly per group
constexpr int kOzGroup = 7;  // 32-pixel sub-chunks per exact group (224 pixels)
constexpr int kOzThreads = 1024;
// elements of a 64-column chunk per staging thread (all warps but the MMA warp), and elements
// per thread per round of the column-scale scan
constexpr int kOzPer = (64 * kTcKC + kOzThreads - 32 - 1) / (kOzThreads - 32);
constexpr int kOzScanBatch = 4;
// staging buffers (chunk ch waits for the MMAs of chunk ch - kOzStages before refilling)
constexpr int kOzStages = 3;

// seven balanced base-256 digits of the double-float h + l (|h + l| < 1/4), as BF16 bits of
// d_k 2^(-8(k+1)).  Each digit is taken from the high part alone (d = rint(h 2^(8(k+1))), and
// h - d 2^(-8(k+1)) is exact); the low part is folded in by an error-free sum before digits 2,
// 4 and 6, while it is still below half a unit of the next digit, so |d_k| <= 129.  d 2^-8(k+1)
// has at most eight significant bits, so its BF16 bits are the top half of its FP32 bits.
__device__ __forceinline__ void oz_digits(float h, float l, uint16_t out[kOzSlices]) {
#pragma unroll
  for (int k = 0; k < kOzSlices; ++k) {
    if (k == 2 || k == 4 || k == 6) {
      const float s2 = __fadd_rn(h, l);
      const float bb = __fsub_rn(s2, h);
      l = __fadd_rn(__fsub_rn(h, __fsub_rn(s2, bb)), __fsub_rn(l, bb));
      h = s2;
    }
    const float sc = __int_as_float((127 + 8 * (k + 1)) << 23);   // 2^(8(k+1))
    const float isc = __int_as_float((127 - 8 * (k + 1)) << 23);  // 2^(-8(k+1))
    const float dv = __fmul_rn(rintf(__fmul_rn(h, sc)), isc);
    out[k] = (uint16_t)(__float_as_uint(dv) >> 16);
    h = __fsub_rn(h, dv);
  }
}

// Column source of the split Gram inside the solve: double-float design block (zero-sum
// columns formed per pixel), R, 1, I2; sqrt(1 / (V1 + V2)) as double-floats.  prepare()
// stages the stamp's per-pixel weights and image values and the per-column psi_k and s_k in
// shared memory once, so that the two passes over the stamp read only the design block.
struct OzStampSource {
  StampParams P;
  // nsplit > 1: block blk takes part blk % nsplit (a range of 32-pixel chunks) of stamp
  // blk / nsplit and writes a partial Gram; the last part to finish adds the partials
  int nsplit;
  int r, cx, cy, part, pix0, np;
  float *wh, *wl, *xr, *xi, *ph, *pl, *sh, *sl;  // shared memory, set by prepare()
  __device__ bool open(int blk) {
    r = blk / nsplit;
    part = blk - r * nsplit;
    const int nch = (P.P + kTcKC - 1) / kTcKC;  // >= nsplit (checked by the launch)
    pix0 = (part * nch / nsplit) * kTcKC;
    np = min(((part + 1) * nch / nsplit) * kTcKC, P.P) - pix0;
    if (P.st->error || P.st->done) return false;
    if (!region_active(P.ptr, P.cand, r, P.max_cand, &cx, &cy)) return false;
    return P.have[r] != P.ptr[r];
  }
  __device__ int ncols() const { return P.Nc; }
  __device__ int npix() const { return np; }
  __host__ __device__ static size_t prep_floats(int npix, int nd) {
    return 4 * (size_t)npix + 4 * (size_t)nd;
  }
  __device__ void bind(float* sm) {
    const int n = P.P, nd = P.Nd;
    wh = sm;
    wl = wh + n;
    xr = wl + n;
    xi = xr + n;
    ph = xi + n;
    pl = ph + nd;
    sh = pl + nd;
    sl = sh + nd;
  }
  __device__ void prepare(int tid, int nthr) {
    for (int lp = tid; lp < np; lp += nthr) {
      const int pix = pix0 + lp;
      const int py = pix / P.sw, px = pix - py * P.sw;
      const int gx = cx - P.s + px, gy = cy - P.s + py;
      float a = 0.f, b = 0.f, h = 0.f, l = 0.f;
      if (gx >= 0 && gx < P.g.W && gy >= 0 && gy < P.g.H) {
        const int64_t o = (int64_t)gy * P.g.pitch + gx;
        a = (P.m1[o] & P.badmask) ? 0.f : P.i1[o];
        b = P.i2[o];
        if (!((P.m1[o] | P.m2[o]) & P.badmask)) {
          // sqrt(w) = (V1 + V2)^(-1/2): the FP32 estimate and two Newton steps in FP64
          // (FP64 division and square root are slow here); the Gram is formed as
          // (sqrt(w) A)^T (sqrt(w) A)
          const double vs = (double)P.v1[o] + (double)P.v2[o];
          double sq;
          if (vs > 1e-30 && vs < 1e30) {
            sq = (double)rsqrtf((float)vs);
            sq = sq * (1.5 - 0.5 * vs * sq * sq);
            sq = sq * (1.5 - 0.5 * vs * sq * sq);
          } else {
            sq = 1.0 / sqrt(vs);  // outside the FP32 estimate's range
          }
          if (!isfinite(P.i1[o]) || !isfinite(b) || !(vs > 0.0) || !isfinite(sq))
            raise_error(P.st, PSFM_ERR_NONFINITE);
          h = (float)sq;
          l = (float)(sq - (double)h);
        }
      }
      xr[lp] = a;
      xi[lp] = b;
      wh[lp] = h;
      wl[lp] = l;
    }
    const int nbk = P.b.Nb;
    for (int c = tid; c < P.Nd; c += nthr) {
      const int k = c < nbk ? c : c - nbk;
      const double psd = P.psi[k], skd = P.sk[k];
      ph[c] = (float)psd;
      pl[c] = (float)(psd - (double)ph[c]);
      sh[c] = (float)skd;
      sl[c] = (float)(skd - (double)sh[c]);
    }
  }
  // pixel indices from here on are the part's (0 .. np - 1)
  __device__ void weight(int pix, float* h, float* l) const {
    *h = pix < np ? wh[pix] : 0.f;
    *l = pix < np ? wl[pix] : 0.f;
  }
  // the design value of column c at pixel pix (the global load, issued ahead of its use)
  __device__ float2 fetch(int c, int pix) const {
    if (pix >= np || c >= P.Nd) return make_float2(0.f, 0.f);
    return reinterpret_cast<const float2*>(P.C)[((int64_t)r * P.Nd + c) * P.P + pix0 + pix];
  }
  __device__ void make(int c, int pix, float2 cv, float* vh, float* vl) const {
    *vh = 0.f;
    *vl = 0.f;
    if (pix >= np || c >= P.Nc) return;
    const int Nd = P.Nd, nbk = P.b.Nb;
    if (c < Nd) {
      // psi C - s X in double-float, X = masked R (or I2 for the dual kernel's terms)
      const float pa = ph[c], pb = pl[c];
      float h = __fmul_rn(pa, cv.x);
      float e = __fmaf_rn(pa, cv.x, -h);
      e = __fmaf_rn(pa, cv.y, e);
      e = __fmaf_rn(pb, cv.x, e);
      const float sa = sh[c];
      if (sa != 0.f) {
        const float x = c < nbk ? xr[pix] : xi[pix], sb = sl[c];
        const float q = __fmul_rn(sa, x);
        const float qe = __fmaf_rn(sb, x, __fmaf_rn(sa, x, -q));
        const float s2 = __fsub_rn(h, q);
        const float bb = __fsub_rn(s2, h);
        const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(s2, bb)), __fsub_rn(-q, bb));
        h = s2;
        e = __fadd_rn(e, __fsub_rn(err, qe));
      }
      const float s2 = __fadd_rn(h, e);
      *vh = s2;
      *vl = __fsub_rn(e, __fsub_rn(s2, h));
      return;
    }
    if (c == Nd) *vh = xr[pix];
    else if (c == Nd + 1) *vh = 1.f;
    else *vh = xi[pix];
  }
  __device__ double* gram() const {
    const int64_t n2 = (int64_t)P.Nc * P.Nc;
    return nsplit == 1 ? P.Gt + r * n2 : P.Gpart + ((int64_t)r * kGramSplit + part) * n2;
  }
  __device__ void fail(int code) const { atomicCAS(&P.st->error, 0, code); }
  // after the block's Gram (or partial) is written, by every thread of the block
  __device__ void finish(int tid) const {
    if (nsplit > 1) {
      __shared__ int s_lastp;
      __threadfence();
      __syncthreads();
      if (tid == 0) s_lastp = atomicAdd(&P.gram_count[r], 1) == nsplit - 1;
      __syncthreads();
      if (!s_lastp) return;
      __threadfence();
      // the partials added in part order, so the Gram does not depend on which part ends last
      const int n2 = P.Nc * P.Nc;
      const double* Gp0 = P.Gpart + (int64_t)r * kGramSplit * n2;
      double* Gr = P.Gt + (int64_t)r * n2;
      for (int q = tid; q < n2; q += blockDim.x) {
        double v = 0.0;
        for (int k = 0; k < nsplit; ++k) v += __ldcg(Gp0 + (int64_t)k * n2 + q);
        Gr[q] = v;
      }
      __syncthreads();
      if (tid == 0) P.gram_count[r] = 0;
    }
    if (tid == 0) {
      P.have[r] = P.ptr[r];
      P.fresh[r] = 1;
    }
  }
};

// Column source of psfm_gram in the split mode: caller FP32 columns and weights (exact).
struct OzPlainSource {
  const float* cols;
  const float* w;
  double* G;
  int32_t* status;
  int n_cols, n_pix, r;
  __device__ bool open(int blk) {
    r = blk;
    return true;
  }
  __device__ int ncols() const { return n_cols; }
  __device__ int npix() const { return n_pix; }
  __host__ __device__ static size_t prep_floats(int, int) { return 0; }
  __device__ void bind(float*) {}
  __device__ void prepare(int, int) {}
  // sqrt(w) as a double-float (the Gram is formed as (sqrt(w) A)^T (sqrt(w) A))
  __device__ void weight(int pix, float* wh, float* wl) const {
    const double sq = pix < n_pix ? sqrt((double)w[(int64_t)r * n_pix + pix]) : 0.0;
    *wh = (float)sq;
    *wl = (float)(sq - (double)*wh);
  }
  __device__ float2 fetch(int c, int pix) const {
    return make_float2(
        (pix < n_pix && c < n_cols) ? cols[((int64_t)r * n_cols + c) * n_pix + pix] : 0.f, 0.f);
  }
  __device__ void make(int, int, float2 cv, float* vh, float* vl) const {
    *vh = cv.x;
    *vl = 0.f;
  }
  __device__ double* gram() const { return G + (int64_t)r * n_cols * n_cols; }
  __device__ void fail(int code) const { atomicCAS(status, 0, code); }
  __device__ void finish(int) const {}
};

// (h, l) * (a, b) in double-float
__device__ __forceinline__ void oz_mul(float h, float l, float a, float b, float* rh, float* rl) {
  const float p = __fmul_rn(h, a);
  float e = __fmaf_rn(h, a, -p);
  e = __fmaf_rn(h, b, e);
  e = __fmaf_rn(l, a, e);
  const float s2 = __fadd_rn(p, e);
  *rh = s2;
  *rl = __fsub_rn(e, __fsub_rn(s2, p));
}

// Element e of a chunk's staging (64 rows x kTcKC pixels) as (row c, pixel j): each warp's 32
// consecutive elements are 4 rows x 8 pixels of one core matrix, 64 contiguous bytes of the
// K-major tile, so its 16-bit stores hit distinct banks.  Rows >= 64 (e >= 2048) map past
// every column.
__device__ __forceinline__ void oz_elem(int e, int* c, int* j) {
  const int w = e >> 5, l = e & 31;
  const int a = w >> 3, b = (w >> 1) & 3, h = w & 1;
  *c = 8 * a + 4 * h + (l >> 3);
  *j = 8 * b + (l & 7);
}

// Power-of-two scale putting max |x| below 1/4 (2^-e with e = ilogb(max) + 3), as the exponent.
__device__ __forceinline__ int oz_exponent(float m) {
  if (!(m > 0.f) || !isfinite(m)) return 0;
  return ilogbf(m) + 3;
}

template <class Src>
__global__ void __launch_bounds__(kOzThreads, 1) k_gram_oz(Src src, int n_tile) {
  constexpr int ESZ = 2;
  extern __shared__ __align__(1024) unsigned char tc_sh[];
  __shared__ __align__(8) uint64_t bars[kOzStages];
  __shared__ uint32_t s_tmem;
  __shared__ unsigned int s_maxa[kTcM];
  __shared__ int s_ea[kTcM];
  __shared__ int s_ok, s_last, s_open;
  const int tid = threadIdx.x, nthr = blockDim.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) s_open = src.open(blockIdx.x) ? 1 : 0;
  __syncthreads();
  if (!s_open) return;
  if (tid != 0) src.open(blockIdx.x);
  const int Nc = src.ncols(), npix = src.npix();
  // one operand: the slices of sqrt(w) A; the B operand of every MMA is the first n_tile rows
  // of an A slice (the same K-major layout)
  constexpr uint32_t a_bytes = kTcM * kTcKC * ESZ;
  const uint32_t stage_bytes = kOzSlices * a_bytes;
  auto a_plane = [&](int s, int k) { return tc_sh + s * stage_bytes + k * a_bytes; };
  // ---- column scales: the largest |sqrt(w) value| of every column (FP32 estimates)
  for (int c = tid; c < kTcM; c += nthr) s_maxa[c] = 0u;
  for (uint32_t i = tid; i < kOzStages * stage_bytes / 4; i += nthr)
    reinterpret_cast<uint32_t*>(tc_sh)[i] = 0u;  // rows >= Nc stay zero throughout
  src.bind(reinterpret_cast<float*>(tc_sh + kOzStages * stage_bytes));
  src.prepare(tid, nthr);
  __syncthreads();
  // Each thread takes one pixel (then the pixel nthr further on) and kOzScanBatch columns at a
  // time, their loads issued together; a warp's lanes share the column, so one warp reduction
  // and one shared-memory atomic per column and warp.  The trip counts are the same for every
  // lane of a warp (the warp reductions need all 32).
  for (int p0 = 0; p0 < npix; p0 += nthr) {
    const int pix = p0 + tid;
    float wh = 0.f, wl = 0.f;
    src.weight(pix, &wh, &wl);
    for (int c0 = 0; c0 < Nc; c0 += kOzScanBatch) {
      float2 cv[kOzScanBatch];
#pragma unroll
      for (int u = 0; u < kOzScanBatch; ++u)
        cv[u] = (pix < npix && c0 + u < Nc) ? src.fetch(c0 + u, pix) : make_float2(0.f, 0.f);
#pragma unroll
      for (int u = 0; u < kOzScanBatch; ++u) {
        const int c = c0 + u;
        if (c >= Nc) break;  // uniform
        unsigned ua = 0u;  // |sqrt(w) value| as order-preserving bits (>= 0)
        if (pix < npix) {
          float vh, vl;
          src.make(c, pix, cv[u], &vh, &vl);
          ua = __float_as_uint(fabsf(vh * wh));
        }
        ua = __reduce_max_sync(0xffffffffu, ua);
        if (lane == 0 && ua) atomicMax(&s_maxa[c], ua);
      }
    }
  }
  __syncthreads();
  for (int c = tid; c < kTcM; c += nthr) s_ea[c] = oz_exponent(__uint_as_float(s_maxa[c]));
  if (tid == 0) {
    for (int b = 0; b < kOzStages; ++b) mbar_init(&bars[b], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_ok = 1;
    s_last = -1;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&s_tmem)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  // tensor-memory columns: exact level L at L n_tile, the small levels at 4 n_tile
  const uint32_t rest_col = (uint32_t)(kOzExact * n_tile);
  const uint32_t idesc = instr_desc(1u, n_tile, kTcM);
  const uint32_t sbo = (kTcKC * ESZ / 16) * 128;
  const int nsub = (npix + kTcKC - 1) / kTcKC;
  // Gram readback: thread = (lane quadrant, 8-column slice), n_tile = 64 columns
  constexpr int kRb = 64 * 4 / (kOzThreads / 32);  // columns a thread reads back
  const int quad = warp & 3, cslice = warp >> 2;
  const int row = quad * 32 + lane, col0 = cslice * kRb;
  long long acc[kRb];
#pragma unroll
  for (int j = 0; j < kRb; ++j) acc[j] = 0;
  // Warp 0 issues the MMAs; warps 1.. stage.  The staging warps go on to the next chunk while
  // the MMAs of this one are issued and run (the chunk's buffer was last read by the MMAs of
  // chunk - kOzStages, whose commit they wait for).  The design values of a chunk (kOzPer
  // elements per staging thread, Nc <= 64 columns) are fetched one chunk ahead, so their
  // global loads are in flight during the previous chunk's staging.
  const int stid = tid - 32, snthr = nthr - 32;
  float2 cvn[kOzPer];
  // a staging thread's elements are the same (row, pixel-in-chunk) slots in every chunk: their
  // tile offset, row and pixel packed once (row 255 marks a slot past the columns)
  uint32_t pk[kOzPer];
#pragma unroll
  for (int u = 0; u < kOzPer; ++u) {
    int c, j;
    oz_elem(stid + u * snthr, &c, &j);
    pk[u] = c < Nc ? tile_off<ESZ>(c, j) | ((uint32_t)c << 16) | ((uint32_t)j << 24)
                   : (255u << 16);
  }
  auto fetch_chunk = [&](int ch2) {
#pragma unroll
    for (int u = 0; u < kOzPer; ++u) {
      const int c = (pk[u] >> 16) & 255, j = pk[u] >> 24;
      cvn[u] = (ch2 < nsub && c != 255) ? src.fetch(c, ch2 * kTcKC + j) : make_float2(0.f, 0.f);
    }
  };
  if (warp != 0) fetch_chunk(0);
  for (int ch = 0; ch < nsub; ++ch) {
    const int s = ch % kOzStages, use = ch / kOzStages;  // use: earlier commits on bars[s]
    const int grp = ch / kOzGroup, q = ch - grp * kOzGroup;
    const int base = ch * kTcKC;
    bool tmo = false;  // this thread's wait for the buffer ran out
    if (warp != 0) {
      tmo = use >= 1 && !mbar_wait(&bars[s], (use - 1) & 1);
      float2 cv[kOzPer];
#pragma unroll
      for (int u = 0; u < kOzPer; ++u) cv[u] = cvn[u];
      fetch_chunk(ch + 1);
#pragma unroll
      for (int u = 0; u < kOzPer; ++u) {
        const int c = (pk[u] >> 16) & 255, j = pk[u] >> 24;
        if (c == 255) continue;  // rows past the columns stay zero
        float vh, vl, wh, wl, bh, bl;
        src.make(c, base + j, cv[u], &vh, &vl);
        src.weight(base + j, &wh, &wl);
        oz_mul(vh, vl, wh, wl, &bh, &bl);
        const float sa = __int_as_float((127 - s_ea[c]) << 23);
        uint16_t da[kOzSlices];
        oz_digits(bh * sa, bl * sa, da);
        const uint32_t off = pk[u] & 0xffffu;
#pragma unroll
        for (int k = 0; k < kOzSlices; ++k)
          *reinterpret_cast<uint16_t*>(a_plane(s, k) + off) = da[k];
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    // the barrier combines the threads' timeouts, so every thread takes the same branch (a
    // shared flag could already be rewritten for the next chunk by a staging warp)
    if (__syncthreads_or(tmo ? 1 : 0)) {
      if (tid == 0) s_ok = 0;
      break;
    }
    if (tid == 0) {
      tc_fence_after();
      // the descriptors of this stage's slices and K steps differ only in the start-address
      // field ((address & 0x3FFFF) >> 4, shared memory being below 256 KB): one descriptor and
      // constant offsets
      const uint64_t d0 = smem_desc(smem_u32(a_plane(s, 0)), 128, sbo);
#pragma unroll
      for (int k0 = 0; k0 < kTcKC; k0 += 16) {
        const uint32_t koff = (uint32_t)(k0 / 8) * 128;
#pragma unroll
        for (int i = 0; i < kOzSlices; ++i) {
          const uint64_t ad = d0 + ((i * a_bytes + koff) >> 4);
#pragma unroll
          for (int j = 0; i + j < kOzSlices; ++j) {
            const uint64_t bd = d0 + ((j * a_bytes + koff) >> 4);
            const int L = i + j;
            uint32_t dst, accf;
            if (L < kOzExact) {
              dst = tmem + (uint32_t)(L * n_tile);
              accf = (q == 0 && k0 == 0 && i == 0) ? 0u : 1u;
            } else {
              dst = tmem + rest_col;
              accf = (ch == 0 && k0 == 0 && i == 0 && j == kOzExact) ? 0u : 1u;
            }
            tc_mma<1>(dst, ad, bd, idesc, accf);
          }
        }
      }
      tc_commit(&bars[s]);
      s_last = ch;
    }
    if (q == kOzGroup - 1 || ch == nsub - 1) {
      // the group's exact levels: wait for its MMAs, read them back, add them as integers (the
      // next group's first MMAs overwrite the tiles only after the barrier below)
      __syncthreads();
      if (!mbar_wait(&bars[s], use & 1) && tid == 0) s_ok = 0;
      __syncthreads();
      if (!s_ok) break;
      tc_fence_after();
      {
        const uint32_t lanebase = ((uint32_t)(quad * 32)) << 16;
#pragma unroll
        for (int L = 0; L < kOzExact; ++L) {
          const uint32_t cb = (uint32_t)(L * n_tile + col0);
          float v0[kRb];
          tc_ld8(tmem + lanebase + cb, v0);
          const float up = __int_as_float((127 + 8 * (L + 2)) << 23);  // 2^(8(L+2))
          const int sh = 8 * (kOzExact - 1 - L);
#pragma unroll
          for (int j = 0; j < kRb; ++j) acc[j] += (long long)__float2int_rn(v0[j] * up) << sh;
        }
      }
      tc_fence_before();
      __syncthreads();
    }
  }
  __syncthreads();
  // drain: every MMA issued is complete before the tensor memory is read or freed
  const int last = s_last;
  const bool drained =
      last < 0 || mbar_wait(&bars[last % kOzStages], (last / kOzStages) & 1);
  __syncthreads();
  if (!drained && tid == 0) s_ok = 0;
  __syncthreads();
  tc_fence_after();
  const bool ok = s_ok != 0 && last == nsub - 1;
  if (ok) {
    float rv0[kRb];
    const uint32_t lanebase = ((uint32_t)(quad * 32)) << 16;
    tc_ld8(tmem + lanebase + rest_col + col0, rv0);
    double* Gr = src.gram();
    if (row < Nc) {
#pragma unroll
      for (int j = 0; j < kRb; ++j) {
        const int d = col0 + j;
        if (d <= row && d < Nc) {
          const double small = (double)rv0[j];
          // acc is in units of 2^(-8 (kOzExact + 1)), the unit of the last exact level; the
          // column scales as an exact power of two built from its exponent bits (ldexp where
          // the exponent leaves the normal range)
          const double lev = (double)acc[j] * 0x1p-48 + small;
          static_assert(8 * (kOzExact + 1) == 48, "unit of the exact levels");
          const int e = s_ea[row] + s_ea[d];
          const double g = (e > -1000 && e < 1000)
                               ? lev * __longlong_as_double((long long)(1023 + e) << 52)
                               : ldexp(lev, e);
          Gr[row * Nc + d] = g;
          Gr[d * Nc + row] = g;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512)
                 : "memory");
  if (!ok) {
    if (tid == 0) src.fail(PSFM_ERR_TIMEOUT);
    return;
  }
  __syncthreads();
  src.finish(tid);
}

}  // namespace

size_t gram_tc_smem(int mode, int n_tile) {
  const size_t esz = mode == 0 ? 4 : 2, nops = mode == 0 ? 1 : 2;
  return 2 * nops * (size_t)(kTcM + n_tile) * kTcKC * esz;
}

template <class Src>
cudaError_t launch_gram_tc_src(int mode, const Src& src, int nblk, int n_cols, cudaStream_t s) {
  const int n_tile = n_cols <= 64 ? 64 : 128;
  const size_t smem = gram_tc_smem(mode, n_tile);
  cudaError_t e;
  if (mode == 0) {
    e = cudaFuncSetAttribute(k_gram_tc<0, Src>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    k_gram_tc<0, Src><<<nblk, kTcThreads, smem, s>>>(src, n_tile);
  } else {
    e = cudaFuncSetAttribute(k_gram_tc<1, Src>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    k_gram_tc<1, Src><<<nblk, kTcThreads, smem, s>>>(src, n_tile);
  }
  return cudaGetLastError();
}

size_t gram_oz_smem(int) { return (size_t)kOzStages * kOzSlices * kTcM * kTcKC * 2; }

template <class Src>
cudaError_t launch_gram_oz_src(const Src& src, int nblk, int n_cols, int n_pix, int n_d,
                               cudaStream_t s) {
  if (n_cols > 64) return cudaErrorInvalidValue;
  const int n_tile = 64;
  const size_t smem = gram_oz_smem(n_tile) + sizeof(float) * Src::prep_floats(n_pix, n_d);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_gram_oz<Src>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_gram_oz<Src><<<nblk, kOzThreads, smem, s>>>(src, n_tile);
  return cudaGetLastError();
}

cudaError_t launch_gram_oz(const StampParams& sp, int nreg, int nsplit, cudaStream_t s) {
  const int nch = (sp.P + kTcKC - 1) / kTcKC;
  nsplit = std::max(1, std::min({nsplit, kGramSplit, nch}));
  OzStampSource src;
  src.P = sp;
  src.nsplit = nsplit;
  return launch_gram_oz_src(src, nreg * nsplit, sp.Nc, sp.P, sp.Nd, s);
}

cudaError_t launch_gram_oz_plain(const float* cols, const float* w, int n_blocks, int n_cols,
                                 int n_pix, double* G, int32_t* status, cudaStream_t s) {
  OzPlainSource src;
  src.cols = cols;
  src.w = w;
  src.G = G;
  src.status = status;
  src.n_cols = n_cols;
  src.n_pix = n_pix;
  return launch_gram_oz_src(src, n_blocks, n_cols, n_pix, 0, s);
}

cudaError_t launch_gram_tc(int mode, const StampParams& sp, int nreg, cudaStream_t s) {
  StampSource src;
  src.P = sp;
  return launch_gram_tc_src(mode, src, nreg, sp.Nc, s);
}

cudaError_t launch_gram_tc_plain(int mode, const float* cols, const float* w, int n_blocks,
                                 int n_cols, int n_pix, double* G, int32_t* status,
                                 cudaStream_t s) {
  PlainSource src;
  src.cols = cols;
  src.w = w;
  src.G = G;
  src.status = status;
  src.n_cols = n_cols;
  src.n_pix = n_pix;
  return launch_gram_tc_src(mode, src, n_blocks, n_cols, s);
}

}  // namespace psfm

namespace psfm {
namespace {

// FP64 reference Gram of psfm_gram: one thread per (i, j <= i), FP64 products and sums in
// pixel order.
__global__ void k_gram_fp64(const float* cols, const float* w, int n_cols, int n_pix,
                            double* G) {
  const int b = blockIdx.y;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = q / n_cols, j = q - i * n_cols;
  if (i >= n_cols || j > i) return;
  const float* ci = cols + ((int64_t)b * n_cols + i) * n_pix;
  const float* cj = cols + ((int64_t)b * n_cols + j) * n_pix;
  const float* wb = w + (int64_t)b * n_pix;
  double s = 0.0;
  for (int p = 0; p < n_pix; ++p) s = fma((double)wb[p] * (double)ci[p], (double)cj[p], s);
  double* Gb = G + (int64_t)b * n_cols * n_cols;
  Gb[i * n_cols + j] = s;
  Gb[j * n_cols + i] = s;
}

}  // namespace
}  // namespace psfm

extern "C" psfm_status psfm_gram(int32_t n_blocks, int32_t n_cols, int32_t n_pix,
                                 const float* cols, const float* weights, int32_t precision,
                                 double* gram, void* workspace, size_t ws_bytes,
                                 psfm_stream stream) {
  if (n_blocks < 0 || n_cols < 1 || n_pix < 1 || !cols || !weights || !gram)
    return n_blocks == 0 ? PSFM_OK : PSFM_ERR_BAD_ARG;
  if (n_blocks == 0) return PSFM_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (precision == PSFM_PREC_FP64) {
    const int64_t nt = (int64_t)n_cols * n_cols;
    dim3 grid((unsigned)((nt + 255) / 256), (unsigned)n_blocks);
    psfm::k_gram_fp64<<<grid, 256, 0, s>>>(cols, weights, n_cols, n_pix, gram);
    return cudaGetLastError() == cudaSuccess ? PSFM_OK : PSFM_ERR_CUDA;
  }
  if (precision != PSFM_PREC_TF32 && precision != PSFM_PREC_BF16X3 &&
      precision != PSFM_PREC_BF16X6)
    return PSFM_ERR_UNSUPPORTED;
  if (n_cols > (precision == PSFM_PREC_BF16X6 ? 64 : 128)) return PSFM_ERR_UNSUPPORTED;
  if (!workspace || ws_bytes < PSFM_GRAM_WORKSPACE ||
      (reinterpret_cast<uintptr_t>(workspace) & 255) != 0)
    return PSFM_ERR_WORKSPACE;
  int32_t* status = static_cast<int32_t*>(workspace);
  if (cudaMemsetAsync(status, 0, sizeof(int32_t), s) != cudaSuccess) return PSFM_ERR_CUDA;
  const cudaError_t e =
      precision == PSFM_PREC_BF16X6
          ? psfm::launch_gram_oz_plain(cols, weights, n_blocks, n_cols, n_pix, gram, status, s)
          : psfm::launch_gram_tc_plain(precision == PSFM_PREC_TF32 ? 0 : 1, cols, weights,
                                       n_blocks, n_cols, n_pix, gram, status, s);
  if (e != cudaSuccess) return PSFM_ERR_CUDA;
  int32_t h = 0;
  if (cudaMemcpyAsync(&h, status, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return PSFM_ERR_CUDA;
  return h;
}

extern "C" psfm_status psfm_set_pipeline_wait_limit(uint32_t polls) {
  return cudaMemcpyToSymbol(psfm::g_pipe_wait_limit, &polls, sizeof(polls)) == cudaSuccess
             ? PSFM_OK
             : PSFM_ERR_CUDA;
}
