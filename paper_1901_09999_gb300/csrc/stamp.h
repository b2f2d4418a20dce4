// Per-stamp kernel parameters and the small device helpers that the stamp kernels (design,
// Gram, chi^2) share across translation units.
#pragma once

#include "psfm_internal.h"

namespace psfm {

__device__ __forceinline__ void raise_error(DevState* st, int code) { atomicCAS(&st->error, 0, code); }

// Whether a block skips its work because the loop has finished or an error was raised, by an
// earlier kernel or by another block of this launch.  Read once by one thread so that the
// decision is uniform across the block's barriers.
__device__ __forceinline__ bool block_skip(const DevState* st) {
  __shared__ int s_skip;
  if (threadIdx.x == 0) s_skip = (st->error || st->done) ? 1 : 0;
  __syncthreads();
  return s_skip != 0;
}

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
  int Nd;  // design columns (N_b, or 2 N_b with the dual kernel)
  const float* f1d;     // [NH][wpad]
  const double* f1d64;  // [NH][w]
  const double* psi;
  const double* sk;
  const int32_t* cand;
  const int32_t* ptr;
  int32_t* have;
  int32_t* fresh;  // [nreg] Gram recomputed in this iteration (added to M by k_system_delta)
  void* C;  // [nreg][Nb][P] of T (float or double, by precision mode)
  double* Gt;      // [nreg][Nc][Nc] Gram of the zero-sum augmented design block
  double* Gpart;        // [nreg][kGramSplit][Nc][Nc] partial Grams (double-float mode)
  int32_t* gram_count;  // [nreg] partials finished, reset by the block that combines them
  double* footsum;
  DevState* st;
};

}  // namespace psfm
