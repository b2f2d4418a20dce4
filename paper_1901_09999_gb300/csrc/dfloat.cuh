// Double-float ("FP32 pair") arithmetic shared by the stamp kernels: a value is hi + lo with
// |lo| <= ulp(hi) / 2.  Products use the exact FMA residual, sums the error-free TwoSum, so
// each operation keeps about 48 significant bits while running on the FP32 pipes (FP64 on this
// GPU runs at 1/64 of the FP32 rate).  Intrinsics keep the compiler from re-associating the
// compensations.
#pragma once

#include <cuda_runtime.h>

namespace psfm {
namespace {

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

__device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }

__device__ __forceinline__ df df_add(df a, df b) {
  df t = a;
  df_acc(t, b.hi, b.lo);
  return df_norm(t);
}

// a + b for FP32 a and b as an exact double-float (TwoSum)
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return df{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

// a + b for double-floats, not renormalised: the high parts are added exactly and the low
// parts and the rounding error go to lo, which may exceed half an ulp of hi.  A product that
// consumes the sum (df_fma) takes both parts, so its error stays at 2^-48 of the operands.
__device__ __forceinline__ df df_sum_raw(df a, df b) {
  df r = two_sum(a.hi, b.hi);
  r.lo = __fadd_rn(r.lo, __fadd_rn(a.lo, b.lo));
  return r;
}

}  // namespace
}  // namespace psfm
