// Float-float value type: a value hi + lo carried by two FP32 numbers (about 48
// significant bits).  On this GPU FP64 arithmetic issues about 68x slower than
// FP32, so arithmetic that needs more than FP32 but not all of FP64 (the inner
// solves of the refined PCG, precision 2) runs on the FP32 pipes with error-free
// transformations: two-sum for additions, the FMA product error for products.
// __fadd_rn / __fmul_rn are never contracted into FMAs, which the error terms
// rely on.  Additions are the cheap variant (errors relative to the operands, as
// an FP64 addition's are to its result rounded once more at 2^-48).
#pragma once
#include <cuda_runtime.h>

namespace mqs {

struct ffv {
  float hi, lo;
  ffv() = default;                                                   // trivial: shared-memory arrays
  __host__ __device__ ffv(int v) : hi((float)v), lo(0.f) {}          // T(0), T x = 0
  __host__ __device__ ffv(float h, float l) : hi(h), lo(l) {}
};

__device__ __forceinline__ ffv ff_norm(float s, float t) {          // s + t, |s| >= |t|
  const float h = __fadd_rn(s, t);
  return ffv(h, __fsub_rn(t, __fsub_rn(h, s)));
}
__device__ __forceinline__ ffv operator+(ffv a, ffv b) {
  const float s = __fadd_rn(a.hi, b.hi), bb = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  return ff_norm(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ffv operator-(ffv a) { return ffv(-a.hi, -a.lo); }
__device__ __forceinline__ ffv operator-(ffv a, ffv b) { return a + (-b); }
// a * b: the FP32 product and its exact error (FMA), plus the cross terms
__device__ __forceinline__ ffv ff_mul(ffv a, ffv b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return ff_norm(p, e);
}
// a * b + c
__device__ __forceinline__ ffv fmaT(ffv a, ffv b, ffv c) { return ff_mul(a, b) + c; }
// a / b: the FP32 quotient q1 corrected by the quotient of the float-float
// remainder a - q1 b (Dekker's division; relative error about 2^-47)
__device__ __forceinline__ ffv ff_div(ffv a, ffv b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const float p = __fmul_rn(q1, b.hi);
  float e = __fmaf_rn(q1, b.hi, -p);
  e = __fmaf_rn(q1, b.lo, e);
  const ffv r = a - ff_norm(p, e);
  return ff_norm(q1, __fdiv_rn(r.hi, b.hi));
}
// a <= b for normalised values (|lo| at most half an ulp of hi)
__device__ __forceinline__ bool ff_le(ffv a, ffv b) { return a.hi < b.hi || (a.hi == b.hi && a.lo <= b.lo); }
__device__ __forceinline__ ffv ff_from(double v) {
  const float hi = __double2float_rn(v);
  return ffv(hi, __double2float_rn(v - (double)hi));
}
__device__ __forceinline__ double ff_to(ffv a) { return (double)a.hi + (double)a.lo; }

// warp shuffle by one lane (the sweeps pass each face flux to the x+1 neighbour)
__device__ __forceinline__ double shfl_up1(double v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ float shfl_up1(float v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ ffv shfl_up1(ffv v) {
  return ffv(__shfl_up_sync(0xffffffffu, v.hi, 1), __shfl_up_sync(0xffffffffu, v.lo, 1));
}

}  // namespace mqs
