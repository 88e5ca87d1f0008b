// Double-float arithmetic ("df"): a value is the unevaluated sum hi + lo of
// two float32 numbers with |lo| <= ulp(hi) / 2, about 48 significant bits.
// Built from the error-free transformations TwoSum (Knuth, TAOCP vol. 2,
// 4.2.2) and TwoProd with a fused multiply-add (Dekker 1971; the FMA form is
// exact because fma(a, b, -a*b) recovers the rounding error of the product).
// The FP64 fine operator computes in this type because FP64 arithmetic on
// GB300 runs at a small fraction of the FP32 rate.  All steps use the _rn
// intrinsics so that the compiler cannot contract or reassociate them.
#pragma once

#include <cuda_runtime.h>

namespace hdcg {

struct dfl {
  float hi, lo;
  dfl() = default;
  __device__ __forceinline__ dfl(float h, float l) : hi(h), lo(l) {}
  __device__ __forceinline__ dfl(int v) : hi((float)v), lo(0.f) {}
  __device__ __forceinline__ dfl(float v) : hi(v), lo(0.f) {}
  __device__ __forceinline__ dfl(double v) {
    hi = __double2float_rn(v);
    lo = __double2float_rn(v - (double)hi);
  }
  __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
};

// s + e = a + b exactly (TwoSum)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// s + e = a + b for |a| >= |b| (FastTwoSum)
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ dfl operator+(dfl a, dfl b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  float h, l;
  fast_two_sum(s, e, h, l);
  return dfl(h, l);
}
__device__ __forceinline__ dfl operator-(dfl a) { return dfl(-a.hi, -a.lo); }
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + (-b); }
__device__ __forceinline__ dfl operator*(dfl a, dfl b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);          // exact error of the product
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  float h, l;
  fast_two_sum(p, e, h, l);
  return dfl(h, l);
}
__device__ __forceinline__ dfl& operator+=(dfl& a, dfl b) { return a = a + b; }
__device__ __forceinline__ dfl& operator-=(dfl& a, dfl b) { return a = a - b; }
__device__ __forceinline__ dfl& operator*=(dfl& a, dfl b) { return a = a * b; }

// lane shuffles of any compute type
__device__ __forceinline__ float shfl_any(float v, int src, int width) {
  return __shfl_sync(0xffffffffu, v, src, width);
}
__device__ __forceinline__ double shfl_any(double v, int src, int width) {
  return __shfl_sync(0xffffffffu, v, src, width);
}
__device__ __forceinline__ dfl shfl_any(dfl v, int src, int width) {
  return dfl(__shfl_sync(0xffffffffu, v.hi, src, width), __shfl_sync(0xffffffffu, v.lo, src, width));
}

}  // namespace hdcg
