// FP32-pair ("double-float") arithmetic for the low-rank kernel's band sums: a
// value is the unevaluated sum hi + lo of two FP32 numbers.  Error-free
// transformations (Knuth's two_sum, the FMA two_prod) keep about 2^-48 relative
// precision per operation on the FP32 pipes.  The _rn intrinsics keep nvcc from
// contracting or reassociating the steps.
#pragma once

#include <cuda_runtime.h>

namespace gf {
namespace pair {

struct f2 {
  float h, l;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// acc += a * b: exact head product, first-order cross terms, head sum by two_sum;
// acc is left unnormalised (its low word collects the rounding errors).
__device__ __forceinline__ void mac(f2& acc, f2 a, f2 b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  float s, t;
  two_sum(acc.h, p, s, t);
  acc.h = s;
  acc.l = __fadd_rn(acc.l, __fadd_rn(t, e));
}

// acc += a (pairs)
__device__ __forceinline__ void add(f2& acc, f2 a) {
  float s, t;
  two_sum(acc.h, a.h, s, t);
  acc.h = s;
  acc.l = __fadd_rn(acc.l, __fadd_rn(t, a.l));
}

__device__ __forceinline__ f2 split(double x) {
  f2 r;
  r.h = __double2float_rn(x);
  r.l = __double2float_rn(x - (double)r.h);
  return r;
}

__device__ __forceinline__ double value(f2 a) { return (double)a.h + (double)a.l; }

}  // namespace pair
}  // namespace gf
