// FP32-pair ("double-float") scalars for the low-rank kernel's band sums: a value
// is the unevaluated sum hi + lo of two FP32 numbers.  The error-free
// transformations are those of gf_complex.cuh (Knuth's two_sum, the FMA
// two_prod), about 2^-48 relative precision per operation on the FP32 pipes.
#pragma once

#include <cuda_runtime.h>

#include "gf_complex.cuh"

namespace gf {
namespace pair {

struct f2 {
  float h, l;
};

using cx::two_sum;

// acc += a * b: exact head product, first-order cross terms, head sum by two_sum;
// acc is left unnormalised (its low word collects the rounding errors).
__device__ __forceinline__ void mac(f2& acc, f2 a, f2 b) { cx::acc_prod(a.h, a.l, b.h, b.l, acc.h, acc.l); }

// acc += a (pairs)
__device__ __forceinline__ void add(f2& acc, f2 a) {
  float s, t;
  two_sum(acc.h, a.h, s, t);
  acc.h = s;
  acc.l = __fadd_rn(acc.l, __fadd_rn(t, a.l));
}

__device__ __forceinline__ f2 split(double x) {
  f2 r;
  cx::split(x, r.h, r.l);
  return r;
}

__device__ __forceinline__ double value(f2 a) { return (double)a.h + (double)a.l; }

}  // namespace pair
}  // namespace gf
