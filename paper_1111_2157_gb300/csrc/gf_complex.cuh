// Complex arithmetic shared by the point kernels of libgf (device code only).
//
//  * double2: complex FP64 multiply-adds and Smith's reciprocal.
//  * cf:      a complex FP32 pair {re.hi, re.lo, im.hi, im.lo}; each part is the
//             unevaluated sum hi + lo of two FP32 numbers, kept with error-free
//             transformations (Knuth's two_sum, the FMA two_prod): about 2^-48
//             relative precision per operation on the FP32 pipes.
//  * float2:  complex FP32 multiply-adds with explicit FMAs, so that two code
//             paths that perform the same update round identically.
// The _rn intrinsics keep nvcc from contracting a product into a later add or
// reassociating sums, which would break the error-free transformations.
#pragma once

#include <cuda_runtime.h>

namespace gf {
namespace cx {

// ------------------------------------------------------------------ complex FP64
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// acc += a * b
__device__ __forceinline__ void cmac(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}
// acc += conj(a) * b
__device__ __forceinline__ void cmac_ca(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(-a.y, b.x, acc.y));
}
// acc += a * conj(b)
__device__ __forceinline__ void cmac_cb(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));
  acc.y = fma(a.y, b.x, fma(-a.x, b.y, acc.y));
}
// 1/a by Smith's algorithm (R. L. Smith, CACM 5(8), 1962): scale by the larger
// component so that no intermediate squares the inputs.
__device__ __forceinline__ double2 crcp(double2 a) {
  if (fabs(a.x) >= fabs(a.y)) {
    const double t = a.y / a.x;
    const double id = 1.0 / fma(a.y, t, a.x);
    return make_double2(id, -t * id);
  } else {
    const double t = a.x / a.y;
    const double id = 1.0 / fma(a.x, t, a.y);
    return make_double2(t * id, -id);
  }
}

// Pivot key of a complex FP64 number: max(|Re|, |Im|) compared through the IEEE
// bit pattern, which orders non-negative doubles like their values; no FP64
// instruction.
__device__ __forceinline__ unsigned long long pivot_key(double2 a) {
  const unsigned long long mask = 0x7fffffffffffffffULL;
  const unsigned long long r = (unsigned long long)__double_as_longlong(a.x) & mask;
  const unsigned long long i = (unsigned long long)__double_as_longlong(a.y) & mask;
  return r > i ? r : i;
}

// ------------------------------------------------------------------ FP32 pairs
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// (sh, sl) += (ah + al)(bh + bl): exact head product, first-order cross terms,
// head sum by two_sum; (sh, sl) is left unnormalised.
__device__ __forceinline__ void acc_prod(float ah, float al, float bh, float bl, float& sh, float& sl) {
  const float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  float s, t;
  two_sum(sh, p, s, t);
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(t, e));
}
// (sh, sl) += (ah + al) b with b a single FP32 number.
__device__ __forceinline__ void acc_prod1(float ah, float al, float b, float& sh, float& sl) {
  const float p = __fmul_rn(ah, b);
  float e = __fmaf_rn(ah, b, -p);
  e = __fmaf_rn(al, b, e);
  float s, t;
  two_sum(sh, p, s, t);
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(t, e));
}
__device__ __forceinline__ void renorm(float& h, float& l) {
  float s, e;
  two_sum(h, l, s, e);
  h = s;
  l = e;
}
__device__ __forceinline__ void renorm_fast(float& h, float& l) {
  const float s = __fadd_rn(h, l);
  l = __fsub_rn(l, __fsub_rn(s, h));
  h = s;
}
__device__ __forceinline__ void split(double x, float& h, float& l) {
  h = __double2float_rn(x);
  l = __double2float_rn(x - (double)h);
}

struct cf {
  float rh, rl, ih, il;
};
__device__ __forceinline__ cf ld4(const float4& v) { return cf{v.x, v.y, v.z, v.w}; }
__device__ __forceinline__ float4 st4(const cf& c) { return make_float4(c.rh, c.rl, c.ih, c.il); }
__device__ __forceinline__ cf cneg(const cf& c) { return cf{-c.rh, -c.rl, -c.ih, -c.il}; }
__device__ __forceinline__ cf czero() { return cf{0.f, 0.f, 0.f, 0.f}; }
__device__ __forceinline__ void cnorm(cf& c) {
  renorm(c.rh, c.rl);
  renorm(c.ih, c.il);
}
__device__ __forceinline__ double2 to_d2(const cf& c) {
  return make_double2((double)c.rh + (double)c.rl, (double)c.ih + (double)c.il);
}
__device__ __forceinline__ cf from_d2(double2 v) {
  cf c;
  split(v.x, c.rh, c.rl);
  split(v.y, c.ih, c.il);
  return c;
}
// acc += a * b
__device__ __forceinline__ void cacc(cf& acc, const cf& a, const cf& b) {
  acc_prod(a.rh, a.rl, b.rh, b.rl, acc.rh, acc.rl);
  acc_prod(-a.ih, -a.il, b.ih, b.il, acc.rh, acc.rl);
  acc_prod(a.rh, a.rl, b.ih, b.il, acc.ih, acc.il);
  acc_prod(a.ih, a.il, b.rh, b.rl, acc.ih, acc.il);
}
// acc += conj(a) * b
__device__ __forceinline__ void cacc_ca(cf& acc, const cf& a, const cf& b) {
  acc_prod(a.rh, a.rl, b.rh, b.rl, acc.rh, acc.rl);
  acc_prod(a.ih, a.il, b.ih, b.il, acc.rh, acc.rl);
  acc_prod(a.rh, a.rl, b.ih, b.il, acc.ih, acc.il);
  acc_prod(-a.ih, -a.il, b.rh, b.rl, acc.ih, acc.il);
}
// acc += a * conj(b)
__device__ __forceinline__ void cacc_cb(cf& acc, const cf& a, const cf& b) {
  acc_prod(a.rh, a.rl, b.rh, b.rl, acc.rh, acc.rl);
  acc_prod(a.ih, a.il, b.ih, b.il, acc.rh, acc.rl);
  acc_prod(a.ih, a.il, b.rh, b.rl, acc.ih, acc.il);
  acc_prod(-a.rh, -a.rl, b.ih, b.il, acc.ih, acc.il);
}
// acc += a * b with b a single-word complex FP32 number
__device__ __forceinline__ void cacc1(cf& acc, const cf& a, float2 b) {
  acc_prod1(a.rh, a.rl, b.x, acc.rh, acc.rl);
  acc_prod1(-a.ih, -a.il, b.y, acc.rh, acc.rl);
  acc_prod1(a.rh, a.rl, b.y, acc.ih, acc.il);
  acc_prod1(a.ih, a.il, b.x, acc.ih, acc.il);
}
// acc += conj(a) * b with b a single-word complex FP32 number
__device__ __forceinline__ void cacc1_ca(cf& acc, const cf& a, float2 b) {
  acc_prod1(a.rh, a.rl, b.x, acc.rh, acc.rl);
  acc_prod1(a.ih, a.il, b.y, acc.rh, acc.rl);
  acc_prod1(a.rh, a.rl, b.y, acc.ih, acc.il);
  acc_prod1(-a.ih, -a.il, b.x, acc.ih, acc.il);
}
// v -= l u
__device__ __forceinline__ void csub_prod(cf& v, const cf& l, const cf& u) {
  acc_prod(-l.rh, -l.rl, u.rh, u.rl, v.rh, v.rl);
  acc_prod(l.ih, l.il, u.ih, u.il, v.rh, v.rl);
  acc_prod(-l.rh, -l.rl, u.ih, u.il, v.ih, v.il);
  acc_prod(-l.ih, -l.il, u.rh, u.rl, v.ih, v.il);
  renorm_fast(v.rh, v.rl);
  renorm_fast(v.ih, v.il);
}
// 1/a in pairs: an FP32 reciprocal refined by one Newton step r0 + r0 (1 - a r0).
__device__ inline cf crcp_df(const cf& a) {
  const float s = fmaxf(fabsf(a.rh), fabsf(a.ih));
  const float is = __frcp_rn(s);
  const float ar = a.rh * is, ai = a.ih * is;
  const float id = __frcp_rn(ar * ar + ai * ai);
  const float r0r = ar * id * is, r0i = -ai * id * is;
  cf e = cf{1.0f, 0.0f, 0.0f, 0.0f};
  const cf r0 = cf{r0r, 0.0f, r0i, 0.0f};
  cacc(e, cneg(a), r0);
  cnorm(e);
  const float cr = __fsub_rn(__fmul_rn(r0r, e.rh), __fmul_rn(r0i, e.ih));
  const float ci = __fadd_rn(__fmul_rn(r0r, e.ih), __fmul_rn(r0i, e.rh));
  cf r;
  two_sum(r0r, cr, r.rh, r.rl);
  two_sum(r0i, ci, r.ih, r.il);
  return r;
}
// Pivot key of a pair: max(|Re.hi|, |Im.hi|) compared through the IEEE bit pattern.
__device__ __forceinline__ unsigned pivot_key_f(const float4& a) {
  const unsigned r = __float_as_uint(a.x) & 0x7fffffffu;
  const unsigned i = __float_as_uint(a.z) & 0x7fffffffu;
  return r > i ? r : i;
}

// ------------------------------------------------------- single-word complex FP32
// acc += a * b
__device__ __forceinline__ void fmac(float2& acc, float2 a, float2 b) {
  acc.x = __fmaf_rn(a.x, b.x, __fmaf_rn(-a.y, b.y, acc.x));
  acc.y = __fmaf_rn(a.x, b.y, __fmaf_rn(a.y, b.x, acc.y));
}
// acc += conj(a) * b
__device__ __forceinline__ void fmac_ca(float2& acc, float2 a, float2 b) {
  acc.x = __fmaf_rn(a.x, b.x, __fmaf_rn(a.y, b.y, acc.x));
  acc.y = __fmaf_rn(a.x, b.y, __fmaf_rn(-a.y, b.x, acc.y));
}
// acc += a * conj(b)
__device__ __forceinline__ void fmac_cb(float2& acc, float2 a, float2 b) {
  acc.x = __fmaf_rn(a.x, b.x, __fmaf_rn(a.y, b.y, acc.x));
  acc.y = __fmaf_rn(a.y, b.x, __fmaf_rn(-a.x, b.y, acc.y));
}
// v -= l u
__device__ __forceinline__ void fsub_prod(float2& v, float2 l, float2 u) {
  v.x = __fmaf_rn(-l.x, u.x, __fmaf_rn(l.y, u.y, v.x));
  v.y = __fmaf_rn(-l.x, u.y, __fmaf_rn(-l.y, u.x, v.y));
}
__device__ __forceinline__ float2 fmul(float2 a, float2 b) {
  return make_float2(__fmaf_rn(a.x, b.x, -__fmul_rn(a.y, b.y)), __fmaf_rn(a.x, b.y, __fmul_rn(a.y, b.x)));
}
// 1/a in FP32 by Smith's scaling (larger component first), two correctly
// rounded reciprocals; a few ulp.
__device__ __forceinline__ float2 frcp(float2 a) {
  const float s = fmaxf(fabsf(a.x), fabsf(a.y));
  const float is = __frcp_rn(s);
  const float ar = __fmul_rn(a.x, is), ai = __fmul_rn(a.y, is);
  const float id = __frcp_rn(__fmaf_rn(ar, ar, __fmul_rn(ai, ai)));
  const float t = __fmul_rn(id, is);
  return make_float2(__fmul_rn(ar, t), -__fmul_rn(ai, t));
}
// Pivot key of a complex FP32 number: max(|Re|, |Im|) as IEEE bits.
__device__ __forceinline__ unsigned pivot_key_s(float2 a) {
  const unsigned r = __float_as_uint(a.x) & 0x7fffffffu;
  const unsigned i = __float_as_uint(a.y) & 0x7fffffffu;
  return r > i ? r : i;
}

}  // namespace cx
}  // namespace gf
