// Float-float arithmetic: a value is carried as hi + lo, two FP32 numbers
// (about 48 significant bits).  GB300 runs FP64 at about 1/70 of its FP32
// rate, so the FP32 form's short-side Gram-Schmidt runs in float-float on the
// FP32 pipes instead of FP64.
//
// Error-free transformations: TwoSum (Knuth, TAOCP vol. 2, 4.2.2), FastTwoSum
// (Dekker 1971, |a| >= |b|) and TwoProduct by one FMA.  Dot products follow
// the compensated scheme of Ogita, Rump and Oishi, "Accurate sum and dot
// product", SIAM J. Sci. Comput. 26 (2005), Algorithm Dot2, with float-float
// operands: the cross terms x_hi y_lo + x_lo y_hi join the error terms.  The
// result is as accurate as a dot product in about twice FP32 precision,
// i.e. errors near n 2^-48 |x| |y| for n terms.
//
// These rely on IEEE FP32 additions in program order: the library is built
// without fast-math, and nothing here is written as a multiply-add that
// contraction could change.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ssa {

struct ff { float hi, lo; };

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ ff ff_norm(float s, float c) {
  ff r;
  fast_two_sum(s, c, r.hi, r.lo);
  return r;
}
// a + b (the "sloppy" sum of the QD library: exact when the sum does not
// cancel; with cancellation the error stays near 2^-48 |a|)
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return ff_norm(s, e);
}
__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.hi, -a.lo}; }
// a * b
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  const float e = __fmaf_rn(a.hi, b.hi, -p);
  const float t = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
  return ff_norm(p, t);
}

// Running sum s + c of a dot product (unnormalised: c collects the rounding
// errors of s and the low-order product terms).
struct ffacc {
  float s = 0.0f, c = 0.0f;
  // += x * y
  __device__ __forceinline__ void fma(float xh, float xl, float yh, float yl) {
    const float p = __fmul_rn(xh, yh);
    const float e = __fmaf_rn(xh, yh, -p);
    float t, q;
    two_sum(s, p, t, q);
    s = t;
    c = __fadd_rn(c, __fadd_rn(q, __fmaf_rn(xh, yl, __fmaf_rn(xl, yh, e))));
  }
  __device__ __forceinline__ void fma(float2 x, float2 y) { fma(x.x, x.y, y.x, y.y); }
  __device__ __forceinline__ void add(const ffacc& o) {
    float t, q;
    two_sum(s, o.s, t, q);
    s = t;
    c = __fadd_rn(c, __fadd_rn(o.c, q));
  }
  __device__ __forceinline__ ff value() const { return ff_norm(s, c); }
};

__device__ __forceinline__ ffacc warp_sum_ff(ffacc a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ffacc b;
    b.s = __shfl_xor_sync(0xffffffffu, a.s, o);
    b.c = __shfl_xor_sync(0xffffffffu, a.c, o);
    a.add(b);
  }
  return a;
}

// hi + lo = d to 2^-48 relative, with integer instructions only (no FP64 pipe):
// hi keeps the leading 24 significant bits of d (truncated), lo the next 29
// rounded to 24.  For |d| < 2^127.  Below 2^-74 lo is dropped (an absolute
// error under 2^-97) and below 2^-100 the result is 0.
__device__ __forceinline__ float2 ff_from_double(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned hw = (unsigned)(b >> 32);
  const unsigned sign = hw & 0x80000000u;
  const int e = (int)((hw >> 20) & 0x7FFu);                   // biased FP64 exponent
  if (e < 1023 - 100) return make_float2(0.0f, 0.0f);
  const unsigned hm = (unsigned)((b >> 29) & 0x7FFFFFu);      // mantissa bits 51..29
  const float hi = __uint_as_float(sign | ((unsigned)(e - 1023 + 127) << 23) | hm);
  const unsigned lm = (unsigned)(b & 0x1FFFFFFFu);            // mantissa bits 28..0
  float lo = 0.0f;
  if (e >= 1075 - 126 && lm != 0) {
    // lm 2^(e - 1075): the scale as an FP32 power of two (e - 1075 >= -126)
    const float sc = __uint_as_float((unsigned)(e - 1075 + 127) << 23);
    lo = __fmul_rn(__uint2float_rn(lm), sc);
    if (sign) lo = -lo;
  }
  return make_float2(hi, lo);
}
// d 2^-shift as hi + lo (the same split, with the exponent lowered by shift
// first; integer instructions only)
__device__ __forceinline__ float2 ff_from_double_scaled(double d, int shift) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const int e = (int)((b >> 52) & 0x7FFull);
  if (e == 0) return make_float2(0.0f, 0.0f);                    // zero (denormals flushed)
  const int es = e - shift;
  if (es < 1) return make_float2(0.0f, 0.0f);
  const unsigned long long bs = (b & ~(0x7FFull << 52)) | ((unsigned long long)es << 52);
  return ff_from_double(__longlong_as_double((long long)bs));
}

// sum over the lanes of a team of W consecutive lanes (W a power of two <= 32)
template <int W>
__device__ __forceinline__ ffacc team_sum_ff(ffacc a) {
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1) {
    ffacc b;
    b.s = __shfl_xor_sync(0xffffffffu, a.s, o);
    b.c = __shfl_xor_sync(0xffffffffu, a.c, o);
    a.add(b);
  }
  return a;
}

// the double nearest hi + lo (two conversions and an FP64 add: off the hot loops)
__device__ __forceinline__ double ff_to_double(float2 v) { return (double)v.x + (double)v.y; }

}  // namespace ssa
