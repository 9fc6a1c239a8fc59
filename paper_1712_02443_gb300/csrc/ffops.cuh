// Double-FP32 ("float-float") arithmetic for the complex128 product's
// contractions.  A value is the unevaluated sum hi + lo of two floats (Dekker
// 1971, "A floating-point technique for extending the available precision";
// the double-double arithmetic of Hida, Li and Bailey with FP32 parts).  GB300
// issues FP32 operations at about sixty times its FP64 rate, so a
// multiply-accumulate in this form (twelve FP32 operations) costs a fraction
// of one FP64 FMA, with about 2^-44 relative error on the sum of |a b|.
//
// Every operation uses the _rn intrinsics: a plain a * b followed by an add may
// be contracted into one FMA, which would break the error-free transformations.
#pragma once

#include <cuda_runtime.h>

namespace mm {

// One complex number in the three-product (Gauss) form, split: re, im and
// re + im, each as hi + lo.  24 bytes, three float2 loads.
struct F6 {
  float rh, ih, sh, rl, il, sl;
};

// Accumulator of a float-float dot product: running sum s (rounded) and the
// sum c of every rounding error and low-order term (c is small against s but
// not renormalised until the end).
struct FF {
  float s, c;
};

__device__ __forceinline__ FF ff_zero() { return FF{0.0f, 0.0f}; }

// acc += (ah + al)(bh + bl).  ah bh = p + e exactly (the FMA gives e); s + p =
// t + z exactly (Knuth's two-sum, six operations); the cross terms ah bl and
// al bh enter the correction (al bl, of order 2^-48, is dropped).
__device__ __forceinline__ void ff_mac(FF& acc, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  const float e = __fmaf_rn(ah, bh, -p);
  const float t = __fadd_rn(acc.s, p);
  const float bb = __fsub_rn(t, acc.s);
  const float z = __fadd_rn(__fsub_rn(acc.s, __fsub_rn(t, bb)), __fsub_rn(p, bb));
  acc.s = t;
  float c = __fadd_rn(acc.c, __fadd_rn(z, e));
  c = __fmaf_rn(ah, bl, c);
  acc.c = __fmaf_rn(al, bh, c);
}

// Renormalised sum a + b of two accumulators: hi + lo with |lo| <= ulp(hi) / 2.
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const float t = __fadd_rn(a.s, b.s);
  const float bb = __fsub_rn(t, a.s);
  float z = __fadd_rn(__fsub_rn(a.s, __fsub_rn(t, bb)), __fsub_rn(b.s, bb));
  z = __fadd_rn(z, __fadd_rn(a.c, b.c));
  const float h = __fadd_rn(t, z);
  return FF{h, __fsub_rn(z, __fsub_rn(h, t))};
}
__device__ __forceinline__ FF ff_neg(FF a) { return FF{-a.s, -a.c}; }

// (double) of a float-float value (exact up to the final FP64 rounding)
__device__ __forceinline__ double ff_to_double(FF a) { return (double)a.s + (double)a.c; }

// x = hi + lo, hi the nearest float to x, lo the nearest float to x - hi
// (|x - hi - lo| <= 2^-48 |x|)
__device__ __forceinline__ void ff_split(double x, float& hi, float& lo) {
  hi = __double2float_rn(x);
  lo = __double2float_rn(x - (double)hi);
}

__device__ __forceinline__ F6 f6_from(double re, double im) {
  F6 f;
  ff_split(re, f.rh, f.rl);
  ff_split(im, f.ih, f.il);
  ff_split(re + im, f.sh, f.sl);
  return f;
}

// The three Gauss sums of a complex dot product: t1 = sum Re a Re b, t2 = sum
// Im a Im b, t3 = sum (Re a + Im a)(Re b + Im b); a b summed = (t1 - t2) + i (t3 - t1 - t2).
struct FF3 {
  FF t1, t2, t3;
};
__device__ __forceinline__ FF3 ff3_zero() { return FF3{ff_zero(), ff_zero(), ff_zero()}; }
__device__ __forceinline__ void ff3_mac(FF3& acc, const F6& a, const F6& b) {
  ff_mac(acc.t1, a.rh, a.rl, b.rh, b.rl);
  ff_mac(acc.t2, a.ih, a.il, b.ih, b.il);
  ff_mac(acc.t3, a.sh, a.sl, b.sh, b.sl);
}
// the complex sum as (re, im) float-float values
__device__ __forceinline__ void ff3_result(const FF3& a, FF& re, FF& im) {
  re = ff_add(a.t1, ff_neg(a.t2));
  im = ff_add(ff_add(a.t3, ff_neg(a.t1)), ff_neg(a.t2));
}

__device__ __forceinline__ F6 f6_load(const F6* p) {
  const float2* q = reinterpret_cast<const float2*>(p);
  const float2 a = q[0], b = q[1], c = q[2];
  return F6{a.x, a.y, b.x, b.y, c.x, c.y};
}
__device__ __forceinline__ void f6_store(F6* p, const F6& f) {
  float2* q = reinterpret_cast<float2*>(p);
  q[0] = make_float2(f.rh, f.ih);
  q[1] = make_float2(f.sh, f.rl);
  q[2] = make_float2(f.il, f.sl);
}
__device__ __forceinline__ F6 f6_zero() { return F6{0, 0, 0, 0, 0, 0}; }

// A renormalised float-float value hi + lo (|lo| <= ulp(hi) / 2) with the
// arithmetic of the FFT stages: a sum is Knuth's two-sum of the high parts plus
// the low parts, a product Dekker's exact product (by FMA) plus the cross
// terms, each renormalised by a fast two-sum (about 2^-47 relative error per
// operation, normwise).  The operators let the FFT's generic complex code run
// on CF = (FFv re, FFv im).
struct FFv {
  float h, l;
  FFv() = default;
  __host__ __device__ constexpr FFv(float v) : h(v), l(0.0f) {}
  __host__ __device__ constexpr FFv(float h_, float l_) : h(h_), l(l_) {}
};
__device__ __forceinline__ FFv ffv_add(FFv a, FFv b) {
  const float s = __fadd_rn(a.h, b.h);
  const float bb = __fsub_rn(s, a.h);
  float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
  e = __fadd_rn(e, __fadd_rn(a.l, b.l));
  const float h = __fadd_rn(s, e);
  return FFv(h, __fsub_rn(e, __fsub_rn(h, s)));
}
__device__ __forceinline__ FFv ffv_mul(FFv a, FFv b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  const float h = __fadd_rn(p, e);
  return FFv(h, __fsub_rn(e, __fsub_rn(h, p)));
}
// a b + c with one renormalisation
__device__ __forceinline__ FFv ffv_fma(FFv a, FFv b, FFv c) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  const float s = __fadd_rn(p, c.h);
  const float bb = __fsub_rn(s, p);
  float z = __fadd_rn(__fsub_rn(p, __fsub_rn(s, bb)), __fsub_rn(c.h, bb));
  z = __fadd_rn(z, __fadd_rn(e, c.l));
  const float h = __fadd_rn(s, z);
  return FFv(h, __fsub_rn(z, __fsub_rn(h, s)));
}
__device__ __forceinline__ FFv operator-(FFv a) { return FFv(-a.h, -a.l); }
__device__ __forceinline__ FFv operator+(FFv a, FFv b) { return ffv_add(a, b); }
__device__ __forceinline__ FFv operator-(FFv a, FFv b) { return ffv_add(a, -b); }
__device__ __forceinline__ FFv operator*(FFv a, FFv b) { return ffv_mul(a, b); }
__device__ __forceinline__ FFv fmx(FFv a, FFv b, FFv c) { return ffv_fma(a, b, c); }

struct CF {
  FFv x, y;
};
// FP64 <-> CF at the FFT stages' boundaries
__device__ __forceinline__ FFv ffv_from(double v) {
  FFv r;
  ff_split(v, r.h, r.l);
  return r;
}
__device__ __forceinline__ double ffv_to_double(FFv v) { return (double)v.h + (double)v.l; }

}  // namespace mm
