// Double-word ("double-float") arithmetic on the FP32 pipe.
//
// A value is held as an unevaluated sum hi + lo of two floats with |lo| <= ulp(hi) / 2, which
// carries about 48 significand bits. GB300 executes FP32 operations at 64 times the rate of
// FP64 ones, so a Krylov inner solve in double-word arithmetic is limited by memory bandwidth
// instead of the FP64 pipe, at a precision close to FP64's.
//
// Building blocks (published error-free transformations, written here from their definitions):
//   two_sum      -- Knuth, TAOCP vol. 2, Sec. 4.2.2: s = fl(a + b) and the exact error e,
//                   a + b = s + e, for any a, b.
//   fast_two_sum -- Dekker (1971): the same with three operations when |a| >= |b|.
//   two_prod     -- with a fused multiply-add: p = fl(a b), e = fma(a, b, -p), a b = p + e.
//   Dot2-style accumulation -- Ogita, Rump & Oishi, "Accurate sum and dot product" (2005): the
//                   running sum s is carried with TwoSum, all rounding errors (and the low-order
//                   cross products of double-word operands) are added into a separate float c;
//                   s + c is as accurate as a dot product in twice the working precision.
// The explicit __fadd_rn / __fmul_rn / __fmaf_rn intrinsics keep the compiler from contracting
// or reordering the error terms.
#pragma once

#include <cuda_runtime.h>

namespace helm {

// complex double-word: (re.hi, re.lo, im.hi, im.lo), one 16-byte load
struct alignas(16) cw {
  float rh, rl, ih, il;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

// Double-word accumulator: value s + c.
struct dacc {
  float s, c;
  __device__ __forceinline__ dacc() : s(0.f), c(0.f) {}
  __device__ __forceinline__ dacc(float h, float l) : s(h), c(l) {}
  // += (ah + al)(xh + xl): exact head product, low-order cross terms into c (al * xl dropped,
  // below the double-word precision)
  __device__ __forceinline__ void mac(float ah, float al, float xh, float xl) {
    const float p = __fmul_rn(ah, xh);
    float e = __fmaf_rn(ah, xh, -p);
    e = __fmaf_rn(ah, xl, e);
    e = __fmaf_rn(al, xh, e);
    float s2, t;
    two_sum(s, p, s2, t);
    s = s2;
    c = __fadd_rn(c, __fadd_rn(t, e));
  }
  // += (h + l)
  __device__ __forceinline__ void add(float h, float l) {
    float s2, t;
    two_sum(s, h, s2, t);
    s = s2;
    c = __fadd_rn(c, __fadd_rn(t, l));
  }
  // += other accumulator
  __device__ __forceinline__ void add(const dacc& o) { add(o.s, o.c); }
  // normalised double-word (hi, lo) of the accumulated value
  __device__ __forceinline__ void get(float& hi, float& lo) const { fast_two_sum(s, c, hi, lo); }
  __device__ __forceinline__ double to_double() const { return (double)s + (double)c; }
};

// double -> double-word (round to nearest for the head, the remainder rounded for the tail)
__device__ __forceinline__ void split_double(double v, float& hi, float& lo) {
  hi = __double2float_rn(v);
  lo = __double2float_rn(v - (double)hi);
}
__device__ __forceinline__ double join_double(float hi, float lo) { return (double)hi + (double)lo; }

// complex double-word scalar from a complex double
struct cws {
  float rh, rl, ih, il;
};
__device__ __forceinline__ cws to_cws(double re, double im) {
  cws a;
  split_double(re, a.rh, a.rl);
  split_double(im, a.ih, a.il);
  return a;
}

// y + a * x for complex double-word y, x and scalar a (all in double-word):
// re = yr + ar xr - ai xi, im = yi + ar xi + ai xr
__device__ __forceinline__ cw cw_axpy(const cw& y, const cws& a, const cw& x) {
  dacc re(y.rh, y.rl), im(y.ih, y.il);
  re.mac(a.rh, a.rl, x.rh, x.rl);
  re.mac(-a.ih, -a.il, x.ih, x.il);
  im.mac(a.rh, a.rl, x.ih, x.il);
  im.mac(a.ih, a.il, x.rh, x.rl);
  cw out;
  re.get(out.rh, out.rl);
  im.get(out.ih, out.il);
  return out;
}

// unconjugated product x^T y accumulated: re += xr yr - xi yi, im += xr yi + xi yr
__device__ __forceinline__ void cw_dotu_acc(dacc& re, dacc& im, const cw& x, const cw& y) {
  re.mac(x.rh, x.rl, y.rh, y.rl);
  re.mac(-x.ih, -x.il, y.ih, y.il);
  im.mac(x.rh, x.rl, y.ih, y.il);
  im.mac(x.ih, x.il, y.rh, y.rl);
}

}  // namespace helm
