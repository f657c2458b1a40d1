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


// ---------------------------------------------------------------------------------------------
// Packed form: two independent double-word accumulations (in practice the real and the
// imaginary component of one complex value) carried in float2 registers and advanced with the
// paired FP32 instructions of sm_100-class GPUs (__ffma2_rn, __fadd2_rn, __fmul2_rn: two
// correctly rounded FP32 operations per instruction). Every component follows exactly the
// operation sequence of `dacc` above, so results are bitwise those of two scalar accumulators;
// subtractions are written as fma(b, -1, a) = fl(a - b) and the product error as the sum of
// ah*xh and the exact negation of its rounded value, so no separate negation is needed.
// ---------------------------------------------------------------------------------------------
namespace dw2 {
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
}  // namespace dw2

struct dacc2 {
  float2 s, c;  // component k holds the double-word value s.k + c.k
  __device__ __forceinline__ dacc2() : s(make_float2(0.f, 0.f)), c(make_float2(0.f, 0.f)) {}
  // += (ah + al)(xh + xl) per component (the scalar mac with the same operations): exact head
  // product, low-order cross terms into c
  __device__ __forceinline__ void mac(float2 ah, float2 al, float2 xh, float2 xl) {
    using namespace dw2;
    const float2 np = mul(f2(-ah.x, -ah.y), xh);  // -fl(ah xh), exactly
    float2 e = fma(ah, xh, np);                    // ah xh - fl(ah xh)
    e = fma(ah, xl, e);
    e = fma(al, xh, e);
    // TwoSum(s, p) with p = -np: s2 = fl(s + p), bb = fl(s2 - s) (kept negated: nbb = fl(s - s2))
    const float2 s2 = sub(s, np);
    const float2 nbb = sub(s, s2);
    const float2 da = sub(s, dw2::add(s2, nbb));  // s - (s2 - bb)
    const float2 db = sub(nbb, np);               // p - bb
    const float2 t = dw2::add(da, db);
    s = s2;
    c = dw2::add(c, dw2::add(t, e));
  }
  // += (h + l) per component
  __device__ __forceinline__ void add(float2 h, float2 l) {
    using namespace dw2;
    const float2 s2 = dw2::add(s, h);
    const float2 bb = sub(s2, s);
    const float2 t = dw2::add(sub(s, sub(s2, bb)), sub(h, bb));
    s = s2;
    c = dw2::add(c, dw2::add(t, l));
  }
  __device__ __forceinline__ void add(const dacc2& o) { add(o.s, o.c); }
  // normalised (hi, lo) per component (FastTwoSum of s and c)
  __device__ __forceinline__ void get(float2& hi, float2& lo) const {
    using namespace dw2;
    hi = dw2::add(s, c);
    lo = sub(c, sub(hi, s));
  }
};

// complex double-word value as the packed pair of its components' heads and tails
__device__ __forceinline__ float2 cw_hi(const cw& v) { return make_float2(v.rh, v.ih); }
__device__ __forceinline__ float2 cw_lo(const cw& v) { return make_float2(v.rl, v.il); }
__device__ __forceinline__ cw cw_from(float2 hi, float2 lo) { return cw{hi.x, lo.x, hi.y, lo.y}; }

// y + a x, bitwise equal to cw_axpy: per component re = yr + ar xr - ai xi, im = yi + ar xi + ai xr
__device__ __forceinline__ cw cw_axpy2(const cw& y, const cws& a, const cw& x) {
  dacc2 acc;
  acc.s = cw_hi(y);
  acc.c = cw_lo(y);
  acc.mac(make_float2(a.rh, a.rh), make_float2(a.rl, a.rl), cw_hi(x), cw_lo(x));
  acc.mac(make_float2(-a.ih, a.ih), make_float2(-a.il, a.il), make_float2(x.ih, x.rh), make_float2(x.il, x.rl));
  float2 hi, lo;
  acc.get(hi, lo);
  return cw_from(hi, lo);
}

// (re, im) += x^T y, bitwise equal to cw_dotu_acc on (re, im)
__device__ __forceinline__ void cw_dotu_acc2(dacc2& acc, const cw& x, const cw& y) {
  acc.mac(make_float2(x.rh, x.rh), make_float2(x.rl, x.rl), cw_hi(y), cw_lo(y));
  acc.mac(make_float2(-x.ih, x.ih), make_float2(-x.il, x.il), make_float2(y.ih, y.rh), make_float2(y.il, y.rl));
}

}  // namespace helm
