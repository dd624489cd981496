// dd.cuh — double-double ("DD") arithmetic on the FP64 pipe.
//
// A DD number is the unevaluated sum hi + lo of two doubles with
// |lo| <= ulp(hi)/2 (arXiv:1806.01036, Sec. 4.2: "numbers represented by two
// doubles").  Every routine here is an error-free transformation or a DD
// algorithm from the literature the paper builds on:
//   two_sum       Knuth / Moller TwoSum (6 flops, no precondition)
//   fast_two_sum  Dekker Fast2Sum (3 flops, needs |a| >= |b| or a == 0)
//   two_prod      TwoProd with a fused multiply-add (2 flops)
//   dd_add        Joldes-Muller-Popescu 2017, "AccurateDWPlusDW"
//   dd_mul        Joldes-Muller-Popescu 2017, "DWTimesDW3"
//   dd_mul_d      Joldes-Muller-Popescu 2017, "DWTimesFP3"
//   dd_div        Newton-Raphson (Karp-Markstein) correction of the FP64
//                 quotient, carried out in DD, as the paper prescribes for
//                 divisions and square roots
//   dd_sqrt       one Newton-Raphson (Karp-Markstein) step from the FP64 root
// The explicit __dadd_rn/__dmul_rn/__fma_rn intrinsics keep the compiler from
// contracting or reassociating any step.
#pragma once

#include <cuda_runtime.h>

namespace eo {

struct dd {
  double hi, lo;
};

__device__ __forceinline__ dd dd_make(double hi, double lo = 0.0) { return dd{hi, lo}; }

__device__ __forceinline__ dd two_sum(double a, double b) {
  double s = __dadd_rn(a, b);
  double bv = __dsub_rn(s, a);
  double av = __dsub_rn(s, bv);
  double e = __dadd_rn(__dsub_rn(a, av), __dsub_rn(b, bv));
  return dd{s, e};
}

__device__ __forceinline__ dd fast_two_sum(double a, double b) {
  double s = __dadd_rn(a, b);
  double e = __dsub_rn(b, __dsub_rn(s, a));
  return dd{s, e};
}

__device__ __forceinline__ dd two_prod(double a, double b) {
  double p = __dmul_rn(a, b);
  double e = __fma_rn(a, b, -p);
  return dd{p, e};
}

__device__ __forceinline__ dd dd_add(dd x, dd y) {
  dd s = two_sum(x.hi, y.hi);
  dd t = two_sum(x.lo, y.lo);
  double c = __dadd_rn(s.lo, t.hi);
  dd v = fast_two_sum(s.hi, c);
  double w = __dadd_rn(t.lo, v.lo);
  return fast_two_sum(v.hi, w);
}

__device__ __forceinline__ dd dd_neg(dd x) { return dd{-x.hi, -x.lo}; }
__device__ __forceinline__ dd dd_sub(dd x, dd y) { return dd_add(x, dd_neg(y)); }

__device__ __forceinline__ dd dd_mul(dd x, dd y) {
  dd c = two_prod(x.hi, y.hi);
  double tl0 = __dmul_rn(x.lo, y.lo);
  double tl1 = __fma_rn(x.hi, y.lo, tl0);
  double cl2 = __fma_rn(x.lo, y.hi, tl1);
  double cl3 = __dadd_rn(c.lo, cl2);
  return fast_two_sum(c.hi, cl3);
}

__device__ __forceinline__ dd dd_mul_d(dd x, double y) {
  dd c = two_prod(x.hi, y);
  double cl3 = __fma_rn(x.lo, y, c.lo);
  return fast_two_sum(c.hi, cl3);
}

// Accumulate the exact product a*b into the DD sum s (Ogita-Rump-Oishi Dot2
// step: TwoProd, TwoSum of the high parts, low parts summed in FP64).
__device__ __forceinline__ void dd_fma_acc(dd& s, double a, double b) {
  dd p = two_prod(a, b);
  dd t = two_sum(s.hi, p.hi);
  s.hi = t.hi;
  s.lo = __dadd_rn(s.lo, __dadd_rn(t.lo, p.lo));
}

// s += x * b for DD x and FP64 b (the Dot2 step with the low part of x folded
// into the FP64 error term).
__device__ __forceinline__ void dd_fma_acc_dd(dd& s, dd x, double b) {
  dd p = two_prod(x.hi, b);
  double pl = __fma_rn(x.lo, b, p.lo);
  dd t = two_sum(s.hi, p.hi);
  s.hi = t.hi;
  s.lo = __dadd_rn(s.lo, __dadd_rn(t.lo, pl));
}

// Renormalize an accumulator so that |lo| <= ulp(hi)/2 (TwoSum: after
// cancellation the low part of a Dot2 accumulator may exceed the high part).
__device__ __forceinline__ dd dd_norm(dd s) { return two_sum(s.hi, s.lo); }

// q = x / y: FP64 quotient, then two Newton-Raphson corrections
// q <- q + (x - y q) / y with the residual evaluated in DD.
__device__ __forceinline__ dd dd_div(dd x, dd y) {
  double q0 = __ddiv_rn(x.hi, y.hi);
  dd r = dd_sub(x, dd_mul_d(y, q0));
  double q1 = __ddiv_rn(r.hi, y.hi);
  dd q = fast_two_sum(q0, q1);
  dd r2 = dd_sub(x, dd_mul(y, q));
  double q2 = __ddiv_rn(r2.hi, y.hi);
  return dd_add(q, dd_make(q2));
}

__device__ __forceinline__ dd dd_recip(dd y) { return dd_div(dd_make(1.0), y); }

// sqrt(x) for x > 0: s = sqrt(x.hi), then s + (x - s^2) / (2 s) in DD.
__device__ __forceinline__ dd dd_sqrt(dd x) {
  if (!(x.hi > 0.0)) return dd_make(0.0);
  double s = __dsqrt_rn(x.hi);
  dd e = dd_sub(x, two_prod(s, s));
  double c = __ddiv_rn(e.hi, __dmul_rn(2.0, s));
  return fast_two_sum(s, c);
}

__device__ __forceinline__ bool dd_finite(dd x) { return isfinite(x.hi) && isfinite(x.lo); }

}  // namespace eo
