// ff.cuh -- float-float ("double-float") arithmetic on the FP32 pipe.
//
// A value is an unevaluated pair h + l of floats with |l| <= ulp(h) / 2, about 48 significant
// bits.  GB300 runs FP64 at 1/64 of the FP32 rate with a 64-cycle latency, so the per-proposal
// constants of the float-float likelihood path are formed here instead of in FP64.  The
// algorithms are the classical error-free transformations (Dekker 1971; Knuth's two-sum) and
// their double-float compositions (as in Hida, Li & Bailey's QD library, reimplemented);
// log and sin/cos use argument reduction and Taylor series written out from the mathematics.
// Accuracy of each operation: a few units of 2^-44 relative (products, quotients, roots, sums
// that do not cancel); log and sin/cos about 1e-13 absolute on the ranges used here -- far
// below the 1e-6 cycle the phase needs.
#pragma once

#include <cstdint>

namespace gwns {

struct ff {
  float h, l;
};

// Compile-time split of a double constant into a float pair.
#define GWNS_FF(x) (::gwns::ff{(float)(x), (float)((x) - (double)(float)(x))})

__device__ __forceinline__ ff ff_make(float h) { return ff{h, 0.0f}; }

// s + e = a + b exactly.
__device__ __forceinline__ ff two_sum_ff(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return ff{s, (a - (s - bb)) + (b - bb)};
}
// s + e = a + b exactly, for |a| >= |b| (or a = 0).
__device__ __forceinline__ ff fast_two_sum_ff(float a, float b) {
  const float s = a + b;
  return ff{s, b - (s - a)};
}
// p + e = a b exactly (FMA).
__device__ __forceinline__ ff two_prod_ff(float a, float b) {
  const float p = a * b;
  return ff{p, fmaf(a, b, -p)};
}

// The low parts are added without their own error term: relative error about 2^-44 times
// (|a| + |b|) / |a + b|.  No sum in this library's uses cancels by more than a few digits.
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  ff s = two_sum_ff(a.h, b.h);
  s.l += a.l + b.l;
  return fast_two_sum_ff(s.h, s.l);
}
__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.h, -a.l}; }
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }
__device__ __forceinline__ ff ff_add_f(ff a, float b) {
  ff s = two_sum_ff(a.h, b);
  s.l += a.l;
  return fast_two_sum_ff(s.h, s.l);
}
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  ff p = two_prod_ff(a.h, b.h);
  p.l = fmaf(a.h, b.l, fmaf(a.l, b.h, p.l));
  return fast_two_sum_ff(p.h, p.l);
}
__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
  ff p = two_prod_ff(a.h, b);
  p.l = fmaf(a.l, b, p.l);
  return fast_two_sum_ff(p.h, p.l);
}
// a * 2^k exactly (no overflow or underflow on the ranges used).
__device__ __forceinline__ ff ff_ldexp(ff a, int k) { return ff{ldexpf(a.h, k), ldexpf(a.l, k)}; }

__device__ __forceinline__ ff ff_div(ff a, ff b) {
  const float q1 = a.h / b.h;
  const ff p = two_prod_ff(q1, b.h);
  const float r = (((a.h - p.h) - p.l) + a.l) - q1 * b.l;
  const float q2 = r / b.h;
  return fast_two_sum_ff(q1, q2);
}
__device__ __forceinline__ ff ff_sqrt(ff a) {
  if (!(a.h > 0.0f)) return ff{0.0f, 0.0f};
  const float s = sqrtf(a.h);
  const ff p = two_prod_ff(s, s);
  const float r = ((a.h - p.h) - p.l) + a.l;
  return fast_two_sum_ff(s, r / (2.0f * s));
}
// a^(-1/3), a > 0: FP32 seed (relative error ~1e-7), one Newton step w <- w + w (1 - a w^3)/3
// with the residual formed in float-float (error ~1e-14 after it).
__device__ __forceinline__ ff ff_rcbrt(ff a) {
  ff w = ff_make(rcbrtf(a.h));
  {
    const ff t = ff_mul(a, ff_mul(ff_mul(w, w), w));
    const float r = (1.0f - t.h) - t.l;
    w = ff_add(w, ff_mul_f(w, r * (1.0f / 3.0f)));
  }
  return w;
}
// a^(-1/5), a > 0: FP32 seed, one Newton step z <- z + z (1 - a z^5) / 5.
__device__ __forceinline__ ff ff_rfifth(ff a) {
  ff z = ff_make(powf(a.h, -0.2f));
  {
    const ff z2 = ff_mul(z, z);
    const ff t = ff_mul(a, ff_mul(ff_mul(z2, z2), z));
    const float r = (1.0f - t.h) - t.l;
    z = ff_add(z, ff_mul_f(z, r * 0.2f));
  }
  return z;
}

// ln a, a > 0: a = m 2^e with m in [1/sqrt 2, sqrt 2), ln a = e ln 2 + 2 atanh(y),
// y = (m - 1) / (m + 1), |y| <= 0.1716, atanh(y) = y (1 + y^2/3 + y^4/5 + ... + y^16/17)
// (truncation below 2e-15).
__device__ __forceinline__ ff ff_log(ff a) {
  int e;
  float m = frexpf(a.h, &e);
  if (m < 0.70710678f) --e;
  const ff x = ff_ldexp(a, -e);
  const ff y = ff_div(ff_add_f(x, -1.0f), ff_add_f(x, 1.0f));
  const ff y2 = ff_mul(y, y);
  ff s = GWNS_FF(1.0 / 17.0);
  s = ff_add(ff_mul(s, y2), GWNS_FF(1.0 / 15.0));
  s = ff_add(ff_mul(s, y2), GWNS_FF(1.0 / 13.0));
  s = ff_add(ff_mul(s, y2), GWNS_FF(1.0 / 11.0));
  s = ff_add(ff_mul(s, y2), GWNS_FF(1.0 / 9.0));
  s = ff_add(ff_mul(s, y2), GWNS_FF(1.0 / 7.0));
  s = ff_add(ff_mul(s, y2), GWNS_FF(1.0 / 5.0));
  s = ff_add(ff_mul(s, y2), GWNS_FF(1.0 / 3.0));
  s = ff_add_f(ff_mul(s, y2), 1.0f);
  const ff at2 = ff_ldexp(ff_mul(y, s), 1);
  return ff_add(ff_mul_f(GWNS_FF(0.6931471805599453), (float)e), at2);
}

// ln(U0 U1 U2 U3) for the open-unit uniforms U_i = ((x_i >> 12) + 1/2) / 2^52 of four Philox
// words: each U_i as a float pair (the 53-bit numerator split exactly into 24 + 29 bits, the
// low part rounded to 24), mantissas multiplied in [2^-4, 1) and the binary exponents summed,
// so nothing underflows; one float-float logarithm.
__device__ __forceinline__ ff ff_log_uniform_product(const uint64_t* x) {
  ff prod = ff_make(1.0f);
  int esum = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint64_t m2 = ((x[i] >> 12) << 1) | 1ull;        // 2 (x >> 12) + 1 < 2^53
    // top 24 bits (exact in a float) and the low 29 bits, each converted from 32 bits
    const float hi = __uint2float_rn((uint32_t)(m2 >> 29)) * 536870912.0f;
    const float lo = __uint2float_rn((uint32_t)(m2 & ((1ull << 29) - 1ull)));
    ff u = fast_two_sum_ff(hi, lo);
    int e;
    frexpf(u.h, &e);
    u = ff_ldexp(u, -e);                                    // u in [0.5, 1)
    esum += e - 53;                                         // U_i = u 2^(e - 53)
    prod = ff_mul(prod, u);
  }
  return ff_add(ff_log(prod), ff_mul_f(GWNS_FF(0.6931471805599453), (float)esum));
}

// sin and cos of a, |a| < 2^20: a = k pi/2 + r with |r| <= pi/4 (pi/2 as float + float pair),
// Taylor series in r^2 to r^15 / r^14 (truncation below 3e-14), then the quadrant.
__device__ __forceinline__ void ff_sincos(ff a, ff& s_out, ff& c_out) {
  const float k = rintf(a.h * 0.63661977f);
  // pi/2 = P1 + P23: P1 = float(pi/2), P23 the remainder as a float pair
  const float P1 = 1.5707963705062866f;
  const ff P23 = GWNS_FF(1.5707963267948966 - 1.5707963705062866);
  ff r = ff_sub(a, two_prod_ff(k, P1));             // k P1 exactly, as a pair
  r = ff_sub(r, ff_mul_f(P23, k));
  const ff r2 = ff_mul(r, r);
  // sin r = r (1 - r^2/3! + r^4/5! - ... - r^14/15!)
  ff ps = GWNS_FF(-1.0 / 1307674368000.0);           // -1/15!
  ps = ff_add(ff_mul(ps, r2), GWNS_FF(1.0 / 6227020800.0));
  ps = ff_add(ff_mul(ps, r2), GWNS_FF(-1.0 / 39916800.0));
  ps = ff_add(ff_mul(ps, r2), GWNS_FF(1.0 / 362880.0));
  ps = ff_add(ff_mul(ps, r2), GWNS_FF(-1.0 / 5040.0));
  ps = ff_add(ff_mul(ps, r2), GWNS_FF(1.0 / 120.0));
  ps = ff_add(ff_mul(ps, r2), GWNS_FF(-1.0 / 6.0));
  ps = ff_add_f(ff_mul(ps, r2), 1.0f);
  const ff sr = ff_mul(r, ps);
  // cos r = 1 - r^2/2! + r^4/4! - ... - r^14/14!
  ff pc = GWNS_FF(-1.0 / 87178291200.0);             // -1/14!
  pc = ff_add(ff_mul(pc, r2), GWNS_FF(1.0 / 479001600.0));
  pc = ff_add(ff_mul(pc, r2), GWNS_FF(-1.0 / 3628800.0));
  pc = ff_add(ff_mul(pc, r2), GWNS_FF(1.0 / 40320.0));
  pc = ff_add(ff_mul(pc, r2), GWNS_FF(-1.0 / 720.0));
  pc = ff_add(ff_mul(pc, r2), GWNS_FF(1.0 / 24.0));
  pc = ff_add(ff_mul(pc, r2), GWNS_FF(-1.0 / 2.0));
  const ff cr = ff_add_f(ff_mul(pc, r2), 1.0f);
  const int q = ((int)k) & 3;
  if (q == 0) { s_out = sr; c_out = cr; }
  else if (q == 1) { s_out = cr; c_out = ff_neg(sr); }
  else if (q == 2) { s_out = ff_neg(sr); c_out = ff_neg(cr); }
  else { s_out = ff_neg(cr); c_out = sr; }
}

}  // namespace gwns
