// Arithmetic on pairs of FP32 values (x = hi + lo, |lo| <= ulp(hi) / 2): about 48
// significant bits on the FP32 pipes.  The building blocks are the error-free
// transformations of Knuth (two-sum) and Dekker (fast two-sum), and the exact product
// error from one FMA.  Every rounded operation is written with an explicit rounding
// intrinsic so that the compiler cannot contract a product and a sum into one FMA,
// which would break the error terms.
#pragma once
#include <cstdint>

namespace iaskit {
namespace fp2 {

struct pair {
  float h, l;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float z = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}
// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ pair renorm(float s, float e) {
  pair r;
  fast_two_sum(s, e, r.h, r.l);
  return r;
}
__device__ __forceinline__ pair add(pair a, pair b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  e = __fadd_rn(e, __fadd_rn(a.l, b.l));
  return renorm(s, e);
}
__device__ __forceinline__ pair add(pair a, float b) {
  float s, e;
  two_sum(a.h, b, s, e);
  return renorm(s, __fadd_rn(e, a.l));
}
__device__ __forceinline__ pair mul(pair a, pair b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return renorm(p, e);
}
__device__ __forceinline__ pair from_double(double x) {
  const float h = __double2float_rn(x);
  return pair{h, __double2float_rn(x - (double)h)};
}

// exp(x) for x <= 0 given as a pair, as a pair with a relative error of a few 2^-48.
// Method: Cody and Waite's additive range reduction x = k ln 2 + r, |r| <= ln 2 / 2,
// with ln 2 split into three FP32 parts (the first with 14 significant bits, so that
// k * LN2_1 is exact for |k| < 512); then r' = r / 32, expm1(r') from its Taylor
// series (terms up to r'^6; the next one is below 2^-60), five doublings
// expm1(2 y) = expm1(y) (expm1(y) + 2), and the scaling by 2^k.  Arguments below -87
// return 0 (the value, below 1.7e-38, is under the FP32 normal range).
// The constants are ln 2 = 0.693147180559945309417232121458... split as
// LN2_1 + LN2_2 + LN2_3 (the remainder is 1.3e-21), and 1/6 as a pair.
__device__ __forceinline__ pair exp_neg(pair x) {
  constexpr float LN2_1 = 0x1.62e4p-1f, LN2_2 = 0x1.7f7d1cp-20f, LN2_3 = 0x1.ef357ap-45f;
  constexpr float LOG2E = 0x1.715476p+0f;
  constexpr float SIXTH_H = 0x1.555556p-3f, SIXTH_L = -0x1.555556p-28f;
  if (!(x.h > -87.0f)) return pair{0.0f, 0.0f};
  if (x.h >= 0.0f && x.l >= 0.0f) x = pair{0.0f, 0.0f};  // the argument of a kernel value is <= 0
  const float k = rintf(__fmul_rn(x.h, LOG2E));
  // r = x - k ln 2 as a pair
  const float t1 = fmaf(-k, LN2_1, x.h);  // exact: k LN2_1 is exact and t1 is near 0 (Sterbenz)
  const float p2 = __fmul_rn(k, LN2_2);
  const float e2 = fmaf(k, LN2_2, -p2);
  float s, e, s2, e3;
  two_sum(t1, -p2, s, e);
  two_sum(s, x.l, s2, e3);
  const float lo = fmaf(-k, LN2_3, __fsub_rn(__fadd_rn(e, e3), e2));
  pair r = renorm(s2, lo);
  r.h = __fmul_rn(r.h, 0.03125f);  // exact scaling by 2^-5
  r.l = __fmul_rn(r.l, 0.03125f);
  // expm1(r) = r + r^2 (1/2 + r (1/6 + r (1/24 + r (1/120 + r / 720))))
  const float q2 = fmaf(r.h, fmaf(r.h, 1.0f / 720.0f, 1.0f / 120.0f), 1.0f / 24.0f);
  const pair q1 = add(pair{SIXTH_H, SIXTH_L}, __fmul_rn(r.h, q2));
  const pair q = add(mul(r, q1), 0.5f);
  pair m = add(r, mul(mul(r, r), q));
  // five doublings: expm1(2 y) = expm1(y) (expm1(y) + 2)
#pragma unroll
  for (int i = 0; i < 5; ++i) m = mul(m, add(m, 2.0f));
  // exp = 1 + expm1, times 2^k (k >= -126 here: a normal power of two)
  const pair v = add(m, 1.0f);
  const float scale = __int_as_float(((int)k + 127) << 23);
  return pair{__fmul_rn(v.h, scale), __fmul_rn(v.l, scale)};
}

}  // namespace fp2
}  // namespace iaskit
