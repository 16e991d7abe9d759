// Float-float ("double-FP32") arithmetic for the mixed-precision path.
//
// GB300 executes FP32 about 55x faster than FP64 (measured 68.6 vs 1.25
// TFLOP/s FMA), so the mixed path evaluates its FP64-class work - the
// temperature Newton solve, transport and the Arrhenius chemistry - on pairs
// of floats.  A value is hi + lo with |lo| <= ulp(hi)/2, about 48 significant
// bits (relative precision ~4e-15), with the exponent range of FP32.
//
// Error-free transformations (published methods):
//   two_sum       Knuth, TAOCP vol. 2: s + e = a + b exactly;
//   fast_two_sum  Dekker 1971: the same when |a| >= |b|;
//   two_prod      with a fused multiply-add: p + e = a * b exactly.
// exp: x = k ln2 + r (|r| <= ln2/2, ln2 carried in three parts so k*ln2 is
// exact), e^r = (e^(r/4))^4 with the Taylor series of e^(r/4) to degree 11
// (truncation below 1e-21), times 2^k.  log: one Newton step
// y <- y + x e^(-y) - 1 from the FP32 logarithm (quadratic convergence takes
// the 1e-7 start to the float-float precision).
// Intrinsics with explicit rounding keep the compiler from contracting or
// reassociating the transformations.
#pragma once

#include <cuda_runtime.h>

namespace lbm {

struct ff {
  float hi, lo;
  __host__ __device__ ff() : hi(0.f), lo(0.f) {}
  __host__ __device__ ff(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ explicit ff(float h) : hi(h), lo(0.f) {}
};

__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return ff(s, e);
}
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return ff(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ ff two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return ff(p, __fmaf_rn(a, b, -p));
}

__device__ __forceinline__ ff operator+(ff a, ff b) {
  ff s = two_sum(a.hi, b.hi);
  const ff t = two_sum(a.lo, b.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = fast_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ ff operator-(ff a) { return ff(-a.hi, -a.lo); }
__device__ __forceinline__ ff operator-(ff a, ff b) { return a + (-b); }
__device__ __forceinline__ ff operator*(ff a, ff b) {
  ff p = two_prod(a.hi, b.hi);
  p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
  p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
  return fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ ff operator/(ff a, ff b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const ff r = a - b * ff(q1);
  const float q2 = __fdiv_rn(r.hi, b.hi);
  const ff r2 = r - b * ff(q2);
  const float q3 = __fdiv_rn(r2.hi, b.hi);
  return fast_two_sum(q1, q2) + ff(q3);
}
__device__ __forceinline__ ff& operator+=(ff& a, ff b) { return a = a + b; }
__device__ __forceinline__ ff& operator-=(ff& a, ff b) { return a = a - b; }
__device__ __forceinline__ ff& operator*=(ff& a, ff b) { return a = a * b; }

// scale by 2^k exactly (k small)
__device__ __forceinline__ ff ff_ldexp(ff a, int k) {
  return ff(ldexpf(a.hi, k), ldexpf(a.lo, k));
}

__device__ __forceinline__ ff ff_exp(ff x) {
  if (x.hi > 88.7f) return ff(__int_as_float(0x7f800000), 0.f);   // +inf
  if (x.hi < -103.0f) return ff(0.f, 0.f);
  // ln2 = L1 + L2 + L3, L1 with 15 significant bits so k * L1 is exact
  const float L1 = 0.693145751953125f, L2 = 1.428606765330187e-06f,
              L3 = 5.497923148104107e-14f;
  const float k = rintf(__fmul_rn(x.hi, 1.4426950408889634f));
  ff r = x - ff(__fmul_rn(k, L1));
  r = r - two_prod(k, L2);
  r = r - ff(__fmul_rn(k, L3));
  const ff s = ff_ldexp(r, -2);
  // Taylor coefficients 1/n!, n = 11..0, split hi + lo
  const float ch[12] = {2.5052107943679403e-08f, 2.755731998149713e-07f,
                        2.7557318844628753e-06f, 2.4801587642286904e-05f,
                        0.00019841270113829523f, 0.0013888889225199819f,
                        0.008333333767950535f, 0.0416666679084301f,
                        0.1666666716337204f, 0.5f, 1.0f, 1.0f};
  const float cl[12] = {4.4176230446483665e-16f, -7.575112209051195e-15f,
                        3.793571224297229e-14f, -3.40699609366682e-13f,
                        -2.725596874933456e-12f, -3.3631094437103215e-11f,
                        -4.34617203337595e-10f, -1.2417634698280722e-09f,
                        -4.967053879312289e-09f, 0.f, 0.f, 0.f};
  ff p(ch[0], cl[0]);
#pragma unroll
  for (int n = 1; n < 12; ++n) p = p * s + ff(ch[n], cl[n]);
  p = p * p;
  p = p * p;
  return ff_ldexp(p, (int)k);
}

__device__ __forceinline__ ff ff_log(ff x) {
  const ff y0(logf(x.hi));
  const ff t = x * ff_exp(-y0) - ff(1.f);
  return y0 + t;
}

__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ ff ff_from_double(double d) {
  const float h = __double2float_rn(d);
  return ff(h, __double2float_rn(d - (double)h));
}
__host__ inline ff ff_host(double d) {
  const float h = (float)d;
  return ff(h, (float)(d - (double)h));
}
__device__ __forceinline__ float ff_abs_hi(ff a) { return fabsf(a.hi); }

}  // namespace lbm
