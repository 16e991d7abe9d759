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
// exp: Tang's table-driven reduction to |r| <= ln2/128 with a 64-entry
// float-float table of 2^(j/64) and a degree-6 polynomial for e^r.
// log: from the FP32 logarithm y, log x = y + log(1 + t) with
// t = x e^(-y) - 1, log(1 + t) to second order (|t| ~ 1e-7).
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

// 2^(j/64), j = 0..63, each as the nearest float plus the nearest float to
// the remainder (generated in 40-digit arithmetic)
static __device__ const float2 kExp2Tab64[64] = {
    {1.000000000e+00f, 0.000000000e+00f}, {1.010889292e+00f, -5.711605411e-09f},
    {1.021897197e+00f, -4.811559862e-08f}, {1.033024907e+00f, -2.809089317e-08f},
    {1.044273734e+00f, 4.833470157e-08f}, {1.055645227e+00f, -4.907169426e-08f},
    {1.067140460e+00f, -5.933751979e-08f}, {1.078760743e+00f, 5.461594554e-08f},
    {1.090507746e+00f, -1.307753994e-08f}, {1.102382541e+00f, 4.260501996e-08f},
    {1.114386797e+00f, -5.435540018e-08f}, {1.126521587e+00f, 3.123641434e-08f},
    {1.138788581e+00f, 5.386222313e-08f}, {1.151189208e+00f, 2.192228266e-08f},
    {1.163724899e+00f, -4.051441493e-08f}, {1.176396966e+00f, 2.566975077e-08f},
    {1.189207077e+00f, 3.797635273e-08f}, {1.202156782e+00f, -5.069756526e-08f},
    {1.215247393e+00f, -3.267394888e-08f}, {1.228480577e+00f, -4.136200360e-08f},
    {1.241857767e+00f, 4.496838102e-08f}, {1.255380750e+00f, 7.322237483e-09f},
    {1.269050956e+00f, 1.419333318e-09f}, {1.282870054e+00f, -3.816621685e-08f},
    {1.296839595e+00f, -4.018999533e-08f}, {1.310961246e+00f, -3.496571566e-08f},
    {1.325236678e+00f, -3.496373324e-08f}, {1.339667559e+00f, -3.461673970e-08f},
    {1.354255557e+00f, -1.012334927e-08f}, {1.369002461e+00f, -3.845881835e-08f},
    {1.383909941e+00f, -5.875577358e-08f}, {1.398979664e+00f, 8.689434061e-09f},
    {1.414213538e+00f, 2.420323497e-08f}, {1.429613352e+00f, -1.342992917e-08f},
    {1.445180774e+00f, 3.324199938e-08f}, {1.460917830e+00f, -3.628657552e-08f},
    {1.476826191e+00f, -4.500898854e-08f}, {1.492907763e+00f, -3.423620143e-08f},
    {1.509164453e+00f, -2.495937323e-08f}, {1.525598168e+00f, -1.762856883e-08f},
    {1.542210817e+00f, 8.070904833e-09f}, {1.559004426e+00f, -2.576466507e-08f},
    {1.575980902e+00f, -5.661025426e-08f}, {1.593142152e+00f, -4.903136785e-10f},
    {1.610490322e+00f, 9.836217174e-09f}, {1.628027439e+00f, -1.726008314e-08f},
    {1.645755529e+00f, -5.124972091e-08f}, {1.663676620e+00f, -3.920298752e-08f},
    {1.681792855e+00f, -2.475532668e-08f}, {1.700106382e+00f, -2.865147231e-08f},
    {1.718619347e+00f, -4.849617596e-08f}, {1.737333894e+00f, -5.850223417e-08f},
    {1.756252170e+00f, -9.235770371e-09f}, {1.775376439e+00f, 5.343197884e-08f},
    {1.794709086e+00f, -1.141504491e-08f}, {1.814252138e+00f, 3.736258236e-08f},
    {1.834008098e+00f, -1.123927795e-08f}, {1.853979111e+00f, 1.436561181e-08f},
    {1.874167681e+00f, -4.663005626e-08f}, {1.894575953e+00f, 2.810338451e-08f},
    {1.915206552e+00f, 9.845328108e-09f}, {1.936061740e+00f, 5.357072297e-08f},
    {1.957144141e+00f, -1.702180441e-08f}, {1.978456020e+00f, 6.032726318e-09f},
};

__device__ __forceinline__ ff ff_exp(ff x) {
  if (x.hi > 88.7f) return ff(__int_as_float(0x7f800000), 0.f);   // +inf
  if (x.hi < -103.0f) return ff(0.f, 0.f);
  // Table-driven reduction (Tang, ACM TOMS 15(2), 1989): x = (64 n + j) ln2/64
  // + r with |r| <= ln2/128; ln2/64 = L1 + L2 + L3, L1 with 9 significant
  // bits so that k * L1 is exact for every k reached here, and x.hi - k L1
  // is exact too (the operands are within a factor 2 of each other, Sterbenz
  // lemma, or k = 0).  k L3 is below 3e-10 and goes into the low part.
  const float L1 = 0.010833740234375f, L2 = -3.3155381515825866e-06f,
              L3 = 2.572804640231345e-14f;
  const float k = rintf(__fmul_rn(x.hi, 92.33248138427734f));   // 64 / ln2
  // r = x - k ln2/64 = (x.hi - k L1) - hi(k L2) + x.lo - lo(k L2) - k L3:
  // the first difference is exact, the next two terms join it by exact
  // two-sums (x.lo is as large as r's own rounding scale), and the last two
  // (below 1e-9) with the two-sums' errors in FP32.
  const float t = __fsub_rn(x.hi, __fmul_rn(k, L1));
  const ff kL2 = two_prod(k, L2);
  const ff s1 = two_sum(t, -kL2.hi);
  const ff s2 = two_sum(s1.hi, x.lo);
  ff r = two_sum(s2.hi, __fadd_rn(__fadd_rn(s1.lo, s2.lo), -__fmaf_rn(k, L3, kL2.lo)));
  // e^r - 1 = r + r^2/2 + r^2 c, c = r/6 + r^2/24 + r^3/120 + r^4/720: c is
  // below 1e-3 and needs only FP32 (its rounding is below 1e-15 of e^r);
  // the Taylor remainder r^7/5040 is below 1e-19.  |r| <= ln2/128, so
  // r^2/2 < |r|/256: the head sum needs no magnitude test, and the terms
  // below ulp(r.hi) (r.lo, the low part of r^2/2, r^2 c) go in FP32.
  const float rh = r.hi;
  const float c = __fmul_rn(rh, __fmaf_rn(rh, __fmaf_rn(rh, __fmaf_rn(rh, 1.3888889225e-3f,
                                                                           8.3333337680e-3f),
                                                       4.1666667908e-2f),
                                          1.6666667163e-1f));
  const ff r2 = two_prod(rh, rh);                       // r.hi^2 exactly
  const float h2 = __fmul_rn(0.5f, r2.hi);
  ff em1 = fast_two_sum(rh, h2);
  float tail = __fmaf_rn(r2.hi, c, __fmaf_rn(0.5f, r2.lo, r.lo));
  tail = __fmaf_rn(rh, r.lo, tail);                     // the cross term r.hi r.lo
  em1 = fast_two_sum(em1.hi, __fadd_rn(em1.lo, tail));
  const int ki = (int)k;
  const float2 t64 = __ldg(&kExp2Tab64[ki & 63]);
  // y = 2^(j/64) (1 + em1): the head product exactly, the rest in FP32
  const ff p = two_prod(t64.x, em1.hi);
  ff y = fast_two_sum(t64.x, p.hi);
  const float lo = __fmaf_rn(t64.x, em1.lo, __fmaf_rn(t64.y, em1.hi, __fadd_rn(p.lo, t64.y)));
  y = fast_two_sum(y.hi, __fadd_rn(y.lo, lo));
  // scale by 2^e: an exact multiply while 2^e is a normal float
  const int e = ki >> 6;
  if (e >= -126) {
    const float sc = __int_as_float((e + 127) << 23);
    return ff(__fmul_rn(y.hi, sc), __fmul_rn(y.lo, sc));
  }
  return ff_ldexp(y, e);
}

__device__ __forceinline__ ff ff_log(ff x) {
  // y0 = log(x.hi) in FP32 (error d below a few 1e-7 relative), then
  // log x = y0 + log(1 + t), t = x e^(-y0) - 1 (|t| ~ |d|): log(1 + t) =
  // t - t^2/2 + O(t^3), the t^2 term in FP32 (a plain Newton step y0 + t
  // would leave t^2/2, up to 1e-11 for large |log x|)
  const ff y0(logf(x.hi));
  ff t = x * ff_exp(-y0) - ff(1.f);
  t = fast_two_sum(t.hi, __fmaf_rn(-0.5f * t.hi, t.hi, t.lo));
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

}  // namespace lbm
