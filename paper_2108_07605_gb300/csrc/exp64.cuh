// FP64 exponential of the reaction rates.  No counterpart in the paper (its
// rates come from Cantera); a published method, restated.
#pragma once

#include <cuda_runtime.h>

namespace lbm {

// exp in FP64 by Tang's table-driven method (P. T. P. Tang, ACM TOMS 15(2),
// 1989): x = (32 m + j) ln2/32 + r with |r| <= ln2/64 (ln2/32 split into
// its double and the double of the remainder, so r is exact to rounding),
// e^x = 2^m 2^(j/32) e^r, e^r - 1 by its Taylor polynomial to degree 6
// (truncation below 4e-18), 2^(j/32) from a table of the nearest doubles
// (60-digit arithmetic), 2^m added to the exponent field.  Within 2 ulp of
// e^x; arguments beyond |x| = 700 (never met by the rates) and NaN go to
// the library exp.
static __device__ const double kExp2Tab32[32] = {
    0x1.0000000000000p+0, 0x1.059b0d3158574p+0, 0x1.0b5586cf9890fp+0,
    0x1.11301d0125b51p+0, 0x1.172b83c7d517bp+0, 0x1.1d4873168b9aap+0,
    0x1.2387a6e756238p+0, 0x1.29e9df51fdee1p+0, 0x1.306fe0a31b715p+0,
    0x1.371a7373aa9cbp+0, 0x1.3dea64c123422p+0, 0x1.44e086061892dp+0,
    0x1.4bfdad5362a27p+0, 0x1.5342b569d4f82p+0, 0x1.5ab07dd485429p+0,
    0x1.6247eb03a5585p+0, 0x1.6a09e667f3bcdp+0, 0x1.71f75e8ec5f74p+0,
    0x1.7a11473eb0187p+0, 0x1.82589994cce13p+0, 0x1.8ace5422aa0dbp+0,
    0x1.93737b0cdc5e5p+0, 0x1.9c49182a3f090p+0, 0x1.a5503b23e255dp+0,
    0x1.ae89f995ad3adp+0, 0x1.b7f76f2fb5e47p+0, 0x1.c199bdd85529cp+0,
    0x1.cb720dcef9069p+0, 0x1.d5818dcfba487p+0, 0x1.dfc97337b9b5fp+0,
    0x1.ea4afa2a490dap+0, 0x1.f50765b6e4540p+0};

__device__ __forceinline__ double exp_tang(double x) {
  if (!(fabs(x) <= 700.0)) return exp(x);
  const double K = 46.16624130844683;                // 32 / ln2
  const double L1 = 0x1.62e42fefa39efp-6;            // double(ln2) / 32
  const double L2 = 0x1.abc9e3b39803fp-61;           // (ln2 - double(ln2)) / 32
  const double SH = 0x1.8p52;                        // rounds to an integer
  const double t = fma(x, K, SH);
  const double n = t - SH;
  const int ni = __double2loint(t);
  double r = fma(-n, L1, x);
  r = fma(-n, L2, r);
  double p = fma(r, 1.0 / 720.0, 1.0 / 120.0);
  p = fma(p, r, 1.0 / 24.0);
  p = fma(p, r, 1.0 / 6.0);
  p = fma(p, r, 0.5);
  p = fma(p * r, r, r);                              // e^r - 1
  const double tj = __ldg(&kExp2Tab32[ni & 31]);
  const double y = fma(tj, p, tj);
  return __longlong_as_double(__double_as_longlong(y) + ((long long)(ni >> 5) << 52));
}

}  // namespace lbm
