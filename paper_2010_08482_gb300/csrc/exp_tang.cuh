// e^x for the propagator arguments x = -dtau (E - E_min) <= 0 with fewer
// float64 instructions than the general exponential: GB300 issues float64
// at 1/64 of the float32 rate, and the small-block trace kernel computes one
// exponential per distinct energy level of every visited sector.
//
// Method: P. T. P. Tang, "Table-driven implementation of the exponential
// function in IEEE floating-point arithmetic", ACM TOMS 15 (1989) 144-157,
// here with 64 table entries:
//   x = (64 m + j) ln2/64 + r,  0 <= j < 64,  |r| <= ln2/128 (+ rounding),
//   e^x = 2^m * 2^{j/64} * e^r,
// e^r from its Taylor polynomial of degree 5 (remainder below
// |r|^6/720 < 3.5e-17 relative), n = 64 m + j the nearest integer of
// x * 64/ln2 (the 1.5 * 2^52 shifter), r by a two-part (Cody-Waite)
// reduction whose high part has 32 significant bits, so n * high is exact
// for |n| < 2^21.  2^{j/64} are the float64 values nearest to the exact
// powers (checked digit by digit on the CPU by the tests); 2^m enters by an
// integer add to the exponent field while the result stays normal.
// Error: within 2 ulp of e^x (table 0.5 ulp, polynomial and its Horner
// roundings about 1 ulp, the final product 0.5 ulp).
#pragma once

#include <cuda_runtime.h>

namespace ctq {
namespace dev {

__device__ const double kExp2Frac64[64] = {
    0x1.0000000000000p+0, 0x1.02c9a3e778061p+0, 0x1.059b0d3158574p+0, 0x1.0874518759bc8p+0,
    0x1.0b5586cf9890fp+0, 0x1.0e3ec32d3d1a2p+0, 0x1.11301d0125b51p+0, 0x1.1429aaea92de0p+0,
    0x1.172b83c7d517bp+0, 0x1.1a35beb6fcb75p+0, 0x1.1d4873168b9aap+0, 0x1.2063b88628cd6p+0,
    0x1.2387a6e756238p+0, 0x1.26b4565e27cddp+0, 0x1.29e9df51fdee1p+0, 0x1.2d285a6e4030bp+0,
    0x1.306fe0a31b715p+0, 0x1.33c08b26416ffp+0, 0x1.371a7373aa9cbp+0, 0x1.3a7db34e59ff7p+0,
    0x1.3dea64c123422p+0, 0x1.4160a21f72e2ap+0, 0x1.44e086061892dp+0, 0x1.486a2b5c13cd0p+0,
    0x1.4bfdad5362a27p+0, 0x1.4f9b2769d2ca7p+0, 0x1.5342b569d4f82p+0, 0x1.56f4736b527dap+0,
    0x1.5ab07dd485429p+0, 0x1.5e76f15ad2148p+0, 0x1.6247eb03a5585p+0, 0x1.6623882552225p+0,
    0x1.6a09e667f3bcdp+0, 0x1.6dfb23c651a2fp+0, 0x1.71f75e8ec5f74p+0, 0x1.75feb564267c9p+0,
    0x1.7a11473eb0187p+0, 0x1.7e2f336cf4e62p+0, 0x1.82589994cce13p+0, 0x1.868d99b4492edp+0,
    0x1.8ace5422aa0dbp+0, 0x1.8f1ae99157736p+0, 0x1.93737b0cdc5e5p+0, 0x1.97d829fde4e50p+0,
    0x1.9c49182a3f090p+0, 0x1.a0c667b5de565p+0, 0x1.a5503b23e255dp+0, 0x1.a9e6b5579fdbfp+0,
    0x1.ae89f995ad3adp+0, 0x1.b33a2b84f15fbp+0, 0x1.b7f76f2fb5e47p+0, 0x1.bcc1e904bc1d2p+0,
    0x1.c199bdd85529cp+0, 0x1.c67f12e57d14bp+0, 0x1.cb720dcef9069p+0, 0x1.d072d4a07897cp+0,
    0x1.d5818dcfba487p+0, 0x1.da9e603db3285p+0, 0x1.dfc97337b9b5fp+0, 0x1.e502ee78b3ff6p+0,
    0x1.ea4afa2a490dap+0, 0x1.efa1bee615a27p+0, 0x1.f50765b6e4540p+0, 0x1.fa7c1819e90d8p+0,
};

// v * 2^k, exact: an integer add to the exponent field when v and the
// result are normal, otherwise a float64 multiply (zero, subnormals,
// underflow).  -1022 <= k <= 1023.
__device__ __forceinline__ double scale_pow2(double v, int k) {
  const long long b = __double_as_longlong(v);
  const int ex = int((b >> 52) & 0x7ff);
  if (ex == 0 || ex + k <= 0 || ex + k >= 0x7ff) return v * __hiloint2double((k + 1023) << 20, 0);
  return __longlong_as_double(b + ((long long)k << 52));
}

// e^x for x <= 0 (any x: NaN passes through; x < -745.2 gives 0).
__device__ __forceinline__ double exp_nonpos(double x) {
  constexpr double INV_STEP = 0x1.71547652b82fep+6;  // 64 / ln2
  constexpr double STEP_HI = 0x1.62e42fee00000p-7;   // ln2 / 64, 32 significant bits
  constexpr double STEP_LO = 0x1.a39ef35793c76p-39;  // ln2 / 64 - STEP_HI
  constexpr double SHIFTER = 0x1.8p52;
  if (!(x >= -745.2)) return (x != x) ? x : 0.0;
  const double t = fma(x, INV_STEP, SHIFTER);  // n in the low bits of t
  const int n = __double2loint(t);
  const double nd = t - SHIFTER;
  double r = fma(-nd, STEP_HI, x);
  r = fma(-nd, STEP_LO, r);
  // Taylor coefficients 1/k!, k = 5 .. 0
  double q = fma(r, 1.0 / 120.0, 1.0 / 24.0);
  q = fma(r, q, 1.0 / 6.0);
  q = fma(r, q, 0.5);
  q = fma(r, q, 1.0);
  q = fma(r, q, 1.0);
  const int j = n & 63, m = n >> 6;  // n = 64 m + j (arithmetic shift: floor)
  const double v = __ldg(&kExp2Frac64[j]) * q;  // in [0.99, 2.02)
  if (m >= -1020) return __longlong_as_double(__double_as_longlong(v) + ((long long)m << 52));
  return (v * __hiloint2double((m + 60 + 1023) << 20, 0)) * 0x1p-60;  // subnormal range: one rounding
}

}  // namespace dev
}  // namespace ctq
