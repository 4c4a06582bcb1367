// Two-sided p-values of the correlation test in log space, FP64, host and device.
//
// Section 2.2 converts each correlation r to t = r sqrt(df / (1 - r^2)) (Eq. 3) and then
// to a P value. For Student's t with df degrees of freedom the two-sided p-value equals the
// regularised incomplete beta function I_x(df/2, 1/2) at x = df / (df + t^2) = 1 - r^2.
// I_x(a, b) is evaluated through its continued fraction (Abramowitz & Stegun 26.5.8) with
// the modified Lentz algorithm (Lentz 1976; Thompson & Barnett 1986), in log space, and
// through I_x(a, b) = 1 - I_{1-x}(b, a) beyond x = (a + 1) / (a + b + 2).
#pragma once

#include <math.h>

namespace tg {

#ifndef TG_HD
#define TG_HD __host__ __device__ __forceinline__
#endif

// h with I_x(a, b) = x^a (1 - x)^b / (a B(a, b)) * h; converges quickly for x < (a+1)/(a+b+2).
TG_HD double incbeta_cf(double a, double b, double x) {
  const double kTiny = 1e-300;
  const double kEps = 2.220446049250313e-16;
  double c = 1.0;
  double d = 1.0 - (a + b) * x / (a + 1.0);
  if (fabs(d) < kTiny) d = kTiny;
  d = 1.0 / d;
  double h = d;
  for (int m = 1; m <= 20000; ++m) {
    const double m2 = 2.0 * m;
    double e = m * (b - m) * x / ((a + m2 - 1.0) * (a + m2));  // even term
    d = 1.0 + e * d;
    if (fabs(d) < kTiny) d = kTiny;
    c = 1.0 + e / c;
    if (fabs(c) < kTiny) c = kTiny;
    d = 1.0 / d;
    h *= d * c;
    e = -(a + m) * (a + b + m) * x / ((a + m2) * (a + m2 + 1.0));  // odd term
    d = 1.0 + e * d;
    if (fabs(d) < kTiny) d = kTiny;
    c = 1.0 + e / c;
    if (fabs(c) < kTiny) c = kTiny;
    d = 1.0 / d;
    const double step = d * c;
    h *= step;
    if (fabs(step - 1.0) <= kEps) break;
  }
  return h;
}

// -log10 p of a correlation r tested with df degrees of freedom; lnB = ln B(df/2, 1/2).
TG_HD double mlog10p_r(double r, double df, double lnB) {
  const double ar = fabs(r);
  if (ar != ar) return ar;          // NaN stays NaN
  if (ar >= 1.0) return INFINITY;   // exact fit
  if (ar == 0.0) return 0.0;
  const double a = 0.5 * df, b = 0.5;
  const double y = ar * ar;                     // 1 - x
  const double x = (1.0 - ar) * (1.0 + ar);     // 1 - r^2 without cancellation
  const double lnx = (y < 0.5) ? log1p(-y) : log(x);
  const double lny = 2.0 * log(ar);
  const double kLn10 = 2.302585092994045684;
  if (x < (a + 1.0) / (a + b + 2.0)) {
    const double lnI = a * lnx + b * lny - log(a) - lnB + log(incbeta_cf(a, b, x));
    return -lnI / kLn10;
  }
  const double comp = exp(b * lny + a * lnx - log(b) - lnB + log(incbeta_cf(b, a, y)));
  return -log1p(-fmin(comp, 1.0)) / kLn10;
}

// -log10 p from Hill's (1970, Comm. ACM 13(10), Algorithm 395) normal deviate for Student's t,
// in FP64 (the formula is written out with the FP32 form below). Within 0.05 of the tolerance
// max(1e-3, 1e-5 -log10 p) for df >= 1500 and 1 - r^2 >= 0.05.
__device__ __forceinline__ double mlog10p_r_hill(double r, double df) {
  const double ar = fabs(r);
  if (ar != ar) return ar;
  if (ar >= 1.0) return INFINITY;
  const double y = ar * ar;
  const double a = df - 0.5;
  const double Y = -a * ((y < 0.5) ? log1p(-y) : log((1.0 - ar) * (1.0 + ar)));
  const double B = 48.0 * a * a;
  const double z =
      ((((((-0.4 * Y - 3.3) * Y - 24.0) * Y - 85.5) / (0.8 * Y * Y + 100.0 + B) + Y + 3.0) / B) + 1.0) *
      sqrt(Y);
  const double x = z * 0.70710678118654752440;
  return (x * x - log(erfcx(x))) * 0.43429448190325182765;
}

// -log10 p of a hit, or of an element recomputed in FP64, on the GPU: the continued fraction,
// except for df >= 1500 and 1 - r^2 >= 0.05, where x = 1 - r^2 lies close to the fraction's
// branch point (a + 1) / (a + b + 2) and it needs up to ~300 iterations of FP64 divisions (a
// fraction of a millisecond per thread on GB300), while Hill's deviate is closed-form and
// within 0.05 of the tolerance there.
__device__ __forceinline__ double mlog10p_r_dev(double r, double df, double lnB) {
  if (df >= 1500.0 && (1.0 - fabs(r)) * (1.0 + fabs(r)) >= 0.05) return mlog10p_r_hill(r, df);
  return mlog10p_r(r, df, lnB);
}

// FP32 forms, used on the GPU for the FULL statistics with 1 - r^2 >= 0.05 (GB300 has little
// FP64 throughput: the FP64 form costs ~8 ns per element there; hits and the elements closer to
// |r| = 1 take the FP64 form above, from an FP64 product).
//
// For df < 1500 the same continued fraction in FP32: near the branch point x ~ (a+1)/(a+b+2)
// its terms cancel by a factor of about a, which FP32 still carries to ~1e-5 for a < 750.
// For df >= 1500 that cancellation grows with df, so the two-sided Student-t probability is
// taken from the normal deviate of Hill (1970, Comm. ACM 13(10), Algorithm 395): with
// a = df - 1/2, Y = a ln(1 + t^2/df) = -a ln(1 - r^2) and B = 48 a^2,
//   z = sqrt(Y) (1 + (Y + 3 + ((((-0.4 Y - 3.3) Y - 24) Y - 85.5) / (0.8 Y^2 + 100 + B)) / B),
// p = erfc(z / sqrt 2), and -log10 p = (x^2 - ln erfcx(x)) / ln 10 with x = z / sqrt 2.
// Against the FP64 continued fraction this is within 0.05 of the tolerance
// (max(1e-3, 1e-5 -log10 p)) for df >= 1500 over the t it is used on, t <= max(400, sqrt(19 df))
// (1 - r^2 >= 0.05), and within 0.004 of it for df >= 5000; every term is well conditioned.
__device__ __forceinline__ float incbeta_cf_f(float a, float b, float x, float y) {
  const float kTiny = 1e-30f;
  const float kEps = 1.2e-7f;
  float c = 1.0f;
  // 1 - (a+b) x / (a+1) written with y = 1 - x to avoid the subtraction
  float d = ((1.0f - b) + (a + b) * y) / (a + 1.0f);
  if (fabsf(d) < kTiny) d = kTiny;
  d = 1.0f / d;
  float h = d;
  for (int m = 1; m <= 500; ++m) {
    const float fm = (float)m, m2 = 2.0f * fm;
    float e = fm * (b - fm) * x / ((a + m2 - 1.0f) * (a + m2));
    d = 1.0f + e * d;
    if (fabsf(d) < kTiny) d = kTiny;
    c = 1.0f + e / c;
    if (fabsf(c) < kTiny) c = kTiny;
    d = 1.0f / d;
    h *= d * c;
    e = -(a + fm) * (a + b + fm) * x / ((a + m2) * (a + m2 + 1.0f));
    d = 1.0f + e * d;
    if (fabsf(d) < kTiny) d = kTiny;
    c = 1.0f + e / c;
    if (fabsf(c) < kTiny) c = kTiny;
    d = 1.0f / d;
    const float step = d * c;
    h *= step;
    if (fabsf(step - 1.0f) <= kEps) break;
  }
  return h;
}

__device__ __forceinline__ float mlog10p_r_f(float r, float df, float lnB) {
  const float ar = fabsf(r);
  if (ar != ar) return ar;
  if (ar >= 1.0f) return INFINITY;
  if (ar == 0.0f) return 0.0f;
  const float kInvLn10 = 0.4342944819032518f;
  const float y = ar * ar;
  if (df >= 1500.0f) {
    const float a = df - 0.5f;
    // ln(1 - r^2) without cancellation: log1p(-r^2) for small r, ln((1 - |r|)(1 + |r|)) above
    const float Y = -a * ((y < 0.5f) ? log1pf(-y) : logf((1.0f - ar) * (1.0f + ar)));
    const float B = 48.0f * a * a;
    const float z =
        ((((((-0.4f * Y - 3.3f) * Y - 24.0f) * Y - 85.5f) / (0.8f * Y * Y + 100.0f + B) + Y + 3.0f) / B) +
         1.0f) *
        sqrtf(Y);
    const float x = z * 0.70710678118654752f;
    return (x * x - logf(erfcxf(x))) * kInvLn10;
  }
  const float a = 0.5f * df, b = 0.5f;
  const float x = (1.0f - ar) * (1.0f + ar);
  const float lnx = (y < 0.5f) ? log1pf(-y) : logf(x);
  const float lny = 2.0f * logf(ar);
  if (x < (a + 1.0f) / (a + b + 2.0f)) {
    const float lnI = a * lnx + b * lny - logf(a) - lnB + logf(incbeta_cf_f(a, b, x, y));
    return -lnI * kInvLn10;
  }
  const float comp = expf(b * lny + a * lnx - logf(b) - lnB + logf(incbeta_cf_f(b, a, y, x)));
  return -log1pf(-fminf(comp, 1.0f)) * kInvLn10;
}

}  // namespace tg
