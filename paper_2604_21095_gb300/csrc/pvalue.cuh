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

}  // namespace tg
