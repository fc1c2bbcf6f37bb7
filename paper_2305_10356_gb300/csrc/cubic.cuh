// The exact line search's cubic (Sec. 3.2): its real roots and the step chosen among them.
// Shared by the iteration and by the unrolled-gradient engine.
#pragma once
#include <cuda_runtime.h>

namespace ofsc {

// Real roots of c3 a^3 + c2 a^2 + c1 a + c0; returns the count (0..3).
__device__ inline int real_roots(double c3, double c2, double c1, double c0, double* r) {
  if (c3 == 0.0) {
    if (c2 == 0.0) {
      if (c1 == 0.0) return 0;
      r[0] = -c0 / c1;
      return 1;
    }
    const double disc = c1 * c1 - 4.0 * c2 * c0;
    if (disc < 0.0) return 0;
    const double q = -0.5 * (c1 + copysign(sqrt(disc), c1));
    if (q == 0.0) {
      r[0] = 0.0;
      return 1;
    }
    r[0] = q / c2;
    r[1] = c0 / q;
    return 2;
  }
  // monic form a^3 + A a^2 + B a + C, shift a = t - A/3: t^3 + p t + q
  const double A = c2 / c3, B = c1 / c3, C = c0 / c3;
  const double p = B - A * A / 3.0;
  const double q = 2.0 * A * A * A / 27.0 - A * B / 3.0 + C;
  const double h = -A / 3.0;
  const double D = 0.25 * q * q + p * p * p / 27.0;
  int cnt;
  if (D > 0.0) {
    const double u = cbrt(-0.5 * q - copysign(sqrt(D), q));
    r[0] = (u != 0.0 ? u - p / (3.0 * u) : 0.0) + h;
    cnt = 1;
  } else if (D == 0.0) {
    if (p == 0.0) {
      r[0] = h;
      return 1;
    }
    r[0] = 3.0 * q / p + h;      // simple root
    r[1] = -1.5 * q / p + h;     // double root
    cnt = 2;
  } else {
    const double m = 2.0 * sqrt(-p / 3.0);
    double arg = 1.5 * q / p * sqrt(-3.0 / p);
    arg = fmax(-1.0, fmin(1.0, arg));
    const double th = acos(arg) / 3.0;
    const double two_pi_3 = 2.0943951023931954923;
    for (int i = 0; i < 3; ++i) r[i] = m * cos(th - two_pi_3 * i) + h;
    cnt = 3;
  }
  for (int i = 0; i < cnt; ++i) {  // two Newton steps on the original cubic
    for (int s = 0; s < 2; ++s) {
      const double x = r[i];
      const double f = ((c3 * x + c2) * x + c1) * x + c0;
      const double d = (3.0 * c3 * x + 2.0 * c2) * x + c1;
      if (d != 0.0) {
        const double nx = x - f / d;
        if (isfinite(nx)) r[i] = nx;
      }
    }
  }
  return cnt;
}

// The step: the real root where q(a) = c3 a^4/4 + c2 a^3/3 + c1 a^2/2 + c0 a is smallest
// (for OFM, q is the objective along the line up to a constant factor). An exact double root
// never beats the simple root, so the paper's three cases all reduce to this rule.
__device__ inline double pick_step(double c3, double c2, double c1, double c0, int* bad) {
  if (!(isfinite(c3) && isfinite(c2) && isfinite(c1) && isfinite(c0))) {
    *bad = 1;
    return 0.0;
  }
  double r[3];
  const int n = real_roots(c3, c2, c1, c0, r);
  if (n == 0) return 0.0;
  double best = r[0], bq = 0.0;
  for (int i = 0; i < n; ++i) {
    const double x = r[i];
    const double qv = ((0.25 * c3 * x + c2 / 3.0) * x + 0.5 * c1) * x * x + c0 * x;
    if (i == 0 || qv < bq || (qv == bq && (fabs(x) < fabs(best) || (fabs(x) == fabs(best) && x < best)))) {
      best = x;
      bq = qv;
    }
  }
  return best;
}

}  // namespace ofsc
