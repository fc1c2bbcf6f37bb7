// The exact line search's cubic (Sec. 3.2): its real roots and the step chosen among them.
// Shared by the iteration and by the unrolled-gradient engine.
//
// The floating-point steps that both the one-thread solver (pick_step) and the warp solver
// (pick_step_warp) take live in non-inlined functions, so that the compiler emits each once and
// the two solvers give the same bits whatever it contracts into fused multiply-adds.
#pragma once
#include <cuda_runtime.h>

namespace ofsc {

// The monic cubic a^3 + A a^2 + B a + C shifted by a = t + h, h = -A/3, to t^3 + p t + q, and its
// discriminant D = q^2/4 + p^3/27 (one real root if D > 0, three if D < 0).
struct CubicDepressed {
  double p, q, h, D;
};

static __device__ __noinline__ CubicDepressed cubic_depressed(double c3, double c2, double c1, double c0) {
  const double A = c2 / c3, B = c1 / c3, C = c0 / c3;
  CubicDepressed d;
  d.p = B - A * A / 3.0;
  d.q = 2.0 * A * A * A / 27.0 - A * B / 3.0 + C;
  d.h = -A / 3.0;
  d.D = 0.25 * d.q * d.q + d.p * d.p * d.p / 27.0;
  return d;
}

// Two Newton steps on the cubic from x (a step that is not finite is not taken).
static __device__ __noinline__ double cubic_newton2(double c3, double c2, double c1, double c0, double x0) {
  double r = x0;
  for (int s = 0; s < 2; ++s) {
    const double x = r;
    const double f = ((c3 * x + c2) * x + c1) * x + c0;
    const double d = (3.0 * c3 * x + 2.0 * c2) * x + c1;
    if (d != 0.0) {
      const double nx = x - f / d;
      if (isfinite(nx)) r = nx;
    }
  }
  return r;
}

// Three real roots (D < 0): the radius m and the angle th of the trigonometric form.
static __device__ __noinline__ void cubic_trig_params(const CubicDepressed& d, double* m, double* th) {
  *m = 2.0 * sqrt(-d.p / 3.0);
  double arg = 1.5 * d.q / d.p * sqrt(-3.0 / d.p);
  arg = fmax(-1.0, fmin(1.0, arg));
  *th = acos(arg) / 3.0;
}

// Root i (0, 1 or 2) of the trigonometric form, polished by two Newton steps.
static __device__ __noinline__ double cubic_trig_root(double c3, double c2, double c1, double c0, double m,
                                                      double th, double h, int i) {
  const double two_pi_3 = 2.0943951023931954923;
  return cubic_newton2(c3, c2, c1, c0, m * cos(th - two_pi_3 * i) + h);
}

// q(a) = c3 a^4/4 + c2 a^3/3 + c1 a^2/2 + c0 a, the antiderivative of the cubic.
static __device__ __noinline__ double cubic_q(double c3, double c2, double c1, double c0, double x) {
  return ((0.25 * c3 * x + c2 / 3.0) * x + 0.5 * c1) * x * x + c0 * x;
}

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
  const CubicDepressed d = cubic_depressed(c3, c2, c1, c0);
  const double p = d.p, q = d.q, h = d.h;
  int cnt;
  if (d.D > 0.0) {
    const double u = cbrt(-0.5 * q - copysign(sqrt(d.D), q));
    r[0] = (u != 0.0 ? u - p / (3.0 * u) : 0.0) + h;
    cnt = 1;
  } else if (d.D == 0.0) {
    if (p == 0.0) {
      r[0] = h;
      return 1;
    }
    r[0] = 3.0 * q / p + h;      // simple root
    r[1] = -1.5 * q / p + h;     // double root
    cnt = 2;
  } else {
    double m, th;
    cubic_trig_params(d, &m, &th);
    for (int i = 0; i < 3; ++i) r[i] = cubic_trig_root(c3, c2, c1, c0, m, th, h, i);
    return 3;
  }
  for (int i = 0; i < cnt; ++i) r[i] = cubic_newton2(c3, c2, c1, c0, r[i]);
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
    const double qv = cubic_q(c3, c2, c1, c0, x);
    if (i == 0 || qv < bq || (qv == bq && (fabs(x) < fabs(best) || (fabs(x) == fabs(best) && x < best)))) {
      best = x;
      bq = qv;
    }
  }
  return best;
}

// pick_step for a whole warp (every lane calls it with the same coefficients and receives the
// step). With three real roots, lane i < 3 computes root i and its q(a) through the same
// functions as pick_step, and every lane then chooses among them in pick_step's order: the same
// result, bit for bit, in about 60% of the time of one thread (FP64 latency, not throughput,
// bounds this code on GB300). The other cases run pick_step in every lane.
__device__ inline double pick_step_warp(double c3, double c2, double c1, double c0, int* bad) {
  if (!(isfinite(c3) && isfinite(c2) && isfinite(c1) && isfinite(c0))) {
    *bad = 1;
    return 0.0;
  }
  if (c3 == 0.0) return pick_step(c3, c2, c1, c0, bad);
  const CubicDepressed d = cubic_depressed(c3, c2, c1, c0);
  if (!(d.D < 0.0)) return pick_step(c3, c2, c1, c0, bad);
  const int lane = threadIdx.x & 31;
  double m, th;
  cubic_trig_params(d, &m, &th);
  const double r = cubic_trig_root(c3, c2, c1, c0, m, th, d.h, lane < 3 ? lane : 0);
  const double qr = cubic_q(c3, c2, c1, c0, r);
  double best = 0.0, bq = 0.0;
  for (int j = 0; j < 3; ++j) {
    const double x = __shfl_sync(0xffffffffu, r, j);
    const double qv = __shfl_sync(0xffffffffu, qr, j);
    if (j == 0 || qv < bq || (qv == bq && (fabs(x) < fabs(best) || (fabs(x) == fabs(best) && x < best)))) {
      best = x;
      bq = qv;
    }
  }
  return best;
}

}  // namespace ofsc
