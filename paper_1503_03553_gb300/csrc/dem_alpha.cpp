// dem_alpha.cpp -- restitution parameter alpha(epsilon) for the library.
//
// The paper (Sec. 2) writes eta_n = eta_t = alpha(eps) sqrt(m* k_n sqrt(dn))
// and calls alpha a function of the coefficient of restitution without
// giving it.  The library takes alpha as the exact inverse of the
// restitution of its own normal law: with dn = d0 x, t = t0 s the two-body
// normal motion m* dn'' = -k_n dn^{3/2} - eta_n dn' becomes
//     x'' = -x^{3/2} - alpha x^{1/4} x',  x(0) = 0, x'(0) = 1,
// whose rebound speed -x'(s_end) at the return to x = 0 is eps, for every
// impact speed, mass and size.  This file integrates that equation with the
// Dormand-Prince 5(4) pair under local error control and solves
// e(alpha) = eps by the Illinois variant of regula falsi.
#include <cmath>

#include "../../include/dem.h"

namespace {

void rhs(double a, double x, double u, double& fx, double& fu) {
  double xp = x > 0.0 ? x : 0.0;
  fx = u;
  fu = -xp * std::sqrt(xp) - a * std::sqrt(std::sqrt(xp)) * u;
}

// one Dormand-Prince step: 5th-order solution and an error estimate
void dp_step(double a, double h, double x, double u, double& x5, double& u5,
             double& err) {
  static const double c21 = 1.0 / 5.0;
  static const double c31 = 3.0 / 40.0, c32 = 9.0 / 40.0;
  static const double c41 = 44.0 / 45.0, c42 = -56.0 / 15.0, c43 = 32.0 / 9.0;
  static const double c51 = 19372.0 / 6561.0, c52 = -25360.0 / 2187.0,
                      c53 = 64448.0 / 6561.0, c54 = -212.0 / 729.0;
  static const double c61 = 9017.0 / 3168.0, c62 = -355.0 / 33.0,
                      c63 = 46732.0 / 5247.0, c64 = 49.0 / 176.0,
                      c65 = -5103.0 / 18656.0;
  static const double b1 = 35.0 / 384.0, b3 = 500.0 / 1113.0,
                      b4 = 125.0 / 192.0, b5 = -2187.0 / 6784.0,
                      b6 = 11.0 / 84.0;
  static const double e1 = 71.0 / 57600.0, e3 = -71.0 / 16695.0,
                      e4 = 71.0 / 1920.0, e5 = -17253.0 / 339200.0,
                      e6 = 22.0 / 525.0, e7 = -1.0 / 40.0;
  double k1x, k1u, k2x, k2u, k3x, k3u, k4x, k4u, k5x, k5u, k6x, k6u, k7x, k7u;
  rhs(a, x, u, k1x, k1u);
  rhs(a, x + h * c21 * k1x, u + h * c21 * k1u, k2x, k2u);
  rhs(a, x + h * (c31 * k1x + c32 * k2x), u + h * (c31 * k1u + c32 * k2u),
      k3x, k3u);
  rhs(a, x + h * (c41 * k1x + c42 * k2x + c43 * k3x),
      u + h * (c41 * k1u + c42 * k2u + c43 * k3u), k4x, k4u);
  rhs(a, x + h * (c51 * k1x + c52 * k2x + c53 * k3x + c54 * k4x),
      u + h * (c51 * k1u + c52 * k2u + c53 * k3u + c54 * k4u), k5x, k5u);
  rhs(a, x + h * (c61 * k1x + c62 * k2x + c63 * k3x + c64 * k4x + c65 * k5x),
      u + h * (c61 * k1u + c62 * k2u + c63 * k3u + c64 * k4u + c65 * k5u),
      k6x, k6u);
  x5 = x + h * (b1 * k1x + b3 * k3x + b4 * k4x + b5 * k5x + b6 * k6x);
  u5 = u + h * (b1 * k1u + b3 * k3u + b4 * k4u + b5 * k5u + b6 * k6u);
  rhs(a, x5, u5, k7x, k7u);
  double ex = h * (e1 * k1x + e3 * k3x + e4 * k4x + e5 * k5x + e6 * k6x + e7 * k7x);
  double eu = h * (e1 * k1u + e3 * k3u + e4 * k4u + e5 * k5u + e6 * k6u + e7 * k7u);
  err = std::fabs(ex) + std::fabs(eu);
}

double rebound(double a) {
  const double tol = 1e-14;
  double x = 0.0, u = 1.0, s = 0.0, h = 1e-6;
  bool left_zero = false;
  for (int it = 0; it < 10000000 && s < 200.0; ++it) {
    double x5, u5, err;
    dp_step(a, h, x, u, x5, u5, err);
    if (err > tol && h > 1e-12) {
      h *= std::fmax(0.1, 0.9 * std::pow(tol / err, 0.2));
      continue;
    }
    if (left_zero && x5 <= 0.0) {
      // the overlap closes inside this step: regula falsi on the step length
      double lo = 0.0, hi = h, flo = x, fhi = x5;
      int side = 0;
      double xm = x, um = u;
      for (int k = 0; k < 200; ++k) {
        double hm = (lo * fhi - hi * flo) / (fhi - flo);
        if (!(hm > lo && hm < hi)) hm = 0.5 * (lo + hi);
        double e2;
        dp_step(a, hm, x, u, xm, um, e2);
        if (xm > 0.0) {
          lo = hm;
          flo = xm;
          if (side == 1) fhi *= 0.5;
          side = 1;
        } else {
          hi = hm;
          fhi = xm;
          if (side == -1) flo *= 0.5;
          side = -1;
        }
        if (std::fabs(xm) < 1e-17 || hi - lo < 1e-18) break;
      }
      return -um;
    }
    x = x5;
    u = u5;
    s += h;
    if (x > 0.0) left_zero = true;
    double grow = err > 0.0 ? 0.9 * std::pow(tol / err, 0.2) : 5.0;
    h *= std::fmin(5.0, std::fmax(0.2, grow));
    if (h > 1e-2) h = 1e-2;
  }
  return 0.0;  // no rebound: fully damped
}

}  // namespace

extern "C" double dem_restitution_of_alpha(double alpha) {
  if (!(alpha >= 0.0)) return NAN;
  return rebound(alpha);
}

extern "C" double dem_alpha_of_restitution(double e) {
  if (!(e > 0.0) || e > 1.0) return NAN;
  if (e == 1.0) return 0.0;
  double lo = 0.0, hi = 4.0;
  double flo = rebound(lo) - e, fhi = rebound(hi) - e;  // e(alpha) decreases
  if (fhi > 0.0) return NAN;  // below the smallest rebound represented
  int side = 0;
  double mid = lo;
  for (int k = 0; k < 300; ++k) {
    mid = (lo * fhi - hi * flo) / (fhi - flo);
    if (!(mid > lo && mid < hi)) mid = 0.5 * (lo + hi);
    double fm = rebound(mid) - e;
    if (fm > 0.0) {
      lo = mid;
      flo = fm;
      if (side == 1) fhi *= 0.5;
      side = 1;
    } else {
      hi = mid;
      fhi = fm;
      if (side == -1) flo *= 0.5;
      side = -1;
    }
    if (std::fabs(fm) < 1e-14 || hi - lo < 1e-14) break;
  }
  return mid;
}
