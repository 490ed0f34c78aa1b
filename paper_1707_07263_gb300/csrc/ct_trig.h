// ct_trig.h -- cos and sin of 2 pi m / R in double precision at compile time,
// for the inner twiddles of the compile-time mixed-radix schedules
// (mixed_ct.cu).  Plain C++17 (constexpr), so the host test suite checks the
// values against the host math library with g++.
#pragma once

namespace gbfft {

// (Taylor series on |x| <= pi/4 after reduction by the octant symmetries of
// the unit circle; double precision, rounded once to FP32 where used)
constexpr double kPiD = 3.14159265358979323846264338327950288;

constexpr double ct_sin_poly(double x) {   // |x| <= pi/4
  double term = x, sum = x;
  for (int k = 1; k < 12; ++k) {
    term *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
    sum += term;
  }
  return sum;
}
constexpr double ct_cos_poly(double x) {   // |x| <= pi/4
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 12; ++k) {
    term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
    sum += term;
  }
  return sum;
}
// cos and sin of 2 pi m / R: the angle in eighths of a turn, e = 8m / R,
// splits into an octant o = floor(e) and a remainder; each octant maps to a
// first-octant angle by an exact rotation or reflection.
constexpr void ct_cossin(int m, int R, double& c, double& s) {
  m %= R;
  if (m < 0) m += R;
  const int o = (8 * m) / R;                          // octant 0..7
  const double frac = (double)(8 * m - o * R) / R;    // in [0, 1)
  double t = frac * kPiD / 4.0;                        // angle within the octant
  double cc = 0, ss = 0;
  // odd octants measure the angle from the next multiple of pi/4 downwards
  if (o & 1) t = kPiD / 4.0 - t;
  const double ct = ct_cos_poly(t), st = ct_sin_poly(t);
  switch (o) {
    case 0: cc = ct; ss = st; break;     // [0, pi/4)
    case 1: cc = st; ss = ct; break;     // [pi/4, pi/2): pi/2 - t
    case 2: cc = -st; ss = ct; break;    // [pi/2, 3pi/4): pi/2 + t
    case 3: cc = -ct; ss = st; break;    // [3pi/4, pi): pi - t
    case 4: cc = -ct; ss = -st; break;   // [pi, 5pi/4): pi + t
    case 5: cc = -st; ss = -ct; break;   // [5pi/4, 3pi/2): 3pi/2 - t
    case 6: cc = st; ss = -ct; break;    // [3pi/2, 7pi/4): 3pi/2 + t
    default: cc = ct; ss = -st; break;   // [7pi/4, 2pi): 2pi - t
  }
  c = cc;
  s = ss;
}
constexpr double ct_cos(int m, int R) {
  double c = 0, s = 0;
  ct_cossin(m, R, c, s);
  return c;
}
constexpr double ct_sin(int m, int R) {
  double c = 0, s = 0;
  ct_cossin(m, R, c, s);
  return s;
}

}  // namespace gbfft
