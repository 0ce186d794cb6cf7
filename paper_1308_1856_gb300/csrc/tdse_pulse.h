// Host arithmetic of the laser pulse (arXiv 1308.1856, Sec. 3), shared by the
// single-instance handle and the batch engine.
//
//   shape TDSE_PULSE_SIN2_E: E(t) = E0 sin^2(pi t/T) sin(omega t + cep), Eq. (EField);
//   shape TDSE_PULSE_SIN2_A: A(t) = -(c E0/omega) sin^2(pi t/T) sin(omega t + cep),
//                            E = -(1/c) dA/dt, Eq. (VecSinSinCosE);
//   T = 2 pi ncycles / omega, zero outside [0, T];
//   A(t) = -c int_0^t E (Eq. (VectorStep)) by 5-point Gauss-Legendre on equal
//   panels of [0, T] no wider than 0.25 a.u., constant after T.
#pragma once

#include <algorithm>
#include <cmath>

#include "../../include/tdse.h"

namespace tdse_dev {

constexpr double kLightAU = 137.035999084;   // speed of light, atomic units

struct PulseParams {
  double E0, omega, ncycles, cep;
  int shape;
};

inline double pulse_field(const PulseParams &p, double t) {
  if (p.E0 == 0.0 || p.omega <= 0.0) return 0.0;
  const double T = 2.0 * M_PI * p.ncycles / p.omega;
  if (t < 0.0 || t > T) return 0.0;
  const double env = std::sin(M_PI * t / T);
  if (p.shape == TDSE_PULSE_SIN2_A) {
    const double W = M_PI / T, ph = p.omega * t + p.cep;
    return p.E0 / p.omega * env * (p.omega * env * std::cos(ph) + 2.0 * W * std::cos(W * t) * std::sin(ph));
  }
  return p.E0 * env * env * std::sin(p.omega * t + p.cep);
}

// int_a^b E by 5-point Gauss-Legendre.
inline double pulse_field_integral(const PulseParams &p, double a, double b) {
  static const double node[5] = {-0.9061798459386640, -0.5384693101056831, 0.0, 0.5384693101056831,
                                 0.9061798459386640};
  static const double weight[5] = {0.2369268850561891, 0.4786286704993665, 0.5688888888888889,
                                   0.4786286704993665, 0.2369268850561891};
  const double mid = 0.5 * (a + b), half = 0.5 * (b - a);
  double acc = 0.0;
  for (int k = 0; k < 5; ++k) acc += weight[k] * pulse_field(p, mid + half * node[k]);
  return half * acc;
}

inline double pulse_vecpot(const PulseParams &p, double t) {
  if (p.E0 == 0.0 || p.omega <= 0.0 || t <= 0.0) return 0.0;
  const double T = 2.0 * M_PI * p.ncycles / p.omega;
  const double tt = std::min(t, T);
  const long panels = (long)std::ceil(T / 0.25);
  const double w = T / (double)panels;
  const long full = (long)std::floor(tt / w);
  double acc = 0.0;
  for (long k = 0; k < full && k < panels; ++k) acc += pulse_field_integral(p, (double)k * w, (double)(k + 1) * w);
  if (full < panels && tt > (double)full * w) acc += pulse_field_integral(p, (double)full * w, tt);
  return -kLightAU * acc;
}

}  // namespace tdse_dev
