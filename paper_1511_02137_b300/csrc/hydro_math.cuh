// Device-side physics and reconstruction for the relativistic-hydro step.
//
// Everything here is templated on the arithmetic type so that one source
// serves the FP64, FP32 and mixed paths.  The formulas follow Eq. 1 of
// arXiv:1511.02137 with p = e/3 (Fig. 3 caption), the WENO reconstruction of
// Sec. 1 and the jet law of Eq. 3.
#pragma once

#include <cuda_runtime.h>

namespace hydro {

template <class T> struct Lim;
template <> struct Lim<double> {
  // cap on |M|/E in the primitive recovery (|M| -> E as v -> 1)
  static constexpr double m_max = 1.0 - 1e-12;
};
template <> struct Lim<float> {
  static constexpr float m_max = 1.0f - 1.0f / 1048576.0f;
};

// Closed-form conserved -> primitive recovery for p = e/3.
// With m = |M|/E the EOS gives m = 4v/(3+v^2), so v = 3m/(2 + sqrt(4-3m^2)),
// e = E (1 - m v), p = e/3 and v^i = v M^i/|M|.  E below e_floor is raised to
// e_floor and m is capped below 1; either floor sets hit.  The stored state is
// never modified.
template <class P>
__device__ __forceinline__ void cons_to_prim(P E, P Mx, P My, P Mz, P e_floor, P& e, P& vx, P& vy, P& vz,
                                             int& hit) {
  P M2 = Mx * Mx + My * My + Mz * Mz;
  P Mabs = sqrt(M2);
  P Ee = E;
  if (!(Ee >= e_floor)) {
    Ee = e_floor;
    hit = 1;
  }
  P m = Mabs / Ee;
  if (!(m <= Lim<P>::m_max)) {
    m = Lim<P>::m_max;
    hit = 1;
  }
  P v = P(3) * m / (P(2) + sqrt(P(4) - P(3) * m * m));
  e = Ee * (P(1) - m * v);
  P s = (Mabs > P(0)) ? v / Mabs : P(0);
  vx = Mx * s;
  vy = My * s;
  vz = Mz * s;
}

// Spectral radius of the flux Jacobian along an axis: max |lambda_pm| with
// lambda_pm = [v_d (1-c^2) +- c sqrt((1-v^2)(1 - v_d^2 - (v^2 - v_d^2) c^2))] / (1 - v^2 c^2),
// c^2 = 1/3.  Both terms of the numerator enter with the sign that maximises |lambda|.
template <class P>
__device__ __forceinline__ P spectral_radius(P vd, P v2) {
  const P third = P(1) / P(3);
  P vd2 = vd * vd;
  P disc = (P(1) - v2) * (P(1) - vd2 - (v2 - vd2) * third);
  disc = disc > P(0) ? disc : P(0);
  return (fabs(vd) * (P(2) * third) + sqrt(disc * third)) / (P(1) - v2 * third);
}

// Nonlinear weights of WENO-JS, w_k ~ d_k / (eps + beta_k)^2, returned as the
// weighted candidate average.  Arguments are 12*q_k (candidates in twelfths),
// 720*beta_k and 720*eps, so that sum_k w_k q_k = num / (12 den).
// FP64: one division, using w_k ~ d_k prod_{j != k} (eps + beta_j)^2.
__device__ __forceinline__ double weno7_combine(double q0, double q1, double q2, double q3, double b0, double b1,
                                                double b2, double b3, double eps720) {
  double s0 = eps720 + b0, s1 = eps720 + b1, s2 = eps720 + b2, s3 = eps720 + b3;
  s0 *= s0;
  s1 *= s1;
  s2 *= s2;
  s3 *= s3;
  double p01 = s0 * s1, p23 = s2 * s3;
  double a0 = s1 * p23;              // d0 = 1
  double a1 = 12.0 * (s0 * p23);     // d1 = 12
  double a2 = 18.0 * (s3 * p01);     // d2 = 18
  double a3 = 4.0 * (s2 * p01);      // d3 = 4   (common factor 1/35 cancels)
  double num = a0 * q0 + a1 * q1 + a2 * q2 + a3 * q3;
  double den = 12.0 * (a0 + a1 + a2 + a3);
  return num / den;
}

// FP32: the product form could overflow, so each weight takes a fast reciprocal.
__device__ __forceinline__ float weno7_combine(float q0, float q1, float q2, float q3, float b0, float b1, float b2,
                                               float b3, float eps720) {
  float s0 = eps720 + b0, s1 = eps720 + b1, s2 = eps720 + b2, s3 = eps720 + b3;
  float a0 = __fdividef(1.0f, s0 * s0);
  float a1 = __fdividef(12.0f, s1 * s1);
  float a2 = __fdividef(18.0f, s2 * s2);
  float a3 = __fdividef(4.0f, s3 * s3);
  float num = a0 * q0 + a1 * q1 + a2 * q2 + a3 * q3;
  float den = 12.0f * (a0 + a1 + a2 + a3);
  return __fdividef(num, den);
}

// WENO7 reconstruction at x_{i+1/2} from f0..f6 = f_{i-3..i+3} (finite-difference
// form: the values are cell averages of the function reconstructed).  Candidate
// cubics on the four 4-cell stencils and Jiang-Shu weights with linear weights
// (1, 12, 18, 4)/35.  The Balsara-Shu smoothness indicators
// beta_k = sum_{l=1..3} int_cell (h^l p_k^(l))^2 dx / h are evaluated as the sum
// of squares they equal, 720 beta_k = 20 A_k^2 + 780 B_k^2 + 781 C_k^2, with
// A_k, B_k, C_k integer combinations of the first, second and third
// differences of the stencil values (p_k = a0 + a1 x + a2 x^2 + a3 x^3 about
// the cell centre gives beta = (a1 + a3/4)^2 + 13/3 a2^2 + 781/20 a3^2).  Being
// a sum of squares it stays non-negative in FP32, where the expanded quadratic
// form cancels to negative values in smooth regions.
template <class F>
__device__ __forceinline__ F weno7(F f0, F f1, F f2, F f3, F f4, F f5, F f6, F eps720) {
  const F q0 = F(-3) * f0 + F(13) * f1 - F(23) * f2 + F(25) * f3;
  const F q1 = f1 - F(5) * f2 + F(13) * f3 + F(3) * f4;
  const F q2 = -f2 + F(7) * f3 + F(7) * f4 - f5;
  const F q3 = F(3) * f3 + F(13) * f4 - F(5) * f5 + f6;
  const F d10 = f1 - f0, d11 = f2 - f1, d12 = f3 - f2, d13 = f4 - f3, d14 = f5 - f4, d15 = f6 - f5;
  const F d20 = d11 - d10, d21 = d12 - d11, d22 = d13 - d12, d23 = d14 - d13, d24 = d15 - d14;
  const F c0 = d21 - d20, c1 = d22 - d21, c2 = d23 - d22, c3 = d24 - d23;
  const F bb0 = F(2) * d21 - d20, bb12 = d22, bb3 = F(2) * d23 - d24;
  const F a0 = F(2) * d10 - F(7) * d11 + F(11) * d12;
  const F a1 = -d11 + F(5) * d12 + F(2) * d13;
  const F a2 = F(2) * d12 + F(5) * d13 - d14;
  const F a3 = F(11) * d13 - F(7) * d14 + F(2) * d15;
  const F m12 = F(780) * bb12 * bb12;
  const F b0 = F(20) * a0 * a0 + F(780) * bb0 * bb0 + F(781) * c0 * c0;
  const F b1 = F(20) * a1 * a1 + m12 + F(781) * c1 * c1;
  const F b2 = F(20) * a2 * a2 + m12 + F(781) * c2 * c2;
  const F b3 = F(20) * a3 * a3 + F(780) * bb3 * bb3 + F(781) * c3 * c3;
  return weno7_combine(q0, q1, q2, q3, b0, b1, b2, b3, eps720);
}

// WENO5 weights (linear weights (1, 6, 3)/10); candidates in sixths.
__device__ __forceinline__ double weno5_combine(double q0, double q1, double q2, double b0, double b1, double b2,
                                                double eps) {
  double s0 = eps + b0, s1 = eps + b1, s2 = eps + b2;
  s0 *= s0;
  s1 *= s1;
  s2 *= s2;
  double a0 = s1 * s2;             // d0 = 1
  double a1 = 6.0 * (s0 * s2);     // d1 = 6
  double a2 = 3.0 * (s0 * s1);     // d2 = 3
  return (a0 * q0 + a1 * q1 + a2 * q2) / (6.0 * (a0 + a1 + a2));
}

__device__ __forceinline__ float weno5_combine(float q0, float q1, float q2, float b0, float b1, float b2,
                                               float eps) {
  float s0 = eps + b0, s1 = eps + b1, s2 = eps + b2;
  float a0 = __fdividef(1.0f, s0 * s0);
  float a1 = __fdividef(6.0f, s1 * s1);
  float a2 = __fdividef(3.0f, s2 * s2);
  return __fdividef(a0 * q0 + a1 * q1 + a2 * q2, 6.0f * (a0 + a1 + a2));
}

// WENO5 (Sec. 1, 5th order): quadratic candidates in sixths on {i-2..i},
// {i-1..i+1}, {i..i+2}; Jiang-Shu indicators 13/12 (2nd difference)^2 +
// 1/4 (1st-derivative combination)^2; linear weights (1, 6, 3)/10.
template <class F>
__device__ __forceinline__ F weno5(F f0, F f1, F f2, F f3, F f4, F eps) {
  F q0 = F(2) * f0 - F(7) * f1 + F(11) * f2;
  F q1 = -f1 + F(5) * f2 + F(2) * f3;
  F q2 = F(2) * f2 + F(5) * f3 - f4;
  F d, g;
  d = f0 - F(2) * f1 + f2;
  g = f0 - F(4) * f1 + F(3) * f2;
  F b0 = F(13.0 / 12.0) * d * d + F(0.25) * g * g;
  d = f1 - F(2) * f2 + f3;
  g = f1 - f3;
  F b1 = F(13.0 / 12.0) * d * d + F(0.25) * g * g;
  d = f2 - F(2) * f3 + f4;
  g = F(3) * f2 - F(4) * f3 + f4;
  F b2 = F(13.0 / 12.0) * d * d + F(0.25) * g * g;
  return weno5_combine(q0, q1, q2, b0, b1, b2, eps);
}

// Temperature from e = (pi^2/30) dof T^4 / (hbar c)^3: T = (e t4coef)^(1/4).
__device__ __forceinline__ double temperature(double e, double t4coef) {
  double x = e * t4coef;
  x = x > 0.0 ? x : 0.0;
  return sqrt(sqrt(x));
}

}  // namespace hydro
