// Reverse-mode derivatives of the FP64 step arithmetic (hand-written adjoints).
//
// Each function takes the same inputs as its forward counterpart in
// hydro_math.cuh plus the adjoint of the output, and returns the adjoints of
// the inputs.  Floors are treated as constants where they act (the derivative
// of a clamped quantity is zero), kinks (|v_d| at 0) take the symmetric
// subgradient 0.
#pragma once

#include "hydro_math.cuh"

namespace hydro {

// Adjoint of the closed-form recovery (E, M) -> (e, v^x, v^y, v^z) for p = e/3:
// with m = |M|/E, v(m) = 3m/(2 + s), s = sqrt(4 - 3m^2),
//   e = E - |M| v(m),  v^i = v(m) M^i/|M|,
//   de/dE = 1 + m^2 v',  de/d|M| = -(v + m v'),
//   dv^i/dE = -m v'/E n^i,  dv^i/dM^j = (v'/E) n^i n^j + (v/|M|)(delta_ij - n^i n^j),
// v' = [3(2 + s) + 9 m^2/s]/(2 + s)^2, n = M/|M|.  Accumulates into Ebar, Mbar.
__device__ __forceinline__ void cons_to_prim_vjp(double E, double Mx, double My, double Mz, double e_floor,
                                                 double ebar, double vbx, double vby, double vbz, double& Ebar,
                                                 double& Mbx, double& Mby, double& Mbz) {
  const double Mabs = sqrt(Mx * Mx + My * My + Mz * Mz);
  bool e_floored = false, m_capped = false;
  double Ee = E;
  if (!(Ee >= e_floor)) {
    Ee = e_floor;
    e_floored = true;
  }
  const double invE = 1.0 / Ee;
  double m = Mabs * invE;
  if (!(m <= MathD::m_max)) {
    m = MathD::m_max;
    m_capped = true;
  }
  const double s = sqrt(4.0 - 3.0 * m * m);
  const double r = 1.0 / (2.0 + s);
  const double v = 3.0 * m * r;
  const double vs = m_capped ? v / Mabs : 3.0 * invE * r;   // v/|M|
  double nx = 0.0, ny = 0.0, nz = 0.0;
  if (Mabs > 0.0) {
    const double im = 1.0 / Mabs;
    nx = Mx * im;
    ny = My * im;
    nz = Mz * im;
  }
  const double vn = vbx * nx + vby * ny + vbz * nz;   // vbar . n
  double dEe, coef;
  if (!m_capped) {
    const double vp = (3.0 * (2.0 + s) + 9.0 * m * m / s) * r * r;   // dv/dm
    dEe = ebar * (1.0 + m * m * vp) - vp * m * invE * vn;
    coef = -ebar * (v + m * vp) + (vp * invE - vs) * vn;
  } else {
    dEe = ebar * (1.0 - m * v);
    coef = -vs * vn;
  }
  if (!e_floored) Ebar += dEe;
  Mbx += vs * vbx + nx * coef;
  Mby += vs * vby + ny * coef;
  Mbz += vs * vbz + nz * coef;
}

// Gradient of the spectral radius rho(v_d, v^2) of hydro_math.cuh.
__device__ __forceinline__ void spectral_radius_grad(double vd, double v2, double& d_vd, double& d_v2) {
  const double third = 1.0 / 3.0;
  const double vd2 = vd * vd;
  const double A = 1.0 - v2, B = 1.0 - v2 * third - 2.0 * third * vd2;
  const double disc = A * B;
  const double D = 1.0 - v2 * third;
  const double sg = (vd > 0.0) ? 1.0 : ((vd < 0.0) ? -1.0 : 0.0);
  double dN_vd = 2.0 * third * sg, dN_v2 = 0.0, s3 = 0.0;
  if (disc > 0.0) {
    s3 = sqrt(disc * third);
    const double k = 1.0 / (6.0 * s3);
    dN_vd += (-4.0 * third * vd * A) * k;
    dN_v2 += (-B - A * third) * k;
  }
  const double rho = (fabs(vd) * 2.0 * third + s3) / D;
  d_vd = dN_vd / D;
  d_v2 = (dN_v2 + rho * third) / D;
}

// WENO7 reconstruction (as weno7<double>) and the adjoint of its 7 inputs for an
// output adjoint gbar.  Returns the reconstructed value.
__device__ __forceinline__ double weno7_vjp(const double f[7], double eps_s, double gbar, double fb[7]) {
  const double a = kW7A, b = kW7B;
  const double Q0 = (-3.0 / 12.0) * f[0] + (13.0 / 12.0) * f[1] + (-23.0 / 12.0) * f[2] + (25.0 / 12.0) * f[3];
  const double Q1 = f[1] - 5.0 * f[2] + 13.0 * f[3] + 3.0 * f[4];
  const double Q2 = -1.5 * f[2] + 10.5 * f[3] + 10.5 * f[4] - 1.5 * f[5];
  const double Q3 = f[3] + (13.0 / 3.0) * f[4] + (-5.0 / 3.0) * f[5] + (1.0 / 3.0) * f[6];
  double d1[6], d2[5], c[4];
  for (int j = 0; j < 6; ++j) d1[j] = f[j + 1] - f[j];
  for (int j = 0; j < 5; ++j) d2[j] = d1[j + 1] - d1[j];
  for (int j = 0; j < 4; ++j) c[j] = d2[j + 1] - d2[j];
  const double A0 = 2 * a * d1[0] - 7 * a * d1[1] + 11 * a * d1[2];
  const double A1 = -a * d1[1] + 5 * a * d1[2] + 2 * a * d1[3];
  const double A2 = 2 * a * d1[2] + 5 * a * d1[3] - a * d1[4];
  const double A3 = 11 * a * d1[3] - 7 * a * d1[4] + 2 * a * d1[5];
  const double B0 = 2 * b * d2[1] - b * d2[0];
  const double B12 = b * d2[2];
  const double B3 = 2 * b * d2[3] - b * d2[4];
  const double be[4] = {A0 * A0 + B0 * B0 + c[0] * c[0], A1 * A1 + B12 * B12 + c[1] * c[1],
                        A2 * A2 + B12 * B12 + c[2] * c[2], A3 * A3 + B3 * B3 + c[3] * c[3]};
  double sq[4], s[4];
  for (int k = 0; k < 4; ++k) {
    sq[k] = eps_s + be[k];
    s[k] = sq[k] * sq[k];
  }
  const double p01 = s[0] * s[1], p23 = s[2] * s[3];
  const double t[4] = {s[1] * p23, s[0] * p23, s[3] * p01, s[2] * p01};
  const double Q[4] = {Q0, Q1, Q2, Q3};
  const double dk[4] = {1.0, 12.0, 18.0, 4.0};
  const double num = t[0] * Q0 + t[1] * Q1 + t[2] * Q2 + t[3] * Q3;
  const double den = t[0] + 12.0 * t[1] + 18.0 * t[2] + 4.0 * t[3];
  const double rden = 1.0 / den;
  const double W = num * rden;
  // reverse
  const double numb = gbar * rden;
  const double denb = -numb * W;
  double tb[4], Qb[4];
  for (int k = 0; k < 4; ++k) {
    tb[k] = numb * Q[k] + denb * dk[k];
    Qb[k] = numb * t[k];
  }
  double sb[4] = {0, 0, 0, 0}, p01b = 0.0, p23b = 0.0;
  sb[1] += tb[0] * p23; p23b += tb[0] * s[1];
  sb[0] += tb[1] * p23; p23b += tb[1] * s[0];
  sb[3] += tb[2] * p01; p01b += tb[2] * s[3];
  sb[2] += tb[3] * p01; p01b += tb[3] * s[2];
  sb[0] += p01b * s[1]; sb[1] += p01b * s[0];
  sb[2] += p23b * s[3]; sb[3] += p23b * s[2];
  double beb[4];
  for (int k = 0; k < 4; ++k) beb[k] = sb[k] * 2.0 * sq[k];
  const double A0b = 2 * A0 * beb[0], A1b = 2 * A1 * beb[1], A2b = 2 * A2 * beb[2], A3b = 2 * A3 * beb[3];
  const double B0b = 2 * B0 * beb[0], B12b = 2 * B12 * (beb[1] + beb[2]), B3b = 2 * B3 * beb[3];
  double cb[4];
  for (int k = 0; k < 4; ++k) cb[k] = 2 * c[k] * beb[k];
  double d2b[5], d1b[6];
  d2b[0] = -b * B0b - cb[0];
  d2b[1] = 2 * b * B0b + cb[0] - cb[1];
  d2b[2] = b * B12b + cb[1] - cb[2];
  d2b[3] = 2 * b * B3b + cb[2] - cb[3];
  d2b[4] = -b * B3b + cb[3];
  d1b[0] = 2 * a * A0b;
  d1b[1] = -7 * a * A0b - a * A1b;
  d1b[2] = 11 * a * A0b + 5 * a * A1b + 2 * a * A2b;
  d1b[3] = 2 * a * A1b + 5 * a * A2b + 11 * a * A3b;
  d1b[4] = -a * A2b - 7 * a * A3b;
  d1b[5] = 2 * a * A3b;
  for (int j = 0; j < 5; ++j) {
    d1b[j] -= d2b[j];
    d1b[j + 1] += d2b[j];
  }
  for (int j = 0; j < 7; ++j) fb[j] = 0.0;
  for (int j = 0; j < 6; ++j) {
    fb[j] -= d1b[j];
    fb[j + 1] += d1b[j];
  }
  fb[0] += Qb[0] * (-3.0 / 12.0);
  fb[1] += Qb[0] * (13.0 / 12.0) + Qb[1];
  fb[2] += Qb[0] * (-23.0 / 12.0) - 5.0 * Qb[1] - 1.5 * Qb[2];
  fb[3] += Qb[0] * (25.0 / 12.0) + 13.0 * Qb[1] + 10.5 * Qb[2] + Qb[3];
  fb[4] += 3.0 * Qb[1] + 10.5 * Qb[2] + (13.0 / 3.0) * Qb[3];
  fb[5] += -1.5 * Qb[2] + (-5.0 / 3.0) * Qb[3];
  fb[6] += (1.0 / 3.0) * Qb[3];
  return W;
}

}  // namespace hydro
