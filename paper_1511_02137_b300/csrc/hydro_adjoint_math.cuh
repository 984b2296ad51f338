// Reverse-mode derivatives of the step arithmetic (hand-written adjoints).
//
// Each function takes the same inputs as its forward counterpart in
// hydro_math.cuh plus the adjoint of the output, and returns the adjoints of
// the inputs.  Floors are treated as constants where they act (the derivative
// of a clamped quantity is zero), kinks (|v_d| at 0) take the symmetric
// subgradient 0.  The templates run in FP64 (MathD) for the FP64 path and in
// FP32 (MathF) for the mixed path, whose forward fluxes are FP32.
#pragma once

#include "hydro_math.cuh"

namespace hydro {

// Adjoint of the closed-form recovery (E, M) -> (e, v^x, v^y, v^z) for p = e/3
// given its intermediate values: with m = |M|/E, v(m) = 3m/(2 + s),
// s = sqrt(4 - 3m^2),
//   e = E - |M| v(m),  v^i = v(m) M^i/|M|,
//   de/dE = 1 + m^2 v',  de/d|M| = -(v + m v'),
//   dv^i/dE = -m v'/E n^i,  dv^i/dM^j = (v'/E) n^i n^j + (v/|M|)(delta_ij - n^i n^j),
// v' = [3(2 + s) + 9 m^2/s]/(2 + s)^2, n = M/|M|, r = 1/(2 + s), vs = v/|M|.
// Accumulates into Ebar, Mbar.
template <class M>
__device__ __forceinline__ void c2p_vjp_core(typename M::T m, typename M::T s, typename M::T r, typename M::T v,
                                             typename M::T vs, typename M::T invE, typename M::T nx,
                                             typename M::T ny, typename M::T nz, bool capped, bool floored,
                                             typename M::T ebar, typename M::T vbx, typename M::T vby,
                                             typename M::T vbz, typename M::T& Ebar, typename M::T& Mbx,
                                             typename M::T& Mby, typename M::T& Mbz) {
  using P = typename M::T;
  const P vn = vbx * nx + vby * ny + vbz * nz;   // vbar . n
  P dEe, coef;
  if (!capped) {
    const P vp = (P(3) * (P(2) + s) + P(9) * m * m * M::rcp(s)) * r * r;   // dv/dm
    dEe = ebar * (P(1) + m * m * vp) - vp * m * invE * vn;
    coef = -ebar * (v + m * vp) + (vp * invE - vs) * vn;
  } else {
    dEe = ebar * (P(1) - m * v);
    coef = -vs * vn;
  }
  if (!floored) Ebar += dEe;
  Mbx += vs * vbx + nx * coef;
  Mby += vs * vby + ny * coef;
  Mbz += vs * vbz + nz * coef;
}

// FP64 recovery adjoint (the recovery of cons_to_prim<MathD>).
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
  c2p_vjp_core<MathD>(m, s, r, v, vs, invE, nx, ny, nz, m_capped, e_floored, ebar, vbx, vby, vbz, Ebar, Mbx, Mby,
                      Mbz);
}

// Intermediate values of the closed-form recovery, kept for its adjoint.
template <class P>
struct C2PTape {
  P m, s, r, v, vs, invE, nx, ny, nz;
  bool capped, floored;
};

// FP64 recovery (the arithmetic of cons_to_prim<MathD>) keeping its intermediates.
__device__ __forceinline__ void cons_to_prim_tape(double E, double Mx, double My, double Mz, double e_floor,
                                                  C2PTape<double>& t, double& e, double& vx, double& vy,
                                                  double& vz) {
  // |M| and 1/|M| from one Newton-Raphson reciprocal square root where |M|^2 is a
  // normal double (always, for |M| above 1.5e-154), IEEE operations below that
  const double M2 = Mx * Mx + My * My + Mz * Mz;
  double Mabs = 0.0, im = 0.0;
  if (M2 >= 2.2250738585072014e-308) {
    sqrt_rsqrt_nr(M2, Mabs, im);
  } else if (M2 > 0.0) {
    Mabs = sqrt(M2);
    im = 1.0 / Mabs;
  }
  double Ee = E;
  t.floored = !(Ee >= e_floor);
  if (t.floored) Ee = e_floor;
  t.invE = rcp_nr(Ee);
  double m = Mabs * t.invE;
  double m_over_M = t.invE;
  t.capped = !(m <= MathD::m_max);
  if (t.capped) {
    m = MathD::m_max;
    m_over_M = m / Mabs;
  }
  t.m = m;
  double ys;
  sqrt_rsqrt_nr(4.0 - 3.0 * m * m, t.s, ys);   // the argument lies in [1, 4]
  t.r = rcp_nr(2.0 + t.s);
  t.v = 3.0 * m * t.r;
  e = Ee * (1.0 - m * t.v);
  t.vs = 3.0 * m_over_M * t.r;
  vx = Mx * t.vs;
  vy = My * t.vs;
  vz = Mz * t.vs;
  t.nx = Mx * im;   // (0 for M = 0)
  t.ny = My * im;
  t.nz = Mz * im;
}

// Mixed recovery from the floored E and om (the arithmetic of cons_to_prim_om)
// keeping its intermediates.
__device__ __forceinline__ void cons_to_prim_om_tape(float Ef_signed, float mx, float my, float mz, float om_in,
                                                     C2PTape<float>& t, float& e, float& vx, float& vy,
                                                     float& vz) {
  t.floored = Ef_signed < 0.0f;
  const float Ef = fabsf(Ef_signed);
  const float Mabs = sqrt_approx(mx * mx + my * my + mz * mz);
  t.invE = rcp_approx(Ef);
  float om = om_in;
  const float om_min = (float)(1.0 - MathD::m_max);
  float m_over_M = t.invE;
  t.capped = !(om >= om_min);
  if (t.capped) {
    om = om_min;
    m_over_M = (1.0f - om) / Mabs;
  }
  t.s = sqrt_approx(1.0f + 3.0f * om * (2.0f - om));
  t.r = rcp_approx(2.0f + t.s);
  const float omv = 3.0f * om * (1.0f + (2.0f - om) * rcp_approx(t.s + 1.0f)) * t.r;   // 1 - v
  t.v = 1.0f - omv;
  t.m = 1.0f - om;
  e = Ef * (omv + t.v * om);
  t.vs = 3.0f * m_over_M * t.r;
  vx = mx * t.vs;
  vy = my * t.vs;
  vz = mz * t.vs;
  t.nx = t.ny = t.nz = 0.0f;
  if (Mabs > 0.0f) {
    const float im = rcp_approx(Mabs);
    t.nx = mx * im;
    t.ny = my * im;
    t.nz = mz * im;
  }
}

// Gradient of the spectral radius rho(v_d, v^2) of hydro_math.cuh.
template <class M>
__device__ __forceinline__ void spectral_radius_grad(typename M::T vd, typename M::T v2, typename M::T& d_vd,
                                                     typename M::T& d_v2) {
  using P = typename M::T;
  const P third = P(1) / P(3);
  const P vd2 = vd * vd;
  const P A = P(1) - v2, B = P(1) - v2 * third - P(2) * third * vd2;
  const P disc = A * B;
  const P D = P(1) - v2 * third;
  const P sg = (vd > P(0)) ? P(1) : ((vd < P(0)) ? P(-1) : P(0));
  P dN_vd = P(2) * third * sg, dN_v2 = P(0), s3 = P(0);
  if (disc > P(0)) {
    s3 = M::sqrt(disc * third);
    const P k = M::rcp(P(6) * s3);
    dN_vd += (P(-4) * third * vd * A) * k;
    dN_v2 += (-B - A * third) * k;
  }
  const P iD = M::rcp(D);
  const P rho = (fabs(vd) * P(2) * third + s3) * iD;
  d_vd = dN_vd * iD;
  d_v2 = (dN_v2 + rho * third) * iD;
}

// WENO7 reconstruction (as weno7_terms: folded candidates, chained indicator
// terms) and the adjoint of its 7 inputs for an output adjoint gbar.  The
// forward keeps the indicator terms a_k, b_k, c_k, the candidate terms z_k and
// the shifted indicators s_k = eps_s + beta'_k; the weights run in product form
// in FP64 (one division) and with one reciprocal per weight in FP32.  Returns
// the reconstructed value.
template <class P>
__device__ __forceinline__ P weno7_vjp(const P f[7], P eps_s, P gbar, P fb[7]) {
  const P kA = P(kW7A), kB = P(kW7B);
  // ---- forward
  P d1[6], d2[5], c[4];
  for (int j = 0; j < 6; ++j) d1[j] = f[j + 1] - f[j];
  for (int j = 0; j < 5; ++j) d2[j] = d1[j + 1] - d1[j];
  for (int j = 0; j < 4; ++j) c[j] = d2[j + 1] - d2[j];
  const P e0 = c[1] - c[0], e1 = c[2] - c[1], e2 = c[3] - c[2];
  P a[4];
  a[0] = P(2 * kW7A) * d1[0] + P(-7 * kW7A) * d1[1] + P(11 * kW7A) * d1[2];
  a[1] = P(2 * kW7A) * e0 + a[0];
  a[2] = P(-kW7A) * e1 + a[1];
  a[3] = P(2 * kW7A) * e2 + a[2];
  const P b12 = kB * d2[2];
  const P b0 = P(-kW7B) * e0 + b12;
  const P b3 = P(-kW7B) * e2 + b12;
  P z[4];
  z[0] = P(1.0 / (12 * kW7A)) * a[0] + P(1.0 / (12 * kW7B)) * b0;
  z[1] = P(1.0 / kW7A) * a[1] + d2[2];
  z[2] = P(1.5 / kW7A) * a[2] + P(1.5) * d2[2];
  z[3] = P(1.0 / (3 * kW7A)) * a[3] + P(1.0 / (3 * kW7B)) * b3;
  const P m12 = b12 * b12 + eps_s;
  P s[4];
  s[0] = a[0] * a[0] + (b0 * b0 + (c[0] * c[0] + eps_s));
  s[1] = a[1] * a[1] + (c[1] * c[1] + m12);
  s[2] = a[2] * a[2] + (c[2] * c[2] + m12);
  s[3] = a[3] * a[3] + (b3 * b3 + (c[3] * c[3] + eps_s));
  const P dk[4] = {P(1), P(12), P(18), P(4)};
  P t[4], q[4], rs[4], p01 = P(0), p23 = P(0);
  if constexpr (sizeof(P) == 8) {
    for (int k = 0; k < 4; ++k) q[k] = s[k] * s[k];
    p01 = q[0] * q[1];
    p23 = q[2] * q[3];
    t[0] = q[1] * p23;
    t[1] = q[0] * p23;
    t[2] = q[3] * p01;
    t[3] = q[2] * p01;
  } else {
    for (int k = 0; k < 4; ++k) {
      rs[k] = rcp_approx(s[k]);
      t[k] = rs[k] * rs[k];
    }
  }
  const P num = t[0] * z[0] + t[1] * z[1] + t[2] * z[2] + t[3] * z[3];
  const P den = t[0] + P(12) * t[1] + P(18) * t[2] + P(4) * t[3];
  P rden;
  if constexpr (sizeof(P) == 8) rden = rcp_nr(den);
  else rden = rcp_approx(den);
  const P corr = num * rden;
  // ---- reverse: weights
  const P numb = gbar * rden;
  const P denb = -numb * corr;
  P tb[4], zb[4], sb[4];
  for (int k = 0; k < 4; ++k) {
    tb[k] = numb * z[k] + denb * dk[k];
    zb[k] = numb * t[k];
  }
  if constexpr (sizeof(P) == 8) {
    P qb[4];
    const P p23b = tb[0] * q[1] + tb[1] * q[0];
    const P p01b = tb[2] * q[3] + tb[3] * q[2];
    qb[0] = tb[1] * p23 + p01b * q[1];
    qb[1] = tb[0] * p23 + p01b * q[0];
    qb[2] = tb[3] * p01 + p23b * q[3];
    qb[3] = tb[2] * p01 + p23b * q[2];
    for (int k = 0; k < 4; ++k) sb[k] = P(2) * s[k] * qb[k];
  } else {
    // t = s^-2: dt/ds = -2 t / s
    for (int k = 0; k < 4; ++k) sb[k] = P(-2) * tb[k] * t[k] * rs[k];
  }
  // ---- reverse: indicators and candidate terms
  P ab[4], cb[4];
  for (int k = 0; k < 4; ++k) {
    ab[k] = P(2) * a[k] * sb[k];
    cb[k] = P(2) * c[k] * sb[k];
  }
  P b0b = P(2) * b0 * sb[0], b12b = P(2) * b12 * (sb[1] + sb[2]), b3b = P(2) * b3 * sb[3];
  P d22b = zb[1] + P(1.5) * zb[2];
  ab[0] += P(1.0 / (12 * kW7A)) * zb[0];
  b0b += P(1.0 / (12 * kW7B)) * zb[0];
  ab[1] += P(1.0 / kW7A) * zb[1];
  ab[2] += P(1.5 / kW7A) * zb[2];
  ab[3] += P(1.0 / (3 * kW7A)) * zb[3];
  b3b += P(1.0 / (3 * kW7B)) * zb[3];
  // b0 = b12 - kB e0, b3 = b12 - kB e2, b12 = kB d2[2]
  b12b += b0b + b3b;
  P e0b = -kB * b0b, e2b = -kB * b3b, e1b = P(0);
  d22b += kB * b12b;
  // a3 = a2 + 2 kA e2, a2 = a1 - kA e1, a1 = a0 + 2 kA e0
  ab[2] += ab[3];
  e2b += P(2) * kA * ab[3];
  ab[1] += ab[2];
  e1b -= kA * ab[2];
  ab[0] += ab[1];
  e0b += P(2) * kA * ab[1];
  // e_k = c[k+1] - c[k]
  cb[0] -= e0b;
  cb[1] += e0b - e1b;
  cb[2] += e1b - e2b;
  cb[3] += e2b;
  // c[k] = d2[k+1] - d2[k]
  P d2b[5];
  d2b[0] = -cb[0];
  d2b[1] = cb[0] - cb[1];
  d2b[2] = cb[1] - cb[2] + d22b;
  d2b[3] = cb[2] - cb[3];
  d2b[4] = cb[3];
  // d2[j] = d1[j+1] - d1[j], and a0 from d1[0..2]
  P d1b[6];
  d1b[0] = P(2 * kW7A) * ab[0] - d2b[0];
  d1b[1] = P(-7 * kW7A) * ab[0] + d2b[0] - d2b[1];
  d1b[2] = P(11 * kW7A) * ab[0] + d2b[1] - d2b[2];
  d1b[3] = d2b[2] - d2b[3];
  d1b[4] = d2b[3] - d2b[4];
  d1b[5] = d2b[4];
  // d1[j] = f[j+1] - f[j]; the reconstruction is f[3] + corr
  fb[0] = -d1b[0];
  for (int j = 1; j < 6; ++j) fb[j] = d1b[j - 1] - d1b[j];
  fb[6] = d1b[5];
  fb[3] += gbar;
  return f[3] + corr;
}

}  // namespace hydro

namespace hydro {

// FP32 pair form of weno7_vjp: the left-biased and the mirrored reconstruction
// of one interface (same operation sequence) in the two lanes of the packed
// FP32x2 instructions, as the forward's weno7_pair.  fb receives the adjoints
// of the 7 inputs of each lane.
__device__ __forceinline__ void weno7_vjp_pair(const float2 f[7], float eps_s, float2 gbar, float2 fb[7]) {
  const float kA = (float)kW7A, kB = (float)kW7B;
  // ---- forward
  float2 d1[6], d2[5], c[4];
#pragma unroll
  for (int j = 0; j < 6; ++j) d1[j] = sub2(f[j + 1], f[j]);
#pragma unroll
  for (int j = 0; j < 5; ++j) d2[j] = sub2(d1[j + 1], d1[j]);
#pragma unroll
  for (int j = 0; j < 4; ++j) c[j] = sub2(d2[j + 1], d2[j]);
  const float2 e0 = sub2(c[1], c[0]), e1 = sub2(c[2], c[1]), e2 = sub2(c[3], c[2]);
  float2 a[4];
  a[0] = fma2(bc2(2 * kA), d1[0], fma2(bc2(-7 * kA), d1[1], mul2(bc2(11 * kA), d1[2])));
  a[1] = fma2(bc2(2 * kA), e0, a[0]);
  a[2] = fma2(bc2(-kA), e1, a[1]);
  a[3] = fma2(bc2(2 * kA), e2, a[2]);
  const float2 b12 = mul2(bc2(kB), d2[2]);
  const float2 b0 = fma2(bc2(-kB), e0, b12);
  const float2 b3 = fma2(bc2(-kB), e2, b12);
  float2 z[4];
  z[0] = fma2(bc2((float)(1.0 / (12 * kW7A))), a[0], mul2(bc2((float)(1.0 / (12 * kW7B))), b0));
  z[1] = fma2(bc2((float)(1.0 / kW7A)), a[1], d2[2]);
  z[2] = fma2(bc2((float)(1.5 / kW7A)), a[2], mul2(bc2(1.5f), d2[2]));
  z[3] = fma2(bc2((float)(1.0 / (3 * kW7A))), a[3], mul2(bc2((float)(1.0 / (3 * kW7B))), b3));
  const float2 e = bc2(eps_s);
  const float2 m12 = fma2(b12, b12, e);
  float2 s[4];
  s[0] = fma2(a[0], a[0], fma2(b0, b0, fma2(c[0], c[0], e)));
  s[1] = fma2(a[1], a[1], fma2(c[1], c[1], m12));
  s[2] = fma2(a[2], a[2], fma2(c[2], c[2], m12));
  s[3] = fma2(a[3], a[3], fma2(b3, b3, fma2(c[3], c[3], e)));
  float2 rs[4], t[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    rs[k] = rcp2(s[k]);
    t[k] = mul2(rs[k], rs[k]);
  }
  const float2 num = fma2(t[0], z[0], fma2(t[1], z[1], fma2(t[2], z[2], mul2(t[3], z[3]))));
  const float2 den = fma2(bc2(12.0f), t[1], fma2(bc2(18.0f), t[2], fma2(bc2(4.0f), t[3], t[0])));
  const float2 rden = rcp2(den);
  const float2 corr = mul2(num, rden);
  // ---- reverse: weights.  numb = gbar/den, tb_k = numb z_k - numb corr d_k,
  // zb_k = numb t_k; t = s^-2, so 2 sb_k = -4 tb_k t_k/s_k (kept doubled: every
  // use below is 2 x value x sb)
  const float2 numb = mul2(gbar, rden);
  const float2 numb4 = mul2(bc2(-4.0f), numb);
  const float2 nc4 = mul2(bc2(4.0f), mul2(numb, corr));
  const float dk[4] = {1.0f, 12.0f, 18.0f, 4.0f};
  float2 zb[4], sb2[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    zb[k] = mul2(numb, t[k]);
    const float2 tb4 = fma2(bc2(dk[k]), nc4, mul2(numb4, z[k]));   // -4 tb_k
    sb2[k] = mul2(tb4, mul2(t[k], rs[k]));
  }
  // ---- reverse: indicators and candidate terms
  float2 ab[4], cb[4];
  ab[0] = fma2(bc2((float)(1.0 / (12 * kW7A))), zb[0], mul2(a[0], sb2[0]));
  ab[1] = fma2(bc2((float)(1.0 / kW7A)), zb[1], mul2(a[1], sb2[1]));
  ab[2] = fma2(bc2((float)(1.5 / kW7A)), zb[2], mul2(a[2], sb2[2]));
  ab[3] = fma2(bc2((float)(1.0 / (3 * kW7A))), zb[3], mul2(a[3], sb2[3]));
#pragma unroll
  for (int k = 0; k < 4; ++k) cb[k] = mul2(c[k], sb2[k]);
  const float2 b0b = fma2(bc2((float)(1.0 / (12 * kW7B))), zb[0], mul2(b0, sb2[0]));
  const float2 b3b = fma2(bc2((float)(1.0 / (3 * kW7B))), zb[3], mul2(b3, sb2[3]));
  const float2 b12b = fma2(b12, add2(sb2[1], sb2[2]), add2(b0b, b3b));
  const float2 d22b = fma2(bc2(kB), b12b, fma2(bc2(1.5f), zb[2], zb[1]));
  // a3 = a2 + 2 kA e2, a2 = a1 - kA e1, a1 = a0 + 2 kA e0; b0 = b12 - kB e0, b3 = b12 - kB e2
  const float2 e2b = fma2(bc2(2 * kA), ab[3], mul2(bc2(-kB), b3b));
  ab[2] = add2(ab[2], ab[3]);
  const float2 e1b = mul2(bc2(-kA), ab[2]);
  ab[1] = add2(ab[1], ab[2]);
  const float2 e0b = fma2(bc2(2 * kA), ab[1], mul2(bc2(-kB), b0b));
  ab[0] = add2(ab[0], ab[1]);
  // e_k = c[k+1] - c[k]
  cb[0] = sub2(cb[0], e0b);
  cb[1] = add2(cb[1], sub2(e0b, e1b));
  cb[2] = add2(cb[2], sub2(e1b, e2b));
  cb[3] = add2(cb[3], e2b);
  // c[k] = d2[k+1] - d2[k]  (d2b[0] = -cb[0], d2b[4] = cb[3])
  const float2 d2b1 = sub2(cb[0], cb[1]);
  const float2 d2b2 = add2(sub2(cb[1], cb[2]), d22b);
  const float2 d2b3 = sub2(cb[2], cb[3]);
  // d2[j] = d1[j+1] - d1[j], and a0 from d1[0..2]
  float2 d1b[6];
  d1b[0] = fma2(bc2(2 * kA), ab[0], cb[0]);
  d1b[1] = fma2(bc2(-7 * kA), ab[0], sub2(mul2(bc2(-1.0f), cb[0]), d2b1));
  d1b[2] = fma2(bc2(11 * kA), ab[0], sub2(d2b1, d2b2));
  d1b[3] = sub2(d2b2, d2b3);
  d1b[4] = sub2(d2b3, cb[3]);
  d1b[5] = cb[3];
  // d1[j] = f[j+1] - f[j]; the reconstruction is f[3] + corr
  fb[0] = mul2(bc2(-1.0f), d1b[0]);
#pragma unroll
  for (int j = 1; j < 6; ++j) fb[j] = sub2(d1b[j - 1], d1b[j]);
  fb[6] = d1b[5];
  fb[3] = add2(fb[3], gbar);
}

}  // namespace hydro
