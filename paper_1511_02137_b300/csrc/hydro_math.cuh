// Device-side physics and reconstruction for the relativistic-hydro step.
//
// The formulas follow Eq. 1 of arXiv:1511.02137 with p = e/3 (Fig. 3
// caption), the WENO reconstruction of Sec. 1 and the jet law of Eq. 3.  They
// are templated on a math policy: MathD is IEEE FP64 (the path held to the
// FP64 oracle), MathF is FP32 with the PTX approximate reciprocal and square
// root (rcp.approx / sqrt.approx, at most 1 ulp and 2^-23 relative error).
#pragma once

#include <cuda_runtime.h>

namespace hydro {

__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ float rsqrt_approx(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// FP64 x^(1/2) and x^(-1/2) together (x > 0, normal): the hardware approximation
// rsqrt.approx.ftz.f64 refined by one third-order Newton-Raphson step for
// y = x^(-1/2), y (1 + e/2 + 3e^2/8) with e = 1 - x y^2, then s = x y.  Measured
// against CUDA's sqrt and IEEE division over 1e6 inputs spanning 60 decades (and
// [1, 4]): at most 2.2e-16 relative error in either (the seed's is 9e-7); half the
// FP64 time of a square root and a division.
__device__ __forceinline__ void sqrt_rsqrt_nr(double x, double& s, double& y) {
  double y0;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y0) : "d"(x));
  const double e = fma(-x, y0 * y0, 1.0);
  y = fma(y0 * e, fma(0.375, e, 0.5), y0);
  s = x * y;
}

// FP64 reciprocal by Newton-Raphson iteration for 1/d (the classical method, e.g.
// P. Markstein, IBM J. Res. Dev. 34 (1990) 111), seeded by the hardware
// approximation rcp.approx.ftz.f64: one third-order step y (1 + e + e^2),
// e = 1 - d y, which takes the seed's ~2^-20 relative error below the rounding
// of the step itself.  Measured against IEEE division over 1e6 divisors spanning
// 80 decades: at most 2.2e-16 relative error (1-2 ulp, not correctly rounded).
// For normal d with a normal reciprocal (every call site: floored energies,
// 2 + s, products of shifted WENO indicators); three FP64 operations where IEEE
// division takes eight.
__device__ __forceinline__ double rcp_nr(double d) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(d));
  const double e = fma(-d, y, 1.0);
  return fma(y, fma(e, e, e), y);
}

// gt_nonneg(a, b) = a > b for a >= 0 or NaN and b >= 0: FP64 compares the bit
// patterns on the integer pipe (non-negative doubles order like them; a NaN with
// the sign bit clear compares greater), FP32 compares the values.
struct MathD {
  using T = double;
  static constexpr double m_max = 1.0 - 1e-12;   // cap on |M|/E (|M| -> E as v -> 1)
  static __device__ __forceinline__ double rcp(double x) { return rcp_nr(x); }
  static __device__ __forceinline__ double sqrt(double x) { return ::sqrt(x); }
  // x^(1/2) and x^(-1/2) for x >= 1
  static __device__ __forceinline__ void sqrt_rsqrt(double x, double& s, double& y) { sqrt_rsqrt_nr(x, s, y); }
  // x^(1/2) for x >= 0 where a result of 1.5e-154 in place of 0 is immaterial:
  // the argument is raised to the smallest normal double
  static __device__ __forceinline__ double sqrt_nonneg(double x) {
    const long long b = __double_as_longlong(x), lo = 0x0010000000000000LL;   // 2^-1022
    double s, y;
    sqrt_rsqrt_nr(__longlong_as_double(b > lo ? b : lo), s, y);
    return s;
  }
  static __device__ __forceinline__ bool gt_nonneg(double a, double b) {
    return __double_as_longlong(a) > __double_as_longlong(b);
  }
};

struct MathF {
  using T = float;
  static constexpr float m_max = 1.0f - 1.0f / 1048576.0f;
  static __device__ __forceinline__ float rcp(float x) { return rcp_approx(x); }
  static __device__ __forceinline__ float sqrt(float x) { return sqrt_approx(x); }
  static __device__ __forceinline__ void sqrt_rsqrt(float x, float& s, float& y) {
    y = rsqrt_approx(x);
    s = x * y;
  }
  static __device__ __forceinline__ float sqrt_nonneg(float x) { return sqrt_approx(x); }
  static __device__ __forceinline__ bool gt_nonneg(float a, float b) { return !(a <= b); }
};

// Closed-form conserved -> primitive recovery for p = e/3.
// With m = |M|/E the EOS gives m = 4v/(3+v^2), so v = 3m/(2 + sqrt(4-3m^2)),
// e = E (1 - m v), p = e/3 and v^i = v M^i/|M| = 3 (m/|M|) M^i / (2 + sqrt(4-3m^2)).
// Everything but the cap test needs m^2 = |M|^2/E^2 only (m v = 3 m^2 r and
// m/|M| = 1/E, r = 1/(2 + sqrt(4 - 3m^2))), so |M| itself, one square root, is
// formed only when the cap acts.  E below e_floor is raised to e_floor and m is
// capped below 1; either floor sets hit.  The stored state is never modified.
template <class M>
__device__ __forceinline__ void cons_to_prim(typename M::T E, typename M::T Mx, typename M::T My,
                                             typename M::T Mz, typename M::T e_floor, typename M::T& e,
                                             typename M::T& vx, typename M::T& vy, typename M::T& vz, int& hit) {
  using P = typename M::T;
  const P M2 = Mx * Mx + My * My + Mz * Mz;
  P Ee = E;
  if (!(Ee >= e_floor)) {
    Ee = e_floor;
    hit = 1;
  }
  const P invE = M::rcp(Ee);
  P m2 = M2 * invE * invE;
  P m_over_M = invE;   // m / |M|, so that v / |M| = 3 r m / |M| stays finite for M = 0
  constexpr P m_max2 = M::m_max * M::m_max;
  if (M::gt_nonneg(m2, m_max2)) {   // m2 >= 0 or NaN (a NaN state takes the cap branch and stays NaN)
    m2 = m_max2;
    m_over_M = M::m_max / M::sqrt(M2);
    hit = 1;
  }
  const P r = M::rcp(P(2) + M::sqrt(P(4) - P(3) * m2));
  e = Ee * (P(1) - P(3) * m2 * r);
  const P vs = P(3) * m_over_M * r;   // v / |M|
  vx = Mx * vs;
  vy = My * vs;
  vz = Mz * vs;
}

// cons_to_prim for the sweeps, also returning the two quantities the spectral
// radius needs: v^2 = 3 r (2 - s) and 1/(1 - v^2/3) = (2 + s)/(2 s), from
// v = 3 m r, r = 1/(2 + s), s^2 = 4 - 3 m^2 (so that v^2 = 9 m^2 r^2 = 3 (2 - s) r
// and 1 - v^2/3 = 2 s r); s and 1/s come from one reciprocal square root.
template <class M>
__device__ __forceinline__ void cons_to_prim_rho(typename M::T E, typename M::T Mx, typename M::T My,
                                                 typename M::T Mz, typename M::T e_floor, typename M::T& e,
                                                 typename M::T& vx, typename M::T& vy, typename M::T& vz,
                                                 typename M::T& v2, typename M::T& rden, int& hit) {
  using P = typename M::T;
  const P M2 = Mx * Mx + My * My + Mz * Mz;
  P Ee = E;
  if (!(Ee >= e_floor)) {
    Ee = e_floor;
    hit = 1;
  }
  const P invE = M::rcp(Ee);
  P m2 = M2 * invE * invE;
  P m_over_M = invE;
  constexpr P m_max2 = M::m_max * M::m_max;
  if (M::gt_nonneg(m2, m_max2)) {
    m2 = m_max2;
    m_over_M = M::m_max / M::sqrt(M2);
    hit = 1;
  }
  P s, ys;
  M::sqrt_rsqrt(P(4) - P(3) * m2, s, ys);   // argument in [1, 4]
  const P twos = P(2) + s;
  const P r = M::rcp(twos);
  e = Ee * (P(1) - P(3) * m2 * r);
  const P vs = P(3) * m_over_M * r;
  vx = Mx * vs;
  vy = My * vs;
  vz = Mz * vs;
  v2 = P(3) * r * (P(2) - s);
  rden = P(0.5) * twos * ys;
}

// Spectral radius from v_d, v^2 and rden = 1/(1 - v^2 c^2) (c^2 = 1/3).
template <class M>
__device__ __forceinline__ typename M::T spectral_radius_r(typename M::T vd, typename M::T v2, typename M::T rden) {
  using P = typename M::T;
  const P third = P(1) / P(3);
  const P vd2 = vd * vd;
  P disc = (P(1) - v2) * (P(1) - vd2 - (v2 - vd2) * third);
  disc = M::gt_nonneg(disc, P(0)) ? disc : P(0);
  return (fabs(vd) * (P(2) * third) + M::sqrt_nonneg(disc * third)) * rden;
}

// Mixed-precision recovery: only the cancelling combination E^2 - |M|^2 (tiny
// as v -> 1) is formed in FP64; everything after it is well conditioned in
// terms of om = 1 - m = (E^2 - |M|^2) / (E (E + |M|)), where E + |M| needs only
// FP32 accuracy, and runs in FP32:
//   4 - 3m^2 = 1 + 3 om (2 - om),  1 - v = 3 om (1 + (2 - om)/(s + 1)) / (2 + s),
//   1 - m v = (1 - v) + v om,  with s = sqrt(4 - 3m^2).
// FP64 <-> FP32 conversions on the integer pipe, from the IEEE 754 binary64 and
// binary32 layouts (B300 runs the hardware conversions at the FP64 rate, 1/64 of
// FP32; the mixed z sweep, whose FP64 pipe also forms the stage combination, and
// the adjoint's elementwise kernels convert with these).  d2f_rn rounds to
// nearest even; results below the FP32 normal range flush to signed zero, above
// it become infinity, NaN stays NaN.  f2d is exact for normal FP32 values and
// zero; FP32 subnormals flush to signed zero.
__device__ __forceinline__ float d2f_rn(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned hb = hi & 0x7fffffffu;
  // biased binary32 exponent and the top 23 fraction bits, then round to nearest
  // even on the 29 dropped bits (a carry lands in the exponent, up to infinity)
  unsigned t = __funnelshift_l(lo, hb - (896u << 20), 3);
  t += ((lo & 0x1fffffffu) + (t & 1u) + 0x0fffffffu) >> 29;
  if (hb - (897u << 20) >= (254u << 20)) {   // outside the binary32 normal range (rare)
    if (hb < (897u << 20)) t = 0u;                                   // flush to zero
    else if (hb > 0x7ff00000u || (hb == 0x7ff00000u && lo != 0u)) t = 0x7fc00000u;   // NaN
    else t = 0x7f800000u;                                            // overflow, infinity
  }
  return __uint_as_float(t | (hi & 0x80000000u));
}

// Finite test of a double on the integer pipe (exponent field not all ones).
__device__ __forceinline__ bool finite_bits(double x) {
  return ((unsigned)__double2hiint(x) & 0x7ff00000u) != 0x7ff00000u;
}
__device__ __forceinline__ bool finite_bits(float x) { return isfinite(x); }

__device__ __forceinline__ double f2d(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned mag = u & 0x7fffffffu;
  // exponent and the top 20 fraction bits move down by 3 and the exponent bias
  // grows by 1023 - 127 = 896; the low 3 fraction bits open the low word
  unsigned hi = ((mag >> 3) + (896u << 20)) | (u & 0x80000000u), lo = u << 29;
  if (mag < 0x00800000u) {   // zero and subnormals: signed zero
    hi = u & 0x80000000u;
    lo = 0u;
  }
  if (mag >= 0x7f800000u) hi += 896u << 20;   // infinity and NaN: exponent 255 + 896 + 896 = 2047
  return __hiloint2double((int)hi, (int)lo);
}

// The FP32 part of the mixed recovery: primitives from the floored E (as FP32,
// negated when the floor acted) and om = 1 - |M|/E (see mixed_shadow).
__device__ __forceinline__ void cons_to_prim_om(float Ef_signed, float mx, float my, float mz, float om_in, float& e,
                                                float& vx, float& vy, float& vz, int& hit) {
  if (Ef_signed < 0.0f) hit = 1;
  const float Ef = fabsf(Ef_signed);
  const float Mabs = sqrt_approx(mx * mx + my * my + mz * mz);
  const float invE = rcp_approx(Ef);
  float om = om_in;
  const float om_min = (float)(1.0 - MathD::m_max);
  float m_over_M = invE;   // m / |M|
  if (!(om >= om_min)) {
    om = om_min;
    m_over_M = (1.0f - om) / Mabs;
    hit = 1;
  }
  const float s = sqrt_approx(1.0f + 3.0f * om * (2.0f - om));
  const float r = rcp_approx(2.0f + s);
  const float omv = 3.0f * om * (1.0f + (2.0f - om) * rcp_approx(s + 1.0f)) * r;   // 1 - v
  const float v = 1.0f - omv;
  e = Ef * (omv + v * om);
  const float vs = 3.0f * m_over_M * r;   // v / |M|
  vx = mx * vs;
  vy = my * vs;
  vz = mz * vs;
}

// !(E >= e_floor) (e_floor > 0) on the integer pipe: non-negative doubles order
// like their bit patterns, negative ones have negative patterns, NaN floors.
__device__ __forceinline__ bool mixed_floored(double E, double e_floor) {
  const long long eb = __double_as_longlong(E);
  const bool nan = !finite_bits(E) && (eb & 0xfffffffffffffLL) != 0;
  return eb < __double_as_longlong(e_floor) || nan;
}

// om = 1 - |M|/E of the mixed recovery: the cancelling E^2 - |M|^2 from the
// floored FP64 energy Ee and the FP64 momentum, the rest from the FP32 roundings.
__device__ __forceinline__ float mixed_om_of(double Ee, double Mx, double My, double Mz, float Eef, float mx,
                                             float my, float mz) {
  const double D = Ee * Ee - (Mx * Mx + My * My + Mz * Mz);
  const float Mabs = sqrt_approx(mx * mx + my * my + mz * mz);
  return d2f_rn(D) * rcp_approx(Eef * (Eef + Mabs));
}

// The FP32 shadow of an FP64 mixed-precision state, six values per cell that
// carry everything the sweeps need from it: the roundings of E, M^x, M^y, M^z
// and R, and om = 1 - |M|/E of the recovery (E^2 - |M|^2 in FP64).  The stored
// E satisfies !(E_s >= e_floor_f) exactly when the FP64 recovery floors E
// (E_s is moved by at most one FP32 ulp, and only for an E within one ulp below
// the floor), so that a sweep reading the shadow takes the FP64 floor decision.
// From a shadow, cons_to_prim_shadow recovers the primitives (the FP64 floor
// decision, om from E^2 - |M|^2 in FP64, the rest in FP32); the sweeps use
// cons_to_prim_shadow_rho, the same closed form with s from a reciprocal
// square root, which also serves the spectral radius.
__device__ __forceinline__ void mixed_shadow(double E, double Mx, double My, double Mz, double R, double e_floor,
                                             float s[6]) {
  const bool floored = mixed_floored(E, e_floor);
  const float ef = d2f_rn(e_floor);
  float Ef = d2f_rn(E);
  const float mx = d2f_rn(Mx), my = d2f_rn(My), mz = d2f_rn(Mz);
  s[5] = mixed_om_of(floored ? e_floor : E, Mx, My, Mz, floored ? ef : Ef, mx, my, mz);
  // E < e_floor rounds to at most ef; equality is the only ambiguous case
  if (floored && Ef >= ef)   // the next float below ef (ef > 0), or a negative one if e_floor rounds to 0
    Ef = ef > 0.0f ? __uint_as_float(__float_as_uint(ef) - 1u) : -1.17549435e-38f;
  s[0] = Ef;
  s[1] = mx;
  s[2] = my;
  s[3] = mz;
  s[4] = d2f_rn(R);
}

// cons_to_prim_om that also returns what the spectral radius needs, v^2 and
// 1/(1 - v^2/3), from the same s: with s^2 = 4 - 3 m^2 = 1 + 3 om (2 - om) and
// r = 1/(2 + s), v^2 = 3 r (2 - s) and 1 - v^2/3 = 2 s r (as cons_to_prim_rho);
// one reciprocal square root gives s and 1/s.
__device__ __forceinline__ void cons_to_prim_om_rho(float Ef_signed, float mx, float my, float mz, float om_in,
                                                    float& e, float& vx, float& vy, float& vz, float& v2,
                                                    float& rden, int& hit) {
  if (Ef_signed < 0.0f) hit = 1;
  const float Ef = fabsf(Ef_signed);
  const float invE = rcp_approx(Ef);
  float om = om_in;
  const float om_min = (float)(1.0 - MathD::m_max);
  float m_over_M = invE;   // m / |M|
  if (!(om >= om_min)) {
    om = om_min;
    m_over_M = (1.0f - om) / sqrt_approx(mx * mx + my * my + mz * mz);
    hit = 1;
  }
  const float s2 = 1.0f + 3.0f * om * (2.0f - om);
  const float ys = rsqrt_approx(s2);
  const float s = s2 * ys;
  const float twos = 2.0f + s;
  const float r = rcp_approx(twos);
  const float omv = 3.0f * om * (1.0f + (2.0f - om) * rcp_approx(s + 1.0f)) * r;   // 1 - v
  const float v = 1.0f - omv;
  e = Ef * (omv + v * om);
  const float vs = 3.0f * m_over_M * r;   // v / |M|
  vx = mx * vs;
  vy = my * vs;
  vz = mz * vs;
  v2 = 3.0f * r * (2.0f - s);
  rden = 0.5f * twos * ys;
}

// The mixed recovery from a shadow (see mixed_shadow); ef = the FP32 rounding of e_floor.
__device__ __forceinline__ void cons_to_prim_shadow(float Es, float mx, float my, float mz, float om, float ef,
                                                    float& e, float& vx, float& vy, float& vz, int& hit) {
  const bool floored = !(Es >= ef);
  cons_to_prim_om(floored ? -ef : Es, mx, my, mz, om, e, vx, vy, vz, hit);
}

// cons_to_prim_shadow with v^2 and 1/(1 - v^2/3) for the spectral radius.
__device__ __forceinline__ void cons_to_prim_shadow_rho(float Es, float mx, float my, float mz, float om, float ef,
                                                        float& e, float& vx, float& vy, float& vz, float& v2,
                                                        float& rden, int& hit) {
  const bool floored = !(Es >= ef);
  cons_to_prim_om_rho(floored ? -ef : Es, mx, my, mz, om, e, vx, vy, vz, v2, rden, hit);
}

// Spectral radius of the flux Jacobian along an axis: max |lambda_pm| with
// lambda_pm = [v_d (1-c^2) +- c sqrt((1-v^2)(1 - v_d^2 - (v^2 - v_d^2) c^2))] / (1 - v^2 c^2),
// c^2 = 1/3.  Both terms of the numerator enter with the sign that maximises |lambda|.
template <class M>
__device__ __forceinline__ typename M::T spectral_radius(typename M::T vd, typename M::T v2) {
  using P = typename M::T;
  const P third = P(1) / P(3);
  const P vd2 = vd * vd;
  P disc = (P(1) - v2) * (P(1) - vd2 - (v2 - vd2) * third);
  disc = M::gt_nonneg(disc, P(0)) ? disc : P(0);   // (against +0 the bit compare also orders negatives)
  return (fabs(vd) * (P(2) * third) + M::sqrt(disc * third)) * M::rcp(P(1) - v2 * third);
}

// Scales of the WENO7 smoothness indicators: 720 beta = 20 A^2 + 780 B^2 + 781 C^2,
// used as beta' = (720/781) beta = (sqrt(20/781) A)^2 + (sqrt(780/781) B)^2 + C^2.
constexpr double kW7EpsScale = 720.0 / 781.0;
constexpr double kW7A = 0.16002560614563885;   // sqrt(20/781)
constexpr double kW7B = 0.999359590072005;     // sqrt(780/781)

// WENO7 reconstruction at x_{i+1/2} from f0..f6 = f_{i-3..i+3} (finite-difference
// form: the values are cell averages of the function reconstructed).
// Candidate cubics q_k on the four 4-cell stencils, linear weights
// (1, 12, 18, 4)/35, Jiang-Shu weights, Balsara-Shu indicators
// beta_k = sum_{l=1..3} int_cell (h^l p_k^(l))^2 dx / h.  With p_k = a0 + a1 x +
// a2 x^2 + a3 x^3 about the cell centre, beta = (a1 + a3/4)^2 + 13/3 a2^2 +
// 781/20 a3^2, i.e. 720 beta_k = 20 A_k^2 + 780 B_k^2 + 781 C_k^2 with A_k, B_k,
// C_k integer combinations of the first (d1), second (d2) and third (c)
// differences of the stencil values:
//   A = (2,-7,11).d1[0..2], (-1,5,2).d1[1..3], (2,5,-1).d1[2..4], (11,-7,2).d1[3..5]
//   B = 2 d2[1] - d2[0], d2[2], d2[2], 2 d2[3] - d2[4];  C_k = c[k].
// The same terms give the candidates: q_k(x_{i+1/2}) - f_i = (A_k + B_k)/12, so
//   reconstruction = f_i + sum_k d_k t_k (A_k + B_k)/12 / sum_k d_k t_k,
// t_k = 1/(eps + beta_k)^2, d = (1, 12, 18, 4).  Neighbouring stencils differ
// by fourth differences e_k = c[k+1] - c[k]:
//   A_1 = A_0 + 2 e_0,  A_2 = A_1 - e_1,  A_3 = A_2 + 2 e_2,
//   B_0 = d2[2] - e_0,  B_3 = d2[2] - e_2.
// The sum of squares stays non-negative in FP32, where the expanded quadratic
// form cancels to negative values in smooth regions.
//
// weno7_terms returns z_k = d_k (A_k + B_k)/12 and s_k = eps_s + beta'_k
// (beta' = 720/781 beta, eps_s = 720/781 eps; the common factor leaves the
// weights unchanged): eps_s enters the innermost FMA of each indicator and the
// scaled a_k = kA A_k, b_k = kB B_k serve both the indicators and z_k.
// From the first differences d1[j] = f_{j+1} - f_j of the stencil values.
template <class F>
__device__ __forceinline__ void weno7_terms_d1(const F d1[6], F eps_s, F z[4], F s[4]) {
  const F d10 = d1[0], d11 = d1[1], d12 = d1[2], d13 = d1[3], d14 = d1[4], d15 = d1[5];
  const F d20 = d11 - d10, d21 = d12 - d11, d22 = d13 - d12, d23 = d14 - d13, d24 = d15 - d14;
  const F c0 = d21 - d20, c1 = d22 - d21, c2 = d23 - d22, c3 = d24 - d23;
  const F e0 = c1 - c0, e1 = c2 - c1, e2 = c3 - c2;
  const F a0 = F(2 * kW7A) * d10 + F(-7 * kW7A) * d11 + F(11 * kW7A) * d12;
  const F a1 = F(2 * kW7A) * e0 + a0;
  const F a2 = F(-kW7A) * e1 + a1;
  const F a3 = F(2 * kW7A) * e2 + a2;
  const F b12 = F(kW7B) * d22;
  const F b0 = F(-kW7B) * e0 + b12;
  const F b3 = F(-kW7B) * e2 + b12;
  z[0] = F(1.0 / (12 * kW7A)) * a0 + F(1.0 / (12 * kW7B)) * b0;
  z[1] = F(1.0 / kW7A) * a1 + d22;
  z[2] = F(1.5 / kW7A) * a2 + F(1.5) * d22;
  z[3] = F(1.0 / (3 * kW7A)) * a3 + F(1.0 / (3 * kW7B)) * b3;
  const F m12 = b12 * b12 + eps_s;
  s[0] = a0 * a0 + (b0 * b0 + (c0 * c0 + eps_s));
  s[1] = a1 * a1 + (c1 * c1 + m12);
  s[2] = a2 * a2 + (c2 * c2 + m12);
  s[3] = a3 * a3 + (b3 * b3 + (c3 * c3 + eps_s));
}

template <class F>
__device__ __forceinline__ void weno7_terms(F f0, F f1, F f2, F f3, F f4, F f5, F f6, F eps_s, F z[4], F s[4]) {
  const F d1[6] = {f1 - f0, f2 - f1, f3 - f2, f4 - f3, f5 - f4, f6 - f5};
  weno7_terms_d1(d1, eps_s, z, s);
}

// FP64 weights in product form, t_k ~ prod_{j != k} s_j^2: the correction is
// num/den with a single division.
__device__ __forceinline__ void weno7_numden(const double z[4], const double s[4], double& num, double& den) {
  const double q0 = s[0] * s[0], q1 = s[1] * s[1], q2 = s[2] * s[2], q3 = s[3] * s[3];
  const double p01 = q0 * q1, p23 = q2 * q3;
  const double t0 = q1 * p23, t1 = q0 * p23, t2 = q3 * p01, t3 = q2 * p01;
  num = t0 * z[0] + t1 * z[1] + t2 * z[2] + t3 * z[3];
  den = t0 + 12.0 * t1 + 18.0 * t2 + 4.0 * t3;
}

// FP64 sum of the two reconstructions of one interface from first differences:
// g3 and dg[6] describe f+ (g3 = f+_i), h3 and dh[6] the negated mirrored f-
// (h3 = -f-_{i+1}); the reconstruction of a negated stencil is the negated
// reconstruction, so the sum is g3 - h3 + (ng dh - nh dg)/(dg dh): both
// corrections over one common denominator, one reciprocal instead of two.
// Each denominator lies in [eps_s^6, (eps_s + beta)^6], so the product neither
// underflows (eps_s >= 1e-20) nor overflows for any indicator below 1e25.
__device__ __forceinline__ double weno7_sum_d1(double g3, const double dg[6], double h3, const double dh[6],
                                               double eps_s) {
  double zg[4], sg[4], zh[4], sh[4], ng, qg, nh, qh;
  weno7_terms_d1(dg, eps_s, zg, sg);
  weno7_terms_d1(dh, eps_s, zh, sh);
  weno7_numden(zg, sg, ng, qg);
  weno7_numden(zh, sh, nh, qh);
  return (g3 - h3) + (ng * qh - nh * qg) * rcp_nr(qg * qh);
}

// ---- FP32 pair form: two reconstructions that run the same operation
// sequence are evaluated together in the two lanes of Blackwell's packed
// FP32x2 instructions (FFMA2, FADD2, FMUL2), halving the issue slots.

__device__ __forceinline__ float2 bc2(float c) { return make_float2(c, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 rcp2(float2 a) { return make_float2(rcp_approx(a.x), rcp_approx(a.y)); }

// The reconstruction of weno7_terms with reciprocal weights per lane.
__device__ __forceinline__ float2 weno7_pair(float2 f0, float2 f1, float2 f2, float2 f3, float2 f4, float2 f5,
                                             float2 f6, float eps_s) {
  const float2 d10 = sub2(f1, f0), d11 = sub2(f2, f1), d12 = sub2(f3, f2), d13 = sub2(f4, f3), d14 = sub2(f5, f4),
               d15 = sub2(f6, f5);
  const float2 d20 = sub2(d11, d10), d21 = sub2(d12, d11), d22 = sub2(d13, d12), d23 = sub2(d14, d13),
               d24 = sub2(d15, d14);
  const float2 c0 = sub2(d21, d20), c1 = sub2(d22, d21), c2 = sub2(d23, d22), c3 = sub2(d24, d23);
  const float2 e0 = sub2(c1, c0), e1 = sub2(c2, c1), e2 = sub2(c3, c2);
  const float kA = (float)kW7A, kB = (float)kW7B;
  const float2 a0 = fma2(bc2(2 * kA), d10, fma2(bc2(-7 * kA), d11, mul2(bc2(11 * kA), d12)));
  const float2 a1 = fma2(bc2(2 * kA), e0, a0);
  const float2 a2 = fma2(bc2(-kA), e1, a1);
  const float2 a3 = fma2(bc2(2 * kA), e2, a2);
  const float2 b12 = mul2(bc2(kB), d22);
  const float2 b0 = fma2(bc2(-kB), e0, b12);
  const float2 b3 = fma2(bc2(-kB), e2, b12);
  const float2 z0 = fma2(bc2((float)(1.0 / (12 * kW7A))), a0, mul2(bc2((float)(1.0 / (12 * kW7B))), b0));
  const float2 z1 = fma2(bc2((float)(1.0 / kW7A)), a1, d22);
  const float2 z2 = fma2(bc2((float)(1.5 / kW7A)), a2, mul2(bc2(1.5f), d22));
  const float2 z3 = fma2(bc2((float)(1.0 / (3 * kW7A))), a3, mul2(bc2((float)(1.0 / (3 * kW7B))), b3));
  const float2 e = bc2(eps_s);
  const float2 m12 = fma2(b12, b12, e);
  float2 t0 = rcp2(fma2(a0, a0, fma2(b0, b0, fma2(c0, c0, e))));
  float2 t1 = rcp2(fma2(a1, a1, fma2(c1, c1, m12)));
  float2 t2 = rcp2(fma2(a2, a2, fma2(c2, c2, m12)));
  float2 t3 = rcp2(fma2(a3, a3, fma2(b3, b3, fma2(c3, c3, e))));
  t0 = mul2(t0, t0);
  t1 = mul2(t1, t1);
  t2 = mul2(t2, t2);
  t3 = mul2(t3, t3);
  const float2 num = fma2(t0, z0, fma2(t1, z1, fma2(t2, z2, mul2(t3, z3))));
  const float2 den = fma2(bc2(12.0f), t1, fma2(bc2(18.0f), t2, fma2(bc2(4.0f), t3, t0)));
  return fma2(num, rcp2(den), f3);
}

// WENO5 weights (linear weights (1, 6, 3)/10), candidates carrying d_k.
__device__ __forceinline__ double weno5_combine(double Q0, double Q1, double Q2, double b0, double b1, double b2,
                                                double eps) {
  double s0 = eps + b0, s1 = eps + b1, s2 = eps + b2;
  s0 *= s0;
  s1 *= s1;
  s2 *= s2;
  const double t0 = s1 * s2, t1 = s0 * s2, t2 = s0 * s1;
  return (t0 * Q0 + t1 * Q1 + t2 * Q2) * rcp_nr(t0 + 6.0 * t1 + 3.0 * t2);
}

__device__ __forceinline__ float weno5_combine(float Q0, float Q1, float Q2, float b0, float b1, float b2, float eps) {
  float t0 = rcp_approx(eps + b0), t1 = rcp_approx(eps + b1), t2 = rcp_approx(eps + b2);
  t0 *= t0;
  t1 *= t1;
  t2 *= t2;
  return (t0 * Q0 + t1 * Q1 + t2 * Q2) * rcp_approx(t0 + 6.0f * t1 + 3.0f * t2);
}

constexpr double kW5EpsScale = 12.0 / 13.0;
constexpr double kW5G = 0.4803844614152614;   // sqrt(3/13)

// WENO5 (Sec. 1, 5th order): quadratic candidates on {i-2..i}, {i-1..i+1},
// {i..i+2}; Jiang-Shu indicators beta = 13/12 (2nd difference)^2 + 1/4 g^2 with g
// the first-derivative combination, used as (12/13) beta = d^2 + (sqrt(3/13) g)^2;
// linear weights (1, 6, 3)/10.  eps_s is (12/13) eps.
template <class F>
__device__ __forceinline__ F weno5(F f0, F f1, F f2, F f3, F f4, F eps_s) {
  const F Q0 = F(2.0 / 6.0) * f0 + F(-7.0 / 6.0) * f1 + F(11.0 / 6.0) * f2;
  const F Q1 = -f1 + F(5) * f2 + F(2) * f3;
  const F Q2 = f2 + F(2.5) * f3 + F(-0.5) * f4;
  const F d0 = f0 - F(2) * f1 + f2, d1 = f1 - F(2) * f2 + f3, d2 = f2 - F(2) * f3 + f4;
  const F g0 = F(kW5G) * f0 + F(-4 * kW5G) * f1 + F(3 * kW5G) * f2;
  const F g1 = F(kW5G) * (f1 - f3);
  const F g2 = F(3 * kW5G) * f2 + F(-4 * kW5G) * f3 + F(kW5G) * f4;
  return weno5_combine(Q0, Q1, Q2, d0 * d0 + g0 * g0, d1 * d1 + g1 * g1, d2 * d2 + g2 * g2, eps_s);
}

// weno5 for FP32 in the two lanes of packed FP32x2 instructions (the left-biased
// reconstruction of an interface in x, the mirrored one in y), the same terms and
// weights as the scalar form.
__device__ __forceinline__ float2 weno5_pair(float2 f0, float2 f1, float2 f2, float2 f3, float2 f4, float eps_s) {
  const float g = (float)kW5G;
  const float2 Q0 = fma2(bc2((float)(11.0 / 6.0)), f2, fma2(bc2((float)(-7.0 / 6.0)), f1,
                                                              mul2(bc2((float)(2.0 / 6.0)), f0)));
  const float2 Q1 = fma2(bc2(2.0f), f3, fma2(bc2(5.0f), f2, mul2(bc2(-1.0f), f1)));
  const float2 Q2 = fma2(bc2(-0.5f), f4, fma2(bc2(2.5f), f3, f2));
  const float2 d0 = add2(fma2(bc2(-2.0f), f1, f0), f2), d1 = add2(fma2(bc2(-2.0f), f2, f1), f3),
               d2 = add2(fma2(bc2(-2.0f), f3, f2), f4);
  const float2 g0 = fma2(bc2(3.0f * g), f2, fma2(bc2(-4.0f * g), f1, mul2(bc2(g), f0)));
  const float2 g1 = mul2(bc2(g), sub2(f1, f3));
  const float2 g2 = fma2(bc2(g), f4, fma2(bc2(-4.0f * g), f3, mul2(bc2(3.0f * g), f2)));
  const float2 e = bc2(eps_s);
  float2 t0 = rcp2(add2(e, fma2(d0, d0, mul2(g0, g0))));
  float2 t1 = rcp2(add2(e, fma2(d1, d1, mul2(g1, g1))));
  float2 t2 = rcp2(add2(e, fma2(d2, d2, mul2(g2, g2))));
  t0 = mul2(t0, t0);
  t1 = mul2(t1, t1);
  t2 = mul2(t2, t2);
  const float2 num = fma2(t2, Q2, fma2(t1, Q1, mul2(t0, Q0)));
  const float2 den = fma2(bc2(3.0f), t2, fma2(bc2(6.0f), t1, t0));
  return mul2(num, rcp2(den));
}

// Temperature from e = (pi^2/30) dof T^4 / (hbar c)^3: T = (e t4coef)^(1/4).
__device__ __forceinline__ double temperature(double e, double t4coef) {
  double x = e * t4coef;
  x = x > 0.0 ? x : 0.0;
  return sqrt(sqrt(x));
}

}  // namespace hydro
