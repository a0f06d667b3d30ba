// Device arithmetic of the stage kernel that is worth testing on its own: the reciprocal and the WENO5
// interface correction. Included by rlb.cu and by the GPU unit test of these two functions.
#pragma once

namespace rlbdev {

// 1/d for positive, normal d: the hardware approximation of rcp.approx.ftz.f64 (relative error ~1e-6,
// measured) refined by one cubically convergent Newton-Raphson step, x1 = x0 (1 + e + e^2) with
// e = 1 - d x0 (the truncated geometric series of 1/(1 - e)); the result is within 2 ulp of the
// correctly rounded quotient. Costs three FP64 FMAs instead of the ~8 FP64-pipe slots of an IEEE division.
__device__ __forceinline__ double rcp_nr(double d) {
  double x0;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(x0) : "d"(d));
  const double e = fma(-d, x0, 1.0);
  return fma(x0, fma(e, e, e), x0);
}

constexpr double WENO_EPS = 1e-6;

// Fifth-order WENO (Jiang & Shu) interface value from five samples ordered along the wind, v2 being the
// upwind cell next to the interface; returns G with interface value v2 + G.
//   Candidates (2,-7,11)/6, (-1,5,2)/6, (2,5,-1)/6 = v2 + r_k/6 with r0 = 5 d2 - 2 d1, r1 = d2 + 2 d3,
//   r2 = 4 d3 - d4 on the first differences d_l = v_l - v_{l-1}.
//   Smoothness indicators (weights 13/12 and 1/4): 3 beta_k are the quadratic forms 4x^2 - 11xy + 10y^2,
//   4x^2 - 5xy + 4y^2, 10x^2 - 11xy + 4y^2 of adjacent differences.
//   alpha_k = d_k / (eps + beta_k)^2 with d = (1, 6, 3)/10 equals 9 / u_k^2 for
//   u_k = (3 eps + 3 beta_k) / sqrt(d_k), so the normalised weights are w_k = prod_{l!=k} s_l / sum_m
//   prod_{l!=m} s_l with s_k = u_k^2 (the sqrt(1/d_k) factors are folded into the coefficients).
__device__ __forceinline__ double weno5_corr(double v0, double v1, double v2, double v3, double v4) {
  constexpr double c0 = 3.1622776601683795;  // sqrt(10)
  constexpr double c1 = 1.2909944487358056;  // sqrt(10/6)
  constexpr double c2 = 1.8257418583505538;  // sqrt(10/3)
  constexpr double E = 3.0 * WENO_EPS;
  const double d1 = v1 - v0, d2 = v2 - v1, d3 = v3 - v2, d4 = v4 - v3;
  const double q1 = d1 * d1, q2 = d2 * d2, q3 = d3 * d3, q4 = d4 * d4;
  const double p12 = d1 * d2, p23 = d2 * d3, p34 = d3 * d4;
  const double u0 = fma(4.0 * c0, q1, fma(-11.0 * c0, p12, fma(10.0 * c0, q2, E * c0)));
  const double u1 = fma(4.0 * c1, q2, fma(-5.0 * c1, p23, fma(4.0 * c1, q3, E * c1)));
  const double u2 = fma(10.0 * c2, q3, fma(-11.0 * c2, p34, fma(4.0 * c2, q4, E * c2)));
  const double s0 = u0 * u0, s1 = u1 * u1, s2 = u2 * u2;
  const double r0 = fma(5.0, d2, -2.0 * d1), r1 = fma(2.0, d3, d2), r2 = fma(4.0, d3, -d4);
  const double a0 = s1 * s2;
  const double num = fma(s0, fma(s2, r1, s1 * r2), a0 * r0);
  const double den = fma(s0, s1 + s2, a0);
  return num * rcp_nr(6.0 * den);
}

}  // namespace rlbdev
