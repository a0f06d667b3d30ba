// Device arithmetic of the stage kernel that is worth testing on its own: the reciprocal and the two halves
// of the WENO5 interface value. Included by rlb.cu and by the GPU unit test of these functions.
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

// Products and sums that are rounded exactly as written. The compiler may contract a product into a following
// addition (an FMA), and may do so differently in different inlined copies of the same expression. The
// reduced-precision kernel evaluates each interface value and each indicator pair at a lane's edges twice (once
// in each lane that uses it), and its compensated sums are error-free only if every addition is rounded as
// written, so its FP32 arithmetic goes through these (mul.rn / add.rn / sub.rn are never contracted). The FP64
// path evaluates every interface once and keeps the compiler's choices.
__device__ __forceinline__ float mul_x(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_x(double a, double b) { return a * b; }
__device__ __forceinline__ float add_x(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_x(double a, double b) { return a + b; }
__device__ __forceinline__ float sub_x(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_x(double a, double b) { return a - b; }

// Fifth-order WENO (Jiang & Shu) written on first differences d_l = v_l - v_{l-1} of five samples
// v0..v4 ordered along the wind (v2 is the upwind cell next to the interface, whose value is v2 + G):
//   candidates (2,-7,11)/6, (-1,5,2)/6, (2,5,-1)/6  =  v2 + r_k/6,  r0 = 5 d2 - 2 d1, r1 = d2 + 2 d3,
//   r2 = 4 d3 - d4;
//   smoothness indicators (weights 13/12 and 1/4): 3 beta_k = SL(d1,d2), SC(d2,d3), SR(d3,d4) with
//   SL(x,y) = 4x^2 - 11xy + 10y^2, SC = 4x^2 - 5xy + 4y^2, SR = 10x^2 - 11xy + 4y^2;
//   alpha_k = d_k / (eps + beta_k)^2 with d = (1, 6, 3)/10 equals 9 / s_k, s_k = u_k^2,
//   u_k = (3 eps + 3 beta_k) / sqrt(d_k); the normalised weights are w_k = prod_{l!=k} s_l / sum_m prod_{l!=m} s_l.
// Each indicator depends on one pair of adjacent differences, and each pair serves three interfaces, so
// the kernel evaluates the three scaled squares once per pair (weno5_pair) and combines three pairs per
// interface (weno5_combine). For a wind toward decreasing index the stencil is mirrored: the differences
// change sign and order, which swaps the roles of SL and SR.
constexpr double C0 = 3.1622776601683795;  // sqrt(10)
constexpr double C1 = 1.2909944487358056;  // sqrt(10/6)
constexpr double C2 = 1.8257418583505538;  // sqrt(10/3)
// epsilon terms 3 eps (C0, C1, C2) of indicators taken on weight-normalised values
constexpr float EPS_A = (float)(3.0 * WENO_EPS * C0);
constexpr float EPS_B = (float)(3.0 * WENO_EPS * C1);
constexpr float EPS_C = (float)(3.0 * WENO_EPS * C2);

// Reciprocal used by the WENO combination: FP64 as above; FP32 the hardware approximation alone (about 1 ulp
// of FP32, below the rounding of the FP32 state it serves).
__device__ __forceinline__ double rcp_fast(double d) { return rcp_nr(d); }
__device__ __forceinline__ float rcp_fast(float d) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(d));
  return r;
}

// Scaled indicator squares of the pair (x, y) = (d_j, d_{j+1}) in memory order. fwd: wind toward increasing
// index; then sA = (C0 (SL + 3eps))^2, sB = (C1 (SC + 3eps))^2, sC = (C2 (SR + 3eps))^2; otherwise SL and SR
// trade places. (eA, eB, eC) = 3 eps (C0, C1, C2): the velocity's epsilon term, which scales with the square
// of its quadrature weight. T is double (FP64 path) or float (reduced-precision path).
template <typename T>
__device__ __forceinline__ void weno5_pair(T x, T y, bool fwd, T eA, T eB, T eC, T& sA, T& sB, T& sC) {
  const T qx = mul_x(x, x), pxy = mul_x(x, y), qy = mul_x(y, y);
  const T ax = fwd ? T(4.0 * C0) : T(10.0 * C0), ay = fwd ? T(10.0 * C0) : T(4.0 * C0);
  const T cx = fwd ? T(10.0 * C2) : T(4.0 * C2), cy = fwd ? T(4.0 * C2) : T(10.0 * C2);
  const T uA = fma(ax, qx, fma(T(-11.0 * C0), pxy, fma(ay, qy, eA)));
  const T uB = fma(T(4.0 * C1), qx, fma(T(-5.0 * C1), pxy, fma(T(4.0 * C1), qy, eB)));
  const T uC = fma(cx, qx, fma(T(-11.0 * C2), pxy, fma(cy, qy, eC)));
  sA = mul_x(uA, uA);
  sB = mul_x(uB, uB);
  sC = mul_x(uC, uC);
}

// weno5_pair from the products x^2, x y, y^2 (the FP64 kernel forms each difference's square once and shares
// it between the two pairs the difference belongs to).
template <typename T>
__device__ __forceinline__ void weno5_pair_q(T qx, T pxy, T qy, bool fwd, T eA, T eB, T eC, T& sA, T& sB, T& sC) {
  const T ax = fwd ? T(4.0 * C0) : T(10.0 * C0), ay = fwd ? T(10.0 * C0) : T(4.0 * C0);
  const T cx = fwd ? T(10.0 * C2) : T(4.0 * C2), cy = fwd ? T(4.0 * C2) : T(10.0 * C2);
  const T uA = fma(ax, qx, fma(T(-11.0 * C0), pxy, fma(ay, qy, eA)));
  const T uB = fma(T(4.0 * C1), qx, fma(T(-5.0 * C1), pxy, fma(T(4.0 * C1), qy, eB)));
  const T uC = fma(cx, qx, fma(T(-11.0 * C2), pxy, fma(cy, qy, eC)));
  sA = uA * uA;
  sB = uB * uB;
  sC = uC * uC;
}

// 6 G of the interface from the three scaled squares (s0, s1, s2) of its stencils and the differences
// d1..d4 in wind order (the FP64 stage kernel applies the 1/6 in the flux difference, where it costs nothing).
template <typename T>
__device__ __forceinline__ T weno5_combine6(T s0, T s1, T s2, T d1, T d2, T d3, T d4) {
  const T r0 = fma(T(5.0), d2, mul_x(T(-2.0), d1)), r1 = fma(T(2.0), d3, d2), r2 = fma(T(4.0), d3, -d4);
  const T a0 = mul_x(s1, s2);
  const T num = fma(s0, fma(s2, r1, mul_x(s1, r2)), mul_x(a0, r0));
  const T den = fma(s0, add_x(s1, s2), a0);
  return mul_x(num, rcp_fast(den));
}

// G of the interface.
template <typename T>
__device__ __forceinline__ T weno5_combine(T s0, T s1, T s2, T d1, T d2, T d3, T d4) {
  return weno5_combine6(s0, s1, s2, d1, d2, d3, d4) * T(1.0 / 6.0);
}

// Interface value v2 + G of five samples in memory order m0..m4 around the interface between m2 and m3
// (wind toward increasing index, fwd) or between m1 and m2 (wind toward decreasing index), computed
// exactly as the stage kernels do: pairs first, then the combination. eps: the limiter's epsilon.
template <typename T>
__device__ __forceinline__ T weno5_interface(T m0, T m1, T m2, T m3, T m4, bool fwd, double eps = WENO_EPS) {
  const T D1 = m1 - m0, D2 = m2 - m1, D3 = m3 - m2, D4 = m4 - m3;
  const T eA = T(3.0 * eps * C0), eB = T(3.0 * eps * C1), eC = T(3.0 * eps * C2);
  T a[3], b[3], c[3];
  weno5_pair(D1, D2, fwd, eA, eB, eC, a[0], b[0], c[0]);
  weno5_pair(D2, D3, fwd, eA, eB, eC, a[1], b[1], c[1]);
  weno5_pair(D3, D4, fwd, eA, eB, eC, a[2], b[2], c[2]);
  if (fwd) return m2 + weno5_combine(a[0], b[1], c[2], D1, D2, D3, D4);
  return m2 + weno5_combine(a[2], b[1], c[0], -D4, -D3, -D2, -D1);
}

// Compensated (double-float) accumulation in FP32 for the moment sums of the reduced-precision path: an
// unevaluated sum hi + lo, the error of each addition recovered with Knuth's TwoSum and of each product with
// an FMA (the error-free transformations of Ogita, Rump and Oishi's accurate dot product). Weights are
// themselves given as hi + lo float pairs, so the sums reach about 1e-13 relative before they are reduced
// in FP64.
struct DF {
  float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// acc += f (whi + wlo)
__device__ __forceinline__ void df_add_prod(DF& acc, float f, float whi, float wlo) {
  const float p = __fmul_rn(f, whi);
  float e = fmaf(f, whi, -p);
  e = fmaf(f, wlo, e);
  float s, t;
  two_sum(acc.hi, p, s, t);
  acc.hi = s;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(t, e));
}

// acc += a (xhi + xlo)
__device__ __forceinline__ void df_add_dfprod(DF& acc, DF a, float xhi, float xlo) {
  const float p = __fmul_rn(a.hi, xhi);
  float e = fmaf(a.hi, xhi, -p);
  e = fmaf(a.hi, xlo, e);
  e = fmaf(a.lo, xhi, e);
  float s, t;
  two_sum(acc.hi, p, s, t);
  acc.hi = s;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(t, e));
}

// acc += a
__device__ __forceinline__ void df_add(DF& acc, DF a) {
  float s, t;
  two_sum(acc.hi, a.hi, s, t);
  acc.hi = s;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(t, a.lo));
}

}  // namespace rlbdev
