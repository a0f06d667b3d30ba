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


// ---------------------------------------------------------------------------------------------------------
// WENO5 limiter of the FP64 stage kernel in double-float arithmetic.
//
// GB300 executes FP32 at 64 times its FP64 rate, and the FP64 stage kernel is bound by the FP64 pipe while
// its issue slots are mostly idle. The limiter (indicators, nonlinear weights, the weighted candidate sum) is
// about two thirds of the kernel's FP64 operations, so the kernel evaluates it in double-float: a value is
// an unevaluated sum hi + lo of two floats (about 47 significant bits), combined with the error-free
// transformations TwoSum (Knuth), FastTwoSum (Dekker) and the FMA-based TwoProduct. Every product and sum is
// written with explicit rounding (fmaf, __fmul_rn, __fadd_rn, __fsub_rn), so that the compiler cannot fuse
// or reorder what the transformations rely on. The differences entering the limiter come from the FP64
// state; the 6 G returned per interface carries an absolute error of a few 1e-14 of the differences around
// it (the error of the limiter's FP64 form is ~1e-16 of them), well inside the FP64 path's 1e-12 parity.
//
// Indicators: with the linear weights d = (1, 6, 3)/10 taken out of the squares, the three indicators of a
// pair of adjacent differences (x, y) are v = S + e with S the integer quadratic forms
//   SL(x, y) = 4x^2 - 11xy + 10y^2, SC = 4x^2 - 5xy + 4y^2, SR = 10x^2 - 11xy + 4y^2  (= 3 beta_k)
// and e = 3 eps ws^2 (the velocity's epsilon term). With t_k = v_k^2 the interface value is
//   6 G = [t1 t2 r0 + 3 t0 (2 t2 r1 + t1 r2)] / [t1 t2 + 3 t0 (2 t2 + t1)],
// the weights d_k / t_k multiplied through by t0 t1 t2 / 10 (r_k as in weno5_combine6). The v_k of one
// interface are first scaled by a common power of two so that the largest lies in [1, 2): the weights are
// homogeneous in t, and the scaling keeps the products of the t's inside the FP32 exponent range.

// a + b = s + e exactly, |a| >= |b| (or a == 0)
__device__ __forceinline__ DF fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// a + b, robust to cancellation of the high parts
__device__ __forceinline__ DF df_plus(DF a, DF b) {
  float s, t;
  two_sum(a.hi, b.hi, s, t);
  t = __fadd_rn(t, __fadd_rn(a.lo, b.lo));
  float u, w;
  two_sum(s, t, u, w);
  return {u, w};
}

// a + b for a, b >= 0 (no cancellation)
__device__ __forceinline__ DF df_plus_pos(DF a, DF b) {
  float s, t;
  two_sum(a.hi, b.hi, s, t);
  return fast_two_sum(s, __fadd_rn(t, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ DF df_neg(DF a) { return {-a.hi, -a.lo}; }

// a * 2^k for a float power of two p (exact)
__device__ __forceinline__ DF df_pow2(DF a, float p) { return {__fmul_rn(a.hi, p), __fmul_rn(a.lo, p)}; }

__device__ __forceinline__ DF df_times(DF a, DF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  const float e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, fmaf(a.hi, b.hi, -p)));
  return fast_two_sum(p, e);
}

__device__ __forceinline__ DF df_square(DF a) {
  const float p = __fmul_rn(a.hi, a.hi);
  const float e = fmaf(__fadd_rn(a.hi, a.hi), a.lo, fmaf(a.hi, a.hi, -p));
  return fast_two_sum(p, e);
}

// a * c for a small integer c (exactly representable), unnormalised: the product of the high parts rounded,
// its rounding error and c a.lo in the second float
__device__ __forceinline__ DF df_times_int(DF a, float c) {
  const float p = __fmul_rn(a.hi, c);
  return {p, fmaf(a.lo, c, fmaf(a.hi, c, -p))};
}

// d = hi + lo with hi the top 24 significant bits of d (truncated) and lo the next 23 (|lo| < ulp(hi)); by
// integer operations on d's bits, so that the split costs no FP64 instruction. |d| < 2^-126 gives 0 (such a
// difference is far below the epsilon term and the values around it); |d| >= 2^128 gives FP32's overflow.
__device__ __forceinline__ DF df_split(double d) {
  const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
  const int e = (int)((hi >> 20) & 0x7FFu);
  if (e <= 896) return {0.0f, 0.0f};
  if (e >= 1151) return {__double2float_rn(d), 0.0f};
  const unsigned sgn = hi & 0x80000000u;
  const float h = __uint_as_float(sgn | ((unsigned)(e - 896) << 23) | (__funnelshift_l(lo, hi, 3) & 0x7FFFFFu));
  float l = 0.0f;
  if (e >= 920) {  // x 2^(E - 46) with x the next 23 bits, E = e - 1023: (2^23 + x) 2^(E - 23) - 2^(E - 23)
    const unsigned k = sgn | ((unsigned)(e - 919) << 23);
    l = __fsub_rn(__uint_as_float(k | ((lo & 0x1FFFFFFFu) >> 6)), __uint_as_float(k));
  }
  return {h, l};
}

// The double equal to the float f (0 for zero and subnormal f), by integer operations on f's bits.
__device__ __forceinline__ double df_widen(float f) {
  const unsigned b = __float_as_uint(f), ef = (b >> 23) & 0xFFu;
  const unsigned hi = (b & 0x80000000u) | ((ef + 896u) << 20) | ((b >> 3) & 0xFFFFFu);
  const double w = __hiloint2double((int)hi, (int)(b << 29));
  return ef == 0u ? 0.0 : w;
}

// Indicators v_A, v_B, v_C of the pair (x, y) = (d_j, d_{j+1}) in memory order, e the epsilon term. fwd (wind
// toward increasing index): (v_A, v_B, v_C) = (SL, SC, SR)(x, y) + e; otherwise SL and SR trade places.
__device__ __forceinline__ void weno5_pair_df(DF x, DF y, bool fwd, DF e, DF& vA, DF& vB, DF& vC) {
  // x^2, x y, y^2 as (rounded product of the high parts, its error plus the cross terms)
  const float px = __fmul_rn(x.hi, x.hi), py = __fmul_rn(y.hi, y.hi), pz = __fmul_rn(x.hi, y.hi);
  const DF X = {px, fmaf(__fadd_rn(x.hi, x.hi), x.lo, fmaf(x.hi, x.hi, -px))};
  const DF Y = {py, fmaf(__fadd_rn(y.hi, y.hi), y.lo, fmaf(y.hi, y.hi, -py))};
  const DF Z = {pz, fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, fmaf(x.hi, y.hi, -pz)))};
  const DF X4 = df_pow2(X, 4.0f), Y4 = df_pow2(Y, 4.0f);
  const DF X10 = df_times_int(X, 10.0f), Y10 = df_times_int(Y, 10.0f);
  const DF Z11 = df_times_int(Z, -11.0f), Z5 = df_times_int(Z, -5.0f);
  // (a, b, c) + e: exact sums of the high parts, then the low parts and the errors; v > 0 is a positive
  // definite form plus e, so the final FastTwoSum's ordering holds
  auto sum3 = [&](DF a, DF b, DF c) {
    float s, t1, t2, t3;
    two_sum(a.hi, b.hi, s, t1);
    two_sum(s, c.hi, s, t2);
    two_sum(s, e.hi, s, t3);
    const float lo = __fadd_rn(__fadd_rn(__fadd_rn(a.lo, b.lo), __fadd_rn(c.lo, e.lo)),
                               __fadd_rn(__fadd_rn(t1, t2), t3));
    return fast_two_sum(s, lo);
  };
  const DF L = sum3(X4, Z11, Y10), R = sum3(X10, Z11, Y4);
  vA = fwd ? L : R;
  vB = sum3(X4, Z5, Y4);
  vC = fwd ? R : L;
}

// 6 G of the interface from the indicators (v0, v1, v2) of its stencils and the differences d1..d4 in wind
// order, in double-float.
__device__ __forceinline__ DF weno5_combine6_df(DF v0, DF v1, DF v2, DF d1, DF d2, DF d3, DF d4) {
  // common power-of-two scale: the largest v lands in [1, 2)
  const unsigned em = __float_as_uint(fmaxf(fmaxf(v0.hi, v1.hi), v2.hi)) >> 23;
  const float sc = __uint_as_float((254u - em) << 23);
  const DF t0 = df_square(df_pow2(v0, sc)), t1 = df_square(df_pow2(v1, sc)), t2 = df_square(df_pow2(v2, sc));
  // r0 = 5 d2 - 2 d1, r1 = d2 + 2 d3, r2 = 4 d3 - d4 (6 times the candidates' corrections)
  const DF r0 = df_plus(df_times_int(d2, 5.0f), df_pow2(d1, -2.0f));
  const DF r1 = df_plus(d2, df_pow2(d3, 2.0f));
  const DF r2 = df_plus(df_pow2(d3, 4.0f), df_neg(d4));
  const DF a0 = df_times(t1, t2);
  const DF t0x3 = df_times_int(t0, 3.0f);
  const DF t03 = fast_two_sum(t0x3.hi, t0x3.lo);
  const DF num = df_plus(df_times(a0, r0),
                         df_times(t03, df_plus(df_pow2(df_times(t2, r1), 2.0f), df_times(t1, r2))));
  const DF den = df_plus_pos(a0, df_times(t03, df_plus_pos(df_pow2(t2, 2.0f), t1)));
  if (den.hi == 0.0f) {  // all but one t below FP32's range (indicator ratios beyond ~1e19): that stencil's value
    const bool k0 = v0.hi <= v1.hi && v0.hi <= v2.hi, k1 = !k0 && v1.hi <= v2.hi;
    return k0 ? r0 : (k1 ? r1 : r2);
  }
  // num / den: a quotient from FP32's reciprocal (approximation refined by one Newton-Raphson step to about
  // half an ulp), then one correction from the remainder
  float rc;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rc) : "f"(den.hi));
  rc = fmaf(rc, fmaf(-den.hi, rc, 1.0f), rc);
  const float q1 = __fmul_rn(num.hi, rc);
  const float p = __fmul_rn(q1, den.hi);
  const float pe = fmaf(q1, den.lo, fmaf(q1, den.hi, -p));
  const float rem = __fadd_rn(__fsub_rn(num.hi, p), __fsub_rn(num.lo, pe));
  float s, t;
  two_sum(q1, __fmul_rn(rem, rc), s, t);
  return {s, t};
}

// Interface value v2 + G computed as the FP64 stage kernel does with the double-float limiter (differences in
// FP64, split, pairs, combination, 6 G widened and divided by 6 in FP64); eps: the limiter's epsilon.
__device__ __forceinline__ double weno5_interface_df(double m0, double m1, double m2, double m3, double m4, bool fwd,
                                                     double eps = WENO_EPS) {
  const DF D1 = df_split(m1 - m0), D2 = df_split(m2 - m1), D3 = df_split(m3 - m2), D4 = df_split(m4 - m3);
  const DF e = df_split(3.0 * eps);
  DF a[3], b[3], c[3];
  weno5_pair_df(D1, D2, fwd, e, a[0], b[0], c[0]);
  weno5_pair_df(D2, D3, fwd, e, a[1], b[1], c[1]);
  weno5_pair_df(D3, D4, fwd, e, a[2], b[2], c[2]);
  const DF G = fwd ? weno5_combine6_df(a[0], b[1], c[2], D1, D2, D3, D4)
                   : weno5_combine6_df(a[2], b[1], c[0], df_neg(D4), df_neg(D3), df_neg(D2), df_neg(D1));
  return fma(df_widen(G.hi), 1.0 / 6.0, fma(df_widen(G.lo), 1.0 / 6.0, m2));
}

}  // namespace rlbdev
