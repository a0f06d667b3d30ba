/*
 * Plain FP64 CPU oracle for the time step of the quadrature-based finite-difference relativistic
 * lattice Boltzmann model for massless particles (Blaga & Ambrus, arXiv:1608.03004).
 *
 * TEST INFRASTRUCTURE ONLY. This file exists to check the CUDA path: only tests/, the smoke check in
 * __graft_entry__.py and the CPU-baseline leg of bench.py may build, load or call it. It shares no code,
 * header, table or constant with the CUDA library, and it is written to be read against the paper, not
 * to be fast: every step is the plain definition, in the paper's order and notation.
 *
 * Notation (paper, section "Lattice Boltzmann model"): momentum magnitude pbar = p/T0 with T0 = 1,
 * direction cosine xi = v^z = cos(theta). The paper's z axis is called x here. The discrete velocity
 * s = i*Qxi + j pairs the radial node pbar_i (generalised Gauss-Laguerre, alpha = 1) with the polar node
 * xi_j (Gauss-Legendre). The azimuthal quadrature is a constant factor 2*pi because f does not depend on
 * phi in the one-dimensional problem (section "Riemann problem").
 *
 * State variable. The stored population is F_ij = 2*pi * w^p_i * w^xi_j * exp(pbar_i) * f(pbar_i, xi_j),
 * so that the moments of section "Relativistic lattice Boltzmann equation" become plain sums:
 *   N^0 = sum F pbar,  N^z = sum F pbar xi,  T^00 = sum F pbar^2,  T^0z = sum F pbar^2 xi,
 *   T^zz = sum F pbar^2 xi^2.
 * The kinetic equation, Eq. (Boltz), is linear in f with a rate that depends on xi only, so F obeys it too.
 *
 * Readings where the paper is silent or garbled:
 *  - Legendre weight, Eq. (polarInt): the printed 2(1-xi_j)^2 is read as 2(1-xi_j^2) (textbook form).
 *  - The expansion coefficients of Eq. (feqtrunc) are omitted in the paper; the truncation is read as the
 *    orthogonal projection of exp(pbar) f^eq onto L^(1)_l(pbar) P_k(xi), l <= Np, k <= Nv, which is what
 *    makes the moments of Eq. (mom_feq) exact.
 *  - n in f^eq is the Landau density n = -u_mu N^mu (it makes the collision conserve N^mu).
 *  - WENO variant: Jiang-Shu WENO5, upwind by the sign of xi, applied to the weight-normalised population
 *    g_s = F_s / (w^p_i w^xi_j / 2) with eps = 1e-6 (equivalently to F_s with eps scaled by the squared
 *    weight), so that the limiter acts alike on every direction whatever the quadrature order.
 *  - Time integration: Shu-Osher SSP-RK3; the collision uses each stage's own moments.
 *  - Open boundary: three zero-gradient ghost cells per side, refreshed every stage.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2
#define ORC_ENONPHYS 4

#define ORC_BC_OPEN 0
#define ORC_BC_PERIODIC 1

#define WENO_EPS 1e-6

/* ------------------------------------------------------------------------------------------------ */
/* Orthogonal polynomials by their three-term recurrences, in long double.                           */
/* ------------------------------------------------------------------------------------------------ */

/* Legendre P_n(x): (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}. */
static long double legendre_P(int n, long double x) {
  long double p0 = 1.0L, p1 = x;
  if (n == 0) return p0;
  for (int k = 1; k < n; ++k) {
    long double p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1);
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

/* Generalised Laguerre L^(1)_n(x): (k+1) L_{k+1} = (2k+2-x) L_k - (k+1) L_{k-1}, L_0 = 1, L_1 = 2-x. */
static long double laguerre1_L(int n, long double x) {
  long double l0 = 1.0L, l1 = 2.0L - x;
  if (n == 0) return l0;
  for (int k = 1; k < n; ++k) {
    long double l2 = ((2 * k + 2 - x) * l1 - (k + 1) * l0) / (k + 1);
    l0 = l1;
    l1 = l2;
  }
  return l1;
}

double orc_legendre_P(int n, double x) { return (double)legendre_P(n, x); }
double orc_laguerre1_L(int n, double x) { return (double)laguerre1_L(n, x); }

/* ------------------------------------------------------------------------------------------------ */
/* Quadrature, section "Discretization of the momentum space using quadrature rules".                */
/* ------------------------------------------------------------------------------------------------ */

/* Roots of a polynomial on [a, b] by scanning for sign changes and bisecting each bracket. */
static int bracket_roots(long double (*poly)(int, long double), int n, long double a, long double b,
                         long nscan, long double *roots) {
  int found = 0;
  long double h = (b - a) / nscan;
  long double x0 = a, f0 = poly(n, x0);
  for (long s = 1; s <= nscan && found < n; ++s) {
    long double x1 = a + h * s, f1 = poly(n, x1);
    if (f0 == 0.0L) {
      roots[found++] = x0;
    } else if ((f0 < 0) != (f1 < 0) && f1 != 0.0L) {
      long double lo = x0, hi = x1, flo = f0;
      for (int it = 0; it < 200; ++it) {
        long double mid = 0.5L * (lo + hi), fm = poly(n, mid);
        if (mid == lo || mid == hi) break;
        if ((fm < 0) == (flo < 0)) {
          lo = mid;
          flo = fm;
        } else {
          hi = mid;
        }
      }
      roots[found++] = 0.5L * (lo + hi);
    }
    x0 = x1;
    f0 = f1;
  }
  return found;
}

/* Legendre roots by Newton from the classical cosine guesses, in long double. */
static int legendre_roots(int n, long double *x) {
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int k = 0; k < n; ++k) {
    /* k-th root counted from -1 upward */
    long double z = -cosl(pi * (k + 0.75L) / (n + 0.5L));
    for (int it = 0; it < 100; ++it) {
      long double p = legendre_P(n, z), pm = legendre_P(n - 1, z);
      long double dp = n * (z * p - pm) / (z * z - 1.0L);
      long double dz = p / dp;
      z -= dz;
      if (fabsl(dz) <= 1e-21L * (1.0L + fabsl(z))) break;
    }
    x[k] = z;
  }
  /* the roots must come out distinct and increasing inside (-1, 1) */
  for (int k = 0; k < n; ++k) {
    if (!(x[k] > -1.0L && x[k] < 1.0L)) return ORC_EINVAL;
    if (k > 0 && !(x[k] > x[k - 1])) return ORC_EINVAL;
  }
  return ORC_OK;
}

/*
 * Nodes and weights. Polar: xi_j are the zeros of P_Qxi, w^xi_j = 2(1 - xi_j^2) / ((Qxi+1)^2 P_{Qxi+1}(xi_j)^2)
 * (Eq. polarInt, read with 1 - xi_j^2). Radial: pbar_i are the zeros of L^(1)_Qp,
 * w^p_i = pbar_i / ((Qp+1) L^(1)_{Qp+1}(pbar_i)^2) (radial rule after Eq. polarInt). Both ascending.
 */
int orc_quadrature(int Qp, int Qxi, double *pbar, double *wp, double *xi, double *wxi) {
  if (Qp < 1 || Qp > 16 || Qxi < 1 || Qxi > 1024) return ORC_EINVAL;
  long double *r = (long double *)malloc(sizeof(long double) * (Qp > Qxi ? Qp : Qxi));
  if (!r) return ORC_ENOMEM;
  /* all zeros of L^(1)_n lie in (0, 4n + 4) */
  int got = bracket_roots(laguerre1_L, Qp, 0.0L, 4.0L * Qp + 4.0L, 200000L, r);
  if (got != Qp) {
    free(r);
    return ORC_EINVAL;
  }
  for (int i = 0; i < Qp; ++i) {
    long double l = laguerre1_L(Qp + 1, r[i]);
    pbar[i] = (double)r[i];
    wp[i] = (double)(r[i] / ((Qp + 1) * l * l));
  }
  if (legendre_roots(Qxi, r) != ORC_OK) {
    free(r);
    return ORC_EINVAL;
  }
  for (int j = 0; j < Qxi; ++j) {
    long double p = legendre_P(Qxi + 1, r[j]);
    xi[j] = (double)r[j];
    wxi[j] = (double)(2.0L * (1.0L - r[j] * r[j]) / ((long double)(Qxi + 1) * (Qxi + 1) * p * p));
  }
  free(r);
  return ORC_OK;
}

/* ------------------------------------------------------------------------------------------------ */
/* Moments and the Landau frame, section "Relativistic lattice Boltzmann equation".                  */
/* ------------------------------------------------------------------------------------------------ */

/* N^mu = int d^3p/p^0 p^mu f and T^{mu nu} = int d^3p/p^0 p^mu p^nu f, as quadrature sums over F. */
void orc_moments_cell(int Qp, int Qxi, const double *pbar, const double *xi, const double *F, long stride,
                      double mom[5]) {
  double N0 = 0, Nz = 0, T00 = 0, T0z = 0, Tzz = 0;
  for (int i = 0; i < Qp; ++i)
    for (int j = 0; j < Qxi; ++j) {
      double f = F[(long)(i * Qxi + j) * stride];
      N0 += f * pbar[i];
      Nz += f * pbar[i] * xi[j];
      T00 += f * pbar[i] * pbar[i];
      T0z += f * pbar[i] * pbar[i] * xi[j];
      Tzz += f * pbar[i] * pbar[i] * xi[j] * xi[j];
    }
  mom[0] = N0;
  mom[1] = Nz;
  mom[2] = T00;
  mom[3] = T0z;
  mom[4] = Tzz;
}

/*
 * Landau-Lifshitz frame: T^mu_nu u^nu = -e u^mu with signature (-,+,+,+). In the (t, z) block the mixed
 * tensor is [[-T00, T0z], [-T0z, Tzz]]; its eigenvalue -e with a timelike eigenvector gives
 *   e = ((T00 - Tzz) + sqrt((T00 + Tzz)^2 - 4 T0z^2)) / 2,  beta = u^z/u^0 = T0z / (Tzz + e).
 * Then gamma = (1 - beta^2)^(-1/2), the Landau density n = -u_mu N^mu = gamma (N0 - beta Nz),
 * P = e/3 and T = P/n (perfect fluid of massless particles, P = nT, e = 3P).
 * out = {e, beta, n, T}.
 */
int orc_landau(const double mom[5], double out[4]) {
  double N0 = mom[0], Nz = mom[1], T00 = mom[2], T0z = mom[3], Tzz = mom[4];
  double disc = (T00 + Tzz) * (T00 + Tzz) - 4.0 * T0z * T0z;
  if (!(disc >= 0.0)) return ORC_ENONPHYS;
  double e = 0.5 * ((T00 - Tzz) + sqrt(disc));
  if (!(e > 0.0)) return ORC_ENONPHYS;
  double beta = T0z / (Tzz + e);
  if (!(fabs(beta) < 1.0)) return ORC_ENONPHYS;
  double gamma = 1.0 / sqrt(1.0 - beta * beta);
  double n = gamma * (N0 - beta * Nz);
  if (!(n > 0.0)) return ORC_ENONPHYS;
  out[0] = e;
  out[1] = beta;
  out[2] = n;
  out[3] = e / (3.0 * n);
  return ORC_OK;
}

/* ------------------------------------------------------------------------------------------------ */
/* Truncated equilibrium, Eq. (feqtrunc) with Eq. (feqMJ).                                            */
/* ------------------------------------------------------------------------------------------------ */

/*
 * Legendre coefficient of h_m(xi) = (1 - beta xi)^(-m):
 *   hhat_{m,k} = (2k+1)/2 * int_{-1}^{1} P_k(xi) (1 - beta xi)^(-m) dxi.
 * Written out by expanding (1 - beta xi)^(-m) = sum_r C(m+r-1, r) beta^r xi^r and integrating each power
 * against P_k exactly: int xi^r P_k = 2^(k+1) r! ((r+k)/2)! / (((r-k)/2)! (r+k+1)!) for r >= k, r - k even,
 * zero otherwise. The terms of one parity class all have one sign, so the sum has no cancellation. The
 * sum stops once a term no longer changes it.
 */
double orc_hhat(int m, int k, double beta) {
  if (beta == 0.0) return k == 0 ? 1.0 : 0.0;
  /* r = k term: C(m+k-1, k) beta^k * 2^(k+1) (k!)^2 / (2k+1)! */
  long double binom = 1.0L;
  for (int q = 1; q <= k; ++q) binom = binom * (m + q - 1) / q;
  long double I = 2.0L;
  for (int q = 1; q <= k; ++q) I = I * 2.0L * q * q / ((2.0L * q) * (2.0L * q + 1.0L));
  long double bk = 1.0L;
  for (int q = 0; q < k; ++q) bk *= beta;
  long double term = binom * bk * I, sum = 0.0L;
  long double b2 = (long double)beta * beta;
  for (long r = k; r < 4000000L; r += 2) {
    long double prev = sum;
    sum += term;
    if (sum == prev && r > k + 8) break;
    /* ratio of the r+2 term to the r term */
    long double a = (r + k) / 2, b = (r - k) / 2;
    long double ratio = b2 * (m + r) * (m + r + 1) / ((r + 1.0L) * (r + 2.0L));
    ratio *= (r + 1.0L) * (r + 2.0L) * (a + 1.0L) / ((b + 1.0L) * (r + k + 2.0L) * (r + k + 3.0L));
    term *= ratio;
  }
  return (double)((2.0L * k + 1.0L) / 2.0L * sum);
}

/*
 * Radial projection, derived from the generating function of L^(1):
 *   exp(-pbar (Lambda - 1)) = sum_l (Lambda - 1)^l / Lambda^(l+2) L^(1)_l(pbar),  Lambda = gamma (1 - beta xi) / T,
 * i.e. with s = T / gamma and h = 1/(1 - beta xi):  A_l(xi) = sum_{q=0}^{l} C(l,q) (-1)^q s^(q+2) h^(q+2).
 * Eq. (feqtrunc) keeps l <= Np and, per Eq. (mom_feq), the angular projection of each A_l of degree <= Nv:
 *   Ahat_{l,k} = sum_q C(l,q) (-1)^q s^(q+2) hhat_{q+2,k}.
 * With f^eq = n/(8 pi T^3) exp(-pbar Lambda) the stored population is
 *   F^eq_ij = 2 pi w^p_i w^xi_j exp(pbar_i) f^eq_trunc = n/(4 T^3) w^p_i w^xi_j sum_l L^(1)_l(pbar_i) sum_k Ahat_{l,k} P_k(xi_j).
 */
int orc_feq_cell(int Qp, int Qxi, int Np, int Nv, const double *pbar, const double *wp, const double *xi,
                 const double *wxi, double n, double T, double beta, double *Feq, long stride) {
  if (Np < 0 || Np > 8 || Nv < 0 || Nv > 32) return ORC_EINVAL;
  if (!(fabs(beta) < 1.0) || !(T > 0.0) || !(n > 0.0)) return ORC_ENONPHYS;
  double gamma = 1.0 / sqrt(1.0 - beta * beta);
  double s = T / gamma;
  double hh[11][33];
  for (int m = 2; m <= Np + 2; ++m)
    for (int k = 0; k <= Nv; ++k) hh[m][k] = orc_hhat(m, k, beta);
  double Ah[9][33];
  for (int l = 0; l <= Np; ++l)
    for (int k = 0; k <= Nv; ++k) {
      double acc = 0.0, c = 1.0; /* c = C(l,q) (-1)^q */
      for (int q = 0; q <= l; ++q) {
        acc += c * pow(s, q + 2) * hh[q + 2][k];
        c = -c * (l - q) / (q + 1);
      }
      Ah[l][k] = acc;
    }
  double pref = n / (4.0 * T * T * T);
  for (int i = 0; i < Qp; ++i)
    for (int j = 0; j < Qxi; ++j) {
      double acc = 0.0;
      for (int l = 0; l <= Np; ++l) {
        double ang = 0.0;
        for (int k = 0; k <= Nv; ++k) ang += Ah[l][k] * orc_legendre_P(k, xi[j]);
        acc += orc_laguerre1_L(l, pbar[i]) * ang;
      }
      Feq[(long)(i * Qxi + j) * stride] = pref * wp[i] * wxi[j] * acc;
    }
  return ORC_OK;
}

/* ------------------------------------------------------------------------------------------------ */
/* Advection: fifth-order WENO (Jiang & Shu), section "Numerical results".                           */
/* ------------------------------------------------------------------------------------------------ */

/*
 * Reconstruction at the interface between v0 and vp1 from the upwind side (v_{-2} .. v_{+2} with the wind
 * blowing from v_{-2} toward v_{+2}): three third-order candidates, smoothness indicators with weights 13/12
 * and 1/4, linear weights 1/10, 6/10, 3/10 and alpha_k = d_k / (eps + beta_k)^2.
 */

/* Smoothness indicator beta_k of candidate stencil k (k = 0: v_{-2} v_{-1} v_0, 1: v_{-1} v_0 v_{+1},
 * 2: v_0 v_{+1} v_{+2}): the sum over l = 1, 2 of h^(2l-1) times the integral over the cell of v0 of the
 * squared l-th derivative of the stencil's quadratic, written out. */
static void weno5_indicators(double vm2, double vm1, double v0, double vp1, double vp2, double b[3]) {
  b[0] = 13.0 / 12.0 * (vm2 - 2.0 * vm1 + v0) * (vm2 - 2.0 * vm1 + v0) +
         0.25 * (vm2 - 4.0 * vm1 + 3.0 * v0) * (vm2 - 4.0 * vm1 + 3.0 * v0);
  b[1] = 13.0 / 12.0 * (vm1 - 2.0 * v0 + vp1) * (vm1 - 2.0 * v0 + vp1) + 0.25 * (vm1 - vp1) * (vm1 - vp1);
  b[2] = 13.0 / 12.0 * (v0 - 2.0 * vp1 + vp2) * (v0 - 2.0 * vp1 + vp2) +
         0.25 * (3.0 * v0 - 4.0 * vp1 + vp2) * (3.0 * v0 - 4.0 * vp1 + vp2);
}

static double weno5_eps(double eps, double vm2, double vm1, double v0, double vp1, double vp2) {
  double q0 = (2.0 * vm2 - 7.0 * vm1 + 11.0 * v0) / 6.0;
  double q1 = (-vm1 + 5.0 * v0 + 2.0 * vp1) / 6.0;
  double q2 = (2.0 * v0 + 5.0 * vp1 - vp2) / 6.0;
  double b[3];
  weno5_indicators(vm2, vm1, v0, vp1, vp2, b);
  double a0 = 0.1 / ((eps + b[0]) * (eps + b[0]));
  double a1 = 0.6 / ((eps + b[1]) * (eps + b[1]));
  double a2 = 0.3 / ((eps + b[2]) * (eps + b[2]));
  return (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2);
}

/* The three smoothness indicators alone, for tests. */
void orc_weno5_indicators(double vm2, double vm1, double v0, double vp1, double vp2, double *out) {
  weno5_indicators(vm2, vm1, v0, vp1, vp2, out);
}

/* The textbook scheme on O(1) data: eps = 1e-6. */
double orc_weno5(double vm2, double vm1, double v0, double vp1, double vp2) {
  return weno5_eps(WENO_EPS, vm2, vm1, v0, vp1, vp2);
}

/* WENO5 on the population F_s of radial node i, direction j: the scheme applied to g_s = F_s / ws,
 * ws = w^p_i w^xi_j / 2, then scaled back, which is the scheme on F_s with eps ws^2. */
double orc_weno5_population(double ws, double vm2, double vm1, double v0, double vp1, double vp2) {
  return weno5_eps(WENO_EPS * ws * ws, vm2, vm1, v0, vp1, vp2);
}

/* ------------------------------------------------------------------------------------------------ */
/* The time step: Eq. (Boltz) discretised with WENO5 in space and SSP-RK3 in time.                    */
/* ------------------------------------------------------------------------------------------------ */

typedef struct {
  int Qp, Qxi, Np, Nv;
  int Nx;
  double dx, dt, tau; /* tau <= 0 or infinite: ballistic (no collision) */
  int bc;
} orc_params;

typedef struct {
  orc_params p;
  int Q;
  double pbar[16], wp[16];
  double *xi, *wxi;
  double *ext;  /* [Q][Nx+6]: one stage input with three ghost cells per side */
  double *flux; /* [Nx+1] */
  double *feq;  /* [Q] */
} orc_work;

static int work_open(orc_work *w, const orc_params *p) {
  memset(w, 0, sizeof(*w));
  if (p->Qp < 1 || p->Qp > 16 || p->Qxi < 1 || p->Qxi > 1024 || p->Nx < 1) return ORC_EINVAL;
  if (p->Np < 0 || p->Np >= p->Qp || p->Nv < 0 || p->Nv > 32) return ORC_EINVAL;
  if (!(p->dx > 0) || !(p->dt >= 0)) return ORC_EINVAL;
  if (p->bc != ORC_BC_OPEN && p->bc != ORC_BC_PERIODIC) return ORC_EINVAL;
  w->p = *p;
  w->Q = p->Qp * p->Qxi;
  w->xi = (double *)malloc(sizeof(double) * p->Qxi);
  w->wxi = (double *)malloc(sizeof(double) * p->Qxi);
  w->ext = (double *)malloc(sizeof(double) * (size_t)w->Q * (p->Nx + 6));
  w->flux = (double *)malloc(sizeof(double) * (p->Nx + 1));
  w->feq = (double *)malloc(sizeof(double) * w->Q);
  if (!w->xi || !w->wxi || !w->ext || !w->flux || !w->feq) return ORC_ENOMEM;
  return orc_quadrature(p->Qp, p->Qxi, w->pbar, w->wp, w->xi, w->wxi);
}

static void work_close(orc_work *w) {
  free(w->xi);
  free(w->wxi);
  free(w->ext);
  free(w->flux);
  free(w->feq);
}

static int ballistic(const orc_params *p) { return !(p->tau > 0.0) || isinf(p->tau); }

/* Copy the interior of G ([Q][Nx]) into ext and fill the ghosts: zero-gradient (open) or periodic. */
static void fill_ghosts(orc_work *w, const double *G) {
  int Nx = w->p.Nx, L = Nx + 6;
  for (int s = 0; s < w->Q; ++s) {
    double *e = w->ext + (size_t)s * L;
    const double *g = G + (size_t)s * Nx;
    for (int x = 0; x < Nx; ++x) e[x + 3] = g[x];
    for (int k = 1; k <= 3; ++k) {
      if (w->p.bc == ORC_BC_OPEN) {
        e[3 - k] = g[0];
        e[Nx + 2 + k] = g[Nx - 1];
      } else {
        e[3 - k] = g[((-k) % Nx + Nx) % Nx];
        e[Nx + 2 + k] = g[(k - 1) % Nx];
      }
    }
  }
}

/* L(G) = -xi_j dG/dx - (gamma (1 - beta xi_j) / tau) (G - G^eq), the right-hand side of Eq. (Boltz). */
static int rhs(orc_work *w, const double *G, double *L) {
  const orc_params *p = &w->p;
  int Nx = p->Nx, Lx = Nx + 6;
  fill_ghosts(w, G);
  /* advection, velocity by velocity, in conservative flux-difference form */
  for (int i = 0; i < p->Qp; ++i)
    for (int j = 0; j < p->Qxi; ++j) {
      int s = i * p->Qxi + j;
      const double *e = w->ext + (size_t)s * Lx; /* e[x + 3] = G[s][x] */
      double xi = w->xi[j];
      double ws = 0.5 * w->wp[i] * w->wxi[j];
      /* flux[x+1] is the reconstruction at the interface x + 1/2, x = -1 .. Nx-1 */
      for (int x = -1; x < Nx; ++x) {
        const double *c = e + x + 3;
        double phi;
        if (xi > 0.0)
          phi = orc_weno5_population(ws, c[-2], c[-1], c[0], c[1], c[2]);
        else if (xi < 0.0)
          phi = orc_weno5_population(ws, c[3], c[2], c[1], c[0], c[-1]);
        else
          phi = 0.0;
        w->flux[x + 1] = phi;
      }
      for (int x = 0; x < Nx; ++x) L[(size_t)s * Nx + x] = -xi * (w->flux[x + 1] - w->flux[x]) / p->dx;
    }
  if (ballistic(p)) return ORC_OK;
  /* Anderson-Witting collision with this stage's own moments */
  for (int x = 0; x < Nx; ++x) {
    double mom[5], lan[4];
    orc_moments_cell(p->Qp, p->Qxi, w->pbar, w->xi, G + x, Nx, mom);
    int st = orc_landau(mom, lan);
    if (st != ORC_OK) return st;
    double e = lan[0], beta = lan[1], n = lan[2], T = lan[3];
    (void)e;
    st = orc_feq_cell(p->Qp, p->Qxi, p->Np, p->Nv, w->pbar, w->wp, w->xi, w->wxi, n, T, beta, w->feq, 1);
    if (st != ORC_OK) return st;
    double gamma = 1.0 / sqrt(1.0 - beta * beta);
    for (int i = 0; i < p->Qp; ++i)
      for (int j = 0; j < p->Qxi; ++j) {
        int s = i * p->Qxi + j;
        double rate = gamma * (1.0 - beta * w->xi[j]) / p->tau;
        L[(size_t)s * Nx + x] -= rate * (G[(size_t)s * Nx + x] - w->feq[s]);
      }
  }
  return ORC_OK;
}

/* The right-hand side alone, for tests. F and L are [Q][Nx]. */
int orc_rhs(const orc_params *p, const double *F, double *L) {
  orc_work w;
  int st = work_open(&w, p);
  if (st == ORC_OK) st = rhs(&w, F, L);
  work_close(&w);
  return st;
}

/*
 * nsteps steps of SSP-RK3 in Shu-Osher form on F ([Q][Nx], in place):
 *   F1 = F + dt L(F);  F2 = 3/4 F + 1/4 (F1 + dt L(F1));  F_new = 1/3 F + 2/3 (F2 + dt L(F2)).
 */
int orc_step(const orc_params *p, double *F, long nsteps) {
  orc_work w;
  int st = work_open(&w, p);
  size_t n = (size_t)w.Q * p->Nx;
  double *F1 = NULL, *F2 = NULL, *L = NULL;
  if (st == ORC_OK) {
    F1 = (double *)malloc(sizeof(double) * n);
    F2 = (double *)malloc(sizeof(double) * n);
    L = (double *)malloc(sizeof(double) * n);
    if (!F1 || !F2 || !L) st = ORC_ENOMEM;
  }
  double dt = p->dt;
  for (long t = 0; t < nsteps && st == ORC_OK; ++t) {
    st = rhs(&w, F, L);
    if (st != ORC_OK) break;
    for (size_t k = 0; k < n; ++k) F1[k] = F[k] + dt * L[k];
    st = rhs(&w, F1, L);
    if (st != ORC_OK) break;
    for (size_t k = 0; k < n; ++k) F2[k] = 0.75 * F[k] + 0.25 * (F1[k] + dt * L[k]);
    st = rhs(&w, F2, L);
    if (st != ORC_OK) break;
    for (size_t k = 0; k < n; ++k) F[k] = F[k] / 3.0 + 2.0 / 3.0 * (F2[k] + dt * L[k]);
  }
  free(F1);
  free(F2);
  free(L);
  work_close(&w);
  return st;
}

/*
 * Initial condition, Eq. (condinit): F = F^eq(n, T = P/n, beta) cell by cell from per-cell pressure P,
 * density n and velocity beta.
 */
int orc_init(const orc_params *p, const double *P, const double *nd, const double *v, double *F) {
  orc_work w;
  int st = work_open(&w, p);
  for (int x = 0; x < p->Nx && st == ORC_OK; ++x) {
    if (!(P[x] > 0) || !(nd[x] > 0)) {
      st = ORC_ENONPHYS;
      break;
    }
    st = orc_feq_cell(p->Qp, p->Qxi, p->Np, p->Nv, w.pbar, w.wp, w.xi, w.wxi, nd[x], P[x] / nd[x], v[x], F + x,
                      p->Nx);
  }
  work_close(&w);
  return st;
}

/* Macroscopic fields per cell: out[f][x] for f = N0, Nz, T00, T0z, Tzz, e, beta, n (Landau). */
int orc_fields(const orc_params *p, const double *F, double *out) {
  orc_work w;
  int st = work_open(&w, p);
  int Nx = p->Nx;
  for (int x = 0; x < Nx && st == ORC_OK; ++x) {
    double mom[5], lan[4];
    orc_moments_cell(p->Qp, p->Qxi, w.pbar, w.xi, F + x, Nx, mom);
    for (int f = 0; f < 5; ++f) out[(size_t)f * Nx + x] = mom[f];
    st = orc_landau(mom, lan);
    if (st != ORC_OK) break;
    out[(size_t)5 * Nx + x] = lan[0];
    out[(size_t)6 * Nx + x] = lan[1];
    out[(size_t)7 * Nx + x] = lan[2];
  }
  work_close(&w);
  return st;
}

/*
 * Riemann initial condition, Eq. (condinit), on cell centres x_c = xleft + (c + 1/2) dx: the left state for
 * x_c < 0, the right state for x_c > 0 and, for a centre exactly on the membrane (odd Nx on a symmetric
 * domain), the mean of the two equilibria. st = {P_L, n_L, v_L, P_R, n_R, v_R}.
 */
int orc_init_riemann(const orc_params *p, double xleft, const double st[6], double *F) {
  orc_work w;
  int rc = work_open(&w, p);
  double *FL = NULL, *FR = NULL;
  if (rc == ORC_OK) {
    FL = (double *)malloc(sizeof(double) * w.Q);
    FR = (double *)malloc(sizeof(double) * w.Q);
    if (!FL || !FR) rc = ORC_ENOMEM;
  }
  if (rc == ORC_OK && (!(st[0] > 0) || !(st[1] > 0) || !(st[3] > 0) || !(st[4] > 0))) rc = ORC_ENONPHYS;
  if (rc == ORC_OK)
    rc = orc_feq_cell(p->Qp, p->Qxi, p->Np, p->Nv, w.pbar, w.wp, w.xi, w.wxi, st[1], st[0] / st[1], st[2], FL, 1);
  if (rc == ORC_OK)
    rc = orc_feq_cell(p->Qp, p->Qxi, p->Np, p->Nv, w.pbar, w.wp, w.xi, w.wxi, st[4], st[3] / st[4], st[5], FR, 1);
  for (int x = 0; x < p->Nx && rc == ORC_OK; ++x) {
    double xc = xleft + (x + 0.5) * p->dx;
    for (int s = 0; s < w.Q; ++s)
      F[(size_t)s * p->Nx + x] = xc < 0.0 ? FL[s] : (xc > 0.0 ? FR[s] : 0.5 * (FL[s] + FR[s]));
  }
  free(FL);
  free(FR);
  work_close(&w);
  return rc;
}
