// Adjoint (reverse mode) of the FP64 stage kernel, and of the initial equilibrium. Included by rlb.cu inside
// its anonymous namespace, after the forward kernels (it uses their helpers and series tables).
//
// One forward stage maps F_in to F_out = a F^n + b (F_in + dt L(F_in)) with
//   L_s(x) = -(xi_j/dx) (Phi_s(x+1/2) - Phi_s(x-1/2)) + r_s(x) (F^eq_s(x) - F_s(x)),  r_s = gamma (1 - beta xi_j)/tau
// (Eq. (Boltz) with WENO5 interface values Phi and the Anderson-Witting collision; F^eq from Eq. (feqtrunc)
// with n, T, beta from the Landau frame of the moments of F_in). Given mu = dL/dF_out, the adjoint stage
// produces b (mu + dt J^T mu) for F_in, a mu for F^n and b dt sum mu dL/dlog(tau) for the relaxation time:
//   advection: psi_X = (xi/dx)(mu(X) - mu(X-1)) for the interface X between cells X-1 and X, and
//              (J^T mu)(y) += sum_X psi_X dPhi_X/dF(y) over the five-cell stencils that contain y (ghost
//              cells of the open boundary pass their share to the edge cell, periodic ones wrap);
//   collision: -r_s mu_s, plus sum_a c_a(s) gM_a with c = (pbar, pbar xi, pbar^2, pbar^2 xi, pbar^2 xi^2)
//              the moment weights and gM = d/dM [sum_s mu_s r_s (F^eq_s - F_s)] at fixed F, carried from
//              (n, T, beta) back through the Landau solve;
//   tau:       d/dlog(tau) of b dt r_s (F^eq_s - F_s) is -b dt r_s (F^eq_s - F_s).
// The equilibrium's parameter derivatives use B[i][k] = n w^p_i/4 sum_q K[i][q] T^(q-1) gamma^-(q+2)
// hhat_{q+2,k}(beta) and the derivative series d hhat_{m,k}/d beta = sum_r r C(m+r-1, r) beta^(r-1) I_{r,k}.
//
// An adjoint tile has TXA = 60 cells, so that the TXA + 4 interfaces whose stencils reach its cells fit
// the 64 lanes of a velocity group.

constexpr int TXA = GW - 4;    // cells per adjoint tile
constexpr int AWF = TXA + 8;   // staged F positions x0-4 .. x0+TXA+3
constexpr int AWU = TXA + 6;   // staged adjoint positions x0-3 .. x0+TXA+2

struct AdjArgs {
  const TubeDev* tubes;
  const int2* tiles;  // adjoint tiles (tube, first cell)
  const double* Fin;  // forward stage input (read with halo)
  const double* mu;   // adjoint of the stage output (read with halo)
  double* out;        // adjoint of the stage input (mode 2, 1), or of F^n (mode 0)
  double* acc;        // adjoint accumulated for F^n over the stages of one step
  const double* tab;
  int* flag;
  double* dlt;        // per-tile accumulators of dL/dlog(tau)
  double a, b;        // the forward stage's Shu-Osher coefficients
  int mode;           // 2: out = b(mu + dt J^T mu), acc = a mu; 1: the same with acc += a mu;
                      // 0: out = acc + b(mu + dt J^T mu)
  int split;          // CTAs per tile (<= 1: one): CTA k of a tile writes velocity rows
                      // [k Q / split, (k + 1) Q / split) after the per-cell reductions over all rows
};

// Legendre coefficients and their beta derivatives (m = 2 .. Np+2, k <= Nv) of the tile's cells
struct AdjCoef {
  double hh[M_MAX - 1][NV_MAX + 1][GW];
  double dh[M_MAX - 1][NV_MAX + 1][GW];
};

// One parity class of hhat_{m,k}(beta) and d hhat_{m,k}/d beta by the positive power series of the forward
// (same tables and summation order), continued until both series have converged.
template <int NPc, int NVc, int PAR>
__device__ bool hhat_parity_d(double beta, double* hh_col, double* dh_col) {
  constexpr int NK = (NVc - PAR) / 2 + 1;
  double acc[NPc + 1][NK], dac[NPc + 1][NK];
#pragma unroll
  for (int m = 0; m <= NPc; ++m)
#pragma unroll
    for (int q = 0; q < NK; ++q) acc[m][q] = dac[m][q] = 0.0;
  const double b2 = beta * beta;
  const double tol = 1e-18 * (1.0 - b2);
  double br = PAR ? beta : 1.0;  // beta^r
  double bm = 1.0;               // beta^(r-1), r >= 1
  bool done = false;
  for (int r = PAR; r <= R_MAX; r += 2) {
    const double* ic = g_ic + r * (NV_MAX + 1);
    const double rb = r == 0 ? 0.0 : r * bm;  // d beta^r / d beta
    double tlast = 0.0, dlast = 0.0;
#pragma unroll
    for (int m = 0; m <= NPc; ++m) {
      const double cb = g_cb[(m + 2) * (R_MAX + 1) + r];
      const double t = cb * br, d = cb * rb;
#pragma unroll
      for (int q = 0; q < NK; ++q) {
        acc[m][q] = fma(ic[PAR + 2 * q], t, acc[m][q]);
        dac[m][q] = fma(ic[PAR + 2 * q], d, dac[m][q]);
      }
      tlast = t;
      dlast = d;
    }
    if (r >= NVc && fabs(tlast) < tol && fabs(dlast) < tol) {
      done = true;
      break;
    }
    br *= b2;
    bm = r == 0 ? beta : bm * b2;
  }
#pragma unroll
  for (int m = 0; m <= NPc; ++m)
#pragma unroll
    for (int q = 0; q < NK; ++q) {
      hh_col[((m * (NV_MAX + 1)) + PAR + 2 * q) * GW] = acc[m][q];
      dh_col[((m * (NV_MAX + 1)) + PAR + 2 * q) * GW] = dac[m][q];
    }
  return done;
}

// hhat and d hhat/d beta of the tile's cells (groups 0/1: even/odd k); cells with ok == 0 keep zeros.
// With Bs != nullptr, group i then builds the equilibrium coefficients B[i][k] as the forward does.
// Ends with a barrier.
template <int NPc, int NVc>
__device__ void tile_coeffs_d(const double* tab, int Qp, const double* cellv /* n, T, beta: [3][GW] */,
                              int* ok, AdjCoef& co, double (*Bs)[GW], int* flag) {
  const int c = threadIdx.x % GW, g = threadIdx.x / GW;
  if (g < 2 && c < TXA) {
    bool conv = true;
    if (ok[c]) {
      const double beta = cellv[2 * GW + c];
      if (g == 0)
        conv = hhat_parity_d<NPc, NVc, 0>(beta, &co.hh[0][0][c], &co.dh[0][0][c]);
      else
        conv = hhat_parity_d<NPc, NVc, 1>(beta, &co.hh[0][0][c], &co.dh[0][0][c]);
    } else {
#pragma unroll
      for (int m = 0; m <= NPc; ++m)
        for (int k = g; k <= NVc; k += 2) co.hh[m][k][c] = co.dh[m][k][c] = 0.0;
    }
    if (!conv) {
      ok[c] = 0;
      atomicOr(flag, 1);
    }
  }
  __syncthreads();
  if (Bs != nullptr && c < TXA) {
    const int i = g;
    double B[NVc + 1];
#pragma unroll
    for (int k = 0; k <= NVc; ++k) B[k] = 0.0;
    if (i < Qp && ok[c]) {
      const double n = cellv[c], T = cellv[GW + c], beta = cellv[2 * GW + c];
      const double s = T * sqrt(1.0 - beta * beta);
      const double pref = n / (4.0 * T * T * T) * tab[TAB_WP + i];
      double sq = s * s;
#pragma unroll
      for (int q = 0; q <= NPc; ++q) {
        const double G = pref * sq * tab[TAB_K + i * (NP_MAX + 1) + q];
#pragma unroll
        for (int k = 0; k <= NVc; ++k) B[k] = fma(G, co.hh[q][k][c], B[k]);
        sq *= s;
      }
    }
    if (i < QP_MAX) {
#pragma unroll
      for (int k = 0; k <= NVc; ++k) Bs[i * (NV_MAX + 1) + k][c] = B[k];
    }
  }
  __syncthreads();
}

// Derivatives of sum_{i,k} B[i][k](n, T, beta) Lam[i][k] with respect to n, T and beta at one cell.
template <int NPc, int NVc>
__device__ void eq_param_grads(const double* tab, int Qp, double n, double T, double beta, const AdjCoef& co,
                               int c, const double (*Lam)[GW] /* [i (NV_MAX+1) + k][GW] */, double& gn,
                               double& gT, double& gb) {
  const double g2 = 1.0 / (1.0 - beta * beta);  // gamma^2
  const double ig = sqrt(1.0 - beta * beta);    // 1/gamma
  double uq = ig * ig / T;                      // T^(q-1) gamma^-(q+2) at q = 0
  double an = 0.0, aT = 0.0, ab = 0.0;
#pragma unroll
  for (int q = 0; q <= NPc; ++q) {
    double sn = 0.0, sb = 0.0;
#pragma unroll
    for (int k = 0; k <= NVc; ++k) {
      double H = 0.0;  // sum_i w_i K[i][q] Lam[i][k]
      for (int i = 0; i < Qp; ++i)
        H = fma(tab[TAB_WP + i] * tab[TAB_K + i * (NP_MAX + 1) + q], Lam[i * (NV_MAX + 1) + k][c], H);
      const double hq = co.hh[q][k][c], dq = co.dh[q][k][c];
      sn = fma(hq, H, sn);
      sb = fma(fma(-(q + 2) * beta * g2, hq, dq), H, sb);
    }
    an = fma(uq, sn, an);
    aT = fma((q - 1) * uq, sn, aT);
    ab = fma(uq, sb, ab);
    uq *= T * ig;
  }
  const double q4 = 0.25 * n;
  gn = 0.25 * an;
  gT = q4 * aT / T;
  gb = q4 * ab;
}

// Landau solve backwards: adjoints (gn, gT, gbeta) of n, T, beta to the adjoints of the five moments.
__device__ __forceinline__ void landau_reverse(const double mom[5], double e, double beta, double n, double T,
                                               double gn, double gT, double gb, double gM[5]) {
  const double gam = 1.0 / sqrt(1.0 - beta * beta);
  // T = e / (3n)
  double ge = gT / (3.0 * n);
  gn -= gT * T / n;
  // n = gamma (N0 - beta Nx)
  gM[0] = gn * gam;
  gM[1] = -gn * gam * beta;
  gb += gn * (gam * gam * beta * n - gam * mom[1]);
  // beta = T0x / (Txx + e)
  const double den = mom[4] + e;
  gM[3] = gb / den;
  gM[4] = -gb * beta / den;
  ge -= gb * beta / den;
  // e = ((T00 - Txx) + sqrt((T00 + Txx)^2 - 4 T0x^2)) / 2
  const double A = mom[2] + mom[4];
  const double sq = sqrt(A * A - 4.0 * mom[3] * mom[3]);
  gM[2] = 0.5 * ge * (1.0 + A / sq);
  gM[4] += 0.5 * ge * (A / sq - 1.0);
  gM[3] -= 2.0 * ge * mom[3] / sq;
}

struct AdjSmem {
  union {
    double red[NG][5][GW];  // A: partial moments
    AdjCoef co;             // B .. B2: hhat and its beta derivative
  } u;
  double B[NBC][GW];        // equilibrium coefficients of the cells
  union {
    struct {
      double lam[NBC][GW];  // Lam[i][k] = sum_j mu_ij r_ij w^xi_j P_k(xi_j) (radial row i summed by group i)
      double s01[NG][2][GW];  // partial S0 = sum mu (F^eq - F), S1 = sum mu xi (F^eq - F)
    } r;
    struct {
      double frow[2][NG][AWF + 1];  // staged F rows
      double urow[2][NG][AWU + 1];  // staged adjoint rows
      double P[NG][5][GW];          // psi_X dPhi_X/dF at the five stencil slots (memory order) of interface X
    } c;
  } v;
  double cellv[3][GW];  // n, T, beta
  double mom[5][GW];
  double ee[GW];        // e
  double r0[GW];        // gamma / tau (0: no collision at this cell)
  double gM[5][GW];     // adjoint of the five moments
  double dl[GW];        // per-cell share of dL/dlog(tau)
  int ok[GW];
  int srcF[AWF + 1];    // source cell of each staged F position
  int srcU[AWU + 1];    // source cell of each staged adjoint position, -1: outside the tube (zero)
};

__device__ __forceinline__ int wrap_cell(int p, int Nx) {
  const int r = p % Nx;
  return r < 0 ? r + Nx : r;
}

// Partial derivatives dPhi/dv_m (m = 0..4, wind order, v2 the upwind cell) of the WENO5 interface value
// Phi = sum_k w_k q_k, w_k = alpha_k / sum alpha, alpha_k = d_k / (eps + beta_k)^2:
//   dPhi/dv = sum_k w_k dq_k/dv + sum_k kappa_k dbeta_k/dv,  kappa_k = -2 w_k (q_k - Phi) / (eps + beta_k).
__device__ void weno5_grad(const double v[5], double eps, double dP[5]) {
  constexpr double S6 = 1.0 / 6.0;
  const double q0 = (2.0 * v[0] - 7.0 * v[1] + 11.0 * v[2]) * S6;
  const double q1 = (-v[1] + 5.0 * v[2] + 2.0 * v[3]) * S6;
  const double q2 = (2.0 * v[2] + 5.0 * v[3] - v[4]) * S6;
  const double a0 = v[0] - 2.0 * v[1] + v[2], b0 = v[0] - 4.0 * v[1] + 3.0 * v[2];
  const double a1 = v[1] - 2.0 * v[2] + v[3], b1 = v[1] - v[3];
  const double a2 = v[2] - 2.0 * v[3] + v[4], b2 = 3.0 * v[2] - 4.0 * v[3] + v[4];
  const double e0 = eps + (13.0 / 12.0 * a0 * a0 + 0.25 * b0 * b0);
  const double e1 = eps + (13.0 / 12.0 * a1 * a1 + 0.25 * b1 * b1);
  const double e2 = eps + (13.0 / 12.0 * a2 * a2 + 0.25 * b2 * b2);
  // alpha_k and the normalised weights, with the refined hardware reciprocal of the forward kernel
  const double i0 = rlbdev::rcp_nr(e0), i1 = rlbdev::rcp_nr(e1), i2 = rlbdev::rcp_nr(e2);
  const double s0 = 0.1 * i0 * i0, s1 = 0.6 * i1 * i1, s2 = 0.3 * i2 * i2;
  const double is = rlbdev::rcp_nr(s0 + s1 + s2);
  const double w0 = s0 * is, w1 = s1 * is, w2 = s2 * is;
  const double Phi = w0 * q0 + w1 * q1 + w2 * q2;
  const double k0 = -2.0 * w0 * (q0 - Phi) * i0;
  const double k1 = -2.0 * w1 * (q1 - Phi) * i1;
  const double k2 = -2.0 * w2 * (q2 - Phi) * i2;
  // dbeta_k/dv = 13/6 a_k da_k/dv + 1/2 b_k db_k/dv
  const double A0 = 13.0 / 6.0 * k0 * a0, B0 = 0.5 * k0 * b0;
  const double A1 = 13.0 / 6.0 * k1 * a1, B1 = 0.5 * k1 * b1;
  const double A2 = 13.0 / 6.0 * k2 * a2, B2 = 0.5 * k2 * b2;
  dP[0] = w0 * (2.0 / 6.0) + A0 + B0;
  dP[1] = w0 * (-7.0 / 6.0) + w1 * (-1.0 / 6.0) - 2.0 * A0 - 4.0 * B0 + A1 + B1;
  dP[2] = w0 * (11.0 / 6.0) + w1 * (5.0 / 6.0) + w2 * (2.0 / 6.0) + A0 + 3.0 * B0 - 2.0 * A1 + A2 + 3.0 * B2;
  dP[3] = w1 * (2.0 / 6.0) + w2 * (5.0 / 6.0) + A1 - B1 - 2.0 * A2 - 4.0 * B2;
  dP[4] = w2 * (-1.0 / 6.0) + A2 + B2;
}

template <int NPc, int NVc>
__device__ void adjoint_tile(const AdjArgs& A, const TubeDev& T, int tile, int x0, int part, int nparts,
                             AdjSmem& sm) {
  const int tid = threadIdx.x, c = tid % GW, g = tid / GW;
  const double* tab = A.tab + T.tab;
  const int Qp = T.Qp, Qxi = T.Qxi, Q = Qp * Qxi, Nx = T.Nx, ld = T.ld;
  const double* Fin = A.Fin + T.off;
  const double* mu = A.mu + T.off;
  double* out = A.out + T.off;
  double* acc = A.acc + T.off;
  const int x = x0 + c;
  const bool cell = (c < TXA) && (x < Nx);
  const bool periodic = T.bc == RLB_BC_PERIODIC;
  for (int k = tid; k < AWF; k += NT) {
    const int p = x0 - 4 + k;
    sm.srcF[k] = periodic ? wrap_cell(p, Nx) : min(max(p, 0), Nx - 1);
  }
  for (int k = tid; k < AWU; k += NT) {
    const int p = x0 - 3 + k;
    sm.srcU[k] = periodic ? wrap_cell(p, Nx) : ((p >= 0 && p < Nx) ? p : -1);
  }
  if (g == 0) {
#pragma unroll
    for (int f = 0; f < 5; ++f) sm.gM[f][c] = 0.0;
    sm.r0[c] = 0.0;
    sm.dl[c] = 0.0;
    sm.cellv[2][c] = 0.0;
  }
  if (T.collide) {
    // A. moments of the forward stage input (as the forward kernel sums them)
    double m0 = 0, m1 = 0, m2 = 0, m3 = 0, m4 = 0;
    if (cell) {
      for (int j = g; j < Qxi; j += NG) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < Qp; ++i) {
          const double f = __ldg(Fin + (size_t)(i * Qxi + j) * ld + x);
          a = fma(f, tab[TAB_PBAR + i], a);
          b = fma(f, tab[TAB_PBAR2 + i], b);
        }
        const double xi = tab[TAB_XI + j];
        m0 += a;
        m1 = fma(a, xi, m1);
        m2 += b;
        m3 = fma(b, xi, m3);
        m4 = fma(b * xi, xi, m4);
      }
    }
    sm.u.red[g][0][c] = m0;
    sm.u.red[g][1][c] = m1;
    sm.u.red[g][2][c] = m2;
    sm.u.red[g][3][c] = m3;
    sm.u.red[g][4][c] = m4;
    __syncthreads();
    // B. Landau frame, then hhat, d hhat/d beta and the equilibrium coefficients
    double mom[5] = {0, 0, 0, 0, 0}, e = 1.0, beta = 0.0, n = 1.0, Tt = 1.0;
    bool ok = false;
    if (g == 0 && cell) {
#pragma unroll
      for (int f = 0; f < 5; ++f) mom[f] = (sm.u.red[0][f][c] + sm.u.red[1][f][c]) + (sm.u.red[2][f][c] + sm.u.red[3][f][c]);
      ok = landau(mom, e, beta, n, Tt);
      if (!ok) atomicOr(A.flag, 1);
    }
    __syncthreads();  // the union now holds the coefficient scratch
    if (g == 0) {
      sm.cellv[0][c] = n;
      sm.cellv[1][c] = Tt;
      sm.cellv[2][c] = ok ? beta : 0.0;
#pragma unroll
      for (int f = 0; f < 5; ++f) sm.mom[f][c] = mom[f];
      sm.ee[c] = e;
      sm.ok[c] = ok ? 1 : 0;
      sm.r0[c] = ok ? T.inv_tau / sqrt(1.0 - beta * beta) : 0.0;
    }
    __syncthreads();
    tile_coeffs_d<NPc, NVc>(tab, Qp, &sm.cellv[0][0], sm.ok, sm.u.co, sm.B, A.flag);
    // R. per cell: Lam[i][k] (group i sums radial row i) and the partial sums S0, S1
    {
      double lam[NVc + 1], B[NVc + 1];
#pragma unroll
      for (int k = 0; k <= NVc; ++k) lam[k] = 0.0;
      double S0 = 0.0, S1 = 0.0;
      if (cell && g < Qp && sm.ok[c]) {
#pragma unroll
        for (int k = 0; k <= NVc; ++k) B[k] = sm.B[g * (NV_MAX + 1) + k][c];
        const double r0 = sm.r0[c], bt = sm.cellv[2][c];
        for (int j = 0; j < Qxi; ++j) {
          const size_t o = (size_t)(g * Qxi + j) * ld + x;
          const double m = __ldg(mu + o), f = __ldg(Fin + o);
          const double xi = tab[TAB_XI + j];
          const double* pw = tab + TAB_XI + Qxi + j * (NV_MAX + 1);
          double feq = 0.0;
#pragma unroll
          for (int k = 0; k <= NVc; ++k) feq = fma(B[k], pw[k], feq);
          const double d = m * (feq - f);
          S0 += d;
          S1 = fma(d, xi, S1);
          const double mr = m * r0 * fma(-bt, xi, 1.0);
#pragma unroll
          for (int k = 0; k <= NVc; ++k) lam[k] = fma(mr, pw[k], lam[k]);
        }
      }
      if (g < QP_MAX) {
#pragma unroll
        for (int k = 0; k <= NVc; ++k) sm.v.r.lam[g * (NV_MAX + 1) + k][c] = lam[k];
      }
      sm.v.r.s01[g][0][c] = S0;
      sm.v.r.s01[g][1][c] = S1;
    }
    __syncthreads();
    // B2. per cell: gradients of the collision term with respect to n, T, beta, then to the moments
    if (g == 0 && cell && sm.ok[c]) {
      const double n_ = sm.cellv[0][c], T_ = sm.cellv[1][c], b_ = sm.cellv[2][c], r0 = sm.r0[c];
      const double S0 = (sm.v.r.s01[0][0][c] + sm.v.r.s01[1][0][c]) + (sm.v.r.s01[2][0][c] + sm.v.r.s01[3][0][c]);
      const double S1 = (sm.v.r.s01[0][1][c] + sm.v.r.s01[1][1][c]) + (sm.v.r.s01[2][1][c] + sm.v.r.s01[3][1][c]);
      double gn, gT, gb;
      eq_param_grads<NPc, NVc>(tab, Qp, n_, T_, b_, sm.u.co, c, sm.v.r.lam, gn, gT, gb);
      // d r_s / d beta = gamma^3 (beta - xi_j) / tau = r0 gamma^2 (beta - xi_j)
      gb += r0 / (1.0 - b_ * b_) * (b_ * S0 - S1);
      double m5[5], gM[5];
#pragma unroll
      for (int f = 0; f < 5; ++f) m5[f] = sm.mom[f][c];
      landau_reverse(m5, sm.ee[c], b_, n_, T_, gn, gT, gb, gM);
#pragma unroll
      for (int f = 0; f < 5; ++f) sm.gM[f][c] = gM[f];
      sm.dl[c] = -A.b * T.dt * r0 * fma(-b_, S1, S0);
    }
  }
  __syncthreads();  // srcF/srcU, gM, r0 ready; the union is free for the row buffers
  if (tid == 0 && part == 0) {
    double s = 0.0;
    for (int k = 0; k < TXA; ++k) s += sm.dl[k];
    A.dlt[tile] += s;
  }

  // C. rows: transposed WENO5 flux differences, collision terms, Runge-Kutta combination
  const double a = A.a, b = A.b, dt = T.dt, inv_dx = 1.0 / T.dx;
  const double bt = sm.cellv[2][c], r0 = sm.r0[c];
  double* P0 = sm.v.c.P[g][0];
  int buf = 0;
  const int r_end = (part + 1) * Q / nparts;
  for (int s0 = part * Q / nparts; s0 < r_end; s0 += NG, buf ^= 1) {
    const int s = s0 + g;
    const bool rv = s < r_end;
    const int i = rv ? s / Qxi : 0, j = rv ? s - i * Qxi : 0;
    double* fr = sm.v.c.frow[buf][g];
    double* ur = sm.v.c.urow[buf][g];
    if (rv) {
      const double* fs = Fin + (size_t)s * ld;
      const double* us = mu + (size_t)s * ld;
      for (int k = c; k < AWF; k += GW) fr[k] = __ldg(fs + sm.srcF[k]);
      for (int k = c; k < AWU; k += GW) {
        const int q = sm.srcU[k];
        ur[k] = q >= 0 ? __ldg(us + q) : 0.0;
      }
    }
    group_sync(g);
    const double xi = tab[TAB_XI + j];
    const bool fwd = xi > 0.0;
    if (rv) {
      // lane c: interface X = x0 - 1 + c (wind toward +x) or x0 - 2 + c (toward -x); its stencil is staged at
      // fr[c .. c+4] in memory order and mu(X), mu(X-1) at ur[c+2], ur[c+1] (resp. ur[c+1], ur[c])
      const double psi = xi * inv_dx * (fwd ? ur[c + 2] - ur[c + 1] : ur[c + 1] - ur[c]);
      double v[5], dP[5];
#pragma unroll
      for (int m = 0; m < 5; ++m) v[m] = fwd ? fr[c + m] : fr[c + 4 - m];
      const double eps = tab[tab_eps(Qxi) + 3 * s] * (1.0 / (3.0 * rlbdev::C0));
      weno5_grad(v, eps, dP);
#pragma unroll
      for (int m = 0; m < 5; ++m) P0[(fwd ? m : 4 - m) * GW + c] = psi * dP[m];
    }
    group_sync(g);
    if (rv && cell) {
      // cell y = x0 + c gathers slot m of interface lane c + 4 - m; the open boundary's ghost positions
      // (copies of the edge cells) add theirs to the edge cells
      double w = 0.0;
#pragma unroll
      for (int m = 0; m < 5; ++m) w += P0[m * GW + c + 4 - m];
      if (!periodic && (x == 0 || x == Nx - 1)) {
        for (int side = 0; side < 2; ++side) {
          if ((side == 0 && x != 0) || (side == 1 && x != Nx - 1)) continue;
          for (int h = 1; h <= 3; ++h) {
            const int p = side == 0 ? -h : Nx - 1 + h;  // ghost position
#pragma unroll
            for (int m = 0; m < 5; ++m) {
              const int lane = p - x0 + 4 - m;
              if (lane >= 0 && lane < GW) w += P0[m * GW + lane];
            }
          }
        }
      }
      const double m_ = ur[c + 3];
      if (r0 != 0.0) {
        const double pb = tab[TAB_PBAR + i], pb2 = tab[TAB_PBAR2 + i];
        w = fma(-r0 * fma(-bt, xi, 1.0), m_, w);
        w = fma(pb, fma(xi, sm.gM[1][c], sm.gM[0][c]), w);
        w = fma(pb2, fma(xi, fma(xi, sm.gM[4][c], sm.gM[3][c]), sm.gM[2][c]), w);
      }
      const double val = b * fma(dt, w, m_);
      const size_t o = (size_t)s * ld + x;
      if (A.mode == 2) {
        out[o] = val;
        acc[o] = a * m_;
      } else if (A.mode == 1) {
        out[o] = val;
        acc[o] = fma(a, m_, acc[o]);
      } else {
        out[o] = acc[o] + val;
      }
    }
  }
}

__global__ void __launch_bounds__(NT) rlb_adjoint_kernel(AdjArgs A) {
  extern __shared__ __align__(16) unsigned char adj_smem_raw[];
  AdjSmem& sm = *reinterpret_cast<AdjSmem*>(adj_smem_raw);
  const int K = A.split > 1 ? A.split : 1;
  const int t = blockIdx.x / K, part = blockIdx.x - t * K;
  const int2 tl = A.tiles[t];
  const TubeDev T = A.tubes[tl.x];
  if (T.Np == 2 && T.Nv == 5)
    adjoint_tile<2, 5>(A, T, t, tl.y, part, K, sm);
  else
    adjoint_tile<NP_MAX, NV_MAX>(A, T, t, tl.y, part, K, sm);
}

// Seed of the state from the adjoint of the five moments of each cell: dL/dF_s = sum_a c_a(s) dL/dM_a.
// gM: [5][nxtot] (field layout); seed: packed state (rows of Nx cells, tube after tube).
__global__ void __launch_bounds__(NT) rlb_moments_vjp_kernel(const TubeDev* tubes, const int2* tiles,
                                                             const double* tabs, const double* gM,
                                                             long long nxtot, double* seed) {
  const int2 tl = tiles[blockIdx.x];
  const TubeDev T = tubes[tl.x];
  const int c = threadIdx.x % GW, g = threadIdx.x / GW, x = tl.y + c;
  if (c >= TXA || x >= T.Nx) return;
  const double* tab = tabs + T.tab;
  const double* gm = gM + T.xoff + x;
  const double g0 = gm[0], g1 = gm[nxtot], g2 = gm[2 * nxtot], g3 = gm[3 * nxtot], g4 = gm[4 * nxtot];
  for (int s = g; s < T.Qp * T.Qxi; s += NG) {
    const int i = s / T.Qxi, j = s - i * T.Qxi;
    const double xi = tab[TAB_XI + j];
    const double v = tab[TAB_PBAR + i] * fma(xi, g1, g0) + tab[TAB_PBAR2 + i] * fma(xi, fma(xi, g4, g3), g2);
    seed[T.poff + (size_t)s * T.Nx + x] = v;
  }
}

// Adjoint of the Landau frame (e, beta, n) with respect to the moments (N0, Nx, T00, T0x, Txx), for the closed
// form of landau(): with A = T00 + Txx, r = sqrt(A^2 - 4 T0x^2), e = (T00 - Txx + r) / 2, W = Txx + e,
// beta = T0x / W, gamma = (1 - beta^2)^-1/2, n = gamma (N0 - beta Nx). Adds ge de/dM + gb dbeta/dM + gn dn/dM to
// G[5]. Returns false for a non-physical cell (G unchanged).
__device__ bool landau_vjp(const double mom[5], double ge, double gb, double gn, double G[5]) {
  double e, beta, n, Tt;
  if (!landau(mom, e, beta, n, Tt)) return false;
  const double A = mom[2] + mom[4], B = mom[3];
  const double r = sqrt(A * A - 4.0 * B * B);
  if (!(r > 0.0)) return false;
  // de/d(T00, T0x, Txx)
  const double e00 = 0.5 * (1.0 + A / r), e0x = -2.0 * B / r, exx = 0.5 * (A / r - 1.0);
  const double W = mom[4] + e, bW = beta / W;  // beta / W = T0x / W^2
  // dbeta/d(T00, T0x, Txx)
  const double b00 = -bW * e00, b0x = 1.0 / W - bW * e0x, bxx = -bW * (1.0 + exx);
  const double g2 = 1.0 / (1.0 - beta * beta), gam = sqrt(g2);
  // dn/dbeta at fixed (N0, Nx); dn/dN0 = gamma, dn/dNx = -gamma beta
  const double nb = gam * (g2 * beta * (mom[0] - beta * mom[1]) - mom[1]);
  const double gbt = gb + gn * nb;  // total adjoint of beta
  G[0] += gn * gam;
  G[1] -= gn * gam * beta;
  G[2] += ge * e00 + gbt * b00;
  G[3] += ge * e0x + gbt * b0x;
  G[4] += ge * exx + gbt * bxx;
  return true;
}

// Seed of the state from the adjoint of the fields of rlb_moments: dL/dF_s = sum_a c_a(s) G_a, where G_a is
// dL/dM_a plus the share of dL/de, dL/dv and dL/dn carried through the Landau frame of the cell's moments.
// gf: [RLB_NFIELDS][nxtot] (field layout); F: the FP64 state (padded rows) the fields were taken at; seed:
// packed state. A non-physical cell raises the flag and seeds only its moments' share.
__global__ void __launch_bounds__(NT) rlb_fields_vjp_kernel(const TubeDev* tubes, const int2* tiles,
                                                            const double* tabs, const double* F, const double* gf,
                                                            long long nxtot, double* seed, int* flag) {
  __shared__ double Gs[5][GW];
  const int2 tl = tiles[blockIdx.x];
  const TubeDev T = tubes[tl.x];
  const int c = threadIdx.x % GW, g = threadIdx.x / GW, x = tl.y + c;
  const bool cell = c < TXA && x < T.Nx;
  const double* tab = tabs + T.tab;
  if (g == 0) {
    double G[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (cell) {
      const double* f = F + T.off + x;
      double mom[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
      for (int j = 0; j < T.Qxi; ++j) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < T.Qp; ++i) {
          const double v = f[(size_t)(i * T.Qxi + j) * T.ld];
          a = fma(v, tab[TAB_PBAR + i], a);
          b = fma(v, tab[TAB_PBAR2 + i], b);
        }
        const double xi = tab[TAB_XI + j];
        mom[0] += a;
        mom[1] = fma(a, xi, mom[1]);
        mom[2] += b;
        mom[3] = fma(b, xi, mom[3]);
        mom[4] = fma(b * xi, xi, mom[4]);
      }
      const double* gx = gf + T.xoff + x;
#pragma unroll
      for (int a = 0; a < 5; ++a) G[a] = gx[a * nxtot];
      if (!landau_vjp(mom, gx[RLB_F_E * nxtot], gx[RLB_F_V * nxtot], gx[RLB_F_N * nxtot], G)) atomicOr(flag, 1);
    }
#pragma unroll
    for (int a = 0; a < 5; ++a) Gs[a][c] = G[a];
  }
  __syncthreads();
  if (!cell) return;
  const double g0 = Gs[0][c], g1 = Gs[1][c], g2 = Gs[2][c], g3 = Gs[3][c], g4 = Gs[4][c];
  for (int s = g; s < T.Qp * T.Qxi; s += NG) {
    const int i = s / T.Qxi, j = s - i * T.Qxi;
    const double xi = tab[TAB_XI + j];
    const double v = tab[TAB_PBAR + i] * fma(xi, g1, g0) + tab[TAB_PBAR2 + i] * fma(xi, fma(xi, g4, g3), g2);
    seed[T.poff + (size_t)s * T.Nx + x] = v;
  }
}

struct InitVjpSmem {
  AdjCoef co;
  double lam[NBC][GW];
  double cellv[3][GW];  // n, T, beta of the initial state
  double P[GW];
  int ok[GW];
};

// Adjoint of the initial condition F = F^eq(n, T = P/n, beta = v): from dL/dF (packed) to dL/dP, dL/dn,
// dL/dv of each cell (field layout).
template <int NPc, int NVc>
__device__ void init_vjp_tile(const TubeDev& T, const double* tab, int x0, const double* P, const double* n,
                              const double* v, const double* gF, double* gP, double* gn, double* gv, int* flag,
                              InitVjpSmem& sm) {
  const int c = threadIdx.x % GW, g = threadIdx.x / GW, x = x0 + c;
  const bool cell = c < TXA && x < T.Nx;
  const size_t k = (size_t)T.xoff + x;
  if (g == 0) {
    const double P_ = cell ? P[k] : 1.0, n_ = cell ? n[k] : 1.0, v_ = cell ? v[k] : 0.0;
    const bool ok = cell && P_ > 0.0 && n_ > 0.0 && fabs(v_) < 1.0;
    if (cell && !ok) atomicOr(flag, 1);
    sm.P[c] = P_;
    sm.cellv[0][c] = n_;
    sm.cellv[1][c] = P_ / n_;
    sm.cellv[2][c] = ok ? v_ : 0.0;
    sm.ok[c] = ok ? 1 : 0;
  }
  __syncthreads();
  tile_coeffs_d<NPc, NVc>(tab, T.Qp, &sm.cellv[0][0], sm.ok, sm.co, nullptr, flag);
  // Lam[i][k] = sum_j dL/dF_ij w^xi_j P_k(xi_j), radial row i summed by group i
  if (g < QP_MAX) {
    double lam[NVc + 1];
#pragma unroll
    for (int q = 0; q <= NVc; ++q) lam[q] = 0.0;
    if (cell && g < T.Qp) {
      for (int j = 0; j < T.Qxi; ++j) {
        const double f = gF[T.poff + (size_t)(g * T.Qxi + j) * T.Nx + x];
        const double* pw = tab + TAB_XI + T.Qxi + j * (NV_MAX + 1);
#pragma unroll
        for (int q = 0; q <= NVc; ++q) lam[q] = fma(f, pw[q], lam[q]);
      }
    }
#pragma unroll
    for (int q = 0; q <= NVc; ++q) sm.lam[g * (NV_MAX + 1) + q][c] = lam[q];
  }
  __syncthreads();
  if (g == 0 && cell) {
    double dn = 0.0, dT = 0.0, db = 0.0;
    if (sm.ok[c])
      eq_param_grads<NPc, NVc>(tab, T.Qp, sm.cellv[0][c], sm.cellv[1][c], sm.cellv[2][c], sm.co, c, sm.lam, dn, dT,
                               db);
    const double n_ = sm.cellv[0][c];
    gP[k] = dT / n_;
    gn[k] = dn - dT * sm.P[c] / (n_ * n_);
    gv[k] = db;
  }
}

__global__ void __launch_bounds__(NT) rlb_init_vjp_kernel(const TubeDev* tubes, const int2* tiles,
                                                          const double* tabs, const double* P, const double* n,
                                                          const double* v, const double* gF, double* gP,
                                                          double* gn, double* gv, int* flag) {
  extern __shared__ __align__(16) unsigned char ivjp_smem_raw[];
  InitVjpSmem& sm = *reinterpret_cast<InitVjpSmem*>(ivjp_smem_raw);
  const int2 tl = tiles[blockIdx.x];
  const TubeDev T = tubes[tl.x];
  if (T.Np == 2 && T.Nv == 5)
    init_vjp_tile<2, 5>(T, tabs + T.tab, tl.y, P, n, v, gF, gP, gn, gv, flag, sm);
  else
    init_vjp_tile<NP_MAX, NV_MAX>(T, tabs + T.tab, tl.y, P, n, v, gF, gP, gn, gv, flag, sm);
}
