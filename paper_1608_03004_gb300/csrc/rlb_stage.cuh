// FP64 stage kernel of the time step and the device helpers that the other kernels share (Landau frame,
// Legendre series of the equilibrium, per-tile coefficients, tile schedules, group barriers). Included by
// rlb.cu inside its anonymous namespace; the file covers the kernel code that the FP64 profile summary was
// captured on, host code lives in rlb.cu.
#pragma once

constexpr int NT = 256;                    // threads per CTA
constexpr int GW = 64;                     // threads per velocity group (one row at a time)
constexpr int NG = NT / GW;                // velocity rows processed together
constexpr int TX = GW - 3;                 // cells per tile: their TX + 1 interfaces need GW indicator pairs
constexpr int HALO = 3;                    // WENO5 reaches three cells upwind/downwind
constexpr int RW = TX + 2 * HALO;          // staged row length
constexpr int NBC = QP_MAX * (NV_MAX + 1); // per-cell equilibrium coefficients

// Series tables for the Legendre coefficients of (1 - beta xi)^-m (filled once per device):
//   g_ic[r][k] = (2k+1)/2 * int_{-1}^{1} xi^r P_k(xi) dxi,   g_cb[m][r] = C(m + r - 1, r).
__device__ double g_ic[(R_MAX + 1) * (NV_MAX + 1)];
__device__ double g_cb[(M_MAX + 1) * (R_MAX + 1)];

struct StageArgs {
  const TubeDev* tubes;
  const int2* tiles;  // (tube, first cell)
  const double* Fn;   // state at the start of the step (read at the cell only)
  const double* Fin;  // stage input (read with halo)
  double* Fout;       // stage output
  const double* tab;
  int* flag;
  int* warn;          // sticky warning bits (RLB_WARN_*) or NULL
  double a, b;        // Shu-Osher combination F_out = a F^n + b (F_in + dt L(F_in))
  int stage;          // 0, 1, 2: selects the b dt xi / dx table
  int ntiles;         // tiles of this launch
  int schedule;       // 0: one CTA per tile; 1: persistent, grid stride; 2: persistent, work counter
  int* counter;       // work counter of schedule 2 (zeroed before the launch)
  int split;          // work items per tile (<= 1: one): item k of a tile advances velocity rows
                      // [k Q / split, (k + 1) Q / split) after reducing the moments over all rows
};

// Tile loop of a stage launch. Schedule 0 gives each CTA one tile; the persistent schedules keep a grid of
// about one wave resident and hand out tiles by a grid stride or by an atomic work counter (cost-ordered
// tiles then balance uneven tubes). No CTA ever waits on another.
template <typename Body>
__device__ __forceinline__ void for_each_tile(int ntiles, int schedule, int* counter, Body body) {
  if (schedule == 0) {
    body((int)blockIdx.x);
    return;
  }
  if (schedule == 1) {
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
      __syncthreads();  // the previous tile's shared-memory readers are done
      body(t);
    }
    return;
  }
  __shared__ int next_tile;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) next_tile = atomicAdd(counter, 1);
    __syncthreads();
    const int t = next_tile;
    if (t >= ntiles) return;
    body(t);
  }
}

// --------------------------------------------------------------------------------------------------
// Device helpers
// --------------------------------------------------------------------------------------------------

// Source of a staged position x in [-HALO, Nx - 1 + GW + HALO] within its row: periodic wrap (Nx >= 3),
// zero-gradient ghosts (open boundary), or, on a halo side of a slab, the ghost cells the caller unpacked beside
// the row (left ghosts -3..-1 at ld-3..ld-1, right ghosts at Nx..Nx+2; ld >= Nx + 6 for slabs; positions past
// Nx + 2 are never read by a cell and map to Nx + 2). Always in [0, ld).
__device__ __forceinline__ int map_cell(int x, int Nx, int bc, int ld) {
  if (bc == RLB_BC_PERIODIC) {
    if (x < 0) x += Nx;
    return x % Nx;
  }
  if (x < 0) return (bc & RLB_BC_HALO_LEFT) ? ld + (x < -HALO ? -HALO : x) : 0;
  if (x >= Nx) return (bc & RLB_BC_HALO_RIGHT) ? (x > Nx + HALO - 1 ? Nx + HALO - 1 : x) : Nx - 1;
  return x;
}

// True where the fastest relaxation of a cell moving at beta, dt gamma (1 + |beta| max|xi|) / tau, is beyond the
// stable region of SSP-RK3 with WENO5 advection at the tube's Courant number (TubeDev::stiff_lim).
__device__ __forceinline__ bool stiff(const TubeDev& T, double beta) {
  const double k = T.dt * T.inv_tau * fma(fabs(beta), T.xi_max, 1.0);  // the rate without gamma = 1 / sqrt(1 - beta^2)
  return k * k > T.stiff_lim * T.stiff_lim * (1.0 - beta * beta);      // (k gamma)^2 > stiff_lim^2, no square root
}

// Landau frame from (N0, Nx, T00, T0x, Txx): e, beta, n (Landau), T, and gamma = (1 - beta^2)^-1/2 if gam_out is
// given. Returns false if non-physical. A cell at rest (T0x = 0, exactly so wherever the state is symmetric in xi)
// skips the division and square root that give beta = 0, gamma = 1 and n = N0.
__device__ __forceinline__ bool landau(const double mom[5], double& e, double& beta, double& n, double& T,
                                       double* gam_out = nullptr) {
  const double A = mom[2] + mom[4];
  const double disc = A * A - 4.0 * mom[3] * mom[3];
  e = 0.5 * ((mom[2] - mom[4]) + sqrt(disc));
  double gam = 1.0;
  if (mom[3] == 0.0) {
    beta = 0.0;
    n = mom[0];
  } else {
    beta = mom[3] / (mom[4] + e);
    gam = 1.0 / sqrt(1.0 - beta * beta);
    n = gam * (mom[0] - beta * mom[1]);
  }
  T = e / (3.0 * n);
  if (gam_out) *gam_out = gam;
  return disc >= 0.0 && e > 0.0 && fabs(beta) < 1.0 && n > 0.0 && T > 0.0;
}

// --------------------------------------------------------------------------------------------------
// Per-cell equilibrium coefficients of a tile (shared by the stage and initial-condition kernels)
// --------------------------------------------------------------------------------------------------

struct CoefSmem {
  double hh[M_MAX - 1][NV_MAX + 1][GW];  // hhat_{m,k}, m = 2 .. Np+2
  double cell[3][GW];                    // n, T, beta of each cell
  int ok[GW];
};

// One parity class of the Legendre coefficients hhat_{m,k} = (2k+1)/2 int P_k(xi) (1 - beta xi)^-m dxi,
// m = 2..NPc+2, k = PAR, PAR+2, .. <= NVc, by the positive power series (1 - beta xi)^-m =
// sum_r C(m+r-1, r) beta^r xi^r with int xi^r P_k tabulated. Terms of one class share one sign, so the sum
// has no cancellation; it stops when the largest-m term drops below 1e-18 (1 - beta^2).
template <int NPc, int NVc, int PAR, int STRIDE = GW>
__device__ bool hhat_parity(double beta, double* hh_col /* [m-2][k][STRIDE] at this cell */) {
  constexpr int NK = (NVc - PAR) / 2 + 1;
  double acc[NPc + 1][NK];
#pragma unroll
  for (int m = 0; m <= NPc; ++m)
#pragma unroll
    for (int q = 0; q < NK; ++q) acc[m][q] = 0.0;
  bool done = (beta == 0.0);
  if (beta == 0.0 && PAR == 0) {
#pragma unroll
    for (int m = 0; m <= NPc; ++m) acc[m][0] = 1.0;
  }
  if (!done) {
    const double b2 = beta * beta;
    const double tol = 1e-18 * (1.0 - b2);
    double br = PAR ? beta : 1.0;  // beta^r
    for (int r = PAR; r <= R_MAX; r += 2) {
      const double* ic = g_ic + r * (NV_MAX + 1);
      double tlast = 0.0;
#pragma unroll
      for (int m = 0; m <= NPc; ++m) {
        const double t = g_cb[(m + 2) * (R_MAX + 1) + r] * br;
#pragma unroll
        for (int q = 0; q < NK; ++q) acc[m][q] = fma(ic[PAR + 2 * q], t, acc[m][q]);
        tlast = t;
      }
      if (r >= NVc && fabs(tlast) < tol) {
        done = true;
        break;
      }
      br *= b2;
    }
  }
#pragma unroll
  for (int m = 0; m <= NPc; ++m)
#pragma unroll
    for (int q = 0; q < NK; ++q) hh_col[((m * (NV_MAX + 1)) + PAR + 2 * q) * STRIDE] = acc[m][q];
  return done;
}

// Fill B[i (NVc+1) + k][c] (radial rows i < Qp) for the TX cells of a tile from cs.cell (n, T, beta) and cs.ok:
//   F^eq_ij = sum_k B[i][k] w^xi_j P_k(xi_j),  B[i][k] = n/(4T^3) w^p_i sum_q s^(q+2) K[i][q] hhat_{q+2,k},
// s = T/gamma (Eq. (feqtrunc): Laguerre generating function for the radial projection, Legendre projection
// of each (1 - beta xi)^-m for the angular one). Groups 0/1 run the even/odd series, then group g builds
// radial row i = g. Cells with ok == 0 get B = 0. Ends with a barrier.
template <int NPc, int NVc>
__device__ void tile_coeffs(const double* tab, int Qp, CoefSmem& cs, double (*Bs)[GW], int* flag) {
  const int c = threadIdx.x % GW, g = threadIdx.x / GW;
  if (g < 2 && c < TX) {
    const double beta = cs.cell[2][c];
    bool conv = true;
    if (cs.ok[c]) {
      if (g == 0)
        conv = hhat_parity<NPc, NVc, 0>(beta, &cs.hh[0][0][c]);
      else
        conv = hhat_parity<NPc, NVc, 1>(beta, &cs.hh[0][0][c]);
    }
    if (!conv) {
      cs.ok[c] = 0;  // both groups may write 0; no other value is written concurrently
      atomicOr(flag, 1);
    }
  }
  __syncthreads();
  if (c < TX) {
    const int i = g;
    double B[NVc + 1];
#pragma unroll
    for (int k = 0; k <= NVc; ++k) B[k] = 0.0;
    if (i < Qp && cs.ok[c]) {
      const double n = cs.cell[0][c], T = cs.cell[1][c], beta = cs.cell[2][c];
      const double s = T * sqrt(1.0 - beta * beta);
      const double pref = n / (4.0 * T * T * T) * tab[TAB_WP + i];
      double sq = s * s;
#pragma unroll
      for (int q = 0; q <= NPc; ++q) {
        const double G = pref * sq * tab[TAB_K + i * (NP_MAX + 1) + q];
#pragma unroll
        for (int k = 0; k <= NVc; ++k) B[k] = fma(G, cs.hh[q][k][c], B[k]);
        sq *= s;
      }
    }
    if (i < Qp) {
#pragma unroll
      for (int k = 0; k <= NVc; ++k) Bs[i * (NVc + 1) + k][c] = B[k];
    }
  }
  __syncthreads();
}

// --------------------------------------------------------------------------------------------------
// Stage kernel
// --------------------------------------------------------------------------------------------------

// Barrier of one 64-thread velocity group (named barrier 1 + g; barrier 0 is __syncthreads).
__device__ __forceinline__ void group_sync(int g) { asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(GW) : "memory"); }

struct StageSmem {
  union {
    double red[NG][3 * QP_MAX][GW];  // per group: the radial sums S0, S1, S2 of each radial node
    CoefSmem coef;
  } u;
  double rate[2][GW];
  double row[2][NG][RW + 1];  // staged velocity rows (double-buffered: written before the first barrier)
  double d1[NG][RW + 1];      // first differences by position, d1[k] = row[k] - row[k-1]
  float2 dd[NG][RW + 1];      // the same differences in double-float (hi, lo)
  float2 sv[NG][3][GW];       // indicators v = S + e (double-float), one triple per pair of adjacent differences
  float2 phi[NG][GW];         // WENO correction of each interface, times 6 (double-float)
  int src[RW + 1];            // source cell of each staged position (boundary condition applied)
  double B[NBC][GW];          // equilibrium coefficients B[i (NVc + 1) + k]; last, so that a launch allocates
                              // only the rows its tubes use (stage_smem_bytes)
};
// Dynamic shared memory of the FP64 stage kernel for `brows` coefficient rows.
constexpr size_t stage_smem_bytes(int brows) { return offsetof(StageSmem, B) + (size_t)brows * GW * sizeof(double); }

template <int NPc, int NVc>
__device__ void stage_tile(const StageArgs& A, const TubeDev& T, int x0, int part, int nparts, StageSmem& sm) {
  const int tid = threadIdx.x, c = tid % GW, g = tid / GW;
  const double* tab = A.tab + T.tab;
  const int Qp = T.Qp, Qxi = T.Qxi, Nx = T.Nx, ld = T.ld;
  const double* Fin = A.Fin + T.off;
  const double* Fn = A.Fn + T.off;
  double* Fout = A.Fout + T.off;
  const int x = x0 + c;
  const bool cell = (c < TX) && (x < Nx);
  for (int k = tid; k < RW; k += NT) sm.src[k] = map_cell(x0 - HALO + k, Nx, T.bc, ld);

  if (T.collide) {
    // A. moments of the stage input. The groups split the mirror pairs of directions (xi_jf = -xi_jb > 0) and
    //    keep, per radial node i, S0 = sum_j F_ij, S1 = sum_j F_ij xi_j and S2 = sum_j F_ij xi_j^2 from the sum
    //    s = F(xi) + F(-xi) and difference d = F(xi) - F(-xi) of each pair (S0 += s, S1 += d xi, S2 += s xi^2):
    //    5 FP64 operations per two populations. An odd Qxi's xi = 0 direction adds to S0 only. Then
    //    N0 = sum_i pbar_i S0_i, Nx = sum_i pbar_i S1_i, T00 = sum_i pbar_i^2 S0_i, T0x = sum_i pbar_i^2 S1_i and
    //    Txx = sum_i pbar_i^2 S2_i.
    double S[3 * QP_MAX];
#pragma unroll
    for (int k = 0; k < 3 * QP_MAX; ++k) S[k] = 0.0;
    const int hq = Qxi / 2;
    if (cell) {
      for (int jb = g; jb < hq; jb += NG) {
        const int jf = Qxi - 1 - jb;
        const double xi = tab[TAB_XI + jf], xi2 = xi * xi;
#pragma unroll
        for (int i = 0; i < QP_MAX; ++i) {
          if (i < Qp) {
            const double ff = __ldg(Fin + (size_t)(i * Qxi + jf) * ld + x);
            const double fb = __ldg(Fin + (size_t)(i * Qxi + jb) * ld + x);
            const double sum = ff + fb, dif = ff - fb;
            S[3 * i] += sum;
            S[3 * i + 1] = fma(dif, xi, S[3 * i + 1]);
            S[3 * i + 2] = fma(sum, xi2, S[3 * i + 2]);
          }
        }
      }
      if ((Qxi & 1) && g == (hq % NG)) {
#pragma unroll
        for (int i = 0; i < QP_MAX; ++i)
          if (i < Qp) S[3 * i] += __ldg(Fin + (size_t)(i * Qxi + hq) * ld + x);
      }
    }
#pragma unroll
    for (int k = 0; k < 3 * QP_MAX; ++k) sm.u.red[g][k][c] = S[k];
    __syncthreads();
    // B. Landau frame (one thread per cell), then the equilibrium coefficients
    double e = 1.0, beta = 0.0, n = 1.0, Tt = 1.0;
    bool ok = false;
    if (g == 0 && cell) {
      double mom[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int i = 0; i < QP_MAX; ++i) {
        if (i < Qp) {
          double Si[3];
#pragma unroll
          for (int q = 0; q < 3; ++q)
            Si[q] = (sm.u.red[0][3 * i + q][c] + sm.u.red[1][3 * i + q][c]) +
                    (sm.u.red[2][3 * i + q][c] + sm.u.red[3][3 * i + q][c]);
          const double p1 = tab[TAB_PBAR + i], p2 = tab[TAB_PBAR2 + i];
          mom[0] = fma(p1, Si[0], mom[0]);
          mom[1] = fma(p1, Si[1], mom[1]);
          mom[2] = fma(p2, Si[0], mom[2]);
          mom[3] = fma(p2, Si[1], mom[3]);
          mom[4] = fma(p2, Si[2], mom[4]);
        }
      }
      ok = landau(mom, e, beta, n, Tt);
      if (!ok) atomicOr(A.flag, 1);
      else if (A.warn != nullptr && stiff(T, beta)) atomicOr(A.warn, RLB_WARN_STIFF);
    }
    __syncthreads();  // the moments are consumed; the union now holds the coefficient scratch
    if (g == 0 && c < GW) {
      sm.u.coef.cell[0][c] = n;
      sm.u.coef.cell[1][c] = Tt;
      sm.u.coef.cell[2][c] = beta;
      sm.u.coef.ok[c] = ok ? 1 : 0;
      // b dt gamma / tau and its beta multiple: the stage's collision rate is r0 - r1 xi_j
      const double r0 = ok ? (A.b * T.dt) * (T.inv_tau / sqrt(1.0 - beta * beta)) : 0.0;
      sm.rate[0][c] = r0;
      sm.rate[1][c] = r0 * beta;
    }
    __syncthreads();
    tile_coeffs<NPc, NVc>(tab, Qp, sm.u.coef, sm.B, A.flag);
  }
  __syncthreads();  // sm.src (and, with collisions, the coefficients) are ready

  // C. advection + collision + Runge-Kutta combination. The work unit of a 64-thread group is a mirror pair
  //    of directions (j, Qxi - 1 - j) of one radial node, processed back to back: the nodes are symmetric, so
  //    w^xi P_k(-xi) = (-1)^k w^xi P_k(xi) and the even and odd Legendre parts of F^eq, summed once, give both
  //    rows' equilibria (the xi = 0 node of an odd Qxi is a unit of its own). Groups synchronise with named
  //    barriers only.
  const double a = A.a, b = A.b;
  const double* cxi_tab = tab + tab_cxi(Qxi) + A.stage * Qxi;
  double* d1 = sm.d1[g];
  float2* dd = sm.dd[g];
  float2* sv0 = sm.sv[g][0];
  float2* sv1 = sm.sv[g][1];
  float2* sv2 = sm.sv[g][2];
  float2* phi = sm.phi[g];
  const float2* epsf = reinterpret_cast<const float2*>(tab + tab_epsf(Qp, Qxi));
  const int hq = Qxi / 2, upr = hq + (Qxi & 1), U = Qp * upr;
  const int u_end = (part + 1) * U / nparts;
  int buf = 0;
  for (int u0 = part * U / nparts; u0 < u_end; u0 += NG) {
    const int u = u0 + g;
    if (u >= u_end) continue;  // uniform over the group
    const int i = u / upr, jA = u - i * upr;  // jA = hq: the xi = 0 node
    const int nrow = jA < hq ? 2 : 1;
    double E = 0.0, O = 0.0;  // even and odd parts of sum_k B[i][k] w^xi P_k(xi_jA) at this cell
    for (int h = 0; h < nrow; ++h, buf ^= 1) {
      const int j = h == 0 ? jA : Qxi - 1 - jA;
      const int s = i * Qxi + j;
      double* row = sm.row[buf][g];
      // stage the row with its first differences, in FP64 and split into double-float (position k needs k - 1
      // as well)
      {
        const double* src = Fin + (size_t)s * ld;
        // positions 0 .. GW-1, one per thread: the previous position's value comes from the lane below by a
        // shuffle (the first lane of each warp loads it)
        {
          const double v = __ldg(src + sm.src[c]);
          row[c] = v;
          const double below = __shfl_up_sync(0xffffffffu, v, 1);
          if (c > 0) {
            const double dk = v - ((c & 31) == 0 ? __ldg(src + sm.src[c - 1]) : below);
            d1[c] = dk;
            const rlbdev::DF q = rlbdev::df_split(dk);
            dd[c] = make_float2(q.hi, q.lo);
          }
        }
        for (int k = c + GW; k < RW; k += GW) {
          const double v = __ldg(src + sm.src[k]);
          row[k] = v;
          const double dk = v - __ldg(src + sm.src[k - 1]);
          d1[k] = dk;
          const rlbdev::DF q = rlbdev::df_split(dk);
          dd[k] = make_float2(q.hi, q.lo);
        }
      }
      // the Runge-Kutta input of this row's cell, loaded now so that its latency hides behind the limiter
      const double fnv = (A.stage != 0 && cell) ? __ldg(Fn + (size_t)s * ld + x) : 0.0;
      group_sync(g);
      const double xi = tab[TAB_XI + j];
      const bool fwd = h == 1;  // the mirror row xi_{Qxi-1-jA} > 0; the first row has xi <= 0
      // pairs: thread c owns the pair of differences at positions (p, p + 1), p = c + 1 (wind toward +x) or
      // c + 2 (toward -x); these are the pairs the TX + 1 interfaces of the tile use
      {
        const int p = c + (fwd ? 1 : 2);
        const float2 e = epsf[s], x = dd[p], y = dd[p + 1];
        rlbdev::DF va, vb, vc;
        rlbdev::weno5_pair_df({x.x, x.y}, {y.x, y.y}, fwd, {e.x, e.y}, va, vb, vc);
        sv0[c] = make_float2(va.hi, va.lo);
        sv1[c] = make_float2(vb.hi, vb.lo);
        sv2[c] = make_float2(vc.hi, vc.lo);
      }
      group_sync(g);
      // interfaces: interface c lies between cells x0 + c - 1 and x0 + c (row index c + 2 | c + 3); its value
      // is v2 + G with v2 the upwind cell; D = v2(c + 1) - v2(c) is the memory-order difference d1[c + 3]
      // (wind toward +x) or d1[c + 4] (toward -x)
      double D = 0.0;
      if (c <= TX) {
        auto get = [](const float2* a, int k) { const float2 q = a[k]; return rlbdev::DF{q.x, q.y}; };
        auto neg = [&](int k) { const float2 q = dd[k]; return rlbdev::DF{-q.x, -q.y}; };
        rlbdev::DF G;
        if (fwd) {
          D = d1[c + 3];
          G = rlbdev::weno5_combine6_df(get(sv0, c), get(sv1, c + 1), get(sv2, c + 2), get(dd, c + 1),
                                        get(dd, c + 2), get(dd, c + 3), get(dd, c + 4));
        } else {
          D = d1[c + 4];
          G = rlbdev::weno5_combine6_df(get(sv0, c + 2), get(sv1, c + 1), get(sv2, c), neg(c + 5), neg(c + 4),
                                        neg(c + 3), neg(c + 2));
        }
        phi[c] = make_float2(G.hi, G.lo);
      }
      group_sync(g);
      if (cell) {
        const double F = row[c + 3];
        // phi holds 6 G: D + (6 G_{x+1/2} - 6 G_{x-1/2}) / 6, the difference taken in double-float
        const float2 pr = phi[c + 1], pl = phi[c];
        const rlbdev::DF dG = rlbdev::df_plus({pr.x, pr.y}, {-pl.x, -pl.y});
        const double dphi = fma(rlbdev::df_widen(dG.hi), 1.0 / 6.0, fma(rlbdev::df_widen(dG.lo), 1.0 / 6.0, D));
        double out = F;
        if (A.stage != 0) out = fma(a, fnv, b * F);  // a = 0 in the first stage
        out = fma(-cxi_tab[j], dphi, out);  // - b dt xi/dx (Phi_{x+1/2} - Phi_{x-1/2})
        if (T.collide) {
          if (h == 0) {
            const double* pw = tab + TAB_XI + Qxi + jA * (NV_MAX + 1);
#pragma unroll
            for (int k = 0; k <= NVc; ++k) {
              const double t = sm.B[i * (NVc + 1) + k][c];
              if (k % 2 == 0)
                E = fma(t, pw[k], E);
              else
                O = fma(t, pw[k], O);
            }
          }
          const double feq = h == 0 ? E + O : E - O;
          const double rate = fma(-sm.rate[1][c], xi, sm.rate[0][c]);
          out = fma(rate, feq - F, out);  // + b dt gamma (1 - beta xi)/tau (F^eq - F)
        }
        Fout[(size_t)s * ld + x] = out;
      }
    }
  }
}

// SCHED is the launch's schedule (compile time, so that the one-CTA-per-tile kernel carries no tile loop).
template <int SCHED>
__global__ void __launch_bounds__(NT, 3) rlb_stage_kernel(StageArgs A) {
  extern __shared__ __align__(16) unsigned char stage_smem_raw[];
  StageSmem& sm = *reinterpret_cast<StageSmem*>(stage_smem_raw);
  const int K = A.split > 1 ? A.split : 1;
  for_each_tile(A.ntiles * K, SCHED, A.counter, [&](int item) {
    const int t = item / K, part = item - t * K;
    const int2 tl = A.tiles[t];
    const TubeDev T = A.tubes[tl.x];
    if (T.Np == 2 && T.Nv == 5)
      stage_tile<2, 5>(A, T, tl.y, part, K, sm);
    else
      stage_tile<NP_MAX, NV_MAX>(A, T, tl.y, part, K, sm);
  });
}
