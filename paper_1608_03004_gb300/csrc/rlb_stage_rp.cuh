// Reduced-precision stage kernel: F stored in FP32 or BF16, advection, equilibrium evaluation, collision and
// the Runge-Kutta combination in FP32; the moments accumulated with compensated FP32 sums (double-float with
// double-float weights) and reduced in FP64; the Landau-frame solve and the equilibrium coefficients in FP64
// (the e, u^mu extraction cancels near |v| -> 1 and in rarefied cells). Included by rlb.cu inside its
// anonymous namespace.
//
// Built for bandwidth rather than for the FP64 pipe:
//  - the moments of a stage's input are not re-read: the stage that wrote F_in accumulated them while
//    storing it and left 5 FP64 moments per cell (M_in); this stage does the same for F_out (M_out), so every
//    stage reads F_in once;
//  - each thread keeps the next PF velocity rows of its tile in flight in registers (a prefetch ring),
//    issuing the loads of row r + PF as soon as row r is consumed;
//  - no FP64 instruction is executed per velocity node; FP64 work is per cell.
// Rows are walked radial-innermost (j = g, g + NG, ...; i = 0 .. Qp-1) so that the radial partial sums
// sum_i F pbar_i and sum_i F pbar_i^2 of one direction xi_j are folded into the five moments once per j.
#pragma once

template <typename S>
__device__ __forceinline__ float ld_s(const S* p);
template <>
__device__ __forceinline__ float ld_s<float>(const float* p) {
  return __ldg(p);
}
template <>
__device__ __forceinline__ float ld_s<__nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(__ldg(p));
}

template <typename S>
__device__ __forceinline__ S to_s(float v);
template <>
__device__ __forceinline__ float to_s<float>(float v) {
  return v;
}
template <>
__device__ __forceinline__ __nv_bfloat16 to_s<__nv_bfloat16>(float v) {
  return __float2bfloat16_rn(v);
}
template <typename S>
__device__ __forceinline__ float from_s(S v);
template <>
__device__ __forceinline__ float from_s<float>(float v) {
  return v;
}
template <>
__device__ __forceinline__ float from_s<__nv_bfloat16>(__nv_bfloat16 v) {
  return __bfloat162float(v);
}

constexpr int PF = 6;  // velocity rows in flight per thread

struct StageArgsRP {
  const TubeDev* tubes;
  const int2* tiles;
  const void* Fn;      // state at the start of the step (read at the cell only)
  const void* Fin;     // stage input (read with halo)
  void* Fout;          // stage output
  const double* Min;   // [5][nxtot] FP64 moments of Fin
  double* Mout;        // [5][nxtot] FP64 moments of Fout, written here
  long long nxtot;
  const double* tab;   // per-tube FP64 tables (as in the FP64 path)
  const float* tabf;   // per-tube FP32 tables
  int* flag;
  float a, b;          // Shu-Osher combination F_out = a F^n + b (F_in + dt L(F_in))
  double bd;           // b in FP64 (for the collision rate)
  int stage;
  int ntiles, schedule;  // as in the FP64 kernel
  int* counter;
};

struct StageSmemRP {
  union {
    double red[NG][5][GW];
    CoefSmem coef;
  } u;
  double B[NBC][GW];  // FP64 equilibrium coefficients from tile_coeffs
  float Bf[NBC][GW];  // their FP32 copy used per velocity node
  float rate[2][GW];
  float row[2][NG][RW + 1];
  float d1[NG][RW + 1];
  float sp[NG][3][GW];
  float phi[NG][GW];
  int src[RW + 1];
};

// Walk of one group's rows: direction j = g, g + NG, ..., radial node i = 0 .. Qp-1 innermost; s = i Qxi + j.
struct RowWalk {
  int i, j;
  __device__ __forceinline__ int s(int Qxi) const { return i * Qxi + j; }
  __device__ __forceinline__ void next(int Qp) {
    if (++i == Qp) {
      i = 0;
      j += NG;
    }
  }
};

template <typename S, int NPc, int NVc>
__device__ void stage_tile_rp(const StageArgsRP& A, const TubeDev& T, int x0, StageSmemRP& sm) {
  using rlbdev::DF;
  const int tid = threadIdx.x, c = tid % GW, g = tid / GW;
  const double* tab = A.tab + T.tab;
  const float* tabf = A.tabf + T.tabf;
  const int Qp = T.Qp, Qxi = T.Qxi, Nx = T.Nx, ld = T.ld;
  const S* Fin = static_cast<const S*>(A.Fin) + T.off;
  const S* Fn = static_cast<const S*>(A.Fn) + T.off;
  S* Fout = static_cast<S*>(A.Fout) + T.off;
  const int x = x0 + c;
  const bool cell = (c < TX) && (x < Nx);
  for (int k = tid; k < RW; k += NT) sm.src[k] = map_cell(x0 - HALO + k, Nx, T.bc);

  // rows of this group and the prefetch ring: thread c holds positions c and c + GW of the staged row
  // (the second only for c < RW - GW) and F^n at its own cell
  const int nj = (Qxi - g + NG - 1) / NG;  // directions j = g, g + NG, ... < Qxi
  const int nrows = nj > 0 ? nj * Qp : 0;
  const bool two = c < RW - GW;
  const bool use_fn = A.a != 0.f;
  __syncthreads();  // sm.src ready
  const int k0 = sm.src[c], k1 = two ? sm.src[c + GW] : 0;
  float pv0[PF], pv1[PF], pfn[PF];
  RowWalk cur{0, g}, ahead{0, g};  // the row being processed and the next row to load
#pragma unroll
  for (int u = 0; u < PF; ++u) {
    pv0[u] = pv1[u] = pfn[u] = 0.f;
    if (u < nrows) {
      const int s = ahead.s(Qxi);
      const S* src = Fin + (size_t)s * ld;
      pv0[u] = ld_s<S>(src + k0);
      if (two) pv1[u] = ld_s<S>(src + k1);
      if (use_fn && cell) pfn[u] = ld_s<S>(Fn + (size_t)s * ld + x);
      ahead.next(Qp);
    }
  }

  if (T.collide) {
    // B. Landau frame from the stored moments of F_in, equilibrium coefficients (FP64, per cell)
    double e = 1.0, beta = 0.0, n = 1.0, Tt = 1.0;
    bool ok = false;
    if (g == 0 && cell) {
      double mom[5];
#pragma unroll
      for (int f = 0; f < 5; ++f) mom[f] = A.Min[f * A.nxtot + T.xoff + x];
      ok = landau(mom, e, beta, n, Tt);
      if (!ok) atomicOr(A.flag, 1);
    }
    if (g == 0) {
      sm.u.coef.cell[0][c] = n;
      sm.u.coef.cell[1][c] = Tt;
      sm.u.coef.cell[2][c] = beta;
      sm.u.coef.ok[c] = ok ? 1 : 0;
      const double r0 = ok ? (A.bd * T.dt) * (T.inv_tau / sqrt(1.0 - beta * beta)) : 0.0;
      sm.rate[0][c] = (float)r0;
      sm.rate[1][c] = (float)(r0 * beta);
    }
    __syncthreads();
    tile_coeffs<NPc, NVc>(tab, Qp, sm.u.coef, sm.B, A.flag);
    if (g < QP_MAX) {
#pragma unroll
      for (int k = 0; k <= NVc; ++k) sm.Bf[g * (NV_MAX + 1) + k][c] = (float)sm.B[g * (NV_MAX + 1) + k][c];
    }
  }
  __syncthreads();

  // C. rows: advection + collision + Runge-Kutta combination in FP32, moments of the output on the fly
  const float a = A.a, b = A.b;
  const float* cxi_tab = tabf + tabf_cxi(Qxi) + A.stage * Qxi;
  float* d1 = sm.d1[g];
  float* sp0 = sm.sp[g][0];
  float* sp1 = sm.sp[g][1];
  float* sp2 = sm.sp[g][2];
  float* phi = sm.phi[g];
  DF m0 = {0.f, 0.f}, m1 = m0, m2 = m0, m3 = m0, m4 = m0, ra = m0, rb = m0;
  int buf = 0;
  const int nchunks = (nrows + PF - 1) / PF;
  for (int ch = 0; ch < nchunks; ++ch) {
#pragma unroll
    for (int u = 0; u < PF; ++u) {
      const int r = ch * PF + u;
      // every thread of the group takes the same branch: r depends on the group only
      if (r < nrows) {
        const int i = cur.i, j = cur.j, s = cur.s(Qxi);
        cur.next(Qp);
        float* row = sm.row[buf][g];
        row[c] = pv0[u];
        if (two) row[c + GW] = pv1[u];
        const float fn = pfn[u];
        // refill this slot with row r + PF
        if (r + PF < nrows) {
          const int s2 = ahead.s(Qxi);
          ahead.next(Qp);
          const S* src = Fin + (size_t)s2 * ld;
          pv0[u] = ld_s<S>(src + k0);
          if (two) pv1[u] = ld_s<S>(src + k1);
          if (use_fn && cell) pfn[u] = ld_s<S>(Fn + (size_t)s2 * ld + x);
        }
        group_sync(g);
        const float xi = tabf[TABF_X + j];
        const bool fwd = xi > 0.f;
        {
          const int p = c + (fwd ? 1 : 2);
          const float xd = row[p] - row[p - 1], yd = row[p + 1] - row[p];
          // indicators of the weight-normalised differences (the squares of those of F would leave FP32's
          // range for small weights); the combination is invariant under that common scale
          const float iws = tabf[tabf_iws(Qxi) + s];
          float sa, sb, sc;
          weno5_pair(xd * iws, yd * iws, fwd, rlbdev::EPS_A, rlbdev::EPS_B, rlbdev::EPS_C, sa, sb, sc);
          sp0[c] = sa;
          sp1[c] = sb;
          sp2[c] = sc;
          d1[p] = xd;
          if (c == GW - 1) d1[p + 1] = yd;
        }
        group_sync(g);
        float D = 0.f;
        if (c <= TX) {
          float G;
          if (fwd) {
            D = d1[c + 3];
            G = weno5_combine(sp0[c], sp1[c + 1], sp2[c + 2], d1[c + 1], d1[c + 2], D, d1[c + 4]);
          } else {
            D = d1[c + 4];
            G = weno5_combine(sp0[c + 2], sp1[c + 1], sp2[c], -d1[c + 5], -D, -d1[c + 3], -d1[c + 2]);
          }
          phi[c] = G;
        }
        group_sync(g);
        if (cell) {
          const float F = row[c + 3];
          const float dphi = D + (phi[c + 1] - phi[c]);
          float out = F;
          if (use_fn) out = fmaf(a, fn, b * F);
          out = fmaf(-cxi_tab[j], dphi, out);
          if (T.collide) {
            const float* pw = tabf + tabf_pw(Qxi) + j * (NV_MAX + 1);
            float feq = 0.f;
#pragma unroll
            for (int k = 0; k <= NVc; ++k) feq = fmaf(sm.Bf[i * (NV_MAX + 1) + k][c], pw[k], feq);
            const float rate = fmaf(-sm.rate[1][c], xi, sm.rate[0][c]);
            out = fmaf(rate, feq - F, out);
          }
          const S stored = to_s<S>(out);
          Fout[(size_t)s * ld + x] = stored;
          if (T.collide) {
            // moments of what was stored: radial partial sums, folded into the five moments per direction
            const float v = from_s<S>(stored);
            rlbdev::df_add_prod(ra, v, tabf[TABF_P1 + i], tabf[TABF_P1 + QP_MAX + i]);
            rlbdev::df_add_prod(rb, v, tabf[TABF_P2 + i], tabf[TABF_P2 + QP_MAX + i]);
            if (i == Qp - 1) {
              const float xh = tabf[TABF_X + j], xl = tabf[TABF_X + Qxi + j];
              const float x2h = tabf[TABF_X + 2 * Qxi + j], x2l = tabf[TABF_X + 3 * Qxi + j];
              rlbdev::df_add(m0, ra);
              rlbdev::df_add_dfprod(m1, ra, xh, xl);
              rlbdev::df_add(m2, rb);
              rlbdev::df_add_dfprod(m3, rb, xh, xl);
              rlbdev::df_add_dfprod(m4, rb, x2h, x2l);
              ra = {0.f, 0.f};
              rb = {0.f, 0.f};
            }
          }
        }
        buf ^= 1;
      }
    }
  }

  // epilogue: FP64 moments of F_out for the next stage (collision tubes only)
  if (T.collide) {
    __syncthreads();  // the coefficient scratch in the union is no longer read
    sm.u.red[g][0][c] = (double)m0.hi + (double)m0.lo;
    sm.u.red[g][1][c] = (double)m1.hi + (double)m1.lo;
    sm.u.red[g][2][c] = (double)m2.hi + (double)m2.lo;
    sm.u.red[g][3][c] = (double)m3.hi + (double)m3.lo;
    sm.u.red[g][4][c] = (double)m4.hi + (double)m4.lo;
    __syncthreads();
    if (g == 0 && cell) {
#pragma unroll
      for (int f = 0; f < 5; ++f)
        A.Mout[f * A.nxtot + T.xoff + x] = (sm.u.red[0][f][c] + sm.u.red[1][f][c]) + (sm.u.red[2][f][c] + sm.u.red[3][f][c]);
    }
  }
}

template <typename S, int SCHED>
__global__ void __launch_bounds__(NT) rlb_stage_rp_kernel(StageArgsRP A) {
  extern __shared__ __align__(16) unsigned char stage_rp_smem_raw[];
  StageSmemRP& sm = *reinterpret_cast<StageSmemRP*>(stage_rp_smem_raw);
  for_each_tile(A.ntiles, SCHED, A.counter, [&](int t) {
    const int2 tl = A.tiles[t];
    const TubeDev T = A.tubes[tl.x];
    if (T.Np == 2 && T.Nv == 5)
      stage_tile_rp<S, 2, 5>(A, T, tl.y, sm);
    else
      stage_tile_rp<S, NP_MAX, NV_MAX>(A, T, tl.y, sm);
  });
}
