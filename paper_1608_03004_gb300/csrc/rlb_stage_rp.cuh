// Reduced-precision stage kernel: F stored in FP32 or BF16, advection, equilibrium evaluation, collision and
// the Runge-Kutta combination in FP32; the moments accumulated with compensated FP32 sums (double-float with
// double-float weights) and reduced in FP64; the Landau-frame solve and the equilibrium coefficients in FP64
// (the e, u^mu extraction cancels near |v| -> 1 and in rarefied cells). Same tiling, row staging and WENO5
// arrangement as the FP64 kernel. Included by rlb.cu inside its anonymous namespace.
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

struct StageArgsRP {
  const TubeDev* tubes;
  const int2* tiles;
  const void* Fn;     // state at the start of the step (read at the cell only)
  const void* Fin;    // stage input (read with halo)
  void* Fout;         // stage output
  const double* tab;  // per-tube FP64 tables (as in the FP64 path)
  const float* tabf;  // per-tube FP32 tables
  int* flag;
  float a, b;         // Shu-Osher combination F_out = a F^n + b (F_in + dt L(F_in))
  double bd;          // b in FP64 (for the collision rate)
  int stage;
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

template <typename S, int NPc, int NVc>
__device__ void stage_tile_rp(const StageArgsRP& A, const TubeDev& T, int x0, StageSmemRP& sm) {
  using rlbdev::DF;
  const int tid = threadIdx.x, c = tid % GW, g = tid / GW;
  const double* tab = A.tab + T.tab;
  const float* tabf = A.tabf + T.tabf;
  const int Qp = T.Qp, Qxi = T.Qxi, Q = Qp * Qxi, Nx = T.Nx, ld = T.ld;
  const S* Fin = static_cast<const S*>(A.Fin) + T.off;
  const S* Fn = static_cast<const S*>(A.Fn) + T.off;
  S* Fout = static_cast<S*>(A.Fout) + T.off;
  const int x = x0 + c;
  const bool cell = (c < TX) && (x < Nx);
  for (int k = tid; k < RW; k += NT) sm.src[k] = map_cell(x0 - HALO + k, Nx, T.bc);

  if (T.collide) {
    // A. moments: compensated FP32 sums over this group's velocity rows, then FP64
    DF m[5] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    if (cell) {
      for (int j = g; j < Qxi; j += NG) {
        DF a = {0.f, 0.f}, b = {0.f, 0.f};
        for (int i = 0; i < Qp; ++i) {
          const float f = ld_s<S>(Fin + (size_t)(i * Qxi + j) * ld + x);
          rlbdev::df_add_prod(a, f, tabf[TABF_P1 + i], tabf[TABF_P1 + QP_MAX + i]);
          rlbdev::df_add_prod(b, f, tabf[TABF_P2 + i], tabf[TABF_P2 + QP_MAX + i]);
        }
        const float xh = tabf[TABF_X + j], xl = tabf[TABF_X + Qxi + j];
        const float x2h = tabf[TABF_X + 2 * Qxi + j], x2l = tabf[TABF_X + 3 * Qxi + j];
        rlbdev::df_add(m[0], a);
        rlbdev::df_add_dfprod(m[1], a, xh, xl);
        rlbdev::df_add(m[2], b);
        rlbdev::df_add_dfprod(m[3], b, xh, xl);
        rlbdev::df_add_dfprod(m[4], b, x2h, x2l);
      }
    }
#pragma unroll
    for (int f = 0; f < 5; ++f) sm.u.red[g][f][c] = (double)m[f].hi + (double)m[f].lo;
    __syncthreads();
    // B. Landau frame and equilibrium coefficients in FP64 (as in the FP64 path)
    double e = 1.0, beta = 0.0, n = 1.0, Tt = 1.0;
    bool ok = false;
    if (g == 0 && cell) {
      double mom[5];
#pragma unroll
      for (int f = 0; f < 5; ++f) mom[f] = (sm.u.red[0][f][c] + sm.u.red[1][f][c]) + (sm.u.red[2][f][c] + sm.u.red[3][f][c]);
      ok = landau(mom, e, beta, n, Tt);
      if (!ok) atomicOr(A.flag, 1);
    }
    __syncthreads();
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

  // C. advection + collision + Runge-Kutta combination in FP32
  const float a = A.a, b = A.b;
  const float* cxi_tab = tabf + tabf_cxi(Qxi) + A.stage * Qxi;
  float* d1 = sm.d1[g];
  float* sp0 = sm.sp[g][0];
  float* sp1 = sm.sp[g][1];
  float* sp2 = sm.sp[g][2];
  float* phi = sm.phi[g];
  int buf = 0;
  for (int s0 = 0; s0 < Q; s0 += NG, buf ^= 1) {
    const int s = s0 + g;
    const bool rv = s < Q;
    const int i = rv ? s / Qxi : 0, j = rv ? s - i * Qxi : 0;
    float* row = sm.row[buf][g];
    if (rv) {
      const S* src = Fin + (size_t)s * ld;
      for (int k = c; k < RW; k += GW) row[k] = ld_s<S>(src + sm.src[k]);
    }
    group_sync(g);
    const float xi = tabf[TABF_X + j];
    const bool fwd = tab[TAB_XI + j] > 0.0;
    if (rv) {
      const int p = c + (fwd ? 1 : 2);
      const float xd = row[p] - row[p - 1], yd = row[p + 1] - row[p];
      float sa, sb, sc;
      weno5_pair(xd, yd, fwd, sa, sb, sc);
      sp0[c] = sa;
      sp1[c] = sb;
      sp2[c] = sc;
      d1[p] = xd;
      if (c == GW - 1) d1[p + 1] = yd;
    }
    group_sync(g);
    float D = 0.f;
    if (rv && c <= TX) {
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
    if (rv && cell) {
      const float F = row[c + 3];
      const float dphi = D + (phi[c + 1] - phi[c]);
      float out = F;
      if (a != 0.f) out = fmaf(a, ld_s<S>(Fn + (size_t)s * ld + x), b * F);
      out = fmaf(-cxi_tab[j], dphi, out);
      if (T.collide) {
        const float* pw = tabf + tabf_pw(Qxi) + j * (NV_MAX + 1);
        float feq = 0.f;
#pragma unroll
        for (int k = 0; k <= NVc; ++k) feq = fmaf(sm.Bf[i * (NV_MAX + 1) + k][c], pw[k], feq);
        const float rate = fmaf(-sm.rate[1][c], xi, sm.rate[0][c]);
        out = fmaf(rate, feq - F, out);
      }
      Fout[(size_t)s * ld + x] = to_s<S>(out);
    }
  }
}

template <typename S>
__global__ void __launch_bounds__(NT) rlb_stage_rp_kernel(StageArgsRP A) {
  extern __shared__ __align__(16) unsigned char stage_rp_smem_raw[];
  StageSmemRP& sm = *reinterpret_cast<StageSmemRP*>(stage_rp_smem_raw);
  const int2 tl = A.tiles[blockIdx.x];
  const TubeDev T = A.tubes[tl.x];
  if (T.Np == 2 && T.Nv == 5)
    stage_tile_rp<S, 2, 5>(A, T, tl.y, sm);
  else
    stage_tile_rp<S, NP_MAX, NV_MAX>(A, T, tl.y, sm);
}
