// Reduced-precision stage kernel: F stored in FP32 or BF16, advection, equilibrium evaluation, collision and
// the Runge-Kutta combination in FP32; the moments accumulated with compensated FP32 sums (double-float with
// double-float weights) and reduced in FP64; the Landau-frame solve and the equilibrium coefficients in FP64
// (the e, u^mu extraction cancels near |v| -> 1 and in rarefied cells). Included by rlb.cu inside its
// anonymous namespace.
//
// Built for instruction throughput and bandwidth rather than for the FP64 pipe:
//  - a warp owns a tile of RP_WT = 128 cells and walks all velocity rows of it; each lane holds RP_C = 4
//    consecutive cells of a row in registers (one 16-byte load and store per lane and row in FP32, 8 bytes in
//    BF16), takes the three neighbour values on each side from the adjacent lanes by shuffles (the edge lanes
//    load the tile's halo, boundary condition applied) and evaluates its pairs of WENO5 indicators, its five
//    interface values, the collision and the Runge-Kutta combination without shared memory or barriers;
//  - the per-velocity constants are one 24-float record (six vector loads, uniform over the warp);
//  - the moments of a stage's input are not re-read: the stage that wrote F_in accumulated them while
//    storing it and left 5 FP64 moments per cell (M_in); this stage does the same for F_out (M_out);
//  - the next row's loads are in flight while a row is evaluated, and F^n is loaded at the start of a row's
//    evaluation (it is needed only at its end);
//  - FP64 work is per cell only (Landau frame, Legendre series, equilibrium coefficients), kept by each lane
//    for its own cells in shared memory, where the lane also keeps its cells' five moment sums between
//    directions (lane-private columns: no barrier).
// Rows are walked radial-innermost (j outer, i = 0 .. Qp-1 inner; s = i Qxi + j) so that the radial partial
// sums sum_i F pbar_i and sum_i F pbar_i^2 of one direction xi_j are folded into the five moments once per j.
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

// The value a float becomes once stored as S.
template <typename S>
__device__ __forceinline__ float rnd_s(float v);
template <>
__device__ __forceinline__ float rnd_s<float>(float v) {
  return v;
}
template <>
__device__ __forceinline__ float rnd_s<__nv_bfloat16>(float v) {
  return __bfloat162float(__float2bfloat16_rn(v));
}

// Four consecutive stored values (16-byte aligned in FP32, 8-byte aligned in BF16) and their store; the
// stored values are already representable in S.
__device__ __forceinline__ float4 ld4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ float4 ld4(const __nv_bfloat16* p) {
  const uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
  const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
  const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
  return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ void st4(__nv_bfloat16* p, float4 v) {
  const __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
  uint2 u;
  u.x = *reinterpret_cast<const unsigned*>(&a);
  u.y = *reinterpret_cast<const unsigned*>(&b);
  *reinterpret_cast<uint2*>(p) = u;
}
template <typename S>
__device__ __forceinline__ void st_s(S* p, float v);
template <>
__device__ __forceinline__ void st_s<float>(float* p, float v) {
  *p = v;
}
template <>
__device__ __forceinline__ void st_s<__nv_bfloat16>(__nv_bfloat16* p, float v) {
  *p = __float2bfloat16_rn(v);
}

constexpr int RP_C = 4;               // cells per lane
constexpr int RP_WT = 32 * RP_C;      // cells per warp tile
constexpr int RP_WARPS = 4;           // warps per CTA, each on its own warp tile
constexpr int RP_NT = 32 * RP_WARPS;  // threads per CTA

struct StageArgsRP {
  const TubeDev* tubes;
  const int2* wtiles;  // warp tiles (tube, first cell), RP_WT cells each
  int nwt;             // warp tiles
  const void* Fn;      // state at the start of the step (read at the cell only)
  const void* Fin;     // stage input (read with halo)
  void* Fout;          // stage output
  const double* Min;   // [5][nxtot] FP64 moments of Fin
  double* Mout;        // [5][nxtot] FP64 moments of Fout, written here
  long long nxtot;
  const double* tab;   // per-tube FP64 tables (as in the FP64 path)
  const float* tabf;   // per-tube FP32 velocity records
  int* flag;
  float a, b;          // Shu-Osher combination F_out = a F^n + b (F_in + dt L(F_in))
  double bd;           // b in FP64 (for the collision rate)
  int stage;
  int ngroups;         // CTA work items: groups of RP_WARPS consecutive warp tiles
  int schedule;        // as in the FP64 kernel
  int* counter;
  int brows;           // coefficient rows per warp region: max over the tubes of Qp (Nv + 1)
};

// Shared memory of one warp tile (lane-private columns 4 lane .. 4 lane + 3): the cells' FP32 equilibrium
// coefficients B[i (Nv + 1) + k][cell] (brows rows), then their five moment sums as (hi, lo) float pairs
// M[f][cell].
struct RpWarp {
  float* B;
  float2* M;
};
// Dynamic shared memory of a CTA for `brows` coefficient rows.
__host__ __device__ constexpr size_t rp_smem_bytes(int brows) {
  return (size_t)RP_WARPS * RP_WT * (brows + 10) * sizeof(float);
}
// Coefficient rows of a tube as the kernel stores them.
__host__ __device__ inline int rp_brows(int Qp, int Np, int Nv) { return Qp * ((Np == 2 && Nv == 5) ? 6 : NV_MAX + 1); }

// Per-cell FP64 phase of one cell: Landau frame of the stored moments, hhat_{m,k} by the positive power
// series (both parities, in registers), B[i][k] = n/(4T^3) w^p_i sum_q s^(q+2) K[i][q] hhat_{q+2,k} (as the
// FP64 kernel's tile_coeffs) stored as FP32 in column `col`, and the stage's collision rate
// b dt gamma (1 - beta xi)/tau = rt0 - rt1 xi. A non-physical cell raises the flag and gets B = 0, rate 0.
template <int NPc, int NVc>
__device__ void cell_coeffs_rp(const TubeDev* Tg, const double* tab, int Qp, const double mom[5], double bdt_itau,
                               int* flag, const RpWarp& w, int col, float& rt0, float& rt1) {
  double e, beta, n, Tt;
  bool ok = landau(mom, e, beta, n, Tt);
  // flag[1] holds the sticky warning bits (RLB_WARN_*); the tube record is read from global memory here
  if (ok && flag != nullptr && stiff(*Tg, beta)) atomicOr(flag + 1, RLB_WARN_STIFF);
  double hh[(NPc + 1) * (NV_MAX + 1)];
#pragma unroll
  for (int k = 0; k < (NPc + 1) * (NV_MAX + 1); ++k) hh[k] = 0.0;
  if (ok) {
    if (beta == 0.0) {
#pragma unroll
      for (int m = 0; m <= NPc; ++m) hh[m * (NV_MAX + 1)] = 1.0;
    } else {
      const bool c0 = hhat_parity<NPc, NVc, 0, 1>(beta, hh);
      const bool c1 = hhat_parity<NPc, NVc, 1, 1>(beta, hh);
      ok = c0 && c1;
    }
  }
  if (!ok && flag) atomicOr(flag, 1);
  const double s = ok ? Tt * sqrt(1.0 - beta * beta) : 0.0;
#pragma unroll
  for (int i = 0; i < QP_MAX; ++i) {
    double B[NVc + 1];
#pragma unroll
    for (int k = 0; k <= NVc; ++k) B[k] = 0.0;
    if (ok && i < Qp) {
      const double pref = n / (4.0 * Tt * Tt * Tt) * tab[TAB_WP + i];
      double sq = s * s;
#pragma unroll
      for (int q = 0; q <= NPc; ++q) {
        const double G = pref * sq * tab[TAB_K + i * (NP_MAX + 1) + q];
#pragma unroll
        for (int k = 0; k <= NVc; ++k) B[k] = fma(G, hh[q * (NV_MAX + 1) + k], B[k]);
        sq *= s;
      }
    }
    if (i < Qp) {
#pragma unroll
      for (int k = 0; k <= NVc; ++k) w.B[(i * (NVc + 1) + k) * RP_WT + col] = (float)B[k];
    }
  }
  const double r0 = ok ? bdt_itau / sqrt(1.0 - beta * beta) : 0.0;
  rt0 = (float)r0;
  rt1 = (float)(r0 * beta);
}

// One velocity row as a lane holds it: its RP_C cells and the tile's halo (edge lanes only).
struct RpRow {
  float v[RP_C];
  float h[3];
};

template <typename S>
__device__ __forceinline__ void rp_load_row(RpRow& r, const S* Fin, size_t row, int xl, bool full,
                                            const int (&csrc)[RP_C], bool edge, const int (&hsrc)[3]) {
  const S* src = Fin + row;
  if (full) {
    const float4 t = ld4(src + xl);
    r.v[0] = t.x;
    r.v[1] = t.y;
    r.v[2] = t.z;
    r.v[3] = t.w;
  } else {
#pragma unroll
    for (int q = 0; q < RP_C; ++q) r.v[q] = ld_s<S>(src + csrc[q]);
  }
#pragma unroll
  for (int h = 0; h < 3; ++h) r.h[h] = edge ? ld_s<S>(src + hsrc[h]) : 0.f;
}

// Radial partial sums of the current direction for a lane's cells (the five moments are in shared memory).
struct RpMom {
  rlbdev::DF ra[RP_C], rb[RP_C];
};

// One velocity row s = i Qxi + j of a lane's RP_C cells: F_out = a F^n + b (F + dt L(F)), stored; with
// collisions, the stored values enter the moment sums.
template <typename S, int NVc>
__device__ __forceinline__ void rp_row(const StageArgsRP& A, const TubeDev& T, const float4* rec, const RpWarp& w,
                                       const RpRow& r, int i, int j, int s, int lane, int xl, bool full,
                                       const float (&rt0)[RP_C], const float (&rt1)[RP_C], const S* Fn, S* Fout,
                                       RpMom& mo) {
  constexpr unsigned ALL = 0xffffffffu;
  const int Qxi = T.Qxi;
  // F^n at the lane's cells, issued first so that the WENO5 arithmetic below covers its latency
  float fn[RP_C] = {0.f, 0.f, 0.f, 0.f};
  if (A.a != 0.f) {
    const S* fs = Fn + (size_t)s * T.ld;
    if (full) {
      const float4 t = ld4(fs + xl);
      fn[0] = t.x;
      fn[1] = t.y;
      fn[2] = t.z;
      fn[3] = t.w;
    } else {
#pragma unroll
      for (int q = 0; q < RP_C; ++q) fn[q] = (xl + q < T.Nx) ? ld_s<S>(fs + xl + q) : 0.f;
    }
  }
  // the velocity's record: xi, b dt xi/dx of this stage, 1/ws, 6/ws, moment weights, w^xi P_k(xi)
  const float4* rp = rec + (size_t)s * (RP_REC / 4);
  const float4 r0 = rp[0], r1 = rp[1], r2 = rp[2], r3 = rp[3], r4 = rp[4], r5 = rp[5];
  const float rv[RP_REC] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w, r2.x, r2.y, r2.z, r2.w,
                            r3.x, r3.y, r3.z, r3.w, r4.x, r4.y, r4.z, r4.w, r5.x, r5.y, r5.z, r5.w};
  const float xi = rv[R_XI], cxi = A.stage == 0 ? rv[R_CXI] : (A.stage == 1 ? rv[R_CXI + 1] : rv[R_CXI + 2]);
  const float iws = rv[R_IWS], c6 = rv[R_C6];
  const bool fwd = xi > 0.f;
  // window of positions -3 .. 6 around the lane's cells 0 .. 3
  float wv[10];
  const float l1 = __shfl_up_sync(ALL, r.v[1], 1), l2 = __shfl_up_sync(ALL, r.v[2], 1),
              l3 = __shfl_up_sync(ALL, r.v[3], 1);
  const float q0 = __shfl_down_sync(ALL, r.v[0], 1), q1 = __shfl_down_sync(ALL, r.v[1], 1),
              q2 = __shfl_down_sync(ALL, r.v[2], 1);
  wv[0] = lane == 0 ? r.h[0] : l1;
  wv[1] = lane == 0 ? r.h[1] : l2;
  wv[2] = lane == 0 ? r.h[2] : l3;
#pragma unroll
  for (int q = 0; q < RP_C; ++q) wv[3 + q] = r.v[q];
  wv[7] = lane == 31 ? r.h[0] : q0;
  wv[8] = lane == 31 ? r.h[1] : q1;
  wv[9] = lane == 31 ? r.h[2] : q2;
  // differences scaled by 1/ws: dd[k] = (w(p) - w(p-1)) / ws at position p = k - 2, k = 0 .. 8
  float dd[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) dd[k] = (wv[k + 1] - wv[k]) * iws;
  // indicator squares of the seven pairs the five interfaces X = 0..4 (between cells X-1 and X) use:
  // pair t = (dd[t], dd[t+1]) toward +x, (dd[t+1], dd[t+2]) toward -x
  float sa[7], sb[7], sc[7];
#pragma unroll
  for (int t = 0; t < 7; ++t) {
    const float x = fwd ? dd[t] : dd[t + 1], y = fwd ? dd[t + 1] : dd[t + 2];
    rlbdev::weno5_pair(x, y, fwd, rlbdev::EPS_A, rlbdev::EPS_B, rlbdev::EPS_C, sa[t], sb[t], sc[t]);
  }
  float G[5];
#pragma unroll
  for (int X = 0; X < 5; ++X) {
    if (fwd)
      G[X] = rlbdev::weno5_combine_scaled(sa[X], sb[X + 1], sc[X + 2], dd[X], dd[X + 1], dd[X + 2], dd[X + 3], c6);
    else
      G[X] = rlbdev::weno5_combine_scaled(sa[X + 2], sb[X + 1], sc[X], -dd[X + 4], -dd[X + 3], -dd[X + 2],
                                          -dd[X + 1], c6);
  }
  // combination, collision, store
  float out[RP_C];
#pragma unroll
  for (int q = 0; q < RP_C; ++q) {
    const float F = wv[3 + q];
    const float up = fwd ? F - wv[2 + q] : wv[4 + q] - F;  // v2(X = q + 1) - v2(X = q)
    const float dphi = up + (G[q + 1] - G[q]);
    float o = A.a != 0.f ? fmaf(A.a, fn[q], A.b * F) : F;
    o = fmaf(-cxi, dphi, o);
    out[q] = o;
  }
  if (T.collide) {
    float feq[RP_C] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k <= NVc; ++k) {
      const float4 b4 = *reinterpret_cast<const float4*>(w.B + (i * (NVc + 1) + k) * RP_WT + RP_C * lane);
      const float pk = rv[R_PW + k];
      feq[0] = fmaf(b4.x, pk, feq[0]);
      feq[1] = fmaf(b4.y, pk, feq[1]);
      feq[2] = fmaf(b4.z, pk, feq[2]);
      feq[3] = fmaf(b4.w, pk, feq[3]);
    }
#pragma unroll
    for (int q = 0; q < RP_C; ++q) {
      const float rate = fmaf(-rt1[q], xi, rt0[q]);
      out[q] = fmaf(rate, feq[q] - wv[3 + q], out[q]);
    }
  }
  float st[RP_C];
#pragma unroll
  for (int q = 0; q < RP_C; ++q) st[q] = rnd_s<S>(out[q]);
  S* dst = Fout + (size_t)s * T.ld;
  if (full) {
    st4(dst + xl, make_float4(st[0], st[1], st[2], st[3]));
  } else {
#pragma unroll
    for (int q = 0; q < RP_C; ++q)
      if (xl + q < T.Nx) st_s<S>(dst + xl + q, st[q]);
  }
  if (T.collide) {
    // moments of what was stored: radial partial sums, folded into the five moments per direction
#pragma unroll
    for (int q = 0; q < RP_C; ++q) {
      rlbdev::df_add_prod(mo.ra[q], st[q], rv[R_P1], rv[R_P1 + 1]);
      rlbdev::df_add_prod(mo.rb[q], st[q], rv[R_P2], rv[R_P2 + 1]);
    }
    if (i == T.Qp - 1) {
#pragma unroll
      for (int f = 0; f < 5; ++f) {
        float4* mp = reinterpret_cast<float4*>(w.M + f * RP_WT + RP_C * lane);
        const float4 u0 = mp[0], u1 = mp[1];
        rlbdev::DF m[RP_C] = {{u0.x, u0.y}, {u0.z, u0.w}, {u1.x, u1.y}, {u1.z, u1.w}};
#pragma unroll
        for (int q = 0; q < RP_C; ++q) {
          if (f == 0) rlbdev::df_add(m[q], mo.ra[q]);
          if (f == 1) rlbdev::df_add_dfprod(m[q], mo.ra[q], rv[R_X], rv[R_X + 1]);
          if (f == 2) rlbdev::df_add(m[q], mo.rb[q]);
          if (f == 3) rlbdev::df_add_dfprod(m[q], mo.rb[q], rv[R_X], rv[R_X + 1]);
          if (f == 4) rlbdev::df_add_dfprod(m[q], mo.rb[q], rv[R_X2], rv[R_X2 + 1]);
        }
        mp[0] = make_float4(m[0].hi, m[0].lo, m[1].hi, m[1].lo);
        mp[1] = make_float4(m[2].hi, m[2].lo, m[3].hi, m[3].lo);
      }
#pragma unroll
      for (int q = 0; q < RP_C; ++q) {
        mo.ra[q] = {0.f, 0.f};
        mo.rb[q] = {0.f, 0.f};
      }
    }
  }
  (void)j;
  (void)Qxi;
}

template <typename S, int NPc, int NVc>
__device__ void warp_tile_rp(const StageArgsRP& A, const TubeDev& T, int x0, const RpWarp& w) {
  const int lane = threadIdx.x & 31;
  const double* tab = A.tab + T.tab;
  const float4* rec = reinterpret_cast<const float4*>(A.tabf + T.tabf);
  const int Qp = T.Qp, Qxi = T.Qxi, Nx = T.Nx, ld = T.ld;
  const S* Fin = static_cast<const S*>(A.Fin) + T.off;
  const S* Fn = static_cast<const S*>(A.Fn) + T.off;
  S* Fout = static_cast<S*>(A.Fout) + T.off;
  const int xl = x0 + RP_C * lane;            // first cell of this lane
  const bool full = x0 + RP_WT <= Nx;         // uniform over the warp
  // sources of the halo (lane 0: x0-3 .. x0-1, lane 31: x0+RP_WT .. +2) and, for a partial tile, of the lane's
  // positions: boundary condition applied, always inside [0, Nx)
  const bool edge = lane == 0 || lane == 31;
  int hsrc[3], csrc[RP_C];
#pragma unroll
  for (int h = 0; h < 3; ++h) hsrc[h] = map_cell(lane == 0 ? x0 - 3 + h : x0 + RP_WT + h, Nx, T.bc);
#pragma unroll
  for (int q = 0; q < RP_C; ++q) csrc[q] = map_cell(xl + q, Nx, T.bc);

  // per-cell FP64 phase
  float rt0[RP_C], rt1[RP_C];
#pragma unroll
  for (int q = 0; q < RP_C; ++q) rt0[q] = rt1[q] = 0.f;
  if (T.collide) {
    const double bdt_itau = A.bd * T.dt * T.inv_tau;
#pragma unroll 1
    for (int q = 0; q < RP_C; ++q) {
      double mom[5] = {1.0, 0.0, 3.0, 0.0, 1.0};  // a rest state for positions past the tube's end
      if (xl + q < Nx) {
#pragma unroll
        for (int f = 0; f < 5; ++f) mom[f] = A.Min[f * A.nxtot + T.xoff + xl + q];
      }
      cell_coeffs_rp<NPc, NVc>(A.tubes + T.index, tab, Qp, mom, bdt_itau, xl + q < Nx ? A.flag : nullptr,
                               w, RP_C * lane + q, rt0[q], rt1[q]);
    }
  }

  RpMom mo;
#pragma unroll
  for (int q = 0; q < RP_C; ++q) {
    mo.ra[q] = mo.rb[q] = {0.f, 0.f};
#pragma unroll
    for (int f = 0; f < 5; ++f) w.M[f * RP_WT + RP_C * lane + q] = make_float2(0.f, 0.f);
  }
  // rows in the order j = 0.., i = 0..Qp-1; two rows in flight
  const int Q = Qp * Qxi;
  RpRow ra_, rb_;
  int ia = 0, ja = 0;  // row held in ra_
  rp_load_row<S>(ra_, Fin, (size_t)(ia * Qxi + ja) * ld, xl, full, csrc, edge, hsrc);
  int ib = Qp > 1 ? 1 : 0, jb = Qp > 1 ? 0 : 1;  // row held in rb_
  if (Q > 1) rp_load_row<S>(rb_, Fin, (size_t)(ib * Qxi + jb) * ld, xl, full, csrc, edge, hsrc);
  auto advance2 = [&](int& i, int& j) {  // two rows further along the walk
#pragma unroll
    for (int u = 0; u < 2; ++u)
      if (++i == Qp) {
        i = 0;
        ++j;
      }
  };
  for (int r = 0; r < Q; r += 2) {
    rp_row<S, NVc>(A, T, rec, w, ra_, ia, ja, ia * Qxi + ja, lane, xl, full, rt0, rt1, Fn, Fout, mo);
    advance2(ia, ja);
    if (r + 2 < Q) rp_load_row<S>(ra_, Fin, (size_t)(ia * Qxi + ja) * ld, xl, full, csrc, edge, hsrc);
    if (r + 1 < Q) {
      rp_row<S, NVc>(A, T, rec, w, rb_, ib, jb, ib * Qxi + jb, lane, xl, full, rt0, rt1, Fn, Fout, mo);
      advance2(ib, jb);
      if (r + 3 < Q) rp_load_row<S>(rb_, Fin, (size_t)(ib * Qxi + jb) * ld, xl, full, csrc, edge, hsrc);
    }
  }
  // FP64 moments of F_out for the next stage (collision tubes only)
  if (T.collide) {
#pragma unroll
    for (int q = 0; q < RP_C; ++q)
      if (xl + q < Nx) {
#pragma unroll
        for (int f = 0; f < 5; ++f) {
          const float2 m = w.M[f * RP_WT + RP_C * lane + q];
          A.Mout[f * A.nxtot + T.xoff + xl + q] = (double)m.x + (double)m.y;
        }
      }
  }
}

template <typename S, int SCHED>
__global__ void __launch_bounds__(RP_NT, 4) rlb_stage_rp_kernel(StageArgsRP A) {
  extern __shared__ __align__(16) float stage_rp_smem[];
  const int warp = threadIdx.x / 32;
  float* base = stage_rp_smem + (size_t)warp * RP_WT * (A.brows + 10);
  const RpWarp w{base, reinterpret_cast<float2*>(base + (size_t)RP_WT * A.brows)};
  for_each_tile(A.ngroups, SCHED, A.counter, [&](int grp) {
    const int wt = grp * RP_WARPS + warp;
    if (wt < A.nwt) {  // uniform over the warp
      const int2 tl = A.wtiles[wt];
      const TubeDev T = A.tubes[tl.x];
      if (T.Np == 2 && T.Nv == 5)
        warp_tile_rp<S, 2, 5>(A, T, tl.y, w);
      else
        warp_tile_rp<S, NP_MAX, NV_MAX>(A, T, tl.y, w);
    }
  });
}
