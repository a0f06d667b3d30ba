// Reduced-precision stage kernel: F stored in FP32 or BF16, advection, equilibrium evaluation, collision and
// the Runge-Kutta combination in FP32; the moments accumulated with compensated FP32 sums (double-float with
// double-float weights) and reduced in FP64; the Landau-frame solve and the equilibrium coefficients in FP64
// (the e, u^mu extraction cancels near |v| -> 1 and in rarefied cells). Included by rlb.cu inside its
// anonymous namespace.
//
// Built for instruction throughput and bandwidth rather than for the FP64 pipe:
//  - a warp holds RP_WT = 128 consecutive cells of a row, RP_C = 4 per lane in registers (one 16-byte load and
//    store per lane and row in FP32, 8 bytes in BF16), and advances the RP_OUT = 120 cells of lanes 1 .. 30:
//    lanes 0 and 31 hold the 4-cell halo on each side. Each lane forms the differences, WENO5 indicator pairs and
//    interface values it owns, once in the warp, takes the few it needs from its neighbours by shuffles, and
//    evaluates the collision and the Runge-Kutta combination without shared memory or barriers;
//  - the per-velocity constants are one 24-float record (vector loads, uniform over the warp);
//  - the moments of a stage's input are not re-read: the stage that wrote F_in accumulated them while
//    storing it and left 5 FP64 moments per cell (M_in); this stage does the same for F_out (M_out);
//  - the next row's loads are in flight while a row is evaluated, and F^n is loaded at the start of a row's
//    evaluation (it is needed only at its end);
//  - FP64 work is per cell only (Landau frame, Legendre series, equilibrium coefficients), kept by each lane
//    for its own cells in shared memory, where the lane also keeps its cells' five moment sums between
//    radial nodes (lane-private columns: no barrier).
// Rows are walked radial node by radial node, each node's directions in mirror pairs (xi, -xi), so that a pair
// shares its velocity record and the even and odd parts of its equilibrium, and the radial sums of a node are
// folded into the five moments once per node.
#pragma once

// Loads of the streamed state rows bypass L1 (ld.global.nc.L1::no_allocate): every row is read once per stage,
// and keeping it out of L1 leaves the little L1 that the shared-memory carveout spares to the per-velocity
// records and tables that every warp reads again and again.
__device__ __forceinline__ float ld_stream(const float* p) {
  float v;
  asm volatile("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ unsigned short ld_stream(const unsigned short* p) {
  unsigned short v;
  asm volatile("ld.global.nc.L1::no_allocate.u16 %0, [%1];" : "=h"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ float4 ld_stream4(const float* p) {
  float4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p));
  return v;
}
__device__ __forceinline__ uint2 ld_stream2(const void* p) {
  uint2 v;
  asm volatile("ld.global.nc.L1::no_allocate.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
  return v;
}

// The FP32 store of four consecutive values (16-byte aligned).
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }

constexpr int RP_C = 4;                   // cells per lane
constexpr int RP_WT = 32 * RP_C;          // cells a warp holds
constexpr int RP_OUT = RP_WT - 2 * RP_C;  // cells a warp tile advances: lanes 1 .. 30 (lanes 0 and 31 hold the halo)
constexpr int RP_WARPS = 4;               // warps per CTA, each on its own warp tile
constexpr int RP_NT = 32 * RP_WARPS;      // threads per CTA

struct StageArgsRP {
  const TubeDev* tubes;
  const int2* wtiles;  // warp tiles (tube, first cell), RP_OUT cells each
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

// Shared memory of one warp tile (lane-private columns 4 lane .. 4 lane + 3), rp_rows(brows) rows of RP_WT
// floats: the cells' FP32 equilibrium coefficients B[i][k] of radial node i at row rp_brow(i, k) (node 0's rows
// last), and their five moment sums as (hi, lo) float pairs M[f][cell] from node 0's first row on: node 0's
// coefficients are no longer read once M is first written (after node 0's walk), so M takes their place and
// RP_MEXTRA rows beyond them.
constexpr int RP_MEXTRA = 10 - 6;  // M's 10 float rows over the Nv + 1 >= 6 rows of node 0
__host__ __device__ constexpr int rp_rows(int brows) { return brows + RP_MEXTRA; }
__device__ __forceinline__ int rp_brow(int i, int k, int Qp, int nk) { return (i == 0 ? Qp - 1 : i - 1) * nk + k; }
struct RpWarp {
  float* B;
};
// Dynamic shared memory of a CTA for `brows` coefficient rows.
__host__ __device__ constexpr size_t rp_smem_bytes(int brows) {
  return (size_t)RP_WARPS * RP_WT * rp_rows(brows) * sizeof(float);
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
  double e, beta, n, Tt, gam;
  bool ok = landau(mom, e, beta, n, Tt, &gam);
  // flag[1] holds the sticky warning bits (RLB_WARN_*); the tube record is read from global memory here
  if (ok && flag != nullptr && stiff(*Tg, beta)) atomicOr(flag + 1, RLB_WARN_STIFF);
  if (ok && beta == 0.0) {
    // at rest hhat_{m,k} = delta_{k0}: only B[i][0] = n/(4T^3) w^p_i sum_q T^(q+2) K[i][q] is nonzero (the same
    // FP64 operations as the general path below takes at beta = 0)
    const double pref = n / (4.0 * Tt * Tt * Tt);
#pragma unroll
    for (int i = 0; i < QP_MAX; ++i) {
      if (i < Qp) {
        const double pw = pref * tab[TAB_WP + i];
        double B0 = 0.0, sq = Tt * Tt;
#pragma unroll
        for (int q = 0; q <= NPc; ++q) {
          const double G = pw * sq * tab[TAB_K + i * (NP_MAX + 1) + q];
          B0 = fma(G, 1.0, B0);
          sq *= Tt;
        }
        w.B[rp_brow(i, 0, Qp, NVc + 1) * RP_WT + col] = (float)B0;
#pragma unroll
        for (int k = 1; k <= NVc; ++k) w.B[rp_brow(i, k, Qp, NVc + 1) * RP_WT + col] = 0.f;
      }
    }
    rt0 = (float)bdt_itau;
    rt1 = 0.f;
    return;
  }
  double hh[(NPc + 1) * (NV_MAX + 1)];
#pragma unroll
  for (int k = 0; k < (NPc + 1) * (NV_MAX + 1); ++k) hh[k] = 0.0;
  if (ok) {
    const bool c0 = hhat_parity<NPc, NVc, 0, 1>(beta, hh);
    const bool c1 = hhat_parity<NPc, NVc, 1, 1>(beta, hh);
    ok = c0 && c1;
  }
  if (!ok && flag) atomicOr(flag, 1);
  const double s = ok ? Tt / gam : 0.0;
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
      for (int k = 0; k <= NVc; ++k) w.B[rp_brow(i, k, Qp, NVc + 1) * RP_WT + col] = (float)B[k];
    }
  }
  const double r0 = ok ? bdt_itau * gam : 0.0;
  rt0 = (float)r0;
  rt1 = (float)(r0 * beta);
}

// One velocity row as a lane holds it: its RP_C cells xl .. xl+3 (xl = x0 - RP_C + RP_C lane, so that lane 0
// holds the tile's left halo x0-4 .. x0-1 and lane 31 its right halo x0+RP_OUT .. +3), as stored: FP32 values,
// or BF16 values two to a word, widened (exactly) only where they are used, so that a warp does not wait for a
// load it issued a row ahead at the load itself.
template <typename S>
struct RpRow;
template <>
struct RpRow<float> {
  float v[RP_C];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int q = 0; q < RP_C; ++q) v[q] = 0.f;
  }
  __device__ __forceinline__ void ld4(const float* p) {
    const float4 t = ld_stream4(p);
    v[0] = t.x;
    v[1] = t.y;
    v[2] = t.z;
    v[3] = t.w;
  }
  __device__ __forceinline__ void ld1(int q, const float* p) { v[q] = ld_stream(p); }
  __device__ __forceinline__ void get(float (&o)[RP_C]) const {
#pragma unroll
    for (int q = 0; q < RP_C; ++q) o[q] = v[q];
  }
};
template <>
struct RpRow<__nv_bfloat16> {
  unsigned u[2];  // cells 0, 1 in u[0] and 2, 3 in u[1], the lower address in the low half
  __device__ __forceinline__ void zero() { u[0] = u[1] = 0u; }
  __device__ __forceinline__ void ld4(const __nv_bfloat16* p) {
    const uint2 t = ld_stream2(p);
    u[0] = t.x;
    u[1] = t.y;
  }
  __device__ __forceinline__ void ld1(int q, const __nv_bfloat16* p) {
    const unsigned h = ld_stream(reinterpret_cast<const unsigned short*>(p));
    u[q >> 1] = (q & 1) ? ((u[q >> 1] & 0xffffu) | (h << 16)) : ((u[q >> 1] & 0xffff0000u) | h);
  }
  __device__ __forceinline__ void get(float (&o)[RP_C]) const {
    o[0] = __uint_as_float(u[0] << 16);
    o[1] = __uint_as_float(u[0] & 0xffff0000u);
    o[2] = __uint_as_float(u[1] << 16);
    o[3] = __uint_as_float(u[1] & 0xffff0000u);
  }
};

// A row's cells: one vector load where the warp's 128 cells all lie inside the tube (full), otherwise one load
// per cell from its source under the boundary condition (positions left of -3 are never used and read -3).
template <typename S>
__device__ __forceinline__ void rp_load_row(RpRow<S>& r, const S* Fin, size_t row, int xl, bool full,
                                            const TubeDev& T) {
  const S* src = Fin + row;
  if (full) {
    r.ld4(src + xl);
  } else {
    r.zero();
#pragma unroll
    for (int q = 0; q < RP_C; ++q) r.ld1(q, src + map_cell(max(xl + q, -HALO), T.Nx, T.bc, T.ld));
  }
}

// F^n of a lane's cells (stages 2 and 3 only; output lanes only, whose cells are >= 0); fn starts zeroed.
template <typename S>
__device__ __forceinline__ void rp_load_fn(RpRow<S>& fn, const S* Fn, size_t row, int xl, bool full, int Nx,
                                           bool out) {
  const S* fs = Fn + row;
  if (!out) return;
  if (full) {
    fn.ld4(fs + xl);
  } else {
#pragma unroll
    for (int q = 0; q < RP_C; ++q)
      if (xl + q < Nx) fn.ld1(q, fs + xl + q);
  }
}

// The first and the last of rlbdev::weno5_pair's squares alone (fwd = true), with the same operations, so the
// same values: sA = (C0 (SL(x, y) + 3eps))^2 and sC = (C2 (SR(x, y) + 3eps))^2.
__device__ __forceinline__ float weno5_square_a(float x, float y) {
  using namespace rlbdev;
  const float qx = mul_x(x, x), pxy = mul_x(x, y), qy = mul_x(y, y);
  const float u = fmaf(float(4.0 * C0), qx, fmaf(float(-11.0 * C0), pxy, fmaf(float(10.0 * C0), qy, EPS_A)));
  return mul_x(u, u);
}
__device__ __forceinline__ float weno5_square_c(float x, float y) {
  using namespace rlbdev;
  const float qx = mul_x(x, x), pxy = mul_x(x, y), qy = mul_x(y, y);
  const float u = fmaf(float(10.0 * C2), qx, fmaf(float(-11.0 * C2), pxy, fmaf(float(4.0 * C2), qy, EPS_C)));
  return mul_x(u, u);
}

// Flux differences Phi(q + 1/2) - Phi(q - 1/2) of a lane's cells q = 0 .. RP_C-1 for a wind toward +x (FWD) or
// toward -x. Interface X lies between cells X-1 and X; its value is the upwind cell (X-1 toward +x, X toward -x)
// plus G, G from the three candidate stencils' indicators on the differences D(k) = F(k) - F(k-1) scaled by 1/ws
// (the limiter acts on F / ws): the combination of the scaled differences returns 6 G / ws, and the flux
// difference scales it back with ws6 = ws / 6 in its one FMA.
// Every pair of adjacent differences and every interface is evaluated once in the warp: a lane with cells
// xl .. xl+3 owns the differences D(xl .. xl+3), the pairs (D(k), D(k+1)) at k = xl .. xl+3 (toward +x) or
// xl+1 .. xl+4 (toward -x), and the interfaces xl+1 .. xl+4 (the right faces of its cells); what its
// interfaces need from beyond (one indicator square and up to three differences of a neighbour lane, and the
// interface xl from the left lane) comes by shuffles. Toward +x interface X takes the pairs at X-2 (sa), X-1
// (sb) and X (sc) and the differences D(X-2 .. X+1); toward -x the pairs at X+1 (sa), X (sb), X-1 (sc) and
// the differences -D(X+2 .. X-1) in wind order. The edge lanes' own outputs are wrong (no neighbour beyond) and
// unused: what lanes 1 and 30 take from them involves their own cells only.
template <bool FWD>
__device__ __forceinline__ void rp_flux_diff(const float (&f)[RP_C], float iws, float ws6, float (&dphi)[RP_C]) {
  constexpr unsigned ALL = 0xffffffffu;
  float D[RP_C], dd[RP_C];
  D[0] = __fsub_rn(f[0], __shfl_up_sync(ALL, f[3], 1));
#pragma unroll
  for (int q = 1; q < RP_C; ++q) D[q] = __fsub_rn(f[q], f[q - 1]);
#pragma unroll
  for (int q = 0; q < RP_C; ++q) dd[q] = __fmul_rn(D[q], iws);
  // D(xl+4), D(xl+5) (and toward -x D(xl+6)) from the right lane, scaled here as that lane scales them
  const float D4 = __shfl_down_sync(ALL, D[0], 1), D5 = __shfl_down_sync(ALL, D[1], 1);
  const float dd4 = __fmul_rn(D4, iws), dd5 = __fmul_rn(D5, iws);
  float sa[RP_C], sb[RP_C], sc[RP_C], G6[RP_C + 1];
  if (FWD) {
    const float ddn[RP_C + 1] = {dd[0], dd[1], dd[2], dd[3], dd4};
#pragma unroll
    for (int q = 0; q < RP_C; ++q)
      rlbdev::weno5_pair(ddn[q], ddn[q + 1], true, rlbdev::EPS_A, rlbdev::EPS_B, rlbdev::EPS_C, sa[q], sb[q], sc[q]);
    // the neighbours' indicator squares this lane needs, formed here from their differences as those lanes form
    // them (same operations, same values): sa of the pair at xl-1, sc of the pair at xl+4
    const float ddm1 = __shfl_up_sync(ALL, dd[3], 1);
    const float sam1 = weno5_square_a(ddm1, dd[0]), sc4 = weno5_square_c(dd4, dd5);
    G6[1] = rlbdev::weno5_combine6(sam1, sb[0], sc[1], ddm1, dd[0], dd[1], dd[2]);
    G6[2] = rlbdev::weno5_combine6(sa[0], sb[1], sc[2], dd[0], dd[1], dd[2], dd[3]);
    G6[3] = rlbdev::weno5_combine6(sa[1], sb[2], sc[3], dd[1], dd[2], dd[3], dd4);
    G6[4] = rlbdev::weno5_combine6(sa[2], sb[3], sc4, dd[2], dd[3], dd4, dd5);
  } else {
    const float D6 = __shfl_down_sync(ALL, D[2], 1);
    const float dd6 = __fmul_rn(D6, iws);
    const float ddn[RP_C + 2] = {dd[1], dd[2], dd[3], dd4, dd5, dd6};
    // pair q at k = xl+1+q, taken in wind order (D(k+1), D(k)): an indicator is even in the differences
#pragma unroll
    for (int q = 0; q < RP_C; ++q)
      rlbdev::weno5_pair(ddn[q + 1], ddn[q], true, rlbdev::EPS_A, rlbdev::EPS_B, rlbdev::EPS_C, sa[q], sb[q], sc[q]);
    // sc of the pair at xl and sa of the pair at xl+5, formed here as the neighbour lanes form them
    const float scm1 = weno5_square_c(dd[1], dd[0]), sa4 = weno5_square_a(dd6, dd5);
    G6[1] = rlbdev::weno5_combine6(sa[1], sb[0], scm1, -dd[3], -dd[2], -dd[1], -dd[0]);
    G6[2] = rlbdev::weno5_combine6(sa[2], sb[1], sc[0], -dd4, -dd[3], -dd[2], -dd[1]);
    G6[3] = rlbdev::weno5_combine6(sa[3], sb[2], sc[1], -dd5, -dd4, -dd[3], -dd[2]);
    G6[4] = rlbdev::weno5_combine6(sa4, sb[3], sc[2], -dd6, -dd5, -dd4, -dd[3]);
  }
  G6[0] = __shfl_up_sync(ALL, G6[4], 1);  // interface xl, the left lane's last
  // the upwind cells of interfaces q+1 and q differ by D(xl+q) toward +x and by D(xl+q+1) toward -x
#pragma unroll
  for (int q = 0; q < RP_C; ++q)
    dphi[q] = fmaf(__fsub_rn(G6[q + 1], G6[q]), ws6, FWD ? D[q] : (q + 1 < RP_C ? D[q + 1] : D4));
}

// Round a lane's four outputs to storage in place (the values the next stage reads and the moments sum) and store
// them if the lane is an output lane; BF16 rounds each pair of values with one packing conversion and stores the
// packed words.
__device__ __forceinline__ void rp_round_store(float (&v)[RP_C], float* dst, int xl, bool full, bool out, int Nx) {
  if (!out) return;
  if (full) {
    st4(dst + xl, make_float4(v[0], v[1], v[2], v[3]));
  } else {
#pragma unroll
    for (int q = 0; q < RP_C; ++q)
      if (xl + q < Nx) dst[xl + q] = v[q];
  }
}
__device__ __forceinline__ void rp_round_store(float (&v)[RP_C], __nv_bfloat16* dst, int xl, bool full, bool out,
                                               int Nx) {
  const __nv_bfloat162 p01 = __floats2bfloat162_rn(v[0], v[1]), p23 = __floats2bfloat162_rn(v[2], v[3]);
  const unsigned u01 = *reinterpret_cast<const unsigned*>(&p01), u23 = *reinterpret_cast<const unsigned*>(&p23);
  v[0] = __uint_as_float(u01 << 16);
  v[1] = __uint_as_float(u01 & 0xffff0000u);
  v[2] = __uint_as_float(u23 << 16);
  v[3] = __uint_as_float(u23 & 0xffff0000u);
  if (!out) return;
  if (full) {
    *reinterpret_cast<uint2*>(dst + xl) = make_uint2(u01, u23);
  } else {
    const unsigned short h[RP_C] = {(unsigned short)(u01 & 0xffffu), (unsigned short)(u01 >> 16),
                                    (unsigned short)(u23 & 0xffffu), (unsigned short)(u23 >> 16)};
#pragma unroll
    for (int q = 0; q < RP_C; ++q)
      if (xl + q < Nx) reinterpret_cast<unsigned short*>(dst)[xl + q] = h[q];
  }
}

// F_out = a F^n + b F - cxi dphi + rate (feq - F) of a lane's cells, rounded to storage and stored by the output
// lanes (out); returns the values in st.
template <typename S>
__device__ __forceinline__ void rp_finish(const StageArgsRP& A, const TubeDev& T, const float (&f)[RP_C],
                                          const float (&dphi)[RP_C], const RpRow<S>& fnr, float cxi,
                                          const float (&rt0)[RP_C], const float (&rt1)[RP_C], float xi,
                                          const float (&feq)[RP_C], S* dst, int xl, bool full, bool out,
                                          float (&st)[RP_C]) {
  float fn[RP_C];
  fnr.get(fn);
#pragma unroll
  for (int q = 0; q < RP_C; ++q) {
    const float F = f[q];
    float o = A.a != 0.f ? fmaf(A.a, fn[q], __fmul_rn(A.b, F)) : F;
    o = fmaf(-cxi, dphi[q], o);
    if (T.collide) o = fmaf(fmaf(-rt1[q], xi, rt0[q]), __fsub_rn(feq[q], F), o);
    st[q] = o;
  }
  rp_round_store(st, dst, xl, full, out, T.Nx);
}

// The compensated radial sums of one radial node i over the directions walked so far, per cell:
// S0 = sum_j F_ij, S1 = sum_j F_ij xi_j, S2 = sum_j F_ij xi_j^2 (double-float).
struct RpSums {
  rlbdev::DF s0[RP_C], s1[RP_C], s2[RP_C];
};

// Add a mirror pair of stored rows (xi, -xi) to the radial sums: with s = F(xi) + F(-xi) and d = F(xi) -
// F(-xi), both exact as float pairs, S0 += s, S1 += d xi, S2 += s xi^2.
__device__ __forceinline__ void rp_sums_pair(RpSums& S, const float (&sf)[RP_C], const float (&sb)[RP_C], float xh,
                                             float xl_, float x2h, float x2l) {
#pragma unroll
  for (int q = 0; q < RP_C; ++q) {
    float s, es, d, ed;
    rlbdev::two_sum(sf[q], sb[q], s, es);
    rlbdev::two_sum(sf[q], -sb[q], d, ed);
    rlbdev::df_add(S.s0[q], {s, es});
    rlbdev::df_add_dfprod(S.s1[q], {d, ed}, xh, xl_);
    rlbdev::df_add_dfprod(S.s2[q], {s, es}, x2h, x2l);
  }
}

// Fold the radial sums of node i into the five moments (double-float pairs M in the lane's shared columns):
// N0 += pbar S0, Nx += pbar S1, T00 += pbar^2 S0, T0x += pbar^2 S1, Txx += pbar^2 S2; the first fold starts from
// zero (M then still holds node 0's coefficients).
__device__ __forceinline__ void rp_fold(float2* M, int lane, bool first, const RpSums& S, float p1h, float p1l,
                                        float p2h, float p2l) {
#pragma unroll
  for (int f = 0; f < 5; ++f) {
    float4* mp = reinterpret_cast<float4*>(M + f * RP_WT + RP_C * lane);
    const float4 u0 = first ? make_float4(0.f, 0.f, 0.f, 0.f) : mp[0], u1 = first ? make_float4(0.f, 0.f, 0.f, 0.f) : mp[1];
    rlbdev::DF m[RP_C] = {{u0.x, u0.y}, {u0.z, u0.w}, {u1.x, u1.y}, {u1.z, u1.w}};
    const float wh = f < 2 ? p1h : p2h, wl = f < 2 ? p1l : p2l;
#pragma unroll
    for (int q = 0; q < RP_C; ++q) {
      const rlbdev::DF src = (f == 0 || f == 2) ? S.s0[q] : ((f == 1 || f == 3) ? S.s1[q] : S.s2[q]);
      rlbdev::df_add_dfprod(m[q], src, wh, wl);
    }
    mp[0] = make_float4(m[0].hi, m[0].lo, m[1].hi, m[1].lo);
    mp[1] = make_float4(m[2].hi, m[2].lo, m[3].hi, m[3].lo);
  }
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
  // the tile's output cells x0 .. x0 + RP_OUT - 1 belong to lanes 1 .. 30; lanes 0 and 31 hold the halo
  const int xl = x0 - RP_C + RP_C * lane;               // first cell of this lane
  const bool out = lane >= 1 && lane <= 30;
  const bool full = x0 >= RP_C && x0 - RP_C + RP_WT <= Nx;  // all the warp's cells inside the tube (uniform)

  // per-cell FP64 phase
  float rt0[RP_C], rt1[RP_C];
#pragma unroll
  for (int q = 0; q < RP_C; ++q) rt0[q] = rt1[q] = 0.f;
  if (T.collide) {
    const double bdt_itau = A.bd * T.dt * T.inv_tau;
#pragma unroll 1
    for (int q = 0; q < RP_C; ++q) {
      double mom[5] = {1.0, 0.0, 3.0, 0.0, 1.0};  // a rest state for the halo lanes and past the tube's end
      const bool own = out && xl + q < Nx;
      if (own) {
#pragma unroll
        for (int f = 0; f < 5; ++f) mom[f] = A.Min[f * A.nxtot + T.xoff + xl + q];
      }
      cell_coeffs_rp<NPc, NVc>(A.tubes + T.index, tab, Qp, mom, bdt_itau, own ? A.flag : nullptr, w,
                               RP_C * lane + q, rt0[q], rt1[q]);
    }
  }
  float2* const M = reinterpret_cast<float2*>(w.B + (size_t)rp_brow(0, 0, Qp, NVc + 1) * RP_WT);

  // Rows in the order i = 0 .. Qp-1 (outer), then the mirror pairs of directions (xi_jf > 0, xi_jb = -xi_jf),
  // jb = 0 .. Qxi/2 - 1, jf = Qxi - 1 - jb: row jf then row jb; an odd Qxi ends each radial node with its xi = 0
  // row. The next row's loads are in flight while a row is evaluated; the walk advances by increments (no
  // division by Qxi per row).
  const int hq = Qxi / 2;
  RpRow<S> ra, rb;
  rp_load_row<S>(ra, Fin, (size_t)(Qxi - 1) * ld, xl, full, T);  // the walk's first row
  // The record's second float4 (1/ws, ws/6), which the first row of a pair needs at once, is loaded one pair
  // ahead; the rest of the record is needed only after that row's flux differences, which cover its latency.
  float4 nr1 = rec[(size_t)(Qxi - 1) * (RP_REC / 4) + 1];
  for (int i = 0; i < Qp; ++i) {
    RpSums Sm;
#pragma unroll
    for (int q = 0; q < RP_C; ++q) Sm.s0[q] = Sm.s1[q] = Sm.s2[q] = {0.f, 0.f};
    const float* Bi = w.B + (size_t)rp_brow(i, 0, Qp, NVc + 1) * RP_WT + RP_C * lane;
    for (int jb = 0; jb < hq; ++jb) {
      const int jf = Qxi - 1 - jb;
      const int sf = i * Qxi + jf, sbk = i * Qxi + jb;
      rp_load_row<S>(rb, Fin, (size_t)sbk * ld, xl, full, T);  // the pair's second row
      // the pair's velocity record (of xi_jf > 0): xi, b dt xi/dx per stage, 1/ws, ws/6, moment weights,
      // w^xi P_k(xi)
      const float4* rp = rec + (size_t)sf * (RP_REC / 4);
      const float4 r1 = nr1;
      {
        const int sn = jb + 1 < hq ? sf - 1 : (i + 1 < Qp ? (i + 1) * Qxi + Qxi - 1 : sf);
        nr1 = rec[(size_t)sn * (RP_REC / 4) + 1];
      }
      const float4 r0 = rp[0], r2 = rp[2], r3 = rp[3], r4 = rp[4], r5 = rp[5];
      const float rv[RP_REC] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w, r2.x, r2.y, r2.z, r2.w,
                                r3.x, r3.y, r3.z, r3.w, r4.x, r4.y, r4.z, r4.w, r5.x, r5.y, r5.z, r5.w};
      const float xi = rv[R_XI], cxi = A.stage == 0 ? rv[R_CXI] : (A.stage == 1 ? rv[R_CXI + 1] : rv[R_CXI + 2]);
      const float iws = rv[R_IWS], ws6 = rv[R_WS6];
      float feq[RP_C], dphi[RP_C], stf[RP_C], stb[RP_C], fv[RP_C];
      // F^n of both rows, loaded now: a whole row's evaluation ahead of the second row's use
      RpRow<S> fn, fnb;
      fn.zero();
      fnb.zero();
      if (A.a != 0.f) {
        rp_load_fn<S>(fn, Fn, (size_t)sf * ld, xl, full, Nx, out);
        rp_load_fn<S>(fnb, Fn, (size_t)sbk * ld, xl, full, Nx, out);
      }
      // row jf: wind toward +x
      ra.get(fv);
      rp_flux_diff<true>(fv, iws, ws6, dphi);
      // even and odd Legendre parts of the pair's equilibria: feq(+xi) = E + O, feq(-xi) = E - O
      float E[RP_C] = {0.f, 0.f, 0.f, 0.f}, O[RP_C] = {0.f, 0.f, 0.f, 0.f};
      if (T.collide) {
#pragma unroll
        for (int kk = 0; kk <= NVc; ++kk) {
          const float4 b4 = *reinterpret_cast<const float4*>(Bi + kk * RP_WT);
          const float pk = rv[R_PW + kk];
          float* acc = (kk & 1) ? O : E;
          acc[0] = fmaf(b4.x, pk, acc[0]);
          acc[1] = fmaf(b4.y, pk, acc[1]);
          acc[2] = fmaf(b4.z, pk, acc[2]);
          acc[3] = fmaf(b4.w, pk, acc[3]);
        }
      }
#pragma unroll
      for (int q = 0; q < RP_C; ++q) feq[q] = __fadd_rn(E[q], O[q]);
      rp_finish<S>(A, T, fv, dphi, fn, cxi, rt0, rt1, xi, feq, Fout + (size_t)sf * ld, xl, full, out, stf);
      {
        const int snx = jb + 1 < hq ? sf - 1 : ((Qxi & 1) ? i * Qxi + hq : (i + 1) * Qxi + Qxi - 1);
        if (jb + 1 < hq || (Qxi & 1) || i + 1 < Qp) rp_load_row<S>(ra, Fin, (size_t)snx * ld, xl, full, T);
      }
      // row jb: wind toward -x
      rb.get(fv);
      rp_flux_diff<false>(fv, iws, ws6, dphi);
#pragma unroll
      for (int q = 0; q < RP_C; ++q) feq[q] = __fsub_rn(E[q], O[q]);
      rp_finish<S>(A, T, fv, dphi, fnb, -cxi, rt0, rt1, -xi, feq, Fout + (size_t)sbk * ld, xl, full, out, stb);
      if (T.collide) rp_sums_pair(Sm, stf, stb, rv[R_X], rv[R_X + 1], rv[R_X2], rv[R_X2 + 1]);
    }
    if (Qxi & 1) {  // the xi = 0 row: no advection; its equilibrium has only even Legendre terms
      const int sc = i * Qxi + hq;
      const float4* rp = rec + (size_t)sc * (RP_REC / 4);
      const float4 r3 = rp[3], r4 = rp[4], r5 = rp[5];
      const float pw[RP_REC - 12] = {r3.x, r3.y, r3.z, r3.w, r4.x, r4.y, r4.z, r4.w, r5.x, r5.y, r5.z, r5.w};
      float feq[RP_C] = {0.f, 0.f, 0.f, 0.f}, st[RP_C], fv[RP_C];
      const float zero[RP_C] = {0.f, 0.f, 0.f, 0.f};
      RpRow<S> fn;
      fn.zero();
      if (T.collide) {
#pragma unroll
        for (int kk = 0; kk <= NVc; kk += 2) {
          const float4 b4 = *reinterpret_cast<const float4*>(Bi + kk * RP_WT);
          const float pk = pw[R_PW - 12 + kk];
          feq[0] = fmaf(b4.x, pk, feq[0]);
          feq[1] = fmaf(b4.y, pk, feq[1]);
          feq[2] = fmaf(b4.z, pk, feq[2]);
          feq[3] = fmaf(b4.w, pk, feq[3]);
        }
      }
      if (A.a != 0.f) rp_load_fn<S>(fn, Fn, (size_t)sc * ld, xl, full, Nx, out);
      ra.get(fv);
      rp_finish<S>(A, T, fv, zero, fn, 0.f, rt0, rt1, 0.f, feq, Fout + (size_t)sc * ld, xl, full, out, st);
      if (i + 1 < Qp) rp_load_row<S>(ra, Fin, (size_t)((i + 1) * Qxi + Qxi - 1) * ld, xl, full, T);
      if (T.collide) {
#pragma unroll
        for (int q = 0; q < RP_C; ++q) rlbdev::df_add(Sm.s0[q], {st[q], 0.f});
      }
    }
    if (T.collide) {
      const float4 p = rec[(size_t)(i * Qxi) * (RP_REC / 4) + 1];  // R_P1 .. R_P2 + 1 of radial node i
      rp_fold(M, lane, i == 0, Sm, p.z, p.w, rec[(size_t)(i * Qxi) * (RP_REC / 4) + 2].x,
              rec[(size_t)(i * Qxi) * (RP_REC / 4) + 2].y);
    }
  }
  // FP64 moments of F_out for the next stage (collision tubes only)
  if (T.collide) {
#pragma unroll
    for (int q = 0; q < RP_C; ++q)
      if (out && xl + q < Nx) {
#pragma unroll
        for (int f = 0; f < 5; ++f) {
          const float2 m = M[f * RP_WT + RP_C * lane + q];
          A.Mout[f * A.nxtot + T.xoff + xl + q] = (double)m.x + (double)m.y;
        }
      }
  }
}

template <typename S, int SCHED>
__global__ void __launch_bounds__(RP_NT, 4) rlb_stage_rp_kernel(StageArgsRP A) {
  extern __shared__ __align__(16) float stage_rp_smem[];
  const int warp = threadIdx.x / 32;
  const RpWarp w{stage_rp_smem + (size_t)warp * RP_WT * rp_rows(A.brows)};
  auto run = [&](int wt) {
    const int2 tl = A.wtiles[wt];
    const TubeDev T = A.tubes[tl.x];
    if (T.Np == 2 && T.Nv == 5)
      warp_tile_rp<S, 2, 5>(A, T, tl.y, w);
    else
      warp_tile_rp<S, NP_MAX, NV_MAX>(A, T, tl.y, w);
  };
  if (SCHED == 2) {
    // counter schedule: every warp takes warp tiles one at a time, so that warps (not CTAs) finish unevenly at
    // the end of the launch; a warp's shared memory is lane-private, so no barrier separates its tiles
    for (;;) {
      int wt = 0;
      if ((threadIdx.x & 31) == 0) wt = atomicAdd(A.counter, 1);
      wt = __shfl_sync(0xffffffffu, wt, 0);
      if (wt >= A.nwt) return;
      run(wt);
    }
  }
  for_each_tile(A.ngroups, SCHED, A.counter, [&](int grp) {
    const int wt = grp * RP_WARPS + warp;
    if (wt < A.nwt) run(wt);  // uniform over the warp
  });
}
