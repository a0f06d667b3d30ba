// Internal declarations of the CUDA library (not part of the public ABI).
#pragma once

#include <cstdint>

#ifndef __CUDACC__
#define __host__
#define __device__
#endif

namespace rlbq {
bool gauss_legendre(int n, double* x, double* w);
bool gauss_laguerre1(int n, double* x, double* w);
double laguerre1(int l, double x);  // L^(1)_l(x)
double legendre(int k, double x);   // P_k(x)
}  // namespace rlbq

namespace rlb {

// Compile-time maxima of the orders the kernels support.
constexpr int QP_MAX = 4;
constexpr int NP_MAX = 3;             // Np < Qp <= QP_MAX
constexpr int NV_MAX = 8;
constexpr int M_MAX = NP_MAX + 2;     // powers (1 - beta xi)^-m, m = 2 .. Np + 2
constexpr int QXI_MAX = 1024;
constexpr int R_MAX = 16383;          // longest series for the Legendre coefficients (|v| up to ~0.995)

// Per-tube description as the kernels see it.
struct TubeDev {
  int Qp, Qxi, Np, Nv;
  int bc;       // 0 open, 1 periodic
  int collide;  // 0: ballistic
  int Nx;       // cells
  int ld;       // row stride in doubles (padded)
  long long off;   // offset of row 0 of this tube in the state buffers
  long long xoff;  // offset of this tube's cells in the field layout
  double dx, dt, inv_tau;
  double x_left;
  int tab;      // offset of this tube's tables in the table buffer
  int index;    // position of the tube in the caller's list
  int tabf;     // offset of this tube's FP32 tables (reduced-precision storage)
  int storage;  // RLB_STORAGE_F64 / F32 / BF16
  long long poff;  // offset of this tube in the packed state layout (rows of Nx cells, tube after tube)
  double xi_max;      // largest |xi_j|
  double stiff_lim;   // rlb_stiffness_limit(xi_max dt / dx): dt gamma (1 + |beta| xi_max) / tau above it warns
};

// Layout of one tube's tables (doubles, starting at TubeDev::tab):
//   [0, QP_MAX)                 pbar_i
//   [QP_MAX, 2 QP_MAX)          pbar_i^2
//   [2 QP_MAX, 3 QP_MAX)        w^p_i
//   [3 QP_MAX, 3 QP_MAX + QP_MAX (NP_MAX+1))   K[i][q] = (-1)^q sum_{l=q}^{Np} C(l,q) L^(1)_l(pbar_i)
//                                               at [i (NP_MAX+1) + q]: the radial factor multiplying
//                                               s^(q+2) hhat_{q+2,k} in the truncated equilibrium
//   then xi_j (Qxi), then w^xi_j P_k(xi_j) at [j (NV_MAX+1) + k] (Qxi (NV_MAX+1)), zero for k > Nv,
//   then b_st dt xi_j / dx at [st Qxi + j] for the three Runge-Kutta stages, b = (1, 1/4, 2/3),
//   then per velocity s = i Qxi + j the WENO5 epsilon terms 3 eps ws^2 (C0, C1, C2) at [3 s + 0..2],
//   ws = w^p_i w^xi_j / 2 (the limiter acts on the weight-normalised population),
//   then per velocity s the term e = 3 eps ws^2 as a float pair (hi, lo) in the 8 bytes of slot s (the FP64
//   stage kernel's double-float limiter)
constexpr int TAB_PBAR = 0;
constexpr int TAB_PBAR2 = QP_MAX;
constexpr int TAB_WP = 2 * QP_MAX;
constexpr int TAB_K = 3 * QP_MAX;
constexpr int TAB_XI = TAB_K + QP_MAX * (NP_MAX + 1);
__host__ __device__ inline int tab_pw(int Qxi) { return TAB_XI + Qxi; }
__host__ __device__ inline int tab_cxi(int Qxi) { return TAB_XI + Qxi + Qxi * (NV_MAX + 1); }
__host__ __device__ inline int tab_eps(int Qxi) { return tab_cxi(Qxi) + 3 * Qxi; }
__host__ __device__ inline int tab_epsf(int Qp, int Qxi) { return tab_eps(Qxi) + 3 * Qp * Qxi; }
inline int tab_size(int Qp, int Qxi) { return tab_epsf(Qp, Qxi) + Qp * Qxi; }
// Per-tube FP32 table of the reduced-precision path (floats, starting at TubeDev::tabf): one record of
// RP_REC floats per velocity s = i Qxi + j, 16-byte aligned, read with vector loads:
//   R_XI          xi_j
//   R_CXI + st    b_st dt xi_j / dx for the three Runge-Kutta stages
//   R_IWS         1 / ws, ws = w^p_i w^xi_j / 2 (the WENO5 limiter acts on F / ws)
//   R_WS6         ws / 6
//   R_P1, R_P2    pbar_i and pbar_i^2 as hi/lo float pairs (moment weights)
//   R_X, R_X2     xi_j and xi_j^2 as hi/lo float pairs
//   R_PW + k      w^xi_j P_k(xi_j), k <= NV_MAX (zero above Nv)
constexpr int RP_REC = 24;
constexpr int R_XI = 0, R_CXI = 1, R_IWS = 4, R_WS6 = 5, R_P1 = 6, R_P2 = 8, R_X = 10, R_X2 = 12, R_PW = 14;
static_assert(R_PW + NV_MAX + 1 <= RP_REC, "record too small");
inline int tabf_size(int Qp, int Qxi) { return Qp * Qxi * RP_REC; }

constexpr double RK_A[3] = {0.0, 0.75, 1.0 / 3.0};  // Shu-Osher SSP-RK3: F_out = a F^n + b (F_in + dt L(F_in))
constexpr double RK_B[3] = {1.0, 0.25, 2.0 / 3.0};

}  // namespace rlb
