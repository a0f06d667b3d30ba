// GB300 (sm_103a) CUDA implementation of the time step of the quadrature-based finite-difference
// relativistic lattice Boltzmann model for massless particles (Blaga & Ambrus, arXiv:1608.03004), and
// its C ABI (include/rlb.h).
//
// One SSP-RK3 stage is one launch of rlb_stage_kernel over every tile of every tube. A CTA owns a tile of
// TX = 61 cells of one tube and, for those cells:
//   A. reduces F over all Q velocities to N^0, N^x, T^00, T^0x, T^xx (section "Relativistic lattice
//      Boltzmann equation");
//   B. solves the Landau-frame eigenproblem T^mu_nu u^nu = -e u^mu for e, v, n and builds the per-cell
//      coefficients of the truncated equilibrium of Eq. (feqtrunc);
//   C. lets each of its four 64-thread groups walk mirror pairs of directions (xi_j, -xi_j) of one radial
//      node: stages a row (tile + 3-cell halo, boundary condition folded into the load) in shared memory with
//      its first differences and their squares, evaluates the WENO5 smoothness indicators once per pair of
//      adjacent differences, combines three pairs into each of the 62 interface values and writes
//      F_out = a F^n + b (F_in + dt L(F_in)), L = advection + Anderson-Witting collision (Eq. (Boltz)); the
//      even and odd Legendre parts of the equilibrium serve both rows of a pair.
// Tiles that cannot fill the GPU are split over several CTAs by velocity rows (StageArgs::split). The FP64
// path is FP64 throughout; on GB300 the FP64 pipe (about 2 DFMA per SM per clock) bounds it, so the
// arithmetic is arranged to spend as few FP64 instructions per velocity-node update as possible. The FP64
// stage kernel and its shared device helpers (rlb_stage.cuh), the reduced-precision kernel (rlb_stage_rp.cuh)
// and the adjoint (rlb_adjoint.cuh) are included below; this file holds the remaining kernels and the host
// side.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstddef>
#include <complex>
#include <cstring>
#include <map>
#include <mutex>
#include <type_traits>
#include <new>
#include <utility>
#include <vector>

#include "../../include/rlb.h"
#include "rlb_device_math.cuh"
#include "rlb_internal.h"

using namespace rlb;
using rlbdev::weno5_combine;
using rlbdev::weno5_pair;

namespace {

#include "rlb_stage.cuh"

#include "rlb_stage_rp.cuh"

// --------------------------------------------------------------------------------------------------
// Initial condition and fields
// --------------------------------------------------------------------------------------------------

// FP64 view of a stored population and its rounding back (storage type S = double, float, bf16)
template <typename S>
__device__ __forceinline__ double ld_d(const S* p) {
  return (double)*p;
}
template <>
__device__ __forceinline__ double ld_d<__nv_bfloat16>(const __nv_bfloat16* p) {
  return (double)__bfloat162float(*p);
}
template <typename S>
__device__ __forceinline__ void st_d(S* p, double v) {
  *p = (S)v;
}
template <>
__device__ __forceinline__ void st_d<__nv_bfloat16>(__nv_bfloat16* p, double v) {
  *p = __double2bfloat16(v);
}

struct InitArgs {
  const TubeDev* tubes;
  const int2* tiles;
  void* F;            // storage type of the handle
  const double* tab;
  const double* P;      // per-cell state (field layout) or NULL
  const double* n;
  const double* v;
  const double* riem;   // per-tube (P_L, n_L, v_L, P_R, n_R, v_R) or NULL
  int* flag;
};

struct InitSmem {
  CoefSmem coef;
  double B[NBC][GW];
  int tie;
};

// Write F = F^eq of the cells' states (pass 0), or average the right-state equilibrium into the cells that
// sit exactly on the membrane (pass 1).
template <typename S, int NVc>
__device__ void init_write(const TubeDev& T, const double* tab, const InitSmem& sm, S* F, int x0, bool pass1,
                           bool tie) {
  const int c = threadIdx.x % GW, g = threadIdx.x / GW, x = x0 + c;
  if (c >= TX || x >= T.Nx || (pass1 && !tie)) return;
  const int Q = T.Qp * T.Qxi;
  for (int s = g; s < Q; s += NG) {
    const int i = s / T.Qxi, j = s - i * T.Qxi;
    const double* pw = tab + TAB_XI + T.Qxi + j * (NV_MAX + 1);
    double f = 0.0;
#pragma unroll
    for (int k = 0; k <= NVc; ++k) f = fma(sm.B[i * (NVc + 1) + k][c], pw[k], f);
    S* dst = F + T.off + (size_t)s * T.ld + x;
    st_d<S>(dst, pass1 ? 0.5 * (ld_d<S>(dst) + f) : f);
  }
}

template <typename S, int NPc, int NVc>
__device__ void init_tile(const InitArgs& A, const TubeDev& T, int x0, InitSmem& sm) {
  const int c = threadIdx.x % GW, g = threadIdx.x / GW, x = x0 + c;
  const double* tab = A.tab + T.tab;
  const bool cell = c < TX && x < T.Nx;
  // Riemann data: side of the membrane from the cell centre, evaluated without contraction so that it
  // matches plain IEEE arithmetic; a centre exactly on x = 0 gets the mean of both equilibria.
  const double xc = __dadd_rn(T.x_left, __dmul_rn((double)x + 0.5, T.dx));
  const bool tie = cell && A.riem != nullptr && xc == 0.0;
  if (threadIdx.x == 0) sm.tie = 0;
  __syncthreads();
  if (tie) sm.tie = 1;
  for (int pass = 0; pass < 2; ++pass) {
    if (g == 0) {
      double P = 1.0, n = 1.0, v = 0.0;
      if (A.riem == nullptr) {
        if (cell) {
          const size_t k = (size_t)T.xoff + x;
          P = A.P[k];
          n = A.n[k];
          v = A.v[k];
        }
      } else {
        const double* st = A.riem + 6 * T.index + ((pass == 1 || xc > 0.0) ? 3 : 0);
        P = st[0];
        n = st[1];
        v = st[2];
      }
      const bool ok = P > 0.0 && n > 0.0 && fabs(v) < 1.0;
      if (cell && !ok) atomicOr(A.flag, 1);
      sm.coef.cell[0][c] = n;
      sm.coef.cell[1][c] = P / n;
      sm.coef.cell[2][c] = v;
      sm.coef.ok[c] = (cell && ok) ? 1 : 0;
    }
    __syncthreads();
    if (pass == 1 && sm.tie == 0) break;  // uniform over the CTA
    tile_coeffs<NPc, NVc>(tab, T.Qp, sm.coef, sm.B, A.flag);
    init_write<S, NVc>(T, tab, sm, static_cast<S*>(A.F), x0, pass == 1, tie);
    __syncthreads();
  }
}

template <typename S>
__global__ void __launch_bounds__(NT) rlb_init_kernel(InitArgs A) {
  __shared__ InitSmem sm;
  const int2 tl = A.tiles[blockIdx.x];
  const TubeDev T = A.tubes[tl.x];
  if (T.Np == 2 && T.Nv == 5)
    init_tile<S, 2, 5>(A, T, tl.y, sm);
  else
    init_tile<S, NP_MAX, NV_MAX>(A, T, tl.y, sm);
}

// Fields of every cell: the five moments summed over F in FP64, or, with M != NULL, read from M for tubes with
// collisions (reduced storage: the stage kernel leaves the FP64 moments of its output there, so F need not be
// read again; ballistic tubes keep no moments and are summed), then the Landau frame.
template <typename S>
__global__ void __launch_bounds__(GW) rlb_fields_kernel(const TubeDev* tubes, const int2* tiles, const void* Fv,
                                                         const double* tabs, double* out, long long nxtot,
                                                         int* flag, const double* M = nullptr) {
  const S* F = static_cast<const S*>(Fv);
  const int2 tl = tiles[blockIdx.x];
  const TubeDev T = tubes[tl.x];
  const int c = threadIdx.x, x = tl.y + c;
  if (c >= TX || x >= T.Nx) return;
  const double* tab = tabs + T.tab;
  const S* f = F + T.off + x;
  double mom[5] = {0, 0, 0, 0, 0};
  if (M != nullptr && T.collide) {
#pragma unroll
    for (int k = 0; k < 5; ++k) mom[k] = M[k * nxtot + T.xoff + x];
  }
  for (int j = 0; j < ((M != nullptr && T.collide) ? 0 : T.Qxi); ++j) {
    double a = 0.0, b = 0.0;
    for (int i = 0; i < T.Qp; ++i) {
      const double v = ld_d<S>(f + (size_t)(i * T.Qxi + j) * T.ld);
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
  double e, beta, n, Tt;
  if (!landau(mom, e, beta, n, Tt)) atomicOr(flag, 1);
  double* o = out + T.xoff + x;
#pragma unroll
  for (int k = 0; k < 5; ++k) o[k * nxtot] = mom[k];
  o[5 * nxtot] = e;
  o[6 * nxtot] = beta;
  o[7 * nxtot] = n;
}

// Packed FP64 <-> stored state of one tube (rows x Nx, stored rows have stride ld).
template <typename S>
__global__ void widen_kernel(const S* src, int ld, double* dst, int Nx) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
  if (x < Nx) dst[(size_t)r * Nx + x] = ld_d<S>(src + (size_t)r * ld + x);
}
template <typename S>
__global__ void narrow_kernel(const double* src, S* dst, int ld, int Nx) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
  if (x < Nx) st_d<S>(dst + (size_t)r * ld + x, src[(size_t)r * Nx + x]);
}

// Exchange blocks of the slabs of a decomposed tube: one block of Q x 3 cells per halo side (left first), row
// by row. pack: the slab's edge cells (0..2 on the left, Nx-3..Nx-1 on the right) into buf; unpack: buf into the
// ghost cells beside each row (left ghosts -3..-1 at ld-3..ld-1, right ghosts Nx..Nx+2). Grid: x over the
// 2 Q 3 cells of a slab's blocks, y over the slabs.
struct HaloDesc {
  int tube;
  int bc;          // RLB_BC_HALO_LEFT and/or RLB_BC_HALO_RIGHT
  long long off;   // first element of the slab's blocks in the buffer
};

template <typename S, bool PACK>
__global__ void halo_kernel(const HaloDesc* hd, const TubeDev* tubes, S* F, S* buf) {
  const HaloDesc d = hd[blockIdx.y];
  const TubeDev T = tubes[d.tube];
  const int Q = T.Qp * T.Qxi;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;  // side, row, cell
  const int left = (d.bc & RLB_BC_HALO_LEFT) ? 1 : 0, sides = left + ((d.bc & RLB_BC_HALO_RIGHT) ? 1 : 0);
  if (k >= sides * Q * HALO) return;
  const int side = k / (Q * HALO), r = k - side * Q * HALO, s = r / HALO, c = r - s * HALO;
  const bool is_left = left && side == 0;
  S* row = F + T.off + (size_t)s * T.ld;
  S* b = buf + d.off + k;
  if (PACK)
    *b = row[is_left ? c : T.Nx - HALO + c];
  else
    row[is_left ? T.ld - HALO + c : T.Nx + c] = *b;
}

#include "rlb_adjoint.cuh"

// --------------------------------------------------------------------------------------------------
// Host side
// --------------------------------------------------------------------------------------------------

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else if (prev == dev) prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

rlb_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return RLB_OK;
  return e == cudaErrorMemoryAllocation ? RLB_ENOMEM : RLB_ECUDA;
}

#define RLB_CUDA(call)                               \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return cuda_status(e_);   \
  } while (0)

std::mutex g_tables_mu;
bool g_tables_ready[64] = {};

// Once per device: fill the series tables (long double on the host) and let the stage kernel use more than
// 48 KB of dynamic shared memory.
rlb_status ensure_series_tables(int dev) {
  std::lock_guard<std::mutex> lk(g_tables_mu);
  if (dev < 0 || dev >= 64) return RLB_EINVAL;
  if (g_tables_ready[dev]) return RLB_OK;
  std::vector<double> ic((size_t)(R_MAX + 1) * (NV_MAX + 1), 0.0), cb((size_t)(M_MAX + 1) * (R_MAX + 1), 0.0);
  for (int k = 0; k <= NV_MAX; ++k) {
    // I_{k,k} = 2^{k+1} (k!)^2 / (2k+1)!; I_{r+2,k}/I_{r,k} = (r+1)(r+2)((r+k)/2+1) / (((r-k)/2+1)(r+k+2)(r+k+3))
    long double I = 2.0L;
    for (int q = 1; q <= k; ++q) I *= 2.0L * q * q / ((2.0L * q) * (2.0L * q + 1.0L));
    for (int r = k; r <= R_MAX; r += 2) {
      ic[(size_t)r * (NV_MAX + 1) + k] = (double)((2.0L * k + 1.0L) / 2.0L * I);
      const long double hp = (r + k) / 2, hm = (r - k) / 2;
      I *= (r + 1.0L) * (r + 2.0L) * (hp + 1.0L) / ((hm + 1.0L) * (r + k + 2.0L) * (r + k + 3.0L));
    }
  }
  for (int m = 1; m <= M_MAX; ++m) {
    long double C = 1.0L;  // C(m - 1, 0)
    for (int r = 0; r <= R_MAX; ++r) {
      cb[(size_t)m * (R_MAX + 1) + r] = (double)C;
      C = C * (m + r) / (r + 1.0L);  // C(m + r, r + 1)
    }
  }
  RLB_CUDA(cudaMemcpyToSymbol(g_ic, ic.data(), ic.size() * sizeof(double)));
  RLB_CUDA(cudaMemcpyToSymbol(g_cb, cb.data(), cb.size() * sizeof(double)));
  const void* fp64[3] = {(const void*)rlb_stage_kernel<0>, (const void*)rlb_stage_kernel<1>,
                         (const void*)rlb_stage_kernel<2>};
  const void* rp[6] = {(const void*)rlb_stage_rp_kernel<float, 0>, (const void*)rlb_stage_rp_kernel<float, 1>,
                       (const void*)rlb_stage_rp_kernel<float, 2>, (const void*)rlb_stage_rp_kernel<__nv_bfloat16, 0>,
                       (const void*)rlb_stage_rp_kernel<__nv_bfloat16, 1>,
                       (const void*)rlb_stage_rp_kernel<__nv_bfloat16, 2>};
  for (const void* k : fp64)
    RLB_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(StageSmem)));
  for (const void* k : rp) {
    RLB_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)rp_smem_bytes(QP_MAX * (NV_MAX + 1))));
    // carveout: enough shared memory for the four CTAs per SM that the registers allow with the default orders
    // (Np = 2, Nv = 5), the rest left to L1, which holds the per-velocity records and the register spills
    const int pct = (int)((100 * 4 * (rp_smem_bytes(rp_brows(3, 2, 5)) + 1024) + 228 * 1024 - 1) / (228 * 1024));
    RLB_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, pct));
  }
  RLB_CUDA(cudaFuncSetAttribute((const void*)rlb_adjoint_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(AdjSmem)));
  RLB_CUDA(cudaFuncSetAttribute((const void*)rlb_init_vjp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(InitVjpSmem)));
  g_tables_ready[dev] = true;
  return RLB_OK;
}

}  // namespace

struct rlb_ctx {
  int dev = 0;
  cudaStream_t stream = nullptr;
  std::vector<rlb_tube> tubes;
  std::vector<TubeDev> td;
  int ntiles = 0;
  int storage = RLB_STORAGE_F64;
  size_t esize = sizeof(double);  // bytes per stored population
  long long state_elems = 0;      // padded elements per buffer
  long long packed = 0;           // sum Q Nx
  long long nxtot = 0;
  TubeDev* d_tubes = nullptr;
  int2* d_tiles = nullptr;
  int2* d_wtiles = nullptr;    // reduced storage: warp tiles of RP_OUT cells
  int nwt = 0;
  int brows = 0;               // reduced storage: coefficient rows per warp region of the stage kernel
  size_t stage_smem = 0;       // FP64: dynamic shared memory of the stage kernel (coefficient rows in use)
  double* d_tab = nullptr;
  float* d_tabf = nullptr;
  void *F = nullptr, *F1 = nullptr, *F2 = nullptr;
  double* d_fields = nullptr;  // scratch for host-side moments
  double* d_stage = nullptr;   // packed FP64 staging for host state copies of reduced storage
  double *M = nullptr, *M1 = nullptr, *M2 = nullptr;  // reduced storage: FP64 moments of F, F1, F2
                                                       // ([RLB_NFIELDS][nxtot]; the first 5 rows are used)
  int* d_flag = nullptr;       // [0]: non-physical cell seen; [1]: warning bits (RLB_WARN_*)
  int* h_flag = nullptr;       // pinned, 2 ints
  // launch shape, CUDA graph of graph_steps steps, work counters of the counter schedule
  rlb_launch cfg = {RLB_SCHED_TILE, 0, 0, RLB_ORDER_COST, 0};
  int occupancy = 1;           // resident CTAs per SM of the stage kernel
  int split = 1;               // automatic FP64 stage work items per tile (several when the tiles cannot fill
                               // the GPU); rlb_launch.split overrides it
  int asplit = 1;              // adjoint work items per adjoint tile
  int nsm = 1;
  cudaStream_t gstream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int* d_counters = nullptr;   // 3 per step, GRAPH_MAX steps
  // adjoint: checkpoints of the last rlb_record, recompute and adjoint scratch, tiles of TXA cells
  double* ckpt = nullptr;
  long long ckpt_cap = 0;      // states allocated
  int64_t rec_steps = 0;
  int rec_every = 0;
  bool rec_kept = false;       // the record kept every stage input in seg (one segment, nothing to recompute)
  double* seg = nullptr;
  long long seg_cap = 0;       // states allocated
  double* adj = nullptr;       // 4 states: adjoints of F^(n+1) / F^n, F^(1), F^(2) and the F^n accumulator
  int2* d_atiles = nullptr;
  std::vector<int> atile_tube;
  double* d_dlt = nullptr;     // per adjoint tile: dL/dlog(tau)
  // slabs of a decomposed tube: their exchange blocks (tube, sides, offset in the buffer)
  std::vector<HaloDesc> halo;
  HaloDesc* d_halo = nullptr;
  long long halo_elems = 0;
};

namespace {

constexpr int GRAPH_MAX = 64;  // longest captured graph, in steps
constexpr int SPLIT_MAX = 8;   // most work items per tile

// Work items per tile of the FP64 stage kernel for the handle's launch shape.
int eff_split(const rlb_ctx* h) {
  if (h->storage != RLB_STORAGE_F64) return 1;
  return h->cfg.split > 0 ? h->cfg.split : h->split;
}

void free_ctx(rlb_ctx* h) {
  if (!h) return;
  DeviceGuard gd(h->dev);
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->gstream) cudaStreamDestroy(h->gstream);
  cudaFree(h->d_counters);
  cudaFree(h->ckpt);
  cudaFree(h->seg);
  cudaFree(h->adj);
  cudaFree(h->d_atiles);
  cudaFree(h->d_dlt);
  cudaFree(h->d_halo);
  cudaFree(h->d_tubes);
  cudaFree(h->d_tiles);
  cudaFree(h->d_wtiles);
  cudaFree(h->d_tab);
  cudaFree(h->d_tabf);
  cudaFree(h->d_stage);
  cudaFree(h->M);
  cudaFree(h->M1);
  cudaFree(h->M2);
  cudaFree(h->F);
  cudaFree(h->F1);
  cudaFree(h->F2);
  cudaFree(h->d_fields);
  cudaFree(h->d_flag);
  cudaFreeHost(h->h_flag);
  delete h;
}

// WENO5 epsilon terms of every velocity: 3 eps ws^2 (C0, C1, C2) into out, ws = w^p_i w^xi_j / 2 (the limiter
// acts on the weight-normalised population F_s / ws with eps = 1e-6), and e = 3 eps ws^2 as the float pair
// (hi, lo), hi + lo = e to about 48 bits, into the 8 bytes of outf[s].
void fill_eps(double* out, double* outf, int Qp, int Qxi, const double* wp, const double* wxi) {
  for (int i = 0; i < Qp; ++i)
    for (int j = 0; j < Qxi; ++j) {
      const double ws = 0.5 * wp[i] * wxi[j];
      const double e = 3.0 * rlbdev::WENO_EPS * ws * ws;
      double* o = out + 3 * (i * Qxi + j);
      o[0] = e * rlbdev::C0;
      o[1] = e * rlbdev::C1;
      o[2] = e * rlbdev::C2;
      const float pair[2] = {(float)e, (float)(e - (double)(float)e)};
      std::memcpy(outf + i * Qxi + j, pair, sizeof(pair));
    }
}

// The FP64 tables of one tube (layout in rlb_internal.h): quadrature nodes and weights, the radial factors
// K[i][q], w^xi_j P_k(xi_j), the per-stage b dt xi_j / dx and the WENO5 epsilon terms. pb, wp, xi, wxi receive
// the quadrature (Qp and Qxi entries). Returns false if a quadrature rule cannot be built.
bool fill_tube_tables(const rlb_tube& t, double* pb, double* wp, double* xi, double* wxi, double* T) {
  if (!rlbq::gauss_laguerre1(t.Qp, pb, wp) || !rlbq::gauss_legendre(t.Qxi, xi, wxi)) return false;
  for (int i = 0; i < t.Qp; ++i) {
    T[TAB_PBAR + i] = pb[i];
    T[TAB_PBAR2 + i] = pb[i] * pb[i];
    T[TAB_WP + i] = wp[i];
    // K[i][q] = (-1)^q sum_{l=q}^{Np} C(l, q) L^(1)_l(pbar_i)
    for (int q = 0; q <= t.Np; ++q) {
      long double acc = 0.0L;
      for (int l = q; l <= t.Np; ++l) {
        long double C = 1.0L;
        for (int u = 1; u <= q; ++u) C = C * (l - q + u) / u;
        acc += C * rlbq::laguerre1(l, pb[i]);
      }
      T[TAB_K + i * (NP_MAX + 1) + q] = (double)((q % 2) ? -acc : acc);
    }
  }
  for (int j = 0; j < t.Qxi; ++j) {
    T[TAB_XI + j] = xi[j];
    for (int k = 0; k <= NV_MAX; ++k)
      T[tab_pw(t.Qxi) + j * (NV_MAX + 1) + k] = k <= t.Nv ? wxi[j] * rlbq::legendre(k, xi[j]) : 0.0;
    for (int st = 0; st < 3; ++st) T[tab_cxi(t.Qxi) + st * t.Qxi + j] = RK_B[st] * t.dt * xi[j] / t.dx;
  }
  fill_eps(T + tab_eps(t.Qxi), T + tab_epsf(t.Qp, t.Qxi), t.Qp, t.Qxi, wp, wxi);
  return true;
}

// Tiles of `width` cells of every tube (TX for the FP64 kernels, RP_OUT warp tiles for the reduced-precision
// kernel): most expensive tubes first (RLB_ORDER_COST), or the tubes interleaved tile by tile
// (RLB_ORDER_INTERLEAVE).
std::vector<int2> build_tiles(const std::vector<rlb_tube>& tubes, int order, int width = TX) {
  const int ntubes = (int)tubes.size();
  std::vector<int> ord(ntubes);
  for (int b = 0; b < ntubes; ++b) ord[b] = b;
  std::stable_sort(ord.begin(), ord.end(), [&](int p, int q) {
    return tubes[p].Qp * tubes[p].Qxi > tubes[q].Qp * tubes[q].Qxi;
  });
  std::vector<int2> tiles;
  if (order == RLB_ORDER_COST) {
    for (int b : ord)
      for (int x0 = 0; x0 < (int)tubes[b].Nx; x0 += width) tiles.push_back(make_int2(b, x0));
  } else {
    bool more = true;
    for (int x0 = 0; more; x0 += width) {
      more = false;
      for (int b : ord)
        if (x0 < (int)tubes[b].Nx) {
          tiles.push_back(make_int2(b, x0));
          more = true;
        }
    }
  }
  return tiles;
}

rlb_status validate(const rlb_tube* t) {
  if (t->Qp < 3 || t->Qp > QP_MAX || t->Np < 2 || t->Np >= t->Qp || t->Np > NP_MAX) return RLB_EINVAL;
  if (t->Nv < 2 || t->Nv > NV_MAX || t->Qxi < 1 || t->Qxi > QXI_MAX || 2 * t->Qxi < t->Nv + 3) return RLB_EINVAL;
  if (t->Nx < 1 || t->Nx > (1LL << 30) || (t->bc != RLB_BC_OPEN && t->Nx < 3)) return RLB_EINVAL;
  if (t->bc != RLB_BC_OPEN && t->bc != RLB_BC_PERIODIC && (t->bc & ~(RLB_BC_HALO_LEFT | RLB_BC_HALO_RIGHT)) != 0)
    return RLB_EINVAL;
  if (!(t->dx > 0.0) || !std::isfinite(t->dx) || !(t->dt > 0.0) || !std::isfinite(t->dt)) return RLB_EINVAL;
  if (std::isnan(t->tau)) return RLB_EINVAL;
  if (t->storage != RLB_STORAGE_F64 && t->storage != RLB_STORAGE_F32 && t->storage != RLB_STORAGE_BF16)
    return RLB_EINVAL;
  return RLB_OK;
}

rlb_status create(rlb_handle* out, const rlb_tube* tubes, int32_t ntubes, const double* xleft, void* stream,
                  rlb_ctx** hp) {
  if (!out || !tubes || ntubes < 1) return RLB_EINVAL;
  *out = nullptr;
  for (int b = 0; b < ntubes; ++b) {
    rlb_status st = validate(&tubes[b]);
    if (st != RLB_OK) return st;
    if (tubes[b].storage != tubes[0].storage) return RLB_EINVAL;
  }
  rlb_ctx* h = new (std::nothrow) rlb_ctx;
  if (!h) return RLB_ENOMEM;
  *hp = h;
  RLB_CUDA(cudaGetDevice(&h->dev));
  h->stream = (cudaStream_t)stream;
  h->tubes.assign(tubes, tubes + ntubes);
  h->storage = tubes[0].storage;
  h->esize = h->storage == RLB_STORAGE_F64 ? sizeof(double) : (h->storage == RLB_STORAGE_F32 ? sizeof(float) : 2);
  // quadrature tables, one block per tube (FP64, and FP32 for reduced storage)
  std::vector<double> tab;
  std::vector<float> tabf;
  std::map<double, double> stiff_memo;  // tubes of one batch often share xi_max dt / dx
  h->td.resize(ntubes);
  long long off = 0, xoff = 0;
  for (int b = 0; b < ntubes; ++b) {
    const rlb_tube& t = tubes[b];
    TubeDev& d = h->td[b];
    d.Qp = t.Qp;
    d.Qxi = t.Qxi;
    d.Np = t.Np;
    d.Nv = t.Nv;
    d.bc = t.bc;
    d.collide = (t.tau > 0.0 && std::isfinite(t.tau)) ? 1 : 0;
    d.Nx = (int)t.Nx;
    // rows start on 256-byte boundaries for every storage type; a slab keeps its ghost cells beside each row
    const bool slab = t.bc == RLB_BC_HALO_LEFT || t.bc == RLB_BC_HALO_RIGHT ||
                      t.bc == (RLB_BC_HALO_LEFT | RLB_BC_HALO_RIGHT);
    d.ld = (int)((t.Nx + (slab ? 2 * HALO : 0) + 127) / 128 * 128);
    if (slab) {
      const int sides = ((t.bc & RLB_BC_HALO_LEFT) ? 1 : 0) + ((t.bc & RLB_BC_HALO_RIGHT) ? 1 : 0);
      h->halo.push_back(HaloDesc{b, t.bc, h->halo_elems});
      h->halo_elems += (long long)sides * t.Qp * t.Qxi * HALO;
    }
    d.storage = t.storage;
    d.off = off;
    d.xoff = xoff;
    d.dx = t.dx;
    d.dt = t.dt;
    d.inv_tau = d.collide ? 1.0 / t.tau : 0.0;
    d.x_left = xleft ? xleft[b] : 0.0;
    d.index = b;
    d.poff = h->packed;
    off += (long long)t.Qp * t.Qxi * d.ld;
    xoff += t.Nx;
    h->packed += (long long)t.Qp * t.Qxi * t.Nx;
    d.tab = (int)tab.size();
    d.tabf = (int)tabf.size();
    tab.resize(tab.size() + tab_size(t.Qp, t.Qxi), 0.0);
    tabf.resize(tabf.size() + tabf_size(t.Qp, t.Qxi), 0.0f);
    double* T = tab.data() + d.tab;
    std::vector<double> pb(t.Qp), wp(t.Qp), xi(t.Qxi), wxi(t.Qxi);
    if (!fill_tube_tables(t, pb.data(), wp.data(), xi.data(), wxi.data(), T)) return RLB_EINVAL;
    d.xi_max = 0.0;
    for (int j = 0; j < t.Qxi; ++j) d.xi_max = std::max(d.xi_max, std::fabs(xi[j]));
    const double nu = d.xi_max * t.dt / t.dx;
    auto memo = stiff_memo.find(nu);
    d.stiff_lim = memo != stiff_memo.end() ? memo->second : (stiff_memo[nu] = rlb_stiffness_limit(nu));
    // FP32 records of the reduced-precision path, one per velocity (hi/lo float pairs of the moment weights)
    float* Tf = tabf.data() + d.tabf;
    auto split = [](double w, float* hl) {
      hl[0] = (float)w;
      hl[1] = (float)(w - (double)hl[0]);
    };
    for (int i = 0; i < t.Qp; ++i)
      for (int j = 0; j < t.Qxi; ++j) {
        float* r = Tf + (size_t)(i * t.Qxi + j) * RP_REC;
        const double iws = 2.0 / (wp[i] * wxi[j]);
        r[R_XI] = (float)xi[j];
        for (int st = 0; st < 3; ++st) r[R_CXI + st] = (float)T[tab_cxi(t.Qxi) + st * t.Qxi + j];
        r[R_IWS] = (float)iws;
        r[R_WS6] = (float)(1.0 / (6.0 * iws));
        split(pb[i], r + R_P1);
        split(pb[i] * pb[i], r + R_P2);
        split(xi[j], r + R_X);
        split(xi[j] * xi[j], r + R_X2);
        for (int k = 0; k <= NV_MAX; ++k) r[R_PW + k] = (float)T[tab_pw(t.Qxi) + j * (NV_MAX + 1) + k];
      }
  }
  h->state_elems = off;
  h->nxtot = xoff;
  // tiles, most expensive tubes first
  const std::vector<int2> tiles = build_tiles(h->tubes, RLB_ORDER_COST);
  h->ntiles = (int)tiles.size();
  DeviceGuard gd(h->dev);
  RLB_CUDA(cudaMalloc(&h->d_tubes, sizeof(TubeDev) * ntubes));
  RLB_CUDA(cudaMalloc(&h->d_tiles, sizeof(int2) * tiles.size()));
  RLB_CUDA(cudaMalloc(&h->d_tab, sizeof(double) * std::max<size_t>(tab.size(), 1)));
  RLB_CUDA(cudaMalloc(&h->d_tabf, sizeof(float) * std::max<size_t>(tabf.size(), 1)));
  RLB_CUDA(cudaMalloc(&h->F, h->esize * h->state_elems));
  RLB_CUDA(cudaMalloc(&h->F1, h->esize * h->state_elems));
  RLB_CUDA(cudaMalloc(&h->F2, h->esize * h->state_elems));
  RLB_CUDA(cudaMalloc(&h->d_flag, 2 * sizeof(int)));
  RLB_CUDA(cudaMallocHost(&h->h_flag, 2 * sizeof(int)));
  RLB_CUDA(cudaMalloc(&h->d_counters, sizeof(int) * 3 * GRAPH_MAX));
  RLB_CUDA(cudaStreamCreateWithFlags(&h->gstream, cudaStreamNonBlocking));
  RLB_CUDA(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
  RLB_CUDA(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
  RLB_CUDA(cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->dev));
  if (h->storage != RLB_STORAGE_F64) {
    const std::vector<int2> wt = build_tiles(h->tubes, RLB_ORDER_COST, RP_OUT);
    h->nwt = (int)wt.size();
    for (const rlb_tube& t : h->tubes) h->brows = std::max(h->brows, rp_brows(t.Qp, t.Np, t.Nv));
    RLB_CUDA(cudaMalloc(&h->d_wtiles, sizeof(int2) * wt.size()));
    RLB_CUDA(cudaMemcpy(h->d_wtiles, wt.data(), sizeof(int2) * wt.size(), cudaMemcpyHostToDevice));
    RLB_CUDA(cudaMalloc(&h->M, sizeof(double) * RLB_NFIELDS * h->nxtot));
    RLB_CUDA(cudaMalloc(&h->M1, sizeof(double) * RLB_NFIELDS * h->nxtot));
    RLB_CUDA(cudaMalloc(&h->M2, sizeof(double) * RLB_NFIELDS * h->nxtot));
  }
  RLB_CUDA(cudaMemcpyAsync(h->d_tubes, h->td.data(), sizeof(TubeDev) * ntubes, cudaMemcpyHostToDevice, h->stream));
  RLB_CUDA(cudaMemcpyAsync(h->d_tiles, tiles.data(), sizeof(int2) * tiles.size(), cudaMemcpyHostToDevice, h->stream));
  RLB_CUDA(cudaMemcpyAsync(h->d_tab, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice, h->stream));
  RLB_CUDA(cudaMemcpyAsync(h->d_tabf, tabf.data(), sizeof(float) * tabf.size(), cudaMemcpyHostToDevice, h->stream));
  RLB_CUDA(cudaMemsetAsync(h->F, 0, h->esize * h->state_elems, h->stream));
  RLB_CUDA(cudaMemsetAsync(h->F1, 0, h->esize * h->state_elems, h->stream));
  RLB_CUDA(cudaMemsetAsync(h->F2, 0, h->esize * h->state_elems, h->stream));
  RLB_CUDA(cudaMemsetAsync(h->d_flag, 0, 2 * sizeof(int), h->stream));
  if (!h->halo.empty()) {
    RLB_CUDA(cudaMalloc(&h->d_halo, sizeof(HaloDesc) * h->halo.size()));
    RLB_CUDA(cudaMemcpyAsync(h->d_halo, h->halo.data(), sizeof(HaloDesc) * h->halo.size(), cudaMemcpyHostToDevice,
                             h->stream));
  }
  rlb_status st = ensure_series_tables(h->dev);
  if (st != RLB_OK) return st;
  // resident CTAs per SM of this handle's stage kernel (the persistent grids' default size)
  if (h->storage == RLB_STORAGE_F64) {
    int rows = 0;
    for (const rlb_tube& t : h->tubes) rows = std::max(rows, rp_brows(t.Qp, t.Np, t.Nv));
    h->stage_smem = stage_smem_bytes(rows);
    RLB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&h->occupancy, rlb_stage_kernel<1>, NT, h->stage_smem));
  }
  else if (h->storage == RLB_STORAGE_F32)
    RLB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&h->occupancy, rlb_stage_rp_kernel<float, 1>, RP_NT,
                                                           rp_smem_bytes(h->brows)));
  else
    RLB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&h->occupancy, rlb_stage_rp_kernel<__nv_bfloat16, 1>, RP_NT,
                                                           rp_smem_bytes(h->brows)));
  if (h->occupancy < 1) h->occupancy = 1;
  // a handle whose tiles cannot fill the resident slots splits each tile's velocity rows over several CTAs
  const long long slots = (long long)h->nsm * h->occupancy;
  if (h->storage == RLB_STORAGE_F64 && h->ntiles < slots)
    h->split = (int)std::min<long long>(SPLIT_MAX, slots / h->ntiles);
  return RLB_OK;
}

rlb_status check_flag(rlb_ctx* h) {
  RLB_CUDA(cudaMemcpyAsync(h->h_flag, h->d_flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  RLB_CUDA(cudaStreamSynchronize(h->stream));
  if (*h->h_flag) {
    RLB_CUDA(cudaMemsetAsync(h->d_flag, 0, sizeof(int), h->stream));
    return RLB_ENONPHYS;
  }
  return RLB_OK;
}

// Reduced storage: the stage kernel reads the moments of its input from M; recompute them (FP64) whenever F is
// written from outside the step (initial condition, rlb_set_state).
rlb_status refresh_moments(rlb_ctx* h) {
  if (h->storage == RLB_STORAGE_F32)
    rlb_fields_kernel<float><<<h->ntiles, GW, 0, h->stream>>>(h->d_tubes, h->d_tiles, h->F, h->d_tab, h->M,
                                                               h->nxtot, h->d_flag);
  else if (h->storage == RLB_STORAGE_BF16)
    rlb_fields_kernel<__nv_bfloat16><<<h->ntiles, GW, 0, h->stream>>>(h->d_tubes, h->d_tiles, h->F, h->d_tab,
                                                                       h->M, h->nxtot, h->d_flag);
  return cuda_status(cudaGetLastError());
}

rlb_status run_init(rlb_ctx* h, const double* P, const double* n, const double* v, int on_device,
                    const double* riem_host) {
  InitArgs A{};
  A.tubes = h->d_tubes;
  A.tiles = h->d_tiles;
  A.F = h->F;
  A.tab = h->d_tab;
  A.flag = h->d_flag;
  double* tmp = nullptr;
  if (riem_host) {
    RLB_CUDA(cudaMalloc(&tmp, sizeof(double) * 6 * h->tubes.size()));
    RLB_CUDA(cudaMemcpyAsync(tmp, riem_host, sizeof(double) * 6 * h->tubes.size(), cudaMemcpyHostToDevice, h->stream));
    A.riem = tmp;
  } else if (on_device) {
    A.P = P;
    A.n = n;
    A.v = v;
  } else {
    RLB_CUDA(cudaMalloc(&tmp, sizeof(double) * 3 * h->nxtot));
    RLB_CUDA(cudaMemcpyAsync(tmp, P, sizeof(double) * h->nxtot, cudaMemcpyHostToDevice, h->stream));
    RLB_CUDA(cudaMemcpyAsync(tmp + h->nxtot, n, sizeof(double) * h->nxtot, cudaMemcpyHostToDevice, h->stream));
    RLB_CUDA(cudaMemcpyAsync(tmp + 2 * h->nxtot, v, sizeof(double) * h->nxtot, cudaMemcpyHostToDevice, h->stream));
    A.P = tmp;
    A.n = tmp + h->nxtot;
    A.v = tmp + 2 * h->nxtot;
  }
  if (h->storage == RLB_STORAGE_F64)
    rlb_init_kernel<double><<<h->ntiles, NT, 0, h->stream>>>(A);
  else if (h->storage == RLB_STORAGE_F32)
    rlb_init_kernel<float><<<h->ntiles, NT, 0, h->stream>>>(A);
  else
    rlb_init_kernel<__nv_bfloat16><<<h->ntiles, NT, 0, h->stream>>>(A);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && h->storage != RLB_STORAGE_F64) {
    const rlb_status sm = refresh_moments(h);
    if (sm != RLB_OK) return sm;
  }
  rlb_status st = check_flag(h);  // also waits for the copies out of the caller's buffers
  if (tmp) cudaFree(tmp);
  if (e != cudaSuccess) return cuda_status(e);
  if (st == RLB_ENONPHYS) return RLB_EINVAL;
  return st;
}

}  // namespace

extern "C" {

rlb_status rlb_init(rlb_handle* out, const rlb_tube* tubes, int32_t ntubes, const double* P, const double* n,
                    const double* v, int32_t ic_on_device, void* stream) {
  if (!P || !n || !v) return RLB_EINVAL;
  rlb_ctx* h = nullptr;
  rlb_status st = create(out, tubes, ntubes, nullptr, stream, &h);
  if (st == RLB_OK) {
    DeviceGuard gd(h->dev);
    st = run_init(h, P, n, v, ic_on_device, nullptr);
  }
  if (st != RLB_OK) {
    free_ctx(h);
    return st;
  }
  *out = h;
  return RLB_OK;
}

rlb_status rlb_init_riemann(rlb_handle* out, const rlb_tube* tubes, int32_t ntubes, const double* states,
                            const double* x_left, void* stream) {
  if (!states || !x_left) return RLB_EINVAL;
  for (int b = 0; b < ntubes; ++b)
    if (!(states[6 * b] > 0) || !(states[6 * b + 1] > 0) || !(states[6 * b + 3] > 0) || !(states[6 * b + 4] > 0) ||
        !(std::fabs(states[6 * b + 2]) < 1) || !(std::fabs(states[6 * b + 5]) < 1) || !std::isfinite(x_left[b]))
      return RLB_EINVAL;
  rlb_ctx* h = nullptr;
  rlb_status st = create(out, tubes, ntubes, x_left, stream, &h);
  if (st == RLB_OK) {
    DeviceGuard gd(h->dev);
    st = run_init(h, nullptr, nullptr, nullptr, 0, states);
  }
  if (st != RLB_OK) {
    free_ctx(h);
    return st;
  }
  *out = h;
  return RLB_OK;
}

}  // extern "C"

namespace {

// One stage st of the current step as one launch on `stream`, with work counter ctr (counter schedule).
rlb_status launch_stage(rlb_ctx* h, cudaStream_t stream, int st, int* ctr) {
  const void* in[3] = {h->F, h->F1, h->F2};
  void* out[3] = {h->F1, h->F2, h->F};
  const int sched = h->cfg.schedule;
  const int split = eff_split(h);
  // work items: tiles (times the split) of the FP64 kernel, groups of RP_WARPS warp tiles otherwise
  const int items = h->storage == RLB_STORAGE_F64 ? h->ntiles * split : (h->nwt + RP_WARPS - 1) / RP_WARPS;
  const int grid = sched == RLB_SCHED_TILE
                       ? items
                       : std::max(1, std::min(items, h->nsm * (h->cfg.ctas_per_sm > 0 ? h->cfg.ctas_per_sm
                                                                                       : h->occupancy)));
  if (h->storage == RLB_STORAGE_F64) {
    StageArgs A{};
    A.tubes = h->d_tubes;
    A.tiles = h->d_tiles;
    A.tab = h->d_tab;
    A.flag = h->d_flag;
    A.warn = h->d_flag + 1;
    A.Fn = static_cast<const double*>(h->F);
    A.Fin = static_cast<const double*>(in[st]);
    A.Fout = static_cast<double*>(out[st]);
    A.a = RK_A[st];
    A.b = RK_B[st];
    A.stage = st;
    A.ntiles = h->ntiles;
    A.schedule = sched;
    A.counter = ctr;
    A.split = split;
    if (sched == RLB_SCHED_TILE)
      rlb_stage_kernel<0><<<grid, NT, h->stage_smem, stream>>>(A);
    else if (sched == RLB_SCHED_STRIDE)
      rlb_stage_kernel<1><<<grid, NT, h->stage_smem, stream>>>(A);
    else
      rlb_stage_kernel<2><<<grid, NT, h->stage_smem, stream>>>(A);
  } else {
    const double* min[3] = {h->M, h->M1, h->M2};
    double* mout[3] = {h->M1, h->M2, h->M};
    StageArgsRP A{};
    A.tubes = h->d_tubes;
    A.wtiles = h->d_wtiles;
    A.nwt = h->nwt;
    A.tab = h->d_tab;
    A.tabf = h->d_tabf;
    A.flag = h->d_flag;  // two words: non-physical flag, warning bits
    A.Fn = h->F;
    A.nxtot = h->nxtot;
    A.Fin = in[st];
    A.Fout = out[st];
    A.Min = min[st];
    A.Mout = mout[st];
    A.a = (float)RK_A[st];
    A.b = (float)RK_B[st];
    A.bd = RK_B[st];
    A.stage = st;
    A.ngroups = items;
    A.schedule = sched;
    A.counter = ctr;
    A.brows = h->brows;
    const size_t sb = rp_smem_bytes(h->brows);
    if (h->storage == RLB_STORAGE_F32) {
      if (sched == RLB_SCHED_TILE)
        rlb_stage_rp_kernel<float, 0><<<grid, RP_NT, sb, stream>>>(A);
      else if (sched == RLB_SCHED_STRIDE)
        rlb_stage_rp_kernel<float, 1><<<grid, RP_NT, sb, stream>>>(A);
      else
        rlb_stage_rp_kernel<float, 2><<<grid, RP_NT, sb, stream>>>(A);
    } else {
      if (sched == RLB_SCHED_TILE)
        rlb_stage_rp_kernel<__nv_bfloat16, 0><<<grid, RP_NT, sb, stream>>>(A);
      else if (sched == RLB_SCHED_STRIDE)
        rlb_stage_rp_kernel<__nv_bfloat16, 1><<<grid, RP_NT, sb, stream>>>(A);
      else
        rlb_stage_rp_kernel<__nv_bfloat16, 2><<<grid, RP_NT, sb, stream>>>(A);
    }
  }
  return cuda_status(cudaGetLastError());
}

// nsteps steps as plain launches on `stream`. in_graph: the launches belong to one captured graph, whose
// counter-schedule launches get counters of their own (zeroed once up front), else each step zeroes three.
rlb_status launch_steps(rlb_ctx* h, cudaStream_t stream, int64_t nsteps, bool in_graph) {
  const int sched = h->cfg.schedule;
  if (sched == RLB_SCHED_COUNTER && in_graph)
    RLB_CUDA(cudaMemsetAsync(h->d_counters, 0, sizeof(int) * 3 * nsteps, stream));
  for (int64_t t = 0; t < nsteps; ++t) {
    if (sched == RLB_SCHED_COUNTER && !in_graph) RLB_CUDA(cudaMemsetAsync(h->d_counters, 0, sizeof(int) * 3, stream));
    int* ctr = h->d_counters + (in_graph ? 3 * t : 0);
    for (int st = 0; st < 3; ++st) {
      const rlb_status r = launch_stage(h, stream, st, ctr + st);
      if (r != RLB_OK) return r;
    }
  }
  return RLB_OK;
}

// Capture graph_steps steps on the private stream (once per launch shape).
rlb_status ensure_graph(rlb_ctx* h) {
  if (h->gexec) return RLB_OK;
  cudaGraph_t graph = nullptr;
  RLB_CUDA(cudaStreamBeginCapture(h->gstream, cudaStreamCaptureModeThreadLocal));
  const rlb_status st = launch_steps(h, h->gstream, h->cfg.graph_steps, true);
  const cudaError_t e = cudaStreamEndCapture(h->gstream, &graph);
  if (st != RLB_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  RLB_CUDA(e);
  const cudaError_t ei = cudaGraphInstantiate(&h->gexec, graph, 0);
  cudaGraphDestroy(graph);
  return cuda_status(ei);
}

void drop_graph(rlb_ctx* h) {
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  h->gexec = nullptr;
}

}  // namespace

extern "C" {

rlb_status rlb_step(rlb_handle h, int64_t nsteps) {
  if (!h || nsteps < 0 || !h->halo.empty()) return RLB_EINVAL;
  DeviceGuard gd(h->dev);
  const int G = h->cfg.graph_steps;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  RLB_CUDA(cudaStreamIsCapturing(h->stream, &cap));
  if (G <= 0 || nsteps < G || cap != cudaStreamCaptureStatusNone) return launch_steps(h, h->stream, nsteps, false);
  rlb_status st = ensure_graph(h);
  if (st != RLB_OK) return st;
  RLB_CUDA(cudaEventRecord(h->ev_fork, h->stream));
  RLB_CUDA(cudaStreamWaitEvent(h->gstream, h->ev_fork, 0));
  for (int64_t k = 0; k < nsteps / G; ++k) RLB_CUDA(cudaGraphLaunch(h->gexec, h->gstream));
  st = launch_steps(h, h->gstream, nsteps % G, false);
  RLB_CUDA(cudaEventRecord(h->ev_join, h->gstream));
  RLB_CUDA(cudaStreamWaitEvent(h->stream, h->ev_join, 0));
  return st;
}

int64_t rlb_halo_size(rlb_handle h) { return h ? h->halo_elems : -1; }

static rlb_status halo_copy(rlb_handle h, int32_t stage, void* buf, bool pack) {
  if (!h || !buf || stage < 0 || stage > 2) return RLB_EINVAL;
  if (h->halo.empty()) return RLB_OK;
  DeviceGuard gd(h->dev);
  void* Fs[3] = {h->F, h->F1, h->F2};
  int most = 0;
  for (const HaloDesc& d : h->halo) most = std::max(most, 2 * h->td[d.tube].Qp * h->td[d.tube].Qxi * HALO);
  const dim3 grid((most + 255) / 256, (unsigned)h->halo.size());
  if (h->storage == RLB_STORAGE_F64) {
    double *F = static_cast<double*>(Fs[stage]), *b = static_cast<double*>(buf);
    if (pack) halo_kernel<double, true><<<grid, 256, 0, h->stream>>>(h->d_halo, h->d_tubes, F, b);
    else halo_kernel<double, false><<<grid, 256, 0, h->stream>>>(h->d_halo, h->d_tubes, F, b);
  } else if (h->storage == RLB_STORAGE_F32) {
    float *F = static_cast<float*>(Fs[stage]), *b = static_cast<float*>(buf);
    if (pack) halo_kernel<float, true><<<grid, 256, 0, h->stream>>>(h->d_halo, h->d_tubes, F, b);
    else halo_kernel<float, false><<<grid, 256, 0, h->stream>>>(h->d_halo, h->d_tubes, F, b);
  } else {
    __nv_bfloat16 *F = static_cast<__nv_bfloat16*>(Fs[stage]), *b = static_cast<__nv_bfloat16*>(buf);
    if (pack) halo_kernel<__nv_bfloat16, true><<<grid, 256, 0, h->stream>>>(h->d_halo, h->d_tubes, F, b);
    else halo_kernel<__nv_bfloat16, false><<<grid, 256, 0, h->stream>>>(h->d_halo, h->d_tubes, F, b);
  }
  return cuda_status(cudaGetLastError());
}

rlb_status rlb_halo_pack(rlb_handle h, int32_t stage, void* send) { return halo_copy(h, stage, send, true); }

rlb_status rlb_halo_unpack(rlb_handle h, int32_t stage, const void* recv) {
  return halo_copy(h, stage, const_cast<void*>(recv), false);
}

rlb_status rlb_stage(rlb_handle h, int32_t stage) {
  if (!h || stage < 0 || stage > 2) return RLB_EINVAL;
  DeviceGuard gd(h->dev);
  if (h->cfg.schedule == RLB_SCHED_COUNTER)
    RLB_CUDA(cudaMemsetAsync(h->d_counters + stage, 0, sizeof(int), h->stream));
  return launch_stage(h, h->stream, stage, h->d_counters + stage);
}

rlb_status rlb_get_launch(rlb_handle h, rlb_launch* out) {
  if (!h || !out) return RLB_EINVAL;
  *out = h->cfg;
  return RLB_OK;
}

rlb_status rlb_set_launch(rlb_handle h, const rlb_launch* cfg) {
  if (!h || !cfg) return RLB_EINVAL;
  if (cfg->schedule < RLB_SCHED_TILE || cfg->schedule > RLB_SCHED_COUNTER || cfg->ctas_per_sm < 0 ||
      cfg->ctas_per_sm > 64 || cfg->graph_steps < 0 || cfg->graph_steps > GRAPH_MAX ||
      (cfg->order != RLB_ORDER_COST && cfg->order != RLB_ORDER_INTERLEAVE) || cfg->split < 0 ||
      cfg->split > SPLIT_MAX)
    return RLB_EINVAL;
  DeviceGuard gd(h->dev);
  if (cfg->order != h->cfg.order) {
    const std::vector<int2> tiles = build_tiles(h->tubes, cfg->order);
    RLB_CUDA(cudaMemcpyAsync(h->d_tiles, tiles.data(), sizeof(int2) * tiles.size(), cudaMemcpyHostToDevice,
                             h->stream));
    std::vector<int2> wt;
    if (h->d_wtiles) {
      wt = build_tiles(h->tubes, cfg->order, RP_OUT);
      RLB_CUDA(cudaMemcpyAsync(h->d_wtiles, wt.data(), sizeof(int2) * wt.size(), cudaMemcpyHostToDevice, h->stream));
    }
    RLB_CUDA(cudaStreamSynchronize(h->stream));  // the host vectors go out of scope
  }
  drop_graph(h);
  h->cfg = *cfg;
  return RLB_OK;
}

rlb_status rlb_autotune(rlb_handle h, int32_t trial_steps, rlb_launch* best, double* best_ms_per_step) {
  if (!h || trial_steps < 1 || trial_steps > GRAPH_MAX || !h->halo.empty()) return RLB_EINVAL;
  DeviceGuard gd(h->dev);
  // save the state (and, for reduced storage, the moments the first stage reads)
  const size_t fbytes = h->esize * h->state_elems;
  const size_t mbytes = h->M ? sizeof(double) * RLB_NFIELDS * h->nxtot : 0;
  char* saved = nullptr;
  RLB_CUDA(cudaMalloc(&saved, fbytes + mbytes));
  auto restore = [&]() -> cudaError_t {
    cudaError_t e = cudaMemcpyAsync(h->F, saved, fbytes, cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess && mbytes) e = cudaMemcpyAsync(h->M, saved + fbytes, mbytes, cudaMemcpyDeviceToDevice, h->stream);
    return e;
  };
  cudaError_t e = cudaMemcpyAsync(saved, h->F, fbytes, cudaMemcpyDeviceToDevice, h->stream);
  if (e == cudaSuccess && mbytes) e = cudaMemcpyAsync(saved + fbytes, h->M, mbytes, cudaMemcpyDeviceToDevice, h->stream);
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  const rlb_launch start = h->cfg;
  rlb_launch win = start;
  float win_ms = -1.0f;
  rlb_status st = cuda_status(e);
  const int scheds[7][2] = {{RLB_SCHED_TILE, 0}, {RLB_SCHED_STRIDE, 0}, {RLB_SCHED_STRIDE, 1}, {RLB_SCHED_STRIDE, 2},
                            {RLB_SCHED_COUNTER, 0}, {RLB_SCHED_COUNTER, 1}, {RLB_SCHED_COUNTER, 2}};
  const int nsplit = (h->storage == RLB_STORAGE_F64 && h->split > 1) ? 2 : 1;  // automatic, and 1 if different
  for (int order = 0; order < 2 && st == RLB_OK; ++order)
    for (int k = 0; k < 7 && st == RLB_OK; ++k)
      for (int graph = 0; graph < 2 && st == RLB_OK; ++graph)
        for (int sp = 0; sp < nsplit && st == RLB_OK; ++sp) {
          const rlb_launch c = {scheds[k][0], scheds[k][1], graph ? trial_steps : 0, order, sp};
          st = rlb_set_launch(h, &c);
          if (st == RLB_OK) st = rlb_step(h, trial_steps);  // warm-up (and graph capture)
          if (st == RLB_OK) st = cuda_status(restore());
          if (st == RLB_OK) st = cuda_status(cudaEventRecord(t0, h->stream));
          if (st == RLB_OK) st = rlb_step(h, trial_steps);
          if (st == RLB_OK) st = cuda_status(cudaEventRecord(t1, h->stream));
          if (st == RLB_OK) st = cuda_status(cudaEventSynchronize(t1));
          float ms = 0.0f;
          if (st == RLB_OK) st = cuda_status(cudaEventElapsedTime(&ms, t0, t1));
          if (st == RLB_OK && (win_ms < 0.0f || ms < win_ms)) {
            win_ms = ms;
            win = c;
          }
          if (st == RLB_OK) st = cuda_status(restore());
        }
  if (st == RLB_OK) st = rlb_set_launch(h, &win);
  else rlb_set_launch(h, &start);
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  cudaStreamSynchronize(h->stream);
  cudaFree(saved);
  if (st != RLB_OK) return st;
  if (best) *best = win;
  if (best_ms_per_step) *best_ms_per_step = win_ms / trial_steps;
  return check_flag(h);
}

rlb_status rlb_moments(rlb_handle h, double* out, int32_t out_on_device) {
  if (!h || !out) return RLB_EINVAL;
  DeviceGuard gd(h->dev);
  double* dst = out;
  if (!out_on_device) {
    if (!h->d_fields) RLB_CUDA(cudaMalloc(&h->d_fields, sizeof(double) * RLB_NFIELDS * h->nxtot));
    dst = h->d_fields;
  }
  if (h->storage == RLB_STORAGE_F64)
    rlb_fields_kernel<double><<<h->ntiles, GW, 0, h->stream>>>(h->d_tubes, h->d_tiles, h->F, h->d_tab, dst,
                                                                h->nxtot, h->d_flag);
  else if (h->storage == RLB_STORAGE_F32)
    rlb_fields_kernel<float><<<h->ntiles, GW, 0, h->stream>>>(h->d_tubes, h->d_tiles, h->F, h->d_tab, dst,
                                                               h->nxtot, h->d_flag, h->M);
  else
    rlb_fields_kernel<__nv_bfloat16><<<h->ntiles, GW, 0, h->stream>>>(h->d_tubes, h->d_tiles, h->F, h->d_tab, dst,
                                                                       h->nxtot, h->d_flag, h->M);
  RLB_CUDA(cudaGetLastError());
  if (!out_on_device)
    RLB_CUDA(cudaMemcpyAsync(out, dst, sizeof(double) * RLB_NFIELDS * h->nxtot, cudaMemcpyDeviceToHost, h->stream));
  return check_flag(h);
}

// Widen (to_handle false) or narrow (true) every tube between the packed FP64 buffer P (device) and F.
static rlb_status convert_state(rlb_handle h, double* P, bool to_handle) {
  long long p = 0;
  for (size_t b = 0; b < h->tubes.size(); ++b) {
    const TubeDev& d = h->td[b];
    const int rows = d.Qp * d.Qxi;
    const dim3 grid((d.Nx + 255) / 256, rows);
    char* base = static_cast<char*>(h->F) + h->esize * d.off;
    if (h->storage == RLB_STORAGE_F32) {
      if (to_handle)
        narrow_kernel<float><<<grid, 256, 0, h->stream>>>(P + p, reinterpret_cast<float*>(base), d.ld, d.Nx);
      else
        widen_kernel<float><<<grid, 256, 0, h->stream>>>(reinterpret_cast<const float*>(base), d.ld, P + p, d.Nx);
    } else {
      if (to_handle)
        narrow_kernel<__nv_bfloat16><<<grid, 256, 0, h->stream>>>(P + p, reinterpret_cast<__nv_bfloat16*>(base),
                                                                   d.ld, d.Nx);
      else
        widen_kernel<__nv_bfloat16><<<grid, 256, 0, h->stream>>>(reinterpret_cast<const __nv_bfloat16*>(base),
                                                                  d.ld, P + p, d.Nx);
    }
    p += (long long)rows * d.Nx;
  }
  return cuda_status(cudaGetLastError());
}

static rlb_status copy_state(rlb_handle h, double* host_or_dev, const double* src_const, int32_t on_device,
                             bool to_handle) {
  DeviceGuard gd(h->dev);
  if (h->storage != RLB_STORAGE_F64) {
    double* P = nullptr;
    if (on_device) {
      P = to_handle ? const_cast<double*>(src_const) : host_or_dev;
    } else {
      if (!h->d_stage) RLB_CUDA(cudaMalloc(&h->d_stage, sizeof(double) * h->packed));
      P = h->d_stage;
      if (to_handle)
        RLB_CUDA(cudaMemcpyAsync(P, src_const, sizeof(double) * h->packed, cudaMemcpyHostToDevice, h->stream));
    }
    rlb_status st = convert_state(h, P, to_handle);
    if (st == RLB_OK && to_handle) st = refresh_moments(h);
    if (st != RLB_OK) return st;
    if (!on_device && !to_handle)
      RLB_CUDA(cudaMemcpyAsync(host_or_dev, P, sizeof(double) * h->packed, cudaMemcpyDeviceToHost, h->stream));
    if (!on_device || !to_handle) return check_flag(h);
    return RLB_OK;
  }
  double* F = static_cast<double*>(h->F);
  // rows without padding (Nx a multiple of the row alignment in every tube): the handle's state is the packed
  // layout itself, one copy
  bool packed = true;
  for (const TubeDev& d : h->td) packed = packed && d.ld == d.Nx;
  if (packed) {
    cudaMemcpyKind kind;
    if (to_handle)
      kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    else
      kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (to_handle)
      RLB_CUDA(cudaMemcpyAsync(F, src_const, sizeof(double) * h->packed, kind, h->stream));
    else
      RLB_CUDA(cudaMemcpyAsync(host_or_dev, F, sizeof(double) * h->packed, kind, h->stream));
    if (!on_device || !to_handle) return check_flag(h);
    return RLB_OK;
  }
  long long p = 0;
  for (size_t b = 0; b < h->tubes.size(); ++b) {
    const TubeDev& d = h->td[b];
    const size_t rows = (size_t)d.Qp * d.Qxi;
    cudaMemcpyKind kind;
    if (to_handle)
      kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    else
      kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (to_handle)
      RLB_CUDA(cudaMemcpy2DAsync(F + d.off, sizeof(double) * d.ld, src_const + p, sizeof(double) * d.Nx,
                                 sizeof(double) * d.Nx, rows, kind, h->stream));
    else
      RLB_CUDA(cudaMemcpy2DAsync(host_or_dev + p, sizeof(double) * d.Nx, F + d.off, sizeof(double) * d.ld,
                                 sizeof(double) * d.Nx, rows, kind, h->stream));
    p += (long long)rows * d.Nx;
  }
  if (!on_device || !to_handle) return check_flag(h);
  return RLB_OK;
}

rlb_status rlb_get_state(rlb_handle h, double* F, int32_t on_device) {
  if (!h || !F) return RLB_EINVAL;
  return copy_state(h, F, nullptr, on_device, false);
}

rlb_status rlb_set_state(rlb_handle h, const double* F, int32_t on_device) {
  if (!h || !F) return RLB_EINVAL;
  return copy_state(h, nullptr, F, on_device, true);
}

rlb_status rlb_sync(rlb_handle h) {
  if (!h) return RLB_EINVAL;
  DeviceGuard gd(h->dev);
  return check_flag(h);
}

rlb_status rlb_destroy(rlb_handle h) {
  if (!h) return RLB_OK;
  {
    DeviceGuard gd(h->dev);
    cudaStreamSynchronize(h->stream);
  }
  free_ctx(h);
  return RLB_OK;
}

int64_t rlb_state_size(rlb_handle h) { return h ? h->packed : -1; }

const char* rlb_error_string(rlb_status s) {
  switch (s) {
    case RLB_OK: return "RLB_OK";
    case RLB_EINVAL: return "RLB_EINVAL: invalid argument";
    case RLB_ENOMEM: return "RLB_ENOMEM: out of memory";
    case RLB_ECUDA: return "RLB_ECUDA: CUDA runtime error";
    case RLB_ENONPHYS: return "RLB_ENONPHYS: non-physical state (e <= 0, |v| >= 1, n <= 0 or NaN)";
  }
  return "unknown rlb_status";
}

double rlb_suggest_dt(double dx, double tau, double cfl) {
  double dt = cfl * dx;
  if (tau > 0.0 && std::isfinite(tau)) dt = std::min(dt, 0.9 * tau);
  return dt;
}

double rlb_stiffness_limit(double nu) {
  // Fourier symbol of the linear fifth-order upwind interface value (the smooth limit of WENO5),
  // phi(th) = (2 e^-2i th - 13 e^-i th + 47 + 27 e^i th - 3 e^2i th) / 60, flux difference phi (1 - e^-i th);
  // a step multiplies a mode by R(z) = 1 + z + z^2/2 + z^3/6, z = -nu phi (1 - e^-i th) - k dt. The symbol at
  // -th is the conjugate of the one at th and R has real coefficients, so th in [0, pi] suffices.
  if (!(nu >= 0.0) || !std::isfinite(nu)) return 0.0;
  constexpr int NTH = 2048;  // 4096 phases over the circle
  static const std::vector<std::complex<double>> psi = [] {
    std::vector<std::complex<double>> t(NTH + 1);
    for (int m = 0; m <= NTH; ++m) {
      const double th = 3.141592653589793 * m / NTH;
      auto E = [th](int k) { return std::complex<double>(std::cos(k * th), std::sin(k * th)); };
      const std::complex<double> phi = (2.0 * E(-2) - 13.0 * E(-1) + 47.0 + 27.0 * E(1) - 3.0 * E(2)) / 60.0;
      t[m] = phi - phi * E(-1);
    }
    return t;
  }();
  auto growth = [nu](double kdt) {
    double worst = 0.0;
    for (int m = 0; m <= NTH; ++m) {
      const std::complex<double> z = -nu * psi[m] - kdt;
      worst = std::max(worst, std::norm(1.0 + z * (1.0 + z * (0.5 + z / 6.0))));
    }
    return std::sqrt(worst);
  };
  const double tol = 1.0 + 1e-12;
  if (growth(0.0) > tol) return 0.0;
  double lo = 0.0, hi = 3.0;  // the real-axis bound of SSP-RK3 is about 2.513
  for (int it = 0; it < 40; ++it) {
    const double mid = 0.5 * (lo + hi);
    (growth(mid) <= tol ? lo : hi) = mid;
  }
  return lo;
}

rlb_status rlb_warnings(rlb_handle h, uint32_t* bits) {
  if (!h || !bits) return RLB_EINVAL;
  DeviceGuard gd(h->dev);
  RLB_CUDA(cudaMemcpyAsync(h->h_flag + 1, h->d_flag + 1, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  RLB_CUDA(cudaStreamSynchronize(h->stream));
  *bits = (uint32_t)h->h_flag[1];
  if (*bits) RLB_CUDA(cudaMemsetAsync(h->d_flag + 1, 0, sizeof(int), h->stream));
  return RLB_OK;
}

rlb_status rlb_quadrature(int32_t Qp, int32_t Qxi, double* pbar, double* wp, double* xi, double* wxi) {
  if (Qp < 1 || Qp > 64 || Qxi < 1 || Qxi > QXI_MAX || !pbar || !wp || !xi || !wxi) return RLB_EINVAL;
  if (!rlbq::gauss_laguerre1(Qp, pbar, wp) || !rlbq::gauss_legendre(Qxi, xi, wxi)) return RLB_EINVAL;
  return RLB_OK;
}

}  // extern "C"

// --------------------------------------------------------------------------------------------------
// Allocation-free single-tube step (rlb_step_static)
// --------------------------------------------------------------------------------------------------
// For callers that cannot allocate device memory when they step. The scratch that rlb_init would allocate
// (intermediate stages F1 and F2, the tube's tables, its descriptor and tile list, a flag) lives in this
// file-scope array instead; the existing stage kernel runs on it unchanged.
namespace {

static __device__ __align__(256) double g_static_scratch[RLB_STATIC_SCRATCH_BYTES / sizeof(double)];

std::mutex g_static_mu;
double* g_static_addr[64] = {};

// Once per device, with that device current: the device address of the array (in host code the symbol is
// only a host-side stand-in and must not be passed to a kernel) and the shared series tables.
rlb_status static_setup(int dev, double** base) {
  if (dev < 0 || dev >= 64) return RLB_EINVAL;
  {
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_addr[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
      if (e != cudaSuccess || p == nullptr) return e != cudaSuccess ? cuda_status(e) : RLB_ECUDA;
      g_static_addr[dev] = static_cast<double*>(p);
    }
    *base = g_static_addr[dev];
  }
  return ensure_series_tables(dev);
}

size_t align256(size_t bytes) { return (bytes + 255) / 256 * 256; }

}  // namespace

extern "C" rlb_status rlb_step_static(const rlb_tube* tube, const double* F_in, double* F_out, int64_t nsteps,
                                      int32_t* flag, void* stream) {
  if (!tube || !F_in || !F_out || nsteps < 0) return RLB_EINVAL;
  rlb_status st = validate(tube);
  if (st != RLB_OK) return st;
  if (tube->storage != RLB_STORAGE_F64 || (tube->bc != RLB_BC_OPEN && tube->bc != RLB_BC_PERIODIC)) return RLB_EINVAL;
  const rlb_tube& t = *tube;
  const int Q = t.Qp * t.Qxi, Nx = (int)t.Nx;
  const int ntiles = (Nx + TX - 1) / TX;
  // layout of the array: descriptor | tiles | flag | tables | F1 | F2, each section 256-byte aligned
  const size_t off_tiles = align256(sizeof(TubeDev));
  const size_t off_flag = off_tiles + align256(sizeof(int2) * (size_t)ntiles);
  const size_t off_tab = off_flag + 256;
  const size_t off_f1 = off_tab + align256(sizeof(double) * (size_t)tab_size(t.Qp, t.Qxi));
  const size_t stage_bytes = align256(sizeof(double) * (size_t)Q * (size_t)Nx);
  const size_t off_f2 = off_f1 + stage_bytes;
  if (off_f2 + stage_bytes > (size_t)RLB_STATIC_SCRATCH_BYTES) return RLB_EINVAL;
  if (nsteps == 0) return RLB_OK;

  cudaStream_t s = (cudaStream_t)stream;
  // the tables below are copied out of host memory that lives only during this call, which a captured graph
  // would read again at every replay: refuse a stream under capture
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  RLB_CUDA(cudaStreamIsCapturing(s, &cap));
  if (cap != cudaStreamCaptureStatusNone) return RLB_EINVAL;
  int dev = 0;
  RLB_CUDA(cudaGetDevice(&dev));
  double* base = nullptr;
  st = static_setup(dev, &base);
  if (st != RLB_OK) return st;
  char* b = reinterpret_cast<char*>(base);

  // descriptor, tiles and tables on the host, then copied into the array on the caller's stream
  TubeDev d{};
  d.Qp = t.Qp;
  d.Qxi = t.Qxi;
  d.Np = t.Np;
  d.Nv = t.Nv;
  d.bc = t.bc;
  d.collide = (t.tau > 0.0 && std::isfinite(t.tau)) ? 1 : 0;
  d.Nx = Nx;
  d.ld = Nx;  // the caller's packed rows
  d.off = 0;
  d.xoff = 0;
  d.dx = t.dx;
  d.dt = t.dt;
  d.inv_tau = d.collide ? 1.0 / t.tau : 0.0;
  d.x_left = 0.0;
  d.tab = 0;
  d.index = 0;
  std::vector<int2> tiles(ntiles);
  for (int k = 0; k < ntiles; ++k) tiles[k] = make_int2(0, k * TX);
  std::vector<double> tab(tab_size(t.Qp, t.Qxi), 0.0), pb(t.Qp), wp(t.Qp), xi(t.Qxi), wxi(t.Qxi);
  if (!fill_tube_tables(t, pb.data(), wp.data(), xi.data(), wxi.data(), tab.data())) return RLB_EINVAL;
  RLB_CUDA(cudaMemcpyAsync(b, &d, sizeof(TubeDev), cudaMemcpyHostToDevice, s));
  RLB_CUDA(cudaMemcpyAsync(b + off_tiles, tiles.data(), sizeof(int2) * ntiles, cudaMemcpyHostToDevice, s));
  RLB_CUDA(cudaMemcpyAsync(b + off_tab, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice, s));
  int* dflag = flag ? flag : reinterpret_cast<int*>(b + off_flag);
  if (!flag) RLB_CUDA(cudaMemsetAsync(dflag, 0, sizeof(int), s));
  // the copies above come from pageable host memory, so they are consumed before cudaMemcpyAsync returns

  double* F1 = reinterpret_cast<double*>(b + off_f1);
  double* F2 = reinterpret_cast<double*>(b + off_f2);
  StageArgs A{};
  A.tubes = reinterpret_cast<const TubeDev*>(b);
  A.tiles = reinterpret_cast<const int2*>(b + off_tiles);
  A.tab = reinterpret_cast<const double*>(b + off_tab);
  A.flag = dflag;
  for (int64_t k = 0; k < nsteps; ++k) {
    const double* Fn = (k == 0) ? F_in : F_out;
    const double* in[3] = {Fn, F1, F2};
    double* out[3] = {F1, F2, F_out};
    A.Fn = Fn;
    for (int st = 0; st < 3; ++st) {
      A.Fin = in[st];
      A.Fout = out[st];
      A.a = RK_A[st];
      A.b = RK_B[st];
      A.stage = st;
      rlb_stage_kernel<0><<<ntiles, NT, sizeof(StageSmem), s>>>(A);
    }
  }
  return cuda_status(cudaGetLastError());
}

// --------------------------------------------------------------------------------------------------
// Adjoint: record with checkpoints, reverse sweep, seeds from the moments, initial-condition adjoint
// --------------------------------------------------------------------------------------------------

namespace {

// One FP64 forward stage between explicit buffers (one CTA per tile; every launch shape gives the same bits).
rlb_status launch_stage_ptrs(rlb_ctx* h, int st, const double* Fn, const double* Fin, double* Fout) {
  StageArgs A{};
  A.tubes = h->d_tubes;
  A.tiles = h->d_tiles;
  A.tab = h->d_tab;
  A.flag = h->d_flag;
  A.warn = h->d_flag + 1;
  A.Fn = Fn;
  A.Fin = Fin;
  A.Fout = Fout;
  A.a = RK_A[st];
  A.b = RK_B[st];
  A.stage = st;
  A.ntiles = h->ntiles;
  A.schedule = RLB_SCHED_TILE;
  A.counter = h->d_counters;
  A.split = eff_split(h);
  rlb_stage_kernel<0><<<h->ntiles * A.split, NT, h->stage_smem, h->stream>>>(A);
  return cuda_status(cudaGetLastError());
}

rlb_status launch_adjoint(rlb_ctx* h, int st, int mode, const double* Fin, const double* mu, double* out,
                          double* acc) {
  AdjArgs A{};
  A.tubes = h->d_tubes;
  A.tiles = h->d_atiles;
  A.Fin = Fin;
  A.mu = mu;
  A.out = out;
  A.acc = acc;
  A.tab = h->d_tab;
  A.flag = h->d_flag;
  A.dlt = h->d_dlt;
  A.a = RK_A[st];
  A.b = RK_B[st];
  A.mode = mode;
  A.split = h->asplit;
  rlb_adjoint_kernel<<<(int)h->atile_tube.size() * h->asplit, NT, sizeof(AdjSmem), h->stream>>>(A);
  return cuda_status(cudaGetLastError());
}

// Tiles of TXA cells (tube after tube) and their dL/dlog(tau) accumulators.
rlb_status ensure_adjoint_tiles(rlb_ctx* h) {
  if (h->d_atiles) return RLB_OK;
  std::vector<int2> tiles;
  for (size_t b = 0; b < h->tubes.size(); ++b)
    for (int x0 = 0; x0 < (int)h->tubes[b].Nx; x0 += TXA) {
      tiles.push_back(make_int2((int)b, x0));
      h->atile_tube.push_back((int)b);
    }
  RLB_CUDA(cudaMalloc(&h->d_atiles, sizeof(int2) * tiles.size()));
  RLB_CUDA(cudaMalloc(&h->d_dlt, sizeof(double) * tiles.size()));
  RLB_CUDA(cudaMemcpyAsync(h->d_atiles, tiles.data(), sizeof(int2) * tiles.size(), cudaMemcpyHostToDevice, h->stream));
  RLB_CUDA(cudaStreamSynchronize(h->stream));  // the host vector goes out of scope
  int occ = 1;
  RLB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, rlb_adjoint_kernel, NT, sizeof(AdjSmem)));
  const long long slots = (long long)h->nsm * std::max(occ, 1);
  if ((long long)tiles.size() < slots) h->asplit = (int)std::min<long long>(8, slots / (long long)tiles.size());
  return RLB_OK;
}

// Recompute buffer of at least `states` states (the stage inputs of a segment).
rlb_status ensure_seg(rlb_ctx* h, long long states) {
  if (h->seg_cap >= states) return RLB_OK;
  cudaFree(h->seg);
  h->seg = nullptr;
  h->seg_cap = 0;
  RLB_CUDA(cudaMalloc(&h->seg, sizeof(double) * h->state_elems * states));
  h->seg_cap = states;
  return RLB_OK;
}

// Packed <-> padded FP64 state of every tube (device to device).
rlb_status packed_to_padded(rlb_ctx* h, const double* P, double* F) {
  for (size_t b = 0; b < h->tubes.size(); ++b) {
    const TubeDev& d = h->td[b];
    RLB_CUDA(cudaMemcpy2DAsync(F + d.off, sizeof(double) * d.ld, P + d.poff, sizeof(double) * d.Nx,
                               sizeof(double) * d.Nx, (size_t)d.Qp * d.Qxi, cudaMemcpyDeviceToDevice, h->stream));
  }
  return RLB_OK;
}

rlb_status padded_to_packed(rlb_ctx* h, const double* F, double* P) {
  for (size_t b = 0; b < h->tubes.size(); ++b) {
    const TubeDev& d = h->td[b];
    RLB_CUDA(cudaMemcpy2DAsync(P + d.poff, sizeof(double) * d.Nx, F + d.off, sizeof(double) * d.ld,
                               sizeof(double) * d.Nx, (size_t)d.Qp * d.Qxi, cudaMemcpyDeviceToDevice, h->stream));
  }
  return RLB_OK;
}

}  // namespace

extern "C" {

rlb_status rlb_record(rlb_handle h, int64_t nsteps, int32_t every) {
  if (!h || nsteps < 1 || every < 1 || h->storage != RLB_STORAGE_F64 || !h->halo.empty()) return RLB_EINVAL;
  DeviceGuard gd(h->dev);
  h->rec_steps = 0;
  h->rec_kept = false;
  const long long se = h->state_elems;
  if (every >= nsteps) {
    // one segment: keep every stage input as the steps run (the buffer the reverse sweep would fill anyway),
    // so that the reverse sweep recomputes nothing
    rlb_status st = ensure_seg(h, 3 * nsteps + 1);
    if (st != RLB_OK) return st;
    double* S = h->seg;
    RLB_CUDA(cudaMemcpyAsync(S, h->F, sizeof(double) * se, cudaMemcpyDeviceToDevice, h->stream));
    for (int64_t t = 0; t < nsteps; ++t) {
      double* Fn = S + 3 * t * se;
      if ((st = launch_stage_ptrs(h, 0, Fn, Fn, Fn + se)) != RLB_OK) return st;
      if ((st = launch_stage_ptrs(h, 1, Fn, Fn + se, Fn + 2 * se)) != RLB_OK) return st;
      if ((st = launch_stage_ptrs(h, 2, Fn, Fn + 2 * se, Fn + 3 * se)) != RLB_OK) return st;
    }
    RLB_CUDA(cudaMemcpyAsync(h->F, S + 3 * nsteps * se, sizeof(double) * se, cudaMemcpyDeviceToDevice, h->stream));
    st = check_flag(h);
    if (st != RLB_OK) return st;
    h->rec_steps = nsteps;
    h->rec_every = (int)nsteps;
    h->rec_kept = true;
    return RLB_OK;
  }
  const long long nck = (nsteps + every - 1) / every;
  if (h->ckpt_cap < nck) {
    cudaFree(h->ckpt);
    h->ckpt = nullptr;
    h->ckpt_cap = 0;
    RLB_CUDA(cudaMalloc(&h->ckpt, sizeof(double) * se * nck));
    h->ckpt_cap = nck;
  }
  for (long long k = 0; k < nck; ++k) {
    RLB_CUDA(cudaMemcpyAsync(h->ckpt + k * se, h->F, sizeof(double) * se, cudaMemcpyDeviceToDevice, h->stream));
    const int64_t len = std::min<int64_t>(every, nsteps - k * every);
    const rlb_status st = rlb_step(h, len);
    if (st != RLB_OK) return st;
  }
  const rlb_status st = check_flag(h);
  if (st != RLB_OK) return st;
  h->rec_steps = nsteps;
  h->rec_every = every;
  return RLB_OK;
}

rlb_status rlb_backward(rlb_handle h, const double* seed, double* grad_state, double* grad_log_tau) {
  if (!h || !seed || h->storage != RLB_STORAGE_F64 || h->rec_steps < 1 || !h->halo.empty()) return RLB_EINVAL;
  DeviceGuard gd(h->dev);
  rlb_status st = ensure_adjoint_tiles(h);
  if (st != RLB_OK) return st;
  const long long se = h->state_elems;
  const int every = h->rec_every;
  if (!h->rec_kept) {
    st = ensure_seg(h, 3 * std::min<int64_t>(every, h->rec_steps) + 1);
    if (st != RLB_OK) return st;
  }
  if (!h->adj) RLB_CUDA(cudaMalloc(&h->adj, sizeof(double) * se * 4));
  double *L = h->adj, *L1 = L + se, *L2 = L1 + se, *LA = L2 + se;
  RLB_CUDA(cudaMemsetAsync(h->adj, 0, sizeof(double) * se * 4, h->stream));
  RLB_CUDA(cudaMemsetAsync(h->d_dlt, 0, sizeof(double) * h->atile_tube.size(), h->stream));
  st = packed_to_padded(h, seed, L);
  if (st != RLB_OK) return st;
  const long long nck = (h->rec_steps + every - 1) / every;
  for (long long k = nck - 1; k >= 0; --k) {
    const int64_t len = std::min<int64_t>(every, h->rec_steps - k * every);
    double* S = h->seg;
    if (!h->rec_kept)
      RLB_CUDA(cudaMemcpyAsync(S, h->ckpt + k * se, sizeof(double) * se, cudaMemcpyDeviceToDevice, h->stream));
    // recompute the segment, keeping the three stage inputs of every step (unless the record kept them)
    for (int64_t t = 0; !h->rec_kept && t < len; ++t) {
      double* Fn = S + 3 * t * se;
      if ((st = launch_stage_ptrs(h, 0, Fn, Fn, Fn + se)) != RLB_OK) return st;
      if ((st = launch_stage_ptrs(h, 1, Fn, Fn + se, Fn + 2 * se)) != RLB_OK) return st;
      if ((st = launch_stage_ptrs(h, 2, Fn, Fn + 2 * se, Fn + 3 * se)) != RLB_OK) return st;
    }
    // reverse: stage 3, 2, 1 of every step, last step first
    for (int64_t t = len - 1; t >= 0; --t) {
      const double* Fn = S + 3 * t * se;
      if ((st = launch_adjoint(h, 2, 2, Fn + 2 * se, L, L2, LA)) != RLB_OK) return st;
      if ((st = launch_adjoint(h, 1, 1, Fn + se, L2, L1, LA)) != RLB_OK) return st;
      if ((st = launch_adjoint(h, 0, 0, Fn, L1, L, LA)) != RLB_OK) return st;
    }
  }
  if (grad_state) {
    st = padded_to_packed(h, L, grad_state);
    if (st != RLB_OK) return st;
  }
  std::vector<double> dl(h->atile_tube.size());
  RLB_CUDA(cudaMemcpyAsync(dl.data(), h->d_dlt, sizeof(double) * dl.size(), cudaMemcpyDeviceToHost, h->stream));
  st = check_flag(h);  // synchronises the stream
  if (st != RLB_OK) return st;
  if (grad_log_tau) {
    for (size_t b = 0; b < h->tubes.size(); ++b) grad_log_tau[b] = 0.0;
    for (size_t t = 0; t < dl.size(); ++t) grad_log_tau[h->atile_tube[t]] += dl[t];
  }
  return RLB_OK;
}

rlb_status rlb_moments_vjp(rlb_handle h, const double* grad_moments, double* seed) {
  if (!h || !grad_moments || !seed || h->storage != RLB_STORAGE_F64 || !h->halo.empty()) return RLB_EINVAL;
  DeviceGuard gd(h->dev);
  rlb_status st = ensure_adjoint_tiles(h);
  if (st != RLB_OK) return st;
  rlb_moments_vjp_kernel<<<(int)h->atile_tube.size(), NT, 0, h->stream>>>(h->d_tubes, h->d_atiles, h->d_tab,
                                                                          grad_moments, h->nxtot, seed);
  RLB_CUDA(cudaGetLastError());
  RLB_CUDA(cudaStreamSynchronize(h->stream));
  return RLB_OK;
}

rlb_status rlb_fields_vjp(rlb_handle h, const double* grad_fields, double* seed) {
  if (!h || !grad_fields || !seed || h->storage != RLB_STORAGE_F64 || !h->halo.empty()) return RLB_EINVAL;
  DeviceGuard gd(h->dev);
  rlb_status st = ensure_adjoint_tiles(h);
  if (st != RLB_OK) return st;
  rlb_fields_vjp_kernel<<<(int)h->atile_tube.size(), NT, 0, h->stream>>>(
      h->d_tubes, h->d_atiles, h->d_tab, static_cast<const double*>(h->F), grad_fields, h->nxtot, seed, h->d_flag);
  RLB_CUDA(cudaGetLastError());
  return check_flag(h);  // synchronises the stream
}

rlb_status rlb_init_vjp(rlb_handle h, const double* P, const double* n, const double* v, const double* grad_state,
                        double* grad_P, double* grad_n, double* grad_v) {
  if (!h || !P || !n || !v || !grad_state || !grad_P || !grad_n || !grad_v || h->storage != RLB_STORAGE_F64 ||
      !h->halo.empty())
    return RLB_EINVAL;
  DeviceGuard gd(h->dev);
  rlb_status st = ensure_adjoint_tiles(h);
  if (st != RLB_OK) return st;
  rlb_init_vjp_kernel<<<(int)h->atile_tube.size(), NT, sizeof(InitVjpSmem), h->stream>>>(
      h->d_tubes, h->d_atiles, h->d_tab, P, n, v, grad_state, grad_P, grad_n, grad_v, h->d_flag);
  RLB_CUDA(cudaGetLastError());
  st = check_flag(h);
  return st == RLB_ENONPHYS ? RLB_EINVAL : st;
}

}  // extern "C"
