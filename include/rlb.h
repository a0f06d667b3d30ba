/*
 * rlb.h - C ABI of the GB300 (sm_103a) time step of the quadrature-based finite-difference relativistic
 * lattice Boltzmann model for massless particles (Blaga & Ambrus, arXiv:1608.03004).
 *
 * The library advances one or more independent one-dimensional tubes ("shock tubes") of the kinetic
 * equation (section "Relativistic lattice Boltzmann equation", Eq. (Boltz)):
 *     (d_t + xi d_x) f = -(u^0 - xi u^x)/tau (f - f^eq),
 * with the Anderson-Witting collision, the Landau-frame equilibrium rebuilt every stage from the
 * stress-energy tensor T^{mu nu} (second moment of f), the truncated Maxwell-Juttner expansion of
 * Eq. (feqtrunc), fifth-order WENO advection and third-order SSP Runge-Kutta time integration (section
 * "Numerical results").
 *
 * Conventions shared by every entry point
 *  - Velocities: s = i*Qxi + j pairs the i-th zero pbar_i of the generalised Laguerre polynomial
 *    L^(1)_Qp (radial, momentum magnitude p/T0, T0 = 1) with the j-th zero xi_j of the Legendre
 *    polynomial P_Qxi (direction cosine along x), both ascending (section "Discretization of the momentum
 *    space using quadrature rules"). The paper's z axis is called x here.
 *  - Stored population: F_s(x) = 2 pi w^p_i w^xi_j exp(pbar_i) f(x, pbar_i, xi_j), so that
 *    N^0 = sum_s F pbar, N^x = sum F pbar xi, T^00 = sum F pbar^2, T^0x = sum F pbar^2 xi,
 *    T^xx = sum F pbar^2 xi^2.
 *  - Packed state layout ("packed"): tubes one after the other; tube b holds Q_b rows of Nx_b doubles
 *    (row s, cell x at offset s*Nx_b + x). With FP32 or BF16 storage the state crosses the ABI as doubles
 *    too: rlb_get_state widens, rlb_set_state rounds to nearest. Fields layout: [RLB_NFIELDS][sum_b Nx_b], each field row holding
 *    the tubes' cells one after the other.
 *  - Pointers flagged "on_device" are CUDA device pointers on the handle's device, otherwise host
 *    pointers (pageable or pinned). Caller buffers are never retained after a call returns.
 *  - Every call is ordered on the stream given to rlb_init. Calls that copy to the host wait for that
 *    stream. Errors are returned, never aborted on. A cell that reaches a non-physical state (e <= 0,
 *    |v| >= 1, n <= 0 or NaN) sets a sticky device flag; the next call that synchronises (rlb_moments,
 *    rlb_get_state, rlb_sync) returns RLB_ENONPHYS.
 *  - Limits: 2 <= Np < Qp <= 4 and 2 <= Nv <= 8 with 2*Qxi >= Nv + 3: T^{mu nu} is of second order in pbar
 *    and in xi, so Eq. (mom_feq) recovers it exactly only with Np >= 2, Nv >= 2 and a polar rule exact to
 *    degree Nv + 2 (section "Riemann problem" gives Qp = 3 for the same reason). Qxi <= 1024, Nx >= 1
 *    (periodic: Nx >= 3), dx > 0, dt > 0.
 *  - Speed limit: the Legendre coefficients of the equilibrium, Eq. (feqtrunc), are summed as a positive
 *    power series in v of at most 16384 terms, which converges for |v| <= 0.9955. A cell faster than that is
 *    treated as non-physical: rlb_init returns RLB_EINVAL, a step sets the sticky non-physical flag.
 */
#ifndef RLB_H
#define RLB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rlb_ctx *rlb_handle;

typedef enum {
  RLB_OK = 0,
  RLB_EINVAL = 1,   /* an argument is out of range or a pointer is NULL */
  RLB_ENOMEM = 2,   /* a device or host allocation failed */
  RLB_ECUDA = 3,    /* a CUDA runtime call failed */
  RLB_ENONPHYS = 4  /* some cell reached a non-physical state since the last check */
} rlb_status;

/* Boundary of a tube. RLB_BC_OPEN: three zero-gradient ghost cells per side (section "Riemann problem").
 * RLB_BC_PERIODIC: the tube wraps around. RLB_BC_HALO_LEFT / RLB_BC_HALO_RIGHT (flags, either or both, the
 * other side open): the tube is one x-slab of a longer tube split over several tubes, handles or GPUs; the
 * three ghost cells on that side are the neighbouring slab's edge cells, which the caller moves with
 * rlb_halo_pack / rlb_halo_unpack before every stage (rlb_stage). */
enum { RLB_BC_OPEN = 0, RLB_BC_PERIODIC = 1, RLB_BC_HALO_LEFT = 2, RLB_BC_HALO_RIGHT = 4 };

/* Storage of F. FP64: everything in FP64 (the parity path). FP32 / BF16: F stored in that type, advection,
 * equilibrium evaluation, collision and the Runge-Kutta combination in FP32, the moments accumulated with
 * compensated FP32 sums and reduced in FP64, the Landau-frame solve and the equilibrium coefficients in FP64.
 * All tubes of one handle use the same storage. */
enum { RLB_STORAGE_F64 = 0, RLB_STORAGE_F32 = 1, RLB_STORAGE_BF16 = 2 };

/* Fields written by rlb_moments, in this order. */
enum {
  RLB_F_N0 = 0, RLB_F_NX, RLB_F_T00, RLB_F_T0X, RLB_F_TXX, RLB_F_E, RLB_F_V, RLB_F_N, RLB_NFIELDS
};

/* One tube. tau <= 0 or tau = +inf means the ballistic regime (no collision). */
typedef struct {
  int32_t Qp;       /* radial Gauss-Laguerre order (the paper uses 3) */
  int32_t Qxi;      /* polar Gauss-Legendre order */
  int32_t Np;       /* radial truncation order of f^eq (the paper uses 2; at least 2) */
  int32_t Nv;       /* angular truncation order of f^eq (the paper uses 5) */
  int64_t Nx;       /* number of cells */
  double dx;        /* cell width; cell c has its centre at x_left + (c + 1/2) dx */
  double dt;        /* time step */
  double tau;       /* relaxation time */
  int32_t bc;       /* RLB_BC_OPEN, RLB_BC_PERIODIC, or RLB_BC_HALO_LEFT and/or RLB_BC_HALO_RIGHT */
  int32_t storage;  /* RLB_STORAGE_F64 (0), RLB_STORAGE_F32 or RLB_STORAGE_BF16; the same for every tube */
} rlb_tube;

/*
 * rlb_init - create a handle for ntubes tubes and set F to the truncated equilibrium of a per-cell state.
 *   Initial condition, Eq. (condinit): F_s(x) = F^eq_s(P(x), n(x), v(x)) with T = P/n.
 *   P, n, v: per-cell pressure, density and velocity, each sum_b Nx_b doubles (tubes one after the
 *   other), host pointers or, with ic_on_device != 0, device pointers. stream: a cudaStream_t (NULL =
 *   default stream). The handle owns all device memory it allocates; rlb_destroy frees it.
 *   Returns RLB_EINVAL for bad orders/sizes or a non-positive P or n, RLB_ENOMEM, RLB_ECUDA.
 */
rlb_status rlb_init(rlb_handle *out, const rlb_tube *tubes, int32_t ntubes, const double *P, const double *n,
                    const double *v, int32_t ic_on_device, void *stream);

/*
 * rlb_init_riemann - as rlb_init for the Riemann problem of Eq. (condinit): per tube b,
 *   states[6b..6b+5] = (P_L, n_L, v_L, P_R, n_R, v_R) and x_left[b] is the left edge of the domain. Cells
 *   whose centre is left of x = 0 take the left equilibrium, right of it the right one, and a centre at
 *   exactly x = 0 the mean of the two. states and x_left are host arrays.
 */
rlb_status rlb_init_riemann(rlb_handle *out, const rlb_tube *tubes, int32_t ntubes, const double *states,
                            const double *x_left, void *stream);

/*
 * rlb_step - advance every tube by nsteps time steps of SSP-RK3 (three stages per step), each stage
 *   computing moments, Landau frame, f^eq, collision and WENO5 advection (section "Numerical results",
 *   Eq. (Boltz)). Asynchronous on the handle's stream; nsteps >= 0. Returns RLB_EINVAL for a NULL handle
 *   or negative nsteps, RLB_ECUDA if a launch fails.
 */
rlb_status rlb_step(rlb_handle h, int64_t nsteps);

/*
 * Domain decomposition: one tube split into x-slabs (the method's one exchange step, section "Numerical
 * results": WENO5 reaches three cells on each side, so every Runge-Kutta stage needs the neighbouring slabs'
 * three edge cells of all Q velocities). A slab is a tube with RLB_BC_HALO_LEFT and/or RLB_BC_HALO_RIGHT; its
 * handle keeps the ghost cells beside each row. The caller runs each step as three stages and, before each
 * stage, moves the edge cells of that stage's input between neighbours (in one process, between handles of
 * one GPU, or between GPUs with NCCL or peer copies):
 *     for stage in 0, 1, 2:  rlb_halo_pack(h, stage, send); <send / receive>; rlb_halo_unpack(h, stage, recv);
 *                            rlb_stage(h, stage);
 * Buffer layout (elements of the handle's storage type, rlb_halo_size() of them): for every slab of the handle,
 * in tube order, a block of Q x 3 elements per halo side, left side first; a block holds, row s by row s, three
 * cells in ascending x. rlb_halo_pack writes a left block with the slab's cells 0, 1, 2 (for the left
 * neighbour's right ghosts) and a right block with cells Nx-3, Nx-2, Nx-1 (for the right neighbour's left
 * ghosts); rlb_halo_unpack reads a left block as the ghost cells -3, -2, -1 (the left neighbour's last three
 * cells) and a right block as Nx, Nx+1, Nx+2 (the right neighbour's first three). A slab result is bit-identical
 * to the same cells of the undivided tube. Slabs need Nx >= 3; rlb_step, rlb_autotune and the adjoint entry
 * points return RLB_EINVAL for handles with slabs.
 */

/* rlb_halo_size - elements of the exchange buffer of a handle (0 without slabs). */
int64_t rlb_halo_size(rlb_handle h);

/* rlb_halo_pack - write the edge cells of stage `stage`'s input (0: the state, 1 and 2: the intermediate
 *   Runge-Kutta states) into send (device pointer, rlb_halo_size() elements of the storage type). Ordered on
 *   the handle's stream, asynchronous. */
rlb_status rlb_halo_pack(rlb_handle h, int32_t stage, void *send);

/* rlb_halo_unpack - set the ghost cells of stage `stage`'s input from recv (device pointer, same layout).
 *   Ordered on the handle's stream, asynchronous. */
rlb_status rlb_halo_unpack(rlb_handle h, int32_t stage, const void *recv);

/* rlb_stage - run Runge-Kutta stage `stage` (0, 1, 2) of the current step for every tube of the handle (one
 *   stage kernel launch; the three in order make one rlb_step). Asynchronous on the handle's stream. */
rlb_status rlb_stage(rlb_handle h, int32_t stage);

/*
 * rlb_moments - write the macroscopic fields of the current state (section "Relativistic lattice
 *   Boltzmann equation"): N^0, N^x, T^00, T^0x, T^xx, the Landau-frame energy density e, velocity v and
 *   density n = -u_mu N^mu, as [RLB_NFIELDS][sum_b Nx_b] doubles into out (device pointer if
 *   out_on_device, else host; a host copy waits for the stream). Returns RLB_ENONPHYS if the sticky flag
 *   is set (the fields are still written). With FP32/BF16 storage the moments of tubes with collisions are
 *   the compensated sums the last stage accumulated while storing F (double-float, about 1e-13 relative to
 *   the exact sums of the stored F); ballistic tubes are summed over F in FP64.
 */
rlb_status rlb_moments(rlb_handle h, double *out, int32_t out_on_device);

/* rlb_get_state / rlb_set_state - copy F out of / into the handle in the packed layout (checkpoint and
 *   restore). F holds rlb_state_size() doubles; host or device pointer as flagged. */
rlb_status rlb_get_state(rlb_handle h, double *F, int32_t on_device);
rlb_status rlb_set_state(rlb_handle h, const double *F, int32_t on_device);

/* rlb_sync - wait for the handle's stream; returns RLB_ENONPHYS (and clears the flag) if it was set. */
rlb_status rlb_sync(rlb_handle h);

/* rlb_destroy - free the handle and its device memory (after waiting for its stream). NULL is a no-op. */
rlb_status rlb_destroy(rlb_handle h);

/* rlb_state_size - number of doubles in the packed state of a handle (sum_b Qp_b Qxi_b Nx_b). */
int64_t rlb_state_size(rlb_handle h);

/* rlb_error_string - static, human-readable name of a status. */
const char *rlb_error_string(rlb_status s);

/*
 * rlb_suggest_dt - time step min(cfl * dx, 0.9 tau): the CFL bound for particle speeds |xi| <= 1 (the
 *   paper bounds its step by the CFL condition in section "Numerical results"; cfl = 0.5 gives its
 *   dt = 0.5e-4 at dx = 1e-4) and the stiffness bound of SSP-RK3 with WENO5 advection: at cfl <= 0.5 the
 *   step is stable while dt gamma (1 + |v|) / tau <= 1.977 (linear analysis), i.e. up to |v| ~ 0.63 with
 *   0.9 tau. Faster flows need a smaller dt: near |v| = 1 the bound of the linear analysis is not enough,
 *   because the relaxation rate gamma (1 - v xi) / tau grows with the speed it relaxes (flows at |v| = 0.97
 *   .. 0.99 stepped at dt gamma (1 + |v|) / tau = 1.8 run away within a few steps; 0.25 .. 0.5 is stable).
 *   tau <= 0 or infinite: cfl * dx.
 */
double rlb_suggest_dt(double dx, double tau, double cfl);

/*
 * rlb_stiffness_limit - the largest k dt for which one SSP-RK3 step of dF/dt = -(xi/dx) D F - k F, with D the
 *   linear fifth-order upwind difference that WENO5 reduces to on smooth data, damps every Fourier mode at
 *   the Courant number nu = |xi| dt / dx (host computation: bisection over k dt, modes sampled on 4096 phases).
 *   About 2.513 at nu = 0, 1.977 at nu = 0.5; 0 if nu alone is unstable. The collision of Eq. (Boltz)
 *   relaxes direction xi at k = gamma (1 - beta xi) / tau, largest at gamma (1 + |beta| max|xi|) / tau.
 */
double rlb_stiffness_limit(double nu);

/*
 * rlb_warnings - read and clear the handle's sticky warning bits (waits for the handle's stream). The step
 *   goes on when a warning is raised; the results may be wrong.
 *   RLB_WARN_STIFF: in some cell of a tube with collisions, dt gamma (1 + |v| max|xi|) / tau exceeded the
 *     tube's rlb_stiffness_limit(max|xi| dt / dx): the relaxation of the fastest direction is outside the
 *     stable region of the scheme (a smaller dt is needed for that velocity).
 *   The bits are set by every stage a handle runs (rlb_step and the forward steps of rlb_record and
 *   rlb_backward); rlb_step_static has no handle and checks nothing. Returns RLB_EINVAL for a null argument,
 *   RLB_ECUDA if the read fails.
 */
enum { RLB_WARN_STIFF = 1 };
rlb_status rlb_warnings(rlb_handle h, uint32_t *bits);

/*
 * rlb_quadrature - the library's own nodes and weights (host, FP64): pbar[Qp], wp[Qp] for the generalised
 *   Gauss-Laguerre rule with weight pbar e^-pbar, xi[Qxi], wxi[Qxi] for Gauss-Legendre, both ascending
 *   (section "Discretization of the momentum space using quadrature rules").
 */
rlb_status rlb_quadrature(int32_t Qp, int32_t Qxi, double *pbar, double *wp, double *xi, double *wxi);

/*
 * Launch shape of a handle's steps (no counterpart in the paper; it changes how the work is scheduled, never
 * the arithmetic: every choice gives bit-identical results).
 *   schedule:     RLB_SCHED_TILE (one CTA per tile, the default), RLB_SCHED_STRIDE (persistent grid, tiles by
 *                 grid stride) or RLB_SCHED_COUNTER (persistent grid, tiles handed out by an atomic counter:
 *                 to whole CTAs in the FP64 kernel, to single warps in the reduced-precision kernel, whose
 *                 tiles are warp tiles; nothing waits on another CTA or warp).
 *   ctas_per_sm:  persistent grid = SMs x ctas_per_sm; 0 takes the occupancy limit.
 *   graph_steps:  rlb_step replays a captured CUDA graph of this many steps (on a private stream joined to the
 *                 handle's stream by events); 0 launches directly. Calls made while the handle's stream is
 *                 being captured by the caller always launch directly. 1 <= graph_steps <= 64 otherwise.
 *   order:        tile order, RLB_ORDER_COST (most expensive tubes first, the default) or RLB_ORDER_INTERLEAVE
 *                 (tubes interleaved tile by tile).
 *   split:        work items per tile of the FP64 stage kernel: item k advances velocity rows [k Q / split,
 *                 (k + 1) Q / split) of the tile after reducing its moments over all rows. 0 (the default)
 *                 chooses: one item per tile when the tiles fill the GPU's resident CTA slots, else
 *                 min(8, slots / tiles). 1 <= split <= 8 fixes it. Handles with reduced storage use one.
 */
enum { RLB_SCHED_TILE = 0, RLB_SCHED_STRIDE = 1, RLB_SCHED_COUNTER = 2 };
enum { RLB_ORDER_COST = 0, RLB_ORDER_INTERLEAVE = 1 };
typedef struct {
  int32_t schedule;
  int32_t ctas_per_sm;
  int32_t graph_steps;
  int32_t order;
  int32_t split;
} rlb_launch;

/* rlb_get_launch / rlb_set_launch - read or change the launch shape (RLB_EINVAL for values out of range). */
rlb_status rlb_get_launch(rlb_handle h, rlb_launch *out);
rlb_status rlb_set_launch(rlb_handle h, const rlb_launch *cfg);

/*
 * rlb_autotune - time every launch shape (schedules x ctas_per_sm in {occupancy, 1, 2} x both tile orders x
 *   graph on/off x split automatic or 1 where the automatic choice is not 1) for trial_steps steps on the handle's own tubes and state, keep the fastest. The state is
 *   saved first and restored after every trial, so the handle's state is unchanged on return. best and
 *   best_ms_per_step (either may be NULL) receive the choice and its time per step. Synchronous.
 */
rlb_status rlb_autotune(rlb_handle h, int32_t trial_steps, rlb_launch *best, double *best_ms_per_step);

/*
 * rlb_step_static - advance ONE tube by nsteps SSP-RK3 steps without allocating device memory.
 *   This entry point has no counterpart in the paper; it exists for callers that cannot call cudaMalloc
 *   (or anything that allocates device memory) at the point where they step: a host application that has
 *   handed the device memory to its own pool allocator, a plugin whose host forbids device allocation once
 *   running, or a latency-critical loop where a cudaMalloc, which can synchronise the device, is not
 *   acceptable. rlb_init allocates the state and scratch buffers of a handle; this call takes the state
 *   from the caller and keeps its scratch (the two intermediate Runge-Kutta stages, the quadrature tables
 *   and the tile list) in one file-scope device array of RLB_STATIC_SCRATCH_BYTES bytes that every GPU which
 *   loads the library holds until the process exits.
 *   tube:  host pointer to the tube (same rules as rlb_init, bc open or periodic, storage RLB_STORAGE_F64).
 *   F_in:  device pointer, packed state [Q][Nx] doubles (Q = Qp * Qxi), read only.
 *   F_out: device pointer, packed state [Q][Nx] doubles, written with the state after nsteps steps; may
 *          equal F_in (in place). With nsteps = 0 nothing is launched and F_out is left untouched.
 *   flag:  optional device pointer; a non-physical cell ORs 1 into it (the caller zeroes it). NULL: such
 *          cells are not reported.
 *   stream: cudaStream_t to launch on. The call returns once its small host-side tables have been copied
 *          out (CUDA may first wait for earlier work on that stream, as for any copy from pageable memory);
 *          the steps themselves run asynchronously.
 *   Size limit: 2 Q Nx doubles of stage scratch plus the tables (about 8 (Qxi + 16) (NV_MAX + 2) bytes) and
 *   8 bytes per 61 cells must fit in RLB_STATIC_SCRATCH_BYTES, e.g. Q = 24 up to Nx of about 170000, Q = 600
 *   up to about 6800; larger tubes return RLB_EINVAL before anything is launched.
 *   Set-up: the first call on a device (with that device current) looks up the array's device address and
 *   uploads the series tables that the kernels share with rlb_init; these steps synchronise, so make the first
 *   call on each device before any stream capture. Later calls only enqueue copies into the array and the
 *   kernel launches.
 *   Every call uses the same array and leaves its contents behind: calls that overlap on the GPU (on two
 *   streams, or from two threads) race on it and must be ordered by the caller.
 *   The small tables are copied into the array from host memory that exists only during the call, so a
 *   stream that is being captured is refused with RLB_EINVAL (a captured copy would read that memory again
 *   at every replay). Unlike the handle-based steps, this call keeps no warning word: it reports
 *   non-physical cells through flag but raises no stiffness warning (RLB_WARN_STIFF).
 *   Returns RLB_EINVAL for bad arguments, a tube over the limit or a capturing stream, RLB_ECUDA if a CUDA
 *   call fails.
 */
#define RLB_STATIC_SCRATCH_BYTES (64u << 20)
rlb_status rlb_step_static(const rlb_tube *tube, const double *F_in, double *F_out, int64_t nsteps,
                           int32_t *flag, void *stream);

/* ---------------------------------------------------------------------------------------------------------
 * Adjoint (reverse-mode gradient) of the time step. The paper has no adjoint; these entry points give the
 * gradient of a scalar loss of the state after a run with respect to the initial state, the initial fields
 * (P, n, v) and log(tau) of every tube, by the exact transpose of each stage of the discrete step (WENO5
 * flux differences, Anderson-Witting collision with the equilibrium of Eq. (feqtrunc) through the Landau
 * frame, SSP-RK3 combination) evaluated in FP64 on the GPU. The time step dt of a tube is held fixed.
 * Handles with reduced-precision storage return RLB_EINVAL from all five.
 * Layouts: "packed state" = the layout of rlb_get_state (per tube [Q][Nx] doubles, tube after tube);
 * "field layout" = [sum of Nx] doubles, tube after tube. All pointers below are device pointers unless
 * stated; the calls run on the handle's stream and return after their work has finished.
 * --------------------------------------------------------------------------------------------------------- */

/*
 * rlb_record - advance every tube by nsteps steps as rlb_step does (bit-identical results), keeping a
 *   checkpoint of the state every `every` steps (the state before steps 0, every, 2 every, ...) in device
 *   memory owned by the handle; a later rlb_backward recomputes each segment of `every` steps from its
 *   checkpoint. Replaces any earlier record. Memory: ceil(nsteps / every) states. With every >= nsteps the
 *   record keeps every stage input instead (3 nsteps + 1 states, the buffer rlb_backward needs anyway) and
 *   rlb_backward recomputes nothing.
 *   Returns RLB_EINVAL (nsteps < 1, every < 1, reduced storage), RLB_ENOMEM, RLB_ECUDA, or RLB_ENONPHYS if a
 *   cell became non-physical during the run.
 */
rlb_status rlb_record(rlb_handle h, int64_t nsteps, int32_t every);

/*
 * rlb_backward - reverse sweep over the last rlb_record.
 *   seed:         packed state, dL/dF of the state after the recorded steps (read only).
 *   grad_state:   packed state, written with dL/dF of the state before the recorded steps; may be NULL.
 *   grad_log_tau: HOST array [ntubes], written with dL/dlog(tau) of each tube (0 for tau = infinity); may be
 *                 NULL.
 *   The handle's state is not changed. Scratch: (3 min(every, nsteps) + 1) + 4 states, allocated on first
 *   use and kept until rlb_destroy. Returns RLB_EINVAL (no record, reduced storage, seed NULL), RLB_ENOMEM, RLB_ECUDA,
 *   RLB_ENONPHYS (a recomputed cell was non-physical).
 */
rlb_status rlb_backward(rlb_handle h, const double *seed, double *grad_state, double *grad_log_tau);

/*
 * rlb_moments_vjp - seed of rlb_backward from the adjoint of the five conserved moments:
 *   grad_moments: [5][sum of Nx] (field layout per row: N^0, N^x, T^00, T^0x, T^xx, as rows 0..4 of
 *                 rlb_moments), read only.
 *   seed:         packed state, written with dL/dF_s(x) = sum_a dL/dM_a(x) c_a(s), c = (pbar, pbar xi,
 *                 pbar^2, pbar^2 xi, pbar^2 xi^2) (the moment sums of the section "Relativistic lattice
 *                 Boltzmann equation").
 */
rlb_status rlb_moments_vjp(rlb_handle h, const double *grad_moments, double *seed);

/*
 * rlb_fields_vjp - seed of rlb_backward from the adjoint of all the fields of rlb_moments at the handle's
 *   current state (after rlb_record, the state after the recorded steps):
 *   grad_fields:  [RLB_NFIELDS][sum of Nx] (field layout per row, rows as in rlb_moments: N^0, N^x, T^00,
 *                 T^0x, T^xx, e, v, n), read only.
 *   seed:         packed state, written with dL/dF_s(x) = sum_a G_a(x) c_a(s), c as in rlb_moments_vjp, where
 *                 G_a = dL/dM_a + dL/de de/dM_a + dL/dv dv/dM_a + dL/dn dn/dM_a: the derivatives of the
 *                 Landau-frame solution (section "Relativistic lattice Boltzmann equation", T^mu_nu u^nu =
 *                 -e u^mu, n = -u_mu N^mu) at each cell's moments.
 *   Returns RLB_EINVAL for NULL pointers or reduced storage, RLB_ENONPHYS if a cell's moments have no Landau
 *   frame (its seed then carries only the moments' share).
 */
rlb_status rlb_fields_vjp(rlb_handle h, const double *grad_fields, double *seed);

/*
 * rlb_init_vjp - adjoint of the initial condition of rlb_init (F = F^eq of Eq. (feqtrunc) with T = P/n and
 *   beta = v in every cell): from dL/dF of that state to dL/dP, dL/dn, dL/dv.
 *   P, n, v:           field layout, the initial fields given to rlb_init (read only).
 *   grad_state:        packed state, dL/dF of the initial state (e.g. grad_state of rlb_backward).
 *   grad_P, grad_n, grad_v: field layout, written.
 *   Returns RLB_EINVAL for NULL pointers, reduced storage or a non-physical initial cell.
 */
rlb_status rlb_init_vjp(rlb_handle h, const double *P, const double *n, const double *v,
                        const double *grad_state, double *grad_P, double *grad_n, double *grad_v);

#ifdef __cplusplus
}
#endif

#endif /* RLB_H */
