/*
 * teno.h -- C-ABI of the GB300 (sm_103a) TENO5-LAD compressible-Euler library.
 *
 * The library computes the semi-discrete right-hand side of the Euler
 * equations with the fifth-order targeted ENO scheme whose cutoff C_T adapts
 * locally between 1e-10 and 1e-4 (Peng et al., arXiv 2003.09145, "TENO5-LAD"),
 * and advances it with SSP-RK3.  All arithmetic is IEEE binary64 on the GPU.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Conservative state U: device memory, float64, structure of arrays
 *   U[nvar][n_z][n_y][n_x] with x fastest, nvar = ndim + 2, components
 *   (rho, rho u, [rho v, [rho w]], E), E = p/(gamma-1) + rho |u|^2 / 2
 *   (eq. 4.7).  Base address 16-byte aligned, no padding, no ghost cells:
 *   boundaries are applied inside the kernels.
 * - Every array is owned by the caller.  The library never allocates device
 *   memory and never synchronises in a compute call: work is enqueued on the
 *   caller's stream (`stream` is a cudaStream_t; NULL = legacy default stream).
 *   Scratch space is the caller's workspace `ws` of at least
 *   teno_workspace_bytes() bytes (256-byte aligned); it also holds the device
 *   status word read by teno_get_device_status().
 * - Arguments are validated on the host before anything is launched; an
 *   invalid call returns TENO_ERR_INVALID_ARG (or TENO_ERR_WORKSPACE /
 *   TENO_ERR_UNSUPPORTED) and enqueues nothing.  Conditions found on the
 *   device (non-physical density or pressure, a time-out of a bounded wait)
 *   are recorded in the workspace's status word.  No call throws.
 * - Flag bytes (optional output of teno_rhs): one byte per interface, per
 *   characteristic field and per side; bits 0..2 = delta_0..delta_2 of
 *   eq. 2.14, bits 3..6 = the magnitude m of eq. 3.1.  Layout: for each
 *   direction d in order, a block [nvar][2 (0 = f^+, 1 = f^-)][interface grid],
 *   where the interface grid of direction d has n_d + 1 points along d (entry
 *   i lies between cells i-1 and i) and n_k along the other axes, x fastest.
 */
#ifndef TENO_H
#define TENO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TENO_ABI_VERSION 2

typedef enum {
  TENO_OK = 0,
  TENO_ERR_INVALID_ARG = 1,   /* bad pointer, size, alignment or parameter   */
  TENO_ERR_UNSUPPORTED = 2,   /* valid request the library does not implement */
  TENO_ERR_CUDA = 3,          /* a CUDA runtime call or launch failed        */
  TENO_ERR_NONPHYSICAL = 4,   /* device saw rho <= 0, p <= 0 or a non-finite */
  TENO_ERR_TIMEOUT = 5,       /* a bounded device wait ran out               */
  TENO_ERR_WORKSPACE = 6,     /* workspace missing, misaligned or too small  */
  TENO_ERR_UNIMPLEMENTED = 7
} teno_status;

typedef enum {
  TENO_BC_PERIODIC = 0,      /* wrap-around                                   */
  TENO_BC_TRANSMISSIVE = 1,  /* zero gradient: the boundary cell is copied    */
  TENO_BC_REFLECTIVE = 2,    /* solid wall: cells mirrored about the wall with */
                             /* the normal velocity reversed (Sec. 4.2's blast */
                             /* waves); teno_rhs, teno_rk3_step and            */
                             /* teno_rhs_noalloc only (the adjoint and batched */
                             /* entry points return TENO_ERR_UNSUPPORTED)      */
  TENO_BC_DIRICHLET = 3      /* fixed state: every ghost cell of a face holds  */
                             /* the face's teno_grid.bc_state (Sec. 4.3.2's    */
                             /* Rayleigh-Taylor top and bottom); teno_rhs,     */
                             /* teno_rk3_step and the staged step only         */
} teno_bc;

/* The reconstruction's cutoff (teno_grid.scheme).  The paper's method is
 * TENO_SCHEME_LAD; the others are the schemes it is compared with (Sec. 4,
 * Tab. 2), on the same characteristic-wise flux and the same kernels. */
typedef enum {
  TENO_SCHEME_LAD = 0,     /* C_T = Lad(m), m = B_l + floor(theta (B_u - B_l))  */
                           /* (eq. 3.1-3.4)                                    */
  TENO_SCHEME_TENO5 = 1,   /* fixed C_T = 10^-ct_m (eq. 2.14; Sec. 4: 1e-7)     */
  TENO_SCHEME_TENO5A = 2,  /* TENO5-A: C_T = 10^-floor(beta) from the sensor    */
                           /* eta of eq. 2.16-2.18 (alpha_1 10.5, alpha_2 3.5,  */
                           /* C_r 0.25, xi 1e-3; eq. 2.18's denominator read    */
                           /* as (df_{i+1/2})^2 + (df_{i-1/2})^2 + eps)         */
  TENO_SCHEME_WENOZ = 3    /* WENO-Z: omega_k = alpha_k / sum alpha,            */
                           /* alpha_k = c_k (1 + tau_5 / (beta_k + eps))        */
                           /* (tau_5 of eq. 2.12); no cutoff                    */
} teno_scheme;

/* Grid and scheme parameters (problem statement: eq. 2.1-2.2, eq. 4.7,
 * eq. 3.1-3.2).  Unused dimensions must have n = 1, dx = 1.  The interfaces
 * along each direction are indexed with 32 bits: a grid with 2^32 or more
 * interfaces along one direction (e.g. 2048 x 2048 x 1024 cells along x) is
 * TENO_ERR_INVALID_ARG. */
typedef struct {
  int ndim;          /* 1, 2 or 3                                            */
  int64_t n[3];      /* cells along x, y, z                                  */
  double dx[3];      /* uniform spacing along x, y, z (> 0)                  */
  int bc[3];         /* teno_bc per direction (both faces alike)             */
  double gamma;      /* ratio of specific heats, eq. 4.7 (paper: 1.4)        */
  double H;          /* discontinuity threshold H of eq. 3.2 (paper: 10)     */
  int b_l, b_u;      /* magnitude bounds B_l, B_u of eq. 3.1 (paper: 4, 10)  */
  double eps;        /* epsilon of eq. 2.8 / eq. 3.2 (paper: 1e-6)           */
  int scheme;        /* teno_scheme (TENO_SCHEME_LAD = 0)                     */
  int ct_m;          /* TENO_SCHEME_TENO5 only: C_T = 10^-ct_m, 1..15         */
  double grav[3];    /* body acceleration g: the source (0, rho g, rho u.g)   */
                     /* is added to L(U) (Sec. 4.3.2: rho in the y momentum,  */
                     /* rho v in the energy, g = (0, 1)); zero: no source.    */
                     /* teno_rhs, teno_rk3_step, the staged step only         */
  double bc_state[3][2][5]; /* TENO_BC_DIRICHLET axes: the conservative      */
                     /* ghost state (rho, rho u.., E; first nvar entries) of  */
                     /* the low [0] and high [1] face; rho, p > 0, finite     */
} teno_grid;

/* Workspace sizes for each operation (teno_workspace_bytes `op`). */
enum {
  TENO_OP_RHS = 0,          /* teno_rhs                                     */
  TENO_OP_RK3 = 1,          /* teno_rk3_step                                */
  TENO_OP_RHS_ADJOINT = 2,  /* teno_rhs_adjoint                             */
  TENO_OP_RK3_ADJOINT = 3   /* teno_rk3_step_adjoint                        */
};

/* Fills `g` with the paper's parameters (gamma 1.4, H 10, B_l 4, B_u 10,
 * eps 1e-6, TENO_SCHEME_LAD, ct_m 7; Sec. 2 and Sec. 4) for an ndim grid of n cells of spacing dx with
 * boundary type bc on every axis. */
void teno_grid_default(teno_grid* g, int ndim, const int64_t* n,
                       const double* dx, int bc);

/* Bytes of workspace `op` needs for grid g (0 if g is invalid). */
size_t teno_workspace_bytes(const teno_grid* g, int op);

/* Number of flag bytes teno_rhs writes for grid g (see the layout above). */
int64_t teno_flag_count(const teno_grid* g);

/*
 * teno_rhs -- the semi-discrete operator L(U) of eq. 2.2,
 *   dU/dt = - sum_d (F^_{d,i+1/2} - F^_{d,i-1/2}) / dx_d,
 * computed dimension by dimension.  At every interface: global
 * Lax-Friedrichs splitting (alpha per direction and characteristic field,
 * the maximum of |lambda| over all cells of U), projection onto the Roe
 * averaged characteristic fields, TENO5 reconstruction of each split flux
 * (eq. 2.4-2.15) with the adaptive cutoff C_T = Lad(m) (eq. 3.1-3.4),
 * back-projection (the convective-term paragraph of Sec. 4).
 *   U     : [in]  device, nvar * ncell doubles (layout above).
 *   dUdt  : [out] device, nvar * ncell doubles; must not alias U.
 *   flags : [out] device, teno_flag_count(g) bytes, or NULL.
 *   ws    : device workspace of >= teno_workspace_bytes(g, TENO_OP_RHS).
 */
teno_status teno_rhs(const teno_grid* g, const double* U, double* dUdt,
                     uint8_t* flags, void* ws, size_t ws_bytes, void* stream);

/*
 * teno_rk3_step -- one SSP-RK3 step (eq. 4.1-4.3) of U in place:
 *   U1 = U + dt L(U);  U2 = 3/4 U + 1/4 U1 + 1/4 dt L(U1);
 *   U <- 1/3 U + 2/3 U2 + 2/3 dt L(U2).
 * dt = dt_fixed if dt_fixed > 0, else the CFL step of eq. dt1 (1D) /
 * eq. dt2 (2D) / sigma / sum_d(max(|u_d|+c)/dx_d) (3D) with sigma = cfl,
 * evaluated on the device from U; in both cases dt is clipped to
 * t_end - t so the step lands on t_end.  When t >= t_end nothing changes.
 *   U      : [in/out] device state.
 *   t_dev  : [in/out] device double, the current time (advanced by dt).
 *   dt_dev : [out] device double receiving the dt used, or NULL.
 *   ws     : >= teno_workspace_bytes(g, TENO_OP_RK3).
 */
teno_status teno_rk3_step(const teno_grid* g, double* U, double cfl,
                          double dt_fixed, double* t_dev, double t_end,
                          double* dt_dev, void* ws, size_t ws_bytes,
                          void* stream);

/* ------------------------------------------------------------------------ */
/* Decomposed stepping: one SSP-RK3 step in stages, so that a caller that    */
/* splits the domain over GPUs (or over slabs) can exchange halos and reduce */
/* the LF speeds between the stages.                                          */
/* ------------------------------------------------------------------------ */

/*
 * A step of teno_rk3_step is, for stage k = 1, 2, 3 with input
 * Uin = U^n, U1, U2 and output Uout = U1, U2, U^n:
 *   teno_rk3_stage_begin(g, Uin, ...)   cell pass: primitives of Uin and this
 *                                       grid's Lax-Friedrichs speeds, written
 *                                       to the workspace as nine 64-bit words
 *                                       at byte teno_alpha_offset() (per
 *                                       direction: max|u-c|, max|u|, max|u+c|
 *                                       as the bit patterns of non-negative
 *                                       doubles, so an integer maximum over
 *                                       ranks is the maximum of the speeds);
 *   [the caller replaces the nine words by their maximum over all ranks]
 *   teno_rk3_stage_end(g, k, Uin, U^n, Uout, ...)
 *                                       stage 1 also takes dt (eq. dt1 / dt2 /
 *                                       the 3D form, from the speeds in the
 *                                       workspace, or dt_fixed) and advances
 *                                       *t_dev; then the interface fluxes,
 *                                       the difference and the stage of
 *                                       eq. 4.1 / 4.2 / 4.3.
 * Called in this order on one grid and workspace with nothing in between,
 * the stages give teno_rk3_step's result bit for bit (global LF speeds and
 * dt are functions of the speeds alone, Sec. 4 and reading C7).
 *
 * Domain decomposition along the slowest axis (z in 3D, y in 2D, x in 1D):
 * a rank stores its slab with three ghost planes on each side (n along that
 * axis = interior planes + 6; transmissive bc on that axis) and fills the
 * ghost planes of every stage input before stage_begin -- from the
 * neighbouring slabs' interior planes (periodic ends wrap), or, at a
 * transmissive end, with copies of the boundary plane.  The interior cells'
 * fluxes then read only real data, and the interior result equals the
 * undivided grid's bit for bit.  The ghost planes' own results are not
 * meaningful.
 *   Uin, Un, Uout : device states of grid g; stage 1: Uin == Un, Uout != Un;
 *                   stage 2: Uout distinct from both; stage 3: Uout may be Un.
 *   t_dev, dt_dev, cfl, dt_fixed, t_end : as teno_rk3_step (stage 1 only).
 *   ws : >= teno_workspace_bytes(g, TENO_OP_RK3), the same for all stages.
 */
teno_status teno_rk3_stage_begin(const teno_grid* g, const double* Uin, void* ws,
                                 size_t ws_bytes, void* stream);
teno_status teno_rk3_stage_end(const teno_grid* g, int stage, const double* Uin,
                               double* Un, double* Uout, double cfl,
                               double dt_fixed, double* t_dev, double t_end,
                               double* dt_dev, void* ws, size_t ws_bytes,
                               void* stream);

/* Byte offset, in any workspace, of the nine LF-speed words (above). */
size_t teno_alpha_offset(void);

/*
 * teno_planes_copy -- copies nplanes consecutive planes along the slowest
 * axis (all nvar fields) from src to dst, both device arrays: a state of
 * grid g (planes from src_plane / dst_plane) or, with *_packed = 1, a packed
 * buffer [nvar][nplanes][plane] (plane = cells of one plane).  One
 * cudaMemcpy2DAsync on `stream`; used for halo exchange (between slabs on
 * one GPU, or packing for a transfer between GPUs).
 */
teno_status teno_planes_copy(const teno_grid* g, const double* src, int64_t src_plane,
                             int src_packed, double* dst, int64_t dst_plane,
                             int dst_packed, int64_t nplanes, void* stream);

/* ------------------------------------------------------------------------ */
/* Batched mode: many independent 1D problems advanced together.             */
/* ------------------------------------------------------------------------ */

/* A batch of nprob 1D Euler problems packed back to back: problem p owns the
 * cells offsets[p] .. offsets[p+1]-1 of the SoA state U[3][ncell]
 * (rho, rho u, E), has its own spacing dx[p], time t[p] and final time
 * t_end[p], and its own global Lax-Friedrichs speeds.  Boundary type and
 * scheme parameters are shared. */
typedef struct {
  int64_t nprob;     /* number of problems (>= 1)                            */
  int64_t ncell;     /* total cells, offsets[nprob]                          */
  int bc;            /* teno_bc of every problem's two ends                   */
  double gamma;      /* eq. 4.7                                               */
  double H;          /* eq. 3.2                                               */
  int b_l, b_u;      /* eq. 3.1                                               */
  double eps;        /* eq. 2.8                                               */
} teno_batch;

/* Launch shape of the batched kernel (NULL = 128 threads, 4 CTAs per SM).
 * block: 64, 128 or 256 threads; ctas_per_sm: persistent CTAs per SM. */
typedef struct {
  int block;
  int ctas_per_sm;
} teno_batch_tuning;

/* Workspace bytes of a batch (0 if b is invalid). */
size_t teno_batch_workspace_bytes(const teno_batch* b);

/*
 * teno_batch_prepare -- checks the host copy of the offsets (offsets[0] = 0,
 * offsets[nprob] = ncell, every problem at least one cell), stores the
 * processing order (largest problems first) in the workspace and clears its
 * status word.  Call once per workspace and batch layout before stepping; it
 * waits for `stream`.
 */
teno_status teno_batch_prepare(const teno_batch* b, const int64_t* offsets_host,
                               void* ws, size_t ws_bytes, void* stream);

/*
 * teno_rk3_step_batched -- one SSP-RK3 step (eq. 4.1-4.3) of every problem,
 * three persistent launches (one per stage).  Per problem: dt = dt_fixed if
 * dt_fixed > 0, else eq. dt1 with sigma = cfl from its own state, clipped to
 * t_end[p] - t[p]; problems with t[p] >= t_end[p] are left unchanged.  The
 * arithmetic per problem is exactly that of teno_rk3_step on the problem
 * alone.
 *   offsets : device int64[nprob + 1];  dx : device double[nprob]
 *   U       : [in/out] device double[3 * ncell]
 *   t_dev   : [in/out] device double[nprob];  t_end_dev : device double[nprob]
 *   ws      : >= teno_batch_workspace_bytes(b), prepared by teno_batch_prepare.
 */
teno_status teno_rk3_step_batched(const teno_batch* b, const int64_t* offsets,
                                  const double* dx, double* U, double* t_dev,
                                  const double* t_end_dev, double cfl,
                                  double dt_fixed,
                                  const teno_batch_tuning* tuning, void* ws,
                                  size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------ */
/* Adjoint (vector-Jacobian products).                                       */
/* ------------------------------------------------------------------------ */

/* Workspace bytes of teno_rhs_adjoint (op = TENO_OP_RHS_ADJOINT) or
 * teno_rk3_step_adjoint (op = TENO_OP_RK3_ADJOINT) on grid g; 0 if invalid. */
size_t teno_adjoint_workspace_bytes(const teno_grid* g, int op);

/*
 * teno_rhs_adjoint -- U_bar += J(U)^T dUdt_bar, J = dL/dU of the right-hand
 * side of teno_rhs (eq. 2.2).  The stencil selections (delta of eq. 2.14 and
 * m of eq. 3.1) are held at their values for U: the cutoff is piecewise
 * constant, so J is the derivative of L almost everywhere.  The global
 * Lax-Friedrichs speed max_cells |lambda_s| is differentiated through its
 * arg-max cell (the lowest linear index on ties).  Deterministic: no atomics
 * on floating-point data.  The TENO schemes (LAD, TENO5, TENO5-A) only:
 * WENO-Z's weights are not piecewise constant (TENO_ERR_UNSUPPORTED).
 *   U, dUdt_bar : [in] device, nvar * ncell doubles.
 *   U_bar       : [in/out] device, accumulated; must not alias the inputs.
 *   ws          : >= teno_adjoint_workspace_bytes(g, TENO_OP_RHS_ADJOINT).
 */
teno_status teno_rhs_adjoint(const teno_grid* g, const double* U,
                             const double* dUdt_bar, double* U_bar, void* ws,
                             size_t ws_bytes, void* stream);

/*
 * teno_rk3_step_adjoint -- reverse of one SSP-RK3 step of fixed size dt
 * (eq. 4.1-4.3) taken from U_n: recomputes the stages U1, U2 and returns
 *   Ubar_n = dJ/dU_n given Ubar_next = dJ/dU_{n+1}
 * (Ubar_n is overwritten; it may alias Ubar_next).  dt carries no gradient.
 *   ws : >= teno_adjoint_workspace_bytes(g, TENO_OP_RK3_ADJOINT).
 */
teno_status teno_rk3_step_adjoint(const teno_grid* g, const double* U_n,
                                  double dt, const double* Ubar_next,
                                  double* Ubar_n, void* ws, size_t ws_bytes,
                                  void* stream);

/*
 * teno_rk3_step_adjoint_staged -- the same reverse step with the stages U1,
 * U2 of eq. 4.1-4.2 supplied by the caller (as teno_rk3_stage_end wrote
 * them for this step with dt_fixed = dt) instead of recomputed: the result
 * equals teno_rk3_step_adjoint's bit for bit when they are.  A rollout that
 * replays its steps anyway keeps the stages and saves two right-hand-side
 * evaluations per reverse step.
 *   U_n, U1, U2 : [in] device, nvar * ncell doubles.
 *   Ubar_n      : [out] may alias Ubar_next, not U_n, U1 or U2.
 *   ws          : >= teno_adjoint_workspace_bytes(g, TENO_OP_RK3_ADJOINT).
 */
teno_status teno_rk3_step_adjoint_staged(const teno_grid* g, const double* U_n,
                                         const double* U1, const double* U2,
                                         double dt, const double* Ubar_next,
                                         double* Ubar_n, void* ws,
                                         size_t ws_bytes, void* stream);

/*
 * teno_get_device_status -- waits for `stream`, then returns in *status the
 * status recorded on the device in workspace `ws` since the last call
 * (TENO_OK, TENO_ERR_NONPHYSICAL or TENO_ERR_TIMEOUT) and clears it.
 * The return value reports the host-side outcome of the query itself.
 */
teno_status teno_get_device_status(void* ws, void* stream, int* status);

/* ------------------------------------------------------------------------ */
/* Scalar mode: linear advection, the paper's scalar test problems.          */
/* ------------------------------------------------------------------------ */

/* Reconstruction used by the scalar mode. */
enum {
  TENO_SCALAR_LAD = 0,      /* TENO5-LAD (eq. 2.4-2.15, 3.1-3.4)               */
  TENO_SCALAR_UPWIND5 = 1   /* the fixed linear weights of eq. 2.3           */
};

/* Bytes of workspace the scalar mode needs for grid g (0 if g is not a valid
 * periodic 1D grid). */
size_t teno_scalar_workspace_bytes(const teno_grid* g);

/*
 * teno_scalar_rhs -- right-hand side of u_t + a u_x = 0 (eq. 4.4) on a
 * periodic 1D grid: the flux f = a u is split by global Lax-Friedrichs
 * (alpha = |a|), f^+ = (a + |a|) u / 2 is reconstructed from u_{i-2..i+2}
 * and f^- = (a - |a|) u / 2 from u_{i+3..i-1} with `mode` (TENO_SCALAR_*),
 * and dudt_i = -(f^_{i+1/2} - f^_{i-1/2}) / dx (eq. 2.2).
 *   g      : ndim = 1, bc[0] = TENO_BC_PERIODIC (else TENO_ERR_UNSUPPORTED);
 *            H, b_l, b_u, eps as for the Euler path; gamma is unused.
 *   a      : advection speed (finite).
 *   u      : [in]  device, n[0] doubles.
 *   dudt   : [out] device, n[0] doubles; must not alias u.
 *   ws     : >= teno_scalar_workspace_bytes(g).
 */
teno_status teno_scalar_rhs(const teno_grid* g, double a, int mode, const double* u,
                            double* dudt, void* ws, size_t ws_bytes, void* stream);

/*
 * teno_scalar_rk3_step -- one SSP-RK3 step (eq. 4.1-4.3) of fixed dt > 0 of
 * the same problem, u in place (the caller clips the last step to its final
 * time).
 */
teno_status teno_scalar_rk3_step(const teno_grid* g, double a, int mode, double* u, double dt,
                                 void* ws, size_t ws_bytes, void* stream);

/*
 * teno_rhs_noalloc -- teno_rhs for callers that cannot allocate device memory.
 * The paper has no counterpart; this is a deployment aid.
 *
 * Who needs it: code that may not call cudaMalloc -- a plugin running inside
 * another framework's memory pool or allocator, a host application that
 * forbids device allocation on its threads, or a deployment with a fixed,
 * pre-planned memory footprint.  Such callers can pass their own input and
 * output arrays but cannot supply the workspace teno_rhs needs.  This entry
 * point computes the same L(U) with the same kernels and allocates nothing:
 * its scratch is one file-scope device array of TENO_NOALLOC_SCRATCH_BYTES,
 * which every GPU that loads the library holds until the process exits.
 *   U    : [in]  device, nvar * ncell doubles (layout above).
 *   dUdt : [out] device, nvar * ncell doubles; must not alias U.
 * Size limit: a call needs 256 + 8 (2 ndim + 3) ncell + 8 (ndim + 2) max_d
 * (#interfaces_d) bytes (each term rounded up to 256); larger grids are
 * rejected with TENO_ERR_WORKSPACE before anything is launched.  In 1D that is
 * up to 131,065 cells; in 2D 308^2; in 3D 42^3.
 * The first call on each device looks up the array's device address (with
 * that device current) and caches it; make that first call before capturing
 * a stream into a CUDA graph.  The cached address dies with the device's
 * context: after cudaDeviceReset on a device, do not call this entry point on
 * that device again in the same process.
 * All calls share the one array and each call starts by clearing the parts
 * that must start at zero, so calls whose work overlaps on the GPU (other
 * streams, other host threads) race and give wrong results: serialise them.
 * Selection flags and device-side status are not reported by this variant.
 */
#define TENO_NOALLOC_SCRATCH_BYTES (8u << 20)
teno_status teno_rhs_noalloc(const teno_grid* g, const double* U, double* dUdt,
                             void* stream);

/* Kernel kinds reported by the launch timer. */
enum {
  TENO_KERNEL_CELL = 0,  /* primitive variables + LF wave-speed reduction   */
  TENO_KERNEL_FLUX = 1,  /* interface fluxes of one direction               */
  TENO_KERNEL_DIFF = 2,  /* conservative difference / fused RK3 stage       */
  TENO_KERNEL_DT = 3,    /* CFL time step                                   */
  TENO_KERNEL_KINDS = 4
};

/*
 * teno_timer_begin / teno_timer_end -- measurement aid (no counterpart in the
 * paper).  Between the two calls every kernel the library launches is
 * bracketed by CUDA events on its stream (at most 8192 launches; later ones
 * are not timed and teno_timer_end then returns TENO_ERR_WORKSPACE).
 * teno_timer_end waits for those events and writes, per kernel kind, the
 * summed device time in ms[TENO_KERNEL_KINDS] and the launch count in
 * launches[TENO_KERNEL_KINDS] (host arrays).  Not thread-safe; do not use
 * while capturing a CUDA graph.
 */
teno_status teno_timer_begin(void);
teno_status teno_timer_end(double* ms, int64_t* launches);

/*
 * teno_probe_fp64 -- measurement aid (no counterpart in the paper): launches
 * `blocks` blocks of 256 threads, each running 8 independent FP64 fused
 * multiply-add chains of `iters` steps (2 * 8 * iters flops per thread), and
 * writes one double per thread to out_dev (device, blocks * 256 doubles).
 * Timing it with events gives the FP64 pipe's throughput on this GPU.
 */
teno_status teno_probe_fp64(double* out_dev, int64_t blocks, int64_t iters,
                            void* stream);

/*
 * teno_probe_recip -- test aid (no counterpart in the paper): for the n
 * doubles x_dev (device) writes, to out_dev (device, 2 n doubles), the
 * library's seeded reciprocal (the one the Roe average uses), then CUDA's
 * 1.0 / x, n entries each.  TENO_ERR_INVALID_ARG for null pointers or n
 * outside 1..2^32.
 */
teno_status teno_probe_recip(const double* x_dev, double* out_dev, int64_t n,
                             void* stream);

/* Human-readable name of a status code (static storage). */
const char* teno_status_string(teno_status s);

/* TENO_ABI_VERSION of the loaded library. */
int teno_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TENO_H */
