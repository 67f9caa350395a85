// teno_launch.h -- host-side launchers of the kernels in teno_kernels.cu
// (internal to the library; the public interface is include/teno.h).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "teno.h"
#include "teno_device.cuh"

namespace teno {

// Scheme constants for the given gas, LAD parameters (eq. 3.1-3.2, 2.8) and
// cutoff variant (teno_scheme; ct_m: TENO5's fixed magnitude).
Scheme make_scheme(double gamma, double H, double eps, int b_l, int b_u, int variant = TENO_SCHEME_LAD,
                   int ct_m = 7);

// The grid's scheme fields are valid: a known teno_scheme, and for
// TENO_SCHEME_TENO5 a magnitude 1..15.
inline bool scheme_fields_ok(const teno_grid* g) {
  if (g->scheme < TENO_SCHEME_LAD || g->scheme > TENO_SCHEME_WENOZ) return false;
  if (g->scheme == TENO_SCHEME_TENO5 && (g->ct_m < 1 || g->ct_m > 15)) return false;
  return true;
}

inline Scheme scheme_of(const teno_grid* g) {
  return make_scheme(g->gamma, g->H, g->eps, g->b_l, g->b_u, g->scheme, g->ct_m);
}

// Primitives (aux) and LF speeds of every cell; with `fh` (nullable) also
// the half physical fluxes F_d/2 without their mass component,
// [ndim][nvar - 1][ncell]; with `cand` (nullable, 18 words per block of
// cell_blocks) the per-block arg-max candidates of the speeds.
int cell_blocks(int64_t ncell, int nsm);
cudaError_t launch_cell(int ndim, const double* U, double* aux, double* fh,
                        unsigned long long* alpha, int* status, int64_t ncell,
                        double gamma, int nsm, cudaStream_t st, unsigned long long* cand = nullptr);
// argidx[3 d + s] = the lowest cell index at which speed s of direction d
// attains its maximum, from the candidates of a launch_cell with `cand`.
cudaError_t launch_argmax_finish(int ndim, const unsigned long long* cand, int64_t ncell, int nsm,
                                 unsigned long long* argidx, cudaStream_t st);

// The interface fluxes of direction `dir` into Fhat.  With `flags`, or
// without a pending list or the cell pass's half fluxes `fh`, one pass; with
// `list` (room for one 32-bit entry per interface), its counter `count`
// (zero on entry) and `fh`, the closed-form pass and the pass over the
// interfaces it leaves pending.  `launches` (optional) receives the number
// of kernels launched.  With `roe_out` (two-pass fluxes without reflecting or
// fixed-state faces only) the closed-form pass also writes every
// interface's Roe state and its certificate's decision, [ndim + 8][#interfaces]
// (flux_closed_kernel).
cudaError_t launch_flux(int ndim, int dir, const double* U, const double* aux, const double* fh,
                        const unsigned long long* alpha, double* Fhat,
                        uint8_t* flags, uint32_t* list, unsigned* count, int* status,
                        const Grid& G, const Scheme& S, int nsm, cudaStream_t st,
                        int* launches, double* roe_out = nullptr);

// The workspace header holds the nine LF speeds (as bit patterns) and, right
// after them, one pending-list counter per direction; one memset of
// kAlphaAndCountBytes from the speeds clears both.
constexpr size_t kPendingCountOffset = 9 * sizeof(unsigned long long);
constexpr size_t kAlphaAndCountBytes = kPendingCountOffset + 3 * sizeof(unsigned);

// The difference of direction `dir` (called for dir = 0..ndim-1 in order,
// each after that direction's fluxes are in Fhat; Usrc = the state whose
// right-hand side this is, for the body-force source when G.has_grav).  R carries the unscaled
// partial sum between the calls (see diff_kernel).  mode 0: the last
// direction writes L(U) into R; 2, 3, 4: the last direction writes the
// SSP-RK3 stage (eq. 4.1-4.3) into Uout, with dt read from the device word
// `dt` (dt <= 0: the state is left unchanged, stage buffers take Un).
cudaError_t launch_diff(int ndim, int dir, const double* Fhat, double* R,
                        const double* Un, const double* Uk, double* Uout,
                        const double* dt, const Grid& G, int mode,
                        int nsm, cudaStream_t st, const double* Usrc);

// The fixed-state (TENO_BC_DIRICHLET) ghost cells: the conservative states of
// the six faces (slot 2 d + side, unused slots ignored per `mask` bit) into
// the ghost block G.gU and their primitives and half fluxes into G.gaux,
// G.gfh (the cell pass's formulas, kGhostSlots entries per field).
struct GhostStates {
  double U[6][5];
};
cudaError_t launch_ghost_cells(int ndim, const GhostStates& gs, unsigned mask, const Grid& G, double gamma,
                               cudaStream_t st);
// doubles of the ghost block for an ndim grid
inline int ghost_block_doubles(int ndim) { return 6 * ((ndim + 2) + aux_fields(ndim) + ndim * (ndim + 1)); }

cudaError_t launch_dt(int ndim, const unsigned long long* alpha, const Grid& G,
                      double cfl, double dt_fixed, double* t_dev, double t_end,
                      double* dt_ws, double* dt_out, cudaStream_t st);

// One right-hand-side evaluation of U fused with the SSP-RK3 stage `mode`
// (2, 3 or 4; see diff_kernel) into Uout, with dt read from the workspace
// word at dt_off.  `ws` offsets locate the status word, the LF speeds (and
// the pending counters after them), the per-cell primitives, the half
// fluxes, the interface-flux buffer and the pending list (fh_off or list_off
// 0: one-pass fluxes); R holds the partial sums of the multi-dimensional
// difference; `cand` (nullable) as for launch_cell; with `roe_out`, direction
// d's Roe states go to roe_out + d roe_stride (see launch_flux).
teno_status forward_stage(const teno_grid* g, char* ws, size_t status_off, size_t dt_off,
                          size_t alpha_off, size_t aux_off, size_t fh_off, size_t fhat_off, size_t list_off,
                          const double* U, double* R, int mode, const double* Un, const double* Uk,
                          double* Uout, cudaStream_t st, unsigned long long* cand = nullptr,
                          double* roe_out = nullptr, size_t roe_stride = 0);

}  // namespace teno
