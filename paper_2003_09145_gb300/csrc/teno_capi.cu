// teno_capi.cu -- the C-ABI of include/teno.h: argument validation, workspace
// layout and the launch sequences of teno_rhs and teno_rk3_step.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>

#include "teno.h"
#include "teno_device.cuh"
#include "teno_launch.h"

namespace {

using teno::Grid;
using teno::Scheme;

constexpr size_t kAlign = 256;
constexpr size_t kHeader = 256;  // status word, dt, alpha bit patterns

size_t round_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// the fixed ghost states of axis k are physical: rho > 0, p > 0, finite
bool fixed_states_ok(const teno_grid* g, int k) {
  const int nvar = g->ndim + 2;
  for (int side = 0; side < 2; ++side) {
    const double* U = g->bc_state[k][side];
    double q = 0.0;
    for (int v = 0; v < nvar; ++v)
      if (!std::isfinite(U[v])) return false;
    if (!(U[0] > 0.0)) return false;
    for (int j = 0; j < g->ndim; ++j) q += U[1 + j] * U[1 + j];
    const double p = (g->gamma - 1.0) * (U[nvar - 1] - 0.5 * q / U[0]);
    if (!(p > 0.0) || !std::isfinite(p)) return false;
  }
  return true;
}

bool grid_ok(const teno_grid* g) {
  if (!g) return false;
  if (g->ndim < 1 || g->ndim > 3) return false;
  for (int k = 0; k < 3; ++k) {
    if (g->n[k] < 1) return false;
    if (k >= g->ndim && g->n[k] != 1) return false;
    if (k < g->ndim) {
      if (!(g->dx[k] > 0.0) || !std::isfinite(g->dx[k])) return false;
      if (g->bc[k] != TENO_BC_PERIODIC && g->bc[k] != TENO_BC_TRANSMISSIVE && g->bc[k] != TENO_BC_REFLECTIVE &&
          g->bc[k] != TENO_BC_DIRICHLET)
        return false;
      if (!std::isfinite(g->grav[k])) return false;
      if (g->bc[k] == TENO_BC_DIRICHLET && !fixed_states_ok(g, k)) return false;
    }
  }
  if (!(g->gamma > 1.0) || !std::isfinite(g->gamma)) return false;
  if (!(g->H > 0.0) || !std::isfinite(g->H)) return false;
  if (!(g->eps > 0.0) || !std::isfinite(g->eps)) return false;
  if (g->b_l < 0 || g->b_u > 15 || g->b_u <= g->b_l) return false;
  if (!teno::scheme_fields_ok(g)) return false;
  // total cell count must stay addressable with 64-bit indices
  const double cells = double(g->n[0]) * double(g->n[1]) * double(g->n[2]);
  if (cells * teno::aux_fields(g->ndim) > 9.0e18 / 8.0) return false;
  // the pending lists hold 32-bit interface indices
  for (int d = 0; d < g->ndim; ++d) {
    double m = 1.0;
    for (int k = 0; k < 3; ++k) m *= double(g->n[k] + (k == d ? 1 : 0));
    if (m >= 4294967296.0) return false;
  }
  return true;
}

int64_t ncell_of(const teno_grid* g) { return g->n[0] * g->n[1] * g->n[2]; }

int64_t nifc_of(const teno_grid* g, int d) {
  int64_t m = 1;
  for (int k = 0; k < 3; ++k) m *= g->n[k] + (k == d ? 1 : 0);
  return m;
}

struct Layout {
  // header: [0] status, [8] dt, [64] LF speeds (9 x 8) then the pending-list
  // counters (3 x 4)
  size_t status = 0, dt = 8, alpha = 64;
  size_t aux = 0, fh = 0, fhat = 0, list = 0, ghost = 0, R = 0, U1 = 0, U2 = 0, total = 0;
};

Layout layout_of(const teno_grid* g, int op) {
  Layout L;
  const int nvar = g->ndim + 2;
  const size_t ncell = size_t(ncell_of(g));
  int64_t maxifc = 0;
  for (int d = 0; d < g->ndim; ++d) maxifc = nifc_of(g, d) > maxifc ? nifc_of(g, d) : maxifc;
  size_t off = kHeader;
  L.aux = off;
  off += round_up(sizeof(double) * teno::aux_fields(g->ndim) * ncell);
  L.fh = off;   // half physical fluxes F_d/2 per cell and direction (no mass component)
  off += round_up(sizeof(double) * g->ndim * (nvar - 1) * ncell);
  L.fhat = off;
  off += round_up(sizeof(double) * nvar * size_t(maxifc));
  L.list = off;
  off += round_up(sizeof(uint32_t) * size_t(maxifc));
  L.ghost = off;   // fixed-state ghost cells (state, primitives, half fluxes of 6 face slots)
  off += round_up(sizeof(double) * size_t(teno::ghost_block_doubles(g->ndim)));
  if (op == TENO_OP_RK3) {
    L.R = off;
    off += round_up(sizeof(double) * nvar * ncell);
    L.U1 = off;
    off += round_up(sizeof(double) * nvar * ncell);
    L.U2 = off;
    off += round_up(sizeof(double) * nvar * ncell);
  }
  L.total = off;
  return L;
}

Grid make_grid(const teno_grid* g) {
  Grid G;
  for (int k = 0; k < 3; ++k) {
    G.n[k] = g->n[k];
    G.bc[k] = k < g->ndim ? g->bc[k] : 0;
    G.dx[k] = k < g->ndim ? g->dx[k] : 1.0;
    G.inv_dx[k] = 1.0 / G.dx[k];
    G.rdx[k] = G.dx[0] / G.dx[k];
  }
  G.ncell = ncell_of(g);
  for (int k = 0; k < 3; ++k) {
    G.grav[k] = k < g->ndim ? g->grav[k] : 0.0;
    if (G.grav[k] != 0.0) G.has_grav = 1;
  }
  return G;
}

Scheme make_scheme(const teno_grid* g) { return teno::scheme_of(g); }

// make_grid with the fixed-state ghost block of workspace ws attached
Grid grid_in(const teno_grid* g, const Layout& L, char* ws) {
  Grid G = make_grid(g);
  double* gb = reinterpret_cast<double*>(ws + L.ghost);
  const int nvar = g->ndim + 2;
  G.gU = gb;
  G.gaux = gb + nvar * teno::kGhostSlots;
  G.gfh = gb + (nvar + teno::aux_fields(g->ndim)) * teno::kGhostSlots;
  return G;
}

bool has_dirichlet(const teno_grid* g) {
  for (int k = 0; k < g->ndim; ++k)
    if (g->bc[k] == TENO_BC_DIRICHLET) return true;
  return false;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// True if p is a device (or managed) allocation the current device can use.
bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int sm_count() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 152;
  static int cache[64] = {0};
  if (dev >= 0 && dev < 64 && cache[dev] > 0) return cache[dev];
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
  if (dev >= 0 && dev < 64) cache[dev] = n;
  return n;
}

// ---------------------------------------------------------------------------
// Optional per-kernel timing: when enabled, every launch of the library is
// bracketed by a pair of CUDA events on its stream; teno_timer_end() sums the
// elapsed times per kernel kind.  Off by default (no events are recorded).
// ---------------------------------------------------------------------------
constexpr int kTimerPairs = 8192;
struct KernelTimer {
  bool on = false;
  bool created = false;
  int used = 0;
  int64_t dropped = 0;
  cudaEvent_t ev[2 * kTimerPairs];
  int kind[kTimerPairs];
  int nlaunch[kTimerPairs];   // kernels launched inside the pair
};
KernelTimer g_timer;

struct TimerScope {
  cudaStream_t st;
  int slot = -1;
  TimerScope(cudaStream_t s, int kind) : st(s) {
    if (!g_timer.on) return;
    if (g_timer.used >= kTimerPairs) { ++g_timer.dropped; return; }
    slot = g_timer.used++;
    g_timer.kind[slot] = kind;
    g_timer.nlaunch[slot] = 1;
    cudaEventRecord(g_timer.ev[2 * slot], st);
  }
  void launches(int n) {
    if (slot >= 0) g_timer.nlaunch[slot] = n;
  }
  ~TimerScope() {
    if (slot >= 0) cudaEventRecord(g_timer.ev[2 * slot + 1], st);
  }
};

#define TENO_CUDA(call)                                  \
  do {                                                   \
    if ((call) != cudaSuccess) return TENO_ERR_CUDA;     \
  } while (0)

// The first half of a right-hand-side evaluation of state `U`: clear the LF
// speeds and pending counters, then the cell pass (primitives, half fluxes
// for the two-pass flux evaluation, this grid's LF speeds).
teno_status stage_begin(const teno_grid* g, const Layout& L, char* ws, const double* U, bool one_pass,
                        cudaStream_t st) {
  const Grid G = grid_in(g, L, ws);
  const int nsm = sm_count();
  int* status = reinterpret_cast<int*>(ws + L.status);
  auto* alpha = reinterpret_cast<unsigned long long*>(ws + L.alpha);
  double* aux = reinterpret_cast<double*>(ws + L.aux);
  double* fh = one_pass ? nullptr : reinterpret_cast<double*>(ws + L.fh);
  TENO_CUDA(cudaMemsetAsync(alpha, 0, teno::kAlphaAndCountBytes, st));
  TimerScope ts(st, TENO_KERNEL_CELL);
  if (has_dirichlet(g)) {
    teno::GhostStates gs;
    std::memset(&gs, 0, sizeof(gs));
    unsigned mask = 0;
    for (int d = 0; d < g->ndim; ++d) {
      if (g->bc[d] != TENO_BC_DIRICHLET) continue;
      for (int side = 0; side < 2; ++side) {
        for (int v = 0; v < g->ndim + 2; ++v) gs.U[2 * d + side][v] = g->bc_state[d][side][v];
        mask |= 1u << (2 * d + side);
      }
    }
    TENO_CUDA(teno::launch_ghost_cells(g->ndim, gs, mask, G, g->gamma, st));
  }
  TENO_CUDA(teno::launch_cell(g->ndim, U, aux, fh, alpha, status, G.ncell, g->gamma, nsm, st));
  return TENO_OK;
}

// The second half, with the LF speeds in the workspace: the CFL step (with_dt),
// then per direction the interface fluxes and the difference; mode_last
// selects what the last direction's difference does (0: dUdt into R; 2/3/4:
// the SSP-RK3 stage into Uout).
teno_status stage_finish(const teno_grid* g, const Layout& L, char* ws, const double* U, double* R,
                         uint8_t* flags, int mode_last, const double* Un, const double* Uk, double* Uout,
                         cudaStream_t st, bool with_dt, double cfl, double dt_fixed, double* t_dev, double t_end,
                         double* dt_out) {
  const Grid G = grid_in(g, L, ws);
  const Scheme S = make_scheme(g);
  const int nsm = sm_count();
  int* status = reinterpret_cast<int*>(ws + L.status);
  double* dt_ws = reinterpret_cast<double*>(ws + L.dt);
  auto* alpha = reinterpret_cast<unsigned long long*>(ws + L.alpha);
  double* aux = reinterpret_cast<double*>(ws + L.aux);
  double* Fhat = reinterpret_cast<double*>(ws + L.fhat);
  uint32_t* list = reinterpret_cast<uint32_t*>(ws + L.list);
  double* fh = flags ? nullptr : reinterpret_cast<double*>(ws + L.fh);   // the flag path is one-pass
  unsigned* count = reinterpret_cast<unsigned*>(ws + L.alpha + teno::kPendingCountOffset);
  if (with_dt) {
    TimerScope ts(st, TENO_KERNEL_DT);
    TENO_CUDA(teno::launch_dt(g->ndim, alpha, G, cfl, dt_fixed, t_dev, t_end, dt_ws, dt_out, st));
  }
  int64_t foff = 0;
  for (int d = 0; d < g->ndim; ++d) {
    uint8_t* fl = flags ? flags + foff : nullptr;
    {
      TimerScope ts(st, TENO_KERNEL_FLUX);
      int nl = 1;
      TENO_CUDA(teno::launch_flux(g->ndim, d, U, aux, fh, alpha, Fhat, fl, list, count + d, status, G, S, nsm, st,
                                  &nl));
      ts.launches(nl);
    }
    foff += int64_t(g->ndim + 2) * 2 * nifc_of(g, d);
    {
      TimerScope ts(st, TENO_KERNEL_DIFF);
      TENO_CUDA(teno::launch_diff(g->ndim, d, Fhat, R, Un, Uk, Uout, dt_ws, G, mode_last, nsm, st, U));
    }
  }
  return TENO_OK;
}

// One right-hand-side evaluation of state `U` (both halves).
teno_status rhs_sequence(const teno_grid* g, const Layout& L, char* ws,
                         const double* U, double* R, uint8_t* flags,
                         int mode_last, const double* Un, const double* Uk,
                         double* Uout, cudaStream_t st, bool with_dt,
                         double cfl, double dt_fixed, double* t_dev,
                         double t_end, double* dt_out) {
  const teno_status s = stage_begin(g, L, ws, U, flags != nullptr, st);
  if (s != TENO_OK) return s;
  return stage_finish(g, L, ws, U, R, flags, mode_last, Un, Uk, Uout, st, with_dt, cfl, dt_fixed, t_dev, t_end,
                      dt_out);
}

}  // namespace

extern "C" {

void teno_grid_default(teno_grid* g, int ndim, const int64_t* n, const double* dx, int bc) {
  if (!g) return;
  std::memset(g, 0, sizeof(*g));
  g->ndim = ndim;
  for (int k = 0; k < 3; ++k) {
    g->n[k] = (k < ndim && n) ? n[k] : 1;
    g->dx[k] = (k < ndim && dx) ? dx[k] : 1.0;
    g->bc[k] = bc;
  }
  g->gamma = 1.4;
  g->H = 10.0;
  g->b_l = 4;
  g->b_u = 10;
  g->eps = 1e-6;
  g->scheme = TENO_SCHEME_LAD;
  g->ct_m = 7;
}

size_t teno_workspace_bytes(const teno_grid* g, int op) {
  if (!grid_ok(g)) return 0;
  if (op != TENO_OP_RHS && op != TENO_OP_RK3) return 0;
  return layout_of(g, op).total;
}

int64_t teno_flag_count(const teno_grid* g) {
  if (!grid_ok(g)) return 0;
  int64_t c = 0;
  for (int d = 0; d < g->ndim; ++d) c += int64_t(g->ndim + 2) * 2 * nifc_of(g, d);
  return c;
}

teno_status teno_rhs(const teno_grid* g, const double* U, double* dUdt, uint8_t* flags,
                     void* ws, size_t ws_bytes, void* stream) {
  if (!grid_ok(g) || !U || !dUdt || U == dUdt) return TENO_ERR_INVALID_ARG;
  if (!aligned(U, 16) || !aligned(dUdt, 16)) return TENO_ERR_INVALID_ARG;
  if (!is_device_ptr(U) || !is_device_ptr(dUdt) || (flags && !is_device_ptr(flags)))
    return TENO_ERR_INVALID_ARG;
  const Layout L = layout_of(g, TENO_OP_RHS);
  if (!ws || !aligned(ws, kAlign) || ws_bytes < L.total || !is_device_ptr(ws)) return TENO_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return rhs_sequence(g, L, static_cast<char*>(ws), U, dUdt, flags, 0, nullptr, nullptr, nullptr,
                      st, false, 0.0, 0.0, nullptr, 0.0, nullptr);
}

teno_status teno_rk3_step(const teno_grid* g, double* U, double cfl, double dt_fixed,
                          double* t_dev, double t_end, double* dt_dev, void* ws,
                          size_t ws_bytes, void* stream) {
  if (!grid_ok(g) || !U || !t_dev) return TENO_ERR_INVALID_ARG;
  if (!aligned(U, 16) || !aligned(t_dev, 8) || (dt_dev && !aligned(dt_dev, 8))) return TENO_ERR_INVALID_ARG;
  if (!(dt_fixed > 0.0) && !(cfl > 0.0 && std::isfinite(cfl))) return TENO_ERR_INVALID_ARG;
  if (!std::isfinite(dt_fixed) || std::isnan(t_end)) return TENO_ERR_INVALID_ARG;
  if (!is_device_ptr(U) || !is_device_ptr(t_dev) || (dt_dev && !is_device_ptr(dt_dev)))
    return TENO_ERR_INVALID_ARG;
  const Layout L = layout_of(g, TENO_OP_RK3);
  if (!ws || !aligned(ws, kAlign) || ws_bytes < L.total || !is_device_ptr(ws)) return TENO_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(ws);
  double* R = reinterpret_cast<double*>(w + L.R);
  double* U1 = reinterpret_cast<double*>(w + L.U1);
  double* U2 = reinterpret_cast<double*>(w + L.U2);
  teno_status s;
  // eq. 4.1: U1 = U + dt L(U); dt from U^n (eq. dt1 / dt2)
  s = rhs_sequence(g, L, w, U, R, nullptr, 2, U, nullptr, U1, st, true, cfl, dt_fixed, t_dev,
                   t_end, dt_dev);
  if (s != TENO_OK) return s;
  // eq. 4.2: U2 = 3/4 U + 1/4 U1 + 1/4 dt L(U1)
  s = rhs_sequence(g, L, w, U1, R, nullptr, 3, U, U1, U2, st, false, 0, 0, nullptr, 0, nullptr);
  if (s != TENO_OK) return s;
  // eq. 4.3: U <- 1/3 U + 2/3 U2 + 2/3 dt L(U2)
  return rhs_sequence(g, L, w, U2, R, nullptr, 4, U, U2, U, st, false, 0, 0, nullptr, 0, nullptr);
}

teno_status teno_rk3_stage_begin(const teno_grid* g, const double* Uin, void* ws, size_t ws_bytes, void* stream) {
  if (!grid_ok(g) || !Uin || !aligned(Uin, 16) || !is_device_ptr(Uin)) return TENO_ERR_INVALID_ARG;
  const Layout L = layout_of(g, TENO_OP_RK3);
  if (!ws || !aligned(ws, kAlign) || ws_bytes < L.total || !is_device_ptr(ws)) return TENO_ERR_WORKSPACE;
  return stage_begin(g, L, static_cast<char*>(ws), Uin, false, static_cast<cudaStream_t>(stream));
}

teno_status teno_rk3_stage_end(const teno_grid* g, int stage, const double* Uin, double* Un, double* Uout,
                               double cfl, double dt_fixed, double* t_dev, double t_end, double* dt_dev, void* ws,
                               size_t ws_bytes, void* stream) {
  if (!grid_ok(g) || stage < 1 || stage > 3 || !Uin || !Un || !Uout) return TENO_ERR_INVALID_ARG;
  if (!aligned(Uin, 16) || !aligned(Un, 16) || !aligned(Uout, 16)) return TENO_ERR_INVALID_ARG;
  if (!is_device_ptr(Uin) || !is_device_ptr(Un) || !is_device_ptr(Uout)) return TENO_ERR_INVALID_ARG;
  // stage 1 reads U^n itself and writes U1 elsewhere; stage 2 writes U2
  // apart from its inputs; stage 3 may write over U^n
  if ((stage == 1 && (Uin != Un || Uout == Un)) || (stage == 2 && (Uout == Un || Uout == Uin)) ||
      (stage == 3 && Uout == Uin))
    return TENO_ERR_INVALID_ARG;
  if (stage == 1) {
    if (!t_dev || !aligned(t_dev, 8) || !is_device_ptr(t_dev) || (dt_dev && !is_device_ptr(dt_dev)))
      return TENO_ERR_INVALID_ARG;
    if (!(dt_fixed > 0.0) && !(cfl > 0.0 && std::isfinite(cfl))) return TENO_ERR_INVALID_ARG;
    if (!std::isfinite(dt_fixed) || std::isnan(t_end)) return TENO_ERR_INVALID_ARG;
  }
  const Layout L = layout_of(g, TENO_OP_RK3);
  if (!ws || !aligned(ws, kAlign) || ws_bytes < L.total || !is_device_ptr(ws)) return TENO_ERR_WORKSPACE;
  char* w = static_cast<char*>(ws);
  double* R = reinterpret_cast<double*>(w + L.R);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // eq. 4.1 / 4.2 / 4.3 (diff modes 2 / 3 / 4); dt from the LF speeds now in ws
  return stage_finish(g, L, w, Uin, R, nullptr, stage + 1, Un, stage == 1 ? nullptr : Uin, Uout, st, stage == 1,
                      cfl, dt_fixed, t_dev, t_end, dt_dev);
}

size_t teno_alpha_offset(void) { return Layout().alpha; }

teno_status teno_planes_copy(const teno_grid* g, const double* src, int64_t src_plane, int src_packed,
                             double* dst, int64_t dst_plane, int dst_packed, int64_t nplanes, void* stream) {
  if (!grid_ok(g) || !src || !dst || nplanes < 1) return TENO_ERR_INVALID_ARG;
  const int ax = g->ndim - 1;
  const int64_t nax = g->n[ax];
  const int64_t plane = ncell_of(g) / nax;
  const int64_t ncell = ncell_of(g);
  if (!src_packed && (src_plane < 0 || src_plane + nplanes > nax)) return TENO_ERR_INVALID_ARG;
  if (!dst_packed && (dst_plane < 0 || dst_plane + nplanes > nax)) return TENO_ERR_INVALID_ARG;
  if (!aligned(src, 8) || !aligned(dst, 8) || !is_device_ptr(src) || !is_device_ptr(dst)) return TENO_ERR_INVALID_ARG;
  const size_t width = sizeof(double) * size_t(nplanes * plane);
  const size_t spitch = src_packed ? width : sizeof(double) * size_t(ncell);
  const size_t dpitch = dst_packed ? width : sizeof(double) * size_t(ncell);
  const double* s0 = src + (src_packed ? 0 : src_plane * plane);
  double* d0 = dst + (dst_packed ? 0 : dst_plane * plane);
  TENO_CUDA(cudaMemcpy2DAsync(d0, dpitch, s0, spitch, width, size_t(g->ndim + 2), cudaMemcpyDeviceToDevice,
                              static_cast<cudaStream_t>(stream)));
  return TENO_OK;
}

teno_status teno_get_device_status(void* ws, void* stream, int* status) {
  if (!ws || !status || !aligned(ws, kAlign)) return TENO_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int h = 0;
  TENO_CUDA(cudaMemcpyAsync(&h, ws, sizeof(int), cudaMemcpyDeviceToHost, st));
  TENO_CUDA(cudaStreamSynchronize(st));
  TENO_CUDA(cudaMemsetAsync(ws, 0, sizeof(int), st));
  TENO_CUDA(cudaStreamSynchronize(st));
  if (h & teno::kStatusTimeout) *status = TENO_ERR_TIMEOUT;
  else if (h & teno::kStatusNonphysical) *status = TENO_ERR_NONPHYSICAL;
  else *status = TENO_OK;
  return TENO_OK;
}

teno_status teno_timer_begin(void) {
  if (!g_timer.created) {
    for (int i = 0; i < 2 * kTimerPairs; ++i)
      if (cudaEventCreate(&g_timer.ev[i]) != cudaSuccess) return TENO_ERR_CUDA;
    g_timer.created = true;
  }
  g_timer.used = 0;
  g_timer.dropped = 0;
  g_timer.on = true;
  return TENO_OK;
}

teno_status teno_timer_end(double* ms, int64_t* launches) {
  if (!ms || !launches) return TENO_ERR_INVALID_ARG;
  g_timer.on = false;
  for (int k = 0; k < TENO_KERNEL_KINDS; ++k) {
    ms[k] = 0.0;
    launches[k] = 0;
  }
  for (int i = 0; i < g_timer.used; ++i) {
    if (cudaEventSynchronize(g_timer.ev[2 * i + 1]) != cudaSuccess) return TENO_ERR_CUDA;
    float t = 0.0f;
    if (cudaEventElapsedTime(&t, g_timer.ev[2 * i], g_timer.ev[2 * i + 1]) != cudaSuccess)
      return TENO_ERR_CUDA;
    ms[g_timer.kind[i]] += t;
    launches[g_timer.kind[i]] += g_timer.nlaunch[i];
  }
  return g_timer.dropped ? TENO_ERR_WORKSPACE : TENO_OK;
}

const char* teno_status_string(teno_status s) {
  switch (s) {
    case TENO_OK: return "TENO_OK";
    case TENO_ERR_INVALID_ARG: return "TENO_ERR_INVALID_ARG";
    case TENO_ERR_UNSUPPORTED: return "TENO_ERR_UNSUPPORTED";
    case TENO_ERR_CUDA: return "TENO_ERR_CUDA";
    case TENO_ERR_NONPHYSICAL: return "TENO_ERR_NONPHYSICAL";
    case TENO_ERR_TIMEOUT: return "TENO_ERR_TIMEOUT";
    case TENO_ERR_WORKSPACE: return "TENO_ERR_WORKSPACE";
    case TENO_ERR_UNIMPLEMENTED: return "TENO_ERR_UNIMPLEMENTED";
  }
  return "TENO_UNKNOWN_STATUS";
}

int teno_abi_version(void) { return TENO_ABI_VERSION; }

}  // extern "C"
