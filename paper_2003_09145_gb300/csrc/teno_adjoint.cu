// teno_adjoint.cu -- adjoint (vector-Jacobian product) of the TENO5-LAD Euler
// right-hand side and of one SSP-RK3 step.
//
// The stencil selections are frozen at their primal values: the cutoff of
// eq. 2.14 is piecewise constant, so with delta fixed the reconstruction is
// linear and L(U) is differentiable almost everywhere.  The global
// Lax-Friedrichs speed alpha_{d,s} = max_cells |lambda_s| is differentiated
// through its arg-max cell (lowest linear index on ties).
//
// teno_rhs_adjoint, per direction d:
//   adj_flux_kernel  : one thread per interface: the selections by the same
//                      device code as the forward pass, then the interface VJP
//                      (teno_adjoint_core.cuh; the closed form when every
//                      stencil is kept) with Fbar from Rbar (eq. 2.2);
//                      the six cells' contributions are written to a buffer
//                      and d/dalpha is summed per block (fixed order);
//   adj_gather_kernel: one thread per cell sums the contributions of every
//                      (interface, stencil slot) that maps to it (boundary
//                      ghost copies included) -- deterministic, no atomics;
//   adj_alpha_kernel : sums the block partials in a fixed order and adds the
//                      alpha terms at the arg-max cells.
#include <cmath>
#include <cstdint>
#include <cstring>

#include <cuda_runtime.h>

#include "teno.h"
#include "teno_adjoint_core.cuh"
#include "teno_device.cuh"
#include "teno_flux.cuh"
#include "teno_launch.h"

namespace {

using teno::Grid;
using teno::Scheme;

constexpr int kAdjThreads = 128;

// Lowest linear cell index at which |lambda_kind| (direction d) equals the
// reduced maximum alpha (same rounding as the forward cell pass).
template <int NDIM>
__global__ void argmax_kernel(const double* __restrict__ U, const unsigned long long* __restrict__ alpha,
                              unsigned long long* __restrict__ argidx, int64_t ncell, double gamma,
                              double* __restrict__ scratch_aux) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell;
       c += (int64_t)gridDim.x * blockDim.x) {
    double u[NDIM], cs;
    teno::cell_primitives<NDIM>(U, ncell, c, gamma, scratch_aux, u, cs);
#pragma unroll
    for (int d = 0; d < NDIM; ++d) {
      const double lam[3] = {fabs(__dsub_rn(u[d], cs)), fabs(u[d]), fabs(__dadd_rn(u[d], cs))};
#pragma unroll
      for (int k = 0; k < 3; ++k)
        if (teno::dbits(lam[k]) == alpha[d * 3 + k]) atomicMin(&argidx[d * 3 + k], (unsigned long long)c);
    }
  }
}

template <int NDIM, int DIR>
__global__ void __launch_bounds__(kAdjThreads) adj_flux_kernel(
    const double* __restrict__ U, const double* __restrict__ aux,
    const unsigned long long* __restrict__ alpha_bits, const double* __restrict__ Rbar, double scale,
    double* __restrict__ contrib, double* __restrict__ apart, int* __restrict__ status, Grid G, Scheme S) {
  constexpr int NVAR = NDIM + 2;
  const int64_t m0 = G.n[0] + (DIR == 0), m1 = G.n[1] + (DIR == 1), m2 = G.n[2] + (DIR == 2);
  const int64_t nifc = m0 * m1 * m2;
  const int64_t ncell = G.ncell;
  const int64_t stride_d = (DIR == 0) ? 1 : (DIR == 1 ? G.n[0] : G.n[0] * G.n[1]);
  const int64_t nd = G.n[DIR];
  const int bcd = G.bc[DIR];
  double ha[NVAR], fa[NVAR];
  {
    const double am = __longlong_as_double((long long)alpha_bits[DIR * 3 + 0]);
    const double a0 = __longlong_as_double((long long)alpha_bits[DIR * 3 + 1]);
    const double ap = __longlong_as_double((long long)alpha_bits[DIR * 3 + 2]);
    fa[0] = am;
    for (int f = 1; f < NVAR - 1; ++f) fa[f] = a0;
    fa[NVAR - 1] = ap;
    for (int f = 0; f < NVAR; ++f) ha[f] = 0.5 * fa[f];
  }
  double nfa[NVAR];
  for (int f = 0; f < NVAR; ++f) nfa[f] = -2.0 * ha[f];
  const double fscale = scale * G.inv_dx[DIR];
  double asum[3] = {0.0, 0.0, 0.0};
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nifc;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i0 = q % m0;
    const int64_t r = q / m0;
    const int64_t i1 = r % m1;
    const int64_t i2 = r / m1;
    const int64_t id = (DIR == 0) ? i0 : (DIR == 1 ? i1 : i2);
    const int64_t base = (DIR == 0) ? (i2 * G.n[1] + i1) * G.n[0]
                       : (DIR == 1) ? i2 * G.n[1] * G.n[0] + i0
                                    : i1 * G.n[0] + i0;
    int64_t cells[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) cells[j] = base + teno::ghost(id - 3 + j, nd, bcd) * stride_d;
    // the primal selections: the forward pass's own device code (the same
    // certified tests and binary64 decisions teno_rhs / teno_rk3_step take)
    double fout[NVAR];
    unsigned fl[NVAR][2];
    teno::interface_flux<NDIM, DIR, false>(U, aux, ncell, cells, ha, nfa, S, fout, fl, status);
    unsigned sel[NVAR][2];
    bool all_kept = true;
    for (int s = 0; s < NVAR; ++s) {
      sel[s][0] = fl[s][0] & 7u;
      sel[s][1] = fl[s][1] & 7u;
      all_kept = all_kept && sel[s][0] == 7u && sel[s][1] == 7u;
    }
    double Up[6][NVAR];
    for (int j = 0; j < 6; ++j)
      for (int v = 0; v < NVAR; ++v) Up[j][v] = U[v * ncell + cells[j]];
    // Fbar of interface id: R_c = -(F^_{c+1/2} - F^_{c-1/2})/dx gives
    // dJ/dF^_id = (Rbar_id [id < n] - Rbar_{id-1} [id >= 1]) / dx
    double Fb[NVAR];
    for (int v = 0; v < NVAR; ++v) {
      double a = 0.0;
      if (id < nd) a += Rbar[v * ncell + base + id * stride_d];
      if (id >= 1) a -= Rbar[v * ncell + base + (id - 1) * stride_d];
      Fb[v] = a * fscale;
    }
    double Ub[6][NVAR], ab[NVAR];
    if (all_kept)
      teno_adj::interface_vjp_kept<NDIM, DIR>(Up, fa, S.gamma, Fb, Ub, ab);
    else
      teno_adj::interface_vjp<NDIM, DIR>(Up, fa, sel, S.gamma, Fb, Ub, ab);
    for (int j = 0; j < 6; ++j)
      for (int v = 0; v < NVAR; ++v) contrib[(int64_t)(j * NVAR + v) * nifc + q] = Ub[j][v];
    asum[0] += ab[0];
    for (int f = 1; f < NVAR - 1; ++f) asum[1] += ab[f];
    asum[2] += ab[NVAR - 1];
  }
  // block sum in a fixed order
  __shared__ double red[kAdjThreads][3];
  for (int k = 0; k < 3; ++k) red[threadIdx.x][k] = asum[k];
  __syncthreads();
  for (int w = kAdjThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int k = 0; k < 3; ++k) red[threadIdx.x][k] += red[threadIdx.x + w][k];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < 3; ++k) apart[blockIdx.x * 3 + k] = red[0][k];
}

// Ubar_c += sum over (interface, slot j) whose stencil point maps to cell c.
template <int NDIM, int DIR>
__global__ void __launch_bounds__(256) adj_gather_kernel(const double* __restrict__ contrib,
                                                         double* __restrict__ Ubar, Grid G) {
  constexpr int NVAR = NDIM + 2;
  const int64_t ncell = G.ncell;
  const int64_t m0 = G.n[0] + (DIR == 0), m1 = G.n[1] + (DIR == 1);
  const int64_t nifc = m0 * m1 * (G.n[2] + (DIR == 2));
  const int64_t sd = (DIR == 0) ? 1 : (DIR == 1 ? m0 : m0 * m1);   // interface-grid stride along DIR
  const int64_t nd = G.n[DIR];
  const int bc = G.bc[DIR];
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i0 = c % G.n[0];
    const int64_t r = c / G.n[0];
    const int64_t i1 = r % G.n[1];
    const int64_t i2 = r / G.n[1];
    const int64_t id = (DIR == 0) ? i0 : (DIR == 1 ? i1 : i2);
    // interface-grid index of this line's interface 0
    const int64_t q0 = (i2 * m1 + i1) * m0 + i0 - id * sd;
    double acc[NVAR];
    for (int v = 0; v < NVAR; ++v) acc[v] = 0.0;
    for (int j = 0; j < 6; ++j) {
      // interfaces qd in [0, nd] whose point j, ghost(qd - 3 + j), is cell id
      if (bc == 0) {
        // x = qd - 3 + j ranges over [j - 3, nd + j - 3]; x = id (mod nd)
        int64_t x = id + ((j - 3 - id) / nd) * nd;
        while (x < j - 3) x += nd;
        while (x - nd >= j - 3) x -= nd;
        for (; x <= nd + j - 3; x += nd) {
          const int64_t qd = x + 3 - j;
          for (int v = 0; v < NVAR; ++v) acc[v] += contrib[(int64_t)(j * NVAR + v) * nifc + q0 + qd * sd];
        }
      } else {
        // transmissive: points below 0 map to cell 0, points above nd-1 to nd-1
        int64_t lo = id + 3 - j, hi = id + 3 - j;
        if (id == 0) lo = 0;
        if (id == nd - 1) hi = nd;
        if (lo < 0) lo = 0;
        if (hi > nd) hi = nd;
        for (int64_t qd = lo; qd <= hi; ++qd) {
          const int64_t x = qd - 3 + j;
          const int64_t mapped = x < 0 ? 0 : (x >= nd ? nd - 1 : x);
          if (mapped != id) continue;
          for (int v = 0; v < NVAR; ++v) acc[v] += contrib[(int64_t)(j * NVAR + v) * nifc + q0 + qd * sd];
        }
      }
    }
    for (int v = 0; v < NVAR; ++v) Ubar[v * ncell + c] += acc[v];
  }
}

// Sum the per-block d/dalpha in a fixed order and add its effect at the
// arg-max cells (one thread: the three kinds may share a cell).
template <int NDIM>
__global__ void adj_alpha_kernel(const double* __restrict__ apart, int nblocks,
                                 const unsigned long long* __restrict__ argidx, int dir,
                                 const double* __restrict__ U, double* __restrict__ Ubar, int64_t ncell,
                                 double gamma) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  constexpr int NVAR = NDIM + 2;
  double s[3] = {0.0, 0.0, 0.0};
  for (int b = 0; b < nblocks; ++b)
    for (int k = 0; k < 3; ++k) s[k] += apart[b * 3 + k];
  for (int k = 0; k < 3; ++k) {
    const unsigned long long c = argidx[dir * 3 + k];
    if (c >= (unsigned long long)ncell) continue;
    double Uc[NVAR], g[NVAR];
    for (int v = 0; v < NVAR; ++v) {
      Uc[v] = U[v * ncell + c];
      g[v] = 0.0;
    }
    teno_adj::wave_speed_grad<NDIM>(Uc, dir, k, gamma, s[k], g);
    for (int v = 0; v < NVAR; ++v) Ubar[v * ncell + c] += g[v];
  }
}

__global__ void set_value_kernel(double* p, double v) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *p = v;
}

// out = a x + b y (y may be null: out = a x)
__global__ void lincomb_kernel(double* __restrict__ out, double a, const double* __restrict__ x, double b,
                               const double* __restrict__ y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = y ? fma(a, x[i], b * y[i]) : a * x[i];
}

// ---------------------------------------------------------------------------
// workspace
// ---------------------------------------------------------------------------
constexpr size_t kAlign = 256;
size_t round_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

bool grid_valid(const teno_grid* g) {
  if (!g || g->ndim < 1 || g->ndim > 3) return false;
  for (int k = 0; k < 3; ++k) {
    if (g->n[k] < 1 || (k >= g->ndim && g->n[k] != 1)) return false;
    if (k < g->ndim && (!(g->dx[k] > 0.0) || !std::isfinite(g->dx[k]))) return false;
    if (k < g->ndim && g->bc[k] != TENO_BC_PERIODIC && g->bc[k] != TENO_BC_TRANSMISSIVE) return false;
  }
  if (!(g->gamma > 1.0) || !(g->H > 0.0) || !(g->eps > 0.0)) return false;
  if (g->b_l < 0 || g->b_u > 15 || g->b_u <= g->b_l) return false;
  return true;
}

int64_t nifc_of(const teno_grid* g, int d) {
  int64_t m = 1;
  for (int k = 0; k < 3; ++k) m *= g->n[k] + (k == d ? 1 : 0);
  return m;
}

int adj_blocks(int nsm) { return nsm * 8; }

struct AdjLayout {
  // header: [0] status, [8] dt, [64] alpha bits (9 x 8), [160] arg-max (9 x 8)
  size_t status = 0, dt = 8, alpha = 64, argidx = 160;
  size_t aux = 0, contrib = 0, apart = 0, R = 0, U1 = 0, U2 = 0, B1 = 0, B2 = 0, total = 0;
};

AdjLayout adj_layout(const teno_grid* g, int op, int nsm) {
  AdjLayout L;
  const size_t ncell = size_t(g->n[0] * g->n[1] * g->n[2]);
  const int nvar = g->ndim + 2;
  int64_t maxifc = 0;
  for (int d = 0; d < g->ndim; ++d) maxifc = nifc_of(g, d) > maxifc ? nifc_of(g, d) : maxifc;
  size_t off = kAlign;
  L.aux = off;
  off += round_up(sizeof(double) * (g->ndim + 3) * ncell);
  L.contrib = off;
  off += round_up(sizeof(double) * 6 * nvar * size_t(maxifc));
  L.apart = off;
  off += round_up(sizeof(double) * 3 * size_t(adj_blocks(nsm)));
  if (op == TENO_OP_RK3_ADJOINT) {
    // forward recomputation (R, U1, U2) and the stage adjoints (B1, B2)
    L.R = off;
    off += round_up(sizeof(double) * nvar * ncell);
    L.U1 = off;
    off += round_up(sizeof(double) * nvar * ncell);
    L.U2 = off;
    off += round_up(sizeof(double) * nvar * ncell);
    L.B1 = off;
    off += round_up(sizeof(double) * nvar * ncell);
    L.B2 = off;
    off += round_up(sizeof(double) * nvar * ncell);
  }
  L.total = off;
  return L;
}

int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
    n = 152;
  return n;
}

Grid make_grid(const teno_grid* g) {
  Grid G;
  for (int k = 0; k < 3; ++k) {
    G.n[k] = g->n[k];
    G.bc[k] = k < g->ndim ? g->bc[k] : 0;
    G.dx[k] = k < g->ndim ? g->dx[k] : 1.0;
    G.inv_dx[k] = 1.0 / G.dx[k];
  }
  G.ncell = g->n[0] * g->n[1] * g->n[2];
  return G;
}

bool is_dev(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

bool al(const void* p, size_t a) { return reinterpret_cast<uintptr_t>(p) % a == 0; }

template <int NDIM, int DIR>
void launch_adj_dir(int nblk, int nsm, cudaStream_t st, const double* U, const double* aux,
                    const unsigned long long* alpha, const double* Rbar, double scale, double* contrib,
                    double* apart, int* status, double* Ubar, const unsigned long long* argidx,
                    const Grid& G, const Scheme& S) {
  adj_flux_kernel<NDIM, DIR><<<nblk, kAdjThreads, 0, st>>>(U, aux, alpha, Rbar, scale, contrib, apart,
                                                          status, G, S);
  int64_t gb = (G.ncell + 255) / 256;
  if (gb > int64_t(nsm) * 16) gb = int64_t(nsm) * 16;
  adj_gather_kernel<NDIM, DIR><<<unsigned(gb), 256, 0, st>>>(contrib, Ubar, G);
  adj_alpha_kernel<NDIM><<<1, 32, 0, st>>>(apart, nblk, argidx, DIR, U, Ubar, G.ncell, S.gamma);
}

// Ubar += scale * J(U)^T Rbar
teno_status adjoint_sequence(const teno_grid* g, const AdjLayout& L, char* ws, const double* U,
                             const double* Rbar, double* Ubar, double scale, cudaStream_t st) {
  const Grid G = make_grid(g);
  const Scheme S = teno::make_scheme(g->gamma, g->H, g->eps, g->b_l, g->b_u);
  const int nsm = sm_count();
  const int nblk = adj_blocks(nsm);
  int* status = reinterpret_cast<int*>(ws + L.status);
  auto* alpha = reinterpret_cast<unsigned long long*>(ws + L.alpha);
  auto* argidx = reinterpret_cast<unsigned long long*>(ws + L.argidx);
  double* aux = reinterpret_cast<double*>(ws + L.aux);
  double* contrib = reinterpret_cast<double*>(ws + L.contrib);
  double* apart = reinterpret_cast<double*>(ws + L.apart);
  if (cudaMemsetAsync(alpha, 0, sizeof(unsigned long long) * 9, st) != cudaSuccess) return TENO_ERR_CUDA;
  if (cudaMemsetAsync(argidx, 0xff, sizeof(unsigned long long) * 9, st) != cudaSuccess) return TENO_ERR_CUDA;
  if (teno::launch_cell(g->ndim, U, aux, alpha, status, G.ncell, g->gamma, nsm, st) != cudaSuccess)
    return TENO_ERR_CUDA;
  int64_t cb = (G.ncell + 255) / 256;
  if (cb > int64_t(nsm) * 16) cb = int64_t(nsm) * 16;
  // the arg-max pass rewrites aux with the same values (same formulas)
  switch (g->ndim) {
    case 1: argmax_kernel<1><<<unsigned(cb), 256, 0, st>>>(U, alpha, argidx, G.ncell, g->gamma, aux); break;
    case 2: argmax_kernel<2><<<unsigned(cb), 256, 0, st>>>(U, alpha, argidx, G.ncell, g->gamma, aux); break;
    default: argmax_kernel<3><<<unsigned(cb), 256, 0, st>>>(U, alpha, argidx, G.ncell, g->gamma, aux); break;
  }
  for (int d = 0; d < g->ndim; ++d) {
    if (g->ndim == 1) launch_adj_dir<1, 0>(nblk, nsm, st, U, aux, alpha, Rbar, scale, contrib, apart, status, Ubar, argidx, G, S);
    else if (g->ndim == 2 && d == 0) launch_adj_dir<2, 0>(nblk, nsm, st, U, aux, alpha, Rbar, scale, contrib, apart, status, Ubar, argidx, G, S);
    else if (g->ndim == 2) launch_adj_dir<2, 1>(nblk, nsm, st, U, aux, alpha, Rbar, scale, contrib, apart, status, Ubar, argidx, G, S);
    else if (d == 0) launch_adj_dir<3, 0>(nblk, nsm, st, U, aux, alpha, Rbar, scale, contrib, apart, status, Ubar, argidx, G, S);
    else if (d == 1) launch_adj_dir<3, 1>(nblk, nsm, st, U, aux, alpha, Rbar, scale, contrib, apart, status, Ubar, argidx, G, S);
    else launch_adj_dir<3, 2>(nblk, nsm, st, U, aux, alpha, Rbar, scale, contrib, apart, status, Ubar, argidx, G, S);
    if (cudaGetLastError() != cudaSuccess) return TENO_ERR_CUDA;
  }
  return TENO_OK;
}

teno_status lincomb(double* out, double a, const double* x, double b, const double* y, int64_t n,
                    cudaStream_t st) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  lincomb_kernel<<<unsigned(blocks), 256, 0, st>>>(out, a, x, b, y, n);
  return cudaGetLastError() == cudaSuccess ? TENO_OK : TENO_ERR_CUDA;
}

}  // namespace

extern "C" {

size_t teno_adjoint_workspace_bytes(const teno_grid* g, int op) {
  if (!grid_valid(g) || (op != TENO_OP_RHS_ADJOINT && op != TENO_OP_RK3_ADJOINT)) return 0;
  return adj_layout(g, op, sm_count()).total;
}

teno_status teno_rhs_adjoint(const teno_grid* g, const double* U, const double* dUdt_bar, double* U_bar,
                             void* ws, size_t ws_bytes, void* stream) {
  if (!grid_valid(g) || !U || !dUdt_bar || !U_bar) return TENO_ERR_INVALID_ARG;
  if (!al(U, 16) || !al(dUdt_bar, 16) || !al(U_bar, 16)) return TENO_ERR_INVALID_ARG;
  if (U_bar == U || U_bar == dUdt_bar) return TENO_ERR_INVALID_ARG;
  if (!is_dev(U) || !is_dev(dUdt_bar) || !is_dev(U_bar)) return TENO_ERR_INVALID_ARG;
  const AdjLayout L = adj_layout(g, TENO_OP_RHS_ADJOINT, sm_count());
  if (!ws || !al(ws, kAlign) || ws_bytes < L.total || !is_dev(ws)) return TENO_ERR_WORKSPACE;
  return adjoint_sequence(g, L, static_cast<char*>(ws), U, dUdt_bar, U_bar, 1.0,
                          static_cast<cudaStream_t>(stream));
}

teno_status teno_rk3_step_adjoint(const teno_grid* g, const double* U_n, double dt, const double* Ubar_next,
                                  double* Ubar_n, void* ws, size_t ws_bytes, void* stream) {
  if (!grid_valid(g) || !U_n || !Ubar_next || !Ubar_n || !(dt >= 0.0) || !std::isfinite(dt))
    return TENO_ERR_INVALID_ARG;
  if (!al(U_n, 16) || !al(Ubar_next, 16) || !al(Ubar_n, 16) || Ubar_n == U_n) return TENO_ERR_INVALID_ARG;
  if (!is_dev(U_n) || !is_dev(Ubar_next) || !is_dev(Ubar_n)) return TENO_ERR_INVALID_ARG;
  const AdjLayout L = adj_layout(g, TENO_OP_RK3_ADJOINT, sm_count());
  if (!ws || !al(ws, kAlign) || ws_bytes < L.total || !is_dev(ws)) return TENO_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(ws);
  const int64_t ntot = int64_t(g->ndim + 2) * g->n[0] * g->n[1] * g->n[2];
  double* R = reinterpret_cast<double*>(w + L.R);
  double* U1 = reinterpret_cast<double*>(w + L.U1);
  double* U2 = reinterpret_cast<double*>(w + L.U2);
  double* B1 = reinterpret_cast<double*>(w + L.B1);
  double* B2 = reinterpret_cast<double*>(w + L.B2);
  double* dtp = reinterpret_cast<double*>(w + L.dt);

  // forward stages of the step (eq. 4.1-4.2) with the given dt
  set_value_kernel<<<1, 1, 0, st>>>(dtp, dt);
  if (cudaGetLastError() != cudaSuccess) return TENO_ERR_CUDA;
  teno_status s = teno::forward_stage(g, w, L.status, L.dt, L.alpha, L.aux, L.contrib, U_n, R, 2, U_n,
                                      nullptr, U1, st);
  if (s != TENO_OK) return s;
  s = teno::forward_stage(g, w, L.status, L.dt, L.alpha, L.aux, L.contrib, U1, R, 3, U_n, U1, U2, st);
  if (s != TENO_OK) return s;

  // reverse of eq. 4.3: B2 = 2/3 Ubar' + 2/3 dt J(U2)^T Ubar';  Ubar_n = 1/3 Ubar'
  if ((s = lincomb(B2, 2.0 / 3.0, Ubar_next, 0.0, nullptr, ntot, st)) != TENO_OK) return s;
  if ((s = adjoint_sequence(g, L, w, U2, Ubar_next, B2, 2.0 / 3.0 * dt, st)) != TENO_OK) return s;
  if ((s = lincomb(Ubar_n, 1.0 / 3.0, Ubar_next, 0.0, nullptr, ntot, st)) != TENO_OK) return s;
  // reverse of eq. 4.2: B1 = 1/4 B2 + 1/4 dt J(U1)^T B2;  Ubar_n += 3/4 B2
  if ((s = lincomb(B1, 0.25, B2, 0.0, nullptr, ntot, st)) != TENO_OK) return s;
  if ((s = adjoint_sequence(g, L, w, U1, B2, B1, 0.25 * dt, st)) != TENO_OK) return s;
  if ((s = lincomb(Ubar_n, 1.0, Ubar_n, 0.75, B2, ntot, st)) != TENO_OK) return s;
  // reverse of eq. 4.1: Ubar_n += B1 + dt J(U_n)^T B1
  if ((s = lincomb(Ubar_n, 1.0, Ubar_n, 1.0, B1, ntot, st)) != TENO_OK) return s;
  return adjoint_sequence(g, L, w, U_n, B1, Ubar_n, dt, st);
}

}  // extern "C"
