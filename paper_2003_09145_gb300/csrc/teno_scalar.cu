// teno_scalar.cu -- scalar mode: linear advection u_t + a u_x = 0 (Sec. 4.1,
// eq. 4.4) on a periodic 1D grid with the same TENO5-LAD reconstruction
// device code as the Euler path (teno5_lad), for the paper's scalar tests
// (Tab. 1 and the composite waves of eq. 4.6).
//
//   scalar_flux_kernel : one thread per interface: global Lax-Friedrichs
//                        split of f = a u (alpha = |a|), f^+ from
//                        u_{i-2..i+2}, f^- from u_{i+3..i-1};
//   scalar_diff_kernel : one thread per cell: -(f^_{i+1/2} - f^_{i-1/2})/dx,
//                        written or fused into the SSP-RK3 stage (eq. 4.1-4.3).
#include <cmath>
#include <cstdint>

#include <cuda_runtime.h>

#include "teno.h"
#include "teno_device.cuh"
#include "teno_flux.cuh"
#include "teno_launch.h"

namespace {

using teno::Scheme;

// f^ of the fixed linear weights of eq. 2.3 (all stencils kept) on v0..v4 =
// (f_{i-2}, ..., f_{i+2}): (2, -13, 47, 27, -3) / 60.
__device__ __forceinline__ double upwind5(double v0, double v1, double v2, double v3, double v4) {
  return (2.0 * v0 - 13.0 * v1 + 47.0 * v2 + 27.0 * v3 - 3.0 * v4) / 60.0;
}

__global__ void __launch_bounds__(128) scalar_flux_kernel(const double* __restrict__ u, int64_t n, double a,
                                                          int mode, Scheme S, double* __restrict__ F) {
  const double ap = 0.5 * (a + fabs(a)), am = 0.5 * (a - fabs(a));
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id <= n;
       id += (int64_t)gridDim.x * blockDim.x) {
    // interface id lies between cells id-1 and id; point j is cell id-3+j
    double w[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) w[j] = u[teno::ghost(id - 3 + j, n, TENO_BC_PERIODIC)];
    double f;
    if (mode == TENO_SCALAR_UPWIND5) {
      f = upwind5(ap * w[0], ap * w[1], ap * w[2], ap * w[3], ap * w[4]) +
          upwind5(am * w[5], am * w[4], am * w[3], am * w[2], am * w[1]);
    } else {
      unsigned fl = 0;
      const double hp = teno::teno5_lad<false>(ap * w[0], ap * w[1], ap * w[2], ap * w[3], ap * w[4], 0.0, S, fl);
      f = teno::teno5_lad<false>(am * w[5], am * w[4], am * w[3], am * w[2], am * w[1], hp, S, fl);
    }
    F[id] = f;
  }
}

// mode 0: R = d; 2, 3, 4: SSP-RK3 stage (stage_value) into out.
__global__ void __launch_bounds__(256) scalar_diff_kernel(const double* __restrict__ F, int64_t n, double idx,
                                                          int mode, double dt, const double* __restrict__ un,
                                                          const double* __restrict__ uk, double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double d = (F[i] - F[i + 1]) * idx;
    out[i] = mode == 0 ? d : teno::stage_value(mode, dt, d, un, uk, i);
  }
}

constexpr size_t kAlign = 256;
size_t round_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct ScalarLayout {
  size_t F = 0, u1 = 0, u2 = 0, total = 0;
};

ScalarLayout scalar_layout(int64_t n) {
  ScalarLayout L;
  size_t off = 0;
  L.F = off;
  off += round_up(sizeof(double) * size_t(n + 1));
  L.u1 = off;
  off += round_up(sizeof(double) * size_t(n));
  L.u2 = off;
  off += round_up(sizeof(double) * size_t(n));
  L.total = off;
  return L;
}

bool scalar_grid_ok(const teno_grid* g) {
  if (!g || g->ndim != 1 || g->n[0] < 1 || g->n[1] != 1 || g->n[2] != 1) return false;
  if (!(g->dx[0] > 0.0) || !std::isfinite(g->dx[0])) return false;
  if (!(g->H > 0.0) || !std::isfinite(g->H) || !(g->eps > 0.0) || !std::isfinite(g->eps)) return false;
  if (g->b_l < 0 || g->b_u > 15 || g->b_u <= g->b_l) return false;
  if (!teno::scheme_fields_ok(g)) return false;
  return true;
}

bool is_dev(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

bool aligned(const void* p, size_t a) { return reinterpret_cast<uintptr_t>(p) % a == 0; }

int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
    n = 152;
  return n;
}

int blocks_for(int64_t n, int threads, int cap) {
  int64_t b = (n + threads - 1) / threads;
  return int(b < 1 ? 1 : (b > cap ? cap : b));
}

teno_status check_args(const teno_grid* g, double a, int mode, const void* u, const void* ws, size_t ws_bytes) {
  if (!g) return TENO_ERR_INVALID_ARG;
  if (g->ndim == 1 && g->bc[0] != TENO_BC_PERIODIC) return TENO_ERR_UNSUPPORTED;
  if (!scalar_grid_ok(g) || !std::isfinite(a) || (mode != TENO_SCALAR_LAD && mode != TENO_SCALAR_UPWIND5))
    return TENO_ERR_INVALID_ARG;
  if (!u || !aligned(u, 16) || !is_dev(u)) return TENO_ERR_INVALID_ARG;
  if (!ws || !aligned(ws, kAlign) || ws_bytes < scalar_layout(g->n[0]).total || !is_dev(ws))
    return TENO_ERR_WORKSPACE;
  return TENO_OK;
}

// flux of u into F, then the difference (mode 0) or stage `mode` into out
teno_status scalar_stage(const teno_grid* g, double a, int mode_recon, const double* u, double* F, int mode,
                         double dt, const double* un, const double* uk, double* out, cudaStream_t st) {
  const int64_t n = g->n[0];
  const int nsm = sm_count();
  const Scheme S = teno::make_scheme(1.4, g->H, g->eps, g->b_l, g->b_u, g->scheme, g->ct_m);
  scalar_flux_kernel<<<blocks_for(n + 1, 128, nsm * 16), 128, 0, st>>>(u, n, a, mode_recon, S, F);
  scalar_diff_kernel<<<blocks_for(n, 256, nsm * 8), 256, 0, st>>>(F, n, 1.0 / g->dx[0], mode, dt, un, uk, out);
  return cudaGetLastError() == cudaSuccess ? TENO_OK : TENO_ERR_CUDA;
}

}  // namespace

extern "C" {

size_t teno_scalar_workspace_bytes(const teno_grid* g) {
  if (!scalar_grid_ok(g) || g->bc[0] != TENO_BC_PERIODIC) return 0;
  return scalar_layout(g->n[0]).total;
}

teno_status teno_scalar_rhs(const teno_grid* g, double a, int mode, const double* u, double* dudt, void* ws,
                            size_t ws_bytes, void* stream) {
  const teno_status s = check_args(g, a, mode, u, ws, ws_bytes);
  if (s != TENO_OK) return s;
  if (!dudt || dudt == u || !aligned(dudt, 16) || !is_dev(dudt)) return TENO_ERR_INVALID_ARG;
  const ScalarLayout L = scalar_layout(g->n[0]);
  double* F = reinterpret_cast<double*>(static_cast<char*>(ws) + L.F);
  return scalar_stage(g, a, mode, u, F, 0, 0.0, nullptr, nullptr, dudt, static_cast<cudaStream_t>(stream));
}

teno_status teno_scalar_rk3_step(const teno_grid* g, double a, int mode, double* u, double dt, void* ws,
                                 size_t ws_bytes, void* stream) {
  const teno_status s = check_args(g, a, mode, u, ws, ws_bytes);
  if (s != TENO_OK) return s;
  if (!(dt > 0.0) || !std::isfinite(dt)) return TENO_ERR_INVALID_ARG;
  const ScalarLayout L = scalar_layout(g->n[0]);
  char* w = static_cast<char*>(ws);
  double* F = reinterpret_cast<double*>(w + L.F);
  double* u1 = reinterpret_cast<double*>(w + L.u1);
  double* u2 = reinterpret_cast<double*>(w + L.u2);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  teno_status r;
  // eq. 4.1: u1 = u + dt L(u); eq. 4.2: u2 = 3/4 u + 1/4 u1 + 1/4 dt L(u1);
  // eq. 4.3: u <- 1/3 u + 2/3 u2 + 2/3 dt L(u2)
  if ((r = scalar_stage(g, a, mode, u, F, 2, dt, u, nullptr, u1, st)) != TENO_OK) return r;
  if ((r = scalar_stage(g, a, mode, u1, F, 3, dt, u, u1, u2, st)) != TENO_OK) return r;
  return scalar_stage(g, a, mode, u2, F, 4, dt, u, u2, u, st);
}

}  // extern "C"
