// teno_batched.cu -- many independent 1D Euler problems of uneven length
// advanced together: one persistent launch per SSP-RK3 stage.
//
// Each problem is a 1D grid of its own (own dx, time, final time and global
// Lax-Friedrichs speeds); the problems are packed back to back in one SoA
// array U[3][sum N].  A persistent grid of CTAs pulls whole problems from a
// device work queue (largest first, the order prepared by
// teno_batch_prepare).  For its problem a CTA
//   (A) evaluates the primitive variables, the half physical fluxes F/2 and
//       the problem's LF speeds (block reduction) and, in stage 1, the CFL
//       step and the new time;
//   (B) sweeps the problem in tiles of BLOCK - 1 cells: one thread per
//       interface flux with the same device code as teno_rhs (the certified
//       closed form; the faces it leaves pending are gathered into the first
//       lanes for the characteristic path), the fluxes of a tile in shared
//       memory, then the conservative difference fused with the stage update.
// No grid-wide synchronisation is needed: every dependency is inside a
// problem, and a problem never spans two CTAs.  The arithmetic is exactly
// that of teno_rk3_step on each problem alone, so results agree bit for bit.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <vector>

#include <cuda_runtime.h>

#include "teno.h"
#include "teno_device.cuh"
#include "teno_flux.cuh"
#include "teno_launch.h"

namespace {

using teno::Scheme;

struct BatchArgs {
  const double* Uin;   // state the fluxes are computed from
  const double* Un;    // U^n
  const double* Uk;    // U1 (stage 2) or U2 (stage 3)
  double* Uout;        // U1, U2 or U^{n+1}
  double* aux;         // [aux_fields(1) = 5][ncell] (the grid path's per-cell primitives)
  double* fh;          // [2][ncell]: F/2 of every cell (eq. 4.7), momentum and energy
  const int64_t* offsets;
  const double* dx;
  double* t;
  const double* t_end;
  double* dtv;
  const int* order;
  int* queue;
  int* status;
  int64_t nprob, ncell;
  int bc;
  double gamma, cfl, dt_fixed;
  int mode;            // 2, 3, 4: SSP-RK3 stage 1, 2, 3 (eq. 4.1-4.3)
};

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) batched_stage_kernel(BatchArgs A, Scheme S) {
  constexpr int NW = BLOCK / 32;
  __shared__ int s_q;
  __shared__ unsigned long long s_red[NW][3];
  __shared__ double s_alpha[3];
  __shared__ double s_dt, s_idx;
  __shared__ double s_F[BLOCK][3];
  __shared__ int s_pend[BLOCK];   // tile faces the certified test leaves pending
  __shared__ int s_npend;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  for (;;) {
    if (tid == 0) s_q = atomicAdd(A.queue, 1);
    __syncthreads();
    const int q = s_q;
    __syncthreads();
    if (q >= A.nprob) return;
    const int p = A.order[q];
    const int64_t off = A.offsets[p];
    const int64_t n = A.offsets[p + 1] - off;
    if (A.mode != 2 && !(A.dtv[p] > 0.0)) continue;  // finished problem

    // (A) primitive variables and LF speeds of this problem
    unsigned long long b0 = 0ull, b1 = 0ull, b2 = 0ull;   // bit patterns of the maxima
    bool bad = false;
    for (int64_t i = tid; i < n; i += BLOCK) {
      double uh[1], cs, ep;
      const int64_t c = off + i;
      if (!teno::cell_primitives<1>(A.Uin, A.ncell, c, A.gamma, A.aux, uh, cs, ep)) bad = true;
      const double Uc[3] = {A.Uin[c], A.Uin[A.ncell + c], A.Uin[2 * A.ncell + c]};
      double Fh[3];
      teno::cell_flux_half_ep<1, 0>(Uc, uh[0], A.aux[A.ncell + c], ep, Fh);
#pragma unroll
      for (int v = 1; v < 3; ++v) A.fh[(v - 1) * A.ncell + c] = Fh[v];
      // u -+ c from u/2 with one rounding; max|u| kept as max|u/2|
      b0 = teno::max_abs_bits(b0, fma(2.0, uh[0], -cs));
      b1 = teno::max_abs_bits(b1, uh[0]);
      b2 = teno::max_abs_bits(b2, fma(2.0, uh[0], cs));
    }
    b1 = teno::dbits(2.0 * __longlong_as_double(static_cast<long long>(b1)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long w0 = __shfl_xor_sync(0xffffffffu, b0, o);
      unsigned long long w1 = __shfl_xor_sync(0xffffffffu, b1, o);
      unsigned long long w2 = __shfl_xor_sync(0xffffffffu, b2, o);
      b0 = b0 > w0 ? b0 : w0;
      b1 = b1 > w1 ? b1 : w1;
      b2 = b2 > w2 ? b2 : w2;
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(A.status, teno::kStatusNonphysical);
    if (lane == 0) {
      s_red[warp][0] = b0;
      s_red[warp][1] = b1;
      s_red[warp][2] = b2;
    }
    __syncthreads();
    if (tid == 0) {
      unsigned long long m0 = 0, m1 = 0, m2 = 0;
      for (int w = 0; w < NW; ++w) {
        m0 = m0 > s_red[w][0] ? m0 : s_red[w][0];
        m1 = m1 > s_red[w][1] ? m1 : s_red[w][1];
        m2 = m2 > s_red[w][2] ? m2 : s_red[w][2];
      }
      s_alpha[0] = 0.5 * __longlong_as_double((long long)m0);
      s_alpha[1] = 0.5 * __longlong_as_double((long long)m1);
      s_alpha[2] = 0.5 * __longlong_as_double((long long)m2);
      const double dxp = A.dx[p];
      if (A.mode == 2) {
        // eq. dt1 with max(|u| + c) = max(max|u - c|, max|u + c|); clipped to t_end
        const double smax = __longlong_as_double((long long)(m0 > m2 ? m0 : m2));
        double dt = A.dt_fixed > 0.0 ? A.dt_fixed : A.cfl * dxp / smax;
        const double t = A.t[p];
        const double rem = A.t_end[p] - t;
        if (rem < dt) dt = rem;
        if (!(dt > 0.0)) dt = 0.0;
        A.dtv[p] = dt;
        A.t[p] = t + dt;
        s_dt = dt;
      } else {
        s_dt = A.dtv[p];
      }
      s_idx = (1.0 / dxp) / teno::kFluxScale;   // the fluxes are stored as kFluxScale F^
    }
    __syncthreads();
    const double dt = s_dt;
    if (!(dt > 0.0)) continue;
    const double alpha[3] = {s_alpha[0], s_alpha[1], s_alpha[2]};
    const double nal[3] = {-2.0 * s_alpha[0], -2.0 * s_alpha[1], -2.0 * s_alpha[2]};
    const double cdt = dt * s_idx;   // dt / (30 dx), as the grid path's stage coefficient

    // (B) fluxes tile by tile, difference fused with the stage update
    for (int64_t i0 = 0; i0 < n; i0 += BLOCK - 1) {
      // the grid path's two passes inside the tile: the certified closed form
      // for every face, then the faces it leaves pending, gathered into the
      // first lanes so that only ceil(pending / 32) warps take the
      // characteristic path (periodic or transmissive ends: no mirrored points)
      if (tid == 0) s_npend = 0;
      __syncthreads();
      const int64_t face = i0 + tid;
      if (face <= n) {
        int64_t cells[6];
#pragma unroll
        for (int j = 0; j < 6; ++j) cells[j] = off + teno::ghost(face - 3 + j, n, A.bc);
        double out[3];
        if (teno::interface_flux_closed<1, 0>(A.Uin, A.aux, A.fh, A.ncell, cells, 0u, alpha, nal, S, out,
                                              A.status)) {
          s_F[tid][0] = out[0];
          s_F[tid][1] = out[1];
          s_F[tid][2] = out[2];
        } else {
          s_pend[atomicAdd(&s_npend, 1)] = tid;
        }
      }
      __syncthreads();
      if (tid < s_npend) {
        const int t = s_pend[tid];
        const int64_t f2 = i0 + t;
        int64_t cells[6];
#pragma unroll
        for (int j = 0; j < 6; ++j) cells[j] = off + teno::ghost(f2 - 3 + j, n, A.bc);
        double out[3];
        unsigned fl[3][2];
        teno::interface_flux<1, 0, false, teno::kFluxChar>(A.Uin, A.aux, A.ncell, cells, 0u, alpha, nal, S, out, fl,
                                                           A.status);
        s_F[t][0] = out[0];
        s_F[t][1] = out[1];
        s_F[t][2] = out[2];
      }
      __syncthreads();
      const int64_t cell = i0 + tid;
      if (tid < BLOCK - 1 && cell < n) {
#pragma unroll
        for (int v = 0; v < 3; ++v) {
          const double t = s_F[tid][v] - s_F[tid + 1][v];
          const int64_t e = v * A.ncell + off + cell;
          A.Uout[e] = teno::stage_value(A.mode, cdt, t, A.Un, A.Uk, e);
        }
      }
      __syncthreads();
    }
  }
}

constexpr size_t kAlign = 256;
size_t round_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct BatchLayout {
  size_t status = 0, queue = 64, order = 0, dt = 0, aux = 0, fh = 0, U1 = 0, U2 = 0, total = 0;
};

bool batch_ok(const teno_batch* b) {
  if (!b || b->nprob < 1 || b->nprob > (int64_t(1) << 30) || b->ncell < b->nprob) return false;
  if (b->ncell > (int64_t(1) << 40)) return false;
  if (b->bc != TENO_BC_PERIODIC && b->bc != TENO_BC_TRANSMISSIVE) return false;
  if (!(b->gamma > 1.0) || !(b->H > 0.0) || !(b->eps > 0.0)) return false;
  if (b->b_l < 0 || b->b_u > 15 || b->b_u <= b->b_l) return false;
  return true;
}

BatchLayout batch_layout(const teno_batch* b) {
  BatchLayout L;
  size_t off = kAlign;
  L.order = off;
  off += round_up(sizeof(int) * size_t(b->nprob));
  L.dt = off;
  off += round_up(sizeof(double) * size_t(b->nprob));
  L.aux = off;
  off += round_up(sizeof(double) * teno::aux_fields(1) * size_t(b->ncell));
  L.fh = off;
  off += round_up(sizeof(double) * 2 * size_t(b->ncell));
  L.U1 = off;
  off += round_up(sizeof(double) * 3 * size_t(b->ncell));
  L.U2 = off;
  off += round_up(sizeof(double) * 3 * size_t(b->ncell));
  L.total = off;
  return L;
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

}  // namespace

extern "C" {

size_t teno_batch_workspace_bytes(const teno_batch* b) {
  if (!batch_ok(b)) return 0;
  return batch_layout(b).total;
}

teno_status teno_batch_prepare(const teno_batch* b, const int64_t* offsets_host, void* ws,
                               size_t ws_bytes, void* stream) {
  if (b && b->bc == TENO_BC_REFLECTIVE) return TENO_ERR_UNSUPPORTED;
  if (!batch_ok(b) || !offsets_host) return TENO_ERR_INVALID_ARG;
  const BatchLayout L = batch_layout(b);
  if (!ws || !al(ws, kAlign) || ws_bytes < L.total || !is_dev(ws)) return TENO_ERR_WORKSPACE;
  if (offsets_host[0] != 0 || offsets_host[b->nprob] != b->ncell) return TENO_ERR_INVALID_ARG;
  std::vector<int64_t> n(size_t(b->nprob));
  for (int64_t p = 0; p < b->nprob; ++p) {
    n[p] = offsets_host[p + 1] - offsets_host[p];
    if (n[p] < 1) return TENO_ERR_INVALID_ARG;
  }
  // largest problems first (longest-processing-time order), ties by index
  std::vector<int> order(size_t(b->nprob));
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return n[a] > n[c]; });
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(ws);
  if (cudaMemsetAsync(w, 0, kAlign, st) != cudaSuccess) return TENO_ERR_CUDA;
  if (cudaMemcpyAsync(w + L.order, order.data(), sizeof(int) * order.size(), cudaMemcpyHostToDevice,
                      st) != cudaSuccess)
    return TENO_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return TENO_ERR_CUDA;
  return TENO_OK;
}

teno_status teno_rk3_step_batched(const teno_batch* b, const int64_t* offsets, const double* dx,
                                  double* U, double* t_dev, const double* t_end_dev, double cfl,
                                  double dt_fixed, const teno_batch_tuning* tuning, void* ws,
                                  size_t ws_bytes, void* stream) {
  if (b && b->bc == TENO_BC_REFLECTIVE) return TENO_ERR_UNSUPPORTED;
  if (!batch_ok(b) || !offsets || !dx || !U || !t_dev || !t_end_dev) return TENO_ERR_INVALID_ARG;
  if (!al(U, 16) || !al(offsets, 8) || !al(dx, 8) || !al(t_dev, 8) || !al(t_end_dev, 8))
    return TENO_ERR_INVALID_ARG;
  if (!(dt_fixed > 0.0) && !(cfl > 0.0 && std::isfinite(cfl))) return TENO_ERR_INVALID_ARG;
  if (!std::isfinite(dt_fixed)) return TENO_ERR_INVALID_ARG;
  if (!is_dev(U) || !is_dev(offsets) || !is_dev(dx) || !is_dev(t_dev) || !is_dev(t_end_dev))
    return TENO_ERR_INVALID_ARG;
  const BatchLayout L = batch_layout(b);
  if (!ws || !al(ws, kAlign) || ws_bytes < L.total || !is_dev(ws)) return TENO_ERR_WORKSPACE;
  int block = tuning ? tuning->block : 128;
  int per_sm = tuning ? tuning->ctas_per_sm : 4;
  if (block != 64 && block != 128 && block != 256) return TENO_ERR_INVALID_ARG;
  if (per_sm < 1 || per_sm > 32) return TENO_ERR_INVALID_ARG;

  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0)
    nsm = 152;
  int64_t grid = int64_t(nsm) * per_sm;
  if (grid > b->nprob) grid = b->nprob;

  char* w = static_cast<char*>(ws);
  BatchArgs A;
  A.aux = reinterpret_cast<double*>(w + L.aux);
  A.fh = reinterpret_cast<double*>(w + L.fh);
  A.offsets = offsets;
  A.dx = dx;
  A.t = t_dev;
  A.t_end = t_end_dev;
  A.dtv = reinterpret_cast<double*>(w + L.dt);
  A.order = reinterpret_cast<const int*>(w + L.order);
  A.queue = reinterpret_cast<int*>(w + L.queue);
  A.status = reinterpret_cast<int*>(w + L.status);
  A.nprob = b->nprob;
  A.ncell = b->ncell;
  A.bc = b->bc;
  A.gamma = b->gamma;
  A.cfl = cfl;
  A.dt_fixed = dt_fixed;
  const Scheme S = teno::make_scheme(b->gamma, b->H, b->eps, b->b_l, b->b_u);
  double* U1 = reinterpret_cast<double*>(w + L.U1);
  double* U2 = reinterpret_cast<double*>(w + L.U2);
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  for (int stage = 0; stage < 3; ++stage) {
    A.mode = 2 + stage;
    A.Un = U;
    if (stage == 0) { A.Uin = U; A.Uk = nullptr; A.Uout = U1; }
    else if (stage == 1) { A.Uin = U1; A.Uk = U1; A.Uout = U2; }
    else { A.Uin = U2; A.Uk = U2; A.Uout = U; }
    if (cudaMemsetAsync(A.queue, 0, sizeof(int), st) != cudaSuccess) return TENO_ERR_CUDA;
    switch (block) {
      case 64: batched_stage_kernel<64><<<unsigned(grid), 64, 0, st>>>(A, S); break;
      case 256: batched_stage_kernel<256><<<unsigned(grid), 256, 0, st>>>(A, S); break;
      default: batched_stage_kernel<128><<<unsigned(grid), 128, 0, st>>>(A, S); break;
    }
    if (cudaGetLastError() != cudaSuccess) return TENO_ERR_CUDA;
  }
  return TENO_OK;
}

}  // extern "C"
