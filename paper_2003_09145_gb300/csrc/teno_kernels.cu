// teno_kernels.cu -- sm_103a kernels of the TENO5-LAD Euler right-hand side
// and the SSP-RK3 stage updates (all FP64).
//
// One right-hand-side evaluation L(U) (eq. 2.2) is
//   cell_kernel    : per cell, primitive variables (u_k, p) and the Roe weights
//                    sqrt(rho), (E + p)/sqrt(rho); the global Lax-Friedrichs
//                    speeds alpha_{d,s} = max |lambda_s| of every direction
//                    (warp-shuffle max, block max, one atomic per block);
//   flux_kernel<D> : per interface of direction D, one thread: the six-point
//                    flux stencil, Roe eigensystem, characteristic projection,
//                    LF splitting, 2 x nvar TENO5-LAD reconstructions and the
//                    back-projection to the interface flux F^;
//   diff_kernel<D> : per cell, -(F^_{i+1/2} - F^_{i-1/2}) / dx_D, written,
//                    accumulated, or fused into the SSP-RK3 stage (eq. 4.1-4.3).
#include <cmath>
#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>

#include "teno_device.cuh"
#include "teno_flux.cuh"
#include "teno_launch.h"

namespace teno {

// ---------------------------------------------------------------------------
// Cell pass: primitive variables, Roe weights and LF speeds.
// The primitive variables come from one reciprocal square root per cell
// (cell_primitives); the wave speeds |u_d - c|, |u_d|, |u_d + c| are reduced
// to their maxima over all cells.
// aux layout: [aux_fields(ndim) = 2 ndim + 3][ncell]: u_0/2..u_{ndim-1}/2,
// p/2, sqrt(rho), (E+p)/sqrt(rho), m_0/sqrt(rho)..m_{ndim-1}/sqrt(rho).
// With `fh`, also the half physical fluxes F_d/2 (eq. 4.7)
// of every direction, momentum and energy components only (the mass one is
// m_d/2), [ndim][nvar - 1][ncell], for the closed-form flux pass.
// alpha layout (bit patterns of non-negative doubles): [ndim][3] =
// max|u_d - c|, max|u_d|, max|u_d + c|.
// ---------------------------------------------------------------------------
// F_d/2 of cell c for d = D..NDIM-1 into fh[d][v - 1][c], v = 1..nvar-1.
template <int NDIM, int D>
__device__ __forceinline__ void store_flux_half(const double (&Uc)[NDIM + 2], const double (&uh)[NDIM], double pn,
                                                double ep, double* __restrict__ fh, int64_t ncell, int64_t c) {
  if constexpr (D < NDIM) {
    constexpr int NVAR = NDIM + 2;
    double Fh[NVAR];
    cell_flux_half_ep<NDIM, D>(Uc, uh[D], pn, ep, Fh);
#pragma unroll
    for (int v = 1; v < NVAR; ++v) fh[(int64_t)(D * (NVAR - 1) + v - 1) * ncell + c] = Fh[v];
    store_flux_half<NDIM, D + 1>(Uc, uh, pn, ep, fh, ncell, c);
  }
}

#ifndef TENO_CELL_MINBLOCKS
#define TENO_CELL_MINBLOCKS 2   // 128 registers, 16 warps per SM: measured 0.1 ms per step
#endif                          // faster than 3 (80 registers) or 4 (64)
// With ARG, every block also writes, per speed, its largest value and the
// lowest cell index attaining it to cand[block][9][2] (value bits, index):
// the arg-max cells through which the adjoint differentiates the global
// speeds (argmax_finish_kernel reduces the candidates).
template <int NDIM, bool ARG>
__global__ void __launch_bounds__(256, TENO_CELL_MINBLOCKS) cell_kernel(const double* __restrict__ U,
                                                   double* __restrict__ aux,
                                                   double* __restrict__ fh,
                                                   unsigned long long* __restrict__ alpha,
                                                   int* __restrict__ status,
                                                   int64_t ncell, double gamma,
                                                   unsigned long long* __restrict__ cand) {
  constexpr int NVAR = NDIM + 2;
  unsigned long long lam[NDIM][3];   // bit patterns of the running maxima (>= 0)
  long long arg[NDIM][3];            // (ARG) the first cell of this thread attaining each
#pragma unroll
  for (int d = 0; d < NDIM; ++d)
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      lam[d][s] = 0ull;
      arg[d][s] = ncell;
    }
  bool bad = false;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell;
       c += (int64_t)gridDim.x * blockDim.x) {
    double uh[NDIM], cs, ep;
    if (!cell_primitives<NDIM>(U, ncell, c, gamma, aux, uh, cs, ep)) bad = true;
    if (fh) {
      double Uc[NVAR];
#pragma unroll
      for (int v = 0; v < NVAR; ++v) Uc[v] = U[v * ncell + c];
      const double pn = aux[NDIM * ncell + c];
      store_flux_half<NDIM, 0>(Uc, uh, pn, ep, fh, ncell, c);
    }
    // u -+ c = 2 (u/2) -+ c with one rounding, as a subtraction of u would;
    // max|u| is kept as max|u/2| and doubled (exactly) below
#pragma unroll
    for (int d = 0; d < NDIM; ++d) {
      const double x[3] = {fma(2.0, uh[d], -cs), uh[d], fma(2.0, uh[d], cs)};
#pragma unroll
      for (int s = 0; s < 3; ++s) {
        if constexpr (ARG) {
          const unsigned long long m = max_abs_bits(lam[d][s], x[s]);
          if (m != lam[d][s]) arg[d][s] = c;
          lam[d][s] = m;
        } else {
          lam[d][s] = max_abs_bits(lam[d][s], x[s]);
        }
      }
    }
  }
#pragma unroll
  for (int d = 0; d < NDIM; ++d) lam[d][1] = dbits(2.0 * __longlong_as_double(static_cast<long long>(lam[d][1])));
  // warp max on bit patterns (all values are >= 0); with ARG the lowest
  // index among the lanes holding the maximum
  __shared__ unsigned long long red[8][NDIM * 3];
  __shared__ long long rarg[ARG ? 8 : 1][NDIM * 3];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int d = 0; d < NDIM; ++d)
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      unsigned long long v = lam[d][s];
      long long a = arg[d][s];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        if constexpr (ARG) {
          const long long b = __shfl_xor_sync(0xffffffffu, a, o);
          if (w > v || (w == v && b < a)) a = b;
        }
        v = v > w ? v : w;
      }
      if (lane == 0) {
        red[warp][d * 3 + s] = v;
        if constexpr (ARG) rarg[warp][d * 3 + s] = a;
      }
    }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(status, kStatusNonphysical);
  __syncthreads();
  if (threadIdx.x < NDIM * 3) {
    unsigned long long v = 0;
    long long a = ncell;
    const int nw = blockDim.x >> 5;
    for (int w = 0; w < nw; ++w) {
      const unsigned long long x = red[w][threadIdx.x];
      if constexpr (ARG) {
        const long long b = rarg[w][threadIdx.x];
        if (x > v || (x == v && b < a)) a = b;
      }
      v = v > x ? v : x;
    }
    atomicMax(&alpha[threadIdx.x], v);
    if constexpr (ARG) {
      cand[(blockIdx.x * 9 + threadIdx.x) * 2] = v;
      cand[(blockIdx.x * 9 + threadIdx.x) * 2 + 1] = static_cast<unsigned long long>(a);
    }
  }
}

// The arg-max cells of the nine LF speeds from the cell pass's per-block
// candidates: the largest value of each speed and the lowest cell index
// attaining it (entries of unused directions stay as they are).
constexpr int kArgThreads = 256;
__global__ void __launch_bounds__(kArgThreads) argmax_finish_kernel(const unsigned long long* __restrict__ cand,
                                                                    int nblocks, int nspeed,
                                                                    unsigned long long* __restrict__ argidx) {
  __shared__ unsigned long long sv[kArgThreads];
  __shared__ unsigned long long sa[kArgThreads];
  for (int k = 0; k < nspeed; ++k) {
    unsigned long long v = 0, a = ~0ull;
    for (int b = threadIdx.x; b < nblocks; b += kArgThreads) {
      const unsigned long long x = cand[(b * 9 + k) * 2], i = cand[(b * 9 + k) * 2 + 1];
      if (x > v || (x == v && i < a)) {
        v = x;
        a = i;
      }
    }
    sv[threadIdx.x] = v;
    sa[threadIdx.x] = a;
    __syncthreads();
    for (int w = kArgThreads / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) {
        const unsigned long long x = sv[threadIdx.x + w], i = sa[threadIdx.x + w];
        if (x > sv[threadIdx.x] || (x == sv[threadIdx.x] && i < sa[threadIdx.x])) {
          sv[threadIdx.x] = x;
          sa[threadIdx.x] = i;
        }
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) argidx[k] = sa[0];
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Interface fluxes of direction DIR.
// ---------------------------------------------------------------------------

#ifndef TENO_FLUX_MINBLOCKS
#define TENO_FLUX_MINBLOCKS 4
#endif

template <int NDIM, int DIR, bool WITH_FLAGS, bool GH>
__global__ void __launch_bounds__(128, TENO_FLUX_MINBLOCKS) flux_kernel(
    const double* __restrict__ U, const double* __restrict__ aux,
    const unsigned long long* __restrict__ alpha_bits, double* __restrict__ Fhat,
    uint8_t* __restrict__ flags, int* __restrict__ status, Grid G, Scheme S) {
  constexpr int NVAR = NDIM + 2;
  // interface grid: n along the other axes, n_DIR + 1 along DIR
  const int64_t m0 = G.n[0] + (DIR == 0), m1 = G.n[1] + (DIR == 1), m2 = G.n[2] + (DIR == 2);
  const int64_t nifc = m0 * m1 * m2;
  const int64_t ncell = G.ncell;
  const int64_t stride_d = (DIR == 0) ? 1 : (DIR == 1 ? G.n[0] : G.n[0] * G.n[1]);
  const int64_t nd = G.n[DIR];
  const int bcd = G.bc[DIR];

  double alpha[NVAR];
  {
    double am = __longlong_as_double((long long)alpha_bits[DIR * 3 + 0]);
    double a0 = __longlong_as_double((long long)alpha_bits[DIR * 3 + 1]);
    double ap = __longlong_as_double((long long)alpha_bits[DIR * 3 + 2]);
    alpha[0] = 0.5 * am;
#pragma unroll
    for (int f = 1; f < NVAR - 1; ++f) alpha[f] = 0.5 * a0;
    alpha[NVAR - 1] = 0.5 * ap;
  }
  double nal[NVAR];
#pragma unroll
  for (int f = 0; f < NVAR; ++f) nal[f] = -2.0 * alpha[f];

  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nifc;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i0 = q % m0;
    const int64_t r = q / m0;
    const int64_t i1 = r % m1;
    const int64_t i2 = r / m1;
    const int64_t id = (DIR == 0) ? i0 : (DIR == 1 ? i1 : i2);
    // linear index of the cell with coordinate 0 along DIR on this line
    const int64_t base = (DIR == 0) ? (i2 * G.n[1] + i1) * G.n[0]
                       : (DIR == 1) ? i2 * G.n[1] * G.n[0] + i0
                                    : i1 * G.n[0] + i0;

    int64_t cells[6];
    unsigned flips = 0u;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      bool f;
      const int64_t k = id - 3 + j;
      cells[j] = (GH && (k < 0 || k >= nd)) ? ncell + 2 * DIR + (k >= nd) : base + ghost(k, nd, bcd, f) * stride_d;
      flips |= GH ? 0u : unsigned(f) << j;
    }
    double out[NVAR];
    unsigned fl[NVAR][2];
    interface_flux<NDIM, DIR, WITH_FLAGS, kFluxFull, GH>(U, aux, ncell, cells, flips, alpha, nal, S, out, fl, status,
                                                        GhostCells{G.gU, G.gaux, G.gfh});
    if (WITH_FLAGS) {
      // direction block offset is applied by the caller through `flags`
#pragma unroll
      for (int s = 0; s < NVAR; ++s)
#pragma unroll
        for (int side = 0; side < 2; ++side)
          flags[(int64_t)(s * 2 + side) * nifc + q] = (uint8_t)fl[s][side];
    }
#pragma unroll
    for (int v = 0; v < NVAR; ++v) Fhat[(int64_t)v * nifc + q] = out[v];
  }
}

// ---------------------------------------------------------------------------
// The same fluxes in two passes (no flags).  flux_closed_kernel evaluates the
// certified closed form -- every interface whose FP32 test keeps all ten
// stencils -- and appends the others to `list` (one atomic per warp);
// flux_pending_kernel then takes the listed interfaces through the
// characteristic path.  Each interface gets the arithmetic of the one-pass
// kernel, except that the closed form's six-point sums are fixed-point sums
// rounded once (teno_fixsum.cuh: terms on a grid of an eighth of the largest
// value's ulp, added exactly) where the one-pass kernel chains binary64
// operations; the closed-form pass stays small (registers,
// instruction cache) and its warps do not diverge into the rare slow path.
// ---------------------------------------------------------------------------
#ifndef TENO_CLOSED_MINBLOCKS
#define TENO_CLOSED_MINBLOCKS 4
#endif
// the z sweep's tiled order (below): 36.93 against 37.36 ms per 256^3 RK3 step
#ifndef TENO_CLOSED_Z_TILE
#define TENO_CLOSED_Z_TILE 1
#endif

// GH: fixed-state faces along DIR, whose ghost points are the virtual cells
// ncell + 2 DIR + side
template <int NDIM, int DIR, bool GH = false>
__device__ __forceinline__ void interface_cells(int64_t q, const Grid& G, int64_t (&cells)[6], unsigned& flips) {
  const int64_t m0 = G.n[0] + (DIR == 0), m1 = G.n[1] + (DIR == 1);
  const int64_t stride_d = (DIR == 0) ? 1 : (DIR == 1 ? G.n[0] : G.n[0] * G.n[1]);
  const int64_t i0 = q % m0;
  const int64_t r = q / m0;
  const int64_t i1 = r % m1;
  const int64_t i2 = r / m1;
  const int64_t id = (DIR == 0) ? i0 : (DIR == 1 ? i1 : i2);
  const int64_t base = (DIR == 0) ? (i2 * G.n[1] + i1) * G.n[0]
                     : (DIR == 1) ? i2 * G.n[1] * G.n[0] + i0
                                  : i1 * G.n[0] + i0;
  flips = 0u;
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    bool f;
    const int64_t k = id - 3 + j;
    if (GH && (k < 0 || k >= G.n[DIR])) {
      cells[j] = G.ncell + 2 * DIR + (k >= G.n[DIR]);
    } else {
      cells[j] = base + ghost(k, G.n[DIR], G.bc[DIR], f) * stride_d;
      flips |= unsigned(f) << j;
    }
  }
}

template <int NDIM, int DIR>
__device__ __forceinline__ void half_speeds(const unsigned long long* __restrict__ alpha_bits,
                                            double (&alpha)[NDIM + 2], double (&nal)[NDIM + 2]) {
  constexpr int NVAR = NDIM + 2;
  const double am = __longlong_as_double((long long)alpha_bits[DIR * 3 + 0]);
  const double a0 = __longlong_as_double((long long)alpha_bits[DIR * 3 + 1]);
  const double ap = __longlong_as_double((long long)alpha_bits[DIR * 3 + 2]);
  alpha[0] = 0.5 * am;
#pragma unroll
  for (int f = 1; f < NVAR - 1; ++f) alpha[f] = 0.5 * a0;
  alpha[NVAR - 1] = 0.5 * ap;
#pragma unroll
  for (int f = 0; f < NVAR; ++f) nal[f] = -2.0 * alpha[f];
}

// WALL: 1 -- the sweep direction has a reflecting wall, so stencil points may
// be mirrored; 2 -- fixed-state faces (ghost points read from the ghost
// block); 0 -- neither: the mirror flags are the constant 0 and their sign
// flips fold away.  With ROE every interface's Roe state (the fields the
// certificate and the adjoint's closed-form VJP read: u~, |u~|^2, H~, c~,
// b1, b1/2, b2/2, 1/(2c~)) and the certificate's decision (1 kept, 0
// pending) also go to roe_out[ndim + 8][nifc], for the adjoint of this
// stage.
template <int NDIM, int DIR, int WALL, bool ROE = false>
__global__ void __launch_bounds__(128, TENO_CLOSED_MINBLOCKS) flux_closed_kernel(
    const double* __restrict__ U, const double* __restrict__ aux, const double* __restrict__ fh,
    const unsigned long long* __restrict__ alpha_bits, double* __restrict__ Fhat,
    uint32_t* __restrict__ list, unsigned* __restrict__ count, int* __restrict__ status, Grid G,
    Scheme S, double* __restrict__ roe_out = nullptr) {
  constexpr int NVAR = NDIM + 2;
  const int64_t nifc = (G.n[0] + (DIR == 0)) * (G.n[1] + (DIR == 1)) * (G.n[2] + (DIR == 2));
  double alpha[NVAR], nal[NVAR];
  half_speeds<NDIM, DIR>(alpha_bits, alpha, nal);
  const unsigned lane = threadIdx.x & 31u;
  // The z sweep takes its interfaces in tiles of 32 along x by 4 along z
  // (a block of 128 threads per tile, a warp per z): the six stencil planes
  // of one interface lie a power of two of bytes apart and share L1 sets,
  // so the second pass's reload misses L1 unless the block's four warps
  // read overlapping planes.  The loop runs over whole tiles; lanes past the
  // grid's edge skip.
  constexpr bool ZT = TENO_CLOSED_Z_TILE && DIR == 2 && NDIM == 3;
  const uint32_t n0 = static_cast<uint32_t>(G.n[0]), n1 = static_cast<uint32_t>(G.n[1]);
  const uint32_t nz1 = static_cast<uint32_t>(G.n[2] + 1);
  const uint32_t ntx = (n0 + 31u) / 32u;
  const int64_t nq = ZT ? (int64_t)ntx * n1 * ((nz1 + 3u) / 4u) * 128 : nifc;
  for (int64_t qq = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; qq < nq;
       qq += (int64_t)gridDim.x * blockDim.x) {
    int64_t q = qq;
    if constexpr (ZT) {
      const uint32_t t = static_cast<uint32_t>(qq >> 7), l = static_cast<uint32_t>(qq) & 127u;
      const uint32_t x = (t % ntx) * 32u + (l & 31u);
      const uint32_t r = t / ntx;
      const uint32_t z = (r / n1) * 4u + (l >> 5);
      if (x >= n0 || z >= nz1) continue;
      q = ((int64_t)z * n1 + (r % n1)) * n0 + x;
    }
    int64_t cells[6];
    unsigned flips;
    interface_cells<NDIM, DIR, WALL == 2>(q, G, cells, flips);
    double out[NVAR];
    RoeIfc<NDIM> R;
    const bool done = interface_flux_closed<NDIM, DIR, WALL == 2>(
        U, aux, fh + (int64_t)DIR * (NVAR - 1) * G.ncell, G.ncell, cells, WALL == 1 ? flips : 0u, alpha, nal, S,
        out, status, GhostCells{G.gU, G.gaux, G.gfh}, ROE ? &R : nullptr);
    if constexpr (ROE) {
      if (S.keep_idx >= 0) {
#pragma unroll
        for (int k = 0; k < NDIM; ++k) roe_out[(int64_t)k * nifc + q] = R.u[k];
        roe_out[(int64_t)(NDIM + 0) * nifc + q] = R.q2;
        roe_out[(int64_t)(NDIM + 1) * nifc + q] = R.H;
        roe_out[(int64_t)(NDIM + 2) * nifc + q] = R.cs;
        roe_out[(int64_t)(NDIM + 3) * nifc + q] = R.b1;
        roe_out[(int64_t)(NDIM + 4) * nifc + q] = R.hb1;
        roe_out[(int64_t)(NDIM + 5) * nifc + q] = R.hb2;
        roe_out[(int64_t)(NDIM + 6) * nifc + q] = R.hic;
        roe_out[(int64_t)(NDIM + 7) * nifc + q] = done ? 1.0 : 0.0;
      }
    }
    if (done) {
#pragma unroll
      for (int v = 0; v < NVAR; ++v) Fhat[(int64_t)v * nifc + q] = out[v];
    }
    // append the undecided interfaces of the lanes converged here
    const unsigned act = __activemask();
    const unsigned m = __ballot_sync(act, !done);
    if (m) {
      const unsigned leader = __ffs(act) - 1;
      unsigned at = 0;
      if (lane == leader) at = atomicAdd(count, __popc(m));
      at = __shfl_sync(act, at, leader);
      if (!done) list[at + __popc(m & ((1u << lane) - 1u))] = static_cast<uint32_t>(q);
    }
  }
}

template <int NDIM, int DIR, bool GH>
__global__ void __launch_bounds__(128) flux_pending_kernel(
    const double* __restrict__ U, const double* __restrict__ aux,
    const unsigned long long* __restrict__ alpha_bits, double* __restrict__ Fhat,
    const uint32_t* __restrict__ list, const unsigned* __restrict__ count, int* __restrict__ status,
    Grid G, Scheme S) {
  constexpr int NVAR = NDIM + 2;
  const int64_t nifc = (G.n[0] + (DIR == 0)) * (G.n[1] + (DIR == 1)) * (G.n[2] + (DIR == 2));
  const int64_t n = *count;
  if (blockIdx.x * (int64_t)blockDim.x >= n) return;
  double alpha[NVAR], nal[NVAR];
  half_speeds<NDIM, DIR>(alpha_bits, alpha, nal);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = list[i];
    int64_t cells[6];
    unsigned flips;
    interface_cells<NDIM, DIR, GH>(q, G, cells, flips);
    double out[NVAR];
    unsigned fl[NVAR][2];
    interface_flux<NDIM, DIR, false, kFluxChar, GH>(U, aux, G.ncell, cells, flips, alpha, nal, S, out, fl, status,
                                                   GhostCells{G.gU, G.gaux, G.gfh});
#pragma unroll
    for (int v = 0; v < NVAR; ++v) Fhat[(int64_t)v * nifc + q] = out[v];
  }
}

// ---------------------------------------------------------------------------
// Conservative difference (eq. 2.2) and SSP-RK3 stage update (eq. 4.1-4.3).
// With t_d = F^_{i-1/2} - F^_{i+1/2} of direction d and r_d = dx_0 / dx_d,
// L(U) = (t_0 + r_1 t_1 + r_2 t_2) / dx_0: R carries the unscaled partial
// sum and 1/dx_0 is applied once (in the stage's coefficient, or at the end
// of a plain right-hand side), one FP64 instruction fewer per element than
// scaling every direction -- the passes are bound by FP64 issue.  The
// fluxes arrive as kFluxScale F^ (teno_flux.cuh), so that factor is
// divided out with dx_0 (dx_0 below stands for kFluxScale dx_0).
// MODE (a template argument, so that every load of a cell is issued before
// its stores):
//   kDiffFirst  R = t_0                        (first of several directions)
//   kDiffAcc    R += r_d t_d                   (a middle direction)
//   kDiffRhs    R = (R + r_d t_d) / dx_0       (last direction of a plain RHS;
//                                               R = t_0 / dx_0 in 1D)
//   2, 3, 4     with s = R + r_d t_d (t_0 in 1D) and c = dt / dx_0:
//               2: U1 = Un + c s;  3: U2 = 3/4 Un + 1/4 U1 + 1/4 c s;
//               4: Un <- 1/3 Un + 2/3 U2 + 2/3 c s.
// ---------------------------------------------------------------------------
constexpr int kDiffFirst = 0, kDiffAcc = 1, kDiffRhs = 5;

// GRAV (last direction only): the body-force source of Sec. 4.3.2,
// S = (0, rho g, rho u.g), is added from the stage input Usrc.
template <int NDIM, int DIR, int MODE, bool GRAV = false>
__global__ void __launch_bounds__(256) diff_kernel(
    const double* __restrict__ Fhat, double* __restrict__ R,
    const double* Un, const double* Uk,   // not restrict: stage 3 writes Uout = Un in place
    double* Uout, const double* __restrict__ dt_ptr, Grid G, const double* Usrc) {
  constexpr bool stage = MODE >= 2 && MODE <= 4;
  constexpr bool acc = DIR > 0;   // R holds the earlier directions' sum
  constexpr int NVAR = NDIM + 2;
  const int64_t ncell = G.ncell;
  const int64_t m0 = G.n[0] + (DIR == 0), m1 = G.n[1] + (DIR == 1);
  const int64_t nifc = m0 * m1 * (G.n[2] + (DIR == 2));
  const double rd = G.rdx[DIR];
  // the interface fluxes are stored as kFluxScale F^: the last direction
  // divides by it together with dx_0
  const double idf = G.inv_dx[0] / kFluxScale;
  double c = 0.0;
  if (stage) {
    const double dt = *dt_ptr;
    if (!(dt > 0.0)) {
      // t >= t_end: the state is left unchanged.  The stage buffers U1, U2
      // take U^n, so that the stages after this one read defined values.
      if (MODE <= 3)
        for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < NVAR * ncell;
             e += (int64_t)gridDim.x * blockDim.x)
          Uout[e] = Un[e];
      return;
    }
    c = dt * idf;
  }
  // The interface left of cell c = (i2 n1 + i1) n0 + i0 is (i2 m1 + i1) m0 + i0:
  // x: c plus the row index c / n0 (one more interface per row); y: c plus
  // n0 times the plane index c / (n0 n1); z: c itself.
  const int64_t span = DIR == 0 ? G.n[0] : G.n[0] * G.n[1];
  const int64_t shift = DIR == 0 ? 1 : G.n[0];
  const bool narrow = ncell <= int64_t(UINT32_MAX);   // 32-bit division suffices
  for (int64_t cc = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cc < ncell;
       cc += (int64_t)gridDim.x * blockDim.x) {
    int64_t left = cc;
    if (DIR < 2) {
      const int64_t q = narrow ? int64_t(uint32_t(cc) / uint32_t(span)) : cc / span;
      left += q * shift;
    }
    const int64_t right = left + (DIR == 0 ? 1 : (DIR == 1 ? m0 : m0 * m1));
    // all loads of the cell first
    double s[NVAR];
#pragma unroll
    for (int v = 0; v < NVAR; ++v) s[v] = Fhat[v * nifc + left] - Fhat[v * nifc + right];
    if (acc)
#pragma unroll
      for (int v = 0; v < NVAR; ++v) s[v] = fma(rd, s[v], R[v * ncell + cc]);
    double src[NVAR];
    if (GRAV) {
      const double rho = Usrc[cc];
      double w = 0.0;
      src[0] = 0.0;
#pragma unroll
      for (int k = 0; k < NDIM; ++k) {
        src[1 + k] = rho * G.grav[k];
        w = fma(Usrc[(1 + k) * ncell + cc], G.grav[k], w);
      }
      src[NVAR - 1] = w;
      // L = s / (30 dx_0) + S: a stage takes c (s + 30 dx_0 S) with c = dt / (30 dx_0)
      if (stage)
#pragma unroll
        for (int v = 1; v < NVAR; ++v) s[v] = fma(kFluxScale * G.dx[0], src[v], s[v]);
    }
    if (MODE == kDiffFirst || MODE == kDiffAcc) {
#pragma unroll
      for (int v = 0; v < NVAR; ++v) R[v * ncell + cc] = s[v];
    } else if (MODE == kDiffRhs) {
#pragma unroll
      for (int v = 0; v < NVAR; ++v) R[v * ncell + cc] = GRAV ? fma(s[v], idf, src[v]) : s[v] * idf;
    } else {
      double o[NVAR];
#pragma unroll
      for (int v = 0; v < NVAR; ++v) o[v] = stage_value(MODE, c, s[v], Un, Uk, v * ncell + cc);
#pragma unroll
      for (int v = 0; v < NVAR; ++v) Uout[v * ncell + cc] = o[v];
    }
  }
}

// ---------------------------------------------------------------------------
// Time step (eq. dt1 / dt2; harmonic 3D form) from the LF speeds of U^n:
// max_i(|u_d| + c) = max(max|u_d - c|, max|u_d + c|).  Clipped to t_end - t.
// ---------------------------------------------------------------------------
template <int NDIM>
__global__ void dt_kernel(const unsigned long long* __restrict__ alpha_bits,
                          Grid G, double cfl, double dt_fixed, double* t_dev,
                          double t_end, double* dt_ws, double* dt_out) {
  const double* dx = G.dx;
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double smax[3];
#pragma unroll
  for (int d = 0; d < NDIM; ++d) {
    unsigned long long a = alpha_bits[d * 3 + 0], b = alpha_bits[d * 3 + 2];
    smax[d] = __longlong_as_double((long long)(a > b ? a : b));
  }
  double dt;
  if (dt_fixed > 0.0) {
    dt = dt_fixed;
  } else if (NDIM == 1) {
    dt = cfl * dx[0] / smax[0];
  } else if (NDIM == 2) {
    const double dtx = dx[0] / smax[0], dty = dx[1] / smax[1];
    dt = cfl * dtx * dty / (dtx + dty);
  } else {
    double acc = 0.0;
#pragma unroll
    for (int d = 0; d < NDIM; ++d) acc += smax[d] / dx[d];
    dt = cfl / acc;
  }
  const double t = *t_dev;
  const double rem = t_end - t;
  if (rem < dt) dt = rem;
  if (!(dt > 0.0)) dt = 0.0;
  *dt_ws = dt;
  if (dt_out) *dt_out = dt;
  *t_dev = t + dt;
}

// ---------------------------------------------------------------------------
// Scheme constants (host side)
// ---------------------------------------------------------------------------
Scheme make_scheme(double gamma, double H, double eps, int b_l, int b_u, int variant, int ct_m) {
  static const double kPow10Neg[16] = {1e-0, 1e-1, 1e-2,  1e-3,  1e-4,  1e-5,  1e-6,  1e-7,
                                       1e-8, 1e-9, 1e-10, 1e-11, 1e-12, 1e-13, 1e-14, 1e-15};
  Scheme S;
  std::memset(&S, 0, sizeof(S));
  S.variant = variant;
  S.m_fixed = ct_m;
  S.eps_a = kTeno5ACr * 0.9 / (1.0 - 0.9 * kTeno5ACr) * kTeno5AXi * kTeno5AXi;
  S.gamma = gamma;
  S.gm1 = gamma - 1.0;
  S.eps = eps;
  S.eps4 = 4.0 * eps;
  S.b_l = b_l;
  S.b_u = b_u;
  S.keep_all = 0;
  S.keep_idx = -1;
  if (variant == kSchemeLad) {
    const int K = b_u - b_l;
    S.nthr = K;
    S.top = 1;
    while (S.top * 2 <= K) S.top *= 2;
    // floor(theta K) >= j  <=>  max chi~ <= H (K/j - 1)   (eq. 3.1-3.2)
    for (int j = 1; j < K; ++j) S.thr[j - 1] = H * (double(K) / double(j) - 1.0);
    // theta == 1 in binary64  <=>  max chi~ / H <= 2^-53
    S.thr[K - 1] = H * 0x1p-53;
    // All stencils are kept whenever 3 (1 + max chi~)^6 C_T < 1 (then
    // chi_k >= gamma_min / (3 gamma_max) >= 1 / (3 (1 + max chi~)^6) > C_T); at
    // a given m, max chi~ <= thr[m - B_l - 1].  A relative margin of 1e-9 covers
    // the rounding of the threshold products.
    for (int c = 1; c <= K; ++c) {
      const int m = b_l + c;
      const double x = 1.0 + S.thr[c - 1];
      const double x6 = x * x * x * x * x * x;
      if (3.0 * x6 * kPow10Neg[m] <= 1.0 - 1e-9) S.keep_all |= 1u << m;
    }
    // the keep-all set is a suffix of B_l..B_u (the bound loosens as m grows)
    for (int c = 1; c <= K; ++c) {
      const unsigned suffix = ((1u << (b_u + 1)) - 1u) & ~((1u << (b_l + c)) - 1u);
      if (S.keep_all == suffix) {
        S.keep_idx = c - 1;
        break;
      }
    }
  } else if (variant == kSchemeTeno5 || variant == kSchemeTeno5A) {
    // The same bound with the largest C_T the scheme can take (TENO5: the
    // fixed one; TENO5-A: 1e-7): every stencil is kept when max chi~ <= thr
    // with 3 (1 + thr)^6 C_T <= 1 - 1e-9.
    const double ct = kPow10Neg[variant == kSchemeTeno5 ? ct_m : 7];
    double thr = std::pow(1.0 / (3.0 * ct), 1.0 / 6.0) - 1.0;
    for (int it = 0; it < 200 && thr > 0.0; ++it) {
      const double x = 1.0 + thr;
      if (3.0 * (x * x * x * x * x * x) * ct <= 1.0 - 1e-9) break;
      thr *= 1.0 - 1e-7;
    }
    if (thr > 0.0) {
      S.thr[0] = thr;
      S.keep_idx = 0;
    }
  }
  // (WENO-Z has no cutoff and no keep-all shortcut: keep_idx stays -1)
  // binary32 constants of the pre-test, rounded towards zero (conservative)
  auto down = [](double x) {
    float f = static_cast<float>(x);
    while (static_cast<double>(f) > x) f = std::nextafter(f, 0.0f);
    return std::nextafter(f, 0.0f);
  };
  // (the FP32 test's rounding analysis wants eps well inside the normal range;
  // thr_keep_f = 0 passes only all-zero stencils, which are kept exactly)
  S.eps4_f = down(4.0 * eps);
  S.thr_keep_f = (S.keep_idx >= 0 && 4.0 * eps >= 0x1p-100) ? down(S.thr[S.keep_idx]) : 0.0f;
  return S;
}

// ---------------------------------------------------------------------------
// Fixed-state ghost cells: one thread per face slot, the cell pass's formulas
// on the face states (kGhostSlots entries per field).
// ---------------------------------------------------------------------------
template <int NDIM>
__global__ void ghost_cell_kernel(GhostStates gs, unsigned mask, double* __restrict__ gU,
                                  double* __restrict__ gaux, double* __restrict__ gfh, double gamma,
                                  int* __restrict__ status) {
  constexpr int NVAR = NDIM + 2;
  const int slot = threadIdx.x;
  if (slot >= kGhostSlots || !((mask >> slot) & 1u)) return;
  double Uc[NVAR];
#pragma unroll
  for (int v = 0; v < NVAR; ++v) gU[v * kGhostSlots + slot] = Uc[v] = gs.U[slot][v];
  double uh[NDIM], cs, ep;
  if (!cell_primitives<NDIM>(gU, kGhostSlots, slot, gamma, gaux, uh, cs, ep) && status)
    atomicOr(status, kStatusNonphysical);
  store_flux_half<NDIM, 0>(Uc, uh, gaux[NDIM * kGhostSlots + slot], ep, gfh, kGhostSlots, slot);
}

cudaError_t launch_ghost_cells(int ndim, const GhostStates& gs, unsigned mask, const Grid& G, double gamma,
                               cudaStream_t st) {
  double* gU = const_cast<double*>(G.gU);
  double* gaux = const_cast<double*>(G.gaux);
  double* gfh = const_cast<double*>(G.gfh);
  switch (ndim) {
    case 1: ghost_cell_kernel<1><<<1, 32, 0, st>>>(gs, mask, gU, gaux, gfh, gamma, nullptr); break;
    case 2: ghost_cell_kernel<2><<<1, 32, 0, st>>>(gs, mask, gU, gaux, gfh, gamma, nullptr); break;
    default: ghost_cell_kernel<3><<<1, 32, 0, st>>>(gs, mask, gU, gaux, gfh, gamma, nullptr); break;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
static inline int blocks_for(int64_t n, int threads, int cap) {
  int64_t b = (n + threads - 1) / threads;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return static_cast<int>(b);
}

int cell_blocks(int64_t ncell, int nsm) { return blocks_for(ncell, 256, nsm * 8); }

cudaError_t launch_cell(int ndim, const double* U, double* aux, double* fh,
                        unsigned long long* alpha, int* status, int64_t ncell,
                        double gamma, int nsm, cudaStream_t st, unsigned long long* cand) {
  const int threads = 256;
  const int blocks = cell_blocks(ncell, nsm);
  if (cand) {
    switch (ndim) {
      case 1: cell_kernel<1, true><<<blocks, threads, 0, st>>>(U, aux, fh, alpha, status, ncell, gamma, cand); break;
      case 2: cell_kernel<2, true><<<blocks, threads, 0, st>>>(U, aux, fh, alpha, status, ncell, gamma, cand); break;
      default: cell_kernel<3, true><<<blocks, threads, 0, st>>>(U, aux, fh, alpha, status, ncell, gamma, cand); break;
    }
    return cudaGetLastError();
  }
  switch (ndim) {
    case 1: cell_kernel<1, false><<<blocks, threads, 0, st>>>(U, aux, fh, alpha, status, ncell, gamma, nullptr); break;
    case 2: cell_kernel<2, false><<<blocks, threads, 0, st>>>(U, aux, fh, alpha, status, ncell, gamma, nullptr); break;
    default: cell_kernel<3, false><<<blocks, threads, 0, st>>>(U, aux, fh, alpha, status, ncell, gamma, nullptr); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_argmax_finish(int ndim, const unsigned long long* cand, int64_t ncell, int nsm,
                                 unsigned long long* argidx, cudaStream_t st) {
  argmax_finish_kernel<<<1, kArgThreads, 0, st>>>(cand, cell_blocks(ncell, nsm), 3 * ndim, argidx);
  return cudaGetLastError();
}

template <int NDIM, int DIR>
static int flux_launch(int blocks, int threads, int pblocks, cudaStream_t st, const double* U,
                       const double* aux, const double* fh, const unsigned long long* alpha, double* Fhat,
                       uint8_t* flags, uint32_t* list, unsigned* count, int* status, const Grid& G,
                       const Scheme& S, double* roe_out) {
  const bool gh = G.bc[DIR] == TENO_BC_DIRICHLET;
  if (flags || !list) {
    if (flags && gh) flux_kernel<NDIM, DIR, true, true><<<blocks, threads, 0, st>>>(U, aux, alpha, Fhat, flags, status, G, S);
    else if (flags) flux_kernel<NDIM, DIR, true, false><<<blocks, threads, 0, st>>>(U, aux, alpha, Fhat, flags, status, G, S);
    else if (gh) flux_kernel<NDIM, DIR, false, true><<<blocks, threads, 0, st>>>(U, aux, alpha, Fhat, flags, status, G, S);
    else flux_kernel<NDIM, DIR, false, false><<<blocks, threads, 0, st>>>(U, aux, alpha, Fhat, flags, status, G, S);
    return 1;
  }
  if (G.bc[DIR] == TENO_BC_REFLECTIVE)
    flux_closed_kernel<NDIM, DIR, 1><<<blocks, threads, 0, st>>>(U, aux, fh, alpha, Fhat, list, count, status, G, S);
  else if (gh)
    flux_closed_kernel<NDIM, DIR, 2><<<blocks, threads, 0, st>>>(U, aux, fh, alpha, Fhat, list, count, status, G, S);
  else if (roe_out)
    flux_closed_kernel<NDIM, DIR, 0, true><<<blocks, threads, 0, st>>>(U, aux, fh, alpha, Fhat, list, count, status,
                                                                      G, S, roe_out);
  else
    flux_closed_kernel<NDIM, DIR, 0><<<blocks, threads, 0, st>>>(U, aux, fh, alpha, Fhat, list, count, status, G, S);
  if (gh)
    flux_pending_kernel<NDIM, DIR, true><<<pblocks, threads, 0, st>>>(U, aux, alpha, Fhat, list, count, status, G, S);
  else
    flux_pending_kernel<NDIM, DIR, false><<<pblocks, threads, 0, st>>>(U, aux, alpha, Fhat, list, count, status, G, S);
  return 2;
}

cudaError_t launch_flux(int ndim, int dir, const double* U, const double* aux, const double* fh,
                        const unsigned long long* alpha, double* Fhat,
                        uint8_t* flags, uint32_t* list, unsigned* count, int* status,
                        const Grid& G, const Scheme& S, int nsm, cudaStream_t st,
                        int* launches, double* roe_out) {
  int64_t nifc = 1;
  for (int k = 0; k < 3; ++k) nifc *= G.n[k] + (k == dir ? 1 : 0);
  if (nifc > int64_t(UINT32_MAX)) list = nullptr;   // list entries are 32-bit
  if (!count || !fh) list = nullptr;
  const int threads = 128;
  const int blocks = blocks_for(nifc, threads, nsm * 64);
  const int pblocks = blocks_for(nifc, threads, nsm * 16);
  int n = 0;
  if (ndim == 1) n = flux_launch<1, 0>(blocks, threads, pblocks, st, U, aux, fh, alpha, Fhat, flags, list, count, status, G, S, roe_out);
  else if (ndim == 2) {
    if (dir == 0) n = flux_launch<2, 0>(blocks, threads, pblocks, st, U, aux, fh, alpha, Fhat, flags, list, count, status, G, S, roe_out);
    else n = flux_launch<2, 1>(blocks, threads, pblocks, st, U, aux, fh, alpha, Fhat, flags, list, count, status, G, S, roe_out);
  } else {
    if (dir == 0) n = flux_launch<3, 0>(blocks, threads, pblocks, st, U, aux, fh, alpha, Fhat, flags, list, count, status, G, S, roe_out);
    else if (dir == 1) n = flux_launch<3, 1>(blocks, threads, pblocks, st, U, aux, fh, alpha, Fhat, flags, list, count, status, G, S, roe_out);
    else n = flux_launch<3, 2>(blocks, threads, pblocks, st, U, aux, fh, alpha, Fhat, flags, list, count, status, G, S, roe_out);
  }
  if (launches) *launches = n;
  return cudaGetLastError();
}

template <int NDIM, int DIR, bool GRAV>
static void diff_launch_last(int blocks, int threads, cudaStream_t st, const double* Fhat, double* R,
                             const double* Un, const double* Uk, double* Uout, const double* dt, const Grid& G,
                             int mode, const double* Usrc) {
  switch (mode) {
    case 0: diff_kernel<NDIM, DIR, kDiffRhs, GRAV><<<blocks, threads, 0, st>>>(Fhat, R, Un, Uk, Uout, dt, G, Usrc); break;
    case 2: diff_kernel<NDIM, DIR, 2, GRAV><<<blocks, threads, 0, st>>>(Fhat, R, Un, Uk, Uout, dt, G, Usrc); break;
    case 3: diff_kernel<NDIM, DIR, 3, GRAV><<<blocks, threads, 0, st>>>(Fhat, R, Un, Uk, Uout, dt, G, Usrc); break;
    default: diff_kernel<NDIM, DIR, 4, GRAV><<<blocks, threads, 0, st>>>(Fhat, R, Un, Uk, Uout, dt, G, Usrc); break;
  }
}

template <int NDIM, int DIR>
static void diff_launch(int blocks, int threads, cudaStream_t st, const double* Fhat,
                        double* R, const double* Un, const double* Uk, double* Uout,
                        const double* dt, const Grid& G, int mode, const double* Usrc) {
  // the first of several directions starts R; a middle one adds to it
  if (DIR < NDIM - 1) {
    if (DIR == 0) diff_kernel<NDIM, DIR, kDiffFirst><<<blocks, threads, 0, st>>>(Fhat, R, Un, Uk, Uout, dt, G, Usrc);
    else diff_kernel<NDIM, DIR, kDiffAcc><<<blocks, threads, 0, st>>>(Fhat, R, Un, Uk, Uout, dt, G, Usrc);
    return;
  }
  if (G.has_grav) diff_launch_last<NDIM, DIR, true>(blocks, threads, st, Fhat, R, Un, Uk, Uout, dt, G, mode, Usrc);
  else diff_launch_last<NDIM, DIR, false>(blocks, threads, st, Fhat, R, Un, Uk, Uout, dt, G, mode, Usrc);
}

cudaError_t launch_diff(int ndim, int dir, const double* Fhat, double* R,
                        const double* Un, const double* Uk, double* Uout,
                        const double* dt, const Grid& G, int mode,
                        int nsm, cudaStream_t st, const double* Usrc) {
  if (mode != 0 && (mode < 2 || mode > 4)) return cudaErrorInvalidValue;
  const int threads = 256;
  const int blocks = blocks_for(G.ncell, threads, nsm * 16);
  if (ndim == 1) diff_launch<1, 0>(blocks, threads, st, Fhat, R, Un, Uk, Uout, dt, G, mode, Usrc);
  else if (ndim == 2) {
    if (dir == 0) diff_launch<2, 0>(blocks, threads, st, Fhat, R, Un, Uk, Uout, dt, G, mode, Usrc);
    else diff_launch<2, 1>(blocks, threads, st, Fhat, R, Un, Uk, Uout, dt, G, mode, Usrc);
  } else {
    if (dir == 0) diff_launch<3, 0>(blocks, threads, st, Fhat, R, Un, Uk, Uout, dt, G, mode, Usrc);
    else if (dir == 1) diff_launch<3, 1>(blocks, threads, st, Fhat, R, Un, Uk, Uout, dt, G, mode, Usrc);
    else diff_launch<3, 2>(blocks, threads, st, Fhat, R, Un, Uk, Uout, dt, G, mode, Usrc);
  }
  return cudaGetLastError();
}

cudaError_t launch_dt(int ndim, const unsigned long long* alpha, const Grid& G,
                      double cfl, double dt_fixed, double* t_dev, double t_end,
                      double* dt_ws, double* dt_out, cudaStream_t st) {
  switch (ndim) {
    case 1: dt_kernel<1><<<1, 32, 0, st>>>(alpha, G, cfl, dt_fixed, t_dev, t_end, dt_ws, dt_out); break;
    case 2: dt_kernel<2><<<1, 32, 0, st>>>(alpha, G, cfl, dt_fixed, t_dev, t_end, dt_ws, dt_out); break;
    default: dt_kernel<3><<<1, 32, 0, st>>>(alpha, G, cfl, dt_fixed, t_dev, t_end, dt_ws, dt_out); break;
  }
  return cudaGetLastError();
}

teno_status forward_stage(const teno_grid* g, char* ws, size_t status_off, size_t dt_off,
                          size_t alpha_off, size_t aux_off, size_t fh_off, size_t fhat_off, size_t list_off,
                          const double* U, double* R, int mode, const double* Un, const double* Uk,
                          double* Uout, cudaStream_t st, unsigned long long* cand, double* roe_out,
                          size_t roe_stride) {
  Grid G;
  for (int k = 0; k < 3; ++k) {
    G.n[k] = g->n[k];
    G.bc[k] = k < g->ndim ? g->bc[k] : 0;
    G.dx[k] = k < g->ndim ? g->dx[k] : 1.0;
    G.inv_dx[k] = 1.0 / G.dx[k];
    G.rdx[k] = G.dx[0] / G.dx[k];
  }
  G.ncell = g->n[0] * g->n[1] * g->n[2];
  const Scheme S = scheme_of(g);
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0)
    nsm = 152;
  int* status = reinterpret_cast<int*>(ws + status_off);
  const double* dt = reinterpret_cast<const double*>(ws + dt_off);
  auto* alpha = reinterpret_cast<unsigned long long*>(ws + alpha_off);
  double* aux = reinterpret_cast<double*>(ws + aux_off);
  double* Fhat = reinterpret_cast<double*>(ws + fhat_off);
  uint32_t* list = list_off ? reinterpret_cast<uint32_t*>(ws + list_off) : nullptr;
  double* fh = fh_off ? reinterpret_cast<double*>(ws + fh_off) : nullptr;
  unsigned* count = reinterpret_cast<unsigned*>(ws + alpha_off + kPendingCountOffset);
  if (cudaMemsetAsync(alpha, 0, kAlphaAndCountBytes, st) != cudaSuccess) return TENO_ERR_CUDA;
  if (launch_cell(g->ndim, U, aux, fh, alpha, status, G.ncell, g->gamma, nsm, st, cand) != cudaSuccess)
    return TENO_ERR_CUDA;
  for (int d = 0; d < g->ndim; ++d) {
    if (launch_flux(g->ndim, d, U, aux, fh, alpha, Fhat, nullptr, list, count + d, status, G, S, nsm, st,
                    nullptr, roe_out ? roe_out + d * roe_stride : nullptr) != cudaSuccess)
      return TENO_ERR_CUDA;
    if (launch_diff(g->ndim, d, Fhat, R, Un, Uk, Uout, dt, G, mode, nsm, st, U) != cudaSuccess)
      return TENO_ERR_CUDA;
  }
  return TENO_OK;
}

}  // namespace teno
