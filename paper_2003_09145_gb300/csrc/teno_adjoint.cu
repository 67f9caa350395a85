// teno_adjoint.cu -- adjoint (vector-Jacobian product) of the TENO5-LAD Euler
// right-hand side and of one SSP-RK3 step.
//
// The stencil selections are frozen at their primal values: the cutoff of
// eq. 2.14 is piecewise constant, so with delta fixed the reconstruction is
// linear and L(U) is differentiable almost everywhere.  The global
// Lax-Friedrichs speed alpha_{d,s} = max_cells |lambda_s| is differentiated
// through its arg-max cell (lowest linear index on ties), which the cell
// pass finds along with the maximum.
//
// One right-hand-side adjoint (adjoint_sequence):
//   cell pass        : primitives, speeds and their arg-max cells (skipped
//                      where the recomputed forward stage already made them);
//   per direction d:
//     adj_kept_kernel  : one thread per interface: the forward pass's certified
//                        FP32 test; where it keeps every stencil, the
//                        closed-form interface VJP (teno_adjoint_core.cuh)
//                        with Fbar from Rbar (eq. 2.2): U~bar and the adjoints
//                        of the two Roe cells' parameters go to kb_d; the
//                        rest is marked pending;
//     list passes      : the pending interfaces in one list, index order;
//     adj_select_kernel: the listed interfaces' selections by the forward
//                        pass's binary64 decisions;
//     partition passes : the list reordered stably, the interfaces that keep
//                        every stencil after all first;
//     adj_general_kernel: the listed interfaces' VJP with those selections
//                        (the closed form for the first kind); the six
//                        cells' contributions go to contrib_d;
// (teno_rk3_step_adjoint runs three of these after recomputing the stages
// U1, U2; teno_rk3_step_adjoint_staged takes the stages from the caller.)
//   adj_gather_kernel: one thread per cell sums, over every direction, the
//                      contributions of every (interface, stencil slot) that
//                      maps to it (boundary ghost copies included) and applies
//                      the per-cell maps once: A_d(U_c)^T to the P-weighted
//                      Fbar of each direction, the Roe-parameter map to the
//                      summed parameter adjoints -- deterministic, no atomics;
//                      it writes out = a X + b Y + (the adjoint);
//   adj_alpha_kernel : sums the per-block d/dalpha in a fixed order and adds
//                      the alpha terms at the arg-max cells.
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

// The adjoint's six-point sums with integer weights in 64-bit fixed point
// (teno_fixsum.cuh, as in the forward's closed form): bit 1 the stencil on
// Rbar (weights 1, -9, 45 on the differences), bit 2 the M-weighted U~bar of
// the slots, bit 4 the kept pass's 60 U~ (from stored Roe states).  A
// component the fixed point does not cover takes the binary64 form.  A
// tuning choice between the FP64 and integer pipes; measured on the 256^3
// reverse RK3 step (ms): none 102.4, bit 1 100.9-101.1 (this default), bit
// 4 101.5, bits 1 and 4 100.0, bits 1 and 2 114.7 (the M sums' seven loads
// per component spill and the integer chains then bound the gather).  Bit 4
// is left off: the kept pass without stored states (the staged reverse
// step's) sums U~ as a binary64 chain, and the two reverse steps agree bit
// for bit only if both do.
#ifndef TENO_ADJ_FIX_MASK
#define TENO_ADJ_FIX_MASK 1
#endif
constexpr unsigned kAdjFixMask = TENO_ADJ_FIX_MASK;

// Geometry of interface q of direction DIR: its index id along DIR, the
// linear index of its line's cell 0 and the six stencil cells (ghosts mapped).
template <int NDIM, int DIR>
struct IfcGeom {
  int64_t m0, m1, nifc, ncell, stride_d, nd;
  int bcd;
  __device__ explicit IfcGeom(const Grid& G)
      : m0(G.n[0] + (DIR == 0)), m1(G.n[1] + (DIR == 1)),
        nifc((G.n[0] + (DIR == 0)) * (G.n[1] + (DIR == 1)) * (G.n[2] + (DIR == 2))), ncell(G.ncell),
        stride_d((DIR == 0) ? 1 : (DIR == 1 ? G.n[0] : G.n[0] * G.n[1])), nd(G.n[DIR]), bcd(G.bc[DIR]) {}
  __device__ void locate(int64_t q, const Grid& G, int64_t& id, int64_t& base, int64_t (&cells)[6]) const {
    const int64_t i0 = q % m0;
    const int64_t r = q / m0;
    const int64_t i1 = r % m1;
    const int64_t i2 = r / m1;
    id = (DIR == 0) ? i0 : (DIR == 1 ? i1 : i2);
    base = (DIR == 0) ? (i2 * G.n[1] + i1) * G.n[0] : (DIR == 1) ? i2 * G.n[1] * G.n[0] + i0 : i1 * G.n[0] + i0;
#pragma unroll
    for (int j = 0; j < 6; ++j) cells[j] = base + teno::ghost(id - 3 + j, nd, bcd) * stride_d;
  }
};

// The three distinct LF speeds of direction DIR per field: fa = alpha,
// ha = alpha / 2, nfa = -alpha (the forward pass's arguments).
template <int NDIM, int DIR>
__device__ __forceinline__ void field_speeds(const unsigned long long* __restrict__ alpha_bits,
                                             double (&fa)[NDIM + 2], double (&ha)[NDIM + 2],
                                             double (&nfa)[NDIM + 2]) {
  constexpr int NVAR = NDIM + 2;
  const double am = __longlong_as_double((long long)alpha_bits[DIR * 3 + 0]);
  const double a0 = __longlong_as_double((long long)alpha_bits[DIR * 3 + 1]);
  const double ap = __longlong_as_double((long long)alpha_bits[DIR * 3 + 2]);
  fa[0] = am;
#pragma unroll
  for (int f = 1; f < NVAR - 1; ++f) fa[f] = a0;
  fa[NVAR - 1] = ap;
#pragma unroll
  for (int f = 0; f < NVAR; ++f) {
    ha[f] = 0.5 * fa[f];
    nfa[f] = -2.0 * ha[f];
  }
}

// Fbar of interface id of a line: R_c = -(F^_{c+1/2} - F^_{c-1/2})/dx gives
// dJ/dF^_id = (Rbar_id [id < n] - Rbar_{id-1} [id >= 1]) / dx (eq. 2.2);
// without fscale the bracket alone.
template <int NVAR>
__device__ __forceinline__ void interface_fbar(const double* __restrict__ Rbar, int64_t ncell, int64_t base,
                                               int64_t id, int64_t nd, int64_t stride_d, double (&Fb)[NVAR]) {
#pragma unroll
  for (int v = 0; v < NVAR; ++v) {
    const double ra = id < nd ? Rbar[v * ncell + base + id * stride_d] : 0.0;
    const double rb = id >= 1 ? Rbar[v * ncell + base + (id - 1) * stride_d] : 0.0;
    Fb[v] = ra - rb;
  }
}
template <int NVAR>
__device__ __forceinline__ void interface_fbar(const double* __restrict__ Rbar, int64_t ncell, int64_t base,
                                               int64_t id, int64_t nd, int64_t stride_d, double fscale,
                                               double (&Fb)[NVAR]) {
  interface_fbar<NVAR>(Rbar, ncell, base, id, nd, stride_d, Fb);
#pragma unroll
  for (int v = 0; v < NVAR; ++v) Fb[v] *= fscale;
}

// Block sum of asum in a fixed order into apart[blockIdx.x].
__device__ __forceinline__ void block_alpha_sum(const double (&asum)[3], double* __restrict__ apart) {
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

template <int NVAR>
__device__ __forceinline__ void add_alpha(const double (&ab)[NVAR], double (&asum)[3]) {
  asum[0] += ab[0];
#pragma unroll
  for (int f = 1; f < NVAR - 1; ++f) asum[1] += ab[f];
  asum[2] += ab[NVAR - 1];
}

// One thread per interface: the forward pass's certified FP32 test (the
// same device code teno_rhs / teno_rk3_step run).  Where it keeps every
// stencil, the interface part of the closed-form VJP: U~bar and the
// adjoints of the Roe parameters of cells i and i+1 go to kb[3 nvar][nifc]
// (the flux Jacobians and the Roe-parameter maps are applied per cell by the
// gather); elsewhere the interface is marked pending for adj_general_kernel.
#ifndef TENO_ADJ_KEPT_MINBLOCKS
#define TENO_ADJ_KEPT_MINBLOCKS 3   // 168 registers: 12 warps per SM
#endif
template <int NDIM, int DIR, bool STORED>
__global__ void __launch_bounds__(kAdjThreads, TENO_ADJ_KEPT_MINBLOCKS) adj_kept_kernel(
    const double* __restrict__ U, const double* __restrict__ aux,
    const unsigned long long* __restrict__ alpha_bits, const double* __restrict__ Rbar, double scale,
    double* __restrict__ kb, unsigned char* __restrict__ pending, double* __restrict__ apart,
    int* __restrict__ status, Grid G, Scheme S, const double* __restrict__ roe_in) {
  constexpr int NVAR = NDIM + 2;
  const IfcGeom<NDIM, DIR> I(G);
  double fa[NVAR], ha[NVAR], nfa[NVAR];
  field_speeds<NDIM, DIR>(alpha_bits, fa, ha, nfa);
  // kept_roe_scaled's inputs: 60 U~ in integer weights, Fbar without the
  // factor scale / dx (carried by the speeds instead); its ab come out times
  // 60 dx / scale, which adj_alpha_kernel divides out of the block sums
  const double fscale = scale * G.inv_dx[DIR];
  const double Mi[6] = {1.0, -5.0, 10.0, -10.0, 5.0, -1.0};
  const double amid = fscale * fa[1], d0 = fscale * (fa[0] - fa[1]), dE = fscale * (fa[NVAR - 1] - fa[1]);
  const double igm1 = 1.0 / (S.gamma - 1.0);
  double asum[3] = {0.0, 0.0, 0.0};
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < I.nifc;
       q += (int64_t)gridDim.x * blockDim.x) {
    int64_t id, base, cells[6];
    I.locate(q, G, id, base, cells);
    // The forward pass's Roe state (roe_interface on the cell pass's
    // primitives) and its certified FP32 test: a pass keeps every stencil
    // exactly where the forward's closed-form pass did.  U~ is accumulated
    // over the same stencil loads.  With STORED the recomputed forward
    // stage's closed-form pass has stored both (roe_in), so neither is
    // evaluated again.
    const double sr2 = aux[(NDIM + 1) * I.ncell + cells[2]], sr3 = aux[(NDIM + 1) * I.ncell + cells[3]];
    const double sh2 = aux[(NDIM + 2) * I.ncell + cells[2]], sh3 = aux[(NDIM + 2) * I.ncell + cells[3]];
    teno::RoeIfc<NDIM> Rf;
    double Ut[NVAR];
    bool kept;
    if constexpr (STORED) {
      kept = roe_in[(int64_t)(NDIM + 7) * I.nifc + q] != 0.0;
    } else {
      double su2[NDIM], su3[NDIM];
#pragma unroll
      for (int k = 0; k < NDIM; ++k) {
        su2[k] = aux[(NDIM + 3 + k) * I.ncell + cells[2]];
        su3[k] = aux[(NDIM + 3 + k) * I.ncell + cells[3]];
      }
      teno::roe_interface<NDIM, DIR>(sr2, sr3, sh2, sh3, su2, su3, S, Rf, status);
      teno::CertIfc<NDIM> C;
      teno::cert_begin<NDIM, DIR>(Rf, ha, C);
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        double Uj[NVAR];
#pragma unroll
        for (int v = 0; v < NVAR; ++v) {
          Uj[v] = U[v * I.ncell + cells[j]];
          Ut[v] = j == 0 ? Uj[v] : (j == 5 ? Ut[v] - Uj[v] : fma(Mi[j], Uj[v], Ut[v]));
        }
        teno::cert_point<NDIM, DIR>(j, Uj, aux[DIR * I.ncell + cells[j]], aux[NDIM * I.ncell + cells[j]], C);
      }
      kept = S.keep_idx >= 0 && teno::cert_keep<NDIM>(C, S);
    }
    pending[q] = kept ? 0 : 1;
    if (!kept) {
      // a pending interface's terms come from adj_general_kernel; zeros
      // here let the gather add kb for every interface alike
#pragma unroll
      for (int v = 0; v < 3 * NVAR; ++v) kb[(int64_t)v * I.nifc + q] = 0.0;
      continue;
    }
    if constexpr (STORED) {
#pragma unroll
      for (int k = 0; k < NDIM; ++k) Rf.u[k] = roe_in[(int64_t)k * I.nifc + q];
      Rf.q2 = roe_in[(int64_t)(NDIM + 0) * I.nifc + q];
      Rf.H = roe_in[(int64_t)(NDIM + 1) * I.nifc + q];
      Rf.cs = roe_in[(int64_t)(NDIM + 2) * I.nifc + q];
      Rf.b1 = roe_in[(int64_t)(NDIM + 3) * I.nifc + q];
      Rf.hb1 = roe_in[(int64_t)(NDIM + 4) * I.nifc + q];
      Rf.hb2 = roe_in[(int64_t)(NDIM + 5) * I.nifc + q];
      Rf.hic = roe_in[(int64_t)(NDIM + 6) * I.nifc + q];
#pragma unroll
      for (int v = 0; v < NVAR; ++v) {
        double us[6];
#pragma unroll
        for (int j = 0; j < 6; ++j) us[j] = U[v * I.ncell + cells[j]];
        const int mw[6] = {1, -5, 10, -10, 5, -1};
        if (!(kAdjFixMask & 4u) || !teno_fix::sum<6>(us, mw, Ut[v])) {
          Ut[v] = us[0];
#pragma unroll
          for (int j = 1; j < 5; ++j) Ut[v] = fma(Mi[j], us[j], Ut[v]);
          Ut[v] -= us[5];
        }
      }
    }
    // the VJP's Roe state: the same average, and the cells' velocity and
    // enthalpy differences
    teno_adj::RoeState<NDIM> R;
    R.sa = sr2;
    R.sb = sr3;
    R.iS = teno::recip_pos(sr2 + sr3);
    R.dH = sh2 * teno::recip_pos(sr2) - sh3 * teno::recip_pos(sr3);
#pragma unroll
    for (int k = 0; k < NDIM; ++k) {
      R.duh[k] = aux[k * I.ncell + cells[2]] - aux[k * I.ncell + cells[3]];
      R.ut[k] = Rf.u[k];
    }
    R.q2 = Rf.q2;
    R.H = Rf.H;
    R.c = Rf.cs;
    R.b1 = Rf.b1;
    R.hb1 = Rf.hb1;
    R.hb2 = Rf.hb2;
    R.hic = Rf.hic;
    R.b1ic2 = (Rf.b1 * Rf.b1) * igm1;   // b1 / c^2 = b1^2 / (gamma - 1)
    double Fb[NVAR];
    interface_fbar<NVAR>(Rbar, I.ncell, base, id, I.nd, I.stride_d, Fb);
    double Utb[NVAR], pa[NVAR], pb[NVAR], ab[NVAR];
    teno_adj::kept_roe_scaled<NDIM, DIR>(R, Ut, amid, d0, dE, R.iS * (1.0 / 60.0), S.gamma, Fb, Utb, pa, pb, ab);
#pragma unroll
    for (int v = 0; v < NVAR; ++v) {
      kb[(int64_t)v * I.nifc + q] = Utb[v];
      kb[(int64_t)(NVAR + v) * I.nifc + q] = pa[v];
      kb[(int64_t)(2 * NVAR + v) * I.nifc + q] = pb[v];
    }
    // the closed form's d/dalpha: the middle speeds' whole derivative in ab[1]
    asum[0] += ab[0];
    asum[1] += ab[1];
    asum[2] += ab[NVAR - 1];
  }
  block_alpha_sum(asum, apart);
}

// The pending interfaces (those the kept kernel's certified test leaves
// undecided) are gathered into one list ordered by interface index, so that
// the general VJP runs on full warps: on the turbulence box they are a few
// per ten thousand, and a warp with one active lane pays the FP64 pipe's full
// cost per instruction.  Three small passes build the list:
//   adj_count_kernel   : block b counts the pending interfaces of its fixed,
//                        contiguous range of 32-interface chunks;
//   adj_scan_kernel    : one block turns the nblk counts into offsets and the
//                        total;
//   adj_scatter_kernel : block b writes its pending interfaces, in index
//                        order, from its offset on.
// The list order depends only on the data, so the general kernel's d/dalpha
// sums (per thread in list order, then per block) are deterministic.
constexpr int kListThreads = 256;

__device__ __forceinline__ void chunk_range(int64_t nchunk, int64_t& c0, int64_t& c1) {
  const int64_t per = (nchunk + gridDim.x - 1) / gridDim.x;
  c0 = (int64_t)blockIdx.x * per;
  c1 = c0 + per < nchunk ? c0 + per : nchunk;
}

__global__ void __launch_bounds__(kListThreads) adj_count_kernel(const unsigned char* __restrict__ pending,
                                                                  int64_t nifc, int* __restrict__ bcount) {
  __shared__ int wsum[kListThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int64_t c0, c1;
  chunk_range((nifc + 31) / 32, c0, c1);
  int cnt = 0;
  for (int64_t c = c0 + wid; c < c1; c += kListThreads / 32) {
    const int64_t q = c * 32 + lane;
    cnt += __popc(__ballot_sync(0xffffffffu, q < nifc && pending[q] != 0));
  }
  if (lane == 0) wsum[wid] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < kListThreads / 32; ++w) t += wsum[w];
    bcount[blockIdx.x] = t;
  }
}

// exclusive offsets boff[b] = sum_{b' < b} bcount[b'] and the total, one
// block of kListThreads (nblk <= 8 kListThreads: eight entries per thread)
__global__ void __launch_bounds__(kListThreads) adj_scan_kernel(const int* __restrict__ bcount, int nblk,
                                                                 int* __restrict__ boff, int* __restrict__ total) {
  __shared__ int wsum[kListThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int v[8], s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int b = threadIdx.x * 8 + k;
    v[k] = b < nblk ? bcount[b] : 0;
    s += v[k];
  }
  int inc = s;   // inclusive scan of the per-thread sums within the warp
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) wsum[wid] = inc;
  __syncthreads();
  int base = 0;
  for (int w = 0; w < wid; ++w) base += wsum[w];
  int run = base + inc - s;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int b = threadIdx.x * 8 + k;
    if (b < nblk) boff[b] = run;
    run += v[k];
  }
  if (threadIdx.x == kListThreads - 1) *total = run;
}

__global__ void __launch_bounds__(kListThreads) adj_scatter_kernel(const unsigned char* __restrict__ pending,
                                                                    int64_t nifc, const int* __restrict__ boff,
                                                                    uint32_t* __restrict__ list) {
  __shared__ int wcnt[kListThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int64_t c0, c1;
  chunk_range((nifc + 31) / 32, c0, c1);
  int run = boff[blockIdx.x];
  for (int64_t cb = c0; cb < c1; cb += kListThreads / 32) {
    const int64_t c = cb + wid;
    const int64_t q = c * 32 + lane;
    const bool p = c < c1 && q < nifc && pending[q] != 0;
    const unsigned m = __ballot_sync(0xffffffffu, p);
    if (lane == 0) wcnt[wid] = __popc(m);
    __syncthreads();
    int before = 0, all = 0;
    for (int w = 0; w < kListThreads / 32; ++w) {
      before += w < wid ? wcnt[w] : 0;
      all += wcnt[w];
    }
    if (p) list[run + before + __popc(m & ((1u << lane) - 1u))] = static_cast<uint32_t>(q);
    run += all;
    __syncthreads();
  }
}

// A stable two-way partition of the list by the selections: the interfaces
// that keep every stencil after all (the certificate is conservative) first,
// in list order, then the others -- so that each kind of VJP runs on full
// warps.  The length n is read on the device; block b takes its fixed,
// contiguous range of 32-entry chunks, as in the list passes above.
//   adj_part_count_kernel  : block b counts its all-kept entries;
//   adj_scan_kernel        : their offsets and total nA;
//   adj_part_scatter_kernel: all-kept entry k of block b goes to boff[b] + k,
//                            other entry k to nA + (first index of b - boff[b]) + k.
__device__ __forceinline__ bool all_kept_sel(uint32_t w, int nvar) { return w == (1u << (6 * nvar)) - 1u; }

__global__ void __launch_bounds__(kListThreads) adj_part_count_kernel(const uint32_t* __restrict__ sel,
                                                                       const int* __restrict__ count, int nvar,
                                                                       int* __restrict__ bcount) {
  __shared__ int wsum[kListThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t n = *count;
  int64_t c0, c1;
  chunk_range((n + 31) / 32, c0, c1);
  int cnt = 0;
  for (int64_t c = c0 + wid; c < c1; c += kListThreads / 32) {
    const int64_t i = c * 32 + lane;
    cnt += __popc(__ballot_sync(0xffffffffu, i < n && all_kept_sel(sel[i], nvar)));
  }
  if (lane == 0) wsum[wid] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < kListThreads / 32; ++w) t += wsum[w];
    bcount[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(kListThreads) adj_part_scatter_kernel(
    const uint32_t* __restrict__ list, const uint32_t* __restrict__ sel, const int* __restrict__ count, int nvar,
    const int* __restrict__ boff, const int* __restrict__ nkept, uint32_t* __restrict__ list2,
    uint32_t* __restrict__ sel2) {
  __shared__ int wa[kListThreads / 32], wg[kListThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t n = *count;
  const int64_t nA = *nkept;
  int64_t c0, c1;
  chunk_range((n + 31) / 32, c0, c1);
  int64_t runA = boff[blockIdx.x];
  int64_t runG = nA + c0 * 32 - runA;
  for (int64_t cb = c0; cb < c1; cb += kListThreads / 32) {
    const int64_t c = cb + wid;
    const int64_t i = c * 32 + lane;
    const bool in = c < c1 && i < n;
    const uint32_t w = in ? sel[i] : 0u;
    const bool a = in && all_kept_sel(w, nvar);
    const bool g = in && !a;
    const unsigned ma = __ballot_sync(0xffffffffu, a), mg = __ballot_sync(0xffffffffu, g);
    if (lane == 0) {
      wa[wid] = __popc(ma);
      wg[wid] = __popc(mg);
    }
    __syncthreads();
    int ba = 0, bg = 0, ta = 0, tg = 0;
    for (int k = 0; k < kListThreads / 32; ++k) {
      ba += k < wid ? wa[k] : 0;
      bg += k < wid ? wg[k] : 0;
      ta += wa[k];
      tg += wg[k];
    }
    const unsigned below = (1u << lane) - 1u;
    if (a) {
      const int64_t pos = runA + ba + __popc(ma & below);
      list2[pos] = list[i];
      sel2[pos] = w;
    } else if (g) {
      const int64_t pos = runG + bg + __popc(mg & below);
      list2[pos] = list[i];
      sel2[pos] = w;
    }
    runA += ta;
    runG += tg;
    __syncthreads();
  }
}

// The listed interfaces in two passes, so that the VJP runs on full warps
// (the forward's cutoff decisions branch per field and lane; the VJP with
// the selections fixed does not branch):
//   adj_select_kernel: one thread per listed interface: the characteristic
//                      path of the forward pass (the same binary64 decisions
//                      its pending pass takes on these very interfaces, as the
//                      kept pass ran the forward's certificate) -> the ten
//                      3-bit selections packed into sel[i];
//   partition passes  : the list reordered, those that keep every stencil
//                      after all first (below);
//   adj_general_kernel: one thread per listed interface: the closed-form VJP
//                      for the first kind, the general VJP with the
//                      selections for the rest; the six cells' contributions,
//                      less the all-kept flux term P_j A(U_j)^T Fbar that the
//                      gather adds for every interface, go to
//                      contrib[6 nvar][nifc].
template <int NDIM, int DIR>
__global__ void __launch_bounds__(kAdjThreads) adj_select_kernel(
    const double* __restrict__ U, const double* __restrict__ aux,
    const unsigned long long* __restrict__ alpha_bits, const uint32_t* __restrict__ list,
    const int* __restrict__ count, uint32_t* __restrict__ sel, int* __restrict__ status, Grid G, Scheme S) {
  constexpr int NVAR = NDIM + 2;
  const IfcGeom<NDIM, DIR> I(G);
  double fa[NVAR], ha[NVAR], nfa[NVAR];
  field_speeds<NDIM, DIR>(alpha_bits, fa, ha, nfa);
  const int64_t n = *count;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = list[i];
    int64_t id, base, cells[6];
    I.locate(q, G, id, base, cells);
    double fout[NVAR];
    unsigned fl[NVAR][2];
    teno::interface_flux<NDIM, DIR, false, teno::kFluxChar>(U, aux, I.ncell, cells, 0u, ha, nfa, S, fout, fl,
                                                            status);
    uint32_t w = 0;
#pragma unroll
    for (int f = 0; f < NVAR; ++f) w |= ((fl[f][0] & 7u) | ((fl[f][1] & 7u) << 3)) << (6 * f);
    sel[i] = w;
  }
}

template <int NDIM, int DIR>
__global__ void __launch_bounds__(kAdjThreads) adj_general_kernel(
    const double* __restrict__ U, const unsigned long long* __restrict__ alpha_bits,
    const double* __restrict__ Rbar, double scale, double* __restrict__ contrib,
    const uint32_t* __restrict__ list, const int* __restrict__ count, const int* __restrict__ nkept,
    const uint32_t* __restrict__ selw, double* __restrict__ apart, Grid G, Scheme S) {
  constexpr int NVAR = NDIM + 2;
  const IfcGeom<NDIM, DIR> I(G);
  double fa[NVAR], ha[NVAR], nfa[NVAR];
  field_speeds<NDIM, DIR>(alpha_bits, fa, ha, nfa);
  const double fscale = scale * G.inv_dx[DIR];
  double asum[3] = {0.0, 0.0, 0.0};
  const int64_t n = *count, nA = *nkept;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = list[i];
    int64_t id, base, cells[6];
    I.locate(q, G, id, base, cells);
    const uint32_t w = selw[i];
    unsigned sel[NVAR][2];
#pragma unroll
    for (int f = 0; f < NVAR; ++f) {
      sel[f][0] = (w >> (6 * f)) & 7u;
      sel[f][1] = (w >> (6 * f + 3)) & 7u;
    }
    double Up[6][NVAR];
#pragma unroll
    for (int j = 0; j < 6; ++j)
#pragma unroll
      for (int v = 0; v < NVAR; ++v) Up[j][v] = U[v * I.ncell + cells[j]];
    double Fb[NVAR];
    interface_fbar<NVAR>(Rbar, I.ncell, base, id, I.nd, I.stride_d, fscale, Fb);
    double Ub[6][NVAR], ab[NVAR];
    if (i < nA)   // the partition puts the all-kept interfaces first
      teno_adj::interface_vjp_kept<NDIM, DIR, true>(Up, fa, S.gamma, Fb, Ub, ab);
    else
      teno_adj::interface_vjp<NDIM, DIR, true>(Up, fa, sel, S.gamma, Fb, Ub, ab);
#pragma unroll
    for (int j = 0; j < 6; ++j)
#pragma unroll
      for (int v = 0; v < NVAR; ++v) contrib[(int64_t)(j * NVAR + v) * I.nifc + q] = Ub[j][v];
    add_alpha<NVAR>(ab, asum);
  }
  block_alpha_sum(asum, apart);
}

// The all-kept weights of the stencil points: P for F~ = sum_j P_j F_j and M
// for U~ = sum_j M_j U_j (indexed by a warp-uniform slot number).
__constant__ double c_adjP[6] = {1.0 / 60.0, -8.0 / 60.0, 37.0 / 60.0, 37.0 / 60.0, -8.0 / 60.0, 1.0 / 60.0};
__constant__ double c_adjM[6] = {1.0 / 60.0, -5.0 / 60.0, 10.0 / 60.0, -10.0 / 60.0, 5.0 / 60.0, -1.0 / 60.0};
__constant__ int c_adjMi[6] = {1, -5, 10, -10, 5, -1};


// What the gather reads per direction, and its output.
struct GatherArgs {
  const double* kb[3];              // [3 nvar][nifc_d]: U~bar, Roe-parameter adjoints of cells i, i+1 (0 if pending)
  const double* contrib[3];         // [6 nvar][nifc_d]: the pending interfaces' contributions, flux term excluded
  const unsigned char* pending[3];  // [nifc_d]
  double fscale[3];                 // scale / dx_d
  double* out;                      // out = a X + b Y + the adjoint (X, Y nullable; out may be X or Y)
  const double* X;
  const double* Y;
  double a, b;
};

// Every interface's share at the cell its slot j maps to: M_j U~bar_q into
// acc and its Roe-parameter adjoints (j = 2: cell i, j = 3: cell i+1) into
// rp (both zero for a pending interface), and for a pending one its own
// contribution into acc.
// (slot_rest: the same without the M_j U~bar term, which the stencil path
// sums in fixed point.)
template <int NVAR>
__device__ __forceinline__ void slot_rest(int j, int64_t q, const double* __restrict__ kb,
                                          const double* __restrict__ contrib,
                                          const unsigned char* __restrict__ pending, int64_t nifc,
                                          double (&acc)[NVAR], double (&rp)[NVAR]) {
  if (j == 2)
#pragma unroll
    for (int v = 0; v < NVAR; ++v) rp[v] += kb[(int64_t)(NVAR + v) * nifc + q];
  if (j == 3)
#pragma unroll
    for (int v = 0; v < NVAR; ++v) rp[v] += kb[(int64_t)(2 * NVAR + v) * nifc + q];
  if (pending[q])
#pragma unroll
    for (int v = 0; v < NVAR; ++v) acc[v] += contrib[(int64_t)(j * NVAR + v) * nifc + q];
}

template <int NVAR>
__device__ __forceinline__ void slot_terms(int j, int64_t q, const double* __restrict__ kb,
                                           const double* __restrict__ contrib,
                                           const unsigned char* __restrict__ pending, int64_t nifc,
                                           double (&acc)[NVAR], double (&rp)[NVAR]) {
  const double Mj = c_adjM[j];
#pragma unroll
  for (int v = 0; v < NVAR; ++v) acc[v] = fma(Mj, kb[(int64_t)v * nifc + q], acc[v]);
  if (j == 2)
#pragma unroll
    for (int v = 0; v < NVAR; ++v) rp[v] += kb[(int64_t)(NVAR + v) * nifc + q];
  if (j == 3)
#pragma unroll
    for (int v = 0; v < NVAR; ++v) rp[v] += kb[(int64_t)(2 * NVAR + v) * nifc + q];
  if (pending[q])
#pragma unroll
    for (int v = 0; v < NVAR; ++v) acc[v] += contrib[(int64_t)(j * NVAR + v) * nifc + q];
}

// The cells the stencil form does not cover (transmissive ends, periodic
// lines shorter than six cells): every (interface qd, slot j) whose point j,
// ghost(qd - 3 + j), is cell id, slot by slot, with fs P_j Fbar_qd into Fsum.
// Out of line: rare, and the hot loop's code stays small.
template <int NVAR>
__device__ __noinline__ void gather_edge(int idl, int ndl, int bc, int64_t q0, int64_t sd, int64_t line,
                                         int64_t cstride, int64_t ncell, int64_t nifc, double fs,
                                         const double* __restrict__ Rbar, const double* __restrict__ kb,
                                         const double* __restrict__ contrib,
                                         const unsigned char* __restrict__ pending, double (&acc)[NVAR],
                                         double (&rp)[NVAR], double (&Fsum)[NVAR]) {
  for (int j = 0; j < 6; ++j) {
    int lo, hi, step;
    if (bc == 0) {
      // x = qd - 3 + j ranges over [j - 3, nd + j - 3]; x = id (mod nd)
      int x = idl;
      while (x - ndl >= j - 3) x -= ndl;
      while (x < j - 3) x += ndl;
      lo = x + 3 - j;
      hi = ndl;
      step = ndl;
    } else {
      // transmissive: points below 0 map to cell 0, points above nd-1 to nd-1
      lo = idl + 3 - j;
      hi = idl + 3 - j;
      if (idl == 0) lo = 0;
      if (idl == ndl - 1) hi = ndl;
      if (lo < 0) lo = 0;
      if (hi > ndl) hi = ndl;
      step = 1;
    }
    for (int qd = lo; qd <= hi; qd += step) {
      if (bc != 0) {
        const int x = qd - 3 + j;
        const int mapped = x < 0 ? 0 : (x >= ndl ? ndl - 1 : x);
        if (mapped != idl) continue;
      }
      const int64_t q = q0 + (int64_t)qd * sd;
      const double Pj = c_adjP[j] * fs;
#pragma unroll
      for (int v = 0; v < NVAR; ++v) {
        const double ra = (qd < ndl) ? Rbar[v * ncell + line + (int64_t)qd * cstride] : 0.0;
        const double rb = (qd >= 1) ? Rbar[v * ncell + line + (int64_t)(qd - 1) * cstride] : 0.0;
        Fsum[v] = fma(Pj, ra - rb, Fsum[v]);
      }
      slot_terms<NVAR>(j, q, kb, contrib, pending, nifc, acc, rp);
    }
  }
}

// Direction DIR's share at cell c (indices i0, i1, i2): acc += the M-weighted
// U~bar and the pending contributions, rp += the Roe-parameter adjoints,
// and acc += A_DIR(U_c)^T applied to the fs P-weighted Fbar sum.
template <int NDIM, int DIR>
__device__ __forceinline__ void gather_dir(const Grid& G, int64_t c, int64_t i0, int64_t i1, int64_t i2,
                                           const double* __restrict__ Rbar, const GatherArgs& A,
                                           const double (&Uc)[NDIM + 2], const teno_adj::CellPrim<NDIM>& P,
                                           double gamma, double (&acc)[NDIM + 2], double (&rp)[NDIM + 2]) {
  constexpr int NVAR = NDIM + 2;
  const double* __restrict__ kb = A.kb[DIR];
  const double* __restrict__ contrib = A.contrib[DIR];
  const unsigned char* __restrict__ pending = A.pending[DIR];
  const double fs = A.fscale[DIR];
  const int64_t ncell = G.ncell;
  const int64_t m0 = G.n[0] + (DIR == 0), m1 = G.n[1] + (DIR == 1);
  const int64_t nifc = m0 * m1 * (G.n[2] + (DIR == 2));
  const int64_t sd = (DIR == 0) ? 1 : (DIR == 1 ? m0 : m0 * m1);   // interface-grid stride along DIR
  const int64_t cstride = (DIR == 0) ? 1 : (DIR == 1 ? G.n[0] : G.n[0] * G.n[1]);
  const int bc = G.bc[DIR];
  const int64_t id = (DIR == 0) ? i0 : (DIR == 1 ? i1 : i2);
  // interface-grid index of this line's interface 0, and the line's cell 0
  const int64_t q0 = (i2 * m1 + i1) * m0 + i0 - id * sd;
  const int64_t line = c - id * cstride;
  double Fsum[NVAR];
  const int idl = int(id), ndl = int(G.n[DIR]);
  // Interior cells (slot j's interface qd = id+3-j) take the P-weighted Fbar
  // sum over the six slots as one stencil on Rbar:
  //   sum_j P_j (Rbar_{id+3-j} - Rbar_{id+2-j}) =
  //   ((Rbar_{id+3} - Rbar_{id-3}) - 9 (Rbar_{id+2} - Rbar_{id-2}) + 45 (Rbar_{id+1} - Rbar_{id-1})) / 60.
  // With periodic ends and at least six cells every cell does: qd and the
  // Rbar stencil wrap modulo nd, and faces 0 and nd -- one physical face
  // computed twice, each copy with its own Fbar -- both add their terms to
  // the slot whose wrapped interface is 0 (their Fbar sum is the wrapped
  // difference the stencil already holds).
  const bool wrap = bc == 0 && ndl >= 6;
  if (wrap || (idl >= 3 && idl <= ndl - 4)) {
    auto wrapped = [ndl](int y) { return y < 0 ? y + ndl : (y >= ndl ? y - ndl : y); };
    const int64_t o1p = wrapped(idl + 1) * cstride, o1m = wrapped(idl - 1) * cstride;
    const int64_t o2p = wrapped(idl + 2) * cstride, o2m = wrapped(idl - 2) * cstride;
    const int64_t o3p = wrapped(idl + 3) * cstride, o3m = wrapped(idl - 3) * cstride;
    const double w1 = fs * (1.0 / 60.0), w9 = fs * (-9.0 / 60.0), w45 = fs * (45.0 / 60.0);
    // slot j's interface; on a periodic line the slot whose interface is 0
    // also takes face nd (jd), whose U~bar enters the M sum as a seventh term
    // (interface indices fit in 32 bits: the C-ABI's grid limit)
    uint32_t qs[6];
    int jd = -1;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const int x = wrapped(idl + 3 - j);
      qs[j] = static_cast<uint32_t>(q0 + (int64_t)x * sd);
      if (x == 0 && bc == 0) jd = j;
    }
    const uint32_t qd = static_cast<uint32_t>(q0 + (int64_t)ndl * sd);
#pragma unroll
    for (int v = 0; v < NVAR; ++v) {
      const double* r = Rbar + v * ncell + line;
      const double r1p = r[o1p], r1m = r[o1m], r2p = r[o2p], r2m = r[o2m], r3p = r[o3p], r3m = r[o3m];
      double S;
      const double rs[6] = {r3p, r3m, r2p, r2m, r1p, r1m};
      const int rw[6] = {1, -1, -9, 9, 45, -45};
      if ((kAdjFixMask & 1u) && teno_fix::sum<6>(rs, rw, S)) Fsum[v] = w1 * S;
      else Fsum[v] = fma(w45, r1p - r1m, fma(w9, r2p - r2m, w1 * (r3p - r3m)));
      if (kAdjFixMask & 2u) {
        const double* k = kb + (int64_t)v * nifc;
        const double ks[7] = {k[qs[0]], k[qs[1]], k[qs[2]], k[qs[3]], k[qs[4]], k[qs[5]], jd >= 0 ? k[qd] : 0.0};
        const int kw[7] = {1, -5, 10, -10, 5, -1, jd >= 0 ? c_adjMi[jd] : 0};
        double T;
        if (teno_fix::sum<7>(ks, kw, T)) {
          acc[v] = fma(1.0 / 60.0, T, acc[v]);
        } else {
#pragma unroll
          for (int j = 0; j < 7; ++j) acc[v] = fma(kw[j] * (1.0 / 60.0), ks[j], acc[v]);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      if (kAdjFixMask & 2u) {
        slot_rest<NVAR>(j, qs[j], kb, contrib, pending, nifc, acc, rp);
        if (j == jd) slot_rest<NVAR>(j, qd, kb, contrib, pending, nifc, acc, rp);
      } else {
        slot_terms<NVAR>(j, qs[j], kb, contrib, pending, nifc, acc, rp);
        if (j == jd) slot_terms<NVAR>(j, qd, kb, contrib, pending, nifc, acc, rp);
      }
    }
  } else {
#pragma unroll
    for (int v = 0; v < NVAR; ++v) Fsum[v] = 0.0;
    gather_edge<NVAR>(idl, ndl, bc, q0, sd, line, cstride, ncell, nifc, fs, Rbar, kb, contrib, pending, acc, rp,
                      Fsum);
  }
  teno_adj::flux_vjp_acc<NDIM, DIR>(Uc, P, gamma, Fsum, acc);
}

template <int NDIM, int DIR>
__device__ __forceinline__ void gather_dirs(const Grid& G, int64_t c, int64_t i0, int64_t i1, int64_t i2,
                                            const double* __restrict__ Rbar, const GatherArgs& A,
                                            const double (&Uc)[NDIM + 2], const teno_adj::CellPrim<NDIM>& P,
                                            double gamma, double (&acc)[NDIM + 2], double (&rp)[NDIM + 2]) {
  if constexpr (DIR < NDIM) {
    gather_dir<NDIM, DIR>(G, c, i0, i1, i2, Rbar, A, Uc, P, gamma, acc, rp);
    gather_dirs<NDIM, DIR + 1>(G, c, i0, i1, i2, Rbar, A, Uc, P, gamma, acc, rp);
  }
}

// out_c = a X_c + b Y_c + sum over directions and over the (interface, slot)
// pairs whose stencil point maps to cell c (boundary ghost copies included)
// of: M_j U~bar of the kept interfaces, the pending interfaces' contributions,
// A_d(U_c)^T applied once per direction to sum_j P_j Fbar of all of them, and
// the Roe-parameter map of cell c applied once to the sum of its parameter
// adjoints.  Deterministic, no atomics.
#ifndef TENO_ADJ_GATHER_MINBLOCKS
#define TENO_ADJ_GATHER_MINBLOCKS 2
#endif
template <int NDIM>
__global__ void __launch_bounds__(256, TENO_ADJ_GATHER_MINBLOCKS) adj_gather_kernel(
    const double* __restrict__ U, const double* __restrict__ aux, const double* __restrict__ Rbar,
    const GatherArgs A, const Grid G, double gamma) {
  constexpr int NVAR = NDIM + 2;
  const int64_t ncell = G.ncell;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i0 = c % G.n[0];
    const int64_t r = c / G.n[0];
    const int64_t i1 = r % G.n[1];
    const int64_t i2 = r / G.n[1];
    double Uc[NVAR], acc[NVAR], rp[NVAR];
#pragma unroll
    for (int v = 0; v < NVAR; ++v) {
      Uc[v] = U[v * ncell + c];
      acc[v] = rp[v] = 0.0;
    }
    teno_adj::CellPrim<NDIM> P;
    teno_adj::cell_prim<NDIM>(Uc, gamma, P);
    gather_dirs<NDIM, 0>(G, c, i0, i1, i2, Rbar, A, Uc, P, gamma, acc, rp);
    // the Roe-parameter map of cell c: sqrt(rho) from the cell pass,
    // H = (E + p) / rho
    const double sx = aux[(NDIM + 1) * ncell + c];
    const double Hx = (Uc[NVAR - 1] + P.p) * P.ir;
    teno_adj::roe_param_vjp_acc<NDIM>(P, sx, Hx, gamma, rp, acc);
#pragma unroll
    for (int v = 0; v < NVAR; ++v) {
      double o = acc[v];
      if (A.X) o = fma(A.a, A.X[v * ncell + c], o);
      if (A.Y) o = fma(A.b, A.Y[v * ncell + c], o);
      A.out[v * ncell + c] = o;
    }
  }
}

// Sum the per-block d/dalpha of every direction in a fixed order (one block
// of kAlphaThreads: strided partial sums, then a tree) and add their effect
// at the arg-max cells (one thread: several speeds may share a cell).
// apart: [ndim][2 nblocks][3], the kept pass's blocks first (their sums in
// units of 60 dx_d / scale: times kscale[d]), then the general pass's.
struct AlphaScale {
  double k[3];
};
constexpr int kAlphaThreads = 256;
template <int NDIM>
__global__ void __launch_bounds__(kAlphaThreads) adj_alpha_kernel(const double* __restrict__ apart, int nblocks,
                                 AlphaScale kscale, const unsigned long long* __restrict__ argidx,
                                 const double* __restrict__ U, double* __restrict__ Ubar, int64_t ncell,
                                 double gamma) {
  constexpr int NVAR = NDIM + 2;
  __shared__ double red[kAlphaThreads][3];
  __shared__ double tot[NDIM][2][3];
  for (int d = 0; d < NDIM; ++d)
    for (int h = 0; h < 2; ++h) {
      const double* ap = apart + ((int64_t)d * 2 + h) * nblocks * 3;
      double s[3] = {0.0, 0.0, 0.0};
      for (int b = threadIdx.x; b < nblocks; b += kAlphaThreads)
        for (int k = 0; k < 3; ++k) s[k] += ap[b * 3 + k];
      for (int k = 0; k < 3; ++k) red[threadIdx.x][k] = s[k];
      __syncthreads();
      for (int w = kAlphaThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
          for (int k = 0; k < 3; ++k) red[threadIdx.x][k] += red[threadIdx.x + w][k];
        __syncthreads();
      }
      if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) tot[d][h][k] = red[0][k];
      __syncthreads();
    }
  if (threadIdx.x != 0) return;
  for (int d = 0; d < NDIM; ++d)
    for (int k = 0; k < 3; ++k) {
      const unsigned long long c = argidx[d * 3 + k];
      if (c >= (unsigned long long)ncell) continue;
      double Uc[NVAR], g[NVAR];
      for (int v = 0; v < NVAR; ++v) {
        Uc[v] = U[v * ncell + c];
        g[v] = 0.0;
      }
      const double s = fma(kscale.k[d], tot[d][0][k], tot[d][1][k]);
      teno_adj::wave_speed_grad<NDIM>(Uc, d, k, gamma, s, g);
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
  if (!teno::scheme_fields_ok(g)) return false;
  // the pending list holds 32-bit interface indices and int counts
  for (int d = 0; d < g->ndim; ++d) {
    double m = 1.0;
    for (int k = 0; k < 3; ++k) m *= double(g->n[k] + (k == d ? 1 : 0));
    if (m >= 2147483647.0) return false;
  }
  return true;
}

// What the adjoint does not differentiate: reflecting walls and fixed-state
// faces (it supports periodic and transmissive boundaries), a body-force
// source, and WENO-Z (its weights are not piecewise constant; the TENO
// cutoffs are).
bool adjoint_unsupported(const teno_grid* g) {
  if (!g || g->ndim < 1 || g->ndim > 3) return false;
  for (int k = 0; k < g->ndim; ++k)
    if (g->bc[k] == TENO_BC_REFLECTIVE || g->bc[k] == TENO_BC_DIRICHLET || g->grav[k] != 0.0) return true;
  return g->scheme == TENO_SCHEME_WENOZ;
}


int64_t nifc_of(const teno_grid* g, int d) {
  int64_t m = 1;
  for (int k = 0; k < 3; ++k) m *= g->n[k] + (k == d ? 1 : 0);
  return m;
}

int adj_blocks(int nsm) { return nsm * 8; }
// blocks of the list-building passes (at most 8 kListThreads, the scan's reach)
int adj_list_blocks(int nsm) { return nsm * 4 < 8 * kListThreads ? nsm * 4 : 8 * kListThreads; }

struct AdjLayout {
  // header: [0] status, [8] dt; per stage s (the RK3 adjoint's three stage
  // inputs; one for a right-hand-side adjoint): the LF speeds (9 x 8) with
  // the pending-list counters of its forward recomputation after them at
  // alpha + 128 s, its arg-max cells (9 x 8) at argidx + 128 s
  static constexpr size_t kStage = 128;
  size_t status = 0, dt = 8, alpha = 64, argidx = 512;
  size_t aux = 0, aux_bytes = 0, cand = 0, fh = 0, kb = 0, kb_bytes = 0, contrib = 0, contrib_bytes = 0,
         pending = 0, pending_bytes = 0, list = 0, sel = 0, lcount = 0, apart = 0, R = 0, U1 = 0, U2 = 0, B1 = 0,
         B2 = 0, roe = 0, roe_stage_bytes = 0, total = 0;
  size_t roe_dir = 0;   // doubles between two directions' Roe states
};

AdjLayout adj_layout(const teno_grid* g, int op, int nsm) {
  AdjLayout L;
  const size_t ncell = size_t(g->n[0] * g->n[1] * g->n[2]);
  const int nvar = g->ndim + 2;
  const int nstage = op == TENO_OP_RK3_ADJOINT ? 3 : 1;
  int64_t maxifc = 0;
  for (int d = 0; d < g->ndim; ++d) maxifc = nifc_of(g, d) > maxifc ? nifc_of(g, d) : maxifc;
  size_t off = 1024;
  // the cell pass's primitives of every stage input
  L.aux = off;
  L.aux_bytes = round_up(sizeof(double) * teno::aux_fields(g->ndim) * ncell);
  off += nstage * L.aux_bytes;
  L.cand = off;   // the cell pass's per-block arg-max candidates
  off += round_up(sizeof(unsigned long long) * 18 * size_t(teno::cell_blocks(int64_t(ncell), nsm)));
  // per direction: the kept interfaces' terms, the pending ones'
  // contributions (the first also the forward recomputation's interface
  // fluxes) and the pending marks
  L.kb = off;
  L.kb_bytes = round_up(sizeof(double) * 3 * nvar * size_t(maxifc));
  off += g->ndim * L.kb_bytes;
  L.contrib = off;
  L.contrib_bytes = round_up(sizeof(double) * 6 * nvar * size_t(maxifc));
  off += g->ndim * L.contrib_bytes;
  L.pending = off;
  L.pending_bytes = round_up(size_t(maxifc));
  off += g->ndim * L.pending_bytes;
  // pending list (recomputed forward stages; the adjoint's general pass) and
  // its partitioned copy, the listed interfaces' packed selections and
  // theirs (each in two halves of 2 maxifc + 2 entries)
  L.list = off;
  off += round_up(sizeof(uint32_t) * (2 * size_t(maxifc) + 2));
  L.sel = off;
  off += round_up(sizeof(uint32_t) * (2 * size_t(maxifc) + 2));
  L.lcount = off;   // the list passes' per-block counts, offsets, total and all-kept total
  off += round_up(sizeof(int) * (2 * size_t(adj_list_blocks(nsm)) + 2));
  L.apart = off;   // [ndim][2 blocks][3]: d/dalpha per block of the kept and general passes
  off += round_up(sizeof(double) * 3 * 2 * size_t(adj_blocks(nsm)) * g->ndim);
  if (op == TENO_OP_RK3_ADJOINT) {
    // half fluxes of the recomputed forward stages (two-pass fluxes)
    L.fh = off;
    off += round_up(sizeof(double) * g->ndim * (nvar - 1) * ncell);
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
    // the recomputed stages' Roe states and decisions (stage slots 0, 1),
    // [ndim][ndim + 8][maxifc]
    L.roe_dir = size_t(g->ndim + 8) * size_t(maxifc);
    L.roe_stage_bytes = round_up(sizeof(double) * g->ndim * L.roe_dir);
    L.roe = off;
    off += 2 * L.roe_stage_bytes;
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
    G.rdx[k] = G.dx[0] / G.dx[k];
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
                    const unsigned long long* alpha, const double* Rbar, double scale, double* kb,
                    double* contrib, unsigned char* pending, uint32_t* list, int* lcount, uint32_t* sel,
                    double* apart, int* status, const Grid& G, const Scheme& S, const double* roe_in) {
  if (roe_in)
    adj_kept_kernel<NDIM, DIR, true><<<nblk, kAdjThreads, 0, st>>>(U, aux, alpha, Rbar, scale, kb, pending, apart,
                                                                  status, G, S, roe_in);
  else
    adj_kept_kernel<NDIM, DIR, false><<<nblk, kAdjThreads, 0, st>>>(U, aux, alpha, Rbar, scale, kb, pending, apart,
                                                                   status, G, S, nullptr);
  int64_t nifc = 1;
  for (int k = 0; k < 3; ++k) nifc *= G.n[k] + (k == DIR ? 1 : 0);
  const int lblk = adj_list_blocks(nsm);
  int* bcount = lcount;
  int* boff = lcount + lblk;
  int* total = lcount + 2 * lblk;
  adj_count_kernel<<<lblk, kListThreads, 0, st>>>(pending, nifc, bcount);
  adj_scan_kernel<<<1, kListThreads, 0, st>>>(bcount, lblk, boff, total);
  adj_scatter_kernel<<<lblk, kListThreads, 0, st>>>(pending, nifc, boff, list);
  adj_select_kernel<NDIM, DIR><<<nblk, kAdjThreads, 0, st>>>(U, aux, alpha, list, total, sel, status, G, S);
  // the partition reuses the counts and offsets; its own total (the number
  // of all-kept entries) goes to the slot after the list's
  int* nkept = total + 1;
  uint32_t* list2 = list + (nifc + 1) / 2 * 2;   // second half of the list region
  uint32_t* sel2 = sel + (nifc + 1) / 2 * 2;
  adj_part_count_kernel<<<lblk, kListThreads, 0, st>>>(sel, total, NDIM + 2, bcount);
  adj_scan_kernel<<<1, kListThreads, 0, st>>>(bcount, lblk, boff, nkept);
  adj_part_scatter_kernel<<<lblk, kListThreads, 0, st>>>(list, sel, total, NDIM + 2, boff, nkept, list2, sel2);
  adj_general_kernel<NDIM, DIR><<<nblk, kAdjThreads, 0, st>>>(U, alpha, Rbar, scale, contrib, list2, total, nkept,
                                                             sel2, apart + 3 * nblk, G, S);
}

template <int NDIM>
void launch_adj_all(int nblk, int nsm, cudaStream_t st, const double* U, const double* aux,
                    const unsigned long long* alpha, const unsigned long long* argidx, const double* Rbar,
                    double scale, const AdjLayout& L, char* ws, int* status, GatherArgs A, const Grid& G,
                    const Scheme& S, const double* roe_in) {
  auto* list = reinterpret_cast<uint32_t*>(ws + L.list);
  auto* lcount = reinterpret_cast<int*>(ws + L.lcount);
  auto* sel = reinterpret_cast<uint32_t*>(ws + L.sel);
  double* apart = reinterpret_cast<double*>(ws + L.apart);
  for (int d = 0; d < NDIM; ++d) {
    double* kb = reinterpret_cast<double*>(ws + L.kb + d * L.kb_bytes);
    double* contrib = reinterpret_cast<double*>(ws + L.contrib + d * L.contrib_bytes);
    auto* pending = reinterpret_cast<unsigned char*>(ws + L.pending + d * L.pending_bytes);
    double* ap = apart + 6 * nblk * d;
    const double* rin = roe_in ? roe_in + d * L.roe_dir : nullptr;
    if (d == 0) launch_adj_dir<NDIM, 0>(nblk, nsm, st, U, aux, alpha, Rbar, scale, kb, contrib, pending, list, lcount, sel, ap, status, G, S, rin);
    if constexpr (NDIM > 1)
      if (d == 1) launch_adj_dir<NDIM, 1>(nblk, nsm, st, U, aux, alpha, Rbar, scale, kb, contrib, pending, list, lcount, sel, ap, status, G, S, rin);
    if constexpr (NDIM > 2)
      if (d == 2) launch_adj_dir<NDIM, 2>(nblk, nsm, st, U, aux, alpha, Rbar, scale, kb, contrib, pending, list, lcount, sel, ap, status, G, S, rin);
    A.kb[d] = kb;
    A.contrib[d] = contrib;
    A.pending[d] = pending;
    A.fscale[d] = scale * G.inv_dx[d];
  }
  int64_t gb = (G.ncell + 255) / 256;
  if (gb > int64_t(nsm) * 16) gb = int64_t(nsm) * 16;
  adj_gather_kernel<NDIM><<<unsigned(gb), 256, 0, st>>>(U, aux, Rbar, A, G, S.gamma);
  AlphaScale ks{};
  for (int d = 0; d < NDIM; ++d) ks.k[d] = scale * G.inv_dx[d] * (1.0 / 60.0);
  adj_alpha_kernel<NDIM><<<1, kAlphaThreads, 0, st>>>(apart, nblk, ks, argidx, U, A.out, G.ncell, S.gamma);
}

// out = a X + b Y + scale J(U)^T Rbar (X, Y nullable; out may alias X or Y,
// not Rbar or U), with stage slot `stage` of the workspace.  With `cell`
// the cell pass of U comes first; without it, the forward recomputation of
// that stage has left its primitives, speeds and arg-max cells there.
teno_status adjoint_sequence(const teno_grid* g, const AdjLayout& L, char* ws, int stage, bool cell,
                             const double* U, const double* Rbar, double scale, double* out, const double* X,
                             double a, const double* Y, double b, cudaStream_t st) {
  const Grid G = make_grid(g);
  const Scheme S = teno::scheme_of(g);
  const int nsm = sm_count();
  const int nblk = adj_blocks(nsm);
  int* status = reinterpret_cast<int*>(ws + L.status);
  auto* alpha = reinterpret_cast<unsigned long long*>(ws + L.alpha + stage * AdjLayout::kStage);
  auto* argidx = reinterpret_cast<unsigned long long*>(ws + L.argidx + stage * AdjLayout::kStage);
  double* aux = reinterpret_cast<double*>(ws + L.aux + stage * L.aux_bytes);
  if (cell) {
    auto* cand = reinterpret_cast<unsigned long long*>(ws + L.cand);
    if (cudaMemsetAsync(alpha, 0, sizeof(unsigned long long) * 9, st) != cudaSuccess) return TENO_ERR_CUDA;
    if (teno::launch_cell(g->ndim, U, aux, nullptr, alpha, status, G.ncell, g->gamma, nsm, st, cand) !=
            cudaSuccess ||
        teno::launch_argmax_finish(g->ndim, cand, G.ncell, nsm, argidx, st) != cudaSuccess)
      return TENO_ERR_CUDA;
  }
  GatherArgs A{};
  A.out = out;
  A.X = X;
  A.a = a;
  A.Y = Y;
  A.b = b;
  // the recomputed forward stage's Roe states, where it stored them (stage
  // slots 0 and 1; none without a keep-all magnitude, as nothing is kept)
  const double* roe_in = (!cell && L.roe && stage < 2 && S.keep_idx >= 0)
                             ? reinterpret_cast<const double*>(ws + L.roe + stage * L.roe_stage_bytes)
                             : nullptr;
  if (g->ndim == 1) launch_adj_all<1>(nblk, nsm, st, U, aux, alpha, argidx, Rbar, scale, L, ws, status, A, G, S, roe_in);
  else if (g->ndim == 2) launch_adj_all<2>(nblk, nsm, st, U, aux, alpha, argidx, Rbar, scale, L, ws, status, A, G, S, roe_in);
  else launch_adj_all<3>(nblk, nsm, st, U, aux, alpha, argidx, Rbar, scale, L, ws, status, A, G, S, roe_in);
  return cudaGetLastError() == cudaSuccess ? TENO_OK : TENO_ERR_CUDA;
}

teno_status lincomb(double* out, double a, const double* x, double b, const double* y, int64_t n,
                    cudaStream_t st) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  lincomb_kernel<<<unsigned(blocks), 256, 0, st>>>(out, a, x, b, y, n);
  return cudaGetLastError() == cudaSuccess ? TENO_OK : TENO_ERR_CUDA;
}

// The reverse of eq. 4.3 -> 4.2 -> 4.1 from the stage inputs U_n, U1, U2;
// with `cells`, every stage input gets its cell pass here, otherwise the
// forward recomputation has left those of U_n and U1 in stage slots 0, 1.
teno_status reverse_stages(const teno_grid* g, const AdjLayout& L, char* w, const double* U_n, const double* U1,
                           const double* U2, bool cells, double dt, const double* Ubar_next, double* Ubar_n,
                           cudaStream_t st) {
  const int64_t ntot = int64_t(g->ndim + 2) * g->n[0] * g->n[1] * g->n[2];
  double* B1 = reinterpret_cast<double*>(w + L.B1);
  double* B2 = reinterpret_cast<double*>(w + L.B2);
  teno_status s;
  // reverse of eq. 4.3: B2 = 2/3 Ubar' + 2/3 dt J(U2)^T Ubar'
  if ((s = adjoint_sequence(g, L, w, 2, true, U2, Ubar_next, 2.0 / 3.0 * dt, B2, Ubar_next, 2.0 / 3.0, nullptr,
                            0.0, st)) != TENO_OK)
    return s;
  // Ubar_n = 1/3 Ubar' + 3/4 B2 (eq. 4.3 and 4.2 reach U^n directly)
  if ((s = lincomb(Ubar_n, 1.0 / 3.0, Ubar_next, 0.75, B2, ntot, st)) != TENO_OK) return s;
  // reverse of eq. 4.2: B1 = 1/4 B2 + 1/4 dt J(U1)^T B2
  if ((s = adjoint_sequence(g, L, w, 1, cells, U1, B2, 0.25 * dt, B1, B2, 0.25, nullptr, 0.0, st)) != TENO_OK)
    return s;
  // reverse of eq. 4.1: Ubar_n += B1 + dt J(U_n)^T B1
  return adjoint_sequence(g, L, w, 0, cells, U_n, B1, dt, Ubar_n, Ubar_n, 1.0, B1, 1.0, st);
}

}  // namespace

extern "C" {

size_t teno_adjoint_workspace_bytes(const teno_grid* g, int op) {
  if (!grid_valid(g) || (op != TENO_OP_RHS_ADJOINT && op != TENO_OP_RK3_ADJOINT)) return 0;
  return adj_layout(g, op, sm_count()).total;
}

teno_status teno_rhs_adjoint(const teno_grid* g, const double* U, const double* dUdt_bar, double* U_bar,
                             void* ws, size_t ws_bytes, void* stream) {
  if (adjoint_unsupported(g)) return TENO_ERR_UNSUPPORTED;
  if (!grid_valid(g) || !U || !dUdt_bar || !U_bar) return TENO_ERR_INVALID_ARG;
  if (!al(U, 16) || !al(dUdt_bar, 16) || !al(U_bar, 16)) return TENO_ERR_INVALID_ARG;
  if (U_bar == U || U_bar == dUdt_bar) return TENO_ERR_INVALID_ARG;
  if (!is_dev(U) || !is_dev(dUdt_bar) || !is_dev(U_bar)) return TENO_ERR_INVALID_ARG;
  const AdjLayout L = adj_layout(g, TENO_OP_RHS_ADJOINT, sm_count());
  if (!ws || !al(ws, kAlign) || ws_bytes < L.total || !is_dev(ws)) return TENO_ERR_WORKSPACE;
  return adjoint_sequence(g, L, static_cast<char*>(ws), 0, true, U, dUdt_bar, 1.0, U_bar, U_bar, 1.0, nullptr,
                          0.0, static_cast<cudaStream_t>(stream));
}

teno_status teno_rk3_step_adjoint(const teno_grid* g, const double* U_n, double dt, const double* Ubar_next,
                                  double* Ubar_n, void* ws, size_t ws_bytes, void* stream) {
  if (adjoint_unsupported(g)) return TENO_ERR_UNSUPPORTED;
  if (!grid_valid(g) || !U_n || !Ubar_next || !Ubar_n || !(dt >= 0.0) || !std::isfinite(dt))
    return TENO_ERR_INVALID_ARG;
  if (!al(U_n, 16) || !al(Ubar_next, 16) || !al(Ubar_n, 16) || Ubar_n == U_n) return TENO_ERR_INVALID_ARG;
  if (!is_dev(U_n) || !is_dev(Ubar_next) || !is_dev(Ubar_n)) return TENO_ERR_INVALID_ARG;
  const AdjLayout L = adj_layout(g, TENO_OP_RK3_ADJOINT, sm_count());
  if (!ws || !al(ws, kAlign) || ws_bytes < L.total || !is_dev(ws)) return TENO_ERR_WORKSPACE;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(ws);
  double* R = reinterpret_cast<double*>(w + L.R);
  double* U1 = reinterpret_cast<double*>(w + L.U1);
  double* U2 = reinterpret_cast<double*>(w + L.U2);
  double* dtp = reinterpret_cast<double*>(w + L.dt);

  // forward stages of the step (eq. 4.1-4.2) with the given dt; each keeps
  // its stage input's primitives, speeds and arg-max cells for the reverse
  // pass (stage slots 0 and 1)
  auto* cand = reinterpret_cast<unsigned long long*>(w + L.cand);
  const int nsm = sm_count();
  const int64_t ncell = int64_t(g->n[0]) * g->n[1] * g->n[2];
  set_value_kernel<<<1, 1, 0, st>>>(dtp, dt);
  if (cudaGetLastError() != cudaSuccess) return TENO_ERR_CUDA;
  double* roe0 = reinterpret_cast<double*>(w + L.roe);
  double* roe1 = reinterpret_cast<double*>(w + L.roe + L.roe_stage_bytes);
  teno_status s = teno::forward_stage(g, w, L.status, L.dt, L.alpha, L.aux, L.fh, L.contrib, L.list, U_n, R,
                                      2, U_n, nullptr, U1, st, cand, roe0, L.roe_dir);
  if (s != TENO_OK) return s;
  if (teno::launch_argmax_finish(g->ndim, cand, ncell, nsm, reinterpret_cast<unsigned long long*>(w + L.argidx),
                                 st) != cudaSuccess)
    return TENO_ERR_CUDA;
  s = teno::forward_stage(g, w, L.status, L.dt, L.alpha + AdjLayout::kStage, L.aux + L.aux_bytes, L.fh, L.contrib,
                          L.list, U1, R, 3, U_n, U1, U2, st, cand, roe1, L.roe_dir);
  if (s != TENO_OK) return s;
  if (teno::launch_argmax_finish(g->ndim, cand, ncell, nsm,
                                 reinterpret_cast<unsigned long long*>(w + L.argidx + AdjLayout::kStage),
                                 st) != cudaSuccess)
    return TENO_ERR_CUDA;

  return reverse_stages(g, L, w, U_n, U1, U2, false, dt, Ubar_next, Ubar_n, st);
}

teno_status teno_rk3_step_adjoint_staged(const teno_grid* g, const double* U_n, const double* U1,
                                         const double* U2, double dt, const double* Ubar_next, double* Ubar_n,
                                         void* ws, size_t ws_bytes, void* stream) {
  if (adjoint_unsupported(g)) return TENO_ERR_UNSUPPORTED;
  if (!grid_valid(g) || !U_n || !U1 || !U2 || !Ubar_next || !Ubar_n || !(dt >= 0.0) || !std::isfinite(dt))
    return TENO_ERR_INVALID_ARG;
  if (!al(U_n, 16) || !al(U1, 16) || !al(U2, 16) || !al(Ubar_next, 16) || !al(Ubar_n, 16))
    return TENO_ERR_INVALID_ARG;
  if (Ubar_n == U_n || Ubar_n == U1 || Ubar_n == U2) return TENO_ERR_INVALID_ARG;
  if (!is_dev(U_n) || !is_dev(U1) || !is_dev(U2) || !is_dev(Ubar_next) || !is_dev(Ubar_n))
    return TENO_ERR_INVALID_ARG;
  const AdjLayout L = adj_layout(g, TENO_OP_RK3_ADJOINT, sm_count());
  if (!ws || !al(ws, kAlign) || ws_bytes < L.total || !is_dev(ws)) return TENO_ERR_WORKSPACE;
  return reverse_stages(g, L, static_cast<char*>(ws), U_n, U1, U2, true, dt, Ubar_next, Ubar_n,
                        static_cast<cudaStream_t>(stream));
}

}  // extern "C"
