// teno_device.cuh -- device-side building blocks of the TENO5-LAD Euler RHS
// for sm_103a.  Everything here is FP64.  The arithmetic of each block follows
// the paper's equations; operation order is chosen for the GPU (FMA, shared
// sub-expressions), so results agree with a plain evaluation to rounding.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace teno {

// Ladder of eq. 3.3: c_lad[m] = 10^-m written as decimal literals, so
// C_T = Lad(m) (eq. 3.4) costs one table read and no power evaluation.
static __constant__ double c_lad[16] = {
    1e-0, 1e-1, 1e-2, 1e-3, 1e-4,  1e-5,  1e-6,  1e-7,
    1e-8, 1e-9, 1e-10, 1e-11, 1e-12, 1e-13, 1e-14, 1e-15};

// TENO weights of eq. 2.15 for each selection pattern sel = delta_0 |
// delta_1 << 1 | delta_2 << 2, with the linear weights c = (0.1, 0.6, 0.3):
// omega_k = delta_k c_k / sum_j delta_j c_j.  Pattern 0 cannot occur (the
// largest chi_k is at least 1/3 > C_T).
static __constant__ double c_omega[8][3] = {
    {0.0, 0.0, 0.0},
    {0.1 / 0.1, 0.0, 0.0},
    {0.0, 0.6 / 0.6, 0.0},
    {0.1 / (0.1 + 0.6), 0.6 / (0.1 + 0.6), 0.0},
    {0.0, 0.0, 0.3 / 0.3},
    {0.1 / (0.1 + 0.3), 0.0, 0.3 / (0.1 + 0.3)},
    {0.0, 0.6 / (0.6 + 0.3), 0.3 / (0.6 + 0.3)},
    {0.1 / (0.1 + 0.6 + 0.3), 0.6 / (0.1 + 0.6 + 0.3), 0.3 / (0.1 + 0.6 + 0.3)}};

constexpr int kMaxDim = 3;
constexpr int kMaxVar = 5;
constexpr int kMaxLadder = 16;

// Device status bits recorded in the workspace header.
enum : int { kStatusNonphysical = 1, kStatusTimeout = 2 };

// Scheme constants, passed to kernels by value.
struct Scheme {
  double gamma;   // ratio of specific heats (eq. 4.7)
  double gm1;     // gamma - 1
  double eps;     // epsilon of eq. 2.8 / 3.2
  int b_l, b_u;   // magnitude bounds of eq. 3.1
  int nthr;       // B_u - B_l
  // m = B_l + #{ j in 1..B_u-B_l : tau <= thr[j-1] * min_k(beta_k + eps) }.
  // With theta = 1/(1 + max_k chi~_k / H) and max_k chi~_k = tau / min_k(beta_k
  // + eps) (eq. 3.2), floor(theta (B_u - B_l)) >= j  <=>  max chi~ <=
  // H ((B_u - B_l)/j - 1); the last threshold (theta == 1 exactly) is the
  // binary64 condition 1 + max chi~ / H == 1, i.e. max chi~ <= H 2^-53.
  double thr[kMaxLadder];
};

struct Grid {
  int64_t n[3];
  int64_t ncell;
  int bc[3];           // 0 periodic, 1 transmissive
  double dx[3];
  double inv_dx[3];
};

// Index of a (possibly ghost) cell along an axis of n cells: periodic wrap or
// zero-gradient copy of the boundary cell.
__device__ __forceinline__ int64_t ghost(int64_t i, int64_t n, int bc) {
  if (bc == 0) {
    if (i < 0) i += n;
    else if (i >= n) i -= n;
    // a stencil reaches at most 3 cells outside; for n < 3 wrap again
    if (i < 0) i = ((i % n) + n) % n;
    else if (i >= n) i = i % n;
    return i;
  }
  return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

// Non-negative doubles order like their bit patterns; used for max / compare
// on the integer pipe.
__device__ __forceinline__ unsigned long long dbits(double x) {
  return static_cast<unsigned long long>(__double_as_longlong(x));
}

// ---------------------------------------------------------------------------
// TENO5-LAD scalar reconstruction of the interface value from five values
// v0..v4 = (f_{i-2}, ..., f_{i+2}).  Returns f^ (eq. 2.7); *flag receives
// delta bits 0..2 and m in bits 3..6.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double teno5_lad(double v0, double v1, double v2,
                                            double v3, double v4,
                                            const Scheme& S, unsigned& flag) {
  // eq. 2.9-2.11
  const double k13_12 = 13.0 / 12.0;
  double a0 = v0 - 2.0 * v1 + v2, c0 = v0 - 4.0 * v1 + 3.0 * v2;
  double a1 = v1 - 2.0 * v2 + v3, c1 = v1 - v3;
  double a2 = v2 - 2.0 * v3 + v4, c2 = 3.0 * v2 - 4.0 * v3 + v4;
  double beta0 = k13_12 * a0 * a0 + 0.25 * c0 * c0;
  double beta1 = k13_12 * a1 * a1 + 0.25 * c1 * c1;
  double beta2 = k13_12 * a2 * a2 + 0.25 * c2 * c2;
  // eq. 2.12
  double tau = fabs(beta2 - beta0);
  double d0 = beta0 + S.eps, d1 = beta1 + S.eps, d2 = beta2 + S.eps;
  // eq. 3.1-3.2 without division: compare tau with thr_j * min_k(beta_k+eps)
  unsigned long long bmin = min(dbits(d0), min(dbits(d1), dbits(d2)));
  double dmin = __longlong_as_double(static_cast<long long>(bmin));
  unsigned long long btau = dbits(tau);
  int m = S.b_l;
#pragma unroll
  for (int j = 0; j < kMaxLadder; ++j) {
    if (j < S.nthr) m += (btau <= dbits(S.thr[j] * dmin)) ? 1 : 0;
  }
  // eq. 3.4
  double ct = c_lad[m];
  // eq. 2.8 with C = 1, q = 6
  double x0 = 1.0 + tau / d0, x1 = 1.0 + tau / d1, x2 = 1.0 + tau / d2;
  double g0 = x0 * x0 * x0; g0 *= g0;
  double g1 = x1 * x1 * x1; g1 *= g1;
  double g2 = x2 * x2 * x2; g2 *= g2;
  // eq. 2.13-2.14 as gamma_k >= C_T * sum(gamma)  (chi_k >= C_T)
  unsigned long long lim = dbits(ct * (g0 + g1 + g2));
  unsigned sel = (dbits(g0) >= lim ? 1u : 0u) | (dbits(g1) >= lim ? 2u : 0u) |
                 (dbits(g2) >= lim ? 4u : 0u);
  flag = sel | (static_cast<unsigned>(m) << 3);
  // eq. 2.4-2.6
  double f0 = (1.0 / 3.0) * v0 - (7.0 / 6.0) * v1 + (11.0 / 6.0) * v2;
  double f1 = -(1.0 / 6.0) * v1 + (5.0 / 6.0) * v2 + (1.0 / 3.0) * v3;
  double f2 = (1.0 / 3.0) * v2 + (5.0 / 6.0) * v3 - (1.0 / 6.0) * v4;
  // eq. 2.15, eq. 2.7
  return c_omega[sel][0] * f0 + c_omega[sel][1] * f1 + c_omega[sel][2] * f2;
}

// Same reconstruction with the selection forced (bits 0..2 of `forced`).
__device__ __forceinline__ double teno5_forced(double v0, double v1, double v2,
                                               double v3, double v4,
                                               const Scheme& S, unsigned forced) {
  double f0 = (1.0 / 3.0) * v0 - (7.0 / 6.0) * v1 + (11.0 / 6.0) * v2;
  double f1 = -(1.0 / 6.0) * v1 + (5.0 / 6.0) * v2 + (1.0 / 3.0) * v3;
  double f2 = (1.0 / 3.0) * v2 + (5.0 / 6.0) * v3 - (1.0 / 6.0) * v4;
  unsigned sel = forced & 7u;
  return c_omega[sel][0] * f0 + c_omega[sel][1] * f1 + c_omega[sel][2] * f2;
}

}  // namespace teno
