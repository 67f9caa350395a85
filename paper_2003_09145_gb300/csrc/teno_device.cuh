// teno_device.cuh -- device-side building blocks of the TENO5-LAD Euler RHS
// for sm_103a.  Everything here is FP64.  The arithmetic of each block follows
// the paper's equations; operation order is chosen for the GPU (FMA, shared
// sub-expressions), so results agree with a plain evaluation to rounding.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "teno_cert.cuh"

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

// The TENO flux of eq. 2.7 written on first differences e_k = v_{k+1} - v_k:
// f^ = v2 + sum_k w_k e_k with, for weights omega = c_omega[sel],
// w = (-omega_0/3, 5 omega_0/6 + omega_1/6, omega_1/3 + 2 omega_2/3, -omega_2/6)
// (candidates of eq. 2.4-2.6 relative to v2: (5 e1/6 - e0/3), (e1/6 + e2/3),
// (2 e2/3 - e3/6)).  With every stencil kept this is eq. 2.3.
#define TENO_COEF_ROW(o0, o1, o2) \
  {-(o0) / 3.0, 5.0 * (o0) / 6.0 + (o1) / 6.0, (o1) / 3.0 + 2.0 * (o2) / 3.0, -(o2) / 6.0}
static __constant__ double c_coef[8][4] = {
    TENO_COEF_ROW(0.0, 0.0, 0.0),
    TENO_COEF_ROW(0.1 / 0.1, 0.0, 0.0),
    TENO_COEF_ROW(0.0, 0.6 / 0.6, 0.0),
    TENO_COEF_ROW(0.1 / (0.1 + 0.6), 0.6 / (0.1 + 0.6), 0.0),
    TENO_COEF_ROW(0.0, 0.0, 0.3 / 0.3),
    TENO_COEF_ROW(0.1 / (0.1 + 0.3), 0.0, 0.3 / (0.1 + 0.3)),
    TENO_COEF_ROW(0.0, 0.6 / (0.6 + 0.3), 0.3 / (0.6 + 0.3)),
    TENO_COEF_ROW(0.1 / (0.1 + 0.6 + 0.3), 0.6 / (0.1 + 0.6 + 0.3), 0.3 / (0.1 + 0.6 + 0.3))};
#undef TENO_COEF_ROW

// The same flux on the point values: f^ = sum_j c_lin[sel][j] v_j with
// (omega_0/3, -7 omega_0/6 - omega_1/6, 11 omega_0/6 + 5 omega_1/6 + omega_2/3,
//  omega_1/3 + 5 omega_2/6, -omega_2/6) (eq. 2.4-2.7).
#define TENO_LIN_ROW(o0, o1, o2)                                                              \
  {(o0) / 3.0, -7.0 * (o0) / 6.0 - (o1) / 6.0, 11.0 * (o0) / 6.0 + 5.0 * (o1) / 6.0 + (o2) / 3.0, \
   (o1) / 3.0 + 5.0 * (o2) / 6.0, -(o2) / 6.0}
static __constant__ double c_lin[8][5] = {
    TENO_LIN_ROW(0.0, 0.0, 0.0),
    TENO_LIN_ROW(0.1 / 0.1, 0.0, 0.0),
    TENO_LIN_ROW(0.0, 0.6 / 0.6, 0.0),
    TENO_LIN_ROW(0.1 / (0.1 + 0.6), 0.6 / (0.1 + 0.6), 0.0),
    TENO_LIN_ROW(0.0, 0.0, 0.3 / 0.3),
    TENO_LIN_ROW(0.1 / (0.1 + 0.3), 0.0, 0.3 / (0.1 + 0.3)),
    TENO_LIN_ROW(0.0, 0.6 / (0.6 + 0.3), 0.3 / (0.6 + 0.3)),
    TENO_LIN_ROW(0.1 / (0.1 + 0.6 + 0.3), 0.6 / (0.1 + 0.6 + 0.3), 0.3 / (0.1 + 0.6 + 0.3))};
#undef TENO_LIN_ROW

constexpr int kMaxDim = 3;
// Per-cell primitive fields the cell pass writes (aux, [aux_fields][ncell]):
// u_k/2 (ndim), p/2, sqrt(rho), (E+p)/sqrt(rho), m_k/sqrt(rho) = sqrt(rho) u_k (ndim).
__host__ __device__ constexpr int aux_fields(int ndim) { return 2 * ndim + 3; }
constexpr int kMaxVar = 5;
constexpr int kMaxLadder = 16;

// Device status bits recorded in the workspace header.
enum : int { kStatusNonphysical = 1, kStatusTimeout = 2 };

// Cutoff variants (teno_scheme of the C-ABI): the paper's LAD cutoff
// (eq. 3.1-3.4) and its comparison schemes -- a fixed C_T (TENO5), TENO5-A's
// sensor (eq. 2.16-2.18) and WENO-Z weights (tau_5 of eq. 2.12, no cutoff).
enum : int { kSchemeLad = 0, kSchemeTeno5 = 1, kSchemeTeno5A = 2, kSchemeWenoZ = 3 };

// TENO5-A's parameters (Sec. 2): alpha_1, alpha_2, C_r = 1/4 (so eta / C_r
// = 4 eta exactly) and eps = 0.9 C_r / (1 - 0.9 C_r) xi^2 with xi = 1e-3,
// evaluated in that order as in the formula (Scheme::eps_a).
constexpr double kTeno5AAlpha1 = 10.5, kTeno5AAlpha2 = 3.5, kTeno5ACr = 0.25, kTeno5AXi = 1e-3;

// Scheme constants, passed to kernels by value.
struct Scheme {
  int variant;    // kScheme*
  int m_fixed;    // kSchemeTeno5: C_T = 10^-m_fixed
  double eps_a;   // kSchemeTeno5A: eps of eq. 2.18
  double gamma;   // ratio of specific heats (eq. 4.7)
  double gm1;     // gamma - 1
  double eps;     // epsilon of eq. 2.8 / 3.2
  double eps4;    // 4 eps (the indicators are carried scaled by 4)
  int b_l, b_u;   // magnitude bounds of eq. 3.1
  int nthr;       // B_u - B_l
  int top;        // largest power of two <= nthr (binary-search start)
  unsigned keep_all;  // bit m set: every chi_k >= C_T is guaranteed at this m
  int keep_idx;   // keep_all = {m >= B_l + keep_idx + 1}: tau <= thr[keep_idx] dmin (-1: none)
  float thr_keep_f;   // thr[keep_idx] rounded down to binary32 (0: no FP32 pre-test)
  float eps4_f;       // 4 eps rounded down to binary32
  // m = B_l + #{ j in 1..B_u-B_l : tau <= thr[j-1] * min_k(beta_k + eps) }.
  // With theta = 1/(1 + max_k chi~_k / H) and max_k chi~_k = tau / min_k(beta_k
  // + eps) (eq. 3.2), floor(theta (B_u - B_l)) >= j  <=>  max chi~ <=
  // H ((B_u - B_l)/j - 1); the last threshold (theta == 1 exactly) is the
  // binary64 condition 1 + max chi~ / H == 1, i.e. max chi~ <= H 2^-53.
  // Entries past B_u - B_l are 0 (the count is clamped to B_u - B_l).
  double thr[kMaxLadder];
};

// entries per field of the fixed-state ghost block: one per face (2 d + side)
constexpr int kGhostSlots = 6;

struct Grid {
  int64_t n[3];
  int64_t ncell;
  int bc[3];           // 0 periodic, 1 transmissive, 2 reflecting, 3 fixed state
  double dx[3];
  double inv_dx[3];
  double rdx[3];       // dx[0] / dx[k] (exactly 1 for equal spacings)
  double grav[3] = {0.0, 0.0, 0.0};   // body acceleration of the source (0, rho g, rho u.g)
  int has_grav = 0;                    // grav is not zero
  // fixed-state (bc 3) ghost cells: state, primitives and half fluxes of the
  // virtual cells ncell + 2 d + side (see GhostCells)
  const double* gU = nullptr;
  const double* gaux = nullptr;
  const double* gfh = nullptr;
};

// Index of a (possibly ghost) cell along an axis of n cells: periodic wrap,
// zero-gradient copy of the boundary cell, or (bc 2, reflecting) the mirror
// image about the wall, cell -1-k for ghost k; `flip` is set when the point is
// a mirror image carrying the reversed normal velocity (an odd number of
// reflections -- more than one only on grids narrower than the stencil).
__device__ __forceinline__ int64_t ghost(int64_t i, int64_t n, int bc, bool& flip) {
  flip = false;
  if (bc == 0) {
    if (i < 0) i += n;
    else if (i >= n) i -= n;
    // a stencil reaches at most 3 cells outside; for n < 3 wrap again
    if (i < 0) i = ((i % n) + n) % n;
    else if (i >= n) i = i % n;
    return i;
  }
  if (bc == 2) {
    // at most 3 cells outside: a few reflections at most
    while (i < 0 || i >= n) {
      i = (i < 0) ? -1 - i : 2 * n - 1 - i;
      flip = !flip;
    }
    return i;
  }
  return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

__device__ __forceinline__ int64_t ghost(int64_t i, int64_t n, int bc) {
  bool flip;
  return ghost(i, n, bc, flip);
}

// x with its sign reversed when f (an integer-pipe sign-bit flip)
__device__ __forceinline__ double flip_sign(double x, bool f) {
  return __longlong_as_double(__double_as_longlong(x) ^ (static_cast<long long>(f) << 63));
}

// Non-negative doubles order like their bit patterns; used for max / compare
// on the integer pipe.
__device__ __forceinline__ unsigned long long dbits(double x) {
  return static_cast<unsigned long long>(__double_as_longlong(x));
}

// Integer-pipe tests and maxima on binary64 bit patterns (GB300's FP64 pipe
// is the scarce unit):
//   max_abs_bits(m, x) = bits of max(value(m), |x|) for m >= 0, skipping a NaN
//                        x as fmax does (non-negative doubles order as
//                        their bit patterns);
//   pos_finite(x)      = 0 < x < inf;
//   is_finite(x)       = x is neither inf nor NaN.
constexpr unsigned long long kExpMask = 0x7FF0000000000000ull;
__device__ __forceinline__ unsigned long long max_abs_bits(unsigned long long m, double x) {
  const unsigned long long b = dbits(x) & 0x7FFFFFFFFFFFFFFFull;
  return (b <= kExpMask && b > m) ? b : m;
}
__device__ __forceinline__ bool pos_finite(double x) {
  const long long b = __double_as_longlong(x);
  return b > 0 && b < static_cast<long long>(kExpMask);
}
__device__ __forceinline__ bool is_finite(double x) { return (dbits(x) & kExpMask) != kExpMask; }

// binary32 approximation of a double on the integer pipe (teno_cert.cuh):
// mantissa truncated to 20 bits, |f - x| < 2^-20 |x| in the normal range.
__device__ __forceinline__ float hi_float(double x) { return teno_cert::hi_float(x); }

// ---------------------------------------------------------------------------
// Reciprocal of a positive double with few FP64 instructions (GB300's FP64
// pipe is the scarce unit): a binary32 seed -- rcp.approx (PTX) of the
// operand truncated by hi_float, widened back exactly on the integer pipe --
// then one third-order step of the Householder iteration for 1/x:
//   e = 1 - x y0,  y = y0 + y0 (e + e^2)   (= (1 - e^3)/x),
// three FMAs against the several of a correctly rounded division.  The seed
// lies within 2^-19 of 1/x, so the step's truncation error is below 2^-55
// relative and the result is within one ulp of the correctly rounded value.
// Operands outside [2^-120, 2^120) -- and zero, negative, infinite or NaN
// ones -- take CUDA's division.  (A seeded reciprocal square root built the
// same way measured more FP64 instructions than CUDA's rsqrt, which stays.)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float rcp_approx_f32(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// binary32 -> binary64 by rebiasing the exponent (exact for normal values)
__device__ __forceinline__ double widen_normal(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned mag = b & 0x7fffffffu;
  return __hiloint2double(static_cast<int>((b & 0x80000000u) | ((mag >> 3) + (896u << 20))),
                          static_cast<int>(mag << 29));
}
// 2^-120 <= x < 2^120 (biased exponent 903..1142, sign clear)
__device__ __forceinline__ bool seed_range(double x) {
  const unsigned hi = static_cast<unsigned>(__double2hiint(x));
  return hi - (903u << 20) < (240u << 20);
}
__device__ __forceinline__ double recip_pos(double x) {
  if (!seed_range(x)) return 1.0 / x;
  const double y0 = widen_normal(rcp_approx_f32(hi_float(x)));
  const double e = fma(-x, y0, 1.0);
  return fma(y0, fma(e, e, e), y0);
}

// ---------------------------------------------------------------------------
// TENO5-A's magnitude m = floor(beta) (eq. 2.16-2.18) from the first
// differences e_k = v_{k+1} - v_k of the five stencil values: the sensor
//   eta_j = (2 |d+ d-| + eps) / ((d+)^2 + (d-)^2 + eps)
// at the stencil points 1, 2, 3 (i-1, i, i+1; d+- the differences on either
// side; the printed denominator repeats d+, read as d+ and d-), their
// minimum eta, m_A = 1 - min(1, eta / C_r), g = (1 - m_A)^4 (1 + 4 m_A),
// beta = alpha_1 - alpha_2 (1 - g).  Every operation is rounded as written
// (no contraction), so the magnitude equals a plain evaluation's bit for bit.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double teno5a_eta(double dp, double dm, double eps_a) {
  const double num = __dadd_rn(2.0 * fabs(__dmul_rn(dp, dm)), eps_a);
  const double den = __dadd_rn(__dadd_rn(__dmul_rn(dp, dp), __dmul_rn(dm, dm)), eps_a);
  return __ddiv_rn(num, den);
}

__device__ __forceinline__ int teno5a_magnitude(double e0, double e1, double e2, double e3, double eps_a) {
  const double eta = fmin(teno5a_eta(e1, e0, eps_a), fmin(teno5a_eta(e2, e1, eps_a), teno5a_eta(e3, e2, eps_a)));
  const double mA = __dsub_rn(1.0, fmin(1.0, __ddiv_rn(eta, kTeno5ACr)));
  const double t = __dsub_rn(1.0, mA);
  const double t2 = __dmul_rn(t, t);
  const double g = __dmul_rn(__dmul_rn(t2, t2), __dadd_rn(1.0, 4.0 * mA));
  const double beta = __dsub_rn(kTeno5AAlpha1, __dmul_rn(kTeno5AAlpha2, __dsub_rn(1.0, g)));
  return static_cast<int>(floor(beta));
}

// ---------------------------------------------------------------------------
// TENO5-LAD scalar reconstruction of the interface value from five values
// v0..v4 = (f_{i-2}, ..., f_{i+2}).  Returns acc + f^ (eq. 2.7); `flag`
// receives delta bits 0..2 and m in bits 3..6.
//
// Arithmetic (all exact rewrites of the paper's formulas, evaluated in FP64):
//  * with first differences e_k = v_{k+1} - v_k, the indicator terms of
//    eq. 2.9-2.11 are a_0 = e1 - e0, c_0 = 3 e1 - e0, a_1 = e2 - e1,
//    c_1 = -(e1 + e2), a_2 = e3 - e2, c_2 = e3 - 3 e2, and the weighted sum
//    of the candidate fluxes (eq. 2.4-2.7) is sum_j c_lin[sel][j] v_j;
//  * m of eq. 3.1 counts the thresholds tau <= thr_j * min_k(beta_k + eps)
//    (see Scheme), found by binary search over the decreasing thresholds;
//  * the cutoff chi_k >= C_T of eq. 2.13-2.14 is decided without division:
//    with D_k = beta_k + eps and N_k = D_k + tau, gamma_k (D0 D1 D2)^6 =
//    (N_k prod_{j!=k} D_j)^6 =: P_k^6, so chi_k >= C_T <=> P_k^6 >= C_T sum P^6;
//  * when max chi~ is small enough that chi_k >= 1/(3 (1 + max chi~)^6) > C_T
//    holds for every k (Scheme::keep_all), all stencils are kept without
//    evaluating gamma.
// ---------------------------------------------------------------------------
template <bool WITH_M>
__device__ __forceinline__ double teno5_lad(double v0, double v1, double v2,
                                            double v3, double v4, double acc,
                                            const Scheme& S, unsigned& flag) {
  if (!WITH_M && S.keep_idx >= 0 &&
      teno_cert::certify_keep_values(v0, v1, v2, v3, v4, S.thr_keep_f, S.eps4_f)) {
    // Certified single-precision pre-test (teno_cert.cuh): the exact values
    // satisfy tau <= thr[keep_idx] * dmin with margin, so the binary64 test
    // below and the bound of Scheme::keep_all would both keep every stencil.
    flag = 7u;
    return fma(c_lin[7][0], v0, fma(c_lin[7][1], v1, fma(c_lin[7][2], v2, fma(c_lin[7][3], v3, fma(c_lin[7][4], v4, acc)))));
  }
  const double e0 = v1 - v0, e1 = v2 - v1, e2 = v3 - v2, e3 = v4 - v3;
  // eq. 2.9-2.11 scaled by 4: 4 beta_k = (13/3) a_k^2 + c_k^2.  Every use of
  // beta_k below is through ratios tau / (beta_k + eps) and products that are
  // homogeneous in (beta, tau, eps), so the common factor 4 (with eps -> 4 eps)
  // leaves m and delta unchanged.
  const double k13_3 = 13.0 / 3.0;
  const double a0 = e1 - e0, a1 = e2 - e1, a2 = e3 - e2;
  const double c0 = fma(3.0, e1, -e0);
  const double c1 = e1 + e2;
  const double c2 = fma(-3.0, e2, e3);
  const double beta0 = fma(k13_3 * a0, a0, c0 * c0);
  const double beta1 = fma(k13_3 * a1, a1, c1 * c1);
  const double beta2 = fma(k13_3 * a2, a2, c2 * c2);
  // eq. 2.12 (scaled)
  const double tau = fabs(beta2 - beta0);
  // eq. 3.1-3.2: m = B_l + #{j : tau <= thr_j * min_k D_k}, D_k = beta_k + eps
  const unsigned long long bmin = min(dbits(beta0), min(dbits(beta1), dbits(beta2)));
  const double dmin = __longlong_as_double(static_cast<long long>(bmin)) + S.eps4;
  const unsigned long long btau = dbits(tau);
  unsigned sel = 7u;
  int m = S.b_u;
  if (S.variant == kSchemeWenoZ) {
    // WENO-Z: omega_k = a_k / sum_j a_j with a_k = c_k (1 + tau / D_k),
    // D_k = beta_k + eps (the common factor 4 cancels); with N_k = D_k + tau
    // and A_k = c_k N_k prod_{j != k} D_j = a_k D_0 D_1 D_2, omega_k =
    // A_k / sum A (one division; three where the products leave the range)
    const double d0 = beta0 + S.eps4, d1 = beta1 + S.eps4, d2 = beta2 + S.eps4;
    double A0 = 0.1 * (d0 + tau) * (d1 * d2), A1 = 0.6 * (d1 + tau) * (d0 * d2), A2 = 0.3 * (d2 + tau) * (d0 * d1);
    double As = A0 + A1 + A2;
    if (!(As > 0.0 && As <= 1.7976931348623157e308)) {
      A0 = 0.1 * (1.0 + tau / d0);
      A1 = 0.6 * (1.0 + tau / d1);
      A2 = 0.3 * (1.0 + tau / d2);
      As = A0 + A1 + A2;
    }
    const double r = 1.0 / As;
    const double o0 = A0 * r, o1 = A1 * r, o2 = A2 * r;
    flag = 7u;
    // f^ = v2 + sum_k w_k e_k (see c_coef)
    const double w0 = o0 * (-1.0 / 3.0), w1 = fma(o0, 5.0 / 6.0, o1 * (1.0 / 6.0));
    const double w2 = fma(o1, 1.0 / 3.0, o2 * (2.0 / 3.0)), w3 = o2 * (-1.0 / 6.0);
    return fma(w0, e0, fma(w1, e1, fma(w2, e2, fma(w3, e3, v2 + acc))));
  }
  if (!WITH_M && S.keep_idx >= 0 && btau <= dbits(S.thr[S.keep_idx] * dmin)) {
    // tau below the keep-all threshold: every stencil is kept (for LAD, m
    // lies in the keep-all range, a suffix of B_l..B_u; for TENO5 and
    // TENO5-A, chi_k >= 1/(3 (1 + max chi~)^6) exceeds the largest C_T)
    flag = 7u;
  } else {
    if (S.variant == kSchemeLad) {
      int cnt = 0;
#pragma unroll
      for (int step = 8; step >= 1; step >>= 1) {
        if (step <= S.top) {
          const int idx = cnt + step - 1;
          if (btau <= dbits(S.thr[idx] * dmin)) cnt += step;
        }
      }
      cnt = min(cnt, S.nthr);
      m = S.b_l + cnt;
    } else if (S.variant == kSchemeTeno5) {
      m = S.m_fixed;
    } else {
      m = teno5a_magnitude(e0, e1, e2, e3, S.eps_a);
    }
    if (!((S.keep_all >> m) & 1u)) {
      // eq. 3.4, eq. 2.8, eq. 2.13-2.14 (division-free form, see above)
      const double ct = c_lad[m];
      const double d0 = beta0 + S.eps4, d1 = beta1 + S.eps4, d2 = beta2 + S.eps4;
      const double n0 = d0 + tau, n1 = d1 + tau, n2 = d2 + tau;
      const double p0 = n0 * (d1 * d2), p1 = n1 * (d0 * d2), p2 = n2 * (d0 * d1);
      double q0 = p0 * p0, q1 = p1 * p1, q2 = p2 * p2;
      q0 = q0 * q0 * q0;
      q1 = q1 * q1 * q1;
      q2 = q2 * q2 * q2;
      const double sum = q0 + q1 + q2;
      if (sum > 0.0 && sum <= 1.7976931348623157e308) {
        const unsigned long long lim = dbits(ct * sum);
        sel = (dbits(q0) >= lim ? 1u : 0u) | (dbits(q1) >= lim ? 2u : 0u) |
              (dbits(q2) >= lim ? 4u : 0u);
      } else {
        // outside the range of the products: gamma_k = (1 + tau/D_k)^6 directly
        const double x0 = 1.0 + tau / d0, x1 = 1.0 + tau / d1, x2 = 1.0 + tau / d2;
        double h0 = x0 * x0 * x0, h1 = x1 * x1 * x1, h2 = x2 * x2 * x2;
        h0 *= h0;
        h1 *= h1;
        h2 *= h2;
        const double gs = h0 + h1 + h2;
        const unsigned long long lim = dbits(ct * gs);
        sel = (dbits(h0) >= lim ? 1u : 0u) | (dbits(h1) >= lim ? 2u : 0u) |
              (dbits(h2) >= lim ? 4u : 0u);
        if (!(gs <= 1.7976931348623157e308)) sel = 7u;  // every chi_k undefined: keep all
      }
    }
    flag = sel | (static_cast<unsigned>(m) << 3);
  }
  // eq. 2.4-2.7 with the weights of eq. 2.15 (c_lin)
  return fma(c_lin[sel][0], v0, fma(c_lin[sel][1], v1, fma(c_lin[sel][2], v2, fma(c_lin[sel][3], v3, fma(c_lin[sel][4], v4, acc)))));
}

}  // namespace teno
