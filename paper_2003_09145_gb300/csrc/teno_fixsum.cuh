// teno_fixsum.cuh -- the closed form's six-point sums with integer weights
// (and the adjoint's sums of the same kind), evaluated in 64-bit fixed point
// on the integer pipes, for host and device.
//
// Where every stencil is kept, the interface flux needs per component two
// sums S = sum_j w_j x_j over the six stencil points, with the integer
// weights c = (1, -8, 37, 37, -8, 1) (the fifth-order upwind and downwind
// reconstructions of eq. 2.3 added) and m = (1, -5, 10, -10, 5, -1) (their
// difference); sum_j |w_j| <= 92 < 2^7.  GB300 issues binary64 at 1/64 of
// its binary32 rate while its integer pipes are mostly idle, so such sums can
// run in fixed point instead of as chains of FP64 fused multiply-adds:
//
//  * E is the largest biased exponent among the six values;
//  * value j becomes the integer X_j = sign(x_j) trunc(|x_j| 2^(1075+G-E)):
//    its 53-bit significand with G = 3 guard bits, aligned to the largest
//    value (|X_j| < 2^56; a zero or subnormal value gives 0 once E >= 64);
//  * A = sum_j w_j X_j is exact in int64 (|A| < 92 2^56 < 2^63);
//  * the sum is A 2^(E - 1075 - G), rounded once to nearest-even binary64.
//
// Besides that one rounding, the only error is each value's truncation below
// 2^(E - 1075 - G), an eighth of the largest value's ulp: at most
// (sum |w|)/8 = 11.5 of its ulps in all.  A binary64 chain of the same sum
// rounds each of five partial sums, as large as 92 times the largest value,
// by up to half of its own ulp, i.e. up to 64 ulps of the largest value each.
// The fixed-point sum does not depend on the order of its terms, and negating
// every value negates it exactly.
//
// The fixed point covers E = 0 (all six values zero or below 2^-1022: the
// sum is taken as 0, an absolute error below 92 * 2^-1022) and
// 64 <= E <= 2030 (the result is then a normal number, and zeros and
// subnormals shift out).  Outside that range (values below 2^-959 or
// above 2^1007, infinities, NaN) callers take a binary64 evaluation.
#pragma once

#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define TENO_FIX_HD __host__ __device__ __forceinline__
#else
#define TENO_FIX_HD inline
#endif

namespace teno_fix {

constexpr int kGuard = 3;
constexpr uint32_t kEmin = 64u, kEmax = 2030u;

TENO_FIX_HD uint32_t hi_word(double x) {
#ifdef __CUDA_ARCH__
  return static_cast<uint32_t>(__double2hiint(x));
#else
  uint64_t b;
  std::memcpy(&b, &x, sizeof(b));
  return static_cast<uint32_t>(b >> 32);
#endif
}

TENO_FIX_HD uint32_t lo_word(double x) {
#ifdef __CUDA_ARCH__
  return static_cast<uint32_t>(__double2loint(x));
#else
  uint64_t b;
  std::memcpy(&b, &x, sizeof(b));
  return static_cast<uint32_t>(b);
#endif
}

TENO_FIX_HD double from_bits(uint64_t b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double(static_cast<long long>(b));
#else
  double x;
  std::memcpy(&x, &b, sizeof(x));
  return x;
#endif
}

TENO_FIX_HD int clz64(uint64_t a) {
#ifdef __CUDA_ARCH__
  return __clzll(static_cast<long long>(a));
#else
  return a ? __builtin_clzll(a) : 64;
#endif
}

// Magnitude key of a value from its high word: the high word without its
// sign, so that key >> 20 is the biased exponent.  E of a sum is the largest
// key's exponent.
TENO_FIX_HD uint32_t key(uint32_t hi) { return hi & 0x7FFFFFFFu; }
TENO_FIX_HD uint32_t exponent(uint32_t key_max) { return key_max >> 20; }

// whether the fixed point covers a sum whose largest exponent is E
TENO_FIX_HD bool in_range(uint32_t E) { return E == 0u || E - kEmin <= kEmax - kEmin; }

// X = sign(x) trunc(|x| 2^(1075 + G - E)) for a value whose exponent is at
// most E.  (Shifting first and multiplying by the weight afterwards measured
// faster on GB300 than multiplying the significand first.)
TENO_FIX_HD int64_t term(double x, uint32_t E) {
  const uint32_t hi = hi_word(x);
  const uint32_t sh = E - ((hi >> 20) & 0x7FFu);
  const uint64_t M = ((static_cast<uint64_t>((hi & 0xFFFFFu) | 0x100000u) << 32) | lo_word(x)) << kGuard;
  const uint64_t X = M >> (sh < 63u ? sh : 63u);
  return static_cast<int32_t>(hi) < 0 ? -static_cast<int64_t>(X) : static_cast<int64_t>(X);
}

// A += w X for a weight |w| <= 37
TENO_FIX_HD void add(int64_t& A, double x, uint32_t E, int w) { A += static_cast<int64_t>(w) * term(x, E); }

// A 2^(E - 1075 - G) rounded to nearest-even binary64 (E in range).  On the
// device with TENO_FIX_ROUND_CVT the rounding is the hardware conversion
// (cvt.rn.f64.s64, the same round-to-nearest-even of the same integer),
// then the power of two is added to the exponent field: the converted |A| is
// at least 1, so the result's exponent E - 55 .. E + 7 stays normal.
#ifndef TENO_FIX_ROUND_CVT
#define TENO_FIX_ROUND_CVT 0
#endif
TENO_FIX_HD double round(int64_t A, uint32_t E) {
#if defined(__CUDA_ARCH__) && TENO_FIX_ROUND_CVT
  const double d = __ll2double_rn(static_cast<long long>(A));
  const int hi = __double2hiint(d) + static_cast<int>((E - 1075u - kGuard) << 20);
  return (E == 0u || A == 0) ? 0.0 : __hiloint2double(hi, __double2loint(d));
#endif
  if (E == 0u || A == 0) return 0.0;
  const uint64_t s = A < 0 ? 1u : 0u;
  const uint64_t a = A < 0 ? uint64_t(0) - static_cast<uint64_t>(A) : static_cast<uint64_t>(A);
  const int lz = clz64(a);                 // 1..63: |A| < 2^63
  const uint64_t n = a << lz;              // leading bit at 2^63
  uint64_t m = n >> 11;                    // 53-bit significand
  const uint64_t r = n & 0x7FFu;           // half-ulp bit and sticky bits
  m += (r > 0x400u || (r == 0x400u && (m & 1u))) ? 1u : 0u;
  // value = m 2^(b - 1075) with b = E + 11 - G - lz; the significand's
  // leading bit (and a carry to 2^53) adds to the exponent field
  const uint64_t b = static_cast<uint64_t>(E) + 11u - kGuard - static_cast<uint64_t>(lz);
  return from_bits(((b - 1u) << 52) + m + (s << 63));
}

// sum_k w_k x_k of n values in fixed point, for weights with sum_k |w_k| < 128
// (so |A| < 2^63): false, with `out` untouched, where the fixed point does not
// cover the values
template <int N>
TENO_FIX_HD bool sum(const double (&x)[N], const int (&w)[N], double& out) {
  uint32_t kmax = 0;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const uint32_t kk = key(hi_word(x[k]));
    kmax = kk > kmax ? kk : kmax;
  }
  const uint32_t E = exponent(kmax);
  if (!in_range(E)) return false;
  int64_t A = 0;
#pragma unroll
  for (int k = 0; k < N; ++k) add(A, x[k], E, w[k]);
  out = round(A, E);
  return true;
}

}  // namespace teno_fix
