// teno_cert.cuh -- certified single-precision test that a TENO5
// reconstruction keeps every stencil (delta_k = 1 for k = 0, 1, 2 in
// eq. 2.14), for host and device.
//
// GB300's FP64 rate is 1/64 of its FP32 rate, so the flux passes first ask
// FP32 whether the binary64 evaluation would keep every stencil, and only
// evaluate the indicators in binary64 when FP32 cannot prove it.  A test
// here passes only if, for the exact values x_j that the FP32 inputs
// approximate, the scaled indicators (4 beta_k of eq. 2.9-2.11, 4 tau_5 of
// eq. 2.12) satisfy
//     tau_5(x) <= thr * (min_k beta_k(x) + eps) * (1 - 1e-5 + 8 u),
// where thr is the threshold below which the cutoff keeps every stencil
// (Scheme::thr_keep_f).  The margin of about 1e-5 is 2^28 times the rounding
// of a binary64 evaluation of the same quantities (whose errors are at most
// 2^-28 of the FP32 bounds below), so the binary64 decision -- the GPU's and
// the oracle's -- is "keep every stencil" whenever a test passes.
//
// Every FP32 operation is written with its rounding explicit (fadd, fsub,
// fmul, ffma: round to nearest, no contraction), so that the host build (used
// by the CPU tests, compiled with -ffp-contract=off) evaluates bit for bit
// what the device evaluates.  u = 2^-24 is the FP32 unit roundoff.
#pragma once

#include <math.h>

#include <cmath>
#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define TENO_CERT_HD __host__ __device__ __forceinline__
#else
#define TENO_CERT_HD inline
#endif

namespace teno_cert {

TENO_CERT_HD float fadd(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
TENO_CERT_HD float fsub(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}
TENO_CERT_HD float fmul(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
TENO_CERT_HD float ffma(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return std::fmaf(a, b, c);
#endif
}
// fabsf, fminf, fmaxf (exact; NaN-ignoring min/max on both sides) are the
// C library's on the host and CUDA's on the device.

// binary32 approximation of a double built from its high word with integer
// operations only: exponent rebiased, mantissa truncated to 20 bits, so
// |f| <= |x| and |f - x| < 2^-20 |x| for 2^-126 <= |x| < 2^128.  Smaller
// magnitudes become 2^-126 (error below 2^-126); larger ones, infinities and
// NaN become the largest value below 2^128 (their squares overflow, so no
// test below can pass on them).
TENO_CERT_HD float hi_float(double x) {
#ifdef __CUDA_ARCH__
  const unsigned hi = static_cast<unsigned>(__double2hiint(x));
#else
  uint64_t b;
  std::memcpy(&b, &x, sizeof(b));
  const unsigned hi = static_cast<unsigned>(b >> 32);
#endif
  unsigned mag = hi & 0x7fffffffu;
  mag = mag < (897u << 20) ? (897u << 20) : mag;
  mag = mag > ((1150u << 20) | 0xFFFFFu) ? ((1150u << 20) | 0xFFFFFu) : mag;
  const unsigned bits = ((mag - (896u << 20)) << 3) | (hi & 0x80000000u);
#ifdef __CUDA_ARCH__
  return __uint_as_float(bits);
#else
  float f;
  std::memcpy(&f, &bits, sizeof(f));
  return f;
#endif
}

// ---------------------------------------------------------------------------
// certify_keep: v0..v4 are FP32 values with |v_j - x_j| <= r, the test is
// given d with
//     d >= (1 + 2^-19) (r + 2 u W),   d >= 2^-21 W,   W = max |v_j|.
//
// Error budget:
//  * first differences e_k = v_{k+1} - v_k: |e| <= 2W, so each rounds by at
//    most 2uW and |e^ - e(x)| <= 2 r + 2uW;
//  * a_0 = e_1 - e_0 (|.| <= 4W, rounding 4uW) and c_0 = 3 e_1 - e_0 (one
//    rounding, |.| <= 8W): |a^ - a(x)| <= 4 (r + 2uW), |c^ - c(x)| <=
//    8 (r + 2uW); likewise a_1, a_2, c_1, c_2.  Hence |da| <= 4 d and
//    |dc| <= 8 d;
//  * 4 beta = (13/3) a^2 + c^2 from a^, c^ differs from its value at (a, c)
//    by at most (13/3)(2|a^| + 4d) 4d + (2|c^| + 8d) 8d, and its own FP32
//    evaluation (13/3 rounded, one product, one fma) by at most 3.02 u beta^:
//    4 u beta^ is charged;
//  * the (at most six) roundings of each error bound's own evaluation are
//    covered by the 2^-19 = 32 u of slack in d;
//  * dmin = min beta^ + eps (eps rounded down) is within max_k dbeta_k +
//    u dmin of the exact value; 4 u dmin is charged, which also covers the
//    rounding of that sum;
//  * the final comparison's own roundings (a few u) sit inside the 1e-5
//    margin;
//  * an overflow anywhere implies W > 2^125, so d > 2^104 and (4d)^2
//    overflows: dtau is then infinite or NaN and the test fails.
// ---------------------------------------------------------------------------
TENO_CERT_HD bool certify_keep(float v0, float v1, float v2, float v3, float v4, float d, float thr_f,
                               float eps4_f) {
  const float u = 0x1p-24f;
  const float e0 = fsub(v1, v0), e1 = fsub(v2, v1), e2 = fsub(v3, v2), e3 = fsub(v4, v3);
  const float a0 = fsub(e1, e0), a1 = fsub(e2, e1), a2 = fsub(e3, e2);
  const float c0 = ffma(3.0f, e1, -e0), c1 = fadd(e1, e2), c2 = ffma(-3.0f, e2, e3);
  const float k = 13.0f / 3.0f;
  const float b0 = ffma(fmul(k, a0), a0, fmul(c0, c0));
  const float b1 = ffma(fmul(k, a1), a1, fmul(c1, c1));
  const float b2 = ffma(fmul(k, a2), a2, fmul(c2, c2));
  const float da = 4.0f * d, dc = 8.0f * d;   // exact scalings
  const float db0 = ffma(4.0f * u, b0, ffma(fmul(k, ffma(2.0f, fabsf(a0), da)), da, fmul(ffma(2.0f, fabsf(c0), dc), dc)));
  const float db1 = ffma(4.0f * u, b1, ffma(fmul(k, ffma(2.0f, fabsf(a1), da)), da, fmul(ffma(2.0f, fabsf(c1), dc), dc)));
  const float db2 = ffma(4.0f * u, b2, ffma(fmul(k, ffma(2.0f, fabsf(a2), da)), da, fmul(ffma(2.0f, fabsf(c2), dc), dc)));
  const float tau = fabsf(fsub(b2, b0));
  const float dtau = ffma(u, tau, fadd(db0, db2));
  const float dmin = fadd(fminf(b0, fminf(b1, b2)), eps4_f);
  const float ddmin = ffma(4.0f * u, dmin, fmaxf(db0, fmaxf(db1, db2)));
  return (dtau <= 1.0e38f) && (fadd(tau, dtau) <= fmul(thr_f, fmul(fsub(dmin, ddmin), 1.0f - 1e-5f)));
}

// The same test on five binary64 values (one scalar reconstruction),
// truncated by hi_float: |g_j - v_j| <= 2^-20 |v_j| + 2^-126 and
// |v_j| <= |g_j| (1 + 2^-19), so r + 2uW <= 0x1.2p-20 W + 2^-126 (plus
// terms of order 2^-39 W); d = 0x1.3p-20 W + 2^-125 leaves more than 5 %
// of slack, which covers 2^-19 and the rounding of d itself.
TENO_CERT_HD bool certify_keep_values(double v0, double v1, double v2, double v3, double v4, float thr_f,
                                      float eps4_f) {
  const float g0 = hi_float(v0), g1 = hi_float(v1), g2 = hi_float(v2), g3 = hi_float(v3), g4 = hi_float(v4);
  const float W = fmaxf(fmaxf(fmaxf(fabsf(g0), fabsf(g1)), fmaxf(fabsf(g2), fabsf(g3))), fabsf(g4));
  return certify_keep(g0, g1, g2, g3, g4, ffma(0x1.3p-20f, W, 0x1p-125f), thr_f, eps4_f);
}

// ---------------------------------------------------------------------------
// The test for all 2 nvar reconstructions of one Euler interface.
// cert_begin takes the interface's Roe state (u~, b1/2, b2/2, 1/(2c)) and the
// halved Lax-Friedrichs speeds; cert_point takes one stencil point (its state
// U_j and half u_d, p) to FP32 split characteristic values v+-[j] together
// with the FP32 evaluation of the same expressions on absolute values
// (mp, mm: bounds of the terms that enter each value); cert_keep runs
// certify_keep on every field and side.
//
// Each split value is a sum of products of at most four truncated inputs
// (e.g. (u_d/2 + alpha) b1/2 u~_k U_j) through at most nine FP32 roundings,
// so |v32 - v| <= (4 2^-20 + 9 u)(1 + 2^-18) |.|_abs < 4.6 2^-20 |.|_abs,
// |.|_abs being the absolute evaluation (which the FP32 one approximates
// from below by at most the same relative amount).  Inputs below 2^-126 add
// an absolute error below 2^-100 for any physical scale.  cert_keep passes
// d = 8 2^-20 |.|_abs + 8 u max|v| + 2^-100, more than 1.7 times the
// r + 2 u W that certify_keep needs, and at least 2^-21 W.
// ---------------------------------------------------------------------------
template <int NDIM>
struct CertIfc {
  float uf[NDIM], hb1f, hb2f, hicf, b1f, hudf, haf[NDIM + 2];
  float vp32[6][NDIM + 2], vm32[6][NDIM + 2], mp[NDIM + 2], mm[NDIM + 2], vmax;
};

template <int NDIM, int DIR>
TENO_CERT_HD void cert_begin(const double (&u)[NDIM], double hb1, double hb2, double hic,
                             const double (&alpha)[NDIM + 2], CertIfc<NDIM>& C) {
  constexpr int NVAR = NDIM + 2;
#pragma unroll
  for (int k = 0; k < NDIM; ++k) C.uf[k] = hi_float(u[k]);
  C.hb1f = hi_float(hb1);
  C.hb2f = hi_float(hb2);
  C.hicf = hi_float(hic);
  // b1 = 2 (b1/2) and u_d/2 from the truncated values (exact scalings: the
  // same 2^-20 relative bound)
  C.b1f = 2.0f * C.hb1f;
  C.hudf = 0.5f * C.uf[DIR];
#pragma unroll
  for (int f = 0; f < NVAR; ++f) {
    C.haf[f] = hi_float(alpha[f]);
    C.mp[f] = C.mm[f] = 0.0f;
  }
  C.vmax = 0.0f;
}

// Point j: U_j (binary64 state, normal momentum already mirrored at a wall),
// unj = u_d/2, pnj = p/2.  The split values follow the binary64
// characteristic path: w = L U_j, t = (p/2) z, v+ = (u_d/2 + alpha) w + t,
// v- = v+ - 2 alpha w.
template <int NDIM, int DIR>
TENO_CERT_HD void cert_point(int j, const double (&Uj)[NDIM + 2], double unj, double pnj, CertIfc<NDIM>& C) {
  constexpr int NVAR = NDIM + 2;
  float X[NVAR], Xa[NVAR];
#pragma unroll
  for (int v = 0; v < NVAR; ++v) {
    X[v] = hi_float(Uj[v]);
    Xa[v] = fabsf(X[v]);
  }
  float Sv = -X[NVAR - 1], Sa = Xa[NVAR - 1];
#pragma unroll
  for (int k = 0; k < NDIM; ++k) {
    Sv = ffma(C.uf[k], X[1 + k], Sv);
    Sa = ffma(fabsf(C.uf[k]), Xa[1 + k], Sa);
  }
  const float A = ffma(C.hb2f, X[0], -fmul(C.hb1f, Sv));
  const float Aa = ffma(fabsf(C.hb2f), Xa[0], fmul(fabsf(C.hb1f), Sa));
  const float B = fmul(ffma(C.uf[DIR], X[0], -X[1 + DIR]), C.hicf);
  const float Ba = fmul(ffma(fabsf(C.uf[DIR]), Xa[0], Xa[1 + DIR]), fabsf(C.hicf));
  float w[NVAR], wa[NVAR];
  w[0] = fadd(A, B);
  wa[0] = fadd(Aa, Ba);
  w[1] = ffma(-2.0f, A, X[0]);
  wa[1] = ffma(2.0f, Aa, Xa[0]);
  {
    int f = 2;
#pragma unroll
    for (int t = 0; t < NDIM; ++t) {
      if (t == DIR) continue;
      w[f] = ffma(-C.uf[t], X[0], X[1 + t]);
      wa[f] = ffma(fabsf(C.uf[t]), Xa[0], Xa[1 + t]);
      ++f;
    }
  }
  w[NVAR - 1] = fsub(A, B);
  wa[NVAR - 1] = fadd(Aa, Ba);
  const float huf = hi_float(unj), hpf = hi_float(pnj);
  const float az = fmul(hpf, fmul(C.b1f, fsub(huf, C.hudf)));
  const float aza = fmul(fabsf(hpf), fmul(fabsf(C.b1f), fadd(fabsf(huf), fabsf(C.hudf))));
  const float bz = fmul(hpf, C.hicf), bza = fmul(fabsf(hpf), fabsf(C.hicf));
#pragma unroll
  for (int f = 0; f < NVAR; ++f) {
    const float t = (f == 0) ? fsub(az, bz) : (f == NVAR - 1) ? fadd(az, bz) : (f == 1) ? -2.0f * az : 0.0f;
    const float ta = (f == 0 || f == NVAR - 1) ? fadd(aza, bza) : (f == 1) ? 2.0f * aza : 0.0f;
    C.vp32[j][f] = ffma(fadd(huf, C.haf[f]), w[f], t);
    C.vm32[j][f] = ffma(-2.0f * C.haf[f], w[f], C.vp32[j][f]);
    const float pa = ffma(fadd(fabsf(huf), C.haf[f]), wa[f], ta);
    const float ma = ffma(2.0f * C.haf[f], wa[f], pa);
    if (j <= 4) C.mp[f] = fmaxf(C.mp[f], pa);
    if (j >= 1) C.mm[f] = fmaxf(C.mm[f], ma);
    C.vmax = fmaxf(C.vmax, fmaxf(fabsf(C.vp32[j][f]), fabsf(C.vm32[j][f])));
  }
}

template <int NDIM>
TENO_CERT_HD bool cert_keep(const CertIfc<NDIM>& C, float thr_f, float eps4_f) {
  constexpr int NVAR = NDIM + 2;
  const float kd = 8.0f * 0x1p-20f;
  const float ku = ffma(8.0f * 0x1p-24f, C.vmax, 0x1p-100f);
  bool keep = true;
#pragma unroll
  for (int f = 0; f < NVAR; ++f) {
    keep = keep && certify_keep(C.vp32[0][f], C.vp32[1][f], C.vp32[2][f], C.vp32[3][f], C.vp32[4][f],
                                ffma(kd, C.mp[f], ku), thr_f, eps4_f);
    keep = keep && certify_keep(C.vm32[5][f], C.vm32[4][f], C.vm32[3][f], C.vm32[2][f], C.vm32[1][f],
                                ffma(kd, C.mm[f], ku), thr_f, eps4_f);
  }
  return keep;
}

}  // namespace teno_cert
