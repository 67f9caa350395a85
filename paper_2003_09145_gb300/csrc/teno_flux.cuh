// teno_flux.cuh -- the numerical flux at one interface (device function shared
// by the grid kernels and the batched kernel).  FP64 throughout.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "teno_device.cuh"
#include "teno_fixsum.cuh"

namespace teno {

// Fixed-state (Dirichlet) ghost cells: a stencil point outside a Dirichlet
// face is the virtual cell ncell + 2 d + side; its state, primitives and half
// fluxes sit in small blocks laid out like the cell arrays with
// kGhostSlots entries per field (U [nvar][6], aux [aux_fields][6],
// fh [ndim][nvar - 1][6]), filled by the cell pass of the fixed states.
struct GhostCells {
  const double* U = nullptr;
  const double* aux = nullptr;
  const double* fh = nullptr;
};

// field `f` of cell c of an array with ncell entries per field, or of the
// ghost block when GH and c is a virtual cell
template <bool GH>
__device__ __forceinline__ double ldc(const double* __restrict__ a, const double* __restrict__ ga, int64_t ncell,
                                      int64_t f, int64_t c) {
  if (GH && c >= ncell) return ga[f * kGhostSlots + (c - ncell)];
  return a[f * ncell + c];
}

// the high word of the same entry (sign, exponent, top of the significand)
template <bool GH>
__device__ __forceinline__ uint32_t ldc_hi(const double* __restrict__ a, const double* __restrict__ ga,
                                           int64_t ncell, int64_t f, int64_t c) {
  const double* p = (GH && c >= ncell) ? ga + f * kGhostSlots + (c - ncell) : a + f * ncell + c;
  return reinterpret_cast<const uint32_t*>(p)[1];
}

// Characteristic projection of one vector X (conservative ordering) onto the
// left eigenvectors of the Roe state (reading of the convective-term
// paragraph of Sec. 4; rows as in the library's design notes):
//   l_0 X = A + B,  l_{nvar-1} X = A - B,  l_1 X = X_0 - 2A,
//   l_t X = X_{1+t} - u_t X_0 (shear, t != DIR),
// with A = (b2 X_0 - b1 (u . X_mom - X_E)) / 2 and B = (u_n X_0 - X_{1+n})/(2c).
template <int NDIM, int DIR>
__device__ __forceinline__ void project(const double (&X)[NDIM + 2],
                                        const double (&u)[NDIM], double hb1,
                                        double hb2, double hic,
                                        double (&w)[NDIM + 2]) {
  constexpr int NVAR = NDIM + 2;
  double S = -X[NVAR - 1];
#pragma unroll
  for (int k = 0; k < NDIM; ++k) S = fma(u[k], X[1 + k], S);
  double A = fma(hb2, X[0], -hb1 * S);
  double B = fma(u[DIR], X[0], -X[1 + DIR]) * hic;
  w[0] = A + B;
  w[1] = fma(-2.0, A, X[0]);
  int f = 2;
#pragma unroll
  for (int t = 0; t < NDIM; ++t) {
    if (t == DIR) continue;
    w[f] = fma(-u[t], X[0], X[1 + t]);
    ++f;
  }
  w[NVAR - 1] = A - B;
}

// ---------------------------------------------------------------------------
// Roe state of the interface i+1/2 from the per-cell primitives of cells i
// and i+1 (sqrt(rho), (E+p)/sqrt(rho) and su = sqrt(rho) u = m/sqrt(rho)):
// u~ = (sr_a u_a + sr_b u_b)/(sr_a + sr_b), H~ = (sh_a + sh_b)/(sr_a + sr_b),
// c~^2 = (gamma-1)(H~ - |u~|^2/2), b1 = (gamma-1)/c~^2, b2 = b1 |u~|^2/2.
// ---------------------------------------------------------------------------
template <int NDIM>
struct RoeIfc {
  double u[NDIM], q2, H, cs, b1, hb1, hb2, hic, hud;
};

template <int NDIM, int DIR>
__device__ __forceinline__ void roe_interface(double sr2, double sr3, double sh2, double sh3,
                                              const double (&su2)[NDIM], const double (&su3)[NDIM],
                                              const Scheme& S, RoeIfc<NDIM>& R, int* __restrict__ status) {
  const double y = recip_pos(sr2 + sr3);
  R.q2 = 0.0;
#pragma unroll
  for (int k = 0; k < NDIM; ++k) {
    R.u[k] = (su2[k] + su3[k]) * y;
    R.q2 = fma(R.u[k], R.u[k], R.q2);
  }
  R.H = (sh2 + sh3) * y;
  const double c2 = S.gm1 * fma(-0.5, R.q2, R.H);
  if (!(c2 > 0.0)) atomicOr(status, kStatusNonphysical);
  const double ic = rsqrt(c2);
  R.cs = c2 * ic;
  // the halved coefficients directly (the factors 1/2 are exact); b1 and
  // hud only for the characteristic path, which reads them
  R.hb1 = (0.5 * S.gm1) * ic * ic;
  R.b1 = R.hb1 + R.hb1;
  R.hb2 = 0.5 * (R.hb1 * R.q2);
  R.hic = 0.5 * ic;
  R.hud = 0.5 * R.u[DIR];
}

// Certified FP32 test that all ten reconstructions of the interface keep
// every stencil: teno_cert.cuh (cert_begin, cert_point, cert_keep).
using teno_cert::CertIfc;

template <int NDIM, int DIR>
__device__ __forceinline__ void cert_begin(const RoeIfc<NDIM>& R, const double (&alpha)[NDIM + 2],
                                           CertIfc<NDIM>& C) {
  teno_cert::cert_begin<NDIM, DIR>(R.u, R.hb1, R.hb2, R.hic, alpha, C);
}

using teno_cert::cert_point;

template <int NDIM>
__device__ __forceinline__ bool cert_keep(const CertIfc<NDIM>& C, const Scheme& S) {
  return teno_cert::cert_keep<NDIM>(C, S.thr_keep_f, S.eps4_f);
}

// ---------------------------------------------------------------------------
// Every stencil kept at every field and side: closed form.  With fixed linear
// weights the characteristic reconstruction is
//   F^ = R [ L sum_j P_j F_j + diag(alpha) L sum_j M_j U_j ]
// with P = (1,-8,37,37,-8,1)/60 (central) and M = (1,-5,10,-10,5,-1)/60;
// R L = I and alpha takes three values, so
//   F^ = F~ + a_mid U~ + (a_0 - a_mid)(l_0.U~) r_0 + (a_E - a_mid)(l_E.U~) r_E.
// cell_flux_half gives F_d(U)/2 of one cell (eq. 4.7) from its half u_d and
// half p -- the grid path stores it per cell and direction, the one-pass
// path forms it per stencil point, with the same rounding; closed_point adds
// point j to F~ and U~ as a binary64 chain (the one-pass form's sums; the
// two-pass kernels use the fixed-point sums below); closed_out forms F^.
//
// The sums are kept in integer weights, 30 F~ = sum_j c_j F_j/2 with
// c = (1,-8,37,37,-8,1) and 60 U~ = sum_j m_j U_j with m = (1,-5,10,-10,5,-1),
// so that point 0 enters by assignment and point 5 by an add (a multiply
// fewer per component than with the fractional weights), and every interface
// flux is stored as 30 F^ (kFluxScale): the speeds enter closed_out halved,
// 30 a U~ = (a/2) 60 U~, and the difference pass divides by 30 together with
// dx (Grid::inv_dx_f).  The mass component of F_d/2 is m_d/2: closed_point
// sums c_j m_d and closed_out halves it, so the half fluxes need only the
// momentum and energy components (v = 1..nvar-1).
// ---------------------------------------------------------------------------
// cell_flux_half_ep takes E + p as given (the cell pass has it);
// cell_flux_half forms it as E + 2 (p/2), the same value, since the
// doubling is exact.
template <int NDIM, int DIR>
__device__ __forceinline__ void cell_flux_half_ep(const double (&Uc)[NDIM + 2], double un, double pn, double ep,
                                                  double (&Fh)[NDIM + 2]) {
  constexpr int NVAR = NDIM + 2;
  Fh[0] = 0.5 * Uc[1 + DIR];
#pragma unroll
  for (int k = 0; k < NDIM; ++k) Fh[1 + k] = k == DIR ? fma(un, Uc[1 + k], pn) : un * Uc[1 + k];
  Fh[NVAR - 1] = un * ep;
}

template <int NDIM, int DIR>
__device__ __forceinline__ void cell_flux_half(const double (&Uc)[NDIM + 2], double un, double pn,
                                               double (&Fh)[NDIM + 2]) {
  constexpr int NVAR = NDIM + 2;
  // F/2 = (u_d/2) U + (p/2) (0, e_d, u_d), per component: mass m_d/2,
  // momentum (u_d/2) m_k (+ p/2 for k = d), energy (u_d/2)(E + p); E + p
  // is formed as E + 2 (p/2), which doubles exactly
  cell_flux_half_ep<NDIM, DIR>(Uc, un, pn, fma(2.0, pn, Uc[NVAR - 1]), Fh);
}

// (Fhj[0] is not read: the mass sum is sum_j c_j m_d.)
template <int NDIM, int DIR>
__device__ __forceinline__ void closed_point(int j, const double (&Uj)[NDIM + 2], const double (&Fhj)[NDIM + 2],
                                             double (&Ft)[NDIM + 2], double (&Ut)[NDIM + 2]) {
  constexpr int NVAR = NDIM + 2;
  const double C[6] = {1.0, -8.0, 37.0, 37.0, -8.0, 1.0};
  const double Mw[6] = {1.0, -5.0, 10.0, -10.0, 5.0, -1.0};
#pragma unroll
  for (int v = 0; v < NVAR; ++v) {
    const double f = v == 0 ? Uj[1 + DIR] : Fhj[v];
    if (j == 0) {
      Ft[v] = f;
      Ut[v] = Uj[v];
    } else if (j == 5) {
      Ft[v] += f;
      Ut[v] -= Uj[v];
    } else {
      Ft[v] = fma(C[j], f, Ft[v]);
      Ut[v] = fma(Mw[j], Uj[v], Ut[v]);
    }
  }
}

// The same two sums in 64-bit fixed point (teno_fixsum.cuh): integer sums
// on the grid 2^(E - 1078) of each component's largest stencil value,
// rounded once to binary64 by closed_fix_out.  EU[v] and EF[v] are the
// largest biased exponents of U[v] and of F/2[v] over the six points
// (EF[0] = EU[1 + DIR]: the mass flux sums m_d); AU and AF accumulate the
// integer terms.  Every U~ sum runs in fixed point; the F~ sums of the
// components named by kFixFluxMask (1 mass, 2 momenta, 4 energy) do too, the
// others stay binary64 chains (Ftd).  The mask balances the integer and FP64
// pipes: it is a tuning choice, both forms being within their stated
// rounding of the exact sum.  Measured on the 256^3 turbulence box (ms per
// RK3 step): all ten sums in fixed point 38.3, U~ and the mass and energy
// fluxes 37.5, U~ and the mass flux 37.4 (this default), every sum a
// binary64 chain 40.4.
#ifndef TENO_FIX_FLUX_MASK
#define TENO_FIX_FLUX_MASK 1
#endif
constexpr unsigned kFixFluxMask = TENO_FIX_FLUX_MASK;

template <int NDIM>
struct ClosedFix {
  uint32_t EU[NDIM + 2], EF[NDIM + 2];
  int64_t AU[NDIM + 2], AF[NDIM + 2];
  double Ftd[NDIM + 2];
};

template <int NVAR>
__device__ __forceinline__ constexpr bool fix_flux(int v) {
  return (kFixFluxMask & (v == 0 ? 1u : v == NVAR - 1 ? 4u : 2u)) != 0u;
}

// exponents from the running maxima of the magnitude keys (KF[v] is read
// only for the fixed-point flux components); false when a component lies
// outside the fixed point's range
template <int NDIM, int DIR>
__device__ __forceinline__ bool closed_fix_begin(const uint32_t (&KU)[NDIM + 2], const uint32_t (&KF)[NDIM + 2],
                                                 ClosedFix<NDIM>& X) {
  constexpr int NVAR = NDIM + 2;
  bool ok = true;
#pragma unroll
  for (int v = 0; v < NVAR; ++v) {
    X.AU[v] = X.AF[v] = 0;
    X.Ftd[v] = 0.0;
    X.EU[v] = teno_fix::exponent(KU[v]);
    ok = ok && teno_fix::in_range(X.EU[v]);
  }
  X.EF[0] = X.EU[1 + DIR];
#pragma unroll
  for (int v = 1; v < NVAR; ++v) {
    X.EF[v] = fix_flux<NVAR>(v) ? teno_fix::exponent(KF[v]) : 0u;
    ok = ok && teno_fix::in_range(X.EF[v]);
  }
  return ok;
}

// the weights c_j and m_j for a point index that may be a loop variable
__constant__ int c_fix_w[2][6] = {{1, -8, 37, 37, -8, 1}, {1, -5, 10, -10, 5, -1}};
__constant__ double c_fix_cd[6] = {1.0, -8.0, 37.0, 37.0, -8.0, 1.0};

// adds point j to the sums (all start at zero)
template <int NDIM, int DIR>
__device__ __forceinline__ void closed_fix_point(int j, const double (&Uj)[NDIM + 2], const double (&Fhj)[NDIM + 2],
                                                 ClosedFix<NDIM>& X) {
  constexpr int NVAR = NDIM + 2;
  const int cw = c_fix_w[0][j], mw = c_fix_w[1][j];
  const double cd = c_fix_cd[j];
  // (a binary64 chain takes point 0 by assignment: j is uniform across the
  // warp, so the branch does not diverge)
  auto chain = [&](double& acc, double f) {
    if (j == 0) acc = f;
    else acc = fma(cd, f, acc);
  };
#pragma unroll
  for (int v = 0; v < NVAR; ++v) {
    teno_fix::add(X.AU[v], Uj[v], X.EU[v], mw);
    if (v == 1 + DIR) {
      if (fix_flux<NVAR>(0)) teno_fix::add(X.AF[0], Uj[v], X.EF[0], cw);
      else chain(X.Ftd[0], Uj[v]);
    }
    if (v >= 1) {
      if (fix_flux<NVAR>(v)) teno_fix::add(X.AF[v], Fhj[v], X.EF[v], cw);
      else chain(X.Ftd[v], Fhj[v]);
    }
  }
}

template <int NDIM>
__device__ __forceinline__ void closed_fix_out(const ClosedFix<NDIM>& X, double (&Ft)[NDIM + 2],
                                               double (&Ut)[NDIM + 2]) {
  constexpr int NVAR = NDIM + 2;
#pragma unroll
  for (int v = 0; v < NVAR; ++v) {
    Ft[v] = fix_flux<NVAR>(v) ? teno_fix::round(X.AF[v], X.EF[v]) : X.Ftd[v];
    Ut[v] = teno_fix::round(X.AU[v], X.EU[v]);
  }
}

// The factor by which interface fluxes are stored (see above).
constexpr double kFluxScale = 30.0;

template <int NDIM, int DIR>
__device__ __forceinline__ void closed_out(const double (&Ft)[NDIM + 2], const double (&Ut)[NDIM + 2],
                                           const RoeIfc<NDIM>& R, const double (&nal)[NDIM + 2],
                                           double (&out)[NDIM + 2]) {
  constexpr int NVAR = NDIM + 2;
  // l_0.U~ = A + B and l_E.U~ = A - B (as in project), so with the speed
  // differences d0, dE of fields 0 and E against the middle ones the two
  // corrections g0 = d0 l_0.U~, gE = dE l_E.U~ enter only as
  //   gs = g0 + gE = (d0 + dE) A + (d0 - dE) B,
  //   gd = gE - g0 = -((d0 - dE) A + (d0 + dE) B)      (ngd = -gd below).
  // Ut is 60 U~ and Ft 30 F~ (F~'s mass component 60 F~_0): with the halved
  // speeds every term below is 30 times its value.
  double Sx = -Ut[NVAR - 1];
#pragma unroll
  for (int k = 0; k < NDIM; ++k) Sx = fma(R.u[k], Ut[1 + k], Sx);
  const double A = fma(R.hb2, Ut[0], -R.hb1 * Sx);
  const double B = fma(R.u[DIR], Ut[0], -Ut[1 + DIR]) * R.hic;
  const double amid = -0.5 * nal[1];
  const double d0 = 0.5 * (nal[1] - nal[0]), dE = 0.5 * (nal[1] - nal[NVAR - 1]);
  const double sg = d0 + dE, df = d0 - dE;
  const double gs = fma(sg, A, df * B);
  const double ngd = fma(df, A, sg * B);
  out[0] = fma(0.5, Ft[0], fma(amid, Ut[0], gs));
#pragma unroll
  for (int k = 0; k < NDIM; ++k) {
    double o = fma(R.u[k], gs, fma(amid, Ut[1 + k], Ft[1 + k]));
    if (k == DIR) o = fma(-R.cs, ngd, o);
    out[1 + k] = o;
  }
  out[NVAR - 1] = fma(R.H, gs, fma(-(R.u[DIR] * R.cs), ngd, fma(amid, Ut[NVAR - 1], Ft[NVAR - 1])));
}

// ---------------------------------------------------------------------------
// The certified closed form alone, with the per-cell F_DIR/2 of the cell
// pass (`fh`, momentum and energy components only: [nvar - 1][ncell]), in
// two passes over the six stencil points: the FP32 test (and the exponents
// of the sums), then the fixed-point sums, so that the test's state is dead
// before the sums' state is live.  Returns false, with `out` unwritten, when
// the test does not keep every stencil or the fixed point does not cover a
// sum; otherwise `out` equals interface_flux's up to the rounding of the
// sums (which that one-pass form evaluates as binary64 chains).
// ---------------------------------------------------------------------------
// (GH: the sweep direction has fixed-state ghost cells, read from gc; the
// half fluxes of the ghost block are taken at direction DIR's block.  With
// `rout` the interface's Roe state is also returned, whatever the test
// decides.)
template <int NDIM, int DIR, bool GH = false>
__device__ __forceinline__ bool interface_flux_closed(const double* __restrict__ U,
                                                      const double* __restrict__ aux,
                                                      const double* __restrict__ fh, int64_t ncell,
                                                      const int64_t (&cells)[6], unsigned flips,
                                                      const double (&alpha)[NDIM + 2],
                                                      const double (&nal)[NDIM + 2], const Scheme& S,
                                                      double (&out)[NDIM + 2], int* __restrict__ status,
                                                      const GhostCells& gc = GhostCells(),
                                                      RoeIfc<NDIM>* rout = nullptr) {
  constexpr int NVAR = NDIM + 2;
  if (S.keep_idx < 0) return false;
  const double* gfh = GH ? gc.fh + DIR * (NVAR - 1) * kGhostSlots : nullptr;
  RoeIfc<NDIM> R;
  {
    double su2[NDIM], su3[NDIM];
#pragma unroll
    for (int k = 0; k < NDIM; ++k) {
      su2[k] = ldc<GH>(aux, gc.aux, ncell, NDIM + 3 + k, cells[2]);
      su3[k] = ldc<GH>(aux, gc.aux, ncell, NDIM + 3 + k, cells[3]);
    }
    su2[DIR] = flip_sign(su2[DIR], (flips >> 2) & 1u);
    su3[DIR] = flip_sign(su3[DIR], (flips >> 3) & 1u);
    roe_interface<NDIM, DIR>(ldc<GH>(aux, gc.aux, ncell, NDIM + 1, cells[2]),
                             ldc<GH>(aux, gc.aux, ncell, NDIM + 1, cells[3]),
                             ldc<GH>(aux, gc.aux, ncell, NDIM + 2, cells[2]),
                             ldc<GH>(aux, gc.aux, ncell, NDIM + 2, cells[3]), su2, su3, S, R, status);
  }
  if (rout) *rout = R;
  // stencil point j: U with the normal momentum reversed at a mirrored wall
  // point, so u_d and every component of F_d/2 but the normal-momentum one
  // change sign
  auto load_point = [&](int j, int64_t c, double (&Uj)[NVAR], double (&Fhj)[NVAR]) {
    const bool fj = (flips >> j) & 1u;
#pragma unroll
    for (int v = 0; v < NVAR; ++v) Uj[v] = ldc<GH>(U, gc.U, ncell, v, c);
    Fhj[0] = 0.0;   // unused: the mass term comes from m_d
#pragma unroll
    for (int v = 1; v < NVAR; ++v) Fhj[v] = flip_sign(ldc<GH>(fh, gfh, ncell, v - 1, c), fj && v != 1 + DIR);
    Uj[1 + DIR] = flip_sign(Uj[1 + DIR], fj);
  };
  // first pass: the certified test, and the magnitude keys of the summed
  // components (high words only; a mirrored point changes signs only)
  uint32_t KU[NVAR], KF[NVAR];
#pragma unroll
  for (int v = 0; v < NVAR; ++v) KF[v] = 0u;
  {
    CertIfc<NDIM> C;
    cert_begin<NDIM, DIR>(R, alpha, C);
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const int64_t c = cells[j];
      const bool fj = (flips >> j) & 1u;
      double Uj[NVAR];
#pragma unroll
      for (int v = 0; v < NVAR; ++v) {
        Uj[v] = ldc<GH>(U, gc.U, ncell, v, c);
        const uint32_t k = teno_fix::key(teno_fix::hi_word(Uj[v]));
        KU[v] = j == 0 ? k : max(KU[v], k);
      }
#pragma unroll
      for (int v = 1; v < NVAR; ++v) {
        if (!fix_flux<NVAR>(v)) continue;
        const uint32_t k = teno_fix::key(ldc_hi<GH>(fh, gfh, ncell, v - 1, c));
        KF[v] = j == 0 ? k : max(KF[v], k);
      }
      Uj[1 + DIR] = flip_sign(Uj[1 + DIR], fj);
      const double unj = flip_sign(ldc<GH>(aux, gc.aux, ncell, DIR, c), fj);
      const double pnj = ldc<GH>(aux, gc.aux, ncell, NDIM, c);
      cert_point<NDIM, DIR>(j, Uj, unj, pnj, C);
    }
    if (!cert_keep<NDIM>(C, S)) return false;
  }
  // second pass: the two sums per component in fixed point.  Where its
  // exponent range does not cover a component (values below 2^-959 or above
  // 2^1007, infinities, NaN) the interface goes to the pending list, whose
  // characteristic path evaluates it in binary64.  The points are taken in
  // two rounds of three (fully unrolled, the sums' temporaries of all six
  // points would not fit in the registers beside the Roe state; the cell
  // indices, read with a loop index, then sit in the stack frame).
  ClosedFix<NDIM> X;
  if (!closed_fix_begin<NDIM, DIR>(KU, KF, X)) return false;
#pragma unroll 3
  for (int j = 0; j < 6; ++j) {
    double Uj[NVAR], Fhj[NVAR];
    load_point(j, cells[j], Uj, Fhj);
    closed_fix_point<NDIM, DIR>(j, Uj, Fhj, X);
  }
  double Ft[NVAR], Ut[NVAR];
  closed_fix_out<NDIM>(X, Ft, Ut);
  closed_out<NDIM, DIR>(Ft, Ut, R, nal, out);
  return true;
}

// ---------------------------------------------------------------------------
// Interface flux F^_{i+1/2} in direction DIR from the six cells i-2..i+3
// (`cells`, linear indices into arrays of `ncell` entries per variable):
// Roe-averaged eigensystem of cells i, i+1, characteristic projection, global
// Lax-Friedrichs split with the halved speeds `alpha` (nal = -2 alpha), TENO5-LAD
// reconstruction of f^+ (cells i-2..i+2) and f^- (mirrored, i+3..i-1) for
// every field, back-projection.  Bit j of `flips` marks stencil point j as a
// mirrored wall point (reflecting boundary: normal velocity reversed).
// `fl` receives the flag bytes when WITH_FLAGS
// (without flags, bits 0..2 still hold the selections used).
// MODE kFluxFull computes the flux.  kFluxSelect only wants the selections:
// it returns without the flux when the certified test keeps every stencil.
// kFluxCertify stops after the certified test: fl = 7 everywhere if it keeps
// every stencil, else fl[0][0] = kUndecided and nothing else is written.
// kFluxChar skips the certified test and takes the characteristic path (for
// interfaces the test has already left undecided: the flux equals
// kFluxFull's).
// ---------------------------------------------------------------------------
constexpr int kFluxFull = 0, kFluxSelect = 1, kFluxCertify = 2, kFluxChar = 4;
constexpr unsigned kUndecided = 0xffu;

// the certify-only instantiation ends early: its remaining code is unreachable
#pragma nv_diag_suppress 128
template <int NDIM, int DIR, bool WITH_FLAGS, int MODE = kFluxFull, bool GH = false>
__device__ __forceinline__ void interface_flux(const double* __restrict__ U,
                                               const double* __restrict__ aux,
                                               int64_t ncell, const int64_t (&cells)[6], unsigned flips,
                                               const double (&alpha)[NDIM + 2],
                                               const double (&nal)[NDIM + 2],
                                               const Scheme& S, double (&out)[NDIM + 2],
                                               unsigned (&fl)[NDIM + 2][2],
                                               int* __restrict__ status,
                                               const GhostCells& gc = GhostCells()) {
  constexpr int NVAR = NDIM + 2;
  {
    // six-point stencil i-2..i+3 with i = id - 1
    double Ux[6][NVAR], un[6], pn[6];
    double sr2, sr3, sh2, sh3, su2[NDIM], su3[NDIM];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const int64_t c = cells[j];
      const bool fj = (flips >> j) & 1u;   // mirrored wall point
#pragma unroll
      for (int v = 0; v < NVAR; ++v) Ux[j][v] = ldc<GH>(U, gc.U, ncell, v, c);
      Ux[j][1 + DIR] = flip_sign(Ux[j][1 + DIR], fj);
      un[j] = flip_sign(ldc<GH>(aux, gc.aux, ncell, DIR, c), fj);
      pn[j] = ldc<GH>(aux, gc.aux, ncell, NDIM, c);
      if (j == 2 || j == 3) {
        double* su = (j == 2) ? su2 : su3;
#pragma unroll
        for (int k = 0; k < NDIM; ++k) su[k] = ldc<GH>(aux, gc.aux, ncell, NDIM + 3 + k, c);
        su[DIR] = flip_sign(su[DIR], fj);
        if (j == 2) {
          sr2 = ldc<GH>(aux, gc.aux, ncell, NDIM + 1, c);
          sh2 = ldc<GH>(aux, gc.aux, ncell, NDIM + 2, c);
        } else {
          sr3 = ldc<GH>(aux, gc.aux, ncell, NDIM + 1, c);
          sh3 = ldc<GH>(aux, gc.aux, ncell, NDIM + 2, c);
        }
      }
    }
    RoeIfc<NDIM> R;
    roe_interface<NDIM, DIR>(sr2, sr3, sh2, sh3, su2, su3, S, R, status);
    const double (&u)[NDIM] = R.u;
    const double q2 = R.q2, H = R.H, cs = R.cs, b1 = R.b1;
    const double hb1 = R.hb1, hb2 = R.hb2, hic = R.hic, hud = R.hud;

    if (!WITH_FLAGS && MODE != kFluxChar && S.keep_idx >= 0) {
      CertIfc<NDIM> C;
      cert_begin<NDIM, DIR>(R, alpha, C);
#pragma unroll
      for (int j = 0; j < 6; ++j) cert_point<NDIM, DIR>(j, Ux[j], un[j], pn[j], C);
      const bool keep = cert_keep<NDIM>(C, S);
      if ((MODE == kFluxSelect || MODE == kFluxCertify) && keep) {
        // only the selections are wanted: every stencil kept
#pragma unroll
        for (int f = 0; f < NVAR; ++f) fl[f][0] = fl[f][1] = 7u;
        return;
      }
      if (keep) {
        // (the sums as binary64 chains: this one-pass form holds the whole
        // stencil in registers already)
        double Ft[NVAR], Ut[NVAR];
#pragma unroll
        for (int j = 0; j < 6; ++j) {
          double Fhj[NVAR];
          cell_flux_half<NDIM, DIR>(Ux[j], un[j], pn[j], Fhj);
          closed_point<NDIM, DIR>(j, Ux[j], Fhj, Ft, Ut);
        }
        closed_out<NDIM, DIR>(Ft, Ut, R, nal, out);
#pragma unroll
        for (int f = 0; f < NVAR; ++f) fl[f][0] = fl[f][1] = 7u;
        return;
      }
    }
    if (MODE == kFluxCertify) {
      fl[0][0] = kUndecided;
      return;
    }

    // Characteristic values w = L U and the split fluxes v+- = (g +- alpha w)/2
    // with g = L F.  Since F(U) = u_d U + p (0, e_d, u_d) (eq. 4.7),
    // g = u_d w + p z with z = (hb1 du - hic, -2 hb1 du, 0.., hb1 du + hic),
    // du = u_d - u~_d, so v+- = (u_d/2 +- alpha/2) w + (p/2) z.
    double fchar[NVAR];
    double vp[6][NVAR], vm[6][NVAR];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      double w[NVAR];
      project<NDIM, DIR>(Ux[j], u, hb1, hb2, hic, w);
      const double hu = un[j];        // u_d / 2
      const double hp = pn[j];        // p / 2
      const double az = hp * (b1 * (hu - hud));   // (p/2) hb1 du
      const double bz = hp * hic;
      const double t0 = az - bz;
      const double tE = az + bz;
      const double t1 = -2.0 * az;
      // v- = v+ - alpha w (nal = -alpha)
      vp[j][0] = fma(hu + alpha[0], w[0], t0);
      vm[j][0] = fma(nal[0], w[0], vp[j][0]);
      vp[j][NVAR - 1] = fma(hu + alpha[NVAR - 1], w[NVAR - 1], tE);
      vm[j][NVAR - 1] = fma(nal[NVAR - 1], w[NVAR - 1], vp[j][NVAR - 1]);
      const double sp = hu + alpha[1];
      vp[j][1] = fma(sp, w[1], t1);
      vm[j][1] = fma(nal[1], w[1], vp[j][1]);
#pragma unroll
      for (int f = 2; f < NVAR - 1; ++f) {
        vp[j][f] = sp * w[f];
        vm[j][f] = fma(nal[1], w[f], vp[j][f]);
      }
    }
#pragma unroll
    for (int s = 0; s < NVAR; ++s) {
      const double hp = teno5_lad<WITH_FLAGS>(vp[0][s], vp[1][s], vp[2][s], vp[3][s], vp[4][s], 0.0, S, fl[s][0]);
      fchar[s] = teno5_lad<WITH_FLAGS>(vm[5][s], vm[4][s], vm[3][s], vm[2][s], vm[1][s], hp, S, fl[s][1]);
    }
    // back-projection F^ = R f^char, columns r_0 = (1, u - c e_n, H - u_n c),
    // r_1 = (1, u, q2/2), r_t = (0, e_t, u_t), r_{nvar-1} = (1, u + c e_n, H + u_n c),
    // stored as kFluxScale F^ like the closed form's
#pragma unroll
    for (int s = 0; s < NVAR; ++s) fchar[s] *= kFluxScale;
    const double sa = fchar[0] + fchar[NVAR - 1];
    const double da = fchar[NVAR - 1] - fchar[0];
    const double rho_f = sa + fchar[1];
    out[0] = rho_f;
    double eng = fma(H, sa, fma(u[DIR] * cs, da, 0.5 * q2 * fchar[1]));
    {
      int f = 2;
#pragma unroll
      for (int k = 0; k < NDIM; ++k) {
        if (k == DIR) {
          out[1 + k] = fma(u[k], rho_f, cs * da);
        } else {
          out[1 + k] = fma(u[k], rho_f, fchar[f]);
          eng = fma(u[k], fchar[f], eng);
          ++f;
        }
      }
    }
    out[NVAR - 1] = eng;
  }
}
#pragma nv_diag_default 128

// ---------------------------------------------------------------------------
// Primitive variables of cell c from one reciprocal square root:
// 1/sqrt(rho), sqrt(rho) = rho/sqrt(rho), 1/(2 rho) = (1/sqrt(rho))^2 / 2,
// u/2 = m/(2 rho), p = (gamma-1)(E - 2 rho |u/2|^2) (eq. 4.7),
// c = sqrt(gamma p / rho).  Writes the aux entries (u_k/2, p/2, sqrt(rho),
// (E+p)/sqrt(rho), sqrt(rho) u_k = m_k/sqrt(rho) -- the Roe average's
// weighted velocities)
// and returns uh = u/2, c and E + p; false if the state is not physical
// (rho <= 0, p <= 0 or non-finite).  Working with u/2 saves the halving
// multiplies; every value equals the u-based evaluation's bit for bit,
// since the factors of 2 are exact.
// ---------------------------------------------------------------------------
template <int NDIM>
__device__ __forceinline__ bool cell_primitives(const double* __restrict__ U, int64_t ncell,
                                                int64_t c, double gamma,
                                                double* __restrict__ aux,
                                                double (&uh)[NDIM], double& cs, double& ep) {
  constexpr int NVAR = NDIM + 2;
  const double rho = U[c];
  const double E = U[(NVAR - 1) * ncell + c];
  const double isr = rsqrt(rho);
  const double sr = rho * isr;
  const double hr = (0.5 * isr) * isr;
  double q2h = 0.0;
#pragma unroll
  for (int k = 0; k < NDIM; ++k) {
    uh[k] = U[(1 + k) * ncell + c] * hr;
    q2h = fma(uh[k], uh[k], q2h);
  }
  const double p = (gamma - 1.0) * fma(-2.0 * rho, q2h, E);
  const double gpr = (2.0 * gamma) * p * hr;
  cs = gpr * rsqrt(gpr);
  ep = E + p;
#pragma unroll
  for (int k = 0; k < NDIM; ++k) aux[k * ncell + c] = uh[k];
  aux[NDIM * ncell + c] = 0.5 * p;
  aux[(NDIM + 1) * ncell + c] = sr;
  aux[(NDIM + 2) * ncell + c] = ep * isr;
#pragma unroll
  for (int k = 0; k < NDIM; ++k) aux[(NDIM + 3 + k) * ncell + c] = U[(1 + k) * ncell + c] * isr;
  return pos_finite(rho) && pos_finite(p) && is_finite(E) && is_finite(q2h) && pos_finite(gpr);
}

// SSP-RK3 stage value (eq. 4.1-4.3) of element e from d = L(U^(k))_e:
// mode 2: U^n + dt d;  3: 3/4 U^n + 1/4 U1 + 1/4 dt d;  4: 1/3 U^n + 2/3 U2 + 2/3 dt d.
__device__ __forceinline__ double stage_value(int mode, double dt, double d,
                                              const double* __restrict__ Un,
                                              const double* __restrict__ Uk, int64_t e) {
  if (mode == 2) return fma(dt, d, Un[e]);
  if (mode == 3) return fma(0.25 * dt, d, fma(0.75, Un[e], 0.25 * Uk[e]));
  return fma((2.0 / 3.0) * dt, d, fma(1.0 / 3.0, Un[e], (2.0 / 3.0) * Uk[e]));
}

}  // namespace teno
