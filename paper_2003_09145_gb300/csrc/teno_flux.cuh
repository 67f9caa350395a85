// teno_flux.cuh -- the numerical flux at one interface (device function shared
// by the grid kernels and the batched kernel).  FP64 throughout.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "teno_device.cuh"

namespace teno {

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
// Interface flux F^_{i+1/2} in direction DIR from the six cells i-2..i+3
// (`cells`, linear indices into arrays of `ncell` entries per variable):
// Roe-averaged eigensystem of cells i, i+1, characteristic projection, global
// Lax-Friedrichs split with the halved speeds `alpha` (nal = -2 alpha), TENO5-LAD
// reconstruction of f^+ (cells i-2..i+2) and f^- (mirrored, i+3..i-1) for
// every field, back-projection.  `fl` receives the flag bytes when WITH_FLAGS.
// ---------------------------------------------------------------------------
template <int NDIM, int DIR, bool WITH_FLAGS>
__device__ __forceinline__ void interface_flux(const double* __restrict__ U,
                                               const double* __restrict__ aux,
                                               int64_t ncell, const int64_t (&cells)[6],
                                               const double (&alpha)[NDIM + 2],
                                               const double (&nal)[NDIM + 2],
                                               const Scheme& S, double (&out)[NDIM + 2],
                                               unsigned (&fl)[NDIM + 2][2],
                                               int* __restrict__ status) {
  constexpr int NVAR = NDIM + 2;
  {
    // six-point stencil i-2..i+3 with i = id - 1
    double Ux[6][NVAR], un[6], pn[6];
    double sr2, sr3, sh2, sh3, uu2[NDIM], uu3[NDIM];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const int64_t c = cells[j];
#pragma unroll
      for (int v = 0; v < NVAR; ++v) Ux[j][v] = U[v * ncell + c];
      un[j] = aux[DIR * ncell + c];
      pn[j] = aux[NDIM * ncell + c];
      if (j == 2 || j == 3) {
        double* uu = (j == 2) ? uu2 : uu3;
#pragma unroll
        for (int k = 0; k < NDIM; ++k) uu[k] = (k == DIR) ? un[j] : aux[k * ncell + c];
        if (j == 2) {
          sr2 = aux[(NDIM + 1) * ncell + c];
          sh2 = aux[(NDIM + 2) * ncell + c];
        } else {
          sr3 = aux[(NDIM + 1) * ncell + c];
          sh3 = aux[(NDIM + 2) * ncell + c];
        }
      }
    }
    // Roe average of cells i and i+1 (uu2, uu3 hold half velocities)
    const double inv2 = 2.0 / (sr2 + sr3);
    double u[NDIM];
    double q2 = 0.0;
#pragma unroll
    for (int k = 0; k < NDIM; ++k) {
      u[k] = fma(sr2, uu2[k], sr3 * uu3[k]) * inv2;
      q2 = fma(u[k], u[k], q2);
    }
    const double H = (sh2 + sh3) * (0.5 * inv2);
    const double c2 = S.gm1 * fma(-0.5, q2, H);
    if (!(c2 > 0.0)) atomicOr(status, kStatusNonphysical);
    const double ic = rsqrt(c2);
    const double cs = c2 * ic;
    const double b1 = S.gm1 * ic * ic;
    const double b2 = 0.5 * b1 * q2;
    const double hb1 = 0.5 * b1, hb2 = 0.5 * b2, hic = 0.5 * ic;
    const double hud = 0.5 * u[DIR];

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
    // r_1 = (1, u, q2/2), r_t = (0, e_t, u_t), r_{nvar-1} = (1, u + c e_n, H + u_n c)
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

// ---------------------------------------------------------------------------
// Primitive variables of cell c from one reciprocal square root:
// 1/sqrt(rho), sqrt(rho) = rho/sqrt(rho), 1/rho = (1/sqrt(rho))^2, u = m/rho,
// p = (gamma-1)(E - rho |u|^2 / 2) (eq. 4.7), c = sqrt(gamma p / rho).  Writes
// the aux entries (u_k/2, p/2, sqrt(rho), (E+p)/sqrt(rho)) and returns u and c;
// false if the state is not physical (rho <= 0, p <= 0 or non-finite).
// ---------------------------------------------------------------------------
template <int NDIM>
__device__ __forceinline__ bool cell_primitives(const double* __restrict__ U, int64_t ncell,
                                                int64_t c, double gamma,
                                                double* __restrict__ aux,
                                                double (&u)[NDIM], double& cs) {
  constexpr int NVAR = NDIM + 2;
  const double rho = U[c];
  const double E = U[(NVAR - 1) * ncell + c];
  const double isr = rsqrt(rho);
  const double sr = rho * isr;
  const double r = isr * isr;
  double q2 = 0.0;
#pragma unroll
  for (int k = 0; k < NDIM; ++k) {
    u[k] = U[(1 + k) * ncell + c] * r;
    q2 = fma(u[k], u[k], q2);
  }
  const double p = (gamma - 1.0) * fma(-0.5 * rho, q2, E);
  const double gpr = gamma * p * r;
  cs = gpr * rsqrt(gpr);
#pragma unroll
  for (int k = 0; k < NDIM; ++k) aux[k * ncell + c] = 0.5 * u[k];
  aux[NDIM * ncell + c] = 0.5 * p;
  aux[(NDIM + 1) * ncell + c] = sr;
  aux[(NDIM + 2) * ncell + c] = (E + p) * isr;
  return (rho > 0.0) && (p > 0.0) && isfinite(E) && isfinite(q2) && (gpr > 0.0);
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
