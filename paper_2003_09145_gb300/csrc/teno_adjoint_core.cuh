// teno_adjoint_core.cuh -- vector-Jacobian product of one interface flux of the
// TENO5-LAD Euler right-hand side, with the stencil selections frozen (the
// cutoff of eq. 2.14 is a piecewise-constant selector, so with delta fixed the
// reconstruction of eq. 2.4-2.7 is linear in the split fluxes).
//
// Forward map at the interface i+1/2 of direction DIR, points j = 0..5 being
// cells i-2..i+3:
//   U_j -> (rho, u, p)_j -> F_j (eq. 4.7)
//   (U_2, U_3) -> Roe state (u~, H~) -> c, b1 = (gamma-1)/c^2, b2 = b1 |u~|^2/2
//            -> L (left eigenvectors, rows), R (right eigenvectors, columns)
//   w_j = L U_j,  g_j = L F_j
//   fchar_s = sum_j P_sj g_js + alpha_s M_sj w_js
//     with P = (A+ + A-)/2, M = (A+ - A-)/2 and A+- the linear weights of the
//     frozen reconstructions of f^+ (points 0..4) and f^- (points 5..1)
//   F^ = R fchar
// Reverse pass: given Fbar = dJ/dF^, returns dJ/dU_j for the six points and
// dJ/dalpha_s.  Plain FP64 arithmetic, usable on host and device.
#pragma once

#include <cmath>

#ifdef __CUDACC__
#define TENO_HD __host__ __device__
#include "teno_device.cuh"
#else
#define TENO_HD
#endif

namespace teno_adj {

// 1/x for x > 0: on the device the seeded reciprocal of the forward pass
// (teno::recip_pos, within one ulp), on the host the division.
TENO_HD inline double recip(double x) {
#ifdef __CUDA_ARCH__
  return teno::recip_pos(x);
#else
  return 1.0 / x;
#endif
}

// Linear weights of the reconstruction with selection `sel` (delta bits):
// f^ = sum_k a[k] v_k over v = (f_{i-2}, ..., f_{i+2}), from the TENO weights
// of eq. 2.15 and the candidate fluxes of eq. 2.4-2.6.  The eight selection
// patterns' weights are a table built at compile time from these formulas
// (selection 0, no stencil, cannot occur: all zeros).
struct LinWeights {
  double a[8][5];
};
constexpr LinWeights make_lin_weights() {
  LinWeights t{};
  for (unsigned sel = 1; sel < 8; ++sel) {
    const double d0 = double(sel & 1u), d1 = double((sel >> 1) & 1u), d2 = double((sel >> 2) & 1u);
    const double s = d0 * 0.1 + d1 * 0.6 + d2 * 0.3;
    const double o0 = d0 * 0.1 / s, o1 = d1 * 0.6 / s, o2 = d2 * 0.3 / s;
    t.a[sel][0] = o0 / 3.0;
    t.a[sel][1] = -7.0 / 6.0 * o0 - 1.0 / 6.0 * o1;
    t.a[sel][2] = 11.0 / 6.0 * o0 + 5.0 / 6.0 * o1 + 1.0 / 3.0 * o2;
    t.a[sel][3] = 1.0 / 3.0 * o1 + 5.0 / 6.0 * o2;
    t.a[sel][4] = -1.0 / 6.0 * o2;
  }
  return t;
}
#ifdef __CUDACC__
__constant__ constexpr LinWeights c_lin_weights = make_lin_weights();
#endif
constexpr LinWeights h_lin_weights = make_lin_weights();

TENO_HD inline void lin_weights(unsigned sel, double a[5]) {
#ifdef __CUDA_ARCH__
  for (int k = 0; k < 5; ++k) a[k] = c_lin_weights.a[sel & 7u][k];
#else
  for (int k = 0; k < 5; ++k) a[k] = h_lin_weights.a[sel & 7u][k];
#endif
}

// With EXCL_P the flux term of the all-kept form, P_j A(U_j)^T Fbar
// (P = (1,-8,37,37,-8,1)/60), is left out of every point's result: the
// adjoint's gather adds that term for every interface alike, through one
// stencil on the right-hand-side adjoint per cell.
template <int NDIM, int DIR, bool EXCL_P = false>
TENO_HD inline void interface_vjp(const double (&Up)[6][NDIM + 2], const double (&alpha)[NDIM + 2],
                                  const unsigned (&sel)[NDIM + 2][2], double gamma,
                                  const double (&Fb)[NDIM + 2], double (&Ub)[6][NDIM + 2],
                                  double (&ab)[NDIM + 2]) {
  constexpr int NV = NDIM + 2;
  constexpr int E = NDIM + 1;
  constexpr int N = DIR;
  const double gm1 = gamma - 1.0;

  // ---- forward --------------------------------------------------------------
  double rho[6], ir[6], u[6][NDIM], p[6], q[6], F[6][NV];
  for (int j = 0; j < 6; ++j) {
    rho[j] = Up[j][0];
    ir[j] = recip(rho[j]);
    q[j] = 0.0;
    for (int k = 0; k < NDIM; ++k) {
      u[j][k] = Up[j][1 + k] * ir[j];
      q[j] += u[j][k] * u[j][k];
    }
    p[j] = gm1 * (Up[j][E] - 0.5 * rho[j] * q[j]);
    F[j][0] = rho[j] * u[j][N];
    for (int k = 0; k < NDIM; ++k) F[j][1 + k] = Up[j][1 + k] * u[j][N] + (k == N ? p[j] : 0.0);
    F[j][E] = u[j][N] * (Up[j][E] + p[j]);
  }
  const double sa = sqrt(rho[2]), sb = sqrt(rho[3]), S = sa + sb, iS = recip(S);
  const double Ha = (Up[2][E] + p[2]) * ir[2], Hb = (Up[3][E] + p[3]) * ir[3];
  double ut[NDIM], q2 = 0.0;
  for (int k = 0; k < NDIM; ++k) {
    ut[k] = (sa * u[2][k] + sb * u[3][k]) * iS;
    q2 += ut[k] * ut[k];
  }
  const double H = (sa * Ha + sb * Hb) * iS;
  const double c2 = gm1 * (H - 0.5 * q2);
  const double c = sqrt(c2);
  const double ic = recip(c), ic2 = ic * ic;
  const double b1 = gm1 * ic2;
  const double b2 = 0.5 * b1 * q2;
  const double un = ut[N];

  double L[NV][NV], R[NV][NV];
  for (int r = 0; r < NV; ++r)
    for (int k = 0; k < NV; ++k) L[r][k] = R[r][k] = 0.0;
  R[0][0] = 1.0;
  for (int k = 0; k < NDIM; ++k) R[1 + k][0] = ut[k] - (k == N ? c : 0.0);
  R[E][0] = H - un * c;
  L[0][0] = 0.5 * (b2 + un * ic);
  for (int k = 0; k < NDIM; ++k) L[0][1 + k] = 0.5 * (-b1 * ut[k] - (k == N ? ic : 0.0));
  L[0][E] = 0.5 * b1;
  R[0][1] = 1.0;
  for (int k = 0; k < NDIM; ++k) R[1 + k][1] = ut[k];
  R[E][1] = 0.5 * q2;
  L[1][0] = 1.0 - b2;
  for (int k = 0; k < NDIM; ++k) L[1][1 + k] = b1 * ut[k];
  L[1][E] = -b1;
  int tf[NDIM > 1 ? NDIM - 1 : 1];   // tangential direction of shear field 2 + i
  {
    int f = 2;
    for (int t = 0; t < NDIM; ++t) {
      if (t == N) continue;
      tf[f - 2] = t;
      R[1 + t][f] = 1.0;
      R[E][f] = ut[t];
      L[f][0] = -ut[t];
      L[f][1 + t] = 1.0;
      ++f;
    }
  }
  R[0][E] = 1.0;
  for (int k = 0; k < NDIM; ++k) R[1 + k][E] = ut[k] + (k == N ? c : 0.0);
  R[E][E] = H + un * c;
  L[E][0] = 0.5 * (b2 - un * ic);
  for (int k = 0; k < NDIM; ++k) L[E][1 + k] = 0.5 * (-b1 * ut[k] + (k == N ? ic : 0.0));
  L[E][E] = 0.5 * b1;

  double w[6][NV], g[6][NV];
  for (int j = 0; j < 6; ++j)
    for (int s = 0; s < NV; ++s) {
      double aw = 0.0, ag = 0.0;
      for (int k = 0; k < NV; ++k) {
        aw += L[s][k] * Up[j][k];
        ag += L[s][k] * F[j][k];
      }
      w[j][s] = aw;
      g[j][s] = ag;
    }
  double Pw[NV][6], Mw[NV][6], fchar[NV];
  for (int s = 0; s < NV; ++s) {
    double ap[5], am[5];
    lin_weights(sel[s][0], ap);
    lin_weights(sel[s][1], am);
    fchar[s] = 0.0;
    for (int j = 0; j < 6; ++j) {
      const double Ap = j < 5 ? ap[j] : 0.0;
      const double Am = j >= 1 ? am[5 - j] : 0.0;
      Pw[s][j] = 0.5 * (Ap + Am);
      Mw[s][j] = 0.5 * (Ap - Am);
      fchar[s] += Pw[s][j] * g[j][s] + alpha[s] * Mw[s][j] * w[j][s];
    }
  }

  // ---- reverse ----------------------------------------------------------------
  double fb[NV];
  for (int s = 0; s < NV; ++s) {
    fb[s] = 0.0;
    for (int r = 0; r < NV; ++r) fb[s] += R[r][s] * Fb[r];
  }
  double wb[6][NV], gb[6][NV];
  for (int s = 0; s < NV; ++s) {
    double sm = 0.0;
    for (int j = 0; j < 6; ++j) {
      wb[j][s] = alpha[s] * Mw[s][j] * fb[s];
      gb[j][s] = Pw[s][j] * fb[s];
      sm += Mw[s][j] * w[j][s];
    }
    ab[s] = fb[s] * sm;
  }
  // direct terms of w = L U, g = L F; X[s][k] = sum_j wb_js U_jk + gb_js F_jk
  double Fbar[6][NV], X[NV][NV];
  for (int j = 0; j < 6; ++j)
    for (int k = 0; k < NV; ++k) {
      double a1 = 0.0, a2 = 0.0;
      for (int s = 0; s < NV; ++s) {
        a1 += L[s][k] * wb[j][s];
        a2 += L[s][k] * gb[j][s];
      }
      Ub[j][k] = a1;
      Fbar[j][k] = a2;
    }
  for (int s = 0; s < NV; ++s)
    for (int k = 0; k < NV; ++k) {
      double a = 0.0;
      for (int j = 0; j < 6; ++j) a += wb[j][s] * Up[j][k] + gb[j][s] * F[j][k];
      X[s][k] = a;
    }

  // gradients of the Roe parameters
  double utb[NDIM];
  for (int k = 0; k < NDIM; ++k) utb[k] = 0.0;
  double Hbar = 0.0, cb = 0.0, b1b = 0.0, b2b = 0.0, q2b = 0.0;
  // from L
  b2b += 0.5 * X[0][0] - X[1][0] + 0.5 * X[E][0];
  utb[N] += 0.5 * ic * (X[0][0] - X[E][0]);
  cb += 0.5 * un * ic2 * (X[E][0] - X[0][0]);
  for (int k = 0; k < NDIM; ++k) {
    b1b += ut[k] * (-0.5 * X[0][1 + k] + X[1][1 + k] - 0.5 * X[E][1 + k]);
    utb[k] += b1 * (-0.5 * X[0][1 + k] + X[1][1 + k] - 0.5 * X[E][1 + k]);
  }
  cb += 0.5 * ic2 * (X[0][1 + N] - X[E][1 + N]);
  b1b += 0.5 * X[0][E] - X[1][E] + 0.5 * X[E][E];
  for (int f = 2; f < NV - 1; ++f) utb[tf[f - 2]] -= X[f][0];
  // from R (Rbar = Fb fchar^T)
  const double fsum = fchar[0] + fchar[1] + fchar[E];
  for (int k = 0; k < NDIM; ++k) utb[k] += Fb[1 + k] * fsum;
  cb += Fb[1 + N] * (fchar[E] - fchar[0]);
  Hbar += Fb[E] * (fchar[0] + fchar[E]);
  utb[N] += c * Fb[E] * (fchar[E] - fchar[0]);
  cb += un * Fb[E] * (fchar[E] - fchar[0]);
  q2b += 0.5 * Fb[E] * fchar[1];
  for (int f = 2; f < NV - 1; ++f) utb[tf[f - 2]] += Fb[E] * fchar[f];
  // chain through b2, b1, c, c2, q2
  b1b += 0.5 * q2 * b2b;
  q2b += 0.5 * b1 * b2b;
  double c2b = -(b1 * ic2) * b1b + 0.5 * ic * cb;
  Hbar += gm1 * c2b;
  q2b += -0.5 * gm1 * c2b;
  for (int k = 0; k < NDIM; ++k) utb[k] += 2.0 * ut[k] * q2b;
  // Roe averages
  double ub2[NDIM], ub3[NDIM], sab = 0.0, sbb = 0.0;
  for (int k = 0; k < NDIM; ++k) {
    ub2[k] = sa * iS * utb[k];
    ub3[k] = sb * iS * utb[k];
    sab += (u[2][k] - ut[k]) * iS * utb[k];
    sbb += (u[3][k] - ut[k]) * iS * utb[k];
  }
  const double Hab = sa * iS * Hbar, Hbb = sb * iS * Hbar;
  sab += (Ha - H) * iS * Hbar;
  sbb += (Hb - H) * iS * Hbar;

  // per point: primitives -> conservative
  if (EXCL_P) {
    const double Pk[6] = {1.0 / 60.0, -8.0 / 60.0, 37.0 / 60.0, 37.0 / 60.0, -8.0 / 60.0, 1.0 / 60.0};
    for (int j = 0; j < 6; ++j)
      for (int k = 0; k < NV; ++k) Fbar[j][k] -= Pk[j] * Fb[k];
  }
  for (int j = 0; j < 6; ++j) {
    double rhob = 0.0, Eb = 0.0, pb = 0.0, ub_[NDIM];
    for (int k = 0; k < NDIM; ++k) ub_[k] = 0.0;
    if (j == 2 || j == 3) {
      const double sx = (j == 2) ? sa : sb;
      const double sxb = (j == 2) ? sab : sbb;
      const double Hx = (j == 2) ? Ha : Hb;
      const double Hxb = (j == 2) ? Hab : Hbb;
      rhob += 0.5 * sx * ir[j] * sxb;   // 1/(2 sqrt(rho)) = sqrt(rho) / (2 rho)
      Eb += Hxb * ir[j];
      pb += Hxb * ir[j];
      rhob += -Hx * ir[j] * Hxb;
      for (int k = 0; k < NDIM; ++k) ub_[k] += (j == 2) ? ub2[k] : ub3[k];
    }
    // F = (rho u_n, m_k u_n + p delta_kn, u_n (E + p))
    double mb[NDIM];
    for (int k = 0; k < NDIM; ++k) mb[k] = 0.0;
    rhob += Fbar[j][0] * u[j][N];
    ub_[N] += Fbar[j][0] * rho[j];
    for (int k = 0; k < NDIM; ++k) {
      mb[k] += Fbar[j][1 + k] * u[j][N];
      ub_[N] += Fbar[j][1 + k] * Up[j][1 + k];
    }
    pb += Fbar[j][1 + N];
    ub_[N] += Fbar[j][E] * (Up[j][E] + p[j]);
    Eb += Fbar[j][E] * u[j][N];
    pb += Fbar[j][E] * u[j][N];
    // p = (gamma-1)(E - rho q / 2)
    Eb += gm1 * pb;
    rhob += -0.5 * gm1 * q[j] * pb;
    for (int k = 0; k < NDIM; ++k) ub_[k] += -gm1 * rho[j] * u[j][k] * pb;
    // u = m / rho
    for (int k = 0; k < NDIM; ++k) {
      mb[k] += ub_[k] * ir[j];
      rhob += -u[j][k] * ir[j] * ub_[k];
    }
    Ub[j][0] += rhob;
    for (int k = 0; k < NDIM; ++k) Ub[j][1 + k] += mb[k];
    Ub[j][E] += Eb;
  }
}

// ---------------------------------------------------------------------------
// Every stencil of every field and side kept (delta = 1 everywhere).  The
// reconstruction then has the fixed linear weights of eq. 2.3 and, with
// R L = I and the three distinct LF speeds (a_0, a_mid, a_E),
//   F^ = F~ + a_mid U~ + (a_0 - a_mid)(l_0 . U~) r_0 + (a_E - a_mid)(l_E . U~) r_E,
//   F~ = sum_j P_j F(U_j),  P = (1,-8,37,37,-8,1)/60,
//   U~ = sum_j M_j U_j,     M = (1,-5,10,-10,5,-1)/60.
// The stencil points enter through U~ (linearly) and F~ (through the flux
// Jacobian of each point); l_0, r_0, l_E, r_E depend on cells i and i+1 only.
// So dJ/dU_j = P_j A(U_j)^T Fbar + M_j U~bar (+ the Roe-parameter terms at
// j = 2, 3), and A(U_j)^T can be applied once per cell to the sum of its
// P-weighted Fbar over the interfaces that reach it.
// ---------------------------------------------------------------------------

// out = A(U)^T G with A = dF/dU the Euler flux Jacobian of direction DIR
// (eq. 4.7): F = u_d U + p (0, e_d, u_d), so
//   A^T G = u_d G + s (-u_d, e_d, 0) + t (|u|^2/2, -u, 1),
//   s = (G.U + p G_E) / rho,  t = (gamma - 1)(G_{1+d} + u_d G_E).
template <int NDIM, int DIR>
TENO_HD inline void flux_vjp(const double (&U)[NDIM + 2], double gamma, const double (&G)[NDIM + 2],
                             double (&out)[NDIM + 2]) {
  constexpr int NV = NDIM + 2;
  constexpr int E = NDIM + 1;
  const double gm1 = gamma - 1.0;
  const double ir = recip(U[0]);
  double u[NDIM], q = 0.0;
  for (int k = 0; k < NDIM; ++k) {
    u[k] = U[1 + k] * ir;
    q += u[k] * u[k];
  }
  const double p = gm1 * (U[E] - 0.5 * U[0] * q);
  double GU = 0.0;
  for (int v = 0; v < NV; ++v) GU += G[v] * U[v];
  const double sc = ir * (GU + p * G[E]);
  const double t = gm1 * (G[1 + DIR] + u[DIR] * G[E]);
  const double ud = u[DIR];
  out[0] = ud * (G[0] - sc) + 0.5 * q * t;
  for (int k = 0; k < NDIM; ++k) out[1 + k] = ud * G[1 + k] - t * u[k] + (k == DIR ? sc : 0.0);
  out[E] = ud * G[E] + t;
}

// The point quantities of one cell that its per-cell adjoint terms share:
// 1/rho, u, |u|^2/2 and p (eq. 4.7).
template <int NDIM>
struct CellPrim {
  double ir, u[NDIM], hq, p;
};

template <int NDIM>
TENO_HD inline void cell_prim(const double (&U)[NDIM + 2], double gamma, CellPrim<NDIM>& P) {
  P.ir = recip(U[0]);
  double q = 0.0;
  for (int k = 0; k < NDIM; ++k) {
    P.u[k] = U[1 + k] * P.ir;
    q = fma(P.u[k], P.u[k], q);
  }
  P.hq = 0.5 * q;
  P.p = (gamma - 1.0) * fma(-U[0], P.hq, U[NDIM + 1]);
}

// acc += A(U)^T G, the product of flux_vjp, from the cell's CellPrim.
template <int NDIM, int DIR>
TENO_HD inline void flux_vjp_acc(const double (&U)[NDIM + 2], const CellPrim<NDIM>& P, double gamma,
                                 const double (&G)[NDIM + 2], double (&acc)[NDIM + 2]) {
  constexpr int NV = NDIM + 2;
  constexpr int E = NDIM + 1;
  double GU = G[0] * U[0];
  for (int v = 1; v < NV; ++v) GU = fma(G[v], U[v], GU);
  const double sc = P.ir * fma(P.p, G[E], GU);
  const double ud = P.u[DIR];
  const double t = (gamma - 1.0) * fma(ud, G[E], G[1 + DIR]);
  acc[0] = fma(ud, G[0] - sc, fma(P.hq, t, acc[0]));
  for (int k = 0; k < NDIM; ++k) acc[1 + k] = fma(ud, G[1 + k], fma(-t, P.u[k], acc[1 + k]));
  acc[1 + DIR] += sc;
  acc[E] = fma(ud, G[E], acc[E] + t);
}

// Roe state of cells i (a) and i+1 (b) with the point quantities its
// derivative needs.  (The adjoint's kept pass fills only what
// kept_roe_scaled reads: sa, sb, iS, duh, dH and the averaged state with
// its halved coefficients.)
template <int NDIM>
struct RoeState {
  double sa, sb, iS, ira, irb, ua[NDIM], ub[NDIM], qa, qb, Ha, Hb;
  double duh[NDIM], dH;   // (u_a - u_b)/2, H_a - H_b
  double ut[NDIM], q2, H, c2, ic, ic2, c, b1, b2;
  double hb1, hb2, hic, b1ic2;   // b1/2, b2/2, 1/(2c), b1/c^2
};

// The averaged state from sqrt(rho), (E+p)/sqrt(rho), u and the differences.
template <int NDIM>
TENO_HD inline void roe_average(double gamma, RoeState<NDIM>& R) {
  const double gm1 = gamma - 1.0;
  R.c2 = gm1 * (R.H - 0.5 * R.q2);
#ifdef __CUDA_ARCH__
  R.ic = rsqrt(R.c2);
#else
  R.ic = 1.0 / sqrt(R.c2);
#endif
  R.ic2 = R.ic * R.ic;
  R.c = R.c2 * R.ic;
  R.b1 = gm1 * R.ic2;
  R.b2 = 0.5 * R.b1 * R.q2;
  R.hb1 = 0.5 * R.b1;
  R.hb2 = 0.5 * R.b2;
  R.hic = 0.5 * R.ic;
  R.b1ic2 = R.b1 * R.ic2;
}

// From sqrt(rho), (E + p)/sqrt(rho) and u of both cells (one reciprocal each).
template <int NDIM>
TENO_HD inline void roe_from_primitives(double sa, double sb, double sha, double shb, const double (&ua)[NDIM],
                                        const double (&ub)[NDIM], double gamma, RoeState<NDIM>& R) {
  const double rsa = recip(sa), rsb = recip(sb);
  R.sa = sa;
  R.sb = sb;
  R.ira = rsa * rsa;
  R.irb = rsb * rsb;
  R.Ha = sha * rsa;
  R.Hb = shb * rsb;
  R.iS = recip(sa + sb);
  R.qa = R.qb = R.q2 = 0.0;
  for (int k = 0; k < NDIM; ++k) {
    R.ua[k] = ua[k];
    R.ub[k] = ub[k];
    R.qa += ua[k] * ua[k];
    R.qb += ub[k] * ub[k];
    R.ut[k] = (sa * ua[k] + sb * ub[k]) * R.iS;
    R.q2 += R.ut[k] * R.ut[k];
  }
  R.H = (sha + shb) * R.iS;
  for (int k = 0; k < NDIM; ++k) R.duh[k] = 0.5 * (ua[k] - ub[k]);
  R.dH = R.Ha - R.Hb;
  roe_average<NDIM>(gamma, R);
}

// From the conservative states of both cells.
template <int NDIM>
TENO_HD inline void roe_from_conservative(const double (&Ua)[NDIM + 2], const double (&Ub)[NDIM + 2], double gamma,
                                          RoeState<NDIM>& R) {
  constexpr int E = NDIM + 1;
  const double gm1 = gamma - 1.0;
  const double ira = 1.0 / Ua[0], irb = 1.0 / Ub[0];
  double ua[NDIM], ub[NDIM], qa = 0.0, qb = 0.0;
  for (int k = 0; k < NDIM; ++k) {
    ua[k] = Ua[1 + k] * ira;
    ub[k] = Ub[1 + k] * irb;
    qa += ua[k] * ua[k];
    qb += ub[k] * ub[k];
  }
  const double pa = gm1 * (Ua[E] - 0.5 * Ua[0] * qa), pb = gm1 * (Ub[E] - 0.5 * Ub[0] * qb);
  const double sa = sqrt(Ua[0]), sb = sqrt(Ub[0]);
  roe_from_primitives<NDIM>(sa, sb, (Ua[E] + pa) / sa, (Ub[E] + pb) / sb, ua, ub, gamma, R);
}

// out += dJ/dU at one of the two Roe cells, from the adjoints of its Roe
// parameters sx = sqrt(rho), Hx = (E + p)/rho and u (ir = 1/rho, q = |u|^2):
// with p = (gamma-1)(E - rho q/2), dHx = (dE + dp - Hx drho)/rho and
// du = (dm - u drho)/rho.
template <int NDIM>
TENO_HD inline void roe_point_vjp(double ir, const double (&u)[NDIM], double q, double sx, double Hx,
                                  double gamma, double sxb, double Hxb, const double (&uxb)[NDIM],
                                  double (&out)[NDIM + 2]) {
  constexpr int E = NDIM + 1;
  const double gm1 = gamma - 1.0;
  double uub = 0.0;
  for (int k = 0; k < NDIM; ++k) uub = fma(u[k], uxb[k], uub);
  const double pb = Hxb * ir;
  // d/drho: sx/(2 rho) sxb + pb ((gamma-1) q/2 - Hx) - u.uxb / rho
  out[0] += fma(0.5 * sx * ir, sxb, fma(pb, fma(0.5 * gm1, q, -Hx), -ir * uub));
  const double gpb = gm1 * pb;
  for (int k = 0; k < NDIM; ++k) out[1 + k] += fma(ir, uxb[k], -gpb * u[k]);
  out[E] = fma(gamma, pb, out[E]);   // pb + (gamma-1) pb
}

// The interface part of the all-kept VJP: from the Roe state of cells i,
// i+1, U~ and Fbar, returns U~bar, the Roe-parameter terms of cells i (roeA)
// and i+1 (roeB), and dJ/dalpha (ab[1] receives the whole derivative with
// respect to a_mid; the other middle entries are zero).
// The Roe-parameter terms are returned as the adjoints of cell a's and cell
// b's own parameters, pa and pb = (d/dsqrt(rho), d/du_0..d/du_{NDIM-1},
// d/dH); roe_param_vjp turns them into conservative terms, so that a cell
// reached by several interfaces applies that per-cell map once to their sum.
//
// kept_roe_scaled is the same computation with its inputs scaled: Ut = s U~,
// Fb = Fbar / f, and the speeds passed as amid = f a_mid, d0 = f (a_0 -
// a_mid), dE = f (a_E - a_mid), iSx = iS / s (iS = 1/(s_a + s_b)).  Every
// output is bilinear in (U~, Fbar) except U~bar, which is linear in Fbar
// alone, so U~bar, pa and pb come out unscaled and ab scaled by s / f.
template <int NDIM, int DIR>
TENO_HD inline void kept_roe_scaled(const RoeState<NDIM>& R, const double (&Ut)[NDIM + 2], double amid,
                                    double d0, double dE, double iSx, double gamma, const double (&Fb)[NDIM + 2],
                                    double (&Utb)[NDIM + 2], double (&pa)[NDIM + 2], double (&pb)[NDIM + 2],
                                    double (&ab)[NDIM + 2]) {
  constexpr int NV = NDIM + 2;
  constexpr int E = NDIM + 1;
  constexpr int N = DIR;
  const double gm1 = gamma - 1.0;
  const double sa = R.sa, sb = R.sb, H = R.H;
  const double q2 = R.q2, c = R.c, b1 = R.b1;
  const double hb1 = R.hb1, hb2 = R.hb2, hic = R.hic;
  const double* ut = R.ut;
  const double un = ut[N];

  // l_0 . X = A + B, l_E . X = A - B with A = (b2 X0 - b1 (u.Xm - XE))/2, B = (un X0 - X_{1+n})/(2c)
  double Sx = -Ut[E];
  for (int k = 0; k < NDIM; ++k) Sx = fma(ut[k], Ut[1 + k], Sx);
  const double Ax = fma(hb2, Ut[0], -hb1 * Sx);
  const double Bx = fma(un, Ut[0], -Ut[1 + N]) * hic;
  const double l0U = Ax + Bx, lEU = Ax - Bx;
  // r_0 . Fb and r_E . Fb
  double rs = fma(H, Fb[E], Fb[0]);
  for (int k = 0; k < NDIM; ++k) rs = fma(ut[k], Fb[1 + k], rs);
  const double rdn = fma(un, Fb[E], Fb[1 + N]);
  const double rho0 = fma(-c, rdn, rs), rhoE = fma(c, rdn, rs);

  // ---- alpha ---------------------------------------------------------------
  double FU = Fb[0] * Ut[0];
  for (int v = 1; v < NV; ++v) FU = fma(Fb[v], Ut[v], FU);
  for (int s = 1; s < NV - 1; ++s) ab[s] = 0.0;
  ab[0] = rho0 * l0U;
  ab[E] = rhoE * lEU;
  ab[1] = FU - ab[0] - ab[E];

  // ---- U~ bar = a_mid Fb + d0 rho0 l_0 + dE rhoE l_E ---------------------------
  const double wE = dE * rhoE;
  const double sX = fma(d0, rho0, wE), dX = fma(d0, rho0, -wE);
  const double hb1sX = hb1 * sX, hicdX = hic * dX;
  Utb[0] = fma(amid, Fb[0], fma(hb2, sX, un * hicdX));
  for (int k = 0; k < NDIM; ++k) {
    double t = fma(-hb1sX, ut[k], amid * Fb[1 + k]);
    if (k == N) t -= hicdX;
    Utb[1 + k] = t;
  }
  Utb[E] = fma(amid, Fb[E], hb1sX);

  // ---- gradients of the Roe parameters -------------------------------------
  // L rows 0 and E contracted with X0 = w0 U~ and XE = wE U~ (the terms of
  // l_0 and l_E in b2, b1, u~ and c), R columns 0 and E with fchar_0 = g0,
  // fchar_E = gE (the other rows / columns do not enter the closed form),
  // with sX = w0 + wE, dX = w0 - wE:
  //   b2bar = sX U~_0 / 2,   b1bar = -sX Sx / 2 + q2 b2bar / 2,
  //   cbar  = dX (U~_{1+n} - un U~_0) / (2 c^2) + (gE - g0)(Fb_{1+n} + un Fb_E),
  // and U~_{1+n} - un U~_0 = -2 c B, so the first term of cbar is -dX B / c.
  // fchar_0 = g0 = d0 l_0.U~ and fchar_E = gE = dE l_E.U~ enter as their
  // sum fs and difference fd
  double utb[NDIM];
  const double gE = dE * lEU;
  const double fs = fma(d0, l0U, gE), fd = fma(-d0, l0U, gE);
  for (int k = 0; k < NDIM; ++k) utb[k] = fma(-hb1sX, Ut[1 + k], Fb[1 + k] * fs);
  utb[N] = fma(hicdX, Ut[0], fma(c * Fb[E], fd, utb[N]));
  const double hsX = 0.5 * sX;
  const double b2b = hsX * Ut[0];
  const double b1b = fma(0.5 * q2, b2b, -hsX * Sx);
  const double cb = fma(-2.0 * hicdX, Bx, fd * rdn);   // ic dX = 2 hic dX
  const double c2b = fma(-R.b1ic2, b1b, hic * cb);
  const double Hbar = fma(gm1, c2b, Fb[E] * fs);
  // twice the q2 adjoint: 2 (b1/2 b2bar - (gamma-1)/2 c2bar)
  const double tq = fma(-gm1, c2b, b1 * b2b);
  for (int k = 0; k < NDIM; ++k) utb[k] = fma(tq, ut[k], utb[k]);
  // u~ = (sa ua + sb ub)/S and H~ = (sa Ha + sb Hb)/S, S = sa + sb, so
  // d/dsa = sb (x_a - x_b)/S^2 and d/dsb = -sa (x_a - x_b)/S^2 for x = u, H
  double Du = 0.0;
  for (int k = 0; k < NDIM; ++k) Du = fma(R.duh[k], utb[k], Du);
  const double Dsum = fma(2.0, Du, R.dH * Hbar);
  const double tS = R.iS * iSx * Dsum;
  const double saS = sa * iSx, sbS = sb * iSx;
  pa[0] = sb * tS;
  pb[0] = -sa * tS;
  for (int k = 0; k < NDIM; ++k) {
    pa[1 + k] = saS * utb[k];
    pb[1 + k] = sbS * utb[k];
  }
  pa[E] = saS * Hbar;
  pb[E] = sbS * Hbar;
}

template <int NDIM, int DIR>
TENO_HD inline void interface_vjp_kept_roe(const RoeState<NDIM>& R, const double (&Ut)[NDIM + 2],
                                           const double (&alpha)[NDIM + 2], double gamma,
                                           const double (&Fb)[NDIM + 2], double (&Utb)[NDIM + 2],
                                           double (&pa)[NDIM + 2], double (&pb)[NDIM + 2],
                                           double (&ab)[NDIM + 2]) {
  constexpr int E = NDIM + 1;
  kept_roe_scaled<NDIM, DIR>(R, Ut, alpha[1], alpha[0] - alpha[1], alpha[E] - alpha[1], R.iS, gamma, Fb, Utb, pa,
                             pb, ab);
}

// out += dJ/dU at one cell from the adjoints p = (d/dsqrt(rho), d/du, d/dH)
// of its Roe parameters (ir = 1/rho, q = |u|^2, sx = sqrt(rho), Hx = (E+p)/rho).
template <int NDIM>
TENO_HD inline void roe_param_vjp(double ir, const double (&u)[NDIM], double q, double sx, double Hx,
                                  double gamma, const double (&p)[NDIM + 2], double (&out)[NDIM + 2]) {
  double uxb[NDIM];
  for (int k = 0; k < NDIM; ++k) uxb[k] = p[1 + k];
  roe_point_vjp<NDIM>(ir, u, q, sx, Hx, gamma, p[0], p[NDIM + 1], uxb, out);
}

// acc += dJ/dU at one cell from the adjoints rp = (d/dsqrt(rho), d/du,
// d/dH) of its Roe parameters, as roe_param_vjp, from the cell's CellPrim
// (sx = sqrt(rho), Hx = (E+p)/rho).
template <int NDIM>
TENO_HD inline void roe_param_vjp_acc(const CellPrim<NDIM>& P, double sx, double Hx, double gamma,
                                      const double (&rp)[NDIM + 2], double (&acc)[NDIM + 2]) {
  constexpr int E = NDIM + 1;
  const double gm1 = gamma - 1.0;
  double uub = 0.0;
  for (int k = 0; k < NDIM; ++k) uub = fma(P.u[k], rp[1 + k], uub);
  const double hb = rp[E] * P.ir;
  acc[0] += fma(0.5 * sx * P.ir, rp[0], fma(hb, fma(gm1, P.hq, -Hx), -P.ir * uub));
  const double ghb = gm1 * hb;
  for (int k = 0; k < NDIM; ++k) acc[1 + k] += fma(P.ir, rp[1 + k], -ghb * P.u[k]);
  acc[E] = fma(gamma, hb, acc[E]);
}

// The interface part of the all-kept VJP with the Roe-parameter terms of
// cells i (roeA) and i+1 (roeB) in conservative form.
template <int NDIM, int DIR>
TENO_HD inline void interface_vjp_kept_ifc(const RoeState<NDIM>& R, const double (&Ut)[NDIM + 2],
                                           const double (&alpha)[NDIM + 2], double gamma,
                                           const double (&Fb)[NDIM + 2], double (&Utb)[NDIM + 2],
                                           double (&roeA)[NDIM + 2], double (&roeB)[NDIM + 2],
                                           double (&ab)[NDIM + 2]) {
  constexpr int NV = NDIM + 2;
  double pa[NV], pb[NV];
  interface_vjp_kept_roe<NDIM, DIR>(R, Ut, alpha, gamma, Fb, Utb, pa, pb, ab);
  for (int v = 0; v < NV; ++v) roeA[v] = roeB[v] = 0.0;
  roe_param_vjp<NDIM>(R.ira, R.ua, R.qa, R.sa, R.Ha, gamma, pa, roeA);
  roe_param_vjp<NDIM>(R.irb, R.ub, R.qb, R.sb, R.Hb, gamma, pb, roeB);
}

// The whole all-kept VJP of one interface, as interface_vjp (same inputs and
// outputs): the interface part plus P_j A(U_j)^T Fbar at every point (left
// out with EXCL_P, as in interface_vjp).
template <int NDIM, int DIR, bool EXCL_P = false>
TENO_HD inline void interface_vjp_kept(const double (&Up)[6][NDIM + 2], const double (&alpha)[NDIM + 2],
                                       double gamma, const double (&Fb)[NDIM + 2],
                                       double (&Ub)[6][NDIM + 2], double (&ab)[NDIM + 2]) {
  constexpr int NV = NDIM + 2;
  const double P[6] = {1.0 / 60.0, -8.0 / 60.0, 37.0 / 60.0, 37.0 / 60.0, -8.0 / 60.0, 1.0 / 60.0};
  const double M[6] = {1.0 / 60.0, -5.0 / 60.0, 10.0 / 60.0, -10.0 / 60.0, 5.0 / 60.0, -1.0 / 60.0};
  double Ut[NV];
  for (int v = 0; v < NV; ++v) {
    Ut[v] = 0.0;
    for (int j = 0; j < 6; ++j) Ut[v] += M[j] * Up[j][v];
  }
  RoeState<NDIM> R;
  roe_from_conservative<NDIM>(Up[2], Up[3], gamma, R);
  double Utb[NV], roeA[NV], roeB[NV];
  interface_vjp_kept_ifc<NDIM, DIR>(R, Ut, alpha, gamma, Fb, Utb, roeA, roeB, ab);
  for (int j = 0; j < 6; ++j) {
    if (EXCL_P) {
      for (int v = 0; v < NV; ++v) Ub[j][v] = M[j] * Utb[v];
    } else {
      double G[NV];
      for (int v = 0; v < NV; ++v) G[v] = P[j] * Fb[v];
      flux_vjp<NDIM, DIR>(Up[j], gamma, G, Ub[j]);
      for (int v = 0; v < NV; ++v) Ub[j][v] += M[j] * Utb[v];
    }
  }
  for (int v = 0; v < NV; ++v) {
    Ub[2][v] += roeA[v];
    Ub[3][v] += roeB[v];
  }
}

// d|lambda|/dU at one cell for lambda = u_d - c (kind 0), u_d (kind 1) or
// u_d + c (kind 2), c = sqrt(gamma p / rho); returns the gradient scaled by s.
template <int NDIM>
TENO_HD inline void wave_speed_grad(const double (&Uc)[NDIM + 2], int d, int kind, double gamma,
                                    double s, double (&out)[NDIM + 2]) {
  constexpr int E = NDIM + 1;
  const double gm1 = gamma - 1.0;
  const double rho = Uc[0];
  double u[NDIM], q = 0.0;
  for (int k = 0; k < NDIM; ++k) {
    u[k] = Uc[1 + k] / rho;
    q += u[k] * u[k];
  }
  const double p = gm1 * (Uc[E] - 0.5 * rho * q);
  const double c = sqrt(gamma * p / rho);
  const double lam = kind == 0 ? u[d] - c : (kind == 1 ? u[d] : u[d] + c);
  const double sg = lam > 0.0 ? 1.0 : (lam < 0.0 ? -1.0 : 0.0);
  const double cs = kind == 0 ? -1.0 : (kind == 1 ? 0.0 : 1.0);   // d lambda / d c
  // d u_d / dU
  double g[NDIM + 2];
  for (int i = 0; i < NDIM + 2; ++i) g[i] = 0.0;
  g[0] += -u[d] / rho;
  g[1 + d] += 1.0 / rho;
  // d c / dU: c = sqrt(gamma p / rho); dc = gamma/(2 rho c) dp - c/(2 rho) drho
  const double cp = gamma / (2.0 * rho * c), cr = -c / (2.0 * rho);
  // dp/drho = gm1 q / 2, dp/dm_k = -gm1 u_k, dp/dE = gm1
  g[0] += cs * (cp * 0.5 * gm1 * q + cr);
  for (int k = 0; k < NDIM; ++k) g[1 + k] += cs * cp * (-gm1 * u[k]);
  g[E] += cs * cp * gm1;
  for (int i = 0; i < NDIM + 2; ++i) out[i] += s * sg * g[i];
}

}  // namespace teno_adj
