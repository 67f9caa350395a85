// adjoint_core_host.cpp -- test helper: the adjoint core's interface VJPs
// (teno_adjoint_core.cuh, plain binary64 host code) behind a C interface for
// the CPU tests.  3D, nvar = 5; arrays row-major as declared.
#include <cmath>
#include <cstring>

#include "teno_adjoint_core.cuh"

namespace {

// The all-kept VJP assembled as the adjoint kernels assemble it: the kept
// pass's interface part with the Roe-parameter adjoints of cells i and i+1
// (interface_vjp_kept_roe), then per point the gather's per-cell maps
// (flux_vjp_acc with P_j Fbar, M_j U~bar, and roe_param_vjp_acc at j = 2, 3).
template <int DIR>
void split(const double (&Up)[6][5], const double (&alpha)[5], double gamma, const double (&Fb)[5],
           double (&Ub)[6][5], double (&Ab)[5]) {
  const double P[6] = {1.0 / 60.0, -8.0 / 60.0, 37.0 / 60.0, 37.0 / 60.0, -8.0 / 60.0, 1.0 / 60.0};
  const double M[6] = {1.0 / 60.0, -5.0 / 60.0, 10.0 / 60.0, -10.0 / 60.0, 5.0 / 60.0, -1.0 / 60.0};
  double Ut[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int v = 0; v < 5; ++v)
    for (int j = 0; j < 6; ++j) Ut[v] += M[j] * Up[j][v];
  teno_adj::RoeState<3> R;
  teno_adj::roe_from_conservative<3>(Up[2], Up[3], gamma, R);
  double Utb[5], pa[5], pb[5];
  teno_adj::interface_vjp_kept_roe<3, DIR>(R, Ut, alpha, gamma, Fb, Utb, pa, pb, Ab);
  for (int j = 0; j < 6; ++j) {
    teno_adj::CellPrim<3> C;
    teno_adj::cell_prim<3>(Up[j], gamma, C);
    double G[5];
    for (int v = 0; v < 5; ++v) {
      Ub[j][v] = M[j] * Utb[v];
      G[v] = P[j] * Fb[v];
    }
    teno_adj::flux_vjp_acc<3, DIR>(Up[j], C, gamma, G, Ub[j]);
    if (j == 2 || j == 3) {
      const double sx = std::sqrt(Up[j][0]);
      const double Hx = (Up[j][4] + C.p) * C.ir;
      teno_adj::roe_param_vjp_acc<3>(C, sx, Hx, gamma, j == 2 ? pa : pb, Ub[j]);
    }
  }
}

template <int DIR>
void run(int kept, const double* up, const double* al, double gamma, const double* fb, double* ub, double* ab) {
  double Up[6][5], alpha[5], Fb[5], Ub[6][5], Ab[5];
  std::memcpy(Up, up, sizeof(Up));
  std::memcpy(alpha, al, sizeof(alpha));
  std::memcpy(Fb, fb, sizeof(Fb));
  if (kept == 2) {
    split<DIR>(Up, alpha, gamma, Fb, Ub, Ab);
  } else if (kept) {
    teno_adj::interface_vjp_kept<3, DIR>(Up, alpha, gamma, Fb, Ub, Ab);
  } else {
    const unsigned sel[5][2] = {{7u, 7u}, {7u, 7u}, {7u, 7u}, {7u, 7u}, {7u, 7u}};
    teno_adj::interface_vjp<3, DIR>(Up, alpha, sel, gamma, Fb, Ub, Ab);
  }
  std::memcpy(ub, Ub, sizeof(Ub));
  std::memcpy(ab, Ab, sizeof(Ab));
}

}  // namespace

extern "C" void adj_flux_vjp3(int dir, const double* u, double gamma, const double* g, double* out) {
  double U[5], G[5], O[5];
  std::memcpy(U, u, sizeof(U));
  std::memcpy(G, g, sizeof(G));
  if (dir == 0) teno_adj::flux_vjp<3, 0>(U, gamma, G, O);
  else if (dir == 1) teno_adj::flux_vjp<3, 1>(U, gamma, G, O);
  else teno_adj::flux_vjp<3, 2>(U, gamma, G, O);
  std::memcpy(out, O, sizeof(O));
}

// acc += A(U)^T G through the cell's shared primitives (flux_vjp_acc)
extern "C" void adj_flux_vjp_acc3(int dir, const double* u, double gamma, const double* g, double* acc) {
  double U[5], G[5], A[5];
  std::memcpy(U, u, sizeof(U));
  std::memcpy(G, g, sizeof(G));
  std::memcpy(A, acc, sizeof(A));
  teno_adj::CellPrim<3> C;
  teno_adj::cell_prim<3>(U, gamma, C);
  if (dir == 0) teno_adj::flux_vjp_acc<3, 0>(U, C, gamma, G, A);
  else if (dir == 1) teno_adj::flux_vjp_acc<3, 1>(U, C, gamma, G, A);
  else teno_adj::flux_vjp_acc<3, 2>(U, C, gamma, G, A);
  std::memcpy(acc, A, sizeof(A));
}

// The general VJP with selections sel[5][2] (delta bits), whole (excl = 0)
// or without the all-kept flux term P_j A(U_j)^T Fbar (excl = 1).
template <int DIR>
void sel_run(int excl, const double* up, const double* al, const unsigned* sl, double gamma, const double* fb,
             double* ub, double* ab) {
  double Up[6][5], alpha[5], Fb[5], Ub[6][5], Ab[5];
  unsigned sel[5][2];
  std::memcpy(Up, up, sizeof(Up));
  std::memcpy(alpha, al, sizeof(alpha));
  std::memcpy(Fb, fb, sizeof(Fb));
  std::memcpy(sel, sl, sizeof(sel));
  if (excl) teno_adj::interface_vjp<3, DIR, true>(Up, alpha, sel, gamma, Fb, Ub, Ab);
  else teno_adj::interface_vjp<3, DIR, false>(Up, alpha, sel, gamma, Fb, Ub, Ab);
  std::memcpy(ub, Ub, sizeof(Ub));
  std::memcpy(ab, Ab, sizeof(Ab));
}

extern "C" void adj_interface_vjp3_sel(int dir, int excl, const double* up, const double* al, const unsigned* sel,
                                       double gamma, const double* fb, double* ub, double* ab) {
  if (dir == 0) sel_run<0>(excl, up, al, sel, gamma, fb, ub, ab);
  else if (dir == 1) sel_run<1>(excl, up, al, sel, gamma, fb, ub, ab);
  else sel_run<2>(excl, up, al, sel, gamma, fb, ub, ab);
}

// The kept pass's scaled form (kept_roe_scaled) with U~ times s, Fbar over f
// and the speeds times f, against the unscaled one: out[0..4] U~bar,
// out[5..9] pa, out[10..14] pb, out[15..19] ab; both calls' results.
extern "C" void adj_kept_scaled3(int dir, const double* up, const double* al, double gamma, const double* fb,
                                 double s, double f, double* plain, double* scaled) {
  double Up[6][5], alpha[5], Fb[5], Fs[5], Ut[5] = {0, 0, 0, 0, 0}, Us[5];
  std::memcpy(Up, up, sizeof(Up));
  std::memcpy(alpha, al, sizeof(alpha));
  std::memcpy(Fb, fb, sizeof(Fb));
  const double M[6] = {1.0 / 60.0, -5.0 / 60.0, 10.0 / 60.0, -10.0 / 60.0, 5.0 / 60.0, -1.0 / 60.0};
  for (int v = 0; v < 5; ++v) {
    for (int j = 0; j < 6; ++j) Ut[v] += M[j] * Up[j][v];
    Us[v] = s * Ut[v];
    Fs[v] = Fb[v] / f;
  }
  teno_adj::RoeState<3> R;
  teno_adj::roe_from_conservative<3>(Up[2], Up[3], gamma, R);
  double o[4][5];
  auto run = [&](double* out, bool sc) {
    if (dir == 0) {
      if (sc) teno_adj::kept_roe_scaled<3, 0>(R, Us, f * alpha[1], f * (alpha[0] - alpha[1]), f * (alpha[4] - alpha[1]), R.iS / s, gamma, Fs, o[0], o[1], o[2], o[3]);
      else teno_adj::interface_vjp_kept_roe<3, 0>(R, Ut, alpha, gamma, Fb, o[0], o[1], o[2], o[3]);
    } else if (dir == 1) {
      if (sc) teno_adj::kept_roe_scaled<3, 1>(R, Us, f * alpha[1], f * (alpha[0] - alpha[1]), f * (alpha[4] - alpha[1]), R.iS / s, gamma, Fs, o[0], o[1], o[2], o[3]);
      else teno_adj::interface_vjp_kept_roe<3, 1>(R, Ut, alpha, gamma, Fb, o[0], o[1], o[2], o[3]);
    } else {
      if (sc) teno_adj::kept_roe_scaled<3, 2>(R, Us, f * alpha[1], f * (alpha[0] - alpha[1]), f * (alpha[4] - alpha[1]), R.iS / s, gamma, Fs, o[0], o[1], o[2], o[3]);
      else teno_adj::interface_vjp_kept_roe<3, 2>(R, Ut, alpha, gamma, Fb, o[0], o[1], o[2], o[3]);
    }
    std::memcpy(out, o, sizeof(o));
  };
  run(plain, false);
  run(scaled, true);
}

// kept: 0 = the general VJP with every stencil selected, 1 = the all-kept
// closed form, 2 = the closed form split as the kernels split it
extern "C" void adj_interface_vjp3(int dir, int kept, const double* up, const double* al, double gamma,
                                   const double* fb, double* ub, double* ab) {
  if (dir == 0) run<0>(kept, up, al, gamma, fb, ub, ab);
  else if (dir == 1) run<1>(kept, up, al, gamma, fb, ub, ab);
  else run<2>(kept, up, al, gamma, fb, ub, ab);
}
