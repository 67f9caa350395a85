// adjoint_core_host.cpp -- test helper: the adjoint core's interface VJPs
// (teno_adjoint_core.cuh, plain binary64 host code) behind a C interface for
// the CPU tests.  3D, nvar = 5; arrays row-major as declared.
#include <cstring>

#include "teno_adjoint_core.cuh"

namespace {

template <int DIR>
void run(int kept, const double* up, const double* al, double gamma, const double* fb, double* ub, double* ab) {
  double Up[6][5], alpha[5], Fb[5], Ub[6][5], Ab[5];
  std::memcpy(Up, up, sizeof(Up));
  std::memcpy(alpha, al, sizeof(alpha));
  std::memcpy(Fb, fb, sizeof(Fb));
  if (kept) {
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

extern "C" void adj_interface_vjp3(int dir, int kept, const double* up, const double* al, double gamma,
                                   const double* fb, double* ub, double* ab) {
  if (dir == 0) run<0>(kept, up, al, gamma, fb, ub, ab);
  else if (dir == 1) run<1>(kept, up, al, gamma, fb, ub, ab);
  else run<2>(kept, up, al, gamma, fb, ub, ab);
}
