/*
 * teno_oracle.c -- plain, slow, FP64 CPU oracle for the TENO5-LAD Euler
 * right-hand side (Peng, Li, Shen, Liu, Zhang, "An efficient targeted ENO
 * scheme with local adaptive dissipation for compressible flow simulation",
 * arXiv 2003.09145).
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load this file.  The GPU library shares no
 * code, header, table or constant with it, and the product path never calls
 * it.
 *
 * Every function restates one step of the paper in plain loops, in the
 * paper's order and notation, with no blocking, fusion or reordering:
 *   - candidate fluxes, eq. 2.4-2.6; linear weights c_k (Sec. 2);
 *   - smoothness indicators beta_k, eq. 2.9-2.11; tau_5, eq. 2.12;
 *   - LAD cutoff: chi~_k and theta (eq. 3.2), m (eq. 3.1), Ladder (eq. 3.3-3.4);
 *   - scale separation gamma_k (eq. 2.8), normalisation (eq. 2.13),
 *     cutoff delta_k (eq. 2.14), weights omega_k (eq. 2.15), flux (eq. 2.7);
 *   - the paper's comparison schemes on the same reconstruction: a fixed
 *     C_T (TENO5, Sec. 2 and Sec. 4), TENO5-A's adaptive C_T (eq. 2.16-2.18)
 *     and WENO-Z weights on tau_5 (eq. 2.12);
 *   - the linear upwind flux, eq. 2.3;
 *   - the Euler flux, eq. 4.7 (extended to 2D/3D by the usual momentum rows);
 *   - global Lax-Friedrichs splitting with characteristic projection (Sec. 4,
 *     the paragraph on convective terms);
 *   - the conservative difference, eq. 2.2;
 *   - the CFL time step, eq. dt1 / dt2; SSP-RK3, eq. 4.1-4.3;
 *   - an exact Riemann solver (textbook pressure-function method) used to
 *     check shock-tube results.
 *
 * Readings of points the paper leaves open (all documented in the design
 * notes): the characteristic eigensystem is the Roe-averaged one with the
 * eigenvector normalisation written in roe_eigensystem(); the LF speed is
 * taken per characteristic field and per direction, as a maximum over all
 * cells, recomputed at every right-hand-side evaluation; the cutoff keeps a
 * stencil when chi_k >= C_T; transmissive boundaries copy the boundary cell
 * into three ghost cells, periodic ones wrap, reflecting ones (the blast-wave
 * test of Sec. 4.2) mirror the cells about the wall with the normal velocity
 * reversed, fixed-state ones (Sec. 4.3.2's top and bottom) hold the given
 * state; the LF speeds and the time step use the interior cells only.  The
 * Rayleigh-Taylor body force of Sec. 4.3.2 (rho added to the y momentum, rho v
 * to the energy) is the source (0, rho g, rho u.g) added to L(U).
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (no FMA contraction,
 * so every product and sum is rounded separately as written).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  double gamma; /* ratio of specific heats (eq. 4.7) */
  double H;     /* discontinuity intensity threshold (eq. 3.2) */
  double eps;   /* small value in eq. 2.8 and eq. 3.2 */
  int b_l;      /* lower magnitude bound B_l (eq. 3.1) */
  int b_u;      /* upper magnitude bound B_u (eq. 3.1) */
  int scheme;   /* OR_SCHEME_*: which cutoff / weights (see or_teno5_lad) */
  int ct_m;     /* OR_SCHEME_TENO5: the fixed C_T = 10^-ct_m (Sec. 4: 7) */
  double grav[3];            /* body acceleration: source (0, rho g, rho u.g) (Sec. 4.3.2) */
  double bc_state[3][2][5];  /* bc 3 (fixed state): conservative ghost state of the
                                low [0] and high [1] face of each direction */
} or_params;

/* The reconstruction's cutoff or weights:
 *   LAD    the paper's adaptive C_T = Lad(m) (eq. 3.1-3.4);
 *   TENO5  a fixed C_T = 10^-ct_m (eq. 2.8-2.15; the paper's comparison
 *          scheme uses 1e-7, Sec. 4);
 *   TENO5A the adaptive C_T of eq. 2.16-2.18 (TENO5-A) with the parameters
 *          alpha_1 = 10.5, alpha_2 = 3.5, C_r = 0.25, xi = 1e-3 (Sec. 2);
 *   WENOZ  the WENO-Z weights built on tau_5 of eq. 2.12:
 *          omega_k = alpha_k / sum alpha, alpha_k = c_k (1 + tau_5/(beta_k + eps)). */
enum { OR_SCHEME_LAD = 0, OR_SCHEME_TENO5 = 1, OR_SCHEME_TENO5A = 2, OR_SCHEME_WENOZ = 3 };

/* Diagnostic record of one scalar reconstruction, in the paper's symbols. */
enum {
  OR_D_BETA0 = 0, OR_D_BETA1, OR_D_BETA2, OR_D_TAU,
  OR_D_CHIT0, OR_D_CHIT1, OR_D_CHIT2, OR_D_THETA, OR_D_M, OR_D_CT,
  OR_D_GAMMA0, OR_D_GAMMA1, OR_D_GAMMA2, OR_D_CHI0, OR_D_CHI1, OR_D_CHI2,
  OR_D_F0, OR_D_F1, OR_D_F2, OR_D_OMEGA0, OR_D_OMEGA1, OR_D_OMEGA2, OR_D_FHAT,
  OR_D_ETA, OR_D_MA, OR_D_GA, OR_D_BETAA, /* TENO5-A: eta_{i+1/2}, m, g(m), beta (eq. 2.16-2.17) */
  OR_D_COUNT
};

int or_diag_count(void) { return OR_D_COUNT; }

static double sq(double x) { return x * x; }

/* 10^-k written out as literals, so the Ladder holds the exact decimal
 * constants of eq. 3.3 without any call to pow(). */
static const double or_powers_of_ten_neg[16] = {
    1e-0, 1e-1, 1e-2, 1e-3, 1e-4,  1e-5,  1e-6,  1e-7,
    1e-8, 1e-9, 1e-10, 1e-11, 1e-12, 1e-13, 1e-14, 1e-15};

/* Ladder of eq. 3.3: Lad(m) = 10^-m for m = B_l .. B_u (eq. 3.4). */
double or_ladder(int m) {
  if (m < 0 || m > 15) return NAN;
  return or_powers_of_ten_neg[m];
}

/* Fifth-order upstream-biased flux, eq. 2.3.  v = (f_{i-2}, ..., f_{i+2}). */
double or_upwind5(const double v[5]) {
  return 2.0 / 60.0 * v[0] - 13.0 / 60.0 * v[1] + 47.0 / 60.0 * v[2] +
         27.0 / 60.0 * v[3] - 3.0 / 60.0 * v[4];
}

/*
 * TENO5-A's sensor eta_i of eq. 2.18 at a point whose neighbouring first
 * differences are dp = f_{i+1} - f_i and dm = f_i - f_{i-1}; the denominator
 * is read as (dp)^2 + (dm)^2 + eps (the printed one repeats dp).
 */
static double teno5a_eta(double dp, double dm, double eps_a) {
  return (2.0 * fabs(dp * dm) + eps_a) / (dp * dp + dm * dm + eps_a);
}

/*
 * One TENO5-LAD reconstruction of the interface flux f^_{i+1/2} from the five
 * values v = (f_{i-2}, f_{i-1}, f_i, f_{i+1}, f_{i+2}).
 *
 * forced < 0: the cutoff is computed (eq. 3.1-3.4, 2.8, 2.13, 2.14).
 * forced >= 0: a flag byte whose bits 0..2 give delta_0..delta_2; the weights
 *   of eq. 2.15 are then formed from those bits (used to compare against a
 *   result whose selections are known).
 * flag (nullable) receives bits 0..2 = delta_k and bits 3..6 = m.
 * diag (nullable) receives OR_D_COUNT values (see the enum above).
 */
double or_teno5_lad(const double v[5], const or_params* P, int forced,
                    unsigned char* flag, double* diag) {
  /* eq. 2.4-2.6: third-order candidate fluxes on S0, S1, S2 */
  double f0 = 1.0 / 3.0 * v[0] - 7.0 / 6.0 * v[1] + 11.0 / 6.0 * v[2];
  double f1 = -1.0 / 6.0 * v[1] + 5.0 / 6.0 * v[2] + 1.0 / 3.0 * v[3];
  double f2 = 1.0 / 3.0 * v[2] + 5.0 / 6.0 * v[3] - 1.0 / 6.0 * v[4];
  /* linear weights (Sec. 2) */
  const double c[3] = {0.1, 0.6, 0.3};

  /* eq. 2.9-2.11: Jiang-Shu smoothness indicators */
  double beta[3];
  beta[0] = 13.0 / 12.0 * sq(v[0] - 2.0 * v[1] + v[2]) +
            1.0 / 4.0 * sq(v[0] - 4.0 * v[1] + 3.0 * v[2]);
  beta[1] = 13.0 / 12.0 * sq(v[1] - 2.0 * v[2] + v[3]) +
            1.0 / 4.0 * sq(v[1] - v[3]);
  beta[2] = 13.0 / 12.0 * sq(v[2] - 2.0 * v[3] + v[4]) +
            1.0 / 4.0 * sq(3.0 * v[2] - 4.0 * v[3] + v[4]);

  /* eq. 2.12: global smoothness indicator tau_5 */
  double tau = fabs(beta[2] - beta[0]);

  /* eq. 3.2: chi~_k and the Runge function theta */
  double chit[3];
  for (int k = 0; k < 3; ++k) chit[k] = tau / (beta[k] + P->eps);
  double chit_max = chit[0];
  for (int k = 1; k < 3; ++k)
    if (chit[k] > chit_max) chit_max = chit[k];
  double theta = 1.0 / (1.0 + chit_max / P->H);

  int m;
  double eta = NAN, mA = NAN, gA = NAN, betaA = NAN;
  if (P->scheme == OR_SCHEME_TENO5) {
    /* a fixed cutoff C_T = 10^-ct_m */
    m = P->ct_m;
  } else if (P->scheme == OR_SCHEME_TENO5A) {
    /* eq. 2.16-2.18: eta at the points i-1, i, i+1 of the stencil, their
     * minimum, m = 1 - min(1, eta / C_r), g(m) = (1 - m)^4 (1 + 4 m),
     * beta = alpha_1 - alpha_2 (1 - g(m)), C_T = 10^-floor(beta) */
    const double a1 = 10.5, a2 = 3.5, Cr = 0.25, xi = 1e-3;
    double eps_a = 0.9 * Cr / (1.0 - 0.9 * Cr) * xi * xi;
    double eta_m1 = teno5a_eta(v[2] - v[1], v[1] - v[0], eps_a);
    double eta_0 = teno5a_eta(v[3] - v[2], v[2] - v[1], eps_a);
    double eta_p1 = teno5a_eta(v[4] - v[3], v[3] - v[2], eps_a);
    eta = fmin(eta_m1, fmin(eta_0, eta_p1));
    mA = 1.0 - fmin(1.0, eta / Cr);
    double t = 1.0 - mA;
    double t2 = t * t;
    gA = t2 * t2 * (1.0 + 4.0 * mA);
    betaA = a1 - a2 * (1.0 - gA);
    m = (int)floor(betaA);
  } else {
    /* eq. 3.1: magnitude m (the Ladder of eq. 3.3-3.4 gives C_T below) */
    m = P->b_l + (int)floor(theta * (double)(P->b_u - P->b_l));
  }
  double CT = or_ladder(m);

  /* eq. 2.8: gamma_k = (C + tau/(beta_k + eps))^q with C = 1, q = 6 */
  const double C = 1.0, q = 6.0;
  double gam[3];
  for (int k = 0; k < 3; ++k) gam[k] = pow(C + tau / (beta[k] + P->eps), q);

  /* eq. 2.13: normalisation */
  double gsum = gam[0] + gam[1] + gam[2];
  double chi[3];
  for (int k = 0; k < 3; ++k) chi[k] = gam[k] / gsum;

  /* eq. 2.14: cutoff */
  int delta[3];
  for (int k = 0; k < 3; ++k) delta[k] = (chi[k] < CT) ? 0 : 1;
  if (forced >= 0)
    for (int k = 0; k < 3; ++k) delta[k] = (forced >> k) & 1;

  /* eq. 2.15: TENO weights */
  double dsum = 0.0;
  for (int k = 0; k < 3; ++k) dsum += delta[k] * c[k];
  double omega[3];
  for (int k = 0; k < 3; ++k) omega[k] = delta[k] * c[k] / dsum;

  if (P->scheme == OR_SCHEME_WENOZ) {
    /* WENO-Z: no cutoff; alpha_k = c_k (1 + tau_5 / (beta_k + eps)),
     * omega_k = alpha_k / sum_j alpha_j.  Flag: every delta set, m = 0. */
    double alpha[3], asum = 0.0;
    for (int k = 0; k < 3; ++k) {
      alpha[k] = c[k] * (1.0 + tau / (beta[k] + P->eps));
      asum += alpha[k];
    }
    for (int k = 0; k < 3; ++k) omega[k] = alpha[k] / asum;
    for (int k = 0; k < 3; ++k) delta[k] = 1;
    m = 0;
    CT = 0.0;
  }

  /* eq. 2.7 */
  double fhat = omega[0] * f0 + omega[1] * f1 + omega[2] * f2;

  if (flag)
    *flag = (unsigned char)(delta[0] | (delta[1] << 1) | (delta[2] << 2) |
                            ((m & 15) << 3));
  if (diag) {
    diag[OR_D_BETA0] = beta[0];
    diag[OR_D_BETA1] = beta[1];
    diag[OR_D_BETA2] = beta[2];
    diag[OR_D_TAU] = tau;
    diag[OR_D_CHIT0] = chit[0];
    diag[OR_D_CHIT1] = chit[1];
    diag[OR_D_CHIT2] = chit[2];
    diag[OR_D_THETA] = theta;
    diag[OR_D_M] = (double)m;
    diag[OR_D_CT] = CT;
    diag[OR_D_GAMMA0] = gam[0];
    diag[OR_D_GAMMA1] = gam[1];
    diag[OR_D_GAMMA2] = gam[2];
    diag[OR_D_CHI0] = chi[0];
    diag[OR_D_CHI1] = chi[1];
    diag[OR_D_CHI2] = chi[2];
    diag[OR_D_F0] = f0;
    diag[OR_D_F1] = f1;
    diag[OR_D_F2] = f2;
    diag[OR_D_OMEGA0] = omega[0];
    diag[OR_D_OMEGA1] = omega[1];
    diag[OR_D_OMEGA2] = omega[2];
    diag[OR_D_FHAT] = fhat;
    diag[OR_D_ETA] = eta;
    diag[OR_D_MA] = mA;
    diag[OR_D_GA] = gA;
    diag[OR_D_BETAA] = betaA;
  }
  return fhat;
}

/* ------------------------------------------------------------------------ */
/* Euler system, eq. 4.7: U = (rho, rho u_1..rho u_ndim, E).                 */
/* ------------------------------------------------------------------------ */

#define OR_MAXVAR 5

/* Primitive variables of one cell: density, velocities, pressure (ideal gas,
 * E = p/(gamma-1) + rho |u|^2 / 2, eq. 4.7). */
static void primitive(int ndim, const double* Uc, double gamma, double* rho,
                      double* vel, double* p) {
  int nvar = ndim + 2;
  *rho = Uc[0];
  double q2 = 0.0;
  for (int k = 0; k < ndim; ++k) {
    vel[k] = Uc[1 + k] / Uc[0];
    q2 += vel[k] * vel[k];
  }
  *p = (gamma - 1.0) * (Uc[nvar - 1] - 0.5 * Uc[0] * q2);
}

/* Physical flux along direction d, eq. 4.7: (rho u_d, rho u_k u_d + p
 * delta_kd, u_d (E + p)). */
static void physical_flux(int ndim, int d, const double* Uc, double gamma,
                          double* F) {
  int nvar = ndim + 2;
  double rho, vel[3], p;
  primitive(ndim, Uc, gamma, &rho, vel, &p);
  F[0] = Uc[0] * vel[d];
  for (int k = 0; k < ndim; ++k) F[1 + k] = Uc[1 + k] * vel[d] + (k == d ? p : 0.0);
  F[nvar - 1] = vel[d] * (Uc[nvar - 1] + p);
}

/*
 * Characteristic eigensystem at the interface between cells a and b, for
 * direction d: Roe averages (sqrt(rho)-weighted velocity and enthalpy), then
 * right eigenvectors (columns of R) and left eigenvectors (rows of L = R^-1):
 *   field 0        : u_d - c   r = (1, u - c e_d, H - u_d c)
 *   field 1        : u_d       r = (1, u, |u|^2/2)            (entropy)
 *   fields 2..     : u_d       r = (0, e_t, u_t), t != d       (shear)
 *   field nvar-1   : u_d + c   r = (1, u + c e_d, H + u_d c)
 * with b1 = (gamma-1)/c^2 and b2 = b1 |u|^2 / 2:
 *   l_0      = 1/2 (b2 + u_d/c, -b1 u_k - delta_kd / c, b1)
 *   l_1      = (1 - b2, b1 u_k, -b1)
 *   l_t      = (-u_t, e_t, 0)
 *   l_nvar-1 = 1/2 (b2 - u_d/c, -b1 u_k + delta_kd / c, b1)
 * Returns 0, or -1 when the averaged sound speed is not real.
 */
int or_roe_eigensystem(int ndim, int d, const double* Ua, const double* Ub,
                       double gamma, double* L, double* R) {
  int nvar = ndim + 2;
  double ra, va[3], pa, rb, vb[3], pb;
  primitive(ndim, Ua, gamma, &ra, va, &pa);
  primitive(ndim, Ub, gamma, &rb, vb, &pb);
  double sa = sqrt(ra), sb = sqrt(rb);
  double Ha = (Ua[nvar - 1] + pa) / ra;
  double Hb = (Ub[nvar - 1] + pb) / rb;
  double u[3], q2 = 0.0;
  for (int k = 0; k < ndim; ++k) {
    u[k] = (sa * va[k] + sb * vb[k]) / (sa + sb);
    q2 += u[k] * u[k];
  }
  double H = (sa * Ha + sb * Hb) / (sa + sb);
  double c2 = (gamma - 1.0) * (H - 0.5 * q2);
  if (!(c2 > 0.0)) return -1;
  double c = sqrt(c2);
  double b1 = (gamma - 1.0) / c2;
  double b2 = 0.5 * b1 * q2;

  for (int i = 0; i < nvar * nvar; ++i) L[i] = R[i] = 0.0;
#define RR(row, col) R[(row) * nvar + (col)]
#define LL(row, col) L[(row) * nvar + (col)]
  /* acoustic field u_d - c */
  RR(0, 0) = 1.0;
  for (int k = 0; k < ndim; ++k) RR(1 + k, 0) = u[k] - (k == d ? c : 0.0);
  RR(nvar - 1, 0) = H - u[d] * c;
  LL(0, 0) = 0.5 * (b2 + u[d] / c);
  for (int k = 0; k < ndim; ++k)
    LL(0, 1 + k) = 0.5 * (-b1 * u[k] - (k == d ? 1.0 / c : 0.0));
  LL(0, nvar - 1) = 0.5 * b1;
  /* entropy field u_d */
  RR(0, 1) = 1.0;
  for (int k = 0; k < ndim; ++k) RR(1 + k, 1) = u[k];
  RR(nvar - 1, 1) = 0.5 * q2;
  LL(1, 0) = 1.0 - b2;
  for (int k = 0; k < ndim; ++k) LL(1, 1 + k) = b1 * u[k];
  LL(1, nvar - 1) = -b1;
  /* shear fields u_d, one per tangential direction in increasing order */
  int f = 2;
  for (int t = 0; t < ndim; ++t) {
    if (t == d) continue;
    RR(1 + t, f) = 1.0;
    RR(nvar - 1, f) = u[t];
    LL(f, 0) = -u[t];
    LL(f, 1 + t) = 1.0;
    ++f;
  }
  /* acoustic field u_d + c */
  RR(0, nvar - 1) = 1.0;
  for (int k = 0; k < ndim; ++k) RR(1 + k, nvar - 1) = u[k] + (k == d ? c : 0.0);
  RR(nvar - 1, nvar - 1) = H + u[d] * c;
  LL(nvar - 1, 0) = 0.5 * (b2 - u[d] / c);
  for (int k = 0; k < ndim; ++k)
    LL(nvar - 1, 1 + k) = 0.5 * (-b1 * u[k] + (k == d ? 1.0 / c : 0.0));
  LL(nvar - 1, nvar - 1) = 0.5 * b1;
#undef RR
#undef LL
  return 0;
}

/* Cell index after the boundary treatment: bc 0 = periodic (wrap),
 * bc 1 = transmissive / zero gradient (the boundary cell is copied into the
 * three ghost cells), bc 2 = reflecting (ghost cell -1-k is the mirror image
 * of cell k about the wall; see ghost_reflects for the velocity). */
static int64_t ghost_index(int64_t i, int64_t n, int bc) {
  if (bc == 0) {
    int64_t r = i % n;
    return r < 0 ? r + n : r;
  }
  if (bc == 2) {
    while (i < 0 || i >= n) i = (i < 0) ? -1 - i : 2 * n - 1 - i;
    return i;
  }
  if (i < 0) return 0;
  if (i >= n) return n - 1;
  return i;
}

/* 1 if the point i of a reflecting direction is a mirror image with the
 * normal velocity reversed (an odd number of reflections), else 0. */
static int ghost_reflects(int64_t i, int64_t n, int bc) {
  int odd = 0;
  if (bc != 2) return 0;
  while (i < 0 || i >= n) {
    i = (i < 0) ? -1 - i : 2 * n - 1 - i;
    odd ^= 1;
  }
  return odd;
}

typedef struct {
  int ndim, nvar;
  int64_t n[3];
  int64_t ncell;
} or_shape;

static or_shape make_shape(int ndim, const int64_t* n) {
  or_shape s;
  s.ndim = ndim;
  s.nvar = ndim + 2;
  for (int k = 0; k < 3; ++k) s.n[k] = (k < ndim) ? n[k] : 1;
  s.ncell = s.n[0] * s.n[1] * s.n[2];
  return s;
}

static int64_t cell_linear(const or_shape* s, const int64_t idx[3]) {
  return (idx[2] * s->n[1] + idx[1]) * s->n[0] + idx[0];
}

static void load_cell(const or_shape* s, const double* U, int64_t lin,
                      double* Uc) {
  for (int v = 0; v < s->nvar; ++v) Uc[v] = U[v * s->ncell + lin];
}

/* Number of interfaces of direction d: n_d + 1 along d, n_k along the others. */
int64_t or_num_interfaces(int ndim, const int64_t* n, int d) {
  or_shape s = make_shape(ndim, n);
  int64_t m = 1;
  for (int k = 0; k < 3; ++k) m *= (k == d) ? s.n[k] + 1 : s.n[k];
  return m;
}

/* Offset of direction d's block in the flag array; the block is laid out
 * [field][side: 0 = f^+, 1 = f^-][interface grid with n_d + 1 along d]. */
int64_t or_flag_offset(int ndim, const int64_t* n, int d) {
  int64_t off = 0;
  for (int k = 0; k < d; ++k) off += (int64_t)(ndim + 2) * 2 * or_num_interfaces(ndim, n, k);
  return off;
}

/*
 * Global Lax-Friedrichs speeds for direction d: alpha_s = max over all cells
 * of |lambda_s| with lambda = (u_d - c, u_d, ..., u_d, u_d + c) from each
 * cell's own velocity and sound speed c = sqrt(gamma p / rho).
 * Returns -1 if a cell has non-positive density or pressure.
 */
int or_lf_alpha(int ndim, const int64_t* n, int d, double gamma,
                const double* U, double* alpha) {
  or_shape s = make_shape(ndim, n);
  double amin = 0.0, amid = 0.0, aplus = 0.0;
  int bad = 0;
  for (int64_t lin = 0; lin < s.ncell; ++lin) {
    double Uc[OR_MAXVAR], rho, vel[3], p;
    load_cell(&s, U, lin, Uc);
    primitive(ndim, Uc, gamma, &rho, vel, &p);
    if (!(rho > 0.0) || !(p > 0.0)) bad = 1;
    double c = sqrt(gamma * p / rho);
    double l0 = fabs(vel[d] - c), l1 = fabs(vel[d]), l2 = fabs(vel[d] + c);
    if (l0 > amin) amin = l0;
    if (l1 > amid) amid = l1;
    if (l2 > aplus) aplus = l2;
  }
  alpha[0] = amin;
  for (int f = 1; f < s.nvar - 1; ++f) alpha[f] = amid;
  alpha[s.nvar - 1] = aplus;
  return bad ? -1 : 0;
}

/*
 * Numerical flux at one interface of direction d.  `ifc` is the interface's
 * position on the interface grid (ifc[d] in 0..n_d): it lies between cells
 * ifc[d]-1 and ifc[d].  The six points i-2..i+3 (i = ifc[d]-1) are projected
 * onto the characteristic fields of the Roe state of cells i and i+1, split by
 * global LF (f^+- = (g +- alpha w)/2), reconstructed with TENO5-LAD (f^- on
 * the mirrored stencil), summed and projected back.
 */
static int interface_flux(const or_shape* s, int d, const int64_t ifc[3],
                          const int* bc, const or_params* P, const double* U,
                          const double* alpha, double* Fhat,
                          unsigned char* flags /* [nvar][2] or NULL */,
                          const unsigned char* forced /* [nvar][2] or NULL */,
                          int diag_field, int diag_side, double* diag) {
  int ndim = s->ndim, nvar = s->nvar;
  double Upt[6][OR_MAXVAR], Fpt[6][OR_MAXVAR];
  int64_t base = ifc[d] - 1; /* i */
  for (int j = 0; j < 6; ++j) {
    int64_t idx[3] = {ifc[0], ifc[1], ifc[2]};
    int64_t k = base - 2 + j;
    if (bc[d] == 3 && (k < 0 || k >= s->n[d])) {
      /* fixed-state face: the ghost cell holds the face's state */
      for (int r = 0; r < nvar; ++r) Upt[j][r] = P->bc_state[d][k < 0 ? 0 : 1][r];
      physical_flux(ndim, d, Upt[j], P->gamma, Fpt[j]);
      continue;
    }
    idx[d] = ghost_index(k, s->n[d], bc[d]);
    load_cell(s, U, cell_linear(s, idx), Upt[j]);
    /* reflecting wall: the ghost state has the normal momentum reversed */
    if (ghost_reflects(base - 2 + j, s->n[d], bc[d])) Upt[j][1 + d] = -Upt[j][1 + d];
    physical_flux(ndim, d, Upt[j], P->gamma, Fpt[j]);
  }
  double L[OR_MAXVAR * OR_MAXVAR], R[OR_MAXVAR * OR_MAXVAR];
  /* Roe state of cells i (point 2) and i+1 (point 3) */
  if (or_roe_eigensystem(ndim, d, Upt[2], Upt[3], P->gamma, L, R) != 0) return -1;

  /* characteristic projection w = L U, g = L F at the six points */
  double w[6][OR_MAXVAR], g[6][OR_MAXVAR];
  for (int j = 0; j < 6; ++j)
    for (int r = 0; r < nvar; ++r) {
      double sw = 0.0, sg = 0.0;
      for (int k = 0; k < nvar; ++k) {
        sw += L[r * nvar + k] * Upt[j][k];
        sg += L[r * nvar + k] * Fpt[j][k];
      }
      w[j][r] = sw;
      g[j][r] = sg;
    }

  double fchar[OR_MAXVAR];
  for (int r = 0; r < nvar; ++r) {
    double vp[5], vm[5];
    for (int k = 0; k < 5; ++k) {
      /* f^+ on points i-2..i+2 */
      vp[k] = 0.5 * (g[k][r] + alpha[r] * w[k][r]);
      /* f^- on the mirrored stencil i+3..i-1 */
      vm[k] = 0.5 * (g[5 - k][r] - alpha[r] * w[5 - k][r]);
    }
    unsigned char fp = 0, fm = 0;
    int forced_p = forced ? forced[r * 2 + 0] : -1;
    int forced_m = forced ? forced[r * 2 + 1] : -1;
    double* dp = (diag && diag_field == r && diag_side == 0) ? diag : NULL;
    double* dm = (diag && diag_field == r && diag_side == 1) ? diag : NULL;
    double hp = or_teno5_lad(vp, P, forced_p, &fp, dp);
    double hm = or_teno5_lad(vm, P, forced_m, &fm, dm);
    fchar[r] = hp + hm;
    if (flags) {
      flags[r * 2 + 0] = fp;
      flags[r * 2 + 1] = fm;
    }
  }
  /* back-projection F^ = R f^char */
  for (int r = 0; r < nvar; ++r) {
    double acc = 0.0;
    for (int k = 0; k < nvar; ++k) acc += R[r * nvar + k] * fchar[k];
    Fhat[r] = acc;
  }
  return 0;
}

/*
 * Semi-discrete right-hand side L(U) = - sum_d (F^_{d,i+1/2} - F^_{d,i-1/2}) /
 * dx_d (eq. 2.2), dimension by dimension.
 *   U, Rhs  : [nvar][n_z][n_y][n_x] (x fastest), nvar = ndim + 2.
 *   flags_out (nullable): per interface, field and side, see or_flag_offset().
 *   flags_in  (nullable): same layout; if given, the selections are forced.
 *   alpha_out (nullable): [ndim][nvar] LF speeds used.
 * Returns 0, -1 for a non-physical state.
 */
/* The body-force source of Sec. 4.3.2, S = (0, rho g, rho u.g), of cell lin
 * added to out[r * ostride], r = 0..nvar-1. */
static void add_source(const or_shape* s, const or_params* P, const double* U, int64_t lin, double* out,
                       int64_t ostride) {
  int ndim = s->ndim, nvar = s->nvar;
  double rho = U[lin];
  double w = 0.0;
  for (int k = 0; k < ndim; ++k) {
    out[(1 + k) * ostride] += rho * P->grav[k];
    w += U[(1 + k) * s->ncell + lin] * P->grav[k];
  }
  out[(nvar - 1) * ostride] += w;
}

int or_euler_rhs(int ndim, const int64_t* n, const double* dx, const int* bc,
                 const or_params* P, const double* U, double* Rhs,
                 unsigned char* flags_out, const unsigned char* flags_in,
                 double* alpha_out) {
  or_shape s = make_shape(ndim, n);
  int nvar = s.nvar;
  int status = 0;
  for (int64_t i = 0; i < nvar * s.ncell; ++i) Rhs[i] = 0.0;

  for (int d = 0; d < ndim; ++d) {
    double alpha[OR_MAXVAR];
    if (or_lf_alpha(ndim, n, d, P->gamma, U, alpha) != 0) status = -1;
    if (alpha_out)
      for (int r = 0; r < nvar; ++r) alpha_out[d * nvar + r] = alpha[r];

    /* lines along d: the other two indices */
    int o1 = (d == 0) ? 1 : 0;
    int o2 = (d == 2) ? 1 : 2;
    int64_t nline = s.n[o1] * s.n[o2];
    int64_t nd = s.n[d];
    int64_t nifc = or_num_interfaces(ndim, n, d);
    int64_t foff = or_flag_offset(ndim, n, d);
    int64_t ifc_stride[3];
    {
      int64_t m0 = s.n[0] + (d == 0), m1 = s.n[1] + (d == 1);
      ifc_stride[0] = 1;
      ifc_stride[1] = m0;
      ifc_stride[2] = m0 * m1;
    }
    int line_status = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : line_status)
    for (int64_t line = 0; line < nline; ++line) {
      int64_t a = line % s.n[o1], b = line / s.n[o1];
      double* Fline = (double*)malloc(sizeof(double) * nvar * (nd + 1));
      for (int64_t id = 0; id <= nd; ++id) {
        int64_t ifc[3];
        ifc[d] = id;
        ifc[o1] = a;
        ifc[o2] = b;
        int64_t ilin = ifc[0] * ifc_stride[0] + ifc[1] * ifc_stride[1] +
                       ifc[2] * ifc_stride[2];
        unsigned char fl[2 * OR_MAXVAR], ff[2 * OR_MAXVAR];
        if (flags_in)
          for (int r = 0; r < nvar; ++r)
            for (int side = 0; side < 2; ++side)
              ff[r * 2 + side] = flags_in[foff + (r * 2 + side) * nifc + ilin];
        if (interface_flux(&s, d, ifc, bc, P, U, alpha, Fline + id * nvar, fl,
                           flags_in ? ff : NULL, -1, -1, NULL) != 0)
          line_status |= 1;
        if (flags_out)
          for (int r = 0; r < nvar; ++r)
            for (int side = 0; side < 2; ++side)
              flags_out[foff + (r * 2 + side) * nifc + ilin] = fl[r * 2 + side];
      }
      /* eq. 2.2: conservative difference */
      for (int64_t i = 0; i < nd; ++i) {
        int64_t idx[3];
        idx[d] = i;
        idx[o1] = a;
        idx[o2] = b;
        int64_t lin = cell_linear(&s, idx);
        for (int r = 0; r < nvar; ++r)
          Rhs[r * s.ncell + lin] +=
              -(Fline[(i + 1) * nvar + r] - Fline[i * nvar + r]) / dx[d];
      }
      free(Fline);
    }
    if (line_status) status = -1;
  }
  for (int64_t lin = 0; lin < s.ncell; ++lin) add_source(&s, P, U, lin, Rhs + lin, s.ncell);
  return status;
}

/*
 * The right-hand side of eq. 2.2 at m sampled cells only (same arithmetic as
 * or_euler_rhs; for grids too large to evaluate whole).  cells[k] is a linear
 * cell index; out is [m][nvar].  flags_in / flags_out use the full flag
 * layout of or_euler_rhs (only the entries of the sampled cells' faces are
 * read or written).  alpha_in (nullable, [ndim][nvar]) supplies the LF
 * speeds; otherwise they are computed from U.
 */
int or_euler_rhs_sample(int ndim, const int64_t* n, const double* dx,
                        const int* bc, const or_params* P, const double* U,
                        int64_t m, const int64_t* cells, double* out,
                        unsigned char* flags_out,
                        const unsigned char* flags_in,
                        const double* alpha_in) {
  or_shape s = make_shape(ndim, n);
  int nvar = s.nvar;
  double alpha[3][OR_MAXVAR];
  int status = 0;
  for (int d = 0; d < ndim; ++d) {
    if (alpha_in) {
      for (int r = 0; r < nvar; ++r) alpha[d][r] = alpha_in[d * nvar + r];
    } else if (or_lf_alpha(ndim, n, d, P->gamma, U, alpha[d]) != 0) {
      status = -1;
    }
  }
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : bad)
  for (int64_t k = 0; k < m; ++k) {
    int64_t lin = cells[k];
    int64_t idx[3] = {lin % s.n[0], (lin / s.n[0]) % s.n[1], lin / (s.n[0] * s.n[1])};
    for (int r = 0; r < nvar; ++r) out[k * nvar + r] = 0.0;
    for (int d = 0; d < ndim; ++d) {
      int64_t nifc = or_num_interfaces(ndim, n, d);
      int64_t foff = or_flag_offset(ndim, n, d);
      int64_t m0 = s.n[0] + (d == 0), m1 = s.n[1] + (d == 1);
      double Fh[2][OR_MAXVAR];
      for (int face = 0; face < 2; ++face) {
        int64_t ifc[3] = {idx[0], idx[1], idx[2]};
        ifc[d] += face;
        int64_t ilin = (ifc[2] * m1 + ifc[1]) * m0 + ifc[0];
        unsigned char fl[2 * OR_MAXVAR], ff[2 * OR_MAXVAR];
        if (flags_in)
          for (int r = 0; r < nvar; ++r)
            for (int side = 0; side < 2; ++side)
              ff[r * 2 + side] = flags_in[foff + (r * 2 + side) * nifc + ilin];
        if (interface_flux(&s, d, ifc, bc, P, U, alpha[d], Fh[face], fl,
                           flags_in ? ff : NULL, -1, -1, NULL) != 0)
          bad |= 1;
        if (flags_out)
          for (int r = 0; r < nvar; ++r)
            for (int side = 0; side < 2; ++side)
              flags_out[foff + (r * 2 + side) * nifc + ilin] = fl[r * 2 + side];
      }
      for (int r = 0; r < nvar; ++r)
        out[k * nvar + r] += -(Fh[1][r] - Fh[0][r]) / dx[d];
    }
    add_source(&s, P, U, lin, out + k * nvar, 1);
  }
  return (status || bad) ? -1 : 0;
}

/*
 * Diagnostic record of one scalar reconstruction inside the Euler RHS: the
 * interface `ifc` of direction d, characteristic field r, side 0 (f^+) or
 * 1 (f^-).  Used to classify selector differences that lie on a rounding
 * boundary.  Returns 0 or -1.
 */
int or_euler_interface_diag(int ndim, const int64_t* n, const double* dx,
                            const int* bc, const or_params* P, const double* U,
                            int d, const int64_t* ifc, int field, int side,
                            double* diag) {
  (void)dx;
  or_shape s = make_shape(ndim, n);
  double alpha[OR_MAXVAR], F[OR_MAXVAR];
  or_lf_alpha(ndim, n, d, P->gamma, U, alpha);
  int64_t idx[3] = {ifc[0], ifc[1], ifc[2]};
  return interface_flux(&s, d, idx, bc, P, U, alpha, F, NULL, NULL, field,
                        side, diag);
}

/*
 * CFL time step (Sec. 4): eq. dt1 in 1D, eq. dt2 in 2D, and in 3D the same
 * harmonic combination sigma / sum_d (max(|u_d| + c) / dx_d).
 */
double or_euler_dt(int ndim, const int64_t* n, const double* dx, double gamma,
                   double sigma, const double* U) {
  or_shape s = make_shape(ndim, n);
  double smax[3] = {0.0, 0.0, 0.0};
  for (int64_t lin = 0; lin < s.ncell; ++lin) {
    double Uc[OR_MAXVAR], rho, vel[3], p;
    load_cell(&s, U, lin, Uc);
    primitive(ndim, Uc, gamma, &rho, vel, &p);
    double c = sqrt(gamma * p / rho);
    for (int d = 0; d < ndim; ++d) {
      double sp = fabs(vel[d]) + c;
      if (sp > smax[d]) smax[d] = sp;
    }
  }
  if (ndim == 1) return sigma * dx[0] / smax[0];
  if (ndim == 2) {
    double dtx = dx[0] / smax[0], dty = dx[1] / smax[1];
    return sigma * dtx * dty / (dtx + dty);
  }
  double acc = 0.0;
  for (int d = 0; d < 3; ++d) acc += smax[d] / dx[d];
  return sigma / acc;
}

/*
 * One SSP-RK3 step of size dt, eq. 4.1-4.3, in place on U.
 * Returns 0 or -1 (non-physical state met in a stage).
 */
int or_euler_rk3_step(int ndim, const int64_t* n, const double* dx,
                      const int* bc, const or_params* P, double* U, double dt) {
  or_shape s = make_shape(ndim, n);
  int64_t tot = s.nvar * s.ncell;
  double* L = (double*)malloc(sizeof(double) * tot);
  double* U1 = (double*)malloc(sizeof(double) * tot);
  double* U2 = (double*)malloc(sizeof(double) * tot);
  int st = 0;
  /* eq. 4.1 */
  st |= or_euler_rhs(ndim, n, dx, bc, P, U, L, NULL, NULL, NULL);
  for (int64_t i = 0; i < tot; ++i) U1[i] = U[i] + dt * L[i];
  /* eq. 4.2 */
  st |= or_euler_rhs(ndim, n, dx, bc, P, U1, L, NULL, NULL, NULL);
  for (int64_t i = 0; i < tot; ++i)
    U2[i] = 3.0 / 4.0 * U[i] + 1.0 / 4.0 * U1[i] + 1.0 / 4.0 * dt * L[i];
  /* eq. 4.3 */
  st |= or_euler_rhs(ndim, n, dx, bc, P, U2, L, NULL, NULL, NULL);
  for (int64_t i = 0; i < tot; ++i)
    U[i] = 1.0 / 3.0 * U[i] + 2.0 / 3.0 * U2[i] + 2.0 / 3.0 * dt * L[i];
  free(L);
  free(U1);
  free(U2);
  return st ? -1 : 0;
}

/*
 * Advance with CFL steps until t_end or max_steps: each step takes
 * dt = min(dt_CFL(U^n), t_end - t) (dt_fixed > 0 replaces dt_CFL).
 * *t is updated; returns the number of steps taken.  With strict != 0 the run
 * stops and returns -1 at the first step in which a stage meets a
 * non-physical state; otherwise it continues and counts such steps in
 * *n_bad (nullable).
 */
int64_t or_euler_run(int ndim, const int64_t* n, const double* dx,
                     const int* bc, const or_params* P, double* U, double* t,
                     double t_end, double sigma, double dt_fixed,
                     int64_t max_steps, int strict, int64_t* n_bad) {
  int64_t k = 0;
  if (n_bad) *n_bad = 0;
  while (k < max_steps && *t < t_end) {
    double dt = dt_fixed > 0.0 ? dt_fixed
                               : or_euler_dt(ndim, n, dx, P->gamma, sigma, U);
    if (t_end - *t < dt) dt = t_end - *t;
    if (or_euler_rk3_step(ndim, n, dx, bc, P, U, dt) != 0) {
      if (strict) return -1;
      if (n_bad) ++*n_bad;
    }
    *t = *t + dt;
    ++k;
  }
  return k;
}

/* ------------------------------------------------------------------------ */
/* Scalar linear advection u_t + u_x = 0 (Sec. 4.1), periodic.               */
/* f = u, global LF with alpha = max|f'| = 1: f^+ = u, f^- = 0.              */
/* ------------------------------------------------------------------------ */

/* mode 0: TENO5-LAD; mode 1: Upwind5 (eq. 2.3). */
void or_scalar_rhs(int64_t n, double dx, const or_params* P, int mode,
                   const double* u, double* rhs) {
  double* F = (double*)malloc(sizeof(double) * (n + 1));
  for (int64_t id = 0; id <= n; ++id) {
    int64_t i = id - 1;
    double vp[5], vm[5];
    for (int k = 0; k < 5; ++k) {
      double fu = u[ghost_index(i - 2 + k, n, 0)];
      vp[k] = 0.5 * (fu + 1.0 * fu);
      double fm = u[ghost_index(i + 3 - k, n, 0)];
      vm[k] = 0.5 * (fm - 1.0 * fm);
    }
    if (mode == 1)
      F[id] = or_upwind5(vp) + or_upwind5(vm);
    else
      F[id] = or_teno5_lad(vp, P, -1, NULL, NULL) +
              or_teno5_lad(vm, P, -1, NULL, NULL);
  }
  for (int64_t i = 0; i < n; ++i) rhs[i] = -(F[i + 1] - F[i]) / dx;
  free(F);
}

/* SSP-RK3 (eq. 4.1-4.3) for the scalar problem from t = 0 to t_end with
 * steps of dt (the last one clipped). Returns the step count. */
int64_t or_scalar_run(int64_t n, double dx, const or_params* P, int mode,
                      double* u, double t_end, double dt) {
  double* L = (double*)malloc(sizeof(double) * n);
  double* u1 = (double*)malloc(sizeof(double) * n);
  double* u2 = (double*)malloc(sizeof(double) * n);
  double t = 0.0;
  int64_t k = 0;
  while (t < t_end) {
    double h = dt;
    if (t_end - t < h) h = t_end - t;
    or_scalar_rhs(n, dx, P, mode, u, L);
    for (int64_t i = 0; i < n; ++i) u1[i] = u[i] + h * L[i];
    or_scalar_rhs(n, dx, P, mode, u1, L);
    for (int64_t i = 0; i < n; ++i)
      u2[i] = 3.0 / 4.0 * u[i] + 1.0 / 4.0 * u1[i] + 1.0 / 4.0 * h * L[i];
    or_scalar_rhs(n, dx, P, mode, u2, L);
    for (int64_t i = 0; i < n; ++i)
      u[i] = 1.0 / 3.0 * u[i] + 2.0 / 3.0 * u2[i] + 2.0 / 3.0 * h * L[i];
    t = t + h;
    ++k;
  }
  free(L);
  free(u1);
  free(u2);
  return k;
}

/* ------------------------------------------------------------------------ */
/* Exact Riemann solver for the ideal-gas Euler equations (textbook          */
/* pressure-function method: Newton iteration on f_L(p) + f_R(p) + du = 0,   */
/* safeguarded by bisection; self-similar sampling).                         */
/* ------------------------------------------------------------------------ */

/* f_K(p) and its derivative: shock branch for p > p_K (Rankine-Hugoniot),
 * rarefaction branch otherwise (isentropic). */
static void pressure_function(double p, double rk, double pk, double ck,
                              double g, double* f, double* df) {
  if (p > pk) {
    double A = 2.0 / ((g + 1.0) * rk);
    double B = (g - 1.0) / (g + 1.0) * pk;
    double s = sqrt(A / (p + B));
    *f = (p - pk) * s;
    *df = s * (1.0 - 0.5 * (p - pk) / (p + B));
  } else {
    double e = (g - 1.0) / (2.0 * g);
    *f = 2.0 * ck / (g - 1.0) * (pow(p / pk, e) - 1.0);
    *df = 1.0 / (rk * ck) * pow(p / pk, -(g + 1.0) / (2.0 * g));
  }
}

/*
 * Star state of the Riemann problem (rl, ul, pl | rr, ur, pr).
 * out[0] = p*, out[1] = u*, out[2] = rho*_L, out[3] = rho*_R,
 * out[4] = left wave type (1 shock, 0 rarefaction), out[5] = right wave type,
 * out[6] = left shock speed or left head speed, out[7] = left tail speed
 * (equal to out[6] for a shock), out[8] = right tail speed, out[9] = right
 * shock or head speed, out[10] = iterations.
 * Returns 0, or -1 if the data generate vacuum or the iteration fails.
 */
int or_riemann_star(double rl, double ul, double pl, double rr, double ur,
                    double pr, double g, double* out) {
  double cl = sqrt(g * pl / rl), cr = sqrt(g * pr / rr);
  double du = ur - ul;
  if (2.0 * (cl + cr) / (g - 1.0) <= du) return -1; /* vacuum */
  /* two-rarefaction initial guess */
  double e = (g - 1.0) / (2.0 * g);
  double p = pow((cl + cr - 0.5 * (g - 1.0) * du) /
                     (cl / pow(pl, e) + cr / pow(pr, e)),
                 1.0 / e);
  if (!(p > 0.0)) p = 1e-8 * (pl < pr ? pl : pr);
  /* bracket for bisection: f is increasing in p */
  double lo = 0.0, hi = (pl > pr ? pl : pr);
  {
    double fl, dfl, fr, dfr;
    for (int k = 0; k < 200; ++k) {
      pressure_function(hi, rl, pl, cl, g, &fl, &dfl);
      pressure_function(hi, rr, pr, cr, g, &fr, &dfr);
      if (fl + fr + du > 0.0) break;
      hi *= 2.0;
    }
  }
  int it = 0;
  for (it = 0; it < 200; ++it) {
    double fl, dfl, fr, dfr;
    pressure_function(p, rl, pl, cl, g, &fl, &dfl);
    pressure_function(p, rr, pr, cr, g, &fr, &dfr);
    double F = fl + fr + du;
    if (F > 0.0) hi = p; else lo = p;
    double pn = p - F / (dfl + dfr);
    if (!(pn > lo && pn < hi)) pn = 0.5 * (lo + hi);
    double change = fabs(pn - p) / (0.5 * (pn + p));
    p = pn;
    if (change < 1e-15 || hi - lo <= 4e-16 * hi) break;
  }
  if (!(p > 0.0) || !isfinite(p)) return -1;
  double fl, dfl, fr, dfr;
  pressure_function(p, rl, pl, cl, g, &fl, &dfl);
  pressure_function(p, rr, pr, cr, g, &fr, &dfr);
  double u = 0.5 * (ul + ur) + 0.5 * (fr - fl);
  double gm = (g - 1.0) / (g + 1.0);
  out[0] = p;
  out[1] = u;
  if (p > pl) { /* left shock */
    out[2] = rl * (p / pl + gm) / (gm * p / pl + 1.0);
    out[4] = 1.0;
    out[6] = ul - cl * sqrt((g + 1.0) / (2.0 * g) * p / pl + (g - 1.0) / (2.0 * g));
    out[7] = out[6];
  } else { /* left rarefaction */
    out[2] = rl * pow(p / pl, 1.0 / g);
    out[4] = 0.0;
    out[6] = ul - cl;
    out[7] = u - cl * pow(p / pl, (g - 1.0) / (2.0 * g));
  }
  if (p > pr) { /* right shock */
    out[3] = rr * (p / pr + gm) / (gm * p / pr + 1.0);
    out[5] = 1.0;
    out[9] = ur + cr * sqrt((g + 1.0) / (2.0 * g) * p / pr + (g - 1.0) / (2.0 * g));
    out[8] = out[9];
  } else { /* right rarefaction */
    out[3] = rr * pow(p / pr, 1.0 / g);
    out[5] = 0.0;
    out[9] = ur + cr;
    out[8] = u + cr * pow(p / pr, (g - 1.0) / (2.0 * g));
  }
  out[10] = (double)it;
  return 0;
}

/* Sample the self-similar exact solution at xi = (x - x0)/t for each of the
 * m points: prim[0][k] = rho, prim[1][k] = u, prim[2][k] = p. */
int or_riemann_sample(double rl, double ul, double pl, double rr, double ur,
                      double pr, double g, const double* xi, int64_t m,
                      double* prim) {
  double st[11];
  if (or_riemann_star(rl, ul, pl, rr, ur, pr, g, st) != 0) return -1;
  double ps = st[0], us = st[1];
  double cl = sqrt(g * pl / rl), cr = sqrt(g * pr / rr);
  for (int64_t k = 0; k < m; ++k) {
    double s = xi[k], r, u, p;
    if (s <= us) { /* left of the contact */
      if (st[4] > 0.5) { /* shock */
        if (s <= st[6]) { r = rl; u = ul; p = pl; }
        else { r = st[2]; u = us; p = ps; }
      } else {
        if (s <= st[6]) { r = rl; u = ul; p = pl; }
        else if (s >= st[7]) { r = st[2]; u = us; p = ps; }
        else { /* inside the left fan */
          u = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * ul + s);
          double c = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * (ul - s));
          r = rl * pow(c / cl, 2.0 / (g - 1.0));
          p = pl * pow(c / cl, 2.0 * g / (g - 1.0));
        }
      }
    } else { /* right of the contact */
      if (st[5] > 0.5) {
        if (s >= st[9]) { r = rr; u = ur; p = pr; }
        else { r = st[3]; u = us; p = ps; }
      } else {
        if (s >= st[9]) { r = rr; u = ur; p = pr; }
        else if (s <= st[8]) { r = st[3]; u = us; p = ps; }
        else { /* inside the right fan */
          u = 2.0 / (g + 1.0) * (-cr + 0.5 * (g - 1.0) * ur + s);
          double c = 2.0 / (g + 1.0) * (cr - 0.5 * (g - 1.0) * (ur - s));
          r = rr * pow(c / cr, 2.0 / (g - 1.0));
          p = pr * pow(c / cr, 2.0 * g / (g - 1.0));
        }
      }
    }
    prim[k] = r;
    prim[m + k] = u;
    prim[2 * m + k] = p;
  }
  return 0;
}

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void or_set_num_threads(int k) {
#ifdef _OPENMP
  if (k > 0) omp_set_num_threads(k);
#else
  (void)k;
#endif
}
