// teno_kernels.cu -- sm_103a kernels of the TENO5-LAD Euler right-hand side
// and the SSP-RK3 stage updates (all FP64).
//
// One right-hand-side evaluation L(U) (eq. 2.2) is
//   cell_kernel    : per cell, primitive variables (u_k, p) and the Roe weights
//                    sqrt(rho), (E + p)/sqrt(rho); the global Lax-Friedrichs
//                    speeds alpha_{d,s} = max |lambda_s| of every direction
//                    (warp-shuffle max, block max, one atomic per block);
//   flux_kernel<D> : per interface of direction D, one thread: the six-point
//                    flux stencil, Roe eigensystem, characteristic projection,
//                    LF splitting, 2 x nvar TENO5-LAD reconstructions and the
//                    back-projection to the interface flux F^;
//   diff_kernel<D> : per cell, -(F^_{i+1/2} - F^_{i-1/2}) / dx_D, written,
//                    accumulated, or fused into the SSP-RK3 stage (eq. 4.1-4.3).
#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>

#include "teno_device.cuh"
#include "teno_launch.h"

namespace teno {

// ---------------------------------------------------------------------------
// Cell pass: primitive variables, Roe weights and LF speeds.
// The primitive variables are evaluated with explicit round-to-nearest
// operations (no contraction) in the order u = m/rho, |u|^2 = sum u_k u_k,
// p = (gamma-1)(E - (rho/2)|u|^2), c = sqrt(gamma p / rho), so the wave
// speeds, and through them alpha and the CFL step, are the correctly rounded
// values of these formulas.
// aux layout: [ndim + 3][ncell]: u_0..u_{ndim-1}, p, sqrt(rho), (E+p)/sqrt(rho).
// alpha layout (bit patterns of non-negative doubles): [ndim][3] =
// max|u_d - c|, max|u_d|, max|u_d + c|.
// ---------------------------------------------------------------------------
template <int NDIM>
__global__ void __launch_bounds__(256) cell_kernel(const double* __restrict__ U,
                                                   double* __restrict__ aux,
                                                   unsigned long long* __restrict__ alpha,
                                                   int* __restrict__ status,
                                                   int64_t ncell, double gamma) {
  constexpr int NVAR = NDIM + 2;
  double lam[NDIM][3];
#pragma unroll
  for (int d = 0; d < NDIM; ++d) lam[d][0] = lam[d][1] = lam[d][2] = 0.0;
  bool bad = false;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell;
       c += (int64_t)gridDim.x * blockDim.x) {
    double rho = U[c];
    double E = U[(NVAR - 1) * ncell + c];
    double u[NDIM];
    double q2 = 0.0;
#pragma unroll
    for (int k = 0; k < NDIM; ++k) {
      u[k] = __ddiv_rn(U[(1 + k) * ncell + c], rho);
      q2 = __dadd_rn(q2, __dmul_rn(u[k], u[k]));
    }
    double p = __dmul_rn(gamma - 1.0, __dsub_rn(E, __dmul_rn(__dmul_rn(0.5, rho), q2)));
    double cs = __dsqrt_rn(__ddiv_rn(__dmul_rn(gamma, p), rho));
    double sr = __dsqrt_rn(rho);
    if (!(rho > 0.0) || !(p > 0.0) || !isfinite(E) || !isfinite(q2)) bad = true;
#pragma unroll
    for (int k = 0; k < NDIM; ++k) aux[k * ncell + c] = u[k];
    aux[NDIM * ncell + c] = p;
    aux[(NDIM + 1) * ncell + c] = sr;
    aux[(NDIM + 2) * ncell + c] = (E + p) / sr;
#pragma unroll
    for (int d = 0; d < NDIM; ++d) {
      lam[d][0] = fmax(lam[d][0], fabs(__dsub_rn(u[d], cs)));
      lam[d][1] = fmax(lam[d][1], fabs(u[d]));
      lam[d][2] = fmax(lam[d][2], fabs(__dadd_rn(u[d], cs)));
    }
  }
  // warp max on bit patterns (all values are >= 0)
  __shared__ unsigned long long red[8][NDIM * 3];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int d = 0; d < NDIM; ++d)
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      unsigned long long v = dbits(lam[d][s]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = v > w ? v : w;
      }
      if (lane == 0) red[warp][d * 3 + s] = v;
    }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(status, kStatusNonphysical);
  __syncthreads();
  if (threadIdx.x < NDIM * 3) {
    unsigned long long v = 0;
    const int nw = blockDim.x >> 5;
    for (int w = 0; w < nw; ++w) v = v > red[w][threadIdx.x] ? v : red[w][threadIdx.x];
    atomicMax(&alpha[threadIdx.x], v);
  }
}

// ---------------------------------------------------------------------------
// Interface fluxes of direction DIR.
// ---------------------------------------------------------------------------

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

template <int NDIM, int DIR>
__global__ void __launch_bounds__(128) flux_kernel(
    const double* __restrict__ U, const double* __restrict__ aux,
    const unsigned long long* __restrict__ alpha_bits, double* __restrict__ Fhat,
    uint8_t* __restrict__ flags, int* __restrict__ status, Grid G, Scheme S) {
  constexpr int NVAR = NDIM + 2;
  // interface grid: n along the other axes, n_DIR + 1 along DIR
  const int64_t m0 = G.n[0] + (DIR == 0), m1 = G.n[1] + (DIR == 1), m2 = G.n[2] + (DIR == 2);
  const int64_t nifc = m0 * m1 * m2;
  const int64_t ncell = G.ncell;
  const int64_t stride_d = (DIR == 0) ? 1 : (DIR == 1 ? G.n[0] : G.n[0] * G.n[1]);
  const int64_t nd = G.n[DIR];
  const int bcd = G.bc[DIR];

  double alpha[NVAR];
  {
    double am = __longlong_as_double((long long)alpha_bits[DIR * 3 + 0]);
    double a0 = __longlong_as_double((long long)alpha_bits[DIR * 3 + 1]);
    double ap = __longlong_as_double((long long)alpha_bits[DIR * 3 + 2]);
    alpha[0] = 0.5 * am;
#pragma unroll
    for (int f = 1; f < NVAR - 1; ++f) alpha[f] = 0.5 * a0;
    alpha[NVAR - 1] = 0.5 * ap;
  }

  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nifc;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i0 = q % m0;
    const int64_t r = q / m0;
    const int64_t i1 = r % m1;
    const int64_t i2 = r / m1;
    const int64_t id = (DIR == 0) ? i0 : (DIR == 1 ? i1 : i2);
    // linear index of the cell with coordinate 0 along DIR on this line
    const int64_t base = (DIR == 0) ? (i2 * G.n[1] + i1) * G.n[0]
                       : (DIR == 1) ? i2 * G.n[1] * G.n[0] + i0
                                    : i1 * G.n[0] + i0;

    // six-point stencil i-2..i+3 with i = id - 1
    double Ux[6][NVAR], un[6], pn[6];
    double sr2, sr3, sh2, sh3, uu2[NDIM], uu3[NDIM];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const int64_t c = base + ghost(id - 3 + j, nd, bcd) * stride_d;
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
    // Roe average of cells i and i+1
    const double inv = 1.0 / (sr2 + sr3);
    double u[NDIM];
    double q2 = 0.0;
#pragma unroll
    for (int k = 0; k < NDIM; ++k) {
      u[k] = fma(sr2, uu2[k], sr3 * uu3[k]) * inv;
      q2 = fma(u[k], u[k], q2);
    }
    const double H = (sh2 + sh3) * inv;
    const double c2 = S.gm1 * fma(-0.5, q2, H);
    if (!(c2 > 0.0)) atomicOr(status, kStatusNonphysical);
    const double ic = rsqrt(c2);
    const double cs = c2 * ic;
    const double b1 = S.gm1 * ic * ic;
    const double b2 = 0.5 * b1 * q2;
    const double hb1 = 0.5 * b1, hb2 = 0.5 * b2, hic = 0.5 * ic;

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
      const double hu = 0.5 * un[j];
      const double hp = 0.5 * pn[j];
      const double zeta = hb1 * (un[j] - u[DIR]);
      const double t0 = hp * (zeta - hic);
      const double tE = hp * (zeta + hic);
      const double t1 = -2.0 * (hp * zeta);
      vp[j][0] = fma(hu + alpha[0], w[0], t0);
      vm[j][0] = fma(hu - alpha[0], w[0], t0);
      vp[j][NVAR - 1] = fma(hu + alpha[NVAR - 1], w[NVAR - 1], tE);
      vm[j][NVAR - 1] = fma(hu - alpha[NVAR - 1], w[NVAR - 1], tE);
      const double sp = hu + alpha[1], sm = hu - alpha[1];
      vp[j][1] = fma(sp, w[1], t1);
      vm[j][1] = fma(sm, w[1], t1);
#pragma unroll
      for (int f = 2; f < NVAR - 1; ++f) {
        vp[j][f] = sp * w[f];
        vm[j][f] = sm * w[f];
      }
    }
    unsigned fl[NVAR][2];
#pragma unroll
    for (int s = 0; s < NVAR; ++s) {
      const double hp = teno5_lad(vp[0][s], vp[1][s], vp[2][s], vp[3][s], vp[4][s], S, fl[s][0]);
      const double hm = teno5_lad(vm[5][s], vm[4][s], vm[3][s], vm[2][s], vm[1][s], S, fl[s][1]);
      fchar[s] = hp + hm;
    }
    if (flags) {
      // direction block offset is applied by the caller through `flags`
#pragma unroll
      for (int s = 0; s < NVAR; ++s)
#pragma unroll
        for (int side = 0; side < 2; ++side)
          flags[(int64_t)(s * 2 + side) * nifc + q] = (uint8_t)fl[s][side];
    }
    // back-projection F^ = R f^char, columns r_0 = (1, u - c e_n, H - u_n c),
    // r_1 = (1, u, q2/2), r_t = (0, e_t, u_t), r_{nvar-1} = (1, u + c e_n, H + u_n c)
    const double sa = fchar[0] + fchar[NVAR - 1];
    const double da = fchar[NVAR - 1] - fchar[0];
    const double rho_f = sa + fchar[1];
    double out[NVAR];
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
#pragma unroll
    for (int v = 0; v < NVAR; ++v) Fhat[(int64_t)v * nifc + q] = out[v];
  }
}

// ---------------------------------------------------------------------------
// Conservative difference (eq. 2.2) and SSP-RK3 stage update (eq. 4.1-4.3).
// mode: 0 R = d; 1 R += d; 2 U1 = Un + dt (R + d); 3 U2 = 3/4 Un + 1/4 U1 +
// 1/4 dt (R + d); 4 Un <- 1/3 Un + 2/3 U2 + 2/3 dt (R + d).  `acc` selects
// whether R already holds the contributions of earlier directions.
// ---------------------------------------------------------------------------
template <int NDIM, int DIR>
__global__ void __launch_bounds__(256) diff_kernel(
    const double* __restrict__ Fhat, double* __restrict__ R,
    const double* __restrict__ Un, const double* __restrict__ Uk,
    double* __restrict__ Uout, const double* __restrict__ dt_ptr, Grid G,
    int mode, int acc) {
  constexpr int NVAR = NDIM + 2;
  const int64_t ncell = G.ncell;
  const int64_t m0 = G.n[0] + (DIR == 0), m1 = G.n[1] + (DIR == 1);
  const int64_t nifc = m0 * m1 * (G.n[2] + (DIR == 2));
  const double idx = G.inv_dx[DIR];
  double dt = 0.0;
  if (mode >= 2) {
    dt = *dt_ptr;
    if (!(dt > 0.0)) return;  // t >= t_end: the state is left unchanged
  }
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i0 = c % G.n[0];
    const int64_t r = c / G.n[0];
    const int64_t i1 = r % G.n[1];
    const int64_t i2 = r / G.n[1];
    const int64_t left = (i2 * m1 + i1) * m0 + i0;
    const int64_t right = left + (DIR == 0 ? 1 : (DIR == 1 ? m0 : m0 * m1));
#pragma unroll
    for (int v = 0; v < NVAR; ++v) {
      double d = (Fhat[v * nifc + left] - Fhat[v * nifc + right]) * idx;
      const int64_t e = v * ncell + c;
      if (acc) d += R[e];
      switch (mode) {
        case 0:
        case 1:
          R[e] = d;
          break;
        case 2:
          Uout[e] = fma(dt, d, Un[e]);
          break;
        case 3:
          Uout[e] = fma(0.25 * dt, d, fma(0.75, Un[e], 0.25 * Uk[e]));
          break;
        default:
          Uout[e] = fma((2.0 / 3.0) * dt, d, fma(1.0 / 3.0, Un[e], (2.0 / 3.0) * Uk[e]));
          break;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Time step (eq. dt1 / dt2; harmonic 3D form) from the LF speeds of U^n:
// max_i(|u_d| + c) = max(max|u_d - c|, max|u_d + c|).  Clipped to t_end - t.
// ---------------------------------------------------------------------------
template <int NDIM>
__global__ void dt_kernel(const unsigned long long* __restrict__ alpha_bits,
                          Grid G, double cfl, double dt_fixed, double* t_dev,
                          double t_end, double* dt_ws, double* dt_out) {
  const double* dx = G.dx;
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double smax[3];
#pragma unroll
  for (int d = 0; d < NDIM; ++d) {
    unsigned long long a = alpha_bits[d * 3 + 0], b = alpha_bits[d * 3 + 2];
    smax[d] = __longlong_as_double((long long)(a > b ? a : b));
  }
  double dt;
  if (dt_fixed > 0.0) {
    dt = dt_fixed;
  } else if (NDIM == 1) {
    dt = cfl * dx[0] / smax[0];
  } else if (NDIM == 2) {
    const double dtx = dx[0] / smax[0], dty = dx[1] / smax[1];
    dt = cfl * dtx * dty / (dtx + dty);
  } else {
    double acc = 0.0;
#pragma unroll
    for (int d = 0; d < NDIM; ++d) acc += smax[d] / dx[d];
    dt = cfl / acc;
  }
  const double t = *t_dev;
  const double rem = t_end - t;
  if (rem < dt) dt = rem;
  if (!(dt > 0.0)) dt = 0.0;
  *dt_ws = dt;
  if (dt_out) *dt_out = dt;
  *t_dev = t + dt;
}

// ---------------------------------------------------------------------------
// Scheme constants (host side)
// ---------------------------------------------------------------------------
Scheme make_scheme(double gamma, double H, double eps, int b_l, int b_u) {
  static const double kPow10Neg[16] = {1e-0, 1e-1, 1e-2,  1e-3,  1e-4,  1e-5,  1e-6,  1e-7,
                                       1e-8, 1e-9, 1e-10, 1e-11, 1e-12, 1e-13, 1e-14, 1e-15};
  Scheme S;
  std::memset(&S, 0, sizeof(S));
  S.gamma = gamma;
  S.gm1 = gamma - 1.0;
  S.eps = eps;
  S.b_l = b_l;
  S.b_u = b_u;
  const int K = b_u - b_l;
  S.nthr = K;
  S.top = 1;
  while (S.top * 2 <= K) S.top *= 2;
  // floor(theta K) >= j  <=>  max chi~ <= H (K/j - 1)   (eq. 3.1-3.2)
  for (int j = 1; j < K; ++j) S.thr[j - 1] = H * (double(K) / double(j) - 1.0);
  // theta == 1 in binary64  <=>  max chi~ / H <= 2^-53
  S.thr[K - 1] = H * 0x1p-53;
  // All stencils are kept whenever 3 (1 + max chi~)^6 C_T < 1 (then
  // chi_k >= gamma_min / (3 gamma_max) >= 1 / (3 (1 + max chi~)^6) > C_T); at
  // a given m, max chi~ <= thr[m - B_l - 1].  A relative margin of 1e-9 covers
  // the rounding of the threshold products.
  S.keep_all = 0;
  for (int c = 1; c <= K; ++c) {
    const int m = b_l + c;
    const double x = 1.0 + S.thr[c - 1];
    const double x6 = x * x * x * x * x * x;
    if (3.0 * x6 * kPow10Neg[m] <= 1.0 - 1e-9) S.keep_all |= 1u << m;
  }
  return S;
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
static inline int blocks_for(int64_t n, int threads, int cap) {
  int64_t b = (n + threads - 1) / threads;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return static_cast<int>(b);
}

cudaError_t launch_cell(int ndim, const double* U, double* aux,
                        unsigned long long* alpha, int* status, int64_t ncell,
                        double gamma, int nsm, cudaStream_t st) {
  const int threads = 256;
  const int blocks = blocks_for(ncell, threads, nsm * 8);
  switch (ndim) {
    case 1: cell_kernel<1><<<blocks, threads, 0, st>>>(U, aux, alpha, status, ncell, gamma); break;
    case 2: cell_kernel<2><<<blocks, threads, 0, st>>>(U, aux, alpha, status, ncell, gamma); break;
    default: cell_kernel<3><<<blocks, threads, 0, st>>>(U, aux, alpha, status, ncell, gamma); break;
  }
  return cudaGetLastError();
}

template <int NDIM, int DIR>
static void flux_launch(int blocks, int threads, cudaStream_t st, const double* U,
                        const double* aux, const unsigned long long* alpha,
                        double* Fhat, uint8_t* flags, int* status, const Grid& G,
                        const Scheme& S) {
  flux_kernel<NDIM, DIR><<<blocks, threads, 0, st>>>(U, aux, alpha, Fhat, flags, status, G, S);
}

cudaError_t launch_flux(int ndim, int dir, const double* U, const double* aux,
                        const unsigned long long* alpha, double* Fhat,
                        uint8_t* flags, int* status, const Grid& G,
                        const Scheme& S, int nsm, cudaStream_t st) {
  int64_t nifc = 1;
  for (int k = 0; k < 3; ++k) nifc *= G.n[k] + (k == dir ? 1 : 0);
  const int threads = 128;
  const int blocks = blocks_for(nifc, threads, nsm * 64);
  if (ndim == 1) flux_launch<1, 0>(blocks, threads, st, U, aux, alpha, Fhat, flags, status, G, S);
  else if (ndim == 2) {
    if (dir == 0) flux_launch<2, 0>(blocks, threads, st, U, aux, alpha, Fhat, flags, status, G, S);
    else flux_launch<2, 1>(blocks, threads, st, U, aux, alpha, Fhat, flags, status, G, S);
  } else {
    if (dir == 0) flux_launch<3, 0>(blocks, threads, st, U, aux, alpha, Fhat, flags, status, G, S);
    else if (dir == 1) flux_launch<3, 1>(blocks, threads, st, U, aux, alpha, Fhat, flags, status, G, S);
    else flux_launch<3, 2>(blocks, threads, st, U, aux, alpha, Fhat, flags, status, G, S);
  }
  return cudaGetLastError();
}

template <int NDIM, int DIR>
static void diff_launch(int blocks, int threads, cudaStream_t st, const double* Fhat,
                        double* R, const double* Un, const double* Uk, double* Uout,
                        const double* dt, const Grid& G, int mode, int acc) {
  diff_kernel<NDIM, DIR><<<blocks, threads, 0, st>>>(Fhat, R, Un, Uk, Uout, dt, G, mode, acc);
}

cudaError_t launch_diff(int ndim, int dir, const double* Fhat, double* R,
                        const double* Un, const double* Uk, double* Uout,
                        const double* dt, const Grid& G, int mode, int acc,
                        int nsm, cudaStream_t st) {
  const int threads = 256;
  const int blocks = blocks_for(G.ncell, threads, nsm * 16);
  if (ndim == 1) diff_launch<1, 0>(blocks, threads, st, Fhat, R, Un, Uk, Uout, dt, G, mode, acc);
  else if (ndim == 2) {
    if (dir == 0) diff_launch<2, 0>(blocks, threads, st, Fhat, R, Un, Uk, Uout, dt, G, mode, acc);
    else diff_launch<2, 1>(blocks, threads, st, Fhat, R, Un, Uk, Uout, dt, G, mode, acc);
  } else {
    if (dir == 0) diff_launch<3, 0>(blocks, threads, st, Fhat, R, Un, Uk, Uout, dt, G, mode, acc);
    else if (dir == 1) diff_launch<3, 1>(blocks, threads, st, Fhat, R, Un, Uk, Uout, dt, G, mode, acc);
    else diff_launch<3, 2>(blocks, threads, st, Fhat, R, Un, Uk, Uout, dt, G, mode, acc);
  }
  return cudaGetLastError();
}

cudaError_t launch_dt(int ndim, const unsigned long long* alpha, const Grid& G,
                      double cfl, double dt_fixed, double* t_dev, double t_end,
                      double* dt_ws, double* dt_out, cudaStream_t st) {
  switch (ndim) {
    case 1: dt_kernel<1><<<1, 32, 0, st>>>(alpha, G, cfl, dt_fixed, t_dev, t_end, dt_ws, dt_out); break;
    case 2: dt_kernel<2><<<1, 32, 0, st>>>(alpha, G, cfl, dt_fixed, t_dev, t_end, dt_ws, dt_out); break;
    default: dt_kernel<3><<<1, 32, 0, st>>>(alpha, G, cfl, dt_fixed, t_dev, t_end, dt_ws, dt_out); break;
  }
  return cudaGetLastError();
}

}  // namespace teno
