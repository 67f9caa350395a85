// cert_host.cpp -- test helper: the certified FP32 keep-all tests of
// teno_cert.cuh (the device code, compiled here for the host with
// -ffp-contract=off, so it rounds exactly as on the GPU) behind a C
// interface for the CPU tests.
#include <cstdint>
#include <cstring>

#include "teno_cert.cuh"

namespace {

template <int NDIM, int DIR>
int interface_case(const double* up, const double* un, const double* pn, const double* u, double hb1, double hb2,
                   double hic, const double* al, float thr_f, float eps4_f) {
  constexpr int NVAR = NDIM + 2;
  double uu[NDIM], alpha[NVAR];
  std::memcpy(uu, u, sizeof(uu));
  std::memcpy(alpha, al, sizeof(alpha));
  teno_cert::CertIfc<NDIM> C;
  teno_cert::cert_begin<NDIM, DIR>(uu, hb1, hb2, hic, alpha, C);
  for (int j = 0; j < 6; ++j) {
    double Uj[NVAR];
    std::memcpy(Uj, up + j * NVAR, sizeof(Uj));
    teno_cert::cert_point<NDIM, DIR>(j, Uj, un[j], pn[j], C);
  }
  return teno_cert::cert_keep<NDIM>(C, thr_f, eps4_f) ? 1 : 0;
}

}  // namespace

// v: n x 5 doubles; out: n ints (1 = certified keep-all)
extern "C" void cert_values_batch(int64_t n, const double* v, float thr_f, float eps4_f, int* out) {
  for (int64_t i = 0; i < n; ++i) {
    const double* w = v + 5 * i;
    out[i] = teno_cert::certify_keep_values(w[0], w[1], w[2], w[3], w[4], thr_f, eps4_f) ? 1 : 0;
  }
}

// One FP32 value test with a given d (the five FP32 inputs as floats).
extern "C" int cert_floats(const float* v, float d, float thr_f, float eps4_f) {
  return teno_cert::certify_keep(v[0], v[1], v[2], v[3], v[4], d, thr_f, eps4_f) ? 1 : 0;
}

extern "C" float cert_hi_float(double x) { return teno_cert::hi_float(x); }

// Interface cases of an ndim-dimensional grid, direction dir: per case the six
// stencil states U[6][nvar], u_d/2 [6], p/2 [6], the Roe state u~[ndim],
// b1/2, b2/2, 1/(2c) and the halved speeds [nvar].
extern "C" void cert_interface_batch(int ndim, int dir, int64_t n, const double* U, const double* un,
                                     const double* pn, const double* u, const double* hb1, const double* hb2,
                                     const double* hic, const double* alpha, float thr_f, float eps4_f, int* out) {
  const int nvar = ndim + 2;
  for (int64_t i = 0; i < n; ++i) {
    const double* up = U + i * 6 * nvar;
    const double* ui = u + i * ndim;
    const double* al = alpha + i * nvar;
    int r = -1;
    if (ndim == 1) r = interface_case<1, 0>(up, un + 6 * i, pn + 6 * i, ui, hb1[i], hb2[i], hic[i], al, thr_f, eps4_f);
    else if (ndim == 2 && dir == 0)
      r = interface_case<2, 0>(up, un + 6 * i, pn + 6 * i, ui, hb1[i], hb2[i], hic[i], al, thr_f, eps4_f);
    else if (ndim == 2 && dir == 1)
      r = interface_case<2, 1>(up, un + 6 * i, pn + 6 * i, ui, hb1[i], hb2[i], hic[i], al, thr_f, eps4_f);
    else if (ndim == 3 && dir == 0)
      r = interface_case<3, 0>(up, un + 6 * i, pn + 6 * i, ui, hb1[i], hb2[i], hic[i], al, thr_f, eps4_f);
    else if (ndim == 3 && dir == 1)
      r = interface_case<3, 1>(up, un + 6 * i, pn + 6 * i, ui, hb1[i], hb2[i], hic[i], al, thr_f, eps4_f);
    else if (ndim == 3 && dir == 2)
      r = interface_case<3, 2>(up, un + 6 * i, pn + 6 * i, ui, hb1[i], hb2[i], hic[i], al, thr_f, eps4_f);
    out[i] = r;
  }
}
