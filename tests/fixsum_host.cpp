// Host build of teno_fixsum.cuh for test_fixsum_host.py: the fixed-point
// six-point sum exactly as the device evaluates it.
#include <cstdint>

#include "teno_fixsum.cuh"

extern "C" {

// n sums of x[i][0..5] with weights w[0..5]; ok[i] = 0 where the fixed
// point does not cover the sum (out[i] is then left 0)
void fix_sum6_batch(int64_t n, const double* x, const int* w, double* out, int* ok, uint32_t* Eout) {
  for (int64_t i = 0; i < n; ++i) {
    const double* xi = x + 6 * i;
    uint32_t kmax = 0;
    for (int j = 0; j < 6; ++j) {
      const uint32_t k = teno_fix::key(teno_fix::hi_word(xi[j]));
      kmax = k > kmax ? k : kmax;
    }
    const uint32_t E = teno_fix::exponent(kmax);
    Eout[i] = E;
    ok[i] = teno_fix::in_range(E) ? 1 : 0;
    out[i] = 0.0;
    if (!ok[i]) continue;
    int64_t A = 0;
    for (int j = 0; j < 6; ++j) teno_fix::add(A, xi[j], E, w[j]);
    out[i] = teno_fix::round(A, E);
  }
}

// the same through teno_fix::sum (n values of 7, weights of any sign with
// sum |w| < 128); ok[i] = 0 where it declines
void fix_sum7_batch(int64_t n, const double* x, const int* w, double* out, int* ok) {
  int wa[7];
  for (int j = 0; j < 7; ++j) wa[j] = w[j];
  for (int64_t i = 0; i < n; ++i) {
    double xi[7];
    for (int j = 0; j < 7; ++j) xi[j] = x[7 * i + j];
    out[i] = 0.0;
    ok[i] = teno_fix::sum<7>(xi, wa, out[i]) ? 1 : 0;
  }
}

}  // extern "C"
