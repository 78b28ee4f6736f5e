// Host entry points over the library's fixed-point sum arithmetic (csrc/pcg_fixed.cuh), for the
// CPU tests: the same functions the CG kernels run on the device, compiled for the host.
#include "pcg_fixed.cuh"

extern "C" {
int fxh_window(double a, double b, double c) { return ccm::fx_window(a, b, c); }

int fxh_digits(double v, int lo, int* d) {
  int dd[ccm::kFxDigits];
  const bool ok = ccm::fx_digits(v, lo, dd);
  for (int k = 0; k < ccm::kFxDigits; ++k) d[k] = dd[k];
  return ok ? 1 : 0;
}

// The fixed-point sum of v[0..n) in the window of bottom 2^lo (digit sums in 64-bit integers,
// as the blocks and the grid form them), and the number of values that did not fit.
double fxh_sum(const double* v, long n, int lo, int* overflow) {
  long long S[ccm::kFxDigits] = {0};
  int bad = 0;
  for (long i = 0; i < n; ++i) {
    int d[ccm::kFxDigits];
    if (!ccm::fx_digits(v[i], lo, d)) ++bad;
    for (int k = 0; k < ccm::kFxDigits; ++k) S[k] += d[k];
  }
  *overflow = bad;
  return ccm::fx_value(S, lo);
}
}
