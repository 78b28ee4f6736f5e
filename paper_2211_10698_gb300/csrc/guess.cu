// Initial guess of the pressure Poisson solve (Eq. pm_poisson) from the solutions of the
// previous steps: the K-orthogonal projection of the new solution onto their span,
//     x0 = sum_i (x~_i, b) x~_i,   with (x~_i, K x~_j) = delta_ij,
// which is the best guess in the energy norm that those solutions allow (Fischer, "Projection
// techniques for iterative solution of Ax = b with successive right-hand sides", Comput.
// Methods Appl. Mech. Engrg. 163, 1998).  After each solve the new solution is
// K-orthonormalised against the basis (classical Gram-Schmidt, twice) and appended; a full
// basis restarts from the newest solution.  The PCG that follows is unchanged: it starts from
// x0 instead of the previous step's Phi and stops at the same relative residual.
//
// Sums are deterministic: a fixed number of blocks, each summing a fixed range in a fixed
// order, then the block partials in block order.
#include "ccm_host.h"

namespace ccm {

namespace {

constexpr int kGT = 256;     // threads per block
constexpr int kGB = 304;     // blocks of the sums (fixed, so the order of the sums is fixed)

// part[i * kGB + b] = sum over block b's range of X_i[k] y[k], i < nb
__global__ void __launch_bounds__(kGT) k_mdot(const double* __restrict__ X, size_t n, int nb,
                                             const double* __restrict__ y, double* part) {
  __shared__ double red[kGT];
  double acc[kGuessMax];
#pragma unroll
  for (int i = 0; i < kGuessMax; ++i) acc[i] = 0.0;
  const size_t chunk = (n + kGB - 1) / kGB;
  const size_t k0 = blockIdx.x * chunk, k1 = min(n, k0 + chunk);
  for (size_t k = k0 + threadIdx.x; k < k1; k += kGT) {
    const double yk = y[k];
#pragma unroll
    for (int i = 0; i < kGuessMax; ++i)
      if (i < nb) acc[i] += X[(size_t)i * n + k] * yk;
  }
#pragma unroll
  for (int i = 0; i < kGuessMax; ++i) {
    if (i >= nb) break;
    red[threadIdx.x] = acc[i];
    __syncthreads();
    for (int h = kGT / 2; h > 0; h >>= 1) {
      if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[(size_t)i * kGB + blockIdx.x] = red[0];
    __syncthreads();
  }
}

// coef[i] = sum_b part[i * kGB + b] in block order (one warp per coefficient)
__global__ void k_msum(const double* part, int nb, double* coef) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = w; i < nb; i += blockDim.x >> 5) {
    double s = 0.0;
    for (int b = lane; b < kGB; b += 32) s += part[(size_t)i * kGB + b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) coef[i] = s;
  }
}

// out[k] = (base ? base[k] : 0) + sign * sum_{i < nb} coef[i] X_i[k]
__global__ void k_combine(const double* __restrict__ X, size_t n, int nb, const double* __restrict__ coef, double sign,
                          const double* base, double* out) {
  __shared__ double c[kGuessMax];
  if ((int)threadIdx.x < nb) c[threadIdx.x] = coef[threadIdx.x];
  __syncthreads();
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < nb; ++i) s += c[i] * X[(size_t)i * n + k];
    out[k] = (base ? base[k] : 0.0) + sign * s;
  }
}

// x *= 1/sqrt(n2), kx likewise, where n2 = (x, K x) from coef[0]; a vector with no energy left
// (the new solution lies in the span already) becomes zero and so adds nothing
__global__ void k_normalize(double* x, double* kx, size_t n, const double* coef, double tiny) {
  const double n2 = coef[0];
  const double s = n2 > tiny ? 1.0 / sqrt(n2) : 0.0;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
    x[k] *= s;
    kx[k] *= s;
  }
}

void mdot(const double* X, size_t n, int nb, const double* y, double* part, double* coef, cudaStream_t st) {
  k_mdot<<<kGB, kGT, 0, st>>>(X, n, nb, y, part);
  k_msum<<<1, 1024, 0, st>>>(part, nb, coef);
}

}  // namespace

size_t guess_scratch_doubles() { return (size_t)kGuessMax * kGB + 2 * kGuessMax; }

void launch_guess_project(const double* X, size_t n, int nb, const double* rhs, double* phi, double* scratch,
                          cudaStream_t st) {
  double* part = scratch;
  double* coef = scratch + (size_t)kGuessMax * kGB;
  mdot(X, n, nb, rhs, part, coef, st);
  k_combine<<<kGB, kGT, 0, st>>>(X, n, nb, coef, 1.0, nullptr, phi);
}

void launch_guess_append(double* X, double* KX, size_t n, int nb, double* scratch, cudaStream_t st) {
  double* part = scratch;
  double* coef = scratch + (size_t)kGuessMax * kGB;
  double* xn = X + (size_t)nb * n;
  double* kxn = KX + (size_t)nb * n;
  // x_n -= sum_i (x~_i, K x_n) x~_i and K x_n likewise, twice (classical Gram-Schmidt with
  // reorthogonalisation keeps the basis K-orthonormal to rounding)
  for (int pass = 0; pass < 2 && nb > 0; ++pass) {
    mdot(X, n, nb, kxn, part, coef, st);
    k_combine<<<kGB, kGT, 0, st>>>(X, n, nb, coef, -1.0, xn, xn);
    k_combine<<<kGB, kGT, 0, st>>>(KX, n, nb, coef, -1.0, kxn, kxn);
  }
  mdot(xn, n, 1, kxn, part, coef, st);
  k_normalize<<<kGB, kGT, 0, st>>>(xn, kxn, n, coef, 1e-300);
}

}  // namespace ccm
