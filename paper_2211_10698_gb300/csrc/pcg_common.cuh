// Building blocks shared by the persistent PCG kernels: the block's cell range, the per-thread
// walk over it, block and grid reductions in a fixed order, the Poisson row in diagonal form
// and the per-block scalar state.
#pragma once
#include "ccm_host.h"

namespace ccm {

constexpr int kPcgThreads = 512;

__device__ __forceinline__ void publish(double* partials, int nb, const double* v, int nv) {
  if (threadIdx.x == 0)
    for (int q = 0; q < nv; ++q) partials[(size_t)q * nb + blockIdx.x] = v[q];
}

// Sum NV per-thread values over the block through shared memory; only warp 0 adds (in a
// fixed order), so the FP64 cost is per block, not per thread.  Result valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum_smem(double (&v)[NV], double (*red)[kPcgThreads]) {
#pragma unroll
  for (int q = 0; q < NV; ++q) red[q][threadIdx.x] = v[q];
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double s = 0.0;
      for (int m = lane; m < (int)blockDim.x; m += 32) s += red[q][m];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      v[q] = s;
    }
  }
}

// Cells of this block: one contiguous chunk of the row-major interior, balanced to +-1 cell
// across blocks (the FP64 pipe of each SM is the bottleneck, so per-SM work must be even).
struct Chunk {
  int t0, t1;
  __device__ Chunk(int ncell) {
    t0 = (int)((long long)ncell * blockIdx.x / gridDim.x);
    t1 = (int)((long long)ncell * (blockIdx.x + 1) / gridDim.x);
  }
};

// Walks t = first, first + stride, ... < end, keeping (i, j) of the interior cell t.
struct CellWalk {
  int t, i, j;
  const int nx, stride, end;
  __device__ CellWalk(int first, int stride_, int end_, int nx_) : t(first), nx(nx_), stride(stride_), end(end_) {
    j = first / nx;
    i = first - j * nx;
  }
  __device__ bool ok() const { return t < end; }
  __device__ void next() {
    t += stride;
    i += stride;
    while (i >= nx) { i -= nx; ++j; }
  }
};

// Chebyshev iteration for K z = r from zero on the Jacobi-scaled operator, eigenvalue
// interval [lmax/30, lmax] with lmax = 2 (Gershgorin bound for a diagonally dominant
// M-matrix scaled by its diagonal), CHEB steps in all (Saad, Chebyshev acceleration).  On
// entry z = w1 = D^-1 r / theta (the first step, written by the caller); each further step
// needs z at the stencil neighbours, so steps are separated by grid barriers and z
// alternates between two buffers.  Returns the buffer that holds the result.
struct ChebCoef {
  static constexpr double lmax = 2.0, lmin = 2.0 / 30.0;
  static constexpr double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin);
};

// K x at one cell in diagonal form, d x_c - sum_f c_f x_nbr.  Cells whose four faces and
// volume are uncut (kind 1) use the constant coefficients of the uniform grid, so their
// coefficient arrays are not read; cut cells (kind 2) read them; other cells (kind 0:
// inactive, identity row) return x_c.
template <class T>
struct KRow {
  const T* cu;
  const T* cv;
  const T* dk;
  const int8_t* kind;
  T cx, cy, dreg;
  size_t P;
  __device__ __forceinline__ T operator()(const T* x, size_t k) const {
    const int8_t t = kind[k];
    const T xc = x[k];
    if (t == 1) return dreg * xc - cx * (x[k - 1] + x[k + 1]) - cy * (x[k - P] + x[k + P]);
    if (t == 2)
      return dk[k] * xc - cu[k] * x[k - 1] - cu[k + 1] * x[k + 1] - cv[k] * x[k - P] - cv[k + P] * x[k + P];
    return xc;
  }
};

// Per-block scalar state of the PCG recurrences, computed by thread 0 only (FP64 division
// is a software sequence on this part) and read by every thread from shared memory.
struct PcgScalars {
  double rz, rr, bb, beta, alpha, zmean;
  int it, stop;  // stop: 0 continue, 1 converged, 2 iteration limit
};

// The cells of one thread taken U at a time (t, t + stride, ... of CellWalk), so that every
// load of a group is issued before the first result is needed.  Slots past the end of the
// range get a valid dummy index and are not stored.
template <int U>
struct Group {
  int k[U];
  bool v[U];
};
template <int U>
__device__ __forceinline__ bool next_group(CellWalk& cw, const Geom& g, int kdummy, Group<U>& gr) {
  if (!cw.ok()) return false;
#pragma unroll
  for (int m = 0; m < U; ++m) {
    gr.v[m] = cw.ok();
    gr.k[m] = gr.v[m] ? (int)g.idx(cw.i, cw.j) : kdummy;
    if (gr.v[m]) cw.next();
  }
  return true;
}

// Block sum of NV per-thread values with one warp per quantity: warps 0..NV-1 sit on
// different SM sub-partitions, so their FP64 additions (the narrow pipe of this part) run
// side by side.  Fixed order: a pairwise tree over a lane's NT/32 values, then the shuffle
// tree.  The sums land in out[0..NV-1] (shared), valid after the closing barrier.
template <int NV, int NT = kPcgThreads>
__device__ __forceinline__ void block_sum_warps(const double (&v)[NV], double (*red)[NT], double* out) {
  constexpr int L = NT / 32;
  static_assert(L >= 2 && (L & (L - 1)) == 0, "a power-of-two number of warps");
#pragma unroll
  for (int q = 0; q < NV; ++q) red[q][threadIdx.x] = v[q];
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (w < NV) {
    double t[L];
#pragma unroll
    for (int m = 0; m < L; ++m) t[m] = red[w][lane + 32 * m];
#pragma unroll
    for (int h = L / 2; h > 0; h >>= 1)
#pragma unroll
      for (int m = 0; m < h; ++m) t[m] += t[m + h];
    double s = t[0];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) out[w] = s;
  }
  __syncthreads();
}

// 1 / y by Newton's iteration x <- x + x (1 - y x) from the correctly rounded single-precision
// reciprocal of y's significand (quadratic convergence: 24, then 48, then beyond 53 bits, so
// two steps), scaled back by y's power of two.  For normal, nonzero y; within a few units in
// the last place, which is all the CG recurrences need.
__device__ __forceinline__ double recip_newton(double y) {
  const long long bits = __double_as_longlong(y);
  const int e = (int)((bits >> 52) & 0x7ff) - 1023;
  const double m = __longlong_as_double((bits & ~(0x7ffLL << 52)) | (1023LL << 52));  // +-[1, 2)
  const double s = __longlong_as_double((long long)(1023 - e) << 52);                // 2^-e
  double x = (double)__frcp_rn((float)m);
  double r = fma(-m, x, 1.0);
  x = fma(x, r, x);
  r = fma(-m, x, 1.0);
  x = fma(x, r, x);
  return x * s;
}

// Sum of the partials of blocks base .. base+count-1 (one case of a batch), quantity w by
// warp w, all of a lane's loads in flight; the result in every thread.
template <int NV>
__device__ __forceinline__ void range_sum(const double* partials, int stride, int base, int count, double (&out)[NV],
                                          double* smem) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (w < NV) {
    const double* src = partials + (size_t)w * stride + base;
    double buf[kGridSumPerLane];
#pragma unroll
    for (int m = 0; m < kGridSumPerLane; ++m) {
      const int b = lane + 32 * m;
      buf[m] = b < count ? __ldcg(&src[b]) : 0.0;
    }
    double s = 0.0;
#pragma unroll
    for (int m = 0; m < kGridSumPerLane; ++m) s += buf[m];
    for (int b = lane + 32 * kGridSumPerLane; b < count; b += 32) s += __ldcg(&src[b]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) smem[w] = s;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) out[k] = smem[k];
}

// FP32 block sum of NV values: shuffle tree per warp, then warps 0..NV-1 add the 16 warp
// partials of one quantity each.  Sums land in out[0..NV-1] (shared).
template <int NV>
__device__ __forceinline__ void block_sum_f32(const float (&v)[NV], float (*wred)[kPcgThreads / 32], float* out) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    float s = v[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) wred[q][w] = s;
  }
  __syncthreads();
  if (w < NV) {
    float s = lane < kPcgThreads / 32 ? wred[w][lane] : 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) out[w] = s;
  }
  __syncthreads();
}

}  // namespace ccm
