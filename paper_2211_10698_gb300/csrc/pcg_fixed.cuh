// Exact sums of FP64 values in fixed point, and a device-wide barrier that carries them.
//
// The dot products of a CG iteration are summed over every thread of every block.  In FP64
// that sum is a chain of dependent additions on the narrow FP64 pipe of this part (64 pipe
// cycles per warp instruction), first inside each block and then, after the grid barrier,
// over the blocks' partials: together more than a microsecond of every iteration.  Here each
// thread turns its partial into integers instead, and the sums run on the integer units:
//
//   * A window 2^lo .. 2^(lo + kFxTop) is shared by all blocks (derived from the previous
//     iteration's sums, which every block holds identically).  A value v = +-m 2^e becomes
//     X = trunc(|v| 2^-lo) < 2^kFxTop, written as kFxDigits digits of kFxBits bits each; the
//     sign is applied to every digit, so no carry ever crosses digits.
//   * A warp adds its lanes' digits with one redux.sync per digit (|sum| < 2^31), a block its
//     warps' digit sums in 64-bit integers (|sum| < 2^35).
//   * Each block adds, per digit, (1 << kFxCountShift) + kFxBias + its digit sum to one 64-bit
//     word in global memory (one release reduction per word).  The top bits of a word count
//     the blocks that have added to it, so a word is complete when its count equals the
//     number of blocks: the wait on the words is the grid barrier, and the same load that
//     ends it delivers the sums (one L2 round trip instead of a barrier and then a load of
//     every block's partial).
//   * The digit sums are recombined in 128-bit integer arithmetic, exactly, and rounded once
//     to FP64 (to nearest, ties to even).
//
// Integer addition is associative, so the result does not depend on the order in which
// threads or blocks add: it is bitwise reproducible and more accurate than an FP64 tree (the
// only errors are the truncation of each value below 2^lo, below 2^-88 of the largest
// previous sum, and the final rounding).  A value that does not fit the window (a sum grew
// more than 2^kFxMargin-fold in one iteration, or is not finite) is counted in an extra
// word; every block then sees the count and repeats the reduction in FP64 (the fallback).
//
// Three buffers of words rotate by reduction index: block 0 clears the buffer of reduction
// i - 1 after the wait of reduction i (every block read it before adding to reduction i), and
// that clearing precedes block 0's release for reduction i + 1, which every block acquires
// before it adds to reduction i + 2, the next user of the buffer.
#pragma once
#include <cstring>

#include "pcg_common.cuh"

namespace ccm {

constexpr int kFxDigits = 5;                             // digits per value
constexpr int kFxBits = 26;                              // bits per digit
constexpr int kFxQ = 3;                                  // values per reduction
static_assert(kFxWords == kFxQ * kFxDigits + 1, "digit sums, then the overflow count");
constexpr int kFxCountShift = 50;                        // arrivals counted in bits 50..63
constexpr long long kFxBias = 1LL << 40;                 // keeps a block's addend positive
constexpr int kFxTop = 108;                              // |X| < 2^108: 2^18 summands stay below 2^126
constexpr int kFxMargin = 20;                            // window top: 2^20 times the largest previous sum
static_assert(kFxDigits * kFxBits >= kFxTop + 18, "digits cover the sum's range");
static_assert(kFxWords <= 32, "one lane per word");

// The arithmetic below is plain integer work on bit patterns, the same on the host (where the
// tests check it against exact rational sums) and on the device.
__host__ __device__ __forceinline__ long long fx_bits(double x) {
#ifdef __CUDA_ARCH__
  return __double_as_longlong(x);
#else
  long long b;
  memcpy(&b, &x, sizeof b);
  return b;
#endif
}
__host__ __device__ __forceinline__ double fx_double(long long b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double(b);
#else
  double x;
  memcpy(&x, &b, sizeof x);
  return x;
#endif
}
__host__ __device__ __forceinline__ int fx_clz64(unsigned long long x) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)x);
#else
  return x == 0 ? 64 : __builtin_clzll(x);
#endif
}

// Window bottom for values of the size of a, b, c: 2^lo with 2^(lo + kFxTop) = 2^kFxMargin
// times the largest of their powers of two.  Integer work on the bit patterns only.
__host__ __device__ __forceinline__ int fx_window(double a, double b, double c) {
  auto ex = [](double x) { return (int)((fx_bits(x) >> 52) & 0x7ff); };
  int e = ex(a), eb = ex(b), ec = ex(c);
  if (eb > e) e = eb;
  if (ec > e) e = ec;
  if (e == 0x7ff) e = 1023;  // not finite: the solve stops on it; any window will do
  if (e == 0) e = 1;         // zero or subnormal
  return (e - 1023) + kFxMargin - kFxTop;
}

// The digits of v in the window of bottom 2^lo; false if v does not fit (or is not finite),
// in which case the digits are zero.
__host__ __device__ __forceinline__ bool fx_digits(double v, int lo, int (&d)[kFxDigits]) {
  const unsigned long long b = (unsigned long long)fx_bits(v);
  const int ex = (int)((b >> 52) & 0x7ff);
  unsigned long long m = b & 0xfffffffffffffULL;
  int e = -1074;
  if (ex != 0) {
    m |= 1ULL << 52;
    e = ex - 1075;
  }
  const int s = e - lo;  // position of m's lowest bit in the window
  const bool ok = ex != 0x7ff && (m == 0 || s + 53 <= kFxTop);
  unsigned __int128 X = 0;
  if (ok && m != 0) {
    if (s >= 0) X = (unsigned __int128)m << s;
    else if (s > -64) X = (unsigned __int128)(m >> (-s));
  }
  const bool neg = (b >> 63) != 0;
#pragma unroll
  for (int k = 0; k < kFxDigits; ++k) {
    const int dk = (int)((unsigned long long)(X >> (kFxBits * k)) & ((1ULL << kFxBits) - 1));
    d[k] = neg ? -dk : dk;
  }
  return ok;
}

// x 2^k for |k| <= 2044: two multiplications by normal powers of two (exact unless the
// result is subnormal).
__host__ __device__ __forceinline__ double fx_scale(double x, int k) {
  const int k1 = k / 2, k2 = k - k1;
  return (x * fx_double((long long)(k1 + 1023) << 52)) * fx_double((long long)(k2 + 1023) << 52);
}

// sum_k S[k] 2^(kFxBits k + lo), exactly in 128-bit integers (the true sum is below 2^126
// in magnitude), then rounded once to FP64.
__host__ __device__ __forceinline__ double fx_value(const long long* S, int lo) {
  unsigned __int128 X = 0;
#pragma unroll
  for (int k = 0; k < kFxDigits; ++k) X += (unsigned __int128)(__int128)S[k] << (kFxBits * k);
  const bool neg = (__int128)X < 0;
  const unsigned __int128 U = neg ? (unsigned __int128)0 - X : X;
  if (U == 0) return 0.0;
  const unsigned long long hi = (unsigned long long)(U >> 64), lw = (unsigned long long)U;
  const int n = hi ? 128 - fx_clz64(hi) : 64 - fx_clz64(lw);  // bit length
  // T = the significand, 53 bits, and the value T 2^(lo + sh)
  unsigned long long T;
  int sh = n - 53;
  if (sh <= 0) {
    T = lw << (-sh);  // exact
  } else {
    T = (unsigned long long)(U >> sh);
    const unsigned __int128 rem = U & (((unsigned __int128)1 << sh) - 1);
    const unsigned __int128 half = (unsigned __int128)1 << (sh - 1);
    if (rem > half || (rem == half && (T & 1))) T += 1;  // to nearest, ties to even
    if (T >> 53) {  // rounded up to 2^53
      T >>= 1;
      sh += 1;
    }
  }
  // assembled from its fields when the result is normal (integer work only), otherwise scaled
  const int E = lo + sh + 52 + 1023;  // biased exponent of T 2^(lo + sh), T in [2^52, 2^53)
  const unsigned long long sign = neg ? 1ULL << 63 : 0ULL;
  if (E >= 1 && E <= 2046)
    return fx_double((long long)(sign | ((unsigned long long)E << 52) | (T & 0xfffffffffffffULL)));
  const double r = fx_scale((double)T, lo + sh);
  return neg ? -r : r;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Shared state of one block's fixed-point reduction.
struct FxShared {
  int w[kPcgThreads / 32][kFxWords];  // per-warp digit sums
  long long s[kFxWords];              // the grid's digit sums (and the overflow count)
  int ok;                             // 0: the wait ran out
};

// Arrival: the block's digits of v[0..2] for reduction buffer `buf` (all threads).  Every
// thread's writes before the call are released with the block's words.
template <int NT>
__device__ __forceinline__ void fx_arrive(const double (&v)[4], int lo, unsigned long long* acc, int buf, int absent,
                                          FxShared& sh) {
  int d[kFxWords];
  bool fit = true;
#pragma unroll
  for (int q = 0; q < kFxQ; ++q) {
    int dq[kFxDigits];
    fit = fx_digits(v[q], lo, dq) && fit;
#pragma unroll
    for (int k = 0; k < kFxDigits; ++k) d[q * kFxDigits + k] = dq[k];
  }
  d[kFxWords - 1] = fit ? 0 : 1;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kFxWords; ++k) d[k] = __reduce_add_sync(0xffffffffu, d[k]);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < kFxWords; ++k) sh.w[wid][k] = d[k];
  __syncthreads();
  if (threadIdx.x < kFxWords) {
    long long s = 0;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) s += sh.w[w][threadIdx.x];
    const unsigned long long word = (1ULL << kFxCountShift) + (unsigned long long)(s + kFxBias);
    unsigned long long* dst = acc + ((size_t)buf * kFxWords + threadIdx.x) * kFxStride;
    if ((int)blockIdx.x != absent) asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(dst), "l"(word) : "memory");
  }
}

// Wait: until every block has added to every word of buffer `buf` (bounded by `budget`
// cycles; on give-up *err is raised and false returned), then the grid's digit sums in
// sh.s.  Block 0 then clears buffer `clear`.  All threads.
__device__ __forceinline__ bool fx_wait(unsigned long long* acc, int buf, int clear, long long budget, int* err,
                                        FxShared& sh) {
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    const unsigned long long* src = acc + ((size_t)buf * kFxWords + (lane < kFxWords ? lane : 0)) * kFxStride;
    const unsigned long long nb = gridDim.x;
    unsigned long long w = 0;
    bool done = lane >= kFxWords;
    int ok = 1;
    const long long t0 = clock64();
    while (true) {
      if (!done) {
        w = ld_acquire_u64(src);
        done = (w >> kFxCountShift) == nb;
      }
      if (__all_sync(0xffffffffu, done)) break;
      if (__shfl_sync(0xffffffffu, clock64() - t0 > budget ? 1 : 0, 0)) {
        ok = 0;
        break;
      }
    }
    if (lane < kFxWords)
      sh.s[lane] = (long long)(w & ((1ULL << kFxCountShift) - 1)) - (long long)nb * kFxBias;
    if (lane == 0) {
      sh.ok = ok;
      if (!ok) atomicExch(err, 1);
    }
    if (ok && blockIdx.x == 0 && lane < kFxWords) acc[((size_t)clear * kFxWords + lane) * kFxStride] = 0ULL;
  }
  __syncthreads();
  return sh.ok != 0;
}

}  // namespace ccm
