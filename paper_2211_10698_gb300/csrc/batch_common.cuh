// Pieces shared by the batched persistent kernels (pcg_batch.cu, pcg_helm.cu): block b of a
// batched launch serves case block_case[b], whose entry records its first block and block
// count; all blocks pass the same grid barriers.
#pragma once
#include "pcg_common.cuh"

namespace ccm {

// Cell range of this block within its case.
struct CaseRange {
  int t0, t1;
  __device__ CaseRange(int ncell, int lb, int nbc) {
    t0 = (int)((long long)ncell * lb / nbc);
    t1 = (int)((long long)ncell * (lb + 1) / nbc);
  }
};

// The block's case entry, copied to shared memory once: the kernels read its pointers and
// scalars in every slot, and shared loads do not compete with the streamed vectors for L1.
template <class Entry>
__device__ __forceinline__ const Entry& stage_entry(const Entry* cases, const int* block_case, void* smem) {
  static_assert(sizeof(Entry) % sizeof(int) == 0, "entries are copied as ints");
  const int* src = reinterpret_cast<const int*>(cases + block_case[blockIdx.x]);
  int* dst = reinterpret_cast<int*>(smem);
  for (int q = threadIdx.x; q < (int)(sizeof(Entry) / sizeof(int)); q += blockDim.x) dst[q] = src[q];
  __syncthreads();
  return *reinterpret_cast<const Entry*>(smem);
}

// Whether any block's flag is set (the same answer in every block; read after a barrier):
// every thread loads at most a few flags, all in flight at once, and the block ORs them.
__device__ __forceinline__ bool any_running(const int* running, int nb) {
  int f = 0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) f |= __ldcg(&running[b]);
  return __syncthreads_or(f) != 0;
}

}  // namespace ccm
