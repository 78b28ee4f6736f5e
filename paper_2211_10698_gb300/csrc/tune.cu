// Launch-shape autotuner for the one-launch Poisson solves: the tile plan of the FP64 CG with
// one barrier per iteration (pcg_fused.cu) or, on small grids, the size of the one cluster
// that holds the whole FP64 solve (pcg_cluster.cu), and the block count of the
// mixed-precision solve (pcg_mixed.cu).  Which shape is fastest depends on the grid: a large
// grid wants every SM busy, a small one loses more to the grid barrier across many blocks
// than it gains from them.  The caller times each candidate on a short solve of the case's
// own operator (a fixed number of iterations on a scratch right-hand side) and keeps the
// fastest; results are cached per grid size and solver setting for the life of the process.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "ccm_host.h"

namespace ccm {

std::vector<TilePlan> fused_plan_candidates(int nx, int ny, int blocks) {
  std::vector<TilePlan> out;
  TilePlan def{};
  fused_tiles(nx, ny, blocks, &def.TX, &def.TY, &def.nbx, &def.ntiles);
  out.push_back(def);
  // every plan also with its tiles' vectors resident in shared memory, where they fit
  // (the launcher refuses the others)
  for (int tx = 32; tx <= 512; tx *= 2) {
    const int bxn = (nx + tx - 1) / tx;
    if (bxn > blocks) continue;
    if (tx > 32 && (nx + tx / 2 - 1) / (tx / 2) == bxn) continue;  // a narrower tile covers nx the same way
    const int byn_max = std::max(1, std::min(blocks / bxn, ny));
    for (int byn = byn_max; byn >= 1; byn /= 2) {
      const int ty = (ny + byn - 1) / byn;
      TilePlan p{tx, ty, bxn, bxn * ((ny + ty - 1) / ty), 0};
      bool seen = false;
      for (const TilePlan& q : out) seen = seen || (q.TX == p.TX && q.TY == p.TY);
      if (!seen && p.ntiles <= blocks && (long long)std::min(tx, nx) * ty <= 64LL * 512) out.push_back(p);
      if (byn == 1) break;
    }
  }
  const size_t n = out.size();
  for (size_t q = 0; q < n; ++q)
    if (fused_resident_smem(out[q].TX, out[q].TY, false) <= 227 * 1024) {
      TilePlan r = out[q];
      r.resident = 1;
      out.push_back(r);
    }
  return out;
}

std::vector<int> mixed_block_candidates(int blocks) {
  std::vector<int> out;
  for (int b = blocks; b >= 1 && out.size() < 6; b /= 2) out.push_back(b);
  return out;
}

std::vector<int> cluster_candidates(int nx, int ny) {
  std::vector<int> out;
  for (int C = 16; C >= 2; C /= 2)
    if (C <= ny && cluster_smem_bytes(nx, ny, C) <= 200 * 1024) out.push_back(C);
  return out;
}

namespace {

using Key = std::tuple<int, int, int, int, int, int>;  // nx, ny, precision, precond, degree, blocks
std::mutex g_tune_mutex;
std::map<Key, TuneResult> g_tune_cache;

}  // namespace

bool tune_cache_get(int nx, int ny, int precision, int precond, int degree, int blocks, TuneResult* r) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  auto it = g_tune_cache.find(Key{nx, ny, precision, precond, degree, blocks});
  if (it == g_tune_cache.end()) return false;
  *r = it->second;
  return true;
}

void tune_cache_put(int nx, int ny, int precision, int precond, int degree, int blocks, const TuneResult& r) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tune_cache[Key{nx, ny, precision, precond, degree, blocks}] = r;
}

cudaError_t time_launches(int n, const std::function<cudaError_t(int)>& launch, cudaStream_t st, int* best,
                          std::vector<float>* ms) {
  *best = -1;
  ms->assign(n, -1.0f);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  // one untimed run first (caches, first-launch set-up)
  if (e == cudaSuccess && n > 0) e = launch(0);
  for (int k = 0; k < n && e == cudaSuccess; ++k) {
    e = cudaEventRecord(e0, st);
    if (e != cudaSuccess) break;
    const cudaError_t le = launch(k);
    if (le == cudaErrorInvalidConfiguration) continue;  // a shape the launcher refuses: skip it
    if ((e = le) != cudaSuccess) break;
    if ((e = cudaEventRecord(e1, st)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess) break;
    float t = 0.0f;
    if ((e = cudaEventElapsedTime(&t, e0, e1)) != cudaSuccess) break;
    (*ms)[k] = t;
    if (*best < 0 || t < (*ms)[*best]) *best = k;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return e;
}

}  // namespace ccm
