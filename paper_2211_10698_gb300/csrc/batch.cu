// Batches of independent cases advanced together (the serving form of the projection step).
//
// All cases of a batch run on the batch's stream.  Per step, each case's explicit stages and
// Helmholtz solve are enqueued case by case, then ONE cooperative launch solves the pressure
// Poisson systems of all cases (each case gets a contiguous range of blocks in proportion to
// its expected work, cells x nx, and reduces over its own blocks), then each case's
// projection is enqueued.  When every case has an outflow side (nonsingular systems) the
// launch is k_sc_batch (FP64 CG on the Jacobi-scaled systems) or k_mixed_batch (FP32 CG with
// FP64 residual replacements, for the MIXED setting), both in pcg_batch.cu.  Otherwise the
// unscaled Jacobi-PCG batch of pcg.cu runs, and for MIXED the FP64 residual refinement runs
// from the host for the whole batch: residuals of the unconverged cases, one host check, one
// batched FP32 inner solve for those cases, corrections, until every case meets tol_p.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "ccm_host.h"

using namespace ccm;

struct ccm_batch_s {
  cudaStream_t st = nullptr;
  int max_cases = 0;
  int blocks = 0;
  std::vector<ccm_case> cases;
  void* dev = nullptr;
  BatchEntry<double>* e64 = nullptr;
  BatchEntry<float>* e32 = nullptr;
  ScaledBatchEntry* esc = nullptr;
  MixedBatchEntry* emx = nullptr;
  int* block_case = nullptr;
  double* partials = nullptr;
  int* running = nullptr;
  unsigned int* bar_count = nullptr;
  int* bar_err = nullptr;
  double* host_sums = nullptr;  // pinned: 2 per case
};

namespace {

ccm_status bfail(ccm_status s, const std::string& m) {
  set_last_error(m);
  return s;
}

// Contiguous block ranges proportional to the expected PCG work (cells x nx: Jacobi
// iterations grow like the grid dimension), at least one block per case.
void allocate_blocks(const std::vector<ccm_case>& cs, int blocks, std::vector<int>& b0, std::vector<int>& nb) {
  const int n = (int)cs.size();
  std::vector<double> w(n);
  double tot = 0.0;
  for (int i = 0; i < n; ++i) {
    w[i] = (double)case_cells(cs[i]) * (double)case_nx(cs[i]);
    tot += w[i];
  }
  nb.assign(n, 1);
  int left = blocks - n;
  std::vector<std::pair<double, int>> rem;
  for (int i = 0; i < n; ++i) {
    const double share = left * w[i] / tot;
    const int f = (int)std::floor(share);
    nb[i] += f;
    rem.push_back({share - f, i});
  }
  int used = 0;
  for (int v : nb) used += v;
  std::sort(rem.begin(), rem.end(), [](const std::pair<double, int>& a, const std::pair<double, int>& b) {
    return a.first > b.first || (a.first == b.first && a.second < b.second);
  });
  for (int k = 0; used < blocks && k < n; ++k, ++used) nb[rem[k].second] += 1;
  b0.assign(n, 0);
  for (int i = 1; i < n; ++i) b0[i] = b0[i - 1] + nb[i - 1];
}

}  // namespace

// One launch of k_sc_batch (FP64) or k_mixed_batch (MIXED) for all cases.
static ccm_status batch_solve_scaled(ccm_batch b, bool mixed) {
  const std::vector<ccm_case>& cs = b->cases;
  const int n = (int)cs.size();
  std::vector<int> b0, nb;
  allocate_blocks(cs, b->blocks, b0, nb);
  std::vector<int> block_case(b->blocks);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < nb[i]; ++k) block_case[b0[i] + k] = i;
  BatchControl ctl{b->partials, b->running, Barrier{b->bar_count, b->bar_err, 2000000000LL}};
  cudaError_t e = cudaMemcpyAsync(b->block_case, block_case.data(), sizeof(int) * b->blocks, cudaMemcpyHostToDevice,
                                  b->st);
  std::vector<ScaledBatchEntry> es;
  std::vector<MixedBatchEntry> em;
  if (e == cudaSuccess && !mixed) {
    es.resize(n);
    for (int i = 0; i < n; ++i) {
      case_scaled_fp64(cs[i], &es[i].a);
      es[i].block0 = b0[i];
      es[i].nblocks = nb[i];
    }
    e = cudaMemcpyAsync(b->esc, es.data(), sizeof(ScaledBatchEntry) * n, cudaMemcpyHostToDevice, b->st);
    if (e == cudaSuccess) e = run_scaled_batch(b->esc, b->block_case, ctl, b->blocks, b->st);
  } else if (e == cudaSuccess) {
    em.resize(n);
    for (int i = 0; i < n; ++i) {
      case_mixed_batch(cs[i], &em[i].a);
      em[i].block0 = b0[i];
      em[i].nblocks = nb[i];
    }
    e = cudaMemcpyAsync(b->emx, em.data(), sizeof(MixedBatchEntry) * n, cudaMemcpyHostToDevice, b->st);
    if (e == cudaSuccess) e = run_mixed_batch(b->emx, b->block_case, ctl, b->blocks, b->st);
  }
  // the host tables must outlive the asynchronous copies
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
  if (e != cudaSuccess) return bfail(CCM_E_CUDA, std::string("batched Poisson solve: ") + cudaGetErrorString(e));
  int err = 0;
  if ((e = cudaMemcpy(&err, b->bar_err, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return bfail(CCM_E_CUDA, cudaGetErrorString(e));
  if (err) {
    cudaMemset(b->bar_err, 0, sizeof(int));
    return bfail(CCM_E_TIMEOUT, "a device-wide barrier gave up waiting");
  }
  return CCM_OK;
}

static bool all_scaled(ccm_batch b) {
  for (ccm_case c : b->cases)
    if (!case_scaled_ok(c)) return false;
  return true;
}

static ccm_status batch_solve(ccm_batch b, const std::vector<ccm_case>& cs, bool fp32) {
  const int n = (int)cs.size();
  if (n == 0) return CCM_OK;
  std::vector<int> b0, nb;
  allocate_blocks(cs, b->blocks, b0, nb);
  std::vector<int> block_case(b->blocks);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < nb[i]; ++k) block_case[b0[i] + k] = i;
  cudaError_t e;
  BatchControl ctl{b->partials, b->running, Barrier{b->bar_count, b->bar_err, 2000000000LL}};
  if ((e = cudaMemcpyAsync(b->block_case, block_case.data(), sizeof(int) * b->blocks, cudaMemcpyHostToDevice, b->st)) !=
      cudaSuccess)
    return bfail(CCM_E_CUDA, std::string("batch table upload: ") + cudaGetErrorString(e));
  if (!fp32) {
    std::vector<PoissonSolve<double>> sv(n);
    std::vector<BatchEntry<double>> ent(n);
    for (int i = 0; i < n; ++i) {
      case_poisson_fp64(cs[i], &sv[i]);
      ent[i].a = sv[i];
      ent[i].block0 = b0[i];
      ent[i].nblocks = nb[i];
    }
    if ((e = cudaMemcpyAsync(b->e64, ent.data(), sizeof(BatchEntry<double>) * n, cudaMemcpyHostToDevice, b->st)) !=
        cudaSuccess)
      return bfail(CCM_E_CUDA, std::string("batch table upload: ") + cudaGetErrorString(e));
    e = run_poisson_batch<double>(sv.data(), n, b->e64, b->block_case, ctl, b->blocks, b->st);
    // the host vectors must outlive the asynchronous copies
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
  } else {
    std::vector<PoissonSolve<float>> sv(n);
    std::vector<BatchEntry<float>> ent(n);
    for (int i = 0; i < n; ++i) {
      case_poisson_fp32(cs[i], &sv[i]);
      ent[i].a = sv[i];
      ent[i].block0 = b0[i];
      ent[i].nblocks = nb[i];
    }
    if ((e = cudaMemcpyAsync(b->e32, ent.data(), sizeof(BatchEntry<float>) * n, cudaMemcpyHostToDevice, b->st)) !=
        cudaSuccess)
      return bfail(CCM_E_CUDA, std::string("batch table upload: ") + cudaGetErrorString(e));
    e = run_poisson_batch<float>(sv.data(), n, b->e32, b->block_case, ctl, b->blocks, b->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
  }
  if (e != cudaSuccess) return bfail(CCM_E_CUDA, std::string("batched Poisson PCG: ") + cudaGetErrorString(e));
  int err = 0;
  if ((e = cudaMemcpy(&err, b->bar_err, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return bfail(CCM_E_CUDA, cudaGetErrorString(e));
  if (err) {
    cudaMemset(b->bar_err, 0, sizeof(int));
    return bfail(CCM_E_TIMEOUT, "a device-wide barrier gave up waiting");
  }
  return CCM_OK;
}

static ccm_status batch_mixed(ccm_batch b) {
  const int n = (int)b->cases.size();
  std::vector<char> done(n, 0);
  std::vector<long long> inner(n, 0);
  std::vector<int> outer(n, 0);
  std::vector<double> rr(n, 0.0), bb(n, 0.0);
  int sweep = 0;
  for (; sweep < 60; ++sweep) {
    std::vector<ccm_case> act;
    for (int i = 0; i < n; ++i)
      if (!done[i]) case_mixed_residual(b->cases[i], b->host_sums + 2 * i);
    cudaError_t e = cudaStreamSynchronize(b->st);
    if (e != cudaSuccess) return bfail(CCM_E_CUDA, std::string("mixed refinement: ") + cudaGetErrorString(e));
    for (int i = 0; i < n; ++i) {
      if (done[i]) continue;
      rr[i] = b->host_sums[2 * i];
      bb[i] = b->host_sums[2 * i + 1];
      CaseSolveView v;
      case_solve_view(b->cases[i], &v);
      const double tolp = v.tol;
      if (bb[i] == 0.0 || rr[i] <= tolp * tolp * bb[i]) {
        done[i] = 1;
        outer[i] = sweep;
        continue;
      }
      act.push_back(b->cases[i]);
    }
    if (act.empty()) break;
    ccm_status s = batch_solve(b, act, true);
    if (s != CCM_OK) return s;
    for (size_t k = 0; k < act.size(); ++k) {
      int it = 0;
      cudaMemcpy(&it, case_inner_iters_dev(act[k]), sizeof(int), cudaMemcpyDeviceToHost);
      for (int i = 0; i < n; ++i)
        if (b->cases[i] == act[k]) inner[i] += it;
      case_mixed_correct(act[k]);
    }
  }
  for (int i = 0; i < n; ++i) case_mixed_account(b->cases[i], inner[i], done[i] ? outer[i] : sweep, rr[i], bb[i], done[i]);
  return CCM_OK;
}

extern "C" {

ccm_status ccm_batch_create(int max_cases, void* stream, ccm_batch* out) {
  set_last_error("");
  if (!out || max_cases < 1) return bfail(CCM_E_INVALID, "max_cases must be >= 1");
  ccm_batch b = new ccm_batch_s();
  b->st = (cudaStream_t)stream;
  b->max_cases = max_cases;
  b->blocks = std::min(batch_blocks(), batch_scaled_blocks());
  if (max_cases > b->blocks) {
    const int most = b->blocks;
    delete b;
    return bfail(CCM_E_INVALID, "a batch holds at most " + std::to_string(most) + " cases on this GPU");
  }
  const size_t pieces[9] = {sizeof(BatchEntry<double>) * max_cases, sizeof(BatchEntry<float>) * max_cases,
                            sizeof(ScaledBatchEntry) * max_cases, sizeof(MixedBatchEntry) * max_cases,
                            sizeof(int) * b->blocks, sizeof(double) * 6 * b->blocks, sizeof(int) * b->blocks,
                            sizeof(unsigned int) * kBarWords, sizeof(int) * 4};
  size_t bytes = 0;
  for (size_t n : pieces) bytes += (n + 255) & ~(size_t)255;
  cudaError_t e = cudaMalloc(&b->dev, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return bfail(CCM_E_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  char* p = (char*)b->dev;
  auto take = [&](size_t n) { char* q = p; p += (n + 255) & ~(size_t)255; return (void*)q; };
  b->e64 = (BatchEntry<double>*)take(sizeof(BatchEntry<double>) * max_cases);
  b->e32 = (BatchEntry<float>*)take(sizeof(BatchEntry<float>) * max_cases);
  b->esc = (ScaledBatchEntry*)take(sizeof(ScaledBatchEntry) * max_cases);
  b->emx = (MixedBatchEntry*)take(sizeof(MixedBatchEntry) * max_cases);
  b->block_case = (int*)take(sizeof(int) * b->blocks);
  b->partials = (double*)take(sizeof(double) * 6 * b->blocks);
  b->running = (int*)take(sizeof(int) * b->blocks);
  b->bar_count = (unsigned int*)take(sizeof(unsigned int) * kBarWords);
  b->bar_err = (int*)take(sizeof(int) * 4);
  (void)take;
  if ((e = cudaMallocHost(&b->host_sums, sizeof(double) * 2 * max_cases)) != cudaSuccess ||
      (e = cudaMemset(b->dev, 0, bytes)) != cudaSuccess) {
    cudaFree(b->dev);
    if (b->host_sums) cudaFreeHost(b->host_sums);
    delete b;
    return bfail(CCM_E_CUDA, cudaGetErrorString(e));
  }
  *out = b;
  return CCM_OK;
}

ccm_status ccm_batch_destroy(ccm_batch b) {
  if (!b) return CCM_OK;
  cudaStreamSynchronize(b->st);
  cudaFree(b->dev);
  cudaFreeHost(b->host_sums);
  delete b;
  return CCM_OK;
}

ccm_status ccm_batch_add(ccm_batch b, ccm_case c) {
  set_last_error("");
  if (!b || !c) return bfail(CCM_E_INVALID, "null argument");
  CaseSolveView v;
  if (!case_solve_view(c, &v)) return bfail(CCM_E_STATE, "set_geometry must come first");
  if (case_stream(c) != b->st) return bfail(CCM_E_INVALID, "the case must use the batch's stream");
  if ((int)b->cases.size() >= b->max_cases) return bfail(CCM_E_INVALID, "batch is full");
  if (!b->cases.empty() && case_is_mixed(b->cases[0]) != case_is_mixed(c))
    return bfail(CCM_E_INVALID, "all cases of a batch use the same precision setting");
  if (std::find(b->cases.begin(), b->cases.end(), c) != b->cases.end())
    return bfail(CCM_E_INVALID, "case already in the batch");
  b->cases.push_back(c);
  return CCM_OK;
}

ccm_status ccm_batch_remove(ccm_batch b, ccm_case c) {
  set_last_error("");
  if (!b || !c) return bfail(CCM_E_INVALID, "null argument");
  auto it = std::find(b->cases.begin(), b->cases.end(), c);
  if (it == b->cases.end()) return bfail(CCM_E_INVALID, "case not in the batch");
  cudaStreamSynchronize(b->st);
  b->cases.erase(it);
  return CCM_OK;
}

int ccm_batch_size(ccm_batch b) { return b ? (int)b->cases.size() : 0; }

ccm_status ccm_batch_step(ccm_batch b, int nsteps, ccm_step_stats* stats) {
  set_last_error("");
  if (!b) return bfail(CCM_E_INVALID, "null batch");
  if (nsteps < 0) return bfail(CCM_E_INVALID, "nsteps < 0");
  if (b->cases.empty()) return CCM_OK;
  const bool mixed = case_is_mixed(b->cases[0]);
  const bool scaled = all_scaled(b);
  ccm_status s;
  for (int n = 0; n < nsteps; ++n) {
    for (ccm_case c : b->cases)
      if ((s = case_stage_predict(c)) != CCM_OK) return s;
    if (scaled) {
      if ((s = batch_solve_scaled(b, mixed)) != CCM_OK) return s;
    } else if (mixed) {
      if ((s = batch_mixed(b)) != CCM_OK) return s;
    } else {
      if ((s = batch_solve(b, b->cases, false)) != CCM_OK) return s;
    }
    for (ccm_case c : b->cases) case_stage_project(c);
  }
  ccm_status worst = CCM_OK;
  for (size_t i = 0; i < b->cases.size(); ++i) {
    s = case_finish(b->cases[i], stats ? &stats[i] : nullptr);
    if (s != CCM_OK && worst == CCM_OK) worst = s;
  }
  return worst;
}

}  // extern "C"
