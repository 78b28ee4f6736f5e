// Batches of independent cases advanced together (the serving form of the projection step).
//
// All cases of a batch run on the batch's stream, and every stage of a step is one launch for
// all cases: the explicit stages (box data, predictor right-hand side, U* and the Poisson
// right-hand side, projection) run the single-case per-point code over a table of cases
// (operators.cu), the CN Helmholtz solves one cooperative launch (pcg_helm.cu), and the
// pressure Poisson solves one cooperative launch (each case gets a contiguous range of blocks
// in proportion to its expected work and reduces over its own blocks).  When every case has
// an outflow side (nonsingular systems) the Poisson launch is k_sc_batch (FP64 CG on the
// Jacobi-scaled systems) or k_mixed_batch (FP32 CG with FP64 residual replacements, Jacobi or
// Chebyshev per case, for the MIXED setting), both in pcg_batch.cu.  Otherwise the unscaled
// Jacobi-PCG batch of pcg.cu runs, and for MIXED the FP64 residual refinement runs from the
// host for the whole batch: residuals of the unconverged cases, one host check, one batched
// FP32 inner solve for those cases, corrections, until every case meets tol_p.
#include <algorithm>
#include <cmath>
#include <queue>
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
  unsigned int* case_bar = nullptr;  // per-case barrier counters of the mixed Poisson launch
  int* bar_err = nullptr;
  double* host_sums = nullptr;  // pinned: 2 per case
  // batched explicit stages and Helmholtz solves: device tables and their pinned staging
  StageCase* stages = nullptr;
  int* stage_starts = nullptr;
  HelmBatchEntry* helm = nullptr;
  int* helm_block_case = nullptr;
  void* pinned = nullptr;
  StageCase* h_stages = nullptr;
  int* h_starts = nullptr;
  HelmBatchEntry* h_helm = nullptr;
  int* h_helm_block_case = nullptr;
  cudaEvent_t tables_done = nullptr;  // the last upload of the pinned tables has completed
  // captured steps: graph k runs a step with stage table k (k = 1: one step ahead)
  StageCase* stages2 = nullptr;
  bool use_graphs = true;
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  std::vector<unsigned long long> gcases;  // serials of the cases the graphs were captured for
  std::vector<int> gcur;         // their time-level parity when graph 0 is next
  int gphase = 0;                // the graph the next step replays
  bool gmixed = false;
  bool gextra = false;               // the captured predictor has the g / D terms
  long long graph_steps = 0;     // steps replayed from graphs
  cudaStream_t cap_st = nullptr; // capture runs here (the legacy default stream cannot capture)
  // online tuning of the Poisson launch's block split (see split_candidates)
  bool tune = true;
  int tune_next = 0;               // candidate the next tuned step uses (== kSplitN: done)
  double tune_cost[3] = {0, 0, 0};
  double tune_cells = 0.0;           // cells of the batch the split was (is being) tuned on
  double split_exp = 0.0;          // the chosen exponent a of the weights cells x nx^a
  cudaEvent_t tev[2] = {nullptr, nullptr};
};

namespace {

ccm_status bfail(ccm_status s, const std::string& m) {
  set_last_error(m);
  return s;
}

// Contiguous block ranges for the cases' expected work w: at least one block per case, then
// each further block to the case whose work per block is largest (this minimises the largest
// work per block, which sets the launch's length: every slot waits for the slowest block).
void allocate_blocks(const std::vector<double>& w, int blocks, std::vector<int>& b0, std::vector<int>& nb) {
  const int n = (int)w.size();
  nb.assign(n, 1);
  std::priority_queue<std::pair<double, int>> q;
  for (int i = 0; i < n; ++i) q.push({w[i], -i});
  for (int left = blocks - n; left > 0; --left) {
    const int i = -q.top().second;
    q.pop();
    nb[i] += 1;
    q.push({w[i] / nb[i], -i});
  }
  b0.assign(n, 0);
  for (int i = 1; i < n; ++i) b0[i] = b0[i - 1] + nb[i - 1];
}

}  // namespace

// Block weights of the cooperative launches: cells x nx^a.  The Poisson launches give every
// case its own barriers, so a case's solve takes about its cells x iterations over its
// blocks, and the largest cases iterate longest, which favours giving them more blocks
// (a > 0); the Helmholtz launch, whose cases share every barrier and take about the same
// iteration count at every size, uses a = 0.  The Poisson launch's a is tuned on the batch's
// own steps (split_candidates).
static std::vector<double> cell_weights(const std::vector<ccm_case>& cs, double a = 0.0) {
  std::vector<double> w(cs.size());
  for (size_t i = 0; i < cs.size(); ++i) w[i] = (double)case_cells(cs[i]) * std::pow((double)case_nx(cs[i]), a);
  return w;
}
// Exponents tried for the Poisson split, one batch step each (the steps advance the cases as
// usual); the one with the least Poisson time per cell-iteration is kept.  With per-case
// barriers the 64-case mix keeps a = 1 (60.3 M cell-steps/s); the expected work as weights
// (cells x the iterations of each case's last solve, refreshed as the counts drift) measured
// 56.4 M with the split fixed, and as a fourth candidate the tuner, which sees each candidate on
// a different step, picked it on one run (56.2 M), so it is not offered.
constexpr int kSplitN = 3;
static const double split_candidates[kSplitN] = {0.0, 0.5, 1.0};

// Waits for the stream and turns a barrier give-up of any launch since the last check into
// CCM_E_TIMEOUT.
static ccm_status check_barrier(ccm_batch b, const char* what) {
  cudaError_t e = cudaStreamSynchronize(b->st);
  if (e != cudaSuccess) return bfail(CCM_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  int err = 0;
  if ((e = cudaMemcpy(&err, b->bar_err, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return bfail(CCM_E_CUDA, cudaGetErrorString(e));
  if (err) {
    cudaMemset(b->bar_err, 0, sizeof(int));
    return bfail(CCM_E_TIMEOUT, "a device-wide barrier gave up waiting");
  }
  return CCM_OK;
}

// Entries and block map of the scaled Poisson launch (k_sc_batch for FP64, k_mixed_batch for
// MIXED), copied to the device; returns once the copies have completed.
static ccm_status upload_poisson_tables(ccm_batch b, bool mixed) {
  const std::vector<ccm_case>& cs = b->cases;
  const int n = (int)cs.size();
  std::vector<int> b0, nb;
  allocate_blocks(cell_weights(cs, b->split_exp), b->blocks, b0, nb);
  std::vector<int> block_case(b->blocks);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < nb[i]; ++k) block_case[b0[i] + k] = i;
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
  } else if (e == cudaSuccess) {
    em.resize(n);
    for (int i = 0; i < n; ++i) {
      case_mixed_batch(cs[i], &em[i].a);
      em[i].block0 = b0[i];
      em[i].nblocks = nb[i];
    }
    e = cudaMemcpyAsync(b->emx, em.data(), sizeof(MixedBatchEntry) * n, cudaMemcpyHostToDevice, b->st);
  }
  // the host tables must outlive the asynchronous copies
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
  if (e != cudaSuccess) return bfail(CCM_E_CUDA, std::string("batched Poisson tables: ") + cudaGetErrorString(e));
  return CCM_OK;
}

// One cooperative launch solves every case's Poisson system (tables already on the device).
static cudaError_t launch_poisson_scaled(ccm_batch b, bool mixed) {
  BatchControl ctl{b->partials, b->running, Barrier{b->bar_count, b->bar_err, 2000000000LL}, b->case_bar,
                   (int)b->cases.size()};
  return mixed ? run_mixed_batch(b->emx, b->block_case, ctl, b->blocks, b->st)
               : run_scaled_batch(b->esc, b->block_case, ctl, b->blocks, b->st);
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
  allocate_blocks(cell_weights(cs), b->blocks, b0, nb);
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
  // singular systems: Phi and the right-hand side onto zero mean in FP64 first (and Phi again
  // at the end), as the single-case refinement does
  for (ccm_case c : b->cases) {
    ccm_status s = case_mixed_project(c, true);
    if (s != CCM_OK) return s;
  }
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
  for (ccm_case c : b->cases) {
    ccm_status s = case_mixed_project(c, false);
    if (s != CCM_OK) return s;
  }
  for (int i = 0; i < n; ++i)
    case_mixed_account(b->cases[i], inner[i], done[i] ? outer[i] : sweep, rr[i], bb[i], done[i]);
  return CCM_OK;
}

// Tables of the batched explicit stages (ahead = 0: the next step; 1: the step after it) and,
// with `helm`, of the Helmholtz launch.  They are written to pinned memory and copied to the
// device on the batch's stream; the previous copy must have completed before the pinned
// tables are rewritten.
static ccm_status upload_stage_tables(ccm_batch b, StageCase* dst, int ahead, bool helm) {
  const std::vector<ccm_case>& cs = b->cases;
  const int n = (int)cs.size();
  cudaError_t e = cudaEventSynchronize(b->tables_done);
  if (e != cudaSuccess) return bfail(CCM_E_CUDA, std::string("batched stages: ") + cudaGetErrorString(e));
  int total = 0;
  for (int i = 0; i < n; ++i) {
    case_stage_case(cs[i], &b->h_stages[i], ahead);
    b->h_starts[i] = total;
    int gx = 0;
    total += stage_case_blocks(b->h_stages[i].g, &gx);
  }
  b->h_starts[n] = total;
  cudaStream_t st = b->st;
  e = cudaMemcpyAsync(dst, b->h_stages, sizeof(StageCase) * n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->stage_starts, b->h_starts, sizeof(int) * (n + 1), cudaMemcpyHostToDevice, st);
  if (helm && e == cudaSuccess) {
    std::vector<int> b0, nb;
    allocate_blocks(cell_weights(cs), b->blocks, b0, nb);
    for (int i = 0; i < n; ++i) {
      case_helm_solve(cs[i], &b->h_helm[i].a);
      b->h_helm[i].block0 = b0[i];
      b->h_helm[i].nblocks = nb[i];
      for (int k = 0; k < nb[i]; ++k) b->h_helm_block_case[b0[i] + k] = i;
    }
    e = cudaMemcpyAsync(b->helm, b->h_helm, sizeof(HelmBatchEntry) * n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->helm_block_case, b->h_helm_block_case, sizeof(int) * b->blocks, cudaMemcpyHostToDevice,
                          st);
  }
  if (e == cudaSuccess) e = cudaEventRecord(b->tables_done, st);
  if (e != cudaSuccess) return bfail(CCM_E_CUDA, std::string("batched stage tables: ") + cudaGetErrorString(e));
  return CCM_OK;
}

// The explicit stages and the Helmholtz solves of one step, one launch per stage for all
// cases (Eq. pm_prediction: box data, right-hand side, CN Helmholtz solve, box data, then U*
// and the Poisson right-hand side cont(U*, D)).
static cudaError_t launch_predict(ccm_batch b, const StageCase* tab) {
  const int n = (int)b->cases.size();
  const int total = b->h_starts[n];
  cudaStream_t st = b->st;
  BatchControl ctl{b->partials, b->running, Barrier{b->bar_count, b->bar_err, 2000000000LL}};
  cudaError_t e = launch_stage_batch(STAGE_FILL_BC, tab, b->stage_starts, n, total, st);
  bool extra = false;
  for (ccm_case c : b->cases) extra = extra || case_has_extras(c);
  if (e == cudaSuccess) e = launch_stage_batch(STAGE_PREDICT, tab, b->stage_starts, n, total, st, extra);
  if (e == cudaSuccess) e = run_helm_batch(b->helm, b->helm_block_case, ctl, b->blocks, st);
  if (e == cudaSuccess) e = launch_stage_batch(STAGE_FILL_BC, tab, b->stage_starts, n, total, st);
  if (e == cudaSuccess) e = launch_stage_batch(STAGE_DIVERGENCE, tab, b->stage_starts, n, total, st);
  return e;
}

// ... and after the Poisson solves: projection and pressure update (Eqs. pm_projection,
// pm_update), then box data.
static cudaError_t launch_project(ccm_batch b, const StageCase* tab) {
  const int n = (int)b->cases.size();
  const int total = b->h_starts[n];
  cudaError_t e = launch_stage_batch(STAGE_PROJECT, tab, b->stage_starts, n, total, b->st);
  if (e == cudaSuccess) e = launch_stage_batch(STAGE_FILL_BC, tab, b->stage_starts, n, total, b->st);
  return e;
}

static void drop_graphs(ccm_batch b) {
  for (cudaGraphExec_t& g : b->gexec)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  b->gcases.clear();
  b->gcur.clear();
}

// Whether the captured graphs still describe the batch: the same cases (by serial number: a
// new case can take a destroyed one's address), each at the time level the graph about to run
// expects (a case stepped on its own in between invalidates).
static bool graphs_valid(ccm_batch b, bool mixed) {
  if (!b->gexec[0] || !b->gexec[1] || b->gcases.size() != b->cases.size() || b->gmixed != mixed) return false;
  bool extra = false;
  for (ccm_case c : b->cases) extra = extra || case_has_extras(c);
  if (extra != b->gextra) return false;  // the graphs hold the predictor variant of their capture
  for (size_t i = 0; i < b->cases.size(); ++i)
    if (case_serial(b->cases[i]) != b->gcases[i] || case_cur(b->cases[i]) != (b->gcur[i] ^ b->gphase)) return false;
  return true;
}

// Captures one step with each stage table (the next step and the one after it): explicit
// stages, Helmholtz launch, Poisson launch, projection.  The tables are uploaded once, before
// capture; a step replays with no host work but the bookkeeping of the time levels.  If the
// capture fails, *ok stays false, the batch stops trying (its steps issue every launch) and
// ccm_last_error says why.
static ccm_status capture_graphs(ccm_batch b, bool mixed, bool* ok) {
  *ok = false;
  drop_graphs(b);
  ccm_status s;
  if ((s = upload_stage_tables(b, b->stages, 0, true)) != CCM_OK) return s;
  if ((s = upload_stage_tables(b, b->stages2, 1, false)) != CCM_OK) return s;
  if ((s = upload_poisson_tables(b, mixed)) != CCM_OK) return s;
  const StageCase* tab[2] = {b->stages, b->stages2};
  if (!b->cap_st && cudaStreamCreateWithFlags(&b->cap_st, cudaStreamNonBlocking) != cudaSuccess) {
    b->cap_st = nullptr;
    cudaGetLastError();
    return CCM_OK;
  }
  const cudaStream_t run_st = b->st;
  for (int k = 0; k < 2; ++k) {
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->cap_st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      set_last_error(std::string("graph capture (steps run without graphs): ") + cudaGetErrorString(e));
      cudaGetLastError();
      drop_graphs(b);
      b->use_graphs = false;  // not again for this batch
      return CCM_OK;
    }
    b->st = b->cap_st;  // the launch helpers issue on b->st
    cudaError_t le = launch_predict(b, tab[k]);
    if (le == cudaSuccess) le = launch_poisson_scaled(b, mixed);
    if (le == cudaSuccess) le = launch_project(b, tab[k]);
    b->st = run_st;
    e = cudaStreamEndCapture(b->cap_st, &graph);
    if (le != cudaSuccess || e != cudaSuccess || !graph) {
      set_last_error(std::string("graph capture (steps run without graphs): ") +
                     cudaGetErrorString(le != cudaSuccess ? le : e));
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      drop_graphs(b);
      b->use_graphs = false;  // not again for this batch
      return CCM_OK;
    }
    e = cudaGraphInstantiate(&b->gexec[k], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      set_last_error(std::string("graph instantiation (steps run without graphs): ") + cudaGetErrorString(e));
      b->gexec[k] = nullptr;
      cudaGetLastError();
      drop_graphs(b);
      b->use_graphs = false;  // not again for this batch
      return CCM_OK;
    }
  }
  b->gcases.clear();
  b->gcur.clear();
  for (ccm_case c : b->cases) {
    b->gcases.push_back(case_serial(c));
    b->gcur.push_back(case_cur(c));
  }
  b->gphase = 0;
  b->gmixed = mixed;
  b->gextra = false;
  for (ccm_case c : b->cases) b->gextra = b->gextra || case_has_extras(c);
  *ok = true;
  return CCM_OK;
}

// One step without graphs: tables uploaded, every launch issued, the stream waited for.
static ccm_status eager_step(ccm_batch b, bool mixed, bool scaled, float* poisson_ms = nullptr) {
  ccm_status s;
  if ((s = upload_stage_tables(b, b->stages, 0, true)) != CCM_OK) return s;
  if (scaled && (s = upload_poisson_tables(b, mixed)) != CCM_OK) return s;
  cudaError_t e = launch_predict(b, b->stages);
  if (e != cudaSuccess) return bfail(CCM_E_CUDA, std::string("batched stages: ") + cudaGetErrorString(e));
  if (scaled) {
    if (poisson_ms && b->tev[0]) cudaEventRecord(b->tev[0], b->st);
    if ((e = launch_poisson_scaled(b, mixed)) != cudaSuccess)
      return bfail(CCM_E_CUDA, std::string("batched Poisson solve: ") + cudaGetErrorString(e));
    if (poisson_ms && b->tev[1]) cudaEventRecord(b->tev[1], b->st);
  } else if (mixed) {
    if ((s = batch_mixed(b)) != CCM_OK) return s;
  } else {
    if ((s = batch_solve(b, b->cases, false)) != CCM_OK) return s;
  }
  if ((e = launch_project(b, b->stages)) != cudaSuccess)
    return bfail(CCM_E_CUDA, std::string("batched stages: ") + cudaGetErrorString(e));
  if ((s = check_barrier(b, "batched step")) != CCM_OK) return s;
  if (poisson_ms && (!b->tev[0] || cudaEventElapsedTime(poisson_ms, b->tev[0], b->tev[1]) != cudaSuccess)) {
    cudaGetLastError();
    *poisson_ms = -1.0f;
  }
  for (ccm_case c : b->cases) case_step_done(c);
  return CCM_OK;
}

// One step with the next candidate split of the Poisson launch, its cost (Poisson time per
// cell-iteration of the step) recorded; after the last candidate the cheapest is kept.
static ccm_status tuning_step(ccm_batch b, bool mixed) {
  const int k = b->tune_next;
  b->split_exp = split_candidates[k];
  if (!b->tev[0] && (cudaEventCreate(&b->tev[0]) != cudaSuccess || cudaEventCreate(&b->tev[1]) != cudaSuccess)) {
    cudaGetLastError();
    b->tune = false;
  }
  float ms = -1.0f;
  ccm_status s = eager_step(b, mixed, true, b->tune ? &ms : nullptr);
  if (s != CCM_OK) return s;
  double work = 0.0;
  for (ccm_case c : b->cases) {
    int it = 0;
    if (cudaMemcpy(&it, case_inner_iters_dev(c), sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      return bfail(CCM_E_CUDA, "batch tuning: reading iteration counts");
    }
    work += (double)case_cells(c) * (double)it;
  }
  b->tune_cost[k] = ms > 0.0f && work > 0.0 ? ms / work : 1e300;
  b->tune_next = k + 1;
  if (b->tune_next == kSplitN) {
    int best = 0;
    for (int q = 1; q < kSplitN; ++q)
      if (b->tune_cost[q] < b->tune_cost[best]) best = q;
    b->split_exp = split_candidates[best];
  }
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
  const size_t pieces[15] = {sizeof(BatchEntry<double>) * max_cases, sizeof(BatchEntry<float>) * max_cases,
                             sizeof(ScaledBatchEntry) * max_cases, sizeof(MixedBatchEntry) * max_cases,
                             sizeof(int) * b->blocks, sizeof(double) * 6 * b->blocks, sizeof(int) * 2 * b->blocks,
                             sizeof(unsigned int) * kBarWords, sizeof(int) * 4, sizeof(StageCase) * max_cases,
                             sizeof(int) * (max_cases + 1), sizeof(HelmBatchEntry) * max_cases,
                             sizeof(int) * b->blocks, sizeof(StageCase) * max_cases,
                             sizeof(unsigned int) * kCaseBarStride * (size_t)max_cases};
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
  b->running = (int*)take(sizeof(int) * 2 * b->blocks);
  b->bar_count = (unsigned int*)take(sizeof(unsigned int) * kBarWords);
  b->bar_err = (int*)take(sizeof(int) * 4);
  b->stages = (StageCase*)take(sizeof(StageCase) * max_cases);
  b->stage_starts = (int*)take(sizeof(int) * (max_cases + 1));
  b->helm = (HelmBatchEntry*)take(sizeof(HelmBatchEntry) * max_cases);
  b->helm_block_case = (int*)take(sizeof(int) * b->blocks);
  b->stages2 = (StageCase*)take(sizeof(StageCase) * max_cases);
  b->case_bar = (unsigned int*)take(sizeof(unsigned int) * kCaseBarStride * (size_t)max_cases);
  const size_t hbytes = sizeof(StageCase) * max_cases + sizeof(HelmBatchEntry) * max_cases +
                        sizeof(int) * (max_cases + 1) + sizeof(int) * b->blocks;
  if ((e = cudaMallocHost(&b->host_sums, sizeof(double) * 2 * max_cases)) != cudaSuccess ||
      (e = cudaMallocHost(&b->pinned, hbytes)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&b->tables_done, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaMemset(b->dev, 0, bytes)) != cudaSuccess) {
    cudaFree(b->dev);
    if (b->host_sums) cudaFreeHost(b->host_sums);
    if (b->pinned) cudaFreeHost(b->pinned);
    if (b->tables_done) cudaEventDestroy(b->tables_done);
    delete b;
    return bfail(CCM_E_CUDA, cudaGetErrorString(e));
  }
  {
    char* h = (char*)b->pinned;
    b->h_stages = (StageCase*)h;
    h += sizeof(StageCase) * max_cases;
    b->h_helm = (HelmBatchEntry*)h;
    h += sizeof(HelmBatchEntry) * max_cases;
    b->h_starts = (int*)h;
    h += sizeof(int) * (max_cases + 1);
    b->h_helm_block_case = (int*)h;
  }
  *out = b;
  return CCM_OK;
}

ccm_status ccm_batch_destroy(ccm_batch b) {
  if (!b) return CCM_OK;
  cudaStreamSynchronize(b->st);
  drop_graphs(b);
  if (b->cap_st) cudaStreamDestroy(b->cap_st);
  for (cudaEvent_t ev : b->tev)
    if (ev) cudaEventDestroy(ev);
  cudaFree(b->dev);
  cudaFreeHost(b->host_sums);
  cudaFreeHost(b->pinned);
  cudaEventDestroy(b->tables_done);
  delete b;
  return CCM_OK;
}

ccm_status ccm_batch_add(ccm_batch b, ccm_case c) {
  set_last_error("");
  if (!b || !c) return bfail(CCM_E_INVALID, "null argument");
  CaseSolveView v;
  if (!case_solve_view(c, &v)) return bfail(CCM_E_STATE, "set_geometry must come first");
  if (case_stream(c) != b->st) return bfail(CCM_E_INVALID, "the case must use the batch's stream");
  if (v.g.px || v.g.py) return bfail(CCM_E_INVALID, "periodic cases are not batched");
  if (case_is_moving(c)) return bfail(CCM_E_INVALID, "cases whose body velocity changes in time are not batched");
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
  StageRange range("ccm batch steps");
  if (!b) return bfail(CCM_E_INVALID, "null batch");
  if (nsteps < 0) return bfail(CCM_E_INVALID, "nsteps < 0");
  if (b->cases.empty()) return CCM_OK;
  for (ccm_case c : b->cases)
    if (case_is_moving(c)) return bfail(CCM_E_INVALID, "cases whose body velocity changes in time are not batched");
  const bool mixed = case_is_mixed(b->cases[0]);
  const bool scaled = all_scaled(b);
  // the split is tuned on the batch as it is; once the batch's cells have changed by more than
  // 30 % (cases joined or left, as in the request loop), it is tuned again
  if (b->tune) {
    double cells = 0.0;
    for (ccm_case c : b->cases) cells += (double)case_cells(c);
    if (b->tune_next == 0) {
      b->tune_cells = cells;
    } else if (std::fabs(cells - b->tune_cells) > 0.3 * b->tune_cells) {
      b->tune_next = 0;
      b->tune_cells = cells;
    }
  }
  ccm_status s;
  int n = 0;
  // a case's first step starts Adams-Bashforth and runs eagerly
  bool first = false;
  for (ccm_case c : b->cases) first = first || case_nstep(c) == 0;
  if (nsteps > 0 && first) {
    if ((s = eager_step(b, mixed, scaled)) != CCM_OK) return s;
    n = 1;
  }
  // the next steps try the candidate splits of the Poisson launch, one each
  for (; n < nsteps && scaled && b->tune && b->tune_next < kSplitN; ++n) {
    drop_graphs(b);
    if ((s = tuning_step(b, mixed)) != CCM_OK) return s;
  }
  if (n < nsteps && scaled && b->use_graphs) {
    bool ok = graphs_valid(b, mixed);
    if (!ok && (s = capture_graphs(b, mixed, &ok)) != CCM_OK) return s;
    if (ok) {
      for (; n < nsteps; ++n) {
        const cudaError_t e = cudaGraphLaunch(b->gexec[b->gphase], b->st);
        if (e != cudaSuccess) return bfail(CCM_E_CUDA, std::string("batch graph: ") + cudaGetErrorString(e));
        b->gphase ^= 1;
        b->graph_steps++;
        for (ccm_case c : b->cases) case_step_done(c);
      }
      if ((s = check_barrier(b, "batch graph")) != CCM_OK) return s;
    }
  }
  for (; n < nsteps; ++n)
    if ((s = eager_step(b, mixed, scaled)) != CCM_OK) return s;
  ccm_status worst = CCM_OK;
  for (size_t i = 0; i < b->cases.size(); ++i) {
    s = case_finish(b->cases[i], stats ? &stats[i] : nullptr);
    if (s != CCM_OK && worst == CCM_OK) worst = s;
  }
  return worst;
}

ccm_status ccm_batch_set_graphs(ccm_batch b, int enable) {
  set_last_error("");
  if (!b) return bfail(CCM_E_INVALID, "null batch");
  cudaStreamSynchronize(b->st);
  b->use_graphs = enable != 0;
  if (!b->use_graphs) drop_graphs(b);
  return CCM_OK;
}

ccm_status ccm_batch_set_tuning(ccm_batch b, int enable) {
  set_last_error("");
  if (!b) return bfail(CCM_E_INVALID, "null batch");
  b->tune = enable != 0;
  if (!b->tune && b->tune_next < kSplitN) b->split_exp = split_candidates[0];
  return CCM_OK;
}

ccm_status ccm_batch_split(ccm_batch b, double* exponent, int* tuned) {
  set_last_error("");
  if (!b || !exponent || !tuned) return bfail(CCM_E_INVALID, "null argument");
  *exponent = b->split_exp;
  *tuned = b->tune_next >= kSplitN ? 1 : 0;
  return CCM_OK;
}

ccm_status ccm_batch_graph_steps(ccm_batch b, long long* steps) {
  set_last_error("");
  if (!b || !steps) return bfail(CCM_E_INVALID, "null argument");
  *steps = b->graph_steps;
  return CCM_OK;
}

}  // extern "C"
