// Request loop for flow-past-body solves (the serving form of the projection step; the paper
// runs one case at a time).  Built only on the public C API of include/ccm.h.
//
// Requests (a case configuration, a body and a number of steps) wait in a FIFO queue.  Each
// round of ccm_server_run
//   1. admits queued requests in arrival order while their device footprint fits the HBM
//      budget and a batch slot is free (continuous batching: requests join between rounds
//      while others are in flight),
//   2. advances every resident case by one chunk of steps through a batch (one batched
//      Poisson solve per step; FP64 and mixed-precision cases in separate batches),
//   3. retires the cases that reached their step count: their velocity and pressure fields
//      are copied to host memory and the case is destroyed, so a finished request holds no
//      device memory; statistics, timestamps and the host copies stay until
//      ccm_server_release.
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <chrono>
#include <deque>
#include <map>
#include <string>
#include <vector>

#include "ccm.h"

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

enum { Q_QUEUED = 0, Q_RUNNING = 1, Q_DONE = 2, Q_FAILED = 3 };

struct Request {
  long long id = 0;
  ccm_config cfg{};
  ccm_geometry geo{};
  int nsteps = 0;
  int done_steps = 0;
  int state = Q_QUEUED;
  size_t bytes = 0;
  ccm_case c = nullptr;
  ccm_step_stats st{};
  double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
  long long iters_p = 0, iters_h = 0;
  std::string error;
  std::vector<double> saved[3];  // U, V, P of a finished request (padded layout)
  std::vector<double> xf, yf;    // copies of a stretched mesh's face abscissas
};

constexpr int kSavedFields[3] = {CCM_F_U, CCM_F_V, CCM_F_P};

}  // namespace

struct ccm_server_s {
  size_t budget = 0, used = 0;
  int max_batch = 0;
  int chunk = 0;
  void* stream = nullptr;
  ccm_batch batch[2] = {nullptr, nullptr};  // FP64, MIXED
  std::vector<Request*> members[2];         // each batch's cases, in the order they joined
  std::deque<Request*> queue;
  std::map<long long, Request*> all;
  long long next_id = 1;
};

// Copy the result fields to the host and free the case's device memory.
static ccm_status retire(ccm_server_s* s, Request* r, int state, double t) {
  ccm_status st = CCM_OK;
  if (r->c) {
    const size_t n = (size_t)(r->cfg.nx + 3) * (size_t)(r->cfg.ny + 3);
    for (int f = 0; f < 3; ++f) {
      r->saved[f].resize(n);
      ccm_status e = ccm_get_field(r->c, kSavedFields[f], r->saved[f].data(), n);
      if (e != CCM_OK && st == CCM_OK) st = e;
    }
    ccm_destroy_case(r->c);
    r->c = nullptr;
    s->used -= r->bytes;
  }
  r->state = st == CCM_OK ? state : Q_FAILED;
  r->t_done = t;
  return st;
}

extern "C" {

ccm_status ccm_server_create(size_t hbm_budget_bytes, int max_batch, int chunk_steps, void* stream, ccm_server* out) {
  if (!out || hbm_budget_bytes == 0 || max_batch < 1 || chunk_steps < 1) return CCM_E_INVALID;
  ccm_server s = new ccm_server_s();
  s->budget = hbm_budget_bytes;
  s->max_batch = max_batch;
  s->chunk = chunk_steps;
  s->stream = stream;
  for (int k = 0; k < 2; ++k) {
    ccm_status st = ccm_batch_create(max_batch, stream, &s->batch[k]);
    if (st != CCM_OK) {
      if (s->batch[0]) ccm_batch_destroy(s->batch[0]);
      delete s;
      return st;
    }
  }
  *out = s;
  return CCM_OK;
}

ccm_status ccm_server_destroy(ccm_server s) {
  if (!s) return CCM_OK;
  for (auto& kv : s->all) {
    Request* r = kv.second;
    if (r->c) ccm_destroy_case(r->c);
    delete r;
  }
  for (int k = 0; k < 2; ++k) ccm_batch_destroy(s->batch[k]);
  delete s;
  return CCM_OK;
}

ccm_status ccm_server_submit(ccm_server s, const ccm_config* cfg, const ccm_geometry* geo, int nsteps, long long* id) {
  if (!s || !cfg || !geo || !id || nsteps < 0) return CCM_E_INVALID;
  for (int q = 0; q < 4; ++q)
    if (cfg->bc_type[q] == CCM_BC_PERIODIC) return CCM_E_INVALID;  // requests advance in batches
  Request* r = new Request();
  r->id = s->next_id++;
  r->cfg = *cfg;
  // a stretched mesh's abscissas are the caller's: the request keeps its own copies
  if (cfg->xf) r->xf.assign(cfg->xf, cfg->xf + cfg->nx + 1);
  if (cfg->yf) r->yf.assign(cfg->yf, cfg->yf + cfg->ny + 1);
  r->cfg.xf = cfg->xf ? r->xf.data() : nullptr;
  r->cfg.yf = cfg->yf ? r->yf.data() : nullptr;
  r->cfg.stream = s->stream;
  r->cfg.autotune = 0;  // requests advance in batches, which do not use the single-case launch plan
  r->geo = *geo;
  r->nsteps = nsteps;
  r->t_submit = now_s();
  ccm_status st = ccm_case_bytes(&r->cfg, &r->bytes);
  if (st != CCM_OK) {
    delete r;
    return st;
  }
  if (r->bytes > s->budget) {
    delete r;
    return CCM_E_OOM;
  }
  s->all[r->id] = r;
  s->queue.push_back(r);
  *id = r->id;
  return CCM_OK;
}

// One admission + one chunk of steps + retirement.  *active receives the number of requests
// queued or running afterwards.
ccm_status ccm_server_run(ccm_server s, int rounds, int* active) {
  if (!s || rounds < 0) return CCM_E_INVALID;
  ccm_status worst = CCM_OK;
  for (int round = 0; round < rounds; ++round) {
    nvtxRangePushA("ccm server round");  // popped at the end of the round
    // admission, in arrival order (a request that does not fit blocks the ones behind it)
    while (!s->queue.empty()) {
      Request* r = s->queue.front();
      const int k = r->cfg.precision == CCM_MIXED ? 1 : 0;
      if (s->used + r->bytes > s->budget || ccm_batch_size(s->batch[k]) >= s->max_batch) break;
      s->queue.pop_front();
      ccm_status st = ccm_create_case(&r->cfg, &r->c);
      if (st == CCM_OK) st = ccm_set_geometry(r->c, &r->geo);
      if (st == CCM_OK) st = ccm_batch_add(s->batch[k], r->c);
      if (st == CCM_OK) s->members[k].push_back(r);
      if (st != CCM_OK) {
        r->state = Q_FAILED;
        r->error = ccm_last_error();
        if (r->c) ccm_destroy_case(r->c);
        r->c = nullptr;
        r->t_done = now_s();
        continue;
      }
      s->used += r->bytes;
      r->state = Q_RUNNING;
      r->t_admit = now_s();
      if (r->nsteps == 0) {
        ccm_batch_remove(s->batch[k], r->c);
        s->members[k].pop_back();
        retire(s, r, Q_DONE, r->t_admit);
      }
    }
    // resident requests of each batch advance by the smallest remaining count, capped at chunk
    for (int k = 0; k < 2; ++k) {
      std::vector<Request*>& order = s->members[k];  // the batch reports stats in this order
      if (order.empty()) continue;
      int n = s->chunk;
      for (Request* r : order) n = std::min(n, r->nsteps - r->done_steps);
      std::vector<ccm_step_stats> st(order.size());
      ccm_status rc = ccm_batch_step(s->batch[k], n, st.data());
      if (rc != CCM_OK && rc != CCM_E_NOT_CONVERGED && worst == CCM_OK) worst = rc;
      for (size_t i = 0; i < order.size(); ++i) {
        Request* r = order[i];
        r->done_steps += n;
        r->st = st[i];
        r->iters_p += st[i].iters_p;
        r->iters_h += st[i].iters_h;
      }
      const double t = now_s();
      std::vector<Request*> keep;
      for (Request* r : order) {
        if (r->done_steps >= r->nsteps) {
          ccm_batch_remove(s->batch[k], r->c);
          retire(s, r, rc == CCM_OK || rc == CCM_E_NOT_CONVERGED ? Q_DONE : Q_FAILED, t);
        } else {
          keep.push_back(r);
        }
      }
      order.swap(keep);
    }
    nvtxRangePop();
  }
  if (active) {
    int a = (int)s->queue.size();
    for (auto& kv : s->all) a += kv.second->state == Q_RUNNING;
    *active = a;
  }
  return worst;
}

// State of a request: 0 queued, 1 running, 2 done, 3 failed; times are seconds on a
// monotonic clock (submit, admit, done); stats holds the last step's statistics with the
// iteration counts summed over all steps.
ccm_status ccm_server_poll(ccm_server s, long long id, int* state, double* times3, ccm_step_stats* stats) {
  if (!s) return CCM_E_INVALID;
  auto it = s->all.find(id);
  if (it == s->all.end()) return CCM_E_INVALID;
  Request* r = it->second;
  if (state) *state = r->state;
  if (times3) {
    times3[0] = r->t_submit;
    times3[1] = r->t_admit;
    times3[2] = r->t_done;
  }
  if (stats) {
    *stats = r->st;
    stats->steps = r->done_steps;
    stats->iters_p = r->iters_p;
    stats->iters_h = r->iters_h;
  }
  return CCM_OK;
}

// Copy a field to the host: any field of a running request (see ccm_get_field), U, V or P
// of a finished one.
ccm_status ccm_server_get_field(ccm_server s, long long id, int field, double* host, size_t count) {
  if (!s || !host) return CCM_E_INVALID;
  auto it = s->all.find(id);
  if (it == s->all.end()) return CCM_E_INVALID;
  Request* r = it->second;
  if (r->c) return ccm_get_field(r->c, field, host, count);
  for (int f = 0; f < 3; ++f)
    if (field == kSavedFields[f] && !r->saved[f].empty()) {
      if (count != r->saved[f].size()) return CCM_E_INVALID;
      std::copy(r->saved[f].begin(), r->saved[f].end(), host);
      return CCM_OK;
    }
  return CCM_E_INVALID;
}

// Free the request's device memory and forget it.
ccm_status ccm_server_release(ccm_server s, long long id) {
  if (!s) return CCM_E_INVALID;
  auto it = s->all.find(id);
  if (it == s->all.end()) return CCM_E_INVALID;
  Request* r = it->second;
  if (r->state == Q_RUNNING) return CCM_E_STATE;
  if (r->state == Q_QUEUED) s->queue.erase(std::find(s->queue.begin(), s->queue.end(), r));
  if (r->c) {
    ccm_destroy_case(r->c);
    s->used -= r->bytes;
  }
  delete r;
  s->all.erase(it);
  return CCM_OK;
}

size_t ccm_server_bytes_in_use(ccm_server s) { return s ? s->used : 0; }

}  // extern "C"
