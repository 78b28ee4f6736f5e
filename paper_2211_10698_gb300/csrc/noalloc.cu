// Pressure solve that allocates nothing.
//
// Some callers cannot call cudaMalloc: a host framework that owns all device memory
// through its own pool and forbids other allocations, a process running under a hard
// device-memory cap, or latency-sensitive code that must not trigger the device-wide
// synchronisation that cudaMalloc and cudaFree imply.  ccm_solve_pressure_noalloc serves
// them: it solves the same system as ccm_solve_pressure in FP64 with the Jacobi
// preconditioner, whatever the case's precision and preconditioner settings, but its scratch
// vectors live in one file-scope __device__ array of fixed size instead of memory the
// library allocates.  Two kernels serve it: a case with an outflow side and the Jacobi
// setting runs CG on the Jacobi-scaled system in the two-barrier layout (k_pcg_poisson_sc,
// which needs fewer work vectors than the tiled one); a singular case (no outflow side,
// zero-mean iterates) or one configured for Chebyshev runs the unscaled Jacobi-PCG
// (k_pcg_poisson_cg with a degree-1 preconditioner).  The caller passes the right-hand side
// and the solution in device memory of its own.
//
// The array (about 6.4 MB) stays resident on every GPU that loads the library until the
// process exits.  Every call uses the same array, so calls that overlap on the GPU (from
// two streams or two threads) race; the array keeps the previous call's contents, so this
// file clears what must start at zero.  The first call on a device looks up the device
// address of the array once (cudaGetSymbolAddress with that device current); make that
// first call before any stream capture.
#include <math.h>
#include <stddef.h>

#include <mutex>
#include <string>

#include "ccm_host.h"

namespace {

using namespace ccm;

constexpr size_t kMaxElems = CCM_NOALLOC_MAX_ELEMS;
constexpr size_t kMaxPartials = 8192;
constexpr int kMaxDevices = 64;

struct Scratch {
  double b[kMaxElems];  // right-hand side restricted to active cells
  double r[kMaxElems];
  double u[kMaxElems];
  double w[kMaxElems];
  double p[kMaxElems];
  double s[kMaxElems];
  double partials[kMaxPartials];
  double rr, bb;
  int iters, converged;
  int bar_err, pad;
  unsigned int bar_count[kBarWords];
};

static __device__ __align__(256) Scratch g_scratch;

std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

__global__ void k_masked_copy(Geom g, const int8_t* act, const double* src, double* dst) {
  const int i = (int)(blockIdx.x * blockDim.x + threadIdx.x) - 1;
  const int j = (int)(blockIdx.y * blockDim.y + threadIdx.y) - 1;
  if (i > g.nx + 1 || j > g.ny + 1) return;
  const size_t k = g.idx(i, j);
  dst[k] = act[k] ? src[k] : 0.0;
}

__global__ void k_mask(Geom g, const int8_t* act, double* x) {
  const int i = (int)(blockIdx.x * blockDim.x + threadIdx.x) - 1;
  const int j = (int)(blockIdx.y * blockDim.y + threadIdx.y) - 1;
  if (i > g.nx + 1 || j > g.ny + 1) return;
  const size_t k = g.idx(i, j);
  if (!act[k]) x[k] = 0.0;
}

ccm_status fail(ccm_status s, const std::string& m) {
  set_last_error(m);
  return s;
}

// Device address of the scratch array on the current device (looked up once per device).
cudaError_t scratch_address(Scratch** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = ptr;
  }
  *out = (Scratch*)g_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" ccm_status ccm_solve_pressure_noalloc(ccm_case c, const double* rhs_dev, double* phi_dev,
                                                 ccm_solve_stats* stats) {
  set_last_error("");
  if (!c || !rhs_dev || !phi_dev) return fail(CCM_E_INVALID, "null argument");
  CaseSolveView v;
  if (!case_solve_view(c, &v)) return fail(CCM_E_STATE, "set_geometry must come first");
  if (v.g.px || v.g.py) return fail(CCM_E_INVALID, "periodic cases are not supported by this solve");
  const size_t n = v.g.count();
  if (n > kMaxElems)
    return fail(CCM_E_INVALID, "grid too large for the fixed scratch: (ny+3)*pitch = " + std::to_string(n) +
                                   " elements, the maximum is " + std::to_string(kMaxElems));
  if ((size_t)pcg_partials_needed() > kMaxPartials) return fail(CCM_E_INVALID, "too many multiprocessors");
  Scratch* S = nullptr;
  cudaError_t e = scratch_address(&S);
  if (e != cudaSuccess) return fail(CCM_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  cudaStream_t st = v.st;
  // the previous call's contents (possibly of another grid size): the first n elements of
  // every work vector are cleared, since the stencils read them on the ghost ring (a solve
  // of this grid touches nothing beyond them), and so are the barrier counter and its
  // error flag
  double* const work[5] = {S->r, S->u, S->w, S->p, S->s};
  for (double* a : work)
    if ((e = cudaMemsetAsync(a, 0, n * sizeof(double), st)) != cudaSuccess)
      return fail(CCM_E_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  if ((e = cudaMemsetAsync(&S->bar_err, 0, 2 * sizeof(int) + sizeof(unsigned int) * kBarWords, st)) != cudaSuccess)
    return fail(CCM_E_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  const dim3 blk(64, 4), grd((v.g.nx + 3 + 63) / 64, (v.g.ny + 3 + 3) / 4);
  k_masked_copy<<<grd, blk, 0, st>>>(v.g, v.act, rhs_dev, S->b);
  k_mask<<<grd, blk, 0, st>>>(v.g, v.act, phi_dev);
  if (!v.zero_mean && v.precond == CCM_JACOBI) {
    ScaledSolve q = scaled_solve_of(v, phi_dev, S->b, S->u, S->r, S->w, S->p, S->s);
    q.partials = S->partials;
    q.bar = Barrier{S->bar_count, &S->bar_err, 2000000000LL};
    q.out = PcgOut{&S->iters, &S->rr, &S->bb, &S->converged, nullptr, nullptr};
    e = run_poisson_scaled(q, st);
  } else {
    PoissonSolve<double> a{};
    a.g = v.g;
    a.cu = v.cu; a.cv = v.cv; a.dk = v.dk; a.invd = v.invd; a.kind = v.kind;
    a.creg_x = v.g.hy / v.g.hx;
    a.creg_y = v.g.hx / v.g.hy;
    a.dreg = 2.0 * (a.creg_x + a.creg_y);
    a.invd_reg = 1.0 / a.dreg;
    a.x = phi_dev; a.b = S->b; a.r = S->r; a.z = S->u; a.q = S->w; a.p0 = S->p; a.p1 = S->s;
    a.z2 = nullptr; a.w1 = nullptr;
    a.cheb = 1;
    a.tol = v.tol; a.max_iter = v.max_iter;
    a.zero_mean = v.zero_mean; a.n_act = v.n_act;
    a.partials = S->partials;
    a.bar = Barrier{S->bar_count, &S->bar_err, 2000000000LL};
    a.out = PcgOut{&S->iters, &S->rr, &S->bb, &S->converged, nullptr, nullptr};
    e = run_poisson_pcg<double>(a, st);
  }
  if (e != cudaSuccess)
    return fail(CCM_E_CUDA, std::string("Poisson PCG launch: ") + cudaGetErrorString(e));
  struct { double rr, bb; int iters, converged; int err, pad; } h{};
  static_assert(sizeof(h) == offsetof(Scratch, bar_count) - offsetof(Scratch, rr), "layout");
  if ((e = cudaMemcpyAsync(&h, &S->rr, sizeof(h), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return fail(CCM_E_CUDA, std::string("reading the solve statistics: ") + cudaGetErrorString(e));
  if (h.err) return fail(CCM_E_TIMEOUT, "a device-wide barrier gave up waiting");
  if (stats) {
    stats->iters = h.iters;
    stats->outer = 1;
    stats->rel_res = h.bb > 0 ? sqrt(h.rr / h.bb) : 0.0;
    stats->converged = h.converged;
  }
  if (!h.converged) return fail(CCM_E_NOT_CONVERGED, "Poisson PCG reached its iteration limit");
  return CCM_OK;
}
