// C ABI of libccm (include/ccm.h): case lifecycle, set-up from the body geometry, field
// exchange, single-operator application, the PmII step (Sec. 4.6) and the pressure solve.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <string>
#include <vector>

#include "ccm_host.h"

using namespace ccm;

namespace {

thread_local std::string g_last_error;

// clock64 cycles a block of a cooperative launch waits at a device-wide barrier before it
// gives up (about one second at 2 GHz)
constexpr long long kBarrierBudget = 2000000000LL;

ccm_status fail(ccm_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

#define CUDA_TRY(expr)                                                                      \
  do {                                                                                      \
    cudaError_t e_ = (expr);                                                                \
    if (e_ != cudaSuccess) return fail(CCM_E_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

struct DevStats {
  long long total_p, total_h;
  int iters_p, iters_h;
  double rr_p, bb_p, rr_h, bb_h;
  int conv_p, conv_h;
  int nconv;
  int nrep;        // FP64 residual replacements of the last mixed solve on the device
  double diag[6];  // max |cont|, kinetic, non-finite flag, mass, momentum x, momentum y
};

}  // namespace

struct ccm_case_s {
  ccm_config cfg;
  Geom g;
  Bc bc;
  Phys ph;
  cudaStream_t st;
  void* slab = nullptr;
  size_t slab_bytes = 0;
  CapPtrs caps;
  CoefPtrs co;
  Coefs cv;
  // state
  double *u, *v, *p, *phi, *cnu[2], *cnv[2];
  int cur = 0;
  long long nstep = 0;
  // step work
  double *ustar, *vstar, *div, *rhs_u, *rhs_v, *rhs_p;
  double *pr, *pz, *pp0, *pp1, *pq, *pz2, *pw1;
  double *hr_u, *hr_v, *hz_u, *hz_v, *hp_u, *hp_v, *hq_u, *hq_v;
  double *hs_u, *hs_v;     // K p of the Helmholtz CG
  HelmCoefPtrs hc;         // the Helmholtz operator, nine coefficients per unknown face
  int* hc_bad;             // set when probing finds a coupling outside that pattern
  float *fx, *fb, *fr, *fz, *fp0, *fp1, *fq, *fz2, *fw1;
  double* mixed_sums;
  double *t0, *t1, *t2, *t3, *t4, *t5;
  double* partials;
  double* dpart;
  unsigned int* bar_count;
  unsigned long long* fxacc;  // words of the fixed-point reduce-barrier (pcg_fixed.cuh)
  int* bar_err;
  DevStats* ds;
  bool geometry = false;
  double n_act = 0.0;
  int zero_mean = 0;
  // timing of the Poisson PCG launches (events recorded on the case's stream)
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  long long launches = 0, poisson_launches = 0;
  long long poisson_iters_timed = 0;
  double poisson_ms = 0.0;
  long long steps_pending = 0;
  // statistics of mixed-precision solves (accumulated on the host)
  long long mixed_total = 0;
  int mixed_last = 0, mixed_outer = 0, mixed_nconv = 0;
  double mixed_rr = 0.0, mixed_bb = 0.0;
  bool mixed_host = false;  // a host-driven refinement ran since the statistics were last read
  TuneResult tune{};        // launch shape of the one-launch Poisson solve (zero: built-in)
  unsigned long long serial = 0;  // unique per case for the life of the process
  // force on the body: block partials and the last value; optional per-step record (a ring of
  // fcap rows of four doubles, allocated on demand; frec steps recorded so far)
  double* fpart = nullptr;
  double* fout = nullptr;
  // body acceleration g at u- and v-faces (zero until set; the predictor reads it once set)
  double *accx = nullptr, *accy = nullptr;
  bool forced = false;
  // the body's Dirichlet velocity D and its constant terms: one allocation of 8 padded arrays,
  // made when D is first set (Dx, Dy, h, S_xx, S_yy, S_xy, visc_u, visc_v)
  double* dblock = nullptr;
  // time law of the body velocity, D(t) = D0 (a0 + a1 sin(omega t + phase)) at t = n dt with D0
  // the field in dblock; steady (D = D0) unless ccm_set_body_motion made it otherwise
  bool moving = false;
  double motion[4] = {1.0, 0.0, 0.0, 0.0};
  double* fhist = nullptr;
  int fcap = 0;
  long long frec = 0;
  // device-wide barriers of the case's cooperative launches: the spin budget, and the block
  // that skips its arrivals (failure-detection tests only; -1 otherwise)
  long long bar_budget = kBarrierBudget;
  int bar_absent = -1;
  // tests only: every k-th fixed-point reduction of the FP64 one-barrier CG takes its FP64
  // fallback (0: only when a value leaves the window)
  int fx_fallback_every = 0;
  // stretched mesh: the face abscissas extended two faces beyond the box (host copies, and
  // their device arrays in the slab); empty for a uniform spacing
  std::vector<double> xfx, yfx;
  double *xfd = nullptr, *yfd = nullptr;
  // projected initial guess of the Poisson solve: K-orthonormal basis X (guess_history padded
  // arrays), its images KX, scratch for the sums (one allocation, made at the first step);
  // gnb vectors in use
  double* gmem = nullptr;
  int gnb = 0;
};

namespace {

Barrier case_barrier(ccm_case c) {
  Barrier b{c->bar_count, c->bar_err, c->bar_budget};
  b.absent = c->bar_absent;
  return b;
}

struct Carver {
  char* base;
  size_t off = 0;
  template <class T>
  T* take(size_t n) {
    off = (off + 255) & ~(size_t)255;
    T* p = base ? (T*)(base + off) : nullptr;
    off += n * sizeof(T);
    return p;
  }
};

void carve(ccm_case c, Carver& cv) {
  const size_t N = c->g.count();
  for (int s = 0; s < 27; ++s) c->caps.a[s] = cv.take<double>(N);
  CoefPtrs& o = c->co;
  o.role_u = cv.take<int8_t>(N);
  o.role_v = cv.take<int8_t>(N);
  o.act = cv.take<int8_t>(N);
  o.kind = cv.take<int8_t>(N);
  double** dd[] = {&o.cu, &o.cv, &o.invdk, &o.diagk, &o.gfu, &o.gfv, &o.pfac, &o.massu, &o.massv, &o.wxx, &o.wyy,
                   &o.wxa, &o.wxb, &o.invdhu, &o.invdhv, &o.liftu, &o.liftv};
  for (double** p : dd) *p = cv.take<double>(N);
  o.cu32 = cv.take<float>(N);
  o.cv32 = cv.take<float>(N);
  o.invdk32 = cv.take<float>(N);
  o.diagk32 = cv.take<float>(N);
  for (double** q : {&o.sdk, &o.isdk, &o.cus, &o.cvs}) *q = cv.take<double>(N);
  for (float** q : {&o.isdk32, &o.cus32, &o.cvs32}) *q = cv.take<float>(N);
  o.kinds = cv.take<int8_t>(N);
  double** st[] = {&c->u, &c->v, &c->p, &c->phi, &c->cnu[0], &c->cnu[1], &c->cnv[0], &c->cnv[1],
                   &c->ustar, &c->vstar, &c->div, &c->rhs_u, &c->rhs_v, &c->rhs_p,
                   &c->pr, &c->pz, &c->pp0, &c->pp1, &c->pq, &c->pz2, &c->pw1,
                   &c->hr_u, &c->hr_v, &c->hz_u, &c->hz_v, &c->hp_u, &c->hp_v, &c->hq_u, &c->hq_v,
                   &c->t0, &c->t1, &c->t2, &c->t3, &c->t4, &c->t5};
  for (double** p : st) *p = cv.take<double>(N);
  float** fl[] = {&c->fx, &c->fb, &c->fr, &c->fz, &c->fp0, &c->fp1, &c->fq, &c->fz2, &c->fw1};
  for (float** p : fl) *p = cv.take<float>(N);
  c->mixed_sums = cv.take<double>(4);
  c->partials = cv.take<double>((size_t)pcg_partials_needed());
  c->dpart = cv.take<double>((size_t)6 * diagnostics_partials(c->g) + 8);
  c->fpart = cv.take<double>((size_t)body_force_partials(c->g));
  c->accx = cv.take<double>(N);
  c->accy = cv.take<double>(N);
  c->fout = cv.take<double>(4);
  c->bar_count = cv.take<unsigned int>(kBarWords);
  c->fxacc = cv.take<unsigned long long>(kFxAccWords);
  c->bar_err = cv.take<int>(4);
  c->ds = cv.take<DevStats>(1);
  c->hs_u = cv.take<double>(N);
  c->hs_v = cv.take<double>(N);
  c->xfd = cv.take<double>((size_t)c->g.nx + 7);
  c->yfd = cv.take<double>((size_t)c->g.ny + 7);
  for (int q = 0; q < 18; ++q) c->hc.a[q] = cv.take<double>(N);
  c->hc_bad = cv.take<int>(4);
}

void make_view(ccm_case c) {
  const CoefPtrs& o = c->co;
  Coefs& v = c->cv;
  v.role_u = o.role_u; v.role_v = o.role_v; v.act = o.act;
  v.ax = c->caps.a[cap_slot(0, CK_AX)];
  v.ay = c->caps.a[cap_slot(0, CK_AY)];
  v.bxx = c->caps.a[cap_slot(1, CK_BX)];
  v.bxy = c->caps.a[cap_slot(1, CK_BY)];
  v.byx = c->caps.a[cap_slot(2, CK_BX)];
  v.byy = c->caps.a[cap_slot(2, CK_BY)];
  v.wxx = o.wxx; v.wyy = o.wyy; v.wxa = o.wxa; v.wxb = o.wxb;
  v.cu = o.cu; v.cv = o.cv; v.invdk = o.invdk;
  v.gfu = o.gfu; v.gfv = o.gfv; v.pfac = o.pfac;
  v.massu = o.massu; v.massv = o.massv;
  v.invdhu = o.invdhu; v.invdhv = o.invdhv;
  v.liftu = o.liftu; v.liftv = o.liftv;
  v.accx = c->forced ? c->accx : nullptr;
  v.accy = c->forced ? c->accy : nullptr;
  const size_t N = c->g.count();
  double* d = c->dblock;
  v.dx = d; v.dy = d ? d + N : nullptr; v.hd = d ? d + 2 * N : nullptr;
  v.sxxd = d ? d + 3 * N : nullptr; v.syyd = d ? d + 4 * N : nullptr; v.sxyd = d ? d + 5 * N : nullptr;
  v.viscdu = d ? d + 6 * N : nullptr; v.viscdv = d ? d + 7 * N : nullptr;
  v.cu32 = o.cu32; v.cv32 = o.cv32; v.invdk32 = o.invdk32;
}

size_t host_count(ccm_case c) { return (size_t)(c->g.nx + 3) * (size_t)(c->g.ny + 3); }

ccm_status upload(ccm_case c, double* dst, const double* host) {
  CUDA_TRY(cudaMemcpy2DAsync(dst, (size_t)c->g.pitch * sizeof(double), host, (size_t)(c->g.nx + 3) * sizeof(double),
                             (size_t)(c->g.nx + 3) * sizeof(double), (size_t)(c->g.ny + 3), cudaMemcpyHostToDevice,
                             c->st));
  return CCM_OK;
}

ccm_status download(ccm_case c, double* host, const double* src) {
  CUDA_TRY(cudaMemcpy2DAsync(host, (size_t)(c->g.nx + 3) * sizeof(double), src, (size_t)c->g.pitch * sizeof(double),
                             (size_t)(c->g.nx + 3) * sizeof(double), (size_t)(c->g.ny + 3), cudaMemcpyDeviceToHost,
                             c->st));
  return CCM_OK;
}

__global__ void k_init_velocity(Geom g, const int8_t* ru, double u0, double* u, double* v) {
  const int i = (int)(blockIdx.x * blockDim.x + threadIdx.x) - 1;
  const int j = (int)(blockIdx.y * blockDim.y + threadIdx.y) - 1;
  if (i > g.nx + 1 || j > g.ny + 1) return;
  const size_t k = g.idx(i, j);
  u[k] = ru[k] == R_UNKNOWN ? u0 : 0.0;
  v[k] = 0.0;
}

// Zero the velocity positions that are not unknowns or Dirichlet faces' neighbours of the
// fill (inactive faces hold zero).
__global__ void k_mask_cells(Geom g, const int8_t* act, double* x) {
  const int i = (int)(blockIdx.x * blockDim.x + threadIdx.x) - 1;
  const int j = (int)(blockIdx.y * blockDim.y + threadIdx.y) - 1;
  if (i > g.nx + 1 || j > g.ny + 1) return;
  const size_t k = g.idx(i, j);
  if (!act[k]) x[k] = 0.0;
}

dim3 grid_of(const Geom& g, dim3 b) { return dim3((g.nx + 3 + b.x - 1) / b.x, (g.ny + 3 + b.y - 1) / b.y); }

// Conservative bounding box of the body, to check the two-cell margin to the box sides.
void body_bbox(const ccm_geometry& geo, double& xa, double& xb, double& ya, double& yb) {
  if (geo.kind == CCM_GEOM_CIRCLE) {
    xa = geo.cx - geo.r; xb = geo.cx + geo.r; ya = geo.cy - geo.r; yb = geo.cy + geo.r;
    return;
  }
  double a = geo.aoa_deg * (M_PI / 180.0), ca = cos(a), sa = sin(a);
  double t = geo.naca_tt / 100.0;
  xa = ya = 1e300; xb = yb = -1e300;
  for (int s = 0; s <= 2000; ++s) {
    double xi = s / 2000.0;
    const double x2 = xi * xi;
    double yt = 5.0 * t * (0.2969 * sqrt(xi) - 0.1260 * xi - 0.3516 * x2 + 0.2843 * x2 * xi - 0.1036 * x2 * x2);
    for (int sg = -1; sg <= 1; sg += 2) {
      double eta = sg * (yt + 1e-3);
      // inverse rotation of (xi, eta) * chord
      double px = geo.chord * (xi * ca + eta * sa), py = geo.chord * (-xi * sa + eta * ca);
      double X = geo.le_x + px, Y = geo.le_y + py;
      xa = fmin(xa, X); xb = fmax(xb, X); ya = fmin(ya, Y); yb = fmax(yb, Y);
    }
  }
}

ccm_status check_cuda_errors(const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(CCM_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
  return CCM_OK;
}

// Face coefficients of an uncut cell, A^2/V = hy/hx (x faces) and hx/hy (y faces).
template <class T>
void set_uniform_coefficients(ccm_case c, PoissonSolve<T>& a) {
  a.creg_x = c->g.hy / c->g.hx;
  a.creg_y = c->g.hx / c->g.hy;
  a.dreg = 2.0 * (a.creg_x + a.creg_y);
  a.invd_reg = 1.0 / a.dreg;
}

ccm_status solve_poisson_fp64(ccm_case c, double* x, double* b) {
  if (!c->zero_mean && c->cfg.precond == CCM_JACOBI && !c->g.px && !c->g.py) {
    // Jacobi-PCG as CG on the symmetrically scaled system (nonsingular systems)
    // with one grid barrier per iteration (tiles that recompute their ring)
    CaseSolveView v;
    case_solve_view(c, &v);
    FusedSolve f{};
    f.a = scaled_solve_of(v, x, b, c->pz, nullptr, nullptr, c->pp0, nullptr);
    f.fxacc = c->fxacc;
    f.fx_fallback_every = c->fx_fallback_every;
    f.a.partials = c->partials;
    f.a.bar = case_barrier(c);
    f.a.out = PcgOut{&c->ds->iters_p, &c->ds->rr_p, &c->ds->bb_p, &c->ds->conv_p, &c->ds->total_p, &c->ds->nconv};
    f.R[0] = c->pr; f.R[1] = c->pz2;
    f.W[0] = c->pq; f.W[1] = c->pw1;
    f.S[0] = c->pp1; f.S[1] = c->t5;
    if (c->tune.cluster > 0) {
      // small grid: the whole solve inside one thread-block cluster
      ClusterSolve cs{};
      cs.a = f.a;
      CUDA_TRY(run_poisson_cluster(cs, c->tune.cluster, c->st));
      return CCM_OK;
    }
    const TilePlan& tp = c->tune.plan;
    f.TX = tp.TX; f.TY = tp.TY; f.nbx = tp.nbx; f.ntiles = tp.ntiles; f.resident = tp.resident;
    CUDA_TRY(run_poisson_fused(f, c->st));
    return CCM_OK;
  }
  PoissonSolve<double> a{};
  a.g = c->g;
  a.cu = c->co.cu; a.cv = c->co.cv; a.dk = c->co.diagk; a.invd = c->co.invdk; a.kind = c->co.kind;
  set_uniform_coefficients(c, a);
  a.x = x; a.b = b; a.r = c->pr; a.z = c->pz; a.p0 = c->pp0; a.p1 = c->pp1; a.q = c->pq;
  a.z2 = c->pz2; a.w1 = c->pw1;
  a.cheb = c->cfg.precond == CCM_CHEBYSHEV ? c->cfg.cheb_degree : 1;
  a.tol = c->cfg.tol_p; a.max_iter = c->cfg.max_iter_p;
  a.zero_mean = c->zero_mean; a.n_act = c->n_act;
  a.partials = c->partials;
  a.bar = case_barrier(c);
  a.out = PcgOut{&c->ds->iters_p, &c->ds->rr_p, &c->ds->bb_p, &c->ds->conv_p, &c->ds->total_p, &c->ds->nconv};
  CUDA_TRY(run_poisson_pcg<double>(a, c->st));
  return CCM_OK;
}

// The CN Helmholtz solve of the predictor (Eq. pm_prediction) on the probed coefficients.
void helm_solve_of(ccm_case c, HelmCSolve* out) {
  HelmCSolve a{};
  a.g = c->g;
  a.ru = c->co.role_u; a.rv = c->co.role_v;
  a.h = c->hc;
  a.invu = c->co.invdhu; a.invv = c->co.invdhv;
  a.xu = c->u; a.xv = c->v; a.bu = c->rhs_u; a.bv = c->rhs_v;
  a.rU = c->hr_u; a.rV = c->hr_v; a.zU = c->hz_u; a.zV = c->hz_v; a.wU = c->hq_u; a.wV = c->hq_v;
  a.pU = c->hp_u; a.pV = c->hp_v; a.sU = c->hs_u; a.sV = c->hs_v;
  a.tol = c->cfg.tol_h; a.max_iter = c->cfg.max_iter_h;
  a.partials = c->partials;
  a.bar = case_barrier(c);
  a.out = PcgOut{&c->ds->iters_h, &c->ds->rr_h, &c->ds->bb_h, &c->ds->conv_h, &c->ds->total_h, &c->ds->nconv};
  *out = a;
}

ccm_status solve_helmholtz(ccm_case c) {
  HelmCSolve a{};
  helm_solve_of(c, &a);
  CUDA_TRY(run_helmholtz_coef(a, c->st));
  return CCM_OK;
}

cudaEvent_t next_event(ccm_case c) {
  if (c->ev_used == c->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    c->ev_pool.push_back(e);
  }
  return c->ev_pool[c->ev_used++];
}

// Mixed precision: FP64 residual, FP32 PCG on the correction equation K d = r to tol_inner,
// x += d, until the FP64 residual meets tol_p (or 60 refinement sweeps).
// The one-launch mixed solve of a case (x = solution in/out, b = right-hand side).
void case_mixed_solve(ccm_case c, double* x, const double* b, MixedSolve* a) {
  CaseSolveView v;
  case_solve_view(c, &v);
  *a = MixedSolve{};
  a->d = scaled_solve_of(v, x, b, nullptr, c->pr, nullptr, nullptr, nullptr);
  a->d.partials = c->partials;
  a->d.bar = case_barrier(c);
  a->d.out = PcgOut{&c->ds->iters_p, &c->ds->rr_p, &c->ds->bb_p, &c->ds->conv_p, &c->ds->total_p, &c->ds->nconv};
  a->cus32 = c->co.cus32; a->cvs32 = c->co.cvs32;
  a->r = c->fr; a->w = c->fq; a->p = c->fp0; a->s = c->fp1; a->e = c->fx;
  a->cheb = c->cfg.precond == CCM_CHEBYSHEV ? c->cfg.cheb_degree : 1;
  a->zA = c->fz2; a->zB = c->fw1; a->dch = c->fb;
  a->fpartials = (float*)(c->partials + pcg_float_partials_offset());
  a->drop = c->cfg.replace_drop > 0 && c->cfg.replace_drop < 1 ? c->cfg.replace_drop : 0.5;
  a->replacements = &c->ds->nrep;
  a->blocks = c->tune.mixed_blocks;
}

// The one-barrier form of the same solve (pcg_mixed1.cu) on the case's FP32 work arrays.
void case_mixed1_solve(ccm_case c, const MixedSolve& a, const TilePlan& tp, Mixed1Solve* f) {
  *f = Mixed1Solve{};
  f->m = a;
  f->R[0] = c->fr; f->R[1] = c->fz;
  f->W[0] = c->fq; f->W[1] = c->fz2;
  f->S[0] = c->fp1; f->S[1] = c->fw1;
  f->P = c->fp0; f->U = c->fb; f->E = c->fx;
  f->TX = tp.TX; f->TY = tp.TY; f->nbx = tp.nbx; f->ntiles = tp.ntiles;
  f->resident = tp.resident;
}

ccm_status solve_poisson_mixed(ccm_case c, double* x, double* b) {
  // periodic sides: the host-driven refinement on the general kernel, which writes the images
  if (!c->zero_mean && !c->g.px && !c->g.py) {
    // one launch: FP32 CG on the scaled system with FP64 residual replacements (Jacobi or
    // Chebyshev preconditioner), with one grid barrier per iteration when the tuner chose it
    MixedSolve a{};
    case_mixed_solve(c, x, b, &a);
    if (c->tune.mixed1.TX > 0) {
      Mixed1Solve f{};
      case_mixed1_solve(c, a, c->tune.mixed1, &f);
      CUDA_TRY(run_poisson_mixed1(f, c->st));
    } else {
      CUDA_TRY(run_poisson_mixed(a, c->st));
    }
    c->launches += 1;
    return CCM_OK;
  }
  c->mixed_host = true;
  const Geom& g = c->g;
  cudaStream_t st = c->st;
  int inner_total = 0, outer = 0;
  double sums[2] = {0.0, 0.0};
  bool conv = false;
  // singular system: warm start and right-hand side projected onto zero mean in FP64, as
  // the FP64 solve does (the FP32 corrections are zero-mean only to FP32 rounding, so the
  // result is projected again at the end)
  CUDA_TRY(project_zero_mean(g, c->co.act, x, c->partials, (double)c->n_act, st));
  CUDA_TRY(project_zero_mean(g, c->co.act, b, c->partials, (double)c->n_act, st));
  launch_wrap_cells(g, x, st);  // periodic sides: the residual's stencil reads x's images
  for (; outer < 60; ++outer) {
    launch_residual64(c->cv, g, x, b, c->fb, c->dpart, c->mixed_sums, st);
    CUDA_TRY(cudaMemcpyAsync(sums, c->mixed_sums, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (sums[1] == 0.0 || sums[0] <= c->cfg.tol_p * c->cfg.tol_p * sums[1]) { conv = true; break; }
    CUDA_TRY(cudaMemsetAsync(c->fx, 0, g.count() * sizeof(float), st));
    PoissonSolve<float> a{};
    a.g = g;
    a.cu = c->co.cu32; a.cv = c->co.cv32; a.dk = c->co.diagk32; a.invd = c->co.invdk32; a.kind = c->co.kind;
    set_uniform_coefficients(c, a);
    a.x = c->fx; a.b = c->fb; a.r = c->fr; a.z = c->fz; a.p0 = c->fp0; a.p1 = c->fp1; a.q = c->fq;
    a.z2 = c->fz2; a.w1 = c->fw1;
    a.cheb = c->cfg.precond == CCM_CHEBYSHEV ? c->cfg.cheb_degree : 1;
    a.tol = c->cfg.tol_inner > 0 ? c->cfg.tol_inner : 1e-5;
    a.max_iter = c->cfg.max_iter_p;
    a.zero_mean = c->zero_mean; a.n_act = c->n_act;
    a.partials = c->partials;
    a.bar = case_barrier(c);
    a.out = PcgOut{&c->ds->iters_p, &c->ds->rr_p, &c->ds->bb_p, &c->ds->conv_p, nullptr, nullptr};
    CUDA_TRY(run_poisson_pcg<float>(a, st));
    c->launches += 1 + (c->zero_mean ? 4 : 0);
    int it = 0;
    CUDA_TRY(cudaMemcpyAsync(&it, &c->ds->iters_p, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    inner_total += it;
    launch_add_correction(g, c->co.act, x, c->fx, st);
    launch_wrap_cells(g, x, st);
    c->launches += 3;
  }
  CUDA_TRY(project_zero_mean(g, c->co.act, x, c->partials, (double)c->n_act, st));
  c->launches += 8;
  c->mixed_total += inner_total;
  c->mixed_last = inner_total;
  c->mixed_outer = outer;
  c->mixed_rr = sums[0];
  c->mixed_bb = sums[1];
  if (!conv) c->mixed_nconv++;
  return check_cuda_errors("mixed Poisson solve");
}

// Launch-shape autotuning of the one-launch Poisson solve, at set-up (see tune.cu): every
// candidate runs kTuneIters iterations of the case's own solve (tolerance 0, so all do the
// same work) from x = 0 on a positive constant right-hand side.  x and b are the copies U*
// and V* of the predicted velocity, outputs of each step and free at set-up; the statistics
// the runs leave are cleared.
constexpr int kTuneIters = 24;

ccm_status autotune_poisson(ccm_case c) {
  if (!c->cfg.autotune || c->zero_mean || c->g.px || c->g.py) return CCM_OK;
  const bool mixed = c->cfg.precision == CCM_MIXED;
  if (!mixed && c->cfg.precond != CCM_JACOBI) return CCM_OK;  // FP64 Chebyshev: no plan to choose
  const Geom& g = c->g;
  cudaStream_t st = c->st;
  const int most = mixed ? mixed_blocks() : fused_blocks();
  const int deg = c->cfg.precond == CCM_CHEBYSHEV ? c->cfg.cheb_degree : 1;
  TuneResult r{};
  if (tune_cache_get(g.nx, g.ny, c->cfg.precision, c->cfg.precond, deg, most, &r)) {
    c->tune = r;
    return CCM_OK;
  }
  double* x = c->ustar;
  double* b = c->vstar;
  const size_t bytes = g.count() * sizeof(double);
  CUDA_TRY(cudaMemsetAsync(b, 0x3f, bytes, st));  // every double 0x3f3f...3f, about 4.8e-4
  int best = -1;
  std::vector<float> ms;
  cudaError_t e = cudaSuccess;
  if (mixed) {
    // block counts of the mixed solve, then tile plans of its one-barrier form
    const std::vector<int> cand = mixed_block_candidates(most);
    const std::vector<TilePlan> cand1 = mixed1_plan_candidates(g.nx, g.ny, deg);
    const int nm = (int)cand.size();
    MixedSolve a{};
    case_mixed_solve(c, x, b, &a);
    a.d.tol = 0.0;
    a.d.max_iter = kTuneIters;
    e = time_launches(nm + (int)cand1.size(), [&](int k) -> cudaError_t {
      cudaError_t me = cudaMemsetAsync(x, 0, bytes, st);
      if (me != cudaSuccess) return me;
      if (k >= nm) {
        Mixed1Solve f{};
        case_mixed1_solve(c, a, cand1[k - nm], &f);
        return run_poisson_mixed1(f, st);
      }
      a.blocks = cand[k];
      return run_poisson_mixed(a, st);
    }, st, &best, &ms);
    if (best >= nm) r.mixed1 = cand1[best - nm];
    else if (best >= 0) r.mixed_blocks = cand[best];
  } else {
    const std::vector<TilePlan> cand = fused_plan_candidates(g.nx, g.ny, most);
    const std::vector<int> ccand = cluster_candidates(g.nx, g.ny);
    const int nf = (int)cand.size();
    CaseSolveView v;
    case_solve_view(c, &v);
    FusedSolve f{};
    f.a = scaled_solve_of(v, x, b, c->pz, nullptr, nullptr, c->pp0, nullptr);
    f.fxacc = c->fxacc;
    f.a.partials = c->partials;
    f.a.bar = case_barrier(c);
    f.a.out = PcgOut{&c->ds->iters_p, &c->ds->rr_p, &c->ds->bb_p, &c->ds->conv_p, nullptr, nullptr};
    f.a.tol = 0.0;
    f.a.max_iter = kTuneIters;
    f.R[0] = c->pr; f.R[1] = c->pz2;
    f.W[0] = c->pq; f.W[1] = c->pw1;
    f.S[0] = c->pp1; f.S[1] = c->t5;
    e = time_launches(nf + (int)ccand.size(), [&](int k) -> cudaError_t {
      cudaError_t me = cudaMemsetAsync(x, 0, bytes, st);
      if (me != cudaSuccess) return me;
      if (k >= nf) {
        ClusterSolve cs{};
        cs.a = f.a;
        return run_poisson_cluster(cs, ccand[k - nf], st);
      }
      f.TX = cand[k].TX; f.TY = cand[k].TY; f.nbx = cand[k].nbx; f.ntiles = cand[k].ntiles;
      f.resident = cand[k].resident;
      return run_poisson_fused(f, st);
    }, st, &best, &ms);
    if (best >= nf) r.cluster = ccand[best - nf];
    else if (best >= 0) r.plan = cand[best];
  }
  if (e != cudaSuccess) return fail(CCM_E_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
  CUDA_TRY(cudaMemsetAsync(x, 0, bytes, st));
  CUDA_TRY(cudaMemsetAsync(b, 0, bytes, st));
  CUDA_TRY(cudaMemsetAsync(c->ds, 0, sizeof(DevStats), st));
  int bar_err = 0;
  CUDA_TRY(cudaMemcpyAsync(&bar_err, c->bar_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  if (bar_err) return fail(CCM_E_TIMEOUT, "autotune: a device-wide barrier gave up waiting");
  if (best >= 0) tune_cache_put(g.nx, g.ny, c->cfg.precision, c->cfg.precond, deg, most, r);
  c->tune = r;
  return CCM_OK;
}

ccm_status poisson_solve(ccm_case c, double* x, double* b) {
  if (c->cfg.precision == CCM_MIXED) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (c->timing) {
      e0 = next_event(c);
      e1 = next_event(c);
      if (e0) cudaEventRecord(e0, c->st);
    }
    ccm_status s = solve_poisson_mixed(c, x, b);
    if (c->timing && e1) cudaEventRecord(e1, c->st);
    c->poisson_launches++;
    launch_wrap_cells(c->g, x, c->st);  // periodic sides: Phi's images for the projection
    return s;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c->timing) {
    e0 = next_event(c);
    e1 = next_event(c);
    if (e0) cudaEventRecord(e0, c->st);
  }
  ccm_status s = solve_poisson_fp64(c, x, b);
  if (c->timing && e1) cudaEventRecord(e1, c->st);
  c->poisson_launches++;
  c->launches += c->zero_mean ? 5 : 1;
  launch_wrap_cells(c->g, x, c->st);  // periodic sides: Phi's images for the projection
  return s;
}

// Sum the recorded Poisson PCG event pairs (after the stream has drained).
void collect_timing(ccm_case c) {
  for (size_t k = 0; k + 1 < c->ev_used; k += 2) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->ev_pool[k], c->ev_pool[k + 1]) == cudaSuccess) c->poisson_ms += ms;
  }
  c->ev_used = 0;
}

}  // namespace

extern "C" {
// The factor f of the body velocity D = f D0 at the time t = n dt of step n (1 when steady).
static double motion_factor(ccm_case c, long long n) {
  if (!c->moving) return 1.0;
  const double t = (double)n * c->ph.dt;
  return c->motion[0] + c->motion[1] * std::sin(c->motion[2] * t + c->motion[3]);
}

static ccm_status stage_predict(ccm_case c);
static void stage_project(ccm_case c);
static ccm_status finish_stats(ccm_case c, ccm_step_stats* stats);
}

namespace ccm {
bool case_solve_view(ccm_case c, CaseSolveView* v) {
  if (!c || !c->geometry) return false;
  v->g = c->g;
  v->st = c->st;
  v->cu = c->co.cu;
  v->cv = c->co.cv;
  v->dk = c->co.diagk;
  v->invd = c->co.invdk;
  v->kind = c->co.kind;
  v->act = c->co.act;
  v->sd = c->co.sdk; v->isd = c->co.isdk; v->cus = c->co.cus; v->cvs = c->co.cvs; v->kinds = c->co.kinds;
  v->precond = c->cfg.precond;
  v->tol = c->cfg.tol_p;
  v->max_iter = c->cfg.max_iter_p;
  v->zero_mean = c->zero_mean;
  v->n_act = c->n_act;
  return true;
}
void set_last_error(const char* msg) { g_last_error = msg; }

ScaledSolve scaled_solve_of(const CaseSolveView& v, double* x, const double* b, double* xs, double* r, double* w,
                            double* p, double* s) {
  ScaledSolve a{};
  a.g = v.g;
  a.cu = v.cu; a.cv = v.cv; a.dk = v.dk; a.kind = v.kind;
  a.sd = v.sd; a.isd = v.isd; a.cus = v.cus; a.cvs = v.cvs; a.kinds = v.kinds;
  a.creg_x = v.g.hy / v.g.hx;
  a.creg_y = v.g.hx / v.g.hy;
  a.dreg = 2.0 * (a.creg_x + a.creg_y);
  a.ax = a.creg_x / a.dreg;
  a.ay = a.creg_y / a.dreg;
  a.x = x; a.b = b;
  a.xs = xs; a.r = r; a.w = w; a.p = p; a.s = s;
  a.tol = v.tol; a.max_iter = v.max_iter;
  return a;
}

// The case's arrays for the batched explicit stages of its next step (ahead = 0) or of the
// step after it (ahead = 1: the two time levels of conv swapped) (csrc/batch.cu).
void case_stage_case(ccm_case c, StageCase* e, int ahead) {
  const int cur = c->cur ^ (ahead & 1);
  const int prev = cur, next = 1 - cur;
  StageCase a{};
  a.c = c->cv; a.g = c->g; a.bc = c->bc; a.ph = c->ph;
  a.u = c->u; a.v = c->v; a.p = c->p; a.phi = c->phi;
  a.cpu = c->cnu[prev]; a.cpv = c->cnv[prev]; a.cnu = c->cnu[next]; a.cnv = c->cnv[next];
  a.ru = c->rhs_u; a.rv = c->rhs_v;
  a.ustar = c->ustar; a.vstar = c->vstar; a.div = c->div; a.rhs = c->rhs_p;
  a.first = c->nstep + ahead == 0 ? 1 : 0;
  stage_case_blocks(c->g, &a.gx);
  *e = a;
}
int case_cur(ccm_case c) { return c->cur; }
unsigned long long case_serial(ccm_case c) { return c->serial; }
bool case_has_extras(ccm_case c) { return c->forced || c->dblock != nullptr; }
bool case_is_moving(ccm_case c) { return c->moving; }
long long case_nstep(ccm_case c) { return c->nstep; }
void case_helm_solve(ccm_case c, HelmCSolve* a) { helm_solve_of(c, a); }
// Host bookkeeping of a step whose stages ran batched (as stage_project does for one case).
void case_step_done(ccm_case c) {
  c->cur = 1 - c->cur;
  c->nstep++;
  c->steps_pending++;
}

// Pieces of the step for the batch driver (csrc/batch.cu).
ccm_status case_finish(ccm_case c, ccm_step_stats* stats) { return finish_stats(c, stats); }
bool case_is_mixed(ccm_case c) { return c->cfg.precision == CCM_MIXED; }
cudaStream_t case_stream(ccm_case c) { return c->st; }
size_t case_cells(ccm_case c) { return (size_t)c->g.nx * c->g.ny; }
int case_nx(ccm_case c) { return c->g.nx; }

// Descriptors of the case's pressure solve (x = Phi, b = the step's right-hand side) for the
// batched kernels; statistics go to the case's device counters as for a single solve.
bool case_scaled_ok(ccm_case c) { return !c->zero_mean && c->geometry; }
void case_scaled_fp64(ccm_case c, ScaledSolve* a) {
  CaseSolveView v;
  case_solve_view(c, &v);
  *a = scaled_solve_of(v, c->phi, c->rhs_p, c->pz, c->pr, c->pq, c->pp0, c->pp1);
  a->out = PcgOut{&c->ds->iters_p, &c->ds->rr_p, &c->ds->bb_p, &c->ds->conv_p, &c->ds->total_p, &c->ds->nconv};
}
void case_mixed_batch(ccm_case c, MixedSolve* a) { case_mixed_solve(c, c->phi, c->rhs_p, a); }

// FP64 Jacobi-PCG descriptor of the case's pressure solve (x = Phi, b = the step's right-hand
// side); statistics go to the case's device counters as for a single solve.
void case_poisson_fp64(ccm_case c, PoissonSolve<double>* a) {
  *a = PoissonSolve<double>{};
  a->g = c->g;
  a->cu = c->co.cu; a->cv = c->co.cv; a->dk = c->co.diagk; a->invd = c->co.invdk; a->kind = c->co.kind;
  a->creg_x = c->g.hy / c->g.hx;
  a->creg_y = c->g.hx / c->g.hy;
  a->dreg = 2.0 * (a->creg_x + a->creg_y);
  a->invd_reg = 1.0 / a->dreg;
  a->x = c->phi; a->b = c->rhs_p; a->r = c->pr; a->z = c->pz; a->q = c->pq; a->p0 = c->pp0; a->p1 = c->pp1;
  a->cheb = 1;
  a->tol = c->cfg.tol_p; a->max_iter = c->cfg.max_iter_p;
  a->zero_mean = c->zero_mean; a->n_act = c->n_act;
  a->out = PcgOut{&c->ds->iters_p, &c->ds->rr_p, &c->ds->bb_p, &c->ds->conv_p, &c->ds->total_p, &c->ds->nconv};
}

// FP32 descriptor of one inner solve of the mixed-precision refinement (x = the FP32
// correction, b = the FP32 residual written by case_mixed_residual).
void case_poisson_fp32(ccm_case c, PoissonSolve<float>* a) {
  *a = PoissonSolve<float>{};
  a->g = c->g;
  a->cu = c->co.cu32; a->cv = c->co.cv32; a->dk = c->co.diagk32; a->invd = c->co.invdk32; a->kind = c->co.kind;
  a->creg_x = c->g.hy / c->g.hx;
  a->creg_y = c->g.hx / c->g.hy;
  a->dreg = 2.0 * (a->creg_x + a->creg_y);
  a->invd_reg = 1.0 / a->dreg;
  a->x = c->fx; a->b = c->fb; a->r = c->fr; a->z = c->fz; a->q = c->fq; a->p0 = c->fp0; a->p1 = c->fp1;
  a->cheb = 1;
  a->tol = c->cfg.tol_inner > 0 ? c->cfg.tol_inner : 1e-5;
  a->max_iter = c->cfg.max_iter_p;
  a->zero_mean = c->zero_mean; a->n_act = c->n_act;
  a->out = PcgOut{&c->ds->iters_p, &c->ds->rr_p, &c->ds->bb_p, &c->ds->conv_p, nullptr, nullptr};
}

// Mixed refinement helpers: FP64 residual into the FP32 right-hand side with its sums copied
// to `host2` (valid after the stream syncs), and x += correction.
// Singular systems: Phi and the right-hand side onto zero mean in FP64 (start and end of the
// batched refinement, as solve_poisson_mixed does for one case); nothing for other systems.
ccm_status case_mixed_project(ccm_case c, bool with_rhs) {
  if (!c->zero_mean) return CCM_OK;
  CUDA_TRY(project_zero_mean(c->g, c->co.act, c->phi, c->partials, (double)c->n_act, c->st));
  if (with_rhs) CUDA_TRY(project_zero_mean(c->g, c->co.act, c->rhs_p, c->partials, (double)c->n_act, c->st));
  c->launches += with_rhs ? 4 : 2;
  return CCM_OK;
}
ccm_status case_mixed_residual(ccm_case c, double* host2) {
  launch_residual64(c->cv, c->g, c->phi, c->rhs_p, c->fb, c->dpart, c->mixed_sums, c->st);
  CUDA_TRY(cudaMemcpyAsync(host2, c->mixed_sums, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CUDA_TRY(cudaMemsetAsync(c->fx, 0, c->g.count() * sizeof(float), c->st));
  c->launches += 2;
  return CCM_OK;
}
void case_mixed_correct(ccm_case c) {
  launch_add_correction(c->g, c->co.act, c->phi, c->fx, c->st);
  c->launches += 1;
}
void case_mixed_account(ccm_case c, long long inner, int outer, double rr, double bb, bool converged) {
  c->mixed_host = true;
  c->mixed_total += inner;
  c->mixed_last = (int)inner;
  c->mixed_outer = outer;
  c->mixed_rr = rr;
  c->mixed_bb = bb;
  if (!converged) c->mixed_nconv++;
}
int* case_inner_iters_dev(ccm_case c) { return &c->ds->iters_p; }
}  // namespace ccm

extern "C" {

int ccm_version(void) { return CCM_VERSION; }

const char* ccm_last_error(void) { return g_last_error.c_str(); }

// Face abscissas f = -3 .. n+3 of a stretched mesh from the n+1 given ones (the second-kind
// capacities of the outermost padded cells reach three faces beyond the box): beyond the box
// the spacing mirrors the spacing inside it, 2 a_0 - a_k (a sum and a difference, which no
// compiler contracts into a fused multiply-add).  Empty if a is NULL.  False if a is not
// strictly increasing from lo to hi.
static bool extend_faces(const double* a, int n, double lo, double hi, std::vector<double>& out, double* hmin) {
  out.clear();
  if (!a) return true;
  if (n < 4 || a[0] != lo || a[n] != hi) return false;
  double m = 1e300;
  for (int k = 0; k < n; ++k) {
    if (!(a[k + 1] > a[k])) return false;
    m = std::min(m, a[k + 1] - a[k]);
  }
  out.resize((size_t)n + 7);
  for (int f = -3; f <= n + 3; ++f)
    out[(size_t)(f + 3)] = f < 0 ? (a[0] + a[0]) - a[-f] : (f > n ? (a[n] + a[n]) - a[2 * n - f] : a[f]);
  *hmin = m;
  return true;
}

ccm_status ccm_create_case(const ccm_config* cfg, ccm_case* out) {
  g_last_error.clear();
  if (!cfg || !out) return fail(CCM_E_INVALID, "null argument");
  if (cfg->nx < 4 || cfg->ny < 4) return fail(CCM_E_INVALID, "nx and ny must be >= 4");
  if ((long long)(cfg->nx + 3) * (cfg->ny + 3) > (1LL << 31) - 1024) return fail(CCM_E_INVALID, "grid too large");
  if (!(cfg->x1 > cfg->x0) || !(cfg->y1 > cfg->y0)) return fail(CCM_E_INVALID, "empty box");
  if (!(cfg->rho > 0) || !(cfg->mu >= 0) || !(cfg->dt > 0)) return fail(CCM_E_INVALID, "rho, dt must be > 0, mu >= 0");
  for (int s = 0; s < 4; ++s)
    if (cfg->bc_type[s] != CCM_BC_DIRICHLET && cfg->bc_type[s] != CCM_BC_OUTFLOW && cfg->bc_type[s] != CCM_BC_PERIODIC)
      return fail(CCM_E_INVALID, "unknown boundary type");
  {
    const bool px = cfg->bc_type[CCM_SIDE_W] == CCM_BC_PERIODIC, py = cfg->bc_type[CCM_SIDE_S] == CCM_BC_PERIODIC;
    if (px != (cfg->bc_type[CCM_SIDE_E] == CCM_BC_PERIODIC) || py != (cfg->bc_type[CCM_SIDE_N] == CCM_BC_PERIODIC))
      return fail(CCM_E_INVALID, "periodic sides come in pairs (W with E, S with N)");
    if ((px && (cfg->nx % 3 != 0 || cfg->xf)) || (py && (cfg->ny % 3 != 0 || cfg->yf)))
      return fail(CCM_E_INVALID, "a periodic axis needs a uniform mesh with a multiple of 3 cells");
  }
  if (cfg->precision != CCM_FP64 && cfg->precision != CCM_MIXED) return fail(CCM_E_INVALID, "unknown precision");
  if (cfg->precond != CCM_JACOBI && cfg->precond != CCM_CHEBYSHEV) return fail(CCM_E_INVALID, "unknown preconditioner");
  if (cfg->pressure_update < 0 || cfg->pressure_update > 2)
    return fail(CCM_E_INVALID, "pressure_update must be 0, 1 or 2");
  if (cfg->precond == CCM_CHEBYSHEV && !cheb_degree_supported(cfg->cheb_degree))
    return fail(CCM_E_INVALID, "cheb_degree must be 1-6 or 8");
  if (cfg->guess_history < 0 || cfg->guess_history > kGuessMax)
    return fail(CCM_E_INVALID, "guess_history must be in 0..32");
  if (!(cfg->tol_p > 0) || !(cfg->tol_h > 0) || cfg->max_iter_p < 1 || cfg->max_iter_h < 1)
    return fail(CCM_E_INVALID, "solver tolerances and limits must be positive");
  ccm_case c = new ccm_case_s();
  static std::atomic<unsigned long long> next_serial{1};
  c->serial = next_serial++;
  c->cfg = *cfg;
  c->g.nx = cfg->nx;
  c->g.ny = cfg->ny;
  c->g.pitch = ((cfg->nx + 3) + 31) / 32 * 32;
  c->g.x0 = cfg->x0;
  c->g.y0 = cfg->y0;
  c->g.hx = (cfg->x1 - cfg->x0) / cfg->nx;
  c->g.hy = (cfg->y1 - cfg->y0) / cfg->ny;
  c->g.xf = c->g.yf = nullptr;
  c->g.px = cfg->bc_type[CCM_SIDE_W] == CCM_BC_PERIODIC;
  c->g.py = cfg->bc_type[CCM_SIDE_S] == CCM_BC_PERIODIC;
  if (!extend_faces(cfg->xf, cfg->nx, cfg->x0, cfg->x1, c->xfx, &c->g.hx) ||
      !extend_faces(cfg->yf, cfg->ny, cfg->y0, cfg->y1, c->yfx, &c->g.hy)) {
    delete c;
    return fail(CCM_E_INVALID, "face abscissas must increase strictly from x0 to x1 (y0 to y1)");
  }
  c->cfg.xf = c->cfg.yf = nullptr;  // the caller's arrays are not retained
  for (int s = 0; s < 4; ++s) {
    c->bc.type[s] = cfg->bc_type[s];
    c->bc.un[s] = cfg->bc_un[s];
    c->bc.ut[s] = cfg->bc_ut[s];
  }
  c->ph = Phys{cfg->rho, cfg->mu, cfg->dt};
  c->st = (cudaStream_t)cfg->stream;
  Carver dry{nullptr};
  carve(c, dry);
  c->slab_bytes = dry.off + 256;
  void* mem = nullptr;
  if (cfg->alloc) {
    mem = cfg->alloc(c->slab_bytes, cfg->alloc_ctx);
    if (!mem) { delete c; return fail(CCM_E_OOM, "allocator hook returned NULL"); }
  } else {
    cudaError_t e = cudaMalloc(&mem, c->slab_bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      delete c;
      return fail(CCM_E_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
  }
  c->slab = mem;
  Carver real{(char*)(((uintptr_t)mem + 255) & ~(uintptr_t)255)};
  carve(c, real);
  if (!c->xfx.empty()) c->g.xf = c->xfd + 3;
  if (!c->yfx.empty()) c->g.yf = c->yfd + 3;
  make_view(c);
  cudaError_t e = cudaMemsetAsync(mem, 0, c->slab_bytes, c->st);
  if (e == cudaSuccess && !c->xfx.empty())
    e = cudaMemcpyAsync(c->xfd, c->xfx.data(), c->xfx.size() * sizeof(double), cudaMemcpyHostToDevice, c->st);
  if (e == cudaSuccess && !c->yfx.empty())
    e = cudaMemcpyAsync(c->yfd, c->yfx.data(), c->yfx.size() * sizeof(double), cudaMemcpyHostToDevice, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) {
    if (cfg->free) cfg->free(mem, cfg->alloc_ctx); else cudaFree(mem);
    delete c;
    return fail(CCM_E_CUDA, std::string("initialising case memory: ") + cudaGetErrorString(e));
  }
  *out = c;
  return CCM_OK;
}

ccm_status ccm_launch_plan(ccm_case c, int plan[7]) {
  g_last_error.clear();
  if (!c || !plan) return fail(CCM_E_INVALID, "null argument");
  if (!c->geometry) return fail(CCM_E_STATE, "set_geometry must come first");
  // the tile plan of the one-barrier solve of the case's precision
  const TilePlan& tp = c->cfg.precision == CCM_MIXED ? c->tune.mixed1 : c->tune.plan;
  plan[0] = tp.TX;
  plan[1] = tp.TY;
  plan[2] = tp.nbx;
  plan[3] = tp.ntiles;
  plan[4] = c->tune.mixed_blocks;
  plan[5] = c->tune.cluster;
  plan[6] = tp.resident;
  return CCM_OK;
}

ccm_status ccm_set_launch_plan(ccm_case c, const int plan[7]) {
  g_last_error.clear();
  if (!c || !plan) return fail(CCM_E_INVALID, "null argument");
  if (!c->geometry) return fail(CCM_E_STATE, "set_geometry must come first");
  TuneResult r{};
  const Geom& g = c->g;
  const bool mixed = c->cfg.precision == CCM_MIXED;
  if (plan[0] != 0 && mixed) {
    // the one-barrier mixed solve: its tiles and their bands must fit the GPU at once
    const int tx = plan[0], ty = plan[1];
    const bool pow2 = tx >= 32 && tx <= 512 && (tx & (tx - 1)) == 0;
    const int nbx = (g.nx + tx - 1) / std::max(tx, 1);
    if (!pow2 || ty < 1 || plan[2] != nbx || plan[3] != nbx * ((g.ny + ty - 1) / ty))
      return fail(CCM_E_INVALID, "tile plan: width a power of two in 32..512, tiles = ceil(nx/w) ceil(ny/h)");
    if (plan[5] != 0 || plan[4] != 0)
      return fail(CCM_E_INVALID, "a mixed tile plan excludes clusters and block counts");
    if (plan[6] != 0 && plan[6] != 1) return fail(CCM_E_INVALID, "resident must be 0 or 1");
    const int deg = c->cfg.precond == CCM_CHEBYSHEV ? c->cfg.cheb_degree : 1;
    if (!mixed1_plan_fits(tx, ty, plan[3], deg, plan[6]))
      return fail(CCM_E_INVALID, "the mixed tiles (and, resident, their vectors) do not fit the GPU at once");
    r.mixed1 = TilePlan{tx, ty, plan[2], plan[3], plan[6]};
    c->tune = r;
    return CCM_OK;
  }
  if (plan[0] != 0) {
    const int tx = plan[0], ty = plan[1];
    const bool pow2 = tx >= 32 && tx <= 512 && (tx & (tx - 1)) == 0;
    const int nbx = (g.nx + tx - 1) / std::max(tx, 1);
    if (!pow2 || ty < 1 || plan[2] != nbx || plan[3] != nbx * ((g.ny + ty - 1) / ty) || plan[3] > fused_blocks())
      return fail(CCM_E_INVALID, "tile plan: width a power of two in 32..512, tiles = ceil(nx/w) ceil(ny/h)");
    if (plan[6] != 0 && plan[6] != 1) return fail(CCM_E_INVALID, "resident must be 0 or 1");
    if (plan[6] == 1 && !fused_resident_ok(tx, ty, plan[3]))
      return fail(CCM_E_INVALID, "resident tiles do not fit in shared memory on this GPU");
    r.plan = TilePlan{tx, ty, plan[2], plan[3], plan[6]};
  } else if (plan[6] != 0) {
    return fail(CCM_E_INVALID, "resident tiles need a tile plan");
  }
  if (plan[4] < 0 || plan[4] > mixed_blocks()) return fail(CCM_E_INVALID, "mixed blocks out of range");
  r.mixed_blocks = plan[4];
  if (plan[5] != 0) {
    bool ok = false;
    for (int C : cluster_candidates(g.nx, g.ny)) ok = ok || C == plan[5];
    if (!ok) return fail(CCM_E_INVALID, "cluster size: 2, 4, 8 or 16 CTAs, at most ny, band in shared memory");
    if (plan[0] != 0) return fail(CCM_E_INVALID, "a tile plan and a cluster exclude each other");
    r.cluster = plan[5];
  }
  c->tune = r;
  return CCM_OK;
}

ccm_status ccm_case_bytes(const ccm_config* cfg, size_t* bytes) {
  if (!cfg || !bytes || cfg->nx < 4 || cfg->ny < 4) return fail(CCM_E_INVALID, "bad configuration");
  ccm_case_s tmp;
  tmp.g.nx = cfg->nx;
  tmp.g.ny = cfg->ny;
  tmp.g.pitch = ((cfg->nx + 3) + 31) / 32 * 32;
  Carver dry{nullptr};
  carve(&tmp, dry);
  *bytes = dry.off + 256;
  return CCM_OK;
}

// Device memory outside the case's slab (force record, D terms), with the case's allocator.
static void* case_alloc(ccm_case c, size_t bytes) {
  void* mem = nullptr;
  if (c->cfg.alloc) return c->cfg.alloc(bytes, c->cfg.alloc_ctx);
  if (cudaMalloc(&mem, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return mem;
}
static void case_free(ccm_case c, void* mem) {
  if (!mem) return;
  if (c->cfg.free) c->cfg.free(mem, c->cfg.alloc_ctx);
  else cudaFree(mem);
}

static void free_force_history(ccm_case c) {
  case_free(c, c->fhist);
  c->fhist = nullptr;
  c->fcap = 0;
  c->frec = 0;
}

ccm_status ccm_destroy_case(ccm_case c) {
  if (!c) return CCM_OK;
  cudaStreamSynchronize(c->st);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  free_force_history(c);
  case_free(c, c->dblock);
  case_free(c, c->gmem);
  if (c->slab) {
    if (c->cfg.free) c->cfg.free(c->slab, c->cfg.alloc_ctx);
    else cudaFree(c->slab);
  }
  delete c;
  return CCM_OK;
}

ccm_status ccm_set_geometry(ccm_case c, const ccm_geometry* geo) {
  g_last_error.clear();
  if (!c || !geo) return fail(CCM_E_INVALID, "null argument");
  if (geo->kind < CCM_GEOM_NONE || geo->kind > CCM_GEOM_HALFPLANE) return fail(CCM_E_INVALID, "unknown geometry kind");
  if (geo->kind == CCM_GEOM_CIRCLE && !(geo->r > 0)) return fail(CCM_E_INVALID, "circle radius must be > 0");
  if (geo->kind == CCM_GEOM_NACA && (!(geo->chord > 0) || geo->naca_tt < 1 || geo->naca_tt > 40))
    return fail(CCM_E_INVALID, "bad NACA parameters");
  if (geo->kind == CCM_GEOM_HALFPLANE && geo->hp_nx == 0.0 && geo->hp_ny == 0.0)
    return fail(CCM_E_INVALID, "half plane normal is zero");
  const Geom& g = c->g;
  if (geo->kind == CCM_GEOM_CIRCLE || geo->kind == CCM_GEOM_NACA) {
    double xa, xb, ya, yb;
    body_bbox(*geo, xa, xb, ya, yb);
    // the body must lie between the u-grid lines 3 and nx-2 (v-grid likewise in y): on a
    // uniform mesh x0 + 2.5 hx and x1 - 2.5 hx
    const Geom gh{g.nx, g.ny, g.pitch, g.x0, g.y0, g.hx, g.hy, c->xfx.empty() ? nullptr : c->xfx.data() + 3,
                  c->yfx.empty() ? nullptr : c->yfx.data() + 3};
    if (xa < line_x(gh, 1, 3) || xb > line_x(gh, 1, g.nx - 2) || ya < line_y(gh, 2, 3) || yb > line_y(gh, 2, g.ny - 2))
      return fail(CCM_E_INVALID, "the body must stay two cells away from every box side");
  }
  cudaStream_t st = c->st;
  CUDA_TRY(launch_capacities(*geo, g, c->caps.a, st));
  launch_derive(g, c->bc, c->ph, c->cfg.literal_offdiag, c->cfg.pressure_update, c->caps, c->co, st);
  launch_scaling(g, c->co, st);
  // lifting of the box data through the viscous operator: visc(S(0, D))
  CUDA_TRY(cudaMemsetAsync(c->t0, 0, g.count() * sizeof(double), st));
  CUDA_TRY(cudaMemsetAsync(c->t1, 0, g.count() * sizeof(double), st));
  launch_fill_bc(g, c->bc, c->t0, c->t1, 1.0, st);
  launch_visc(c->cv, g, c->bc, c->t0, c->t1, c->co.liftu, c->co.liftv, st);
  // Jacobi diagonal of the Helmholtz operator by colour probing
  launch_helmholtz_diag(c->cv, g, c->bc, c->ph, c->t0, c->t1, c->t2, c->t3, c->t4, c->t5, c->co.invdhu, c->co.invdhv,
                        st);
  // its nine coefficients per unknown face, by colour probing
  launch_helmholtz_coefs(c->cv, g, c->bc, c->ph, c->t0, c->t1, c->t2, c->t3, c->hc, c->hc_bad, st);
  // state
  const size_t bytes = g.count() * sizeof(double);
  for (double* a : {c->p, c->phi, c->cnu[0], c->cnu[1], c->cnv[0], c->cnv[1], c->ustar, c->vstar, c->div})
    CUDA_TRY(cudaMemsetAsync(a, 0, bytes, st));
  const dim3 b(64, 4);
  k_init_velocity<<<grid_of(g, b), b, 0, st>>>(g, c->co.role_u, c->cfg.bc_un[CCM_SIDE_W], c->u, c->v);
  launch_fill_bc(g, c->bc, c->u, c->v, 1.0, st);
  CUDA_TRY(cudaMemsetAsync(c->ds, 0, sizeof(DevStats), st));
  CUDA_TRY(cudaMemsetAsync(c->bar_err, 0, sizeof(int), st));
  // number of active cells
  std::vector<int8_t> act(g.count());
  CUDA_TRY(cudaMemcpyAsync(act.data(), c->co.act, g.count(), cudaMemcpyDeviceToHost, st));
  int hc_bad = 0;
  CUDA_TRY(cudaMemcpyAsync(&hc_bad, c->hc_bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  ccm_status s = check_cuda_errors("set_geometry");
  if (s != CCM_OK) return s;
  if (hc_bad) return fail(CCM_E_INVALID, "the Helmholtz operator couples faces outside its nine-point pattern");
  long long na = 0;
  for (int8_t a : act) na += a;
  if (na == 0) return fail(CCM_E_INVALID, "no fluid cell");
  c->n_act = (double)na;
  c->zero_mean = 1;
  for (int q = 0; q < 4; ++q)
    if (c->bc.type[q] == CCM_BC_OUTFLOW) c->zero_mean = 0;
  c->cur = 0;
  c->gnb = 0;
  c->nstep = 0;
  c->geometry = true;
  return autotune_poisson(c);
}

static double* field_ptr(ccm_case c, int field) {
  switch (field) {
    case CCM_F_U: return c->u;
    case CCM_F_V: return c->v;
    case CCM_F_P: return c->p;
    case CCM_F_PHI: return c->phi;
    case CCM_F_CONV_U: return c->cnu[c->cur];
    case CCM_F_CONV_V: return c->cnv[c->cur];
    case CCM_F_USTAR: return c->ustar;
    case CCM_F_VSTAR: return c->vstar;
    case CCM_F_DIV: return c->div;
    case CCM_F_GX: return c->accx;
    case CCM_F_GY: return c->accy;
    case CCM_F_DX: return c->dblock;
    case CCM_F_DY: return c->dblock ? c->dblock + c->g.count() : nullptr;
    default:
      if (field >= CCM_F_CAP && field < CCM_F_CAP + 27) return c->caps.a[field - CCM_F_CAP];
      return nullptr;
  }
}

ccm_status ccm_set_field(ccm_case c, int field, const double* host, size_t count) {
  g_last_error.clear();
  if (!c || !host) return fail(CCM_E_INVALID, "null argument");
  if (!c->geometry) return fail(CCM_E_STATE, "set_geometry must come first");
  // the initial-guess history is only a guess for the next solves, good for any state; a new
  // warm start or step counter (a restored checkpoint) starts a new one, so that a restored
  // run repeats a fresh run from the same fields bit for bit
  if (field == CCM_F_PHI || field == CCM_F_STEP) c->gnb = 0;
  if (field == CCM_F_STEP) {
    if (count < 1) return fail(CCM_E_INVALID, "count");
    c->nstep = (long long)host[0];
    return CCM_OK;
  }
  const bool accel = field == CCM_F_GX || field == CCM_F_GY;
  const bool body = field == CCM_F_DX || field == CCM_F_DY;
  if ((field > CCM_F_CONV_V || field < 0) && !accel && !body) return fail(CCM_E_INVALID, "field is read-only or unknown");
  if (count != host_count(c)) return fail(CCM_E_INVALID, "count must be (nx+3)*(ny+3)");
  if (body && !c->dblock) {
    CUDA_TRY(cudaStreamSynchronize(c->st));
    void* mem = case_alloc(c, 8 * c->g.count() * sizeof(double));
    if (!mem) return fail(CCM_E_OOM, "cannot allocate the body-velocity terms");
    CUDA_TRY(cudaMemsetAsync(mem, 0, 8 * c->g.count() * sizeof(double), c->st));
    c->dblock = (double*)mem;
    make_view(c);
  }
  ccm_status s = upload(c, field_ptr(c, field), host);
  if (s != CCM_OK) return s;
  if (accel && !c->forced) {
    // from now on the predictor adds rho V g (the other component stays zero until set)
    c->forced = true;
    make_view(c);
  }
  const dim3 b(64, 4);
  if (field == CCM_F_U || field == CCM_F_V) {
    // faces whose control volume holds no fluid carry the body's velocity (zero: no-slip)
    launch_inactive_to_body(c->g, c->co.role_u, c->co.role_v, c->cv.dx, c->cv.dy, c->u, c->v, c->st,
                            motion_factor(c, c->nstep));
    launch_fill_bc(c->g, c->bc, c->u, c->v, 1.0, c->st);
  }
  if (body) {
    // the constant D-terms of the step, and D on the faces without fluid
    launch_body_dterms(c->g, c->bc, c->caps, c->cv, c->cv.dx, c->cv.dy, (double*)c->cv.hd, (double*)c->cv.sxxd,
                       (double*)c->cv.syyd, (double*)c->cv.sxyd, (double*)c->cv.viscdu, (double*)c->cv.viscdv,
                       c->st);
    launch_inactive_to_body(c->g, c->co.role_u, c->co.role_v, c->cv.dx, c->cv.dy, c->u, c->v, c->st,
                            motion_factor(c, c->nstep));
  }
  if (field == CCM_F_P || field == CCM_F_PHI) {
    // only active cells carry pressure; the ghost ring stays zero (periodic sides: images)
    k_mask_cells<<<grid_of(c->g, b), b, 0, c->st>>>(c->g, c->co.act, field_ptr(c, field));
    launch_wrap_cells(c->g, field_ptr(c, field), c->st);
  }
  CUDA_TRY(cudaStreamSynchronize(c->st));
  return check_cuda_errors("set_field");
}

ccm_status ccm_get_field(ccm_case c, int field, double* host, size_t count) {
  g_last_error.clear();
  if (!c || !host) return fail(CCM_E_INVALID, "null argument");
  if (field == CCM_F_STEP) {
    if (count < 1) return fail(CCM_E_INVALID, "count");
    host[0] = (double)c->nstep;
    return CCM_OK;
  }
  double* src = field_ptr(c, field);
  if (!src) return fail(CCM_E_INVALID, "unknown field");
  if (count != host_count(c)) return fail(CCM_E_INVALID, "count must be (nx+3)*(ny+3)");
  ccm_status s = download(c, host, src);
  if (s != CCM_OK) return s;
  CUDA_TRY(cudaStreamSynchronize(c->st));
  return CCM_OK;
}

ccm_status ccm_field_device_ptr(ccm_case c, int field, void** dptr, int* pitch) {
  if (!c || !dptr) return fail(CCM_E_INVALID, "null argument");
  double* p = field_ptr(c, field);
  if (!p) return fail(CCM_E_INVALID, "unknown field");
  *dptr = p;
  if (pitch) *pitch = c->g.pitch;
  return CCM_OK;
}

ccm_status ccm_apply_op(ccm_case c, int op, const double* in0, const double* in1, double* out0, double* out1) {
  g_last_error.clear();
  if (!c) return fail(CCM_E_INVALID, "null case");
  if (!c->geometry) return fail(CCM_E_STATE, "set_geometry must come first");
  const Geom& g = c->g;
  cudaStream_t st = c->st;
  ccm_status s = CCM_OK;
  auto need = [&](const void* p) { return p != nullptr; };
  switch (op) {
    case CCM_OP_CONT:
      if (!need(in0) || !need(in1) || !need(out0)) return fail(CCM_E_INVALID, "CONT needs in0, in1, out0");
      if ((s = upload(c, c->t0, in0)) || (s = upload(c, c->t1, in1))) return s;
      launch_cont(c->cv, g, c->t0, c->t1, c->t2, st);
      if ((s = download(c, out0, c->t2))) return s;
      break;
    case CCM_OP_PRES:
      if (!need(in0) || !need(out0) || !need(out1)) return fail(CCM_E_INVALID, "PRES needs in0, out0, out1");
      if ((s = upload(c, c->t0, in0))) return s;
      launch_pres(c->cv, g, c->t0, c->t2, c->t3, st);
      if ((s = download(c, out0, c->t2)) || (s = download(c, out1, c->t3))) return s;
      break;
    case CCM_OP_CONV:
    case CCM_OP_VISC:
      if (!need(in0) || !need(in1) || !need(out0) || !need(out1))
        return fail(CCM_E_INVALID, "needs in0, in1, out0, out1");
      if ((s = upload(c, c->t0, in0)) || (s = upload(c, c->t1, in1))) return s;
      launch_fill_bc(g, c->bc, c->t0, c->t1, 1.0, st);
      if (op == CCM_OP_CONV) launch_conv(c->cv, g, c->t0, c->t1, c->t2, c->t3, st);
      else launch_visc(c->cv, g, c->bc, c->t0, c->t1, c->t2, c->t3, st);
      if ((s = download(c, out0, c->t2)) || (s = download(c, out1, c->t3))) return s;
      break;
    case CCM_OP_HELMHOLTZ:
      if (!need(in0) || !need(in1) || !need(out0) || !need(out1))
        return fail(CCM_E_INVALID, "needs in0, in1, out0, out1");
      if ((s = upload(c, c->t0, in0)) || (s = upload(c, c->t1, in1))) return s;
      launch_helmholtz(c->cv, g, c->bc, c->ph, c->t0, c->t1, c->t2, c->t3, st);
      if ((s = download(c, out0, c->t2)) || (s = download(c, out1, c->t3))) return s;
      break;
    case CCM_OP_POISSON:
      if (!need(in0) || !need(out0)) return fail(CCM_E_INVALID, "POISSON needs in0, out0");
      if ((s = upload(c, c->t0, in0))) return s;
      launch_poisson(c->cv, g, c->t0, c->t2, c->t1, st);
      if ((s = download(c, out0, c->t2))) return s;
      break;
    case CCM_OP_POISSON_DIAG:
      if (!need(out0)) return fail(CCM_E_INVALID, "needs out0");
      if ((s = download(c, out0, c->co.diagk))) return s;
      break;
    case CCM_OP_HELMHOLTZ_DIAG:
      if (!need(out0) || !need(out1)) return fail(CCM_E_INVALID, "needs out0, out1");
      launch_helmholtz_diag(c->cv, g, c->bc, c->ph, c->t0, c->t1, c->t2, c->t3, c->t4, c->t5, nullptr, nullptr, st);
      if ((s = download(c, out0, c->t4)) || (s = download(c, out1, c->t5))) return s;
      break;
    default:
      return fail(CCM_E_INVALID, "unknown operator");
  }
  CUDA_TRY(cudaStreamSynchronize(st));
  return check_cuda_errors("apply_op");
}

static ccm_status read_stats(ccm_case c, DevStats& h) {
  CUDA_TRY(cudaMemcpyAsync(&h, c->ds, sizeof(DevStats), cudaMemcpyDeviceToHost, c->st));
  int err = 0;
  CUDA_TRY(cudaMemcpyAsync(&err, c->bar_err, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  CUDA_TRY(cudaStreamSynchronize(c->st));
  if (err) {
    cudaMemsetAsync(c->bar_err, 0, sizeof(int), c->st);
    cudaStreamSynchronize(c->st);
    return fail(CCM_E_TIMEOUT, "a device-wide barrier gave up waiting");
  }
  return check_cuda_errors("solver");
}

// Stages of one step around the Poisson solve: box data, predictor right-hand side,
// Helmholtz solve, U* and its divergence (Eq. pm_prediction, right-hand side of
// Eq. pm_poisson) ...
static ccm_status stage_predict(ccm_case c) {
  const Geom& g = c->g;
  cudaStream_t st = c->st;
  const int prev = c->cur, next = 1 - c->cur;
  // D^n in conv^n and S^n, D^{n+1} in the implicit half's lift and in cont(U*, D^{n+1})
  c->ph.dn = motion_factor(c, c->nstep);
  c->ph.dn1 = motion_factor(c, c->nstep + 1);
  launch_fill_bc(g, c->bc, c->u, c->v, 1.0, st);
  launch_predictor_rhs(c->cv, g, c->bc, c->ph, c->u, c->v, c->p, c->cnu[prev], c->cnv[prev], c->cnu[next],
                       c->cnv[next], c->rhs_u, c->rhs_v, c->nstep == 0 ? 1 : 0, st);
  ccm_status s;
  if ((s = solve_helmholtz(c)) != CCM_OK) return s;
  // the faces of U* without fluid carry the next level's body velocity
  if (c->moving && c->dblock) {
    launch_inactive_to_body(g, c->co.role_u, c->co.role_v, c->cv.dx, c->cv.dy, c->u, c->v, st, c->ph.dn1);
    c->launches += 1;
  }
  launch_fill_bc(g, c->bc, c->u, c->v, 1.0, st);
  CUDA_TRY(cudaMemcpyAsync(c->ustar, c->u, g.count() * sizeof(double), cudaMemcpyDeviceToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(c->vstar, c->v, g.count() * sizeof(double), cudaMemcpyDeviceToDevice, st));
  launch_divergence(c->cv, g, c->ph, c->u, c->v, c->div, c->rhs_p, st);
  return CCM_OK;
}

// ... and after it: projection, pressure update, box data (Eqs. pm_projection, pm_update).
static void stage_project(ccm_case c) {
  const Geom& g = c->g;
  cudaStream_t st = c->st;
  launch_project(c->cv, g, c->phi, c->u, c->v, c->p, st);
  launch_wrap_cells(g, c->p, st);
  launch_fill_bc(g, c->bc, c->u, c->v, 1.0, st);
  c->launches += 7;  // fill_bc x3, predictor, Helmholtz PCG, divergence, projection
  if (c->fcap > 0) {
    // the force of the new state (U^{n+1}, P^{n+1/2}) into the next row of the record
    Phys pf = c->ph;
    pf.dn = motion_factor(c, c->nstep + 1);
    launch_body_force(c->cv, g, pf, c->u, c->v, c->p, c->fpart, c->fhist + 4 * (c->frec % c->fcap), st);
    c->frec++;
    c->launches += 2;
  }
  c->cur = 1 - c->cur;
  c->nstep++;
  c->steps_pending++;
}

// The projected initial guess around one Poisson solve (guess.cu): before it, Phi = the
// projection of the new solution onto the basis; after it, the solution joins the basis (a
// full basis restarts from the newest solution).
static ccm_status guess_before(ccm_case c) {
  const int L = c->cfg.guess_history;
  if (L <= 0 || c->zero_mean) return CCM_OK;
  const size_t n = c->g.count();
  if (!c->gmem) {
    CUDA_TRY(cudaStreamSynchronize(c->st));
    void* mem = case_alloc(c, (2 * (size_t)L * n + guess_scratch_doubles()) * sizeof(double));
    if (!mem) return fail(CCM_E_OOM, "cannot allocate the initial-guess basis");
    c->gmem = (double*)mem;
    c->gnb = 0;
  }
  if (c->gnb > 0) {
    launch_guess_project(c->gmem, n, c->gnb, c->rhs_p, c->phi, c->gmem + 2 * (size_t)L * n, c->st);
    c->launches += 3;
  }
  return CCM_OK;
}

static ccm_status guess_after(ccm_case c) {
  const int L = c->cfg.guess_history;
  if (L <= 0 || c->zero_mean || !c->gmem) return CCM_OK;
  const size_t n = c->g.count();
  if (c->gnb >= L) c->gnb = 0;
  double* X = c->gmem;
  double* KX = c->gmem + (size_t)L * n;
  CUDA_TRY(cudaMemcpyAsync(X + (size_t)c->gnb * n, c->phi, n * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  launch_poisson(c->cv, c->g, c->phi, KX + (size_t)c->gnb * n, c->t0, c->st);
  launch_guess_append(X, KX, n, c->gnb, c->gmem + 2 * (size_t)L * n, c->st);
  c->launches += 1 + (c->gnb > 0 ? 8 : 0) + 3;
  c->gnb += 1;
  return CCM_OK;
}

static ccm_status enqueue_steps(ccm_case c, int nsteps) {
  ccm_status s;
  for (int n = 0; n < nsteps; ++n) {
    StageRange step("ccm step");
    {
      StageRange r("predictor + Helmholtz + divergence");
      if ((s = stage_predict(c)) != CCM_OK) return s;
    }
    {
      StageRange r("Poisson");
      if ((s = guess_before(c)) != CCM_OK) return s;
      if ((s = poisson_solve(c, c->phi, c->rhs_p)) != CCM_OK) return s;
      if ((s = guess_after(c)) != CCM_OK) return s;
    }
    StageRange r("projection");
    stage_project(c);
  }
  return check_cuda_errors("step");
}

static ccm_status finish_stats(ccm_case c, ccm_step_stats* stats) {
  const Geom& g = c->g;
  launch_diagnostics(c->cv, g, c->caps.a[cap_slot(1, CK_V)], c->caps.a[cap_slot(2, CK_V)], c->u, c->v, c->dpart,
                     c->ds->diag, c->st, motion_factor(c, c->nstep));
  DevStats h{};
  ccm_status s;
  if ((s = read_stats(c, h)) != CCM_OK) {
    // the statistics of the abandoned steps are dropped with them
    c->steps_pending = 0;
    cudaMemsetAsync(c->ds, 0, sizeof(DevStats), c->st);
    cudaStreamSynchronize(c->st);
    return s;
  }
  if (c->timing) collect_timing(c);
  if (c->mixed_host) {
    // host-driven refinements report through the case; one-launch mixed solves through the
    // device counters, like FP64 solves
    h.total_p += c->mixed_total;
    h.iters_p = c->mixed_last;
    h.rr_p = c->mixed_rr;
    h.bb_p = c->mixed_bb;
    h.nconv += c->mixed_nconv;
    c->mixed_total = 0;
    c->mixed_nconv = 0;
    c->mixed_host = false;
  }
  if (stats) {
    stats->steps = (int)c->steps_pending;
    stats->iters_p = h.total_p;
    stats->iters_h = h.total_h;
    stats->last_iters_p = h.iters_p;
    stats->last_iters_h = h.iters_h;
    stats->last_res_p = h.bb_p > 0 ? sqrt(h.rr_p / h.bb_p) : 0.0;
    stats->last_res_h = h.bb_h > 0 ? sqrt(h.rr_h / h.bb_h) : 0.0;
    stats->max_div = h.diag[0];
    stats->kinetic = h.diag[1];
    stats->mass = h.diag[3];
    stats->momentum_x = h.diag[4];
    stats->momentum_y = h.diag[5];
    stats->converged = h.nconv == 0;
  }
  if (c->timing) c->poisson_iters_timed += h.total_p;
  c->steps_pending = 0;
  CUDA_TRY(cudaMemsetAsync(c->ds, 0, sizeof(DevStats), c->st));
  if (h.diag[2] != 0.0) return fail(CCM_E_NONFINITE, "non-finite velocity");
  if (h.nconv) return fail(CCM_E_NOT_CONVERGED, "a PCG reached its iteration limit");
  return CCM_OK;
}

ccm_status ccm_step(ccm_case c, int nsteps, ccm_step_stats* stats) {
  g_last_error.clear();
  if (!c) return fail(CCM_E_INVALID, "null case");
  if (!c->geometry) return fail(CCM_E_STATE, "set_geometry must come first");
  if (nsteps < 0) return fail(CCM_E_INVALID, "nsteps < 0");
  ccm_status s = enqueue_steps(c, nsteps);
  if (s != CCM_OK) return s;
  return finish_stats(c, stats);
}

ccm_status ccm_set_barrier_fault(ccm_case c, long long budget_cycles, int absent_block) {
  g_last_error.clear();
  if (!c) return fail(CCM_E_INVALID, "null case");
  if (budget_cycles < 0 || absent_block < -1) return fail(CCM_E_INVALID, "budget_cycles >= 0, absent_block >= -1");
  c->bar_budget = budget_cycles > 0 ? budget_cycles : kBarrierBudget;
  c->bar_absent = absent_block;
  return CCM_OK;
}

ccm_status ccm_set_sum_fallback(ccm_case c, int every) {
  g_last_error.clear();
  if (!c) return fail(CCM_E_INVALID, "null case");
  if (every < 0) return fail(CCM_E_INVALID, "every >= 0");
  c->fx_fallback_every = every;
  return CCM_OK;
}

ccm_status ccm_set_body_motion(ccm_case c, double a0, double a1, double omega, double phase) {
  g_last_error.clear();
  if (!c) return fail(CCM_E_INVALID, "null case");
  if (!std::isfinite(a0) || !std::isfinite(a1) || !std::isfinite(omega) || !std::isfinite(phase))
    return fail(CCM_E_INVALID, "non-finite motion parameter");
  c->motion[0] = a0; c->motion[1] = a1; c->motion[2] = omega; c->motion[3] = phase;
  c->moving = !(a0 == 1.0 && a1 == 0.0);
  if (c->geometry && c->dblock) {
    // the present state's faces without fluid take the body velocity of its time level
    launch_inactive_to_body(c->g, c->co.role_u, c->co.role_v, c->cv.dx, c->cv.dy, c->u, c->v, c->st,
                            motion_factor(c, c->nstep));
    launch_fill_bc(c->g, c->bc, c->u, c->v, 1.0, c->st);
    CUDA_TRY(cudaStreamSynchronize(c->st));
  }
  return check_cuda_errors("set_body_motion");
}

ccm_status ccm_step_async(ccm_case c, int nsteps) {
  g_last_error.clear();
  if (!c) return fail(CCM_E_INVALID, "null case");
  if (!c->geometry) return fail(CCM_E_STATE, "set_geometry must come first");
  if (nsteps < 0) return fail(CCM_E_INVALID, "nsteps < 0");
  return enqueue_steps(c, nsteps);
}

ccm_status ccm_read_stats(ccm_case c, ccm_step_stats* stats) {
  g_last_error.clear();
  if (!c) return fail(CCM_E_INVALID, "null case");
  if (!c->geometry) return fail(CCM_E_STATE, "set_geometry must come first");
  return finish_stats(c, stats);
}

ccm_status ccm_body_force(ccm_case c, double force[4]) {
  g_last_error.clear();
  if (!c || !force) return fail(CCM_E_INVALID, "null argument");
  if (!c->geometry) return fail(CCM_E_STATE, "set_geometry must come first");
  Phys pf = c->ph;
  pf.dn = motion_factor(c, c->nstep);
  launch_body_force(c->cv, c->g, pf, c->u, c->v, c->p, c->fpart, c->fout, c->st);
  CUDA_TRY(cudaMemcpyAsync(force, c->fout, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CUDA_TRY(cudaStreamSynchronize(c->st));
  return check_cuda_errors("body_force");
}

ccm_status ccm_set_force_history(ccm_case c, int capacity) {
  g_last_error.clear();
  if (!c) return fail(CCM_E_INVALID, "null case");
  if (capacity < 0) return fail(CCM_E_INVALID, "capacity < 0");
  CUDA_TRY(cudaStreamSynchronize(c->st));
  free_force_history(c);
  if (capacity == 0) return CCM_OK;
  void* mem = case_alloc(c, (size_t)capacity * 4 * sizeof(double));
  if (!mem) return fail(CCM_E_OOM, "cannot allocate the force record");
  c->fhist = (double*)mem;
  c->fcap = capacity;
  c->frec = 0;
  return CCM_OK;
}

ccm_status ccm_get_force_history(ccm_case c, double* host, int max_rows, int* rows, long long* total) {
  g_last_error.clear();
  if (!c || !rows || (max_rows > 0 && !host) || max_rows < 0) return fail(CCM_E_INVALID, "bad argument");
  if (total) *total = c->frec;
  const long long kept = std::min<long long>(c->frec, c->fcap);
  const int n = (int)std::min<long long>(kept, max_rows);
  *rows = n;
  if (n == 0) return CCM_OK;
  CUDA_TRY(cudaStreamSynchronize(c->st));
  // the newest n rows, oldest first: ring positions (frec - n) .. (frec - 1) modulo fcap
  const long long first = c->frec - n;
  const int r0 = (int)(first % c->fcap);
  const int part = std::min(n, c->fcap - r0);
  CUDA_TRY(cudaMemcpy(host, c->fhist + 4 * (size_t)r0, (size_t)part * 4 * sizeof(double), cudaMemcpyDeviceToHost));
  if (part < n)
    CUDA_TRY(cudaMemcpy(host + 4 * (size_t)part, c->fhist, (size_t)(n - part) * 4 * sizeof(double),
                        cudaMemcpyDeviceToHost));
  return CCM_OK;
}

ccm_status ccm_enable_kernel_timing(ccm_case c, int enable) {
  if (!c) return fail(CCM_E_INVALID, "null case");
  CUDA_TRY(cudaStreamSynchronize(c->st));
  collect_timing(c);
  c->timing = enable != 0;
  c->poisson_ms = 0.0;
  c->poisson_launches = 0;
  c->poisson_iters_timed = 0;
  c->launches = 0;
  return CCM_OK;
}

ccm_status ccm_kernel_timing(ccm_case c, double* poisson_ms, long long* poisson_launches, long long* poisson_iters,
                             long long* kernel_launches) {
  if (!c) return fail(CCM_E_INVALID, "null case");
  CUDA_TRY(cudaStreamSynchronize(c->st));
  collect_timing(c);
  if (poisson_ms) *poisson_ms = c->poisson_ms;
  if (poisson_launches) *poisson_launches = c->poisson_launches;
  if (poisson_iters) *poisson_iters = c->poisson_iters_timed;
  if (kernel_launches) *kernel_launches = c->launches;
  c->poisson_ms = 0.0;
  c->poisson_launches = 0;
  c->poisson_iters_timed = 0;
  c->launches = 0;
  return CCM_OK;
}

ccm_status ccm_solve_pressure(ccm_case c, const double* rhs_host, ccm_solve_stats* stats) {
  g_last_error.clear();
  if (!c || !rhs_host) return fail(CCM_E_INVALID, "null argument");
  if (!c->geometry) return fail(CCM_E_STATE, "set_geometry must come first");
  ccm_status s = upload(c, c->rhs_p, rhs_host);
  if (s != CCM_OK) return s;
  const dim3 b(64, 4);
  k_mask_cells<<<grid_of(c->g, b), b, 0, c->st>>>(c->g, c->co.act, c->rhs_p);
  k_mask_cells<<<grid_of(c->g, b), b, 0, c->st>>>(c->g, c->co.act, c->phi);
  CUDA_TRY(cudaMemsetAsync(c->ds, 0, sizeof(DevStats), c->st));
  if ((s = poisson_solve(c, c->phi, c->rhs_p)) != CCM_OK) return s;
  DevStats h{};
  if ((s = read_stats(c, h)) != CCM_OK) return s;
  int conv = h.conv_p, outer = c->cfg.precision == CCM_MIXED ? h.nrep : 1;
  if (c->mixed_host) {
    h.iters_p = c->mixed_last;
    h.rr_p = c->mixed_rr;
    h.bb_p = c->mixed_bb;
    conv = c->mixed_nconv == 0;
    outer = c->mixed_outer;
    c->mixed_total = 0;
    c->mixed_nconv = 0;
    c->mixed_host = false;
  }
  if (stats) {
    stats->iters = h.iters_p;
    stats->outer = outer;
    stats->rel_res = h.bb_p > 0 ? sqrt(h.rr_p / h.bb_p) : 0.0;
    stats->converged = conv;
  }
  if (!conv) return fail(CCM_E_NOT_CONVERGED, "Poisson solve reached its iteration limit");
  return CCM_OK;
}

}  // extern "C"
