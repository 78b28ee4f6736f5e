// Host-side declarations shared by the libccm translation units: argument bundles of the
// solver kernels and the launchers each .cu file provides.
#pragma once
#include <nvtx3/nvToolsExt.h>

#include <functional>
#include <string>
#include <vector>

#include "ccm_internal.cuh"

namespace ccm {

struct CapPtrs {
  double* a[27];
};

// Writable view of the derived coefficients (Coefs is the read-only kernel view).
struct CoefPtrs {
  int8_t* role_u;
  int8_t* role_v;
  int8_t* act;
  int8_t* kind;           // Poisson row kind: 0 inactive, 1 uncut, 2 cut
  double *cu, *cv, *invdk, *diagk, *gfu, *gfv, *pfac, *massu, *massv;
  double *wxx, *wyy, *wxa, *wxb;
  double *invdhu, *invdhv, *liftu, *liftv;
  float *cu32, *cv32, *invdk32, *diagk32;
  // symmetric Jacobi scaling of the Poisson matrix, D^-1/2 K D^-1/2 (unit diagonal):
  // sqrt(d), 1/sqrt(d) per cell, the scaled face coefficients, and the scaled row kind
  // (1: the cell and its four neighbours are uncut, so the scaled row is a constant stencil)
  double *sdk, *isdk, *cus, *cvs;
  float *isdk32, *cus32, *cvs32;
  int8_t* kinds;
};

// Where a solver kernel reports: iterations, final squared residual and right-hand side
// norms, convergence flag; `total` and `nconv` accumulate over calls (may be null).
struct PcgOut {
  int* iters;
  double* rr;
  double* bb;
  int* converged;
  long long* total;
  int* nconv;
};

template <class T>
struct PoissonSolve {
  Geom g;
  const T* cu;
  const T* cv;
  const T* dk;            // diagonal of K
  const T* invd;          // 1 / diagonal
  const int8_t* kind;     // 0 inactive (identity row), 1 uncut (constant coefficients), 2 cut
  double creg_x, creg_y;  // face coefficients of an uncut cell: hy/hx and hx/hy
  double dreg, invd_reg;  // their diagonal 2 (creg_x + creg_y) and its inverse
  T* x;
  T* b;
  T* r;
  T* z;
  T* p0;
  T* p1;
  T* q;
  T* z2;          // second z buffer (Chebyshev)
  T* w1;          // Chebyshev increment
  int cheb;       // 1: Jacobi; k > 1: k-step Chebyshev preconditioner
  double tol;
  int max_iter;
  int zero_mean;
  double n_act;
  double* partials;
  Barrier bar;
  PcgOut out;
};

// Poisson solve on the symmetrically scaled system (FP64 Jacobi-PCG in exact arithmetic):
// x~ = D^1/2 x, b~ = D^-1/2 b, K~ x~ = b~ by CG, then x = D^-1/2 x~.
struct ScaledSolve {
  Geom g;
  const double *cu, *cv, *dk;   // K itself, for the initial residual b - K x
  const int8_t* kind;
  const double *sd, *isd, *cus, *cvs;
  const int8_t* kinds;
  double creg_x, creg_y, dreg;  // uncut-cell constants of K
  double ax, ay;                // and of K~: creg / dreg
  double* x;                    // in: warm start; out: solution
  const double* b;
  double *xs, *r, *w, *p, *s;   // scaled iterate, residual, K~ r, direction, K~ p
  double tol;
  int max_iter;
  double* partials;
  Barrier bar;
  PcgOut out;
};
cudaError_t run_poisson_scaled(const ScaledSolve& a, cudaStream_t st);

// The same solve with one grid barrier per iteration (pcg_fused.cu): 2-D tiles, the ring of
// each tile recomputed by its block, r, w, s double-buffered.  a.xs and a.p are used, a.r,
// a.w, a.s are not.
// Words of the fixed-point reduce-barrier (pcg_fixed.cuh): three rotating buffers of kFxWords
// 64-bit words, each word on its own 128-byte line.
constexpr int kFxWords = 16;
constexpr int kFxStride = 16;
constexpr int kFxAccWords = 3 * kFxWords * kFxStride;

struct FusedSolve {
  ScaledSolve a;
  unsigned long long* fxacc;  // kFxAccWords words (cleared by the kernel itself)
  int fx_fallback_every;      // tests only: every k-th reduction takes the FP64 fallback (0: on overflow only)
  double* R[2];
  double* W[2];
  double* S[2];
  int TX, TY, nbx, ntiles;  // tile plan; TX = 0 lets the launcher choose
  int list_cap;             // set by the launcher: entries of the per-tile list of non-uniform cells
  int resident;             // 1: each tile keeps its vectors in shared memory (k_pcg_poisson_f2)
  int lcache;               // set by the launcher (resident): the listed cells' coefficients cached in shared memory
};
cudaError_t run_poisson_fused(FusedSolve f, cudaStream_t st);
void fused_tiles(int nx, int ny, int blocks, int* TX, int* TY, int* nbx, int* ntiles);
int fused_blocks();
size_t fused_resident_smem(int TX, int TY, bool cache);
bool fused_resident_fits(int TX, int TY, int ntiles, bool cache);
int fused_resident_fit(int TX, int TY, int ntiles);
bool fused_resident_ok(int TX, int TY, int ntiles);

// The same solve for small grids inside one thread-block cluster (pcg_cluster.cu).
struct ClusterSolve {
  ScaledSolve a;  // partials and bar unused
  int nmax;       // set by the launcher: cells of the largest band
};
size_t cluster_smem_bytes(int nx, int ny, int C);
// C CTAs (1..16); cudaErrorInvalidConfiguration if the grid or the GPU does not allow it
cudaError_t run_poisson_cluster(ClusterSolve f, int C, cudaStream_t st);

// Launch-shape autotuner (tune.cu).
struct TilePlan {
  int TX, TY, nbx, ntiles;
  int resident;  // 1: the tiles keep their vectors in shared memory (k_pcg_poisson_f2)
};
struct TuneResult {
  TilePlan plan;     // FP64 one-barrier solve (TX = 0: not tuned)
  int mixed_blocks;  // mixed one-launch solve (0: not tuned)
  int cluster;       // FP64 solve inside one cluster of this many CTAs (0: not chosen)
  TilePlan mixed1;   // mixed solve with one barrier per iteration (TX = 0: not chosen)
};
std::vector<TilePlan> fused_plan_candidates(int nx, int ny, int blocks);
std::vector<int> mixed_block_candidates(int blocks);
std::vector<int> cluster_candidates(int nx, int ny);
bool tune_cache_get(int nx, int ny, int precision, int precond, int degree, int blocks, TuneResult* r);
void tune_cache_put(int nx, int ny, int precision, int precond, int degree, int blocks, const TuneResult& r);
// Times launch(k) for k = 0 .. n-1 with CUDA events on st (after one untimed launch(0));
// candidates whose launch returns cudaErrorInvalidConfiguration are skipped.  best = the
// fastest index, ms = the times (-1 where skipped).
cudaError_t time_launches(int n, const std::function<cudaError_t(int)>& launch, cudaStream_t st, int* best,
                          std::vector<float>* ms);

// Mixed-precision solve of the same system: FP32 CG on K~ with FP64 residual replacements.
// d.r serves as the FP64 residual; d.xs, d.w, d.p, d.s are unused.
struct MixedSolve {
  ScaledSolve d;
  const float *cus32, *cvs32;
  float *r, *w, *p, *s, *e;   // FP32 residual, K~ u, direction, K~ p, correction
  int cheb;                   // 1: Jacobi (u = r); k > 1: k-step Chebyshev preconditioner
  float *zA, *zB, *dch;       // Chebyshev iterates and direction (cheb > 1)
  float* fpartials;           // 4 x blocks
  double drop;                // FP32 residual reduction that triggers a replacement
  int* replacements;          // out: FP64 replacements made
  int blocks;                 // single-case launch size (0: two blocks per SM)
};
int mixed_blocks();
cudaError_t run_poisson_mixed(const MixedSolve& a, cudaStream_t st);

// Initial guess of the Poisson solve by projection onto earlier solutions (guess.cu).  X and
// KX hold up to kGuessMax K-orthonormal vectors of n doubles each (and their images under K).
constexpr int kGuessMax = 32;
size_t guess_scratch_doubles();
// phi = sum_{i < nb} (X_i, rhs) X_i
void launch_guess_project(const double* X, size_t n, int nb, const double* rhs, double* phi, double* scratch,
                          cudaStream_t st);
// X_nb, KX_nb hold a new solution and its image under K: K-orthonormalise them against X_0..X_{nb-1}
void launch_guess_append(double* X, double* KX, size_t n, int nb, double* scratch, cudaStream_t st);

// The same mixed solve with one grid barrier per FP32 iteration (pcg_mixed1.cu): 2-D tiles
// whose blocks recompute the band of width k (the preconditioner's degree; 1 for Jacobi)
// around their tile from the previous iteration's vectors and run the Chebyshev steps in
// shared memory.  m.d.x, m.d.b, m.d.r (FP64 residual), m.d.partials and the scalars of m are
// used; m's FP32 vectors are not.
struct Mixed1Solve {
  MixedSolve m;
  float* R[2];   // FP32 residual, double-buffered by iteration parity
  float* W[2];   // K~ u
  float* S[2];   // K~ p
  float *P, *U, *E;  // direction, preconditioned residual (Chebyshev), correction
  int TX, TY, nbx, ntiles;
  int resident;      // 1: the tile's vectors in shared memory (k_pcg_poisson_m2)
};
cudaError_t run_poisson_mixed1(Mixed1Solve f, cudaStream_t st);
size_t mixed1_smem(int TX, int TY, int cheb, int resident);
// Whether a tile plan of the one-barrier mixed solve fits the GPU at once (cooperative launch).
bool mixed1_plan_fits(int TX, int TY, int ntiles, int cheb, int resident);
// Tile plans of the one-barrier mixed solve that fit the GPU at once, resident ones first.
std::vector<TilePlan> mixed1_plan_candidates(int nx, int ny, int cheb);

// One case of a batched solve and its contiguous range of blocks (pcg_batch.cu).
struct ScaledBatchEntry {
  ScaledSolve a;  // partials and bar unused: the batch has its own
  int block0, nblocks;
};
struct MixedBatchEntry {
  MixedSolve a;
  int block0, nblocks;
};
void launch_scaling(const Geom& g, const CoefPtrs& o, cudaStream_t st);

// One case of a batched Poisson solve and the contiguous range of blocks that serves it.
template <class T>
struct BatchEntry {
  PoissonSolve<T> a;  // partials, bar of the entry are unused (the batch has its own)
  int block0, nblocks;
};

// Counters of the per-case barriers of k_mixed_batch, kCaseBarStride words apart.
constexpr int kCaseBarStride = 32;
struct BatchControl {
  double* partials;  // 6 values x blocks
  int* running;      // per block: its case is still iterating (two halves of gridDim.x)
  Barrier bar;
  unsigned int* case_bar = nullptr;  // k_mixed_batch: one barrier counter per case
  int ncases = 0;
};

// The Helmholtz operator of the predictor (Eq. pm_prediction, homogeneous part) as nine
// coefficients per unknown face, found by colour probing at set-up.  u-row (face (i, j)):
// 0 u(i,j), 1 u(i-1,j), 2 u(i+1,j), 3 u(i,j-1), 4 u(i,j+1), 5 v(i-1,j), 6 v(i,j), 7 v(i-1,j+1),
// 8 v(i,j+1).  v-row: 9 v(i,j), 10 v(i-1,j), 11 v(i+1,j), 12 v(i,j-1), 13 v(i,j+1), 14 u(i,j-1),
// 15 u(i+1,j-1), 16 u(i,j), 17 u(i+1,j).  Ghost reflections are folded into these; faces that
// are not unknowns get coefficient 0.
struct HelmCoefPtrs {
  double* a[18];
};
void launch_helmholtz_coefs(const Coefs& c, const Geom& g, const Bc& bc, const Phys& ph, double* eu, double* ev,
                            double* ou, double* ov, const HelmCoefPtrs& h, int* bad, cudaStream_t st);

// Helmholtz PCG on the coefficient form (pcg_helm.cu): single-reduction Jacobi CG over the
// unknown u and v faces.
struct HelmCSolve {
  Geom g;
  const int8_t* ru;
  const int8_t* rv;
  HelmCoefPtrs h;
  const double* invu;  // 1 / diagonal
  const double* invv;
  double *xu, *xv;
  const double *bu, *bv;
  double *rU, *rV, *zU, *zV, *wU, *wV, *pU, *pV, *sU, *sV;
  double tol;
  int max_iter;
  double* partials;
  Barrier bar;
  PcgOut out;
};
cudaError_t run_helmholtz_coef(const HelmCSolve& a, cudaStream_t st);
// One case of a batched explicit stage (operators.cu): its arrays for the step and its range
// of the launch's blocks (starts[] is the prefix over cases of stage_case_blocks()).
enum { STAGE_FILL_BC = 0, STAGE_PREDICT = 1, STAGE_DIVERGENCE = 2, STAGE_PROJECT = 3, STAGE_KINDS = 4 };
struct StageCase {
  Coefs c;
  Geom g;
  Bc bc;
  Phys ph;
  double *u, *v, *p;
  const double* phi;
  const double *cpu, *cpv;          // conv at the previous step (Adams-Bashforth)
  double *cnu, *cnv, *ru, *rv;      // conv now, the predictor's right-hand side
  double *ustar, *vstar, *div, *rhs;
  int first;                        // first step: conv^{n-1} := conv^n
  int gx;                           // blocks per padded row (stage_case_blocks)
};
int stage_case_blocks(const Geom& g, int* gx);
// extra: some case has a body acceleration or a body velocity (the predictor's extra terms)
cudaError_t launch_stage_batch(int kind, const StageCase* dev_cases, const int* dev_starts, int n, int blocks,
                               cudaStream_t st, bool extra = false);
struct HelmBatchEntry {
  HelmCSolve a;  // partials and bar unused: the batch has its own
  int block0, nblocks;
};
int batch_helm_blocks();
cudaError_t run_helm_batch(const HelmBatchEntry* dev_cases, const int* dev_block_case, BatchControl ctl, int blocks,
                           cudaStream_t st);

// What a solver outside api.cu needs from a case (read-only view).
struct CaseSolveView {
  Geom g;
  cudaStream_t st;
  const double* cu;
  const double* cv;
  const double* dk;
  const double* invd;
  const int8_t* kind;
  const int8_t* act;
  const double *sd, *isd, *cus, *cvs;  // symmetric Jacobi scaling (see ScaledSolve)
  const int8_t* kinds;
  int precond;
  double tol;
  int max_iter;
  int zero_mean;
  double n_act;
};
// The FP64 Poisson solve of a case on the scaled system, x and b in device memory, work
// vectors xs, r, w, p, s given by the caller (r must be zero on the ghost ring).
ScaledSolve scaled_solve_of(const CaseSolveView& v, double* x, const double* b, double* xs, double* r, double* w,
                            double* p, double* s);
// api.cu: false when the case has no geometry yet.
bool case_solve_view(ccm_case c, CaseSolveView* v);
// api.cu: the thread-local message returned by ccm_last_error.
void set_last_error(const char* msg);
inline void set_last_error(const std::string& msg) { set_last_error(msg.c_str()); }

// geometry.cu
cudaError_t launch_capacities(const ccm_geometry& geo, const Geom& g, double* const* caps_dev, cudaStream_t st);

// operators.cu
void launch_derive(const Geom& g, const Bc& bc, const Phys& ph, int literal, int pupdate, const CapPtrs& cp,
                   const CoefPtrs& o, cudaStream_t st);
void launch_fill_bc(const Geom& g, const Bc& bc, double* u, double* v, double scale, cudaStream_t st);
// periodic sides: the cells beyond them take their images' values (no-op otherwise)
void launch_wrap_cells(const Geom& g, double* p, cudaStream_t st);
void launch_cont(const Coefs& c, const Geom& g, const double* u, const double* v, double* out, cudaStream_t st);
void launch_pres(const Coefs& c, const Geom& g, const double* p, double* ou, double* ov, cudaStream_t st);
void launch_conv(const Coefs& c, const Geom& g, const double* u, const double* v, double* ou, double* ov,
                 cudaStream_t st);
void launch_visc(const Coefs& c, const Geom& g, const Bc& bc, const double* u, const double* v, double* ou, double* ov,
                 cudaStream_t st);
void launch_helmholtz(const Coefs& c, const Geom& g, const Bc& bc, const Phys& ph, const double* u, const double* v,
                      double* ou, double* ov, cudaStream_t st);
void launch_poisson(const Coefs& c, const Geom& g, const double* x, double* out, double* tmp, cudaStream_t st);
void launch_helmholtz_diag(const Coefs& c, const Geom& g, const Bc& bc, const Phys& ph, double* eu, double* ev,
                           double* ou, double* ov, double* du, double* dv, double* iu, double* iv, cudaStream_t st);
void launch_predictor_rhs(const Coefs& c, const Geom& g, const Bc& bc, const Phys& ph, const double* u, const double* v,
                          const double* p, const double* cpu, const double* cpv, double* cnu, double* cnv, double* ru,
                          double* rv, int first, cudaStream_t st);
void launch_divergence(const Coefs& c, const Geom& g, const Phys& ph, const double* u, const double* v, double* b,
                       double* rhs, cudaStream_t st);
void launch_project(const Coefs& c, const Geom& g, const double* phi, double* u, double* v, double* p, cudaStream_t st);
int diagnostics_partials(const Geom& g);
// The body's steady Dirichlet velocity (dterms.cu): h = cont(0, D), strain(0, D), visc(S(0, D));
// and D on the faces whose control volume holds no fluid (Dx, Dy null: zero).
void launch_body_dterms(const Geom& g, const Bc& bc, const CapPtrs& cp, const Coefs& c, const double* Dx,
                        const double* Dy, double* hd, double* sxxd, double* syyd, double* sxyd, double* vu,
                        double* vv, cudaStream_t st);
// f: the factor of a time-dependent body velocity D = f D0 at the level of u, v (1: steady)
void launch_inactive_to_body(const Geom& g, const int8_t* ru, const int8_t* rv, const double* Dx, const double* Dy,
                             double* u, double* v, cudaStream_t st, double f = 1.0);
// Force of the fluid on the body, out[4] = (Fp_x, Fp_y, Fv_x, Fv_y) (operators.cu); partials
// holds body_force_partials(g) doubles.
int body_force_partials(const Geom& g);
void launch_body_force(const Coefs& c, const Geom& g, const Phys& ph, const double* u, const double* v,
                       const double* p, double* partials, double* out, cudaStream_t st);
void launch_residual64(const Coefs& c, const Geom& g, const double* x, const double* b, float* r32, double* partials,
                       double* out2, cudaStream_t st);
void launch_add_correction(const Geom& g, const int8_t* act, double* x, const float* d, cudaStream_t st);
// fd: the factor of a time-dependent body velocity at the level of u, v (1: steady)
void launch_diagnostics(const Coefs& c, const Geom& g, const double* Vu, const double* Vv, const double* u,
                        const double* v, double* partials, double* out, cudaStream_t st, double fd = 1.0);

// pcg.cu
int pcg_partials_needed();
size_t pcg_float_partials_offset();  // in doubles, within a partials buffer of that size
bool cheb_degree_supported(int k);
template <class T>
cudaError_t run_poisson_pcg(PoissonSolve<T> a, cudaStream_t st);
int batch_blocks();
// pcg_batch.cu: blocks of a batched launch, and the two batched solves (ctl.partials holds
// 5 rows of blocks)
int batch_scaled_blocks();
int poisson_zero_mean_blocks();
cudaError_t project_zero_mean(const Geom& g, const int8_t* act, double* x, double* partials, double n_act,
                              cudaStream_t st);
cudaError_t run_scaled_batch(const ScaledBatchEntry* dev_cases, const int* dev_block_case, BatchControl ctl,
                             int blocks, cudaStream_t st);
cudaError_t run_mixed_batch(const MixedBatchEntry* dev_cases, const int* dev_block_case, BatchControl ctl,
                            int blocks, cudaStream_t st);
template <class T>
cudaError_t run_poisson_batch(const PoissonSolve<T>* host_cases, int ncase, const BatchEntry<T>* dev_cases,
                              const int* dev_block_case, BatchControl ctl, int blocks, cudaStream_t st);

// api.cu: pieces of one step for the batch driver
ccm_status case_finish(ccm_case c, ccm_step_stats* stats);
bool case_is_mixed(ccm_case c);
cudaStream_t case_stream(ccm_case c);
size_t case_cells(ccm_case c);
int case_nx(ccm_case c);
void case_poisson_fp64(ccm_case c, PoissonSolve<double>* a);
bool case_scaled_ok(ccm_case c);  // nonsingular: the scaled and mixed batched kernels apply
void case_scaled_fp64(ccm_case c, ScaledSolve* a);
void case_mixed_batch(ccm_case c, MixedSolve* a);
void case_helm_solve(ccm_case c, HelmCSolve* a);
void case_stage_case(ccm_case c, StageCase* e, int ahead);
int case_cur(ccm_case c);
unsigned long long case_serial(ccm_case c);  // unique per case (addresses can be reused)
bool case_has_extras(ccm_case c);            // a body acceleration or a body velocity is set
bool case_is_moving(ccm_case c);             // the body velocity has a time law (not batched)
long long case_nstep(ccm_case c);
void case_step_done(ccm_case c);
void case_poisson_fp32(ccm_case c, PoissonSolve<float>* a);
ccm_status case_mixed_project(ccm_case c, bool with_rhs);
ccm_status case_mixed_residual(ccm_case c, double* host2);
void case_mixed_correct(ccm_case c);
void case_mixed_account(ccm_case c, long long inner, int outer, double rr, double bb, bool converged);
int* case_inner_iters_dev(ccm_case c);

// Named NVTX range of one stage of a step (header-only NVTX: without a profiler attached the
// calls return at once), so that a timeline shows predictor, Helmholtz, Poisson and projection.
struct StageRange {
  explicit StageRange(const char* name) { nvtxRangePushA(name); }
  ~StageRange() { nvtxRangePop(); }
  StageRange(const StageRange&) = delete;
  StageRange& operator=(const StageRange&) = delete;
};

}  // namespace ccm
