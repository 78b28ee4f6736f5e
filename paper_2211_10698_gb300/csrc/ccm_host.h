// Host-side declarations shared by the libccm translation units: argument bundles of the
// solver kernels and the launchers each .cu file provides.
#pragma once

#include <string>

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

// One case of a batched Poisson solve and the contiguous range of blocks that serves it.
template <class T>
struct BatchEntry {
  PoissonSolve<T> a;  // partials, bar of the entry are unused (the batch has its own)
  int block0, nblocks;
};

struct BatchControl {
  double* partials;  // 6 values x blocks
  int* running;      // per block: its case is still iterating
  Barrier bar;
};

struct HelmholtzSolve {
  Coefs c;
  Geom g;
  Bc bc;
  Phys ph;
  double* xu;
  double* xv;
  const double* bu;
  const double* bv;
  double *ru, *rv, *zu, *zv, *pu, *pv, *qu, *qv;
  double tol;
  int max_iter;
  double* partials;
  Barrier bar;
  PcgOut out;
};

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
  double tol;
  int max_iter;
  int zero_mean;
  double n_act;
};
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
void launch_residual64(const Coefs& c, const Geom& g, const double* x, const double* b, float* r32, double* partials,
                       double* out2, cudaStream_t st);
void launch_add_correction(const Geom& g, const int8_t* act, double* x, const float* d, cudaStream_t st);
void launch_diagnostics(const Coefs& c, const Geom& g, const double* Vu, const double* Vv, const double* u,
                        const double* v, double* partials, double* out, cudaStream_t st);

// pcg.cu
int pcg_partials_needed();
bool cheb_degree_supported(int k);
template <class T>
cudaError_t run_poisson_pcg(PoissonSolve<T> a, cudaStream_t st);
int batch_blocks();
template <class T>
cudaError_t run_poisson_batch(const PoissonSolve<T>* host_cases, int ncase, const BatchEntry<T>* dev_cases,
                              const int* dev_block_case, BatchControl ctl, int blocks, cudaStream_t st);

// api.cu: pieces of one step for the batch driver
ccm_status case_stage_predict(ccm_case c);
void case_stage_project(ccm_case c);
ccm_status case_finish(ccm_case c, ccm_step_stats* stats);
bool case_is_mixed(ccm_case c);
cudaStream_t case_stream(ccm_case c);
size_t case_cells(ccm_case c);
int case_nx(ccm_case c);
void case_poisson_fp64(ccm_case c, PoissonSolve<double>* a);
void case_poisson_fp32(ccm_case c, PoissonSolve<float>* a);
ccm_status case_mixed_residual(ccm_case c, double* host2);
void case_mixed_correct(ccm_case c);
void case_mixed_account(ccm_case c, long long inner, int outer, double rr, double bb, bool converged);
int* case_inner_iters_dev(ccm_case c);
cudaError_t run_helmholtz_pcg(HelmholtzSolve a, cudaStream_t st);

}  // namespace ccm
