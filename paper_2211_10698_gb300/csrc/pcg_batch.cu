// Batched Poisson solves (Eq. pm_poisson) of independent cases in one cooperative launch: the
// FP64 CG on the Jacobi-scaled system of pcg_scaled.cu, and the mixed-precision solve of
// pcg_mixed.cu (FP32 CG with FP64 residual replacements).
//
// Block b serves case block_case[b]: each case owns a contiguous range of blocks, sized by
// the host to its expected work, and reduces over its own blocks only, in the same fixed
// order as a single solve.  Every block passes the same grid barriers: each iteration has
// two slots separated by barriers, and a case fills them according to where it is.  After
// the first barrier every block counts the blocks whose case is still working (the same
// count in every block), and the launch ends when none is.
//
// Mixed solve, per case:
//   ITERATE  slot 1: vector update A;   slot 2: w = K~ r and its sums;  then the scalars and
//            the replacement test (FP32 residual fallen by `drop`, a loss of positivity, or
//            the iteration limit)
//   REPLACE  slot 1: x += D^-1/2 e / sigma;  slot 2: the FP64 residual and its norms; then the
//            convergence test on ||b - K x|| and the new normalisation sigma
//   FRESH    slot 1: r = sigma D^-1/2 (b - K x), w = K~ r and their sums (reduced after the
//            first barrier);  slot 2: p, K~ p formed and (p, K~ p) summed; then alpha
//   DONE     idle
// The first pass starts in REPLACE with e = 0.
#include "pcg_common.cuh"

namespace ccm {

namespace {

constexpr int kGroup = 1;  // cells per thread whose loads k_sc_batch issues together (two would spill)

// Cell range of this block within its case.
struct CaseRange {
  int t0, t1;
  __device__ CaseRange(int ncell, int lb, int nbc) {
    t0 = (int)((long long)ncell * lb / nbc);
    t1 = (int)((long long)ncell * (lb + 1) / nbc);
  }
};

// Number of blocks whose flag is set (same value in every block; read after a barrier).
__device__ __forceinline__ int count_running(const int* running, int nb, int* s_count) {
  if (threadIdx.x < 32) {
    int c = 0;
    for (int b = threadIdx.x; b < nb; b += 32) c += __ldcg(&running[b]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if (threadIdx.x == 0) *s_count = c;
  }
  __syncthreads();
  return *s_count;
}

__device__ __forceinline__ void publish(double* partials, int nb, const double* v, int nv) {
  if (threadIdx.x == 0)
    for (int q = 0; q < nv; ++q) partials[(size_t)q * nb + blockIdx.x] = v[q];
}

// Rows of the partials: sums published before the first barrier of an iteration use rows 0-1,
// those published before the second use rows 2-4, so a block that runs ahead never writes
// a row that another block of its case may still be reading.
constexpr int kRow1 = 0, kRow2 = 2;

// ---------------------------------------------------------------------------------------
// FP64 CG on the scaled system, batched.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kPcgThreads, 2) k_sc_batch(const ScaledBatchEntry* __restrict__ cases,
                                                             const int* __restrict__ block_case, BatchControl ctl) {
  __shared__ double red[4][kPcgThreads];
  __shared__ double bsum[8];
  __shared__ double gsum[8];
  __shared__ double sc_alpha, sc_beta, sc_igamma, sc_ialpha, sc_rr, sc_bb;
  __shared__ int sc_it, sc_stop, s_count;
  unsigned int target = 0;
  const int NB = gridDim.x;
  const ScaledBatchEntry& E = cases[block_case[blockIdx.x]];
  const ScaledSolve& a = E.a;
  const Geom g = a.g;
  const int nx = g.nx, P = g.pitch;
  const int lb = blockIdx.x - E.block0, nbc = E.nblocks;
  const CaseRange ch(g.nx * g.ny, lb, nbc);
  const int first = ch.t0 + threadIdx.x, stride = blockDim.x;
  const int kdummy = (int)g.idx(0, 0);
  const KRow<double> K{a.cu, a.cv, a.dk, a.kind, a.creg_x, a.creg_y, a.dreg, (size_t)P};
  const int8_t* __restrict__ kinds = a.kinds;
  const double* __restrict__ cus = a.cus;
  const double* __restrict__ cvs = a.cvs;
  const double* __restrict__ sd = a.sd;
  const double dreg = a.dreg;
  double* __restrict__ xs = a.xs;
  double* __restrict__ r = a.r;
  double* __restrict__ w = a.w;
  double* __restrict__ p = a.p;
  double* __restrict__ s = a.s;

  auto phase_b = [&](double (&v)[4]) {
    CellWalk cw(first, stride, ch.t1, nx);
    Group<kGroup> gr;
    while (next_group(cw, g, kdummy, gr)) {
      int8_t km[kGroup];
      double rc[kGroup], rw[kGroup], re[kGroup], rs[kGroup], rn[kGroup];
      double cw[kGroup], ce[kGroup], cs[kGroup], cn[kGroup];
#pragma unroll
      for (int m = 0; m < kGroup; ++m) {
        const int k = gr.k[m];
        km[m] = kinds[k];
        rc[m] = r[k];
        rw[m] = r[k - 1];
        re[m] = r[k + 1];
        rs[m] = r[k - P];
        rn[m] = r[k + P];
        cw[m] = cus[k];
        ce[m] = cus[k + 1];
        cs[m] = cvs[k];
        cn[m] = cvs[k + P];
      }
#pragma unroll
      for (int m = 0; m < kGroup; ++m) {
        if (!gr.v[m]) continue;
        const int k = gr.k[m];
        // the scaled coefficient arrays hold the constant stencil on uniform rows and zeros on
        // inactive ones, so one branch-free row serves every cell: a warp never runs two FP64
        // paths (an FP64 warp instruction costs the same however few lanes are active)
        const double wk = rc[m] - cw[m] * rw[m] - ce[m] * re[m] - cs[m] * rs[m] - cn[m] * rn[m];
        if (km[m] != 1) {
          const double dk = km[m] == 2 ? sd[k] * sd[k] : 1.0;
          v[1] += (dk - dreg) * (rc[m] * rc[m]);
        }
        w[k] = wk;
        v[0] += rc[m] * rc[m];
        v[2] += wk * rc[m];
      }
    }
  };

  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (CellWalk cw(first, stride, ch.t1, nx); cw.ok(); cw.next()) {
    const size_t k = g.idx(cw.i, cw.j);
    const double bk = a.b[k];
    const double rk = bk - K(a.x, k);
    xs[k] = sd[k] * a.x[k];
    r[k] = a.isd[k] * rk;
    p[k] = 0.0;
    s[k] = 0.0;
    v[3] += bk * bk;
  }
  bool ok = grid_sync(ctl.bar, target);
  if (ok) {
    phase_b(v);
    block_sum_warps<4>(v, red, bsum);
    publish(ctl.partials, NB, bsum, 4);
    ok = grid_sync(ctl.bar, target);
  }
  if (ok) {
    double t[4];
    range_sum<4>(ctl.partials, NB, E.block0, nbc, t, gsum);
    if (threadIdx.x == 0) {
      const double gamma = t[0], delta = t[2];
      sc_rr = dreg * t[0] + t[1];
      sc_bb = t[3];
      sc_it = 0;
      sc_stop = (sc_bb == 0.0 || sc_rr <= a.tol * a.tol * sc_bb) ? 1 : (a.max_iter <= 0 ? 2 : 0);
      if (sc_stop == 0) {
        sc_igamma = recip_newton(gamma);
        sc_alpha = gamma * recip_newton(delta);
        sc_ialpha = delta * sc_igamma;
        sc_beta = 0.0;
      }
    }
    __syncthreads();
  }
  while (ok) {
    const bool run = sc_stop == 0;
    if (run) {
      const double al = sc_alpha, be = sc_beta;
      CellWalk cw(first, stride, ch.t1, nx);
      Group<kGroup> gr;
      while (next_group(cw, g, kdummy, gr)) {
        double pm[kGroup], rm[kGroup], wm[kGroup], sm[kGroup], xm[kGroup];
#pragma unroll
        for (int m = 0; m < kGroup; ++m) {
          const int k = gr.k[m];
          pm[m] = p[k];
          rm[m] = r[k];
          wm[m] = w[k];
          sm[m] = s[k];
          xm[m] = xs[k];
        }
#pragma unroll
        for (int m = 0; m < kGroup; ++m) {
          if (!gr.v[m]) continue;
          const int k = gr.k[m];
          const double pk = rm[m] + be * pm[m];
          const double sk = wm[m] + be * sm[m];
          p[k] = pk;
          s[k] = sk;
          xs[k] = xm[m] + al * pk;
          r[k] = rm[m] - al * sk;
        }
      }
    }
    if (threadIdx.x == 0) ctl.running[blockIdx.x] = run ? 1 : 0;
    if (!grid_sync(ctl.bar, target)) { ok = false; break; }
    if (count_running(ctl.running, NB, &s_count) == 0) break;
    if (run) {
      v[0] = v[1] = v[2] = 0.0;
      phase_b(v);
      const double v3[3] = {v[0], v[1], v[2]};
      block_sum_warps<3>(v3, red, bsum);
      publish(ctl.partials, NB, bsum, 3);
    }
    if (!grid_sync(ctl.bar, target)) { ok = false; break; }
    if (run) {
      double t[3];
      range_sum<3>(ctl.partials, NB, E.block0, nbc, t, gsum);
      if (threadIdx.x == 0) {
        const double gamma = t[0], delta = t[2];
        sc_rr = dreg * t[0] + t[1];
        sc_it += 1;
        sc_stop = sc_rr <= a.tol * a.tol * sc_bb ? 1 : (sc_it >= a.max_iter ? 2 : 0);
        if (sc_stop == 0) {
          const double beta = gamma * sc_igamma;
          const double den = delta - beta * gamma * sc_ialpha;
          const double ig = recip_newton(gamma);
          sc_beta = beta;
          sc_alpha = gamma * recip_newton(den);
          sc_ialpha = den * ig;
          sc_igamma = ig;
        }
      }
      __syncthreads();
    }
  }
  for (CellWalk cw(first, stride, ch.t1, nx); cw.ok(); cw.next()) {
    const size_t k = g.idx(cw.i, cw.j);
    a.x[k] = a.isd[k] * xs[k];
  }
  if (lb == 0 && threadIdx.x == 0) {
    const bool conv = ok && sc_stop == 1;
    a.out.iters[0] = ok ? sc_it : 0;
    a.out.rr[0] = ok ? sc_rr : 0.0;
    a.out.bb[0] = ok ? sc_bb : 0.0;
    a.out.converged[0] = conv ? 1 : 0;
    if (a.out.total && ok) a.out.total[0] += sc_it;
    if (!conv && a.out.nconv) a.out.nconv[0] += 1;
  }
}

// ---------------------------------------------------------------------------------------
// Mixed-precision solve, batched.
// ---------------------------------------------------------------------------------------
enum { ST_ITERATE = 0, ST_REPLACE = 1, ST_FRESH = 2, ST_DONE = 3 };

__global__ void __launch_bounds__(kPcgThreads, 2) k_mixed_batch(const MixedBatchEntry* __restrict__ cases,
                                                                const int* __restrict__ block_case, BatchControl ctl) {
  __shared__ double red[3][kPcgThreads];
  __shared__ float wred[2][kPcgThreads / 32];
  __shared__ double dsum[8];
  __shared__ float fsum[8];
  __shared__ double sc_sigma, sc_rr, sc_bb, sc_rr_ref;
  __shared__ float sc_alpha, sc_beta, sc_pscale, sc_igamma, sc_ialpha, sc_gref, sc_gfresh;
  __shared__ int sc_state, sc_it, sc_stop, sc_nrep, sc_rep_it, sc_keep, sc_restart, sc_final, sc_init, s_count;
  unsigned int target = 0;
  const int NB = gridDim.x;
  const MixedBatchEntry& E = cases[block_case[blockIdx.x]];
  const MixedSolve& A = E.a;
  const ScaledSolve& d = A.d;
  const Geom g = d.g;
  const int nx = g.nx, P = g.pitch;
  const int lb = blockIdx.x - E.block0, nbc = E.nblocks;
  const CaseRange ch(g.nx * g.ny, lb, nbc);
  const int first = ch.t0 + threadIdx.x, stride = blockDim.x;
  // the FP32 phases work on aligned quads of the case's arrays (see QuadOpsF32)
  const Quads Q(g);
  const int u0 = (int)((long long)Q.nquad * lb / nbc), u1 = (int)((long long)Q.nquad * (lb + 1) / nbc);
  const QuadOpsF32 ops{d.kinds, A.cus32, A.cvs32, (float)d.ax, (float)d.ay, P};
  const KRow<double> K{d.cu, d.cv, d.dk, d.kind, d.creg_x, d.creg_y, d.dreg, (size_t)P};
  const double* __restrict__ isd = d.isd;
  double* __restrict__ x = d.x;
  double* __restrict__ r64 = d.r;
  float* __restrict__ r = A.r;
  float* __restrict__ w = A.w;
  float* __restrict__ p = A.p;
  float* __restrict__ s = A.s;
  float* __restrict__ e = A.e;
  const double tol2 = d.tol * d.tol;

  if (threadIdx.x == 0) {
    sc_state = ST_REPLACE;
    sc_init = 1;
    sc_sigma = 0.0;
    sc_bb = 0.0;
    sc_igamma = 1.0f;
    sc_pscale = 1.0f;
    sc_it = sc_stop = sc_nrep = sc_keep = sc_restart = sc_final = 0;
    sc_rep_it = -1000;
  }
  __syncthreads();
  bool ok = true;
  while (ok) {
    const int st = sc_state;
    // ---- slot 1
    if (st == ST_ITERATE) {
      const float al = sc_alpha, be = sc_beta;
      const bool keep = sc_keep != 0;
      for (int u = u0 + threadIdx.x; u < u1; u += blockDim.x) ops.update(p, r, w, s, e, Q.k(u), al, be, keep);
    } else if (st == ST_REPLACE) {
      if (sc_init) {
        const float4 z = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        for (int u = u0 + threadIdx.x; u < u1; u += blockDim.x) {
          const int k0 = Q.k(u);
          st4(p, k0, z);
          st4(s, k0, z);
          st4(e, k0, z);
        }
      } else {
        const double isig = 1.0 / sc_sigma;
        for (int u = u0 + threadIdx.x; u < u1; u += blockDim.x) quad_fold(x, isd, e, Q.k(u), isig, true);
      }
    } else if (st == ST_FRESH) {
      // r = sigma r64 (FP32), w = K~ r, sums (r, r), (w, r)
      float v[2] = {0.0f, 0.0f};
      const double sig = sc_sigma;
      for (int u = u0 + threadIdx.x; u < u1; u += blockDim.x) ops.stencil(r, w, r64, sig, Q.k(u), v);
      block_sum_f32<2>(v, wred, fsum);
      const double dv[2] = {(double)fsum[0], (double)fsum[1]};
      publish(ctl.partials + kRow1 * NB, NB, dv, 2);
    }
    if (threadIdx.x == 0) ctl.running[blockIdx.x] = st != ST_DONE ? 1 : 0;
    if (!grid_sync(ctl.bar, target)) { ok = false; break; }
    if (count_running(ctl.running, NB, &s_count) == 0) break;
    if (st == ST_FRESH) {
      double t[2];
      range_sum<2>(ctl.partials + kRow1 * NB, NB, E.block0, nbc, t, dsum);
      if (threadIdx.x == 0) {
        const float gamma = (float)t[0];
        sc_gref = gamma;
        sc_gfresh = gamma;
        if ((sc_it == 0 && sc_nrep == 0) || sc_restart) {
          sc_beta = 0.0f;
          sc_restart = 0;
        } else {
          sc_beta = gamma * sc_igamma;
        }
      }
      __syncthreads();
    }
    // ---- slot 2
    if (st == ST_ITERATE) {
      float v[2] = {0.0f, 0.0f};
      for (int u = u0 + threadIdx.x; u < u1; u += blockDim.x) ops.stencil(r, w, nullptr, 0.0, Q.k(u), v);
      block_sum_f32<2>(v, wred, fsum);
      const double dv[2] = {(double)fsum[0], (double)fsum[1]};
      publish(ctl.partials + kRow2 * NB, NB, dv, 2);
    } else if (st == ST_REPLACE) {
      double v[3] = {0.0, 0.0, 0.0};
      for (CellWalk cw(first, stride, ch.t1, nx); cw.ok(); cw.next()) {
        const size_t k = g.idx(cw.i, cw.j);
        const double bk = d.b[k];
        const double rk = bk - K(x, k);
        const double rs = isd[k] * rk;
        r64[k] = rs;
        v[0] += rs * rs;
        v[1] += rk * rk;
        v[2] += bk * bk;
      }
      block_sum_warps<3>(v, red, dsum);
      publish(ctl.partials + kRow2 * NB, NB, dsum, 3);
    } else if (st == ST_FRESH) {
      // p = r + beta' p, s = w + beta' s with beta' = beta sigma_new / sigma_old, and (p, s)
      const float be = sc_beta * sc_pscale;
      float v[1] = {0.0f};
      for (int u = u0 + threadIdx.x; u < u1; u += blockDim.x) v[0] += ops.form(p, r, w, s, Q.k(u), be);
      block_sum_f32<1>(v, wred, fsum);
      const double dv[1] = {(double)fsum[0]};
      publish(ctl.partials + kRow2 * NB, NB, dv, 1);
    }
    if (!grid_sync(ctl.bar, target)) { ok = false; break; }
    // ---- after the second barrier: scalars and the next state
    if (st == ST_ITERATE) {
      double t[2];
      range_sum<2>(ctl.partials + kRow2 * NB, NB, E.block0, nbc, t, dsum);
      if (threadIdx.x == 0) {
        const float gamma = (float)t[0], delta = (float)t[1];
        sc_it += 1;
        sc_keep = 0;
        const double ratio = (double)gamma / (double)sc_gref;
        int replace = (ratio <= A.drop * A.drop || sc_rr_ref * ratio <= tol2 * sc_bb) ? 1 : 0;
        if (!replace) {
          const float beta = gamma * sc_igamma;
          const float den = delta - beta * gamma * sc_ialpha;
          if (den > 0.0f && den < INFINITY) {
            sc_beta = beta;
            sc_alpha = gamma / den;
            sc_igamma = 1.0f / gamma;
            sc_ialpha = 1.0f / sc_alpha;
          } else {
            replace = 1;
            sc_restart = 1;
          }
        }
        if (!replace && sc_it >= d.max_iter) {
          replace = 1;
          sc_final = 1;
        }
        if (replace) {
          sc_nrep += 1;
          if (sc_it - sc_rep_it < 3) sc_restart = 1;
          sc_rep_it = sc_it;
          sc_state = ST_REPLACE;
        }
      }
    } else if (st == ST_REPLACE) {
      double t[3];
      range_sum<3>(ctl.partials + kRow2 * NB, NB, E.block0, nbc, t, dsum);
      if (threadIdx.x == 0) {
        if (sc_init) sc_bb = t[2];
        sc_rr = t[1];
        sc_rr_ref = t[1];
        const double old = sc_init ? 0.0 : sc_sigma;
        sc_sigma = t[0] > 0.0 ? 1.0 / sqrt(t[0]) : 1.0;
        const double c = old > 0.0 ? sc_sigma / old : 0.0;
        sc_pscale = (float)c;
        sc_igamma = (float)((double)sc_igamma / (c * c + (c == 0.0)));
        sc_init = 0;
        if (sc_bb == 0.0 || sc_rr <= tol2 * sc_bb) {
          sc_stop = 1;
          sc_state = ST_DONE;
        } else if (sc_final) {
          sc_stop = 2;
          sc_state = ST_DONE;
        } else {
          sc_state = ST_FRESH;
        }
      }
    } else if (st == ST_FRESH) {
      double t[1];
      range_sum<1>(ctl.partials + kRow2 * NB, NB, E.block0, nbc, t, dsum);
      if (threadIdx.x == 0) {
        sc_alpha = sc_gfresh / (float)t[0];
        sc_igamma = 1.0f / sc_gfresh;
        sc_ialpha = 1.0f / sc_alpha;
        sc_keep = 1;
        sc_state = ST_ITERATE;
      }
    }
    __syncthreads();
  }
  if (lb == 0 && threadIdx.x == 0) {
    const bool conv = ok && sc_stop == 1;
    d.out.iters[0] = ok ? sc_it : 0;
    d.out.rr[0] = ok ? sc_rr : 0.0;
    d.out.bb[0] = ok ? sc_bb : 0.0;
    d.out.converged[0] = conv ? 1 : 0;
    if (d.out.total && ok) d.out.total[0] += sc_it;
    if (!conv && d.out.nconv) d.out.nconv[0] += 1;
    if (A.replacements) A.replacements[0] = sc_nrep;
  }
}

}  // namespace

int batch_scaled_blocks() {
  int dev = 0, sms = 0, per1 = 0, per2 = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per1, k_sc_batch, kPcgThreads, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per2, k_mixed_batch, kPcgThreads, 0);
  int per = per1 < per2 ? per1 : per2;
  per = per > 2 ? 2 : (per < 1 ? 1 : per);
  return sms * per;
}

cudaError_t run_scaled_batch(const ScaledBatchEntry* dev_cases, const int* dev_block_case, BatchControl ctl,
                             int blocks, cudaStream_t st) {
  cudaMemsetAsync(ctl.bar.count, 0, sizeof(unsigned int) * kBarWords, st);
  void* params[] = {(void*)&dev_cases, (void*)&dev_block_case, &ctl};
  return cudaLaunchCooperativeKernel((const void*)k_sc_batch, blocks, kPcgThreads, params, 0, st);
}

cudaError_t run_mixed_batch(const MixedBatchEntry* dev_cases, const int* dev_block_case, BatchControl ctl,
                            int blocks, cudaStream_t st) {
  cudaMemsetAsync(ctl.bar.count, 0, sizeof(unsigned int) * kBarWords, st);
  void* params[] = {(void*)&dev_cases, (void*)&dev_block_case, &ctl};
  return cudaLaunchCooperativeKernel((const void*)k_mixed_batch, blocks, kPcgThreads, params, 0, st);
}

}  // namespace ccm
