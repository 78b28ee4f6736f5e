// Batched Poisson solves (Eq. pm_poisson) of independent cases in one cooperative launch: the
// FP64 CG on the Jacobi-scaled system of pcg_scaled.cu, and the mixed-precision solve of
// pcg_mixed.cu (FP32 CG with FP64 residual replacements).
//
// Block b serves case block_case[b]: each case owns a contiguous range of blocks, sized by
// the host to its expected work, and reduces over its own blocks only, in the same fixed
// order as a single solve.  The barriers are the case's own (a counter per case that only its
// blocks pass; a case on one block needs only the block barrier), so every case iterates at
// its own pace and its blocks leave the launch when it has converged.
//
// FP64 solve: two barriers per CG iteration, as in pcg_scaled.cu.
//
// Mixed solve: each case steps through slots, one barrier after each, according to where it
// is.  The barrier after a slot is the case's own (a counter per case that only its blocks
// pass), so every case iterates at its own pace and its blocks leave the launch when it is
// done; the host gives each case blocks in proportion to its expected work (cells x
// iterations), so that the cases finish together:
//   iteration      UPDATE (vector update A),
//                  CHEB x (degree - 1) (Chebyshev steps from z1 = r / theta; none with Jacobi),
//                  APPLY (w = K~ u and its sums), then the scalars and the replacement test
//                  (FP32 residual fallen by `drop`, a loss of positivity, or the limit)
//   replacement    FOLD (x += D^-1/2 e / sigma), RESID (FP64 residual and its norms; the
//                  convergence test and the new normalisation sigma), FRESH (r = sigma r64;
//                  Jacobi: also w = K~ r and its sums; Chebyshev: then CHEB and APPLY),
//                  FORM (p, K~ p formed and (p, K~ p) summed; then alpha)
//   DONE           the case's blocks leave
// The first pass starts in FOLD with p = s = e = 0.
#include "batch_common.cuh"
#include "pcg_quad.cuh"

namespace ccm {

namespace {

constexpr int kGroup = 1;  // cells per thread whose loads k_sc_batch issues together (two would spill)

// ---------------------------------------------------------------------------------------
// FP64 CG on the scaled system, batched.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kPcgThreads, 2) k_sc_batch(const ScaledBatchEntry* __restrict__ cases,
                                                             const int* __restrict__ block_case, BatchControl ctl) {
  __shared__ double red[4][kPcgThreads];
  __shared__ double bsum[8];
  __shared__ double gsum[8];
  __shared__ double sc_alpha, sc_beta, sc_igamma, sc_den, sc_rr, sc_bb;
  __shared__ double sc_igamma_next, sc_den_next;
  __shared__ int sc_it, sc_stop;
  unsigned int target = 0;
  const int NB = gridDim.x;
  __shared__ __align__(16) unsigned char s_entry[sizeof(ScaledBatchEntry)];
  const ScaledBatchEntry& E = stage_entry(cases, block_case, s_entry);
  const ScaledSolve& a = E.a;
  const Geom g = a.g;
  const int nx = g.nx, P = g.pitch;
  const int lb = blockIdx.x - E.block0, nbc = E.nblocks;
  const CaseRange ch(g.nx * g.ny, lb, nbc);
  const int first = ch.t0 + threadIdx.x, stride = blockDim.x;
  const int kdummy = (int)g.idx(0, 0);
  const KRow<double> K{a.cu, a.cv, a.dk, a.kind, a.creg_x, a.creg_y, a.dreg, (size_t)P};
  unsigned int* const case_bar = ctl.case_bar + (size_t)kCaseBarStride * block_case[blockIdx.x];
  auto case_sync = [&]() -> bool {
    if (nbc == 1) {
      __syncthreads();
      return true;
    }
    return range_sync(ctl.bar, case_bar, (unsigned int)nbc, target);
  };
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
  bool ok = case_sync();
  if (ok) {
    phase_b(v);
    block_sum_warps<4>(v, red, bsum);
    publish(ctl.partials, NB, bsum, 4);
    ok = case_sync();
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
        sc_den = delta;  // 1/alpha = den / gamma
        sc_beta = 0.0;
      }
    }
    __syncthreads();
  }
  while (ok) {
    if (sc_stop != 0) break;  // every block of the case sees the same scalars
    {
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
    if (!case_sync()) { ok = false; break; }
    {
      v[0] = v[1] = v[2] = 0.0;
      phase_b(v);
      const double v3[3] = {v[0], v[1], v[2]};
      block_sum_warps<3>(v3, red, bsum);
      publish(ctl.partials, NB, bsum, 3);
    }
    if (!case_sync()) { ok = false; break; }
    {
      double t[3];
      range_sum<3>(ctl.partials, NB, E.block0, nbc, t, gsum);
      // the two reciprocals in different warps (different sub-partitions' FP64 pipes):
      // 1/gamma for the next beta in warp 0, 1/den for alpha in warp 1
      if (threadIdx.x == 0) {
        const double gamma = t[0];
        sc_rr = dreg * t[0] + t[1];
        sc_it += 1;
        sc_stop = sc_rr <= a.tol * a.tol * sc_bb ? 1 : (sc_it >= a.max_iter ? 2 : 0);
        if (sc_stop == 0) {
          sc_beta = gamma * sc_igamma;
          sc_igamma_next = recip_newton(gamma);
        }
      } else if (threadIdx.x == 32) {
        const double gamma = t[0], delta = t[2];
        const double beta = gamma * sc_igamma;
        const double den = delta - beta * gamma * (sc_den * sc_igamma);
        sc_den_next = den;
        if (den != 0.0) sc_alpha = gamma * recip_newton(den);
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        // read by warp 1 before the barrier above; next read after this iteration's barriers
        sc_igamma = sc_igamma_next;
        sc_den = sc_den_next;
      }
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
// Slots of the mixed solve; the case's barrier follows each, and the sums a slot publishes
// are reduced after it.
enum : int {
  SL_FOLD = 0,    // x += D^-1/2 e / sigma, e = 0 (first pass: p = s = e = 0)
  SL_RESID = 1,   // r64 = D^-1/2 (b - K x) and its norms
  SL_FRESH = 2,   // r = sigma r64; Jacobi: also w = K~ r and the sums
  SL_CHEB = 3,    // Chebyshev step j (1 .. cheb - 1) for K~ z = r (step 1 from z1 = r / theta)
  SL_APPLY = 4,   // w = K~ u and the sums (r, u), (w, u), (r, r)
  SL_FORM = 5,    // p = u + beta' p, s = w + beta' s and (p, s)
  SL_UPDATE = 6,  // vector update A
  SL_DONE = 7     // the case's solve has ended
};

__global__ void __launch_bounds__(kPcgThreads, 2) k_mixed_batch(const MixedBatchEntry* __restrict__ cases,
                                                                const int* __restrict__ block_case, BatchControl ctl) {
  __shared__ double red[3][kPcgThreads];
  __shared__ float wred[3][kPcgThreads / 32];
  __shared__ double dsum[8];
  __shared__ float fsum[8];
  __shared__ double sc_sigma, sc_rr, sc_bb, sc_rr_ref, sc_racc[3];
  __shared__ float sc_alpha, sc_beta, sc_pscale, sc_igamma, sc_ialpha, sc_gref, sc_gfresh;
  __shared__ int sc_slot, sc_part, sc_j, sc_fresh, sc_it, sc_stop, sc_nrep, sc_rep_it, sc_keep, sc_restart, sc_final,
      sc_init;
  unsigned int target = 0;
  const int NB = gridDim.x;
  __shared__ __align__(16) unsigned char s_entry[sizeof(MixedBatchEntry)];
  const MixedBatchEntry& E = stage_entry(cases, block_case, s_entry);
  const MixedSolve& A = E.a;
  const ScaledSolve& d = A.d;
  const Geom g = d.g;
  const int nx = g.nx;
  const int lb = blockIdx.x - E.block0, nbc = E.nblocks;
  const CaseRange ch(g.nx * g.ny, lb, nbc);
  // The FP64 residual of a replacement is one slot: with per-case barriers no other case waits
  // for it (the slot code still takes it in parts when asked to).
  const int nparts = 1;
  unsigned int* const case_bar = ctl.case_bar + (size_t)kCaseBarStride * block_case[blockIdx.x];
  // the FP32 phases work on aligned quads of the case's arrays (see QuadOpsF32)
  const Quads Q(g);
  const int u0 = (int)((long long)Q.nquad * lb / nbc), u1 = (int)((long long)Q.nquad * (lb + 1) / nbc);
  const QuadOpsF32 ops{d.kinds, A.cus32, A.cvs32, (float)d.ax, (float)d.ay, g.pitch};
  const double* __restrict__ r64 = d.r;
  float* __restrict__ r = A.r;
  float* __restrict__ w = A.w;
  float* __restrict__ p = A.p;
  float* __restrict__ s = A.s;
  float* __restrict__ e = A.e;
  // Chebyshev preconditioner (cheb > 1): z1 = r / theta, then cheb - 1 steps alternating
  // between zA and zB; u = M^-1 r is the last iterate.  With Jacobi u is r itself.
  const int cheb = A.cheb > 1 ? A.cheb : 1;
  constexpr float ith = (float)(1.0 / ChebCoef::theta);
  const double tol2 = d.tol * d.tol;

  if (threadIdx.x == 0) {
    sc_slot = SL_FOLD;
    sc_part = 0;
    sc_init = 1;
    sc_sigma = 0.0;
    sc_bb = 0.0;
    sc_igamma = 1.0f;
    sc_pscale = 1.0f;
    sc_j = sc_fresh = sc_it = sc_stop = sc_nrep = sc_keep = sc_restart = sc_final = 0;
    sc_rep_it = -1000;
  }
  __syncthreads();
  bool ok = true;
  // Slot t publishes its sums in rows 3 (t & 1) .. 3 (t & 1) + 2 of the partials: the rows a
  // slot reads after its barrier are written again two slots later, after a barrier that every
  // block reaches only once it has read them.
  for (unsigned int t = 0; ok; ++t) {
    const int sl = sc_slot, part = sc_part;
    if (sl == SL_DONE) break;  // every block of the case sees the same slot
    const bool last_part = part == nparts - 1;
    double* prow = ctl.partials + (size_t)(3 * (t & 1)) * NB;
    if (sl == SL_FOLD) {
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
        for (int u = u0 + threadIdx.x; u < u1; u += blockDim.x) quad_fold(d.x, d.isd, e, Q.k(u), isig, true);
      }
    } else if (sl == SL_RESID) {
      // part `part` of the block's cells: r64 = D^-1/2 (b - K x) and the norms, summed over
      // the parts in shared memory and published with the last
      const KRow<double> K{d.cu, d.cv, d.dk, d.kind, d.creg_x, d.creg_y, d.dreg, (size_t)g.pitch};
      const int len = ch.t1 - ch.t0;
      const int a0 = ch.t0 + (int)((long long)len * part / nparts);
      const int a1 = ch.t0 + (int)((long long)len * (part + 1) / nparts);
      double v[3] = {0.0, 0.0, 0.0};
      for (CellWalk cw(a0 + threadIdx.x, blockDim.x, a1, nx); cw.ok(); cw.next()) {
        const size_t k = g.idx(cw.i, cw.j);
        const double bk = d.b[k];
        const double rk = bk - K(d.x, k);
        const double rs = d.isd[k] * rk;
        d.r[k] = rs;
        v[0] += rs * rs;
        v[1] += rk * rk;
        v[2] += bk * bk;
      }
      block_sum_warps<3>(v, red, dsum);
      if (threadIdx.x == 0) {
        for (int q = 0; q < 3; ++q) sc_racc[q] = part == 0 ? dsum[q] : sc_racc[q] + dsum[q];
        if (last_part) publish(prow, NB, sc_racc, 3);
      }
    } else if (sl == SL_FRESH) {
      const double sig = sc_sigma;
      if (cheb == 1) {
        // r = sigma r64 (FP32), w = K~ r, sums (r, r), (w, r)
        float v[2] = {0.0f, 0.0f};
        for (int u = u0 + threadIdx.x; u < u1; u += blockDim.x) ops.stencil(r, w, r64, sig, Q.k(u), v);
        block_sum_f32<2>(v, wred, fsum);
        const double dv[3] = {(double)fsum[0], (double)fsum[1], (double)fsum[0]};
        publish(prow, NB, dv, 3);
      } else {
        for (int u = u0 + threadIdx.x; u < u1; u += blockDim.x) {
          const int k0 = Q.k(u);
          st4(r, k0, ld4_scaled(r64, k0, sig));
        }
      }
    } else if (sl == SL_CHEB) {
      const int j = sc_j;
      float c1, c2;
      cheb_step_coef(j, c1, c2);
      float* zout = (j & 1) ? A.zB : A.zA;
      if (j == 1) {
        for (int u = u0 + threadIdx.x; u < u1; u += blockDim.x) ops.cheb_first(r, A.dch, zout, Q.k(u), ith, c1, c2);
      } else {
        const float* zin = (j & 1) ? A.zA : A.zB;
        for (int u = u0 + threadIdx.x; u < u1; u += blockDim.x) ops.cheb_step(zin, r, A.dch, zout, Q.k(u), c1, c2);
      }
    } else if (sl == SL_APPLY) {
      float v[3] = {0.0f, 0.0f, 0.0f};
      if (cheb == 1) {
        float v2[2] = {0.0f, 0.0f};
        for (int u = u0 + threadIdx.x; u < u1; u += blockDim.x) ops.stencil(r, w, nullptr, 0.0, Q.k(u), v2);
        v[0] = v2[0];
        v[1] = v2[1];
        v[2] = v2[0];
      } else {
        const float* uvec = (cheb & 1) ? A.zA : A.zB;
        for (int u = u0 + threadIdx.x; u < u1; u += blockDim.x) ops.apply_sums(uvec, r, w, Q.k(u), v);
      }
      block_sum_f32<3>(v, wred, fsum);
      const double dv[3] = {(double)fsum[0], (double)fsum[1], (double)fsum[2]};
      publish(prow, NB, dv, 3);
    } else if (sl == SL_FORM) {
      // p = u + beta' p, s = w + beta' s with beta' = beta sigma_new / sigma_old, and (p, s)
      const float be = sc_beta * sc_pscale;
      const float* uvec = cheb == 1 ? r : ((cheb & 1) ? A.zA : A.zB);
      float v[1] = {0.0f};
      for (int u = u0 + threadIdx.x; u < u1; u += blockDim.x) v[0] += ops.form(p, uvec, w, s, Q.k(u), be);
      block_sum_f32<1>(v, wred, fsum);
      const double dv[1] = {(double)fsum[0]};
      publish(prow, NB, dv, 1);
    } else if (sl == SL_UPDATE) {
      const float al = sc_alpha, be = sc_beta;
      const bool keep = sc_keep != 0;
      if (cheb == 1) {
        for (int u = u0 + threadIdx.x; u < u1; u += blockDim.x) ops.update(p, r, w, s, e, Q.k(u), al, be, keep);
      } else {
        // the same update with u = M^-1 r
        const float* uvec = (cheb & 1) ? A.zA : A.zB;
        for (int u = u0 + threadIdx.x; u < u1; u += blockDim.x)
          ops.update_u(p, uvec, r, w, s, e, Q.k(u), al, be, keep);
      }
    }
    // the case's barrier (a case on one block needs only the block barrier: its own global
    // writes are visible to its threads after it)
    if (nbc == 1) __syncthreads();
    else if (!range_sync(ctl.bar, case_bar, (unsigned int)nbc, target)) { ok = false; break; }
    // ---- after the barrier: the slot's sums, the scalars and the next slot
    const bool sums3 = (sl == SL_RESID && last_part) || sl == SL_APPLY || (sl == SL_FRESH && cheb == 1);
    double t3[3] = {0.0, 0.0, 0.0};
    if (sums3) range_sum<3>(prow, NB, E.block0, nbc, t3, dsum);
    else if (sl == SL_FORM) {
      double t1[1];
      range_sum<1>(prow, NB, E.block0, nbc, t1, dsum);
      t3[0] = t1[0];
    }
    if (threadIdx.x == 0) {
      if (sl == SL_FOLD) {
        sc_slot = SL_RESID;
      } else if (sl == SL_RESID && !last_part) {
        sc_part = part + 1;
      } else if (sl == SL_RESID) {
        sc_part = 0;
        if (sc_init) sc_bb = t3[2];
        sc_rr = t3[1];
        sc_rr_ref = t3[1];
        const double old = sc_init ? 0.0 : sc_sigma;
        sc_sigma = t3[0] > 0.0 ? 1.0 / sqrt(t3[0]) : 1.0;
        // directions and K~ p carried over are rescaled to the new normalisation
        const double c = old > 0.0 ? sc_sigma / old : 0.0;
        sc_pscale = (float)c;
        sc_igamma = (float)((double)sc_igamma / (c * c + (c == 0.0)));
        sc_init = 0;
        if (sc_bb == 0.0 || sc_rr <= tol2 * sc_bb) {
          sc_stop = 1;
          sc_slot = SL_DONE;
        } else if (sc_final) {
          sc_stop = 2;
          sc_slot = SL_DONE;
        } else {
          sc_fresh = 1;
          sc_slot = SL_FRESH;
        }
      } else if (sl == SL_FRESH && cheb > 1) {
        sc_j = 1;
        sc_slot = SL_CHEB;
      } else if (sl == SL_CHEB) {
        if (sc_j + 1 < cheb) sc_j += 1;
        else sc_slot = SL_APPLY;
      } else if (sl == SL_FORM) {
        sc_alpha = sc_gfresh / (float)t3[0];
        sc_igamma = 1.0f / sc_gfresh;
        sc_ialpha = 1.0f / sc_alpha;
        sc_keep = 1;
        sc_slot = SL_UPDATE;
      } else if (sl == SL_UPDATE) {
        sc_fresh = 0;
        if (cheb > 1) {
          sc_j = 1;
          sc_slot = SL_CHEB;
        } else {
          sc_slot = SL_APPLY;
        }
      } else if (sums3) {
        // SL_APPLY, or SL_FRESH with Jacobi: gamma = (r, u), delta = (w, u), (r, r)
        const float gamma = (float)t3[0], delta = (float)t3[1], rr32 = (float)t3[2];
        if (sc_fresh) {
          // after a replacement: beta as usual (none at the start or after a restart), and
          // alpha = gamma / (p, K~ p) from the formed direction
          sc_gref = rr32;
          sc_gfresh = gamma;
          if ((sc_it == 0 && sc_nrep == 0) || sc_restart) {
            sc_beta = 0.0f;
            sc_restart = 0;
          } else {
            sc_beta = gamma * sc_igamma;
          }
          sc_slot = SL_FORM;
        } else {
          sc_it += 1;
          sc_keep = 0;
          // replace when the FP32 residual fell by `drop`, or when the estimate of the unscaled
          // residual norm meets the tolerance
          // (multiplied out: no FP64 division on the serial path)
          const double gref = sc_gref;
          int replace = gref > 0.0 && ((double)rr32 <= A.drop * A.drop * gref ||
                                       sc_rr_ref * (double)rr32 <= tol2 * sc_bb * gref) ? 1 : 0;
          if (!replace) {
            // Chronopoulos-Gear: beta = gamma / gamma_old, alpha = gamma / (delta - beta gamma / alpha_old)
            const float beta = gamma * sc_igamma;
            const float den = delta - beta * gamma * sc_ialpha;
            if (den > 0.0f && den < INFINITY) {
              sc_beta = beta;
              sc_alpha = gamma / den;
              sc_igamma = 1.0f / gamma;
              sc_ialpha = 1.0f / sc_alpha;
            } else {
              replace = 1;  // loss of positivity in FP32: replace and restart
              sc_restart = 1;
            }
          }
          if (!replace && sc_it >= d.max_iter) {
            replace = 1;
            sc_final = 1;
          }
          if (replace) {
            sc_nrep += 1;
            if (sc_it - sc_rep_it < 3) sc_restart = 1;  // replacements back to back: no progress
            sc_rep_it = sc_it;
            sc_slot = SL_FOLD;
          } else {
            sc_slot = SL_UPDATE;
          }
        }
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
  if (!ctl.case_bar || ctl.ncases < 1) return cudaErrorInvalidValue;
  cudaMemsetAsync(ctl.case_bar, 0, sizeof(unsigned int) * kCaseBarStride * (size_t)ctl.ncases, st);
  void* params[] = {(void*)&dev_cases, (void*)&dev_block_case, &ctl};
  return cudaLaunchCooperativeKernel((const void*)k_sc_batch, blocks, kPcgThreads, params, 0, st);
}

cudaError_t run_mixed_batch(const MixedBatchEntry* dev_cases, const int* dev_block_case, BatchControl ctl,
                            int blocks, cudaStream_t st) {
  if (!ctl.case_bar || ctl.ncases < 1) return cudaErrorInvalidValue;
  cudaMemsetAsync(ctl.case_bar, 0, sizeof(unsigned int) * kCaseBarStride * (size_t)ctl.ncases, st);
  void* params[] = {(void*)&dev_cases, (void*)&dev_block_case, &ctl};
  return cudaLaunchCooperativeKernel((const void*)k_mixed_batch, blocks, kPcgThreads, params, 0, st);
}

}  // namespace ccm
