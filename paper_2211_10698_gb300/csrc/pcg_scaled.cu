// FP64 pressure Poisson solve (Eq. pm_poisson) by conjugate gradients on the symmetrically
// Jacobi-scaled system.
//
// With D the diagonal of K, Jacobi-preconditioned CG on K x = b and plain CG on
//     K~ x~ = b~,   K~ = D^-1/2 K D^-1/2,   x~ = D^1/2 x,   b~ = D^-1/2 b
// produce the same iterates in exact arithmetic (x = D^-1/2 x~ at every step), so the method is
// the Jacobi-PCG of the pressure step.  The scaled form saves FP64 work on a part whose FP64
// pipe is narrow: K~ has a unit diagonal, the preconditioned residual is the residual itself,
// and on cells whose four neighbours are uncut the row of K~ is one constant stencil
// x~_c - ax (x~_W + x~_E) - ay (x~_S + x~_N).  Per cell and iteration that leaves 4 FMA in the
// vector updates, 4 in the stencil and 2 in the dot products.
//
// The recurrences are the single-reduction arrangement of Chronopoulos and Gear: with w = K~ r
// and s = K~ p carried along, one grid reduction per iteration yields gamma = (r, r),
// delta = (w, r) and the convergence norm ||r_K||^2 = ||D^1/2 r~||^2 of the unscaled residual,
// so the stopping test ||r|| <= tol ||b|| is the one of the unscaled system.
//
// Per iteration:  A: p = r + beta p, s = w + beta s, x~ += alpha p, r -= alpha s   | barrier
//                 B: w = K~ r, partial sums                                         | barrier
// then every block sums the partials in the same order and computes the same scalars.
// Only nonsingular systems (an outflow side) take this path.
#include "pcg_common.cuh"

namespace ccm {

namespace {

constexpr int kGroup = 2;  // cells per thread whose loads are in flight together

// Set-up: sqrt(d), 1/sqrt(d), the scaled face coefficients and the scaled row kinds.
// d is the diagonal of K on active cells, 1 on inactive cells (identity rows) and 0 outside
// the domain, where every iterate is zero; 1/sqrt(d) is taken as 0 there so that faces to
// ghost cells get a zero scaled coefficient.
__global__ void k_scaling(Geom g, CoefPtrs o) {
  const int i = (int)(blockIdx.x * blockDim.x + threadIdx.x) - 1;
  const int j = (int)(blockIdx.y * blockDim.y + threadIdx.y) - 1;
  if (i > g.nx + 1 || j > g.ny + 1) return;
  const size_t k = g.idx(i, j);
  auto isd_at = [&](size_t q) {
    const double d = o.diagk[q];
    return d > 0.0 ? 1.0 / sqrt(d) : 0.0;
  };
  const double d = o.diagk[k];
  const double sd = d > 0.0 ? sqrt(d) : 0.0;
  const double isd = isd_at(k);
  o.sdk[k] = sd;
  o.isdk[k] = isd;
  o.isdk32[k] = (float)isd;
  const double cus = i >= 0 ? o.cu[k] * isd * isd_at(k - 1) : 0.0;
  const double cvs = j >= 0 ? o.cv[k] * isd * isd_at(k - g.pitch) : 0.0;
  o.cus[k] = cus;
  o.cvs[k] = cvs;
  o.cus32[k] = (float)cus;
  o.cvs32[k] = (float)cvs;
  int8_t ks = 0;
  if (i >= 0 && i < g.nx && j >= 0 && j < g.ny && o.kind[k] != 0) {
    ks = 2;
    if (o.kind[k] == 1) {
      // uncut row; the scaled row is the constant stencil when every in-domain neighbour has
      // the uncut diagonal too (ghost neighbours hold zero in every iterate)
      const double cx = g.hy / g.hx, cy = g.hx / g.hy, dreg = 2.0 * (cx + cy), e = 1e-14 * dreg;
      bool uni = true;
      if (i > 0) uni = uni && fabs(o.diagk[k - 1] - dreg) <= e;
      if (i < g.nx - 1) uni = uni && fabs(o.diagk[k + 1] - dreg) <= e;
      if (j > 0) uni = uni && fabs(o.diagk[k - g.pitch] - dreg) <= e;
      if (j < g.ny - 1) uni = uni && fabs(o.diagk[k + g.pitch] - dreg) <= e;
      if (uni) ks = 1;
    }
  }
  o.kinds[k] = ks;
}

template <int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_pcg_poisson_sc(ScaledSolve a) {
  __shared__ double red[4][NT];
  __shared__ double bsum[8];
  __shared__ double gsum[8];
  __shared__ double sc_alpha, sc_beta;  // scalars of the next vector update
  __shared__ double sc_igamma, sc_ialpha, sc_rr, sc_bb;
  __shared__ int sc_it, sc_stop;        // stop: 0 continue, 1 converged, 2 iteration limit
  unsigned int target = 0;
  const int nb = gridDim.x;
  const Geom g = a.g;
  const int nx = g.nx, P = g.pitch;
  const Chunk ch(g.nx * g.ny);
  const int first = ch.t0 + threadIdx.x, stride = blockDim.x;
  const int kdummy = (int)g.idx(0, 0);
  const KRow<double> K{a.cu, a.cv, a.dk, a.kind, a.creg_x, a.creg_y, a.dreg, (size_t)P};
  const int8_t* __restrict__ kinds = a.kinds;
  const double* __restrict__ cus = a.cus;
  const double* __restrict__ cvs = a.cvs;
  const double* __restrict__ sd = a.sd;
  const double ax = a.ax, ay = a.ay, dreg = a.dreg;
  double* __restrict__ xs = a.xs;
  double* __restrict__ r = a.r;
  double* __restrict__ w = a.w;
  double* __restrict__ p = a.p;
  double* __restrict__ s = a.s;

  // Phase B: w = K~ r on this thread's cells and the sums
  //   v0 = (r, r), v1 = sum over rows without the uncut diagonal of (d - dreg) r^2, v2 = (w, r),
  // so that ||D^1/2 r||^2 = dreg v0 + v1.  Slots past the end of the range do no work (the
  // branch is uniform for all but one warp).
  auto phase_b = [&](double (&v)[4]) {
    CellWalk cw(first, stride, ch.t1, nx);
    Group<kGroup> gr;
    while (next_group(cw, g, kdummy, gr)) {
      int8_t km[kGroup];
      double rc[kGroup], rw[kGroup], re[kGroup], rs[kGroup], rn[kGroup];
#pragma unroll
      for (int m = 0; m < kGroup; ++m) {
        const int k = gr.k[m];
        km[m] = kinds[k];
        rc[m] = r[k];
        rw[m] = r[k - 1];
        re[m] = r[k + 1];
        rs[m] = r[k - P];
        rn[m] = r[k + P];
      }
#pragma unroll
      for (int m = 0; m < kGroup; ++m) {
        if (!gr.v[m]) continue;
        const int k = gr.k[m];
        double wk;
        if (km[m] == 1) {
          wk = rc[m] - ax * (rw[m] + re[m]) - ay * (rs[m] + rn[m]);
        } else {
          const double dk = km[m] == 2 ? sd[k] * sd[k] : 1.0;
          wk = km[m] == 2 ? rc[m] - cus[k] * rw[m] - cus[k + 1] * re[m] - cvs[k] * rs[m] - cvs[k + P] * rn[m]
                          : rc[m];
          v[1] += (dk - dreg) * (rc[m] * rc[m]);
        }
        w[k] = wk;
        v[0] += rc[m] * rc[m];
        v[2] += wk * rc[m];
      }
    }
  };
  auto reduce = [&](const double (&v)[4], int nv) {
    if (nv == 4) block_sum_warps<4, NT>(v, red, bsum);
    else {
      const double v3[3] = {v[0], v[1], v[2]};
      block_sum_warps<3, NT>(v3, red, bsum);
    }
    if (threadIdx.x == 0)
      for (int q = 0; q < nv; ++q) a.partials[(size_t)q * nb + blockIdx.x] = bsum[q];
  };

  // Phase 0: x~ = D^1/2 x, r~ = D^-1/2 (b - K x), p = s = 0, ||b||^2.
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  {
    double bb = 0.0;
    for (CellWalk cw(first, stride, ch.t1, nx); cw.ok(); cw.next()) {
      const size_t k = g.idx(cw.i, cw.j);
      const double bk = a.b[k];
      const double rk = bk - K(a.x, k);
      xs[k] = sd[k] * a.x[k];
      r[k] = a.isd[k] * rk;
      p[k] = 0.0;
      s[k] = 0.0;
      bb += bk * bk;
    }
    v[3] = bb;
  }
  bool ok = grid_sync(a.bar, target);
  if (ok) {
    phase_b(v);
    reduce(v, 4);
    ok = grid_sync(a.bar, target);
  }
  if (ok) {
    double t[4];
    grid_sum<4>(a.partials, nb, t, gsum);
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
  while (ok && sc_stop == 0) {
    // phase A
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
    if (!grid_sync(a.bar, target)) { ok = false; break; }
    v[0] = v[1] = v[2] = 0.0;
    phase_b(v);
    reduce(v, 3);
    if (!grid_sync(a.bar, target)) { ok = false; break; }
    double t[3];
    grid_sum<3>(a.partials, nb, t, gsum);
    if (threadIdx.x == 0) {
      // beta = gamma / gamma_old; alpha = gamma / (delta - beta gamma / alpha_old)
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
  // x = D^-1/2 x~ on this block's cells (also after a failed barrier: the cells are local)
  for (CellWalk cw(first, stride, ch.t1, nx); cw.ok(); cw.next()) {
    const size_t k = g.idx(cw.i, cw.j);
    a.x[k] = a.isd[k] * xs[k];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const bool conv = ok && sc_stop == 1;
    a.out.iters[0] = ok ? sc_it : 0;
    a.out.rr[0] = ok ? sc_rr : 0.0;
    a.out.bb[0] = ok ? sc_bb : 0.0;
    a.out.converged[0] = conv ? 1 : 0;
    if (a.out.total && ok) a.out.total[0] += sc_it;
    if (!conv && a.out.nconv) a.out.nconv[0] += 1;
  }
}

// Block shape of the solve: NT threads, at most MINB blocks per SM.
constexpr int kScThreads = 512, kScBlocksPerSM = 2;
const void* const kScKernel = (const void*)k_pcg_poisson_sc<kScThreads, kScBlocksPerSM>;

int sc_blocks() {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kScKernel, kScThreads, 0);
  if (per > kScBlocksPerSM) per = kScBlocksPerSM;
  if (per < 1) per = 1;
  return sms * per;
}

}  // namespace

void launch_scaling(const Geom& g, const CoefPtrs& o, cudaStream_t st) {
  const dim3 b(32, 8);
  const dim3 grid((g.nx + 3 + b.x - 1) / b.x, (g.ny + 3 + b.y - 1) / b.y);
  k_scaling<<<grid, b, 0, st>>>(g, o);
}

cudaError_t run_poisson_scaled(const ScaledSolve& a, cudaStream_t st) {
  const int blocks = sc_blocks();
  cudaMemsetAsync(a.bar.count, 0, sizeof(unsigned int) * kBarWords, st);
  ScaledSolve arg = a;
  void* params[] = {&arg};
  return cudaLaunchCooperativeKernel(kScKernel, blocks, kScThreads, params, 0, st);
}

}  // namespace ccm
