// Mixed-precision pressure Poisson solve (Eq. pm_poisson): conjugate gradients in FP32 on the
// symmetrically Jacobi-scaled system, anchored by FP64 residual replacements ("reliable
// updates": Sleijpen and van der Vorst, Computing 56, 1996; used for mixed-precision GPU
// solvers by Clark et al., Comput. Phys. Commun. 181, 2010).
//
// The iterate x and the right-hand side b stay in FP64.  Between replacements the kernel runs
// the single-reduction CG of pcg_scaled.cu in FP32 on the correction equation
//     K~ e~ = r~,   r~ = sigma D^-1/2 (b - K x),
// normalised by sigma = 1 / ||D^-1/2 (b - K x)|| so the FP32 values stay near unit size
// whatever the scale of b.  When the FP32 residual has dropped by the factor `drop` since the
// last replacement (or its estimate says the FP64 test may be met) the kernel
//   R1: folds the correction into x (x += D^-1/2 e~ / sigma, e~ = 0),
//   R2: forms the true residual b - K x in FP64 and its norms; stops if ||b - K x|| <= tol ||b||,
//   R3: restarts the FP32 residual from it with the new normalisation,
// and continues with the same search direction (rescaled to the new normalisation) instead of
// restarting the Krylov space, which is what keeps the iteration count close to FP64 CG.
// The FP32 dot products are summed in FP32 per thread, warp and block, the block partials in
// FP32 across the grid (fixed order, deterministic); the replacement norms are FP64.
//
// Layout: the FP32 phases work on aligned quads of the padded arrays (padded indices 4q ..
// 4q+3, one float4 per vector; the pitch is a multiple of 32, so every row starts a quad).
// A row's quads span its interior cells plus the ghost and padding slots beside them; those
// slots hold zero in every FP32 vector and stay zero (their inputs are zero and their row kind
// is the identity), so a quad is processed whole, without masks.  Blocks take balanced
// contiguous ranges of quads; on the 1024x512 grid a thread holds at most one quad, so every
// FP32 phase needs a single round of loads.  The FP64 residual of a replacement walks cells.
#include "pcg_quad.cuh"

namespace ccm {

namespace {

// FP32 grid sum: warp q adds the nb block partials of quantity q (all loads in flight).
template <int NV>
__device__ __forceinline__ void grid_sum_f32(const float* partials, int nb, float (&out)[NV], float* smem) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (w < NV) {
    const float* src = partials + (size_t)w * nb;
    float buf[kGridSumPerLane];
#pragma unroll
    for (int m = 0; m < kGridSumPerLane; ++m) {
      const int b = lane + 32 * m;
      buf[m] = b < nb ? __ldcg(&src[b]) : 0.0f;
    }
    float s = 0.0f;
#pragma unroll
    for (int m = 0; m < kGridSumPerLane; ++m) s += buf[m];
    for (int b = lane + 32 * kGridSumPerLane; b < nb; b += 32) s += __ldcg(&src[b]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) smem[w] = s;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) out[k] = smem[k];
}

__global__ void __launch_bounds__(kPcgThreads, 2) k_pcg_poisson_mixed(MixedSolve a) {
  __shared__ double red[4][kPcgThreads];
  __shared__ float wred[3][kPcgThreads / 32];
  __shared__ double dsum[8];
  __shared__ float fsum[8];
  __shared__ double sc_sigma, sc_rr, sc_bb, sc_rr_ref;
  __shared__ float sc_alpha, sc_beta, sc_pscale, sc_igamma, sc_ialpha, sc_gref, sc_gfresh;
  __shared__ int sc_it, sc_stop, sc_replace, sc_nrep;  // stop: 1 converged, 2 iteration limit
  __shared__ int sc_keep;     // the next phase A uses the stored p and s (formed by phase P)
  __shared__ int sc_restart;  // the next replacement also restarts the direction (beta = 0)
  __shared__ int sc_rep_it;   // iteration of the last replacement
  unsigned int target = 0;
  const int nb = gridDim.x;
  const ScaledSolve& d = a.d;
  const Geom g = d.g;
  const int nx = g.nx, P = g.pitch;
  const Chunk ch(g.nx * g.ny);
  const Quads Q(g);
  const int u0 = (int)((long long)Q.nquad * blockIdx.x / gridDim.x);
  const int u1 = (int)((long long)Q.nquad * (blockIdx.x + 1) / gridDim.x);
  const QuadOpsF32 ops{d.kinds, a.cus32, a.cvs32, (float)d.ax, (float)d.ay, P};
  const int first = ch.t0 + threadIdx.x, stride = blockDim.x;
  const double* __restrict__ isd = d.isd;
  double* __restrict__ x = d.x;
  double* __restrict__ r64 = d.r;  // scaled FP64 residual D^-1/2 (b - K x) at a replacement
  float* __restrict__ r = a.r;
  float* __restrict__ w = a.w;
  float* __restrict__ p = a.p;
  float* __restrict__ s = a.s;
  float* __restrict__ e = a.e;
  float* fpart = a.fpartials;
  // Chebyshev preconditioner (cheb > 1): z1 = r / theta, then cheb - 1 steps of the Chebyshev
  // iteration for K~ z = r, alternating between zA and zB; u = M^-1 r is the last iterate.
  // With Jacobi (cheb = 1) u is r itself.
  const int cheb = a.cheb > 1 ? a.cheb : 1;
  constexpr float ith = (float)(1.0 / ChebCoef::theta);
  const double tol2 = d.tol * d.tol;

  // with Jacobi, phase A leaves e += alpha p to the wait of phase B's reduction barrier (no other
  // block reads e)
  float e_al = 0.0f;
  bool e_pending = false;
  // R2 (and the start): r64 = D^-1/2 (b - K x); sums ||r64||^2, ||b - K x||^2 (and ||b||^2).
  auto residual64 = [&](bool with_b) -> bool {
    const KRow<double> K{d.cu, d.cv, d.dk, d.kind, d.creg_x, d.creg_y, d.dreg, (size_t)P};
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
    if (with_b) block_sum_warps<3>(v, red, dsum);
    else {
      const double v2[2] = {v[0], v[1]};
      block_sum_warps<2>(v2, red, dsum);
    }
    if (threadIdx.x == 0)
      for (int q = 0; q < (with_b ? 3 : 2); ++q) d.partials[(size_t)q * nb + blockIdx.x] = dsum[q];
    if (!grid_sync(d.bar, target)) return false;
    double t[3];
    grid_sum<3>(d.partials, nb, t, dsum);
    if (threadIdx.x == 0) {
      if (with_b) sc_bb = t[2];
      sc_rr = t[1];
      sc_rr_ref = t[1];
      const double old = sc_sigma;
      sc_sigma = t[0] > 0.0 ? 1.0 / sqrt(t[0]) : 1.0;
      // directions and K~ p carried over are rescaled to the new normalisation
      const double c = old > 0.0 ? sc_sigma / old : 0.0;
      sc_pscale = (float)c;
      sc_igamma = (float)((double)sc_igamma / (c * c + (c == 0.0)));
      if (sc_bb == 0.0 || sc_rr <= tol2 * sc_bb) sc_stop = 1;
    }
    __syncthreads();
    return true;
  };
  // The Chebyshev steps 1 .. cheb - 1 (Saad, Chebyshev acceleration; eigenvalue interval of
  // the scaled operator as in ChebCoef), a grid barrier after each (the next step and phase
  // B read the neighbours).  Step 1 starts from z1 = d1 = r / theta, formed from r on the fly.
  auto cheb_steps = [&]() -> bool {
    for (int j = 1; j < cheb; ++j) {
      float c1, c2;
      cheb_step_coef(j, c1, c2);
      float* zout = (j & 1) ? a.zB : a.zA;
      if (j == 1) {
        for (int u = u0 + threadIdx.x; u < u1; u += blockDim.x) ops.cheb_first(r, a.dch, zout, Q.k(u), ith, c1, c2);
      } else {
        const float* zin = (j & 1) ? a.zA : a.zB;
        for (int u = u0 + threadIdx.x; u < u1; u += blockDim.x) ops.cheb_step(zin, r, a.dch, zout, Q.k(u), c1, c2);
      }
      if (!grid_sync(d.bar, target)) return false;
    }
    return true;
  };
  // Phase B: w = K~ u (FP32) and the sums gamma = (r, u), delta = (w, u), (r, r).  With `fresh`,
  // r is first set from the FP64 residual, r = sigma r64: with Jacobi it is read at the
  // neighbours the same way; with Chebyshev it is stored and the steps run first.
  auto phase_b = [&](bool fresh) -> bool {
    float v[3] = {0.0f, 0.0f, 0.0f};
    const double sig = sc_sigma;
    if (cheb == 1) {
      float v2[2] = {0.0f, 0.0f};
      for (int u = u0 + threadIdx.x; u < u1; u += blockDim.x)
        ops.stencil(r, w, fresh ? r64 : nullptr, sig, Q.k(u), v2);
      v[0] = v2[0];
      v[1] = v2[1];
      v[2] = v2[0];
    } else {
      if (fresh) {
        for (int u = u0 + threadIdx.x; u < u1; u += blockDim.x) {
          const int k0 = Q.k(u);
          st4(r, k0, ld4_scaled(r64, k0, sig));
        }
        if (!grid_sync(d.bar, target)) return false;
      }
      if (!cheb_steps()) return false;
      const float* uvec = (cheb & 1) ? a.zA : a.zB;
      for (int u = u0 + threadIdx.x; u < u1; u += blockDim.x) ops.apply_sums(uvec, r, w, Q.k(u), v);
    }
    block_sum_f32<3>(v, wred, fsum);
    if (threadIdx.x == 0) {
      fpart[blockIdx.x] = fsum[0];
      fpart[nb + blockIdx.x] = fsum[1];
      fpart[2 * nb + blockIdx.x] = fsum[2];
    }
    grid_arrive(d.bar, target);
    if (e_pending) {
      for (int u = u0 + threadIdx.x; u < u1; u += blockDim.x) ops.add_e(e, p, Q.k(u), e_al);
      e_pending = false;
    }
    if (!grid_wait(d.bar, target)) return false;
    float t[3];
    grid_sum_f32<3>(fpart, nb, t, fsum);
    if (threadIdx.x == 0) {
      const float gamma = t[0], delta = t[1], rr32 = t[2];
      if (!fresh) {
        sc_it += 1;         // one more phase A done
        sc_pscale = 1.0f;   // its rescaling (after a replacement) is spent
        sc_keep = 0;
      }
      if (fresh) sc_gref = rr32;
      // replace when the FP32 residual fell by `drop`, or when the estimate of the unscaled
      // residual norm (scaled by the last FP64 value) meets the tolerance
      // rr32 / gref <= drop^2, or the estimate rr_ref rr32 / gref of the unscaled residual
      // meets the tolerance (multiplied out: no FP64 division on the serial path)
      const double gref = sc_gref;
      sc_replace = !fresh && gref > 0.0 &&
                   ((double)rr32 <= a.drop * a.drop * gref || sc_rr_ref * (double)rr32 <= tol2 * sc_bb * gref) ? 1 : 0;
      // A residual about to be replaced is not used: the scalars are formed from the replacing
      // residual instead (next call, fresh), against the same previous gamma and alpha.
      if (!sc_replace) {
        if (fresh && sc_it == 0 && sc_nrep == 0) {
          sc_beta = 0.0f;
          sc_alpha = gamma / delta;  // (p, K~ p) = (r, w) exactly
          sc_igamma = 1.0f / gamma;
          sc_ialpha = 1.0f / sc_alpha;
        } else if (fresh && sc_restart) {
          // restart after a breakdown or back-to-back replacements: steepest descent step
          sc_beta = 0.0f;
          sc_alpha = gamma / delta;
          sc_igamma = 1.0f / gamma;
          sc_ialpha = 1.0f / sc_alpha;
          sc_pscale = 0.0f;
          sc_restart = 0;
        } else if (fresh) {
          // after a replacement the recurrences no longer hold exactly: beta as usual, and
          // alpha = gamma / (p, K~ p) from the formed direction (phase P)
          sc_beta = gamma * sc_igamma;
          sc_gfresh = gamma;
          sc_keep = 1;
        } else {
          // Chronopoulos-Gear: beta = gamma / gamma_old, alpha = gamma / (delta - beta gamma / alpha_old)
          const float beta = gamma * sc_igamma;
          const float den = delta - beta * gamma * sc_ialpha;
          if (den > 0.0f && den < INFINITY) {
            sc_beta = beta;
            sc_alpha = gamma / den;
            sc_igamma = 1.0f / gamma;
            sc_ialpha = 1.0f / sc_alpha;
          } else {
            sc_replace = 1;  // loss of positivity in FP32: replace and restart
            sc_restart = 1;
          }
        }
      }
    }
    __syncthreads();
    return true;
  };

  // Phase P (after a replacement): p = r + beta' p, s = w + beta' s stored, and
  // alpha = gamma / (p, s) from a direct reduction.
  auto phase_p = [&]() -> bool {
    const float be = sc_beta * sc_pscale;
    float v[1] = {0.0f};
    const float* uvec = cheb == 1 ? r : ((cheb & 1) ? a.zA : a.zB);
    for (int u = u0 + threadIdx.x; u < u1; u += blockDim.x) v[0] += ops.form(p, uvec, w, s, Q.k(u), be);
    // row 3 of the FP32 partials: rows 0-2 (the sums of phase B) may still be read by other
    // blocks, since no barrier separates that read from this write
    block_sum_f32<1>(v, wred, fsum);
    if (threadIdx.x == 0) fpart[3 * nb + blockIdx.x] = fsum[0];
    if (!grid_sync(d.bar, target)) return false;
    float t[1];
    grid_sum_f32<1>(fpart + 3 * nb, nb, t, fsum);
    if (threadIdx.x == 0) {
      sc_alpha = sc_gfresh / t[0];
      sc_igamma = 1.0f / sc_gfresh;
      sc_ialpha = 1.0f / sc_alpha;
    }
    __syncthreads();
    return true;
  };

  // R1 on this block's quads
  auto fold = [&](double isig, bool clear) {
    for (int u = u0 + threadIdx.x; u < u1; u += blockDim.x) quad_fold(x, isd, e, Q.k(u), isig, clear);
  };

  if (threadIdx.x == 0) {
    sc_keep = 0;
    sc_restart = 0;
    sc_rep_it = -1000;
    sc_sigma = 0.0;
    sc_igamma = 1.0f;
    sc_pscale = 1.0f;
    sc_it = 0;
    sc_stop = 0;
    sc_nrep = 0;
    sc_bb = 0.0;
  }
  for (int u = u0 + threadIdx.x; u < u1; u += blockDim.x) {
    const int k0 = Q.k(u);
    const float4 z = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    st4(p, k0, z);
    st4(s, k0, z);
    st4(e, k0, z);
  }
  __syncthreads();
  bool ok = residual64(true);
  if (ok && sc_stop == 0) ok = phase_b(true);
  bool limit = false;
  while (ok && sc_stop == 0) {
    if (sc_it >= d.max_iter) {
      limit = true;
      break;
    }
    // phase A (FP32): p = r + beta' p, s = w + beta' s, e += alpha p, r -= alpha s (p and s as
    // stored when phase P formed them)
    {
      const float al = sc_alpha, be = sc_keep ? 0.0f : sc_beta * sc_pscale;
      const bool keep = sc_keep != 0;
      if (cheb == 1) {
        // Jacobi: e += alpha p waits for phase B's reduction barrier (measured faster there; with
        // the Chebyshev steps the barrier waits are shorter and it stays here)
        for (int u = u0 + threadIdx.x; u < u1; u += blockDim.x) ops.update(p, r, w, s, nullptr, Q.k(u), al, be, keep);
        e_al = al;
        e_pending = true;
      } else {
        // the same update with u = M^-1 r
        const float* uvec = (cheb & 1) ? a.zA : a.zB;
        for (int u = u0 + threadIdx.x; u < u1; u += blockDim.x)
          ops.update_u(p, uvec, r, w, s, e, Q.k(u), al, be, keep);
      }
    }
    if (!grid_sync(d.bar, target)) { ok = false; break; }
    if (!phase_b(false)) { ok = false; break; }
    if (sc_replace) {
      // R1: x += D^-1/2 e / sigma, e = 0 (cell-local), then R2 after a barrier, then R3 + B
      const double isig = 1.0 / sc_sigma;
      fold(isig, true);
      if (threadIdx.x == 0) {
        sc_nrep += 1;
        if (sc_it - sc_rep_it < 3) sc_restart = 1;  // replacements back to back: no progress
        sc_rep_it = sc_it;
      }
      if (!grid_sync(d.bar, target)) { ok = false; break; }
      if (!residual64(false)) { ok = false; break; }
      if (sc_stop != 0) break;
      if (!phase_b(true)) { ok = false; break; }
      if (sc_keep && !phase_p()) { ok = false; break; }
    }
  }
  if (ok && limit) {
    // iteration limit: keep the progress of the last segment and report the true residual
    const double isig = 1.0 / sc_sigma;
    fold(isig, false);
    if (!grid_sync(d.bar, target) || !residual64(false)) ok = false;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const bool conv = ok && sc_stop == 1;
    d.out.iters[0] = ok ? sc_it : 0;
    d.out.rr[0] = ok ? sc_rr : 0.0;
    d.out.bb[0] = ok ? sc_bb : 0.0;
    d.out.converged[0] = conv ? 1 : 0;
    if (d.out.total && ok) d.out.total[0] += sc_it;
    if (!conv && d.out.nconv) d.out.nconv[0] += 1;
    if (a.replacements) a.replacements[0] = sc_nrep;
  }
}

}  // namespace

int mixed_blocks() {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pcg_poisson_mixed, kPcgThreads, 0);
  per = per > 2 ? 2 : (per < 1 ? 1 : per);
  return sms * per;
}

cudaError_t run_poisson_mixed(const MixedSolve& a, cudaStream_t st) {
  const int most = mixed_blocks();
  const int blocks = a.blocks > 0 && a.blocks <= most ? a.blocks : most;
  cudaMemsetAsync(a.d.bar.count, 0, sizeof(unsigned int) * kBarWords, st);
  MixedSolve arg = a;
  void* params[] = {&arg};
  return cudaLaunchCooperativeKernel((const void*)k_pcg_poisson_mixed, blocks, kPcgThreads, params, 0, st);
}

}  // namespace ccm
