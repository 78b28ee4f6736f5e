// Crank-Nicolson Helmholtz solve of the predictor (Eq. pm_prediction): (rho/tau) M U* -
// mu visc(S_hom(U*)) = rhs, coupled in u and v, by Jacobi-preconditioned CG on the operator's
// coefficient form.
//
// The operator is symmetric positive definite (mass plus the negative semidefinite viscous
// operator with the averaged off-diagonal weight).  Set-up extracts its nine coefficients per
// unknown face by colour probing (operators.cu), so an application here is nine FMA per row
// instead of the strain and viscous-flux evaluation with its boundary branches.  The
// recurrences are the single-reduction arrangement of Chronopoulos and Gear (one grid
// reduction and two barriers per iteration), as for the Poisson solve:
//   A: p = z + beta p, s = w + beta s, x += alpha p, r -= alpha s, z = D^-1 r    | barrier
//   B: w = H z, (r, z), (w, z), (r, r)                                          | barrier
// Rows are the unknown faces of both components; a block takes a balanced contiguous range of
// the padded index, where faces that are not unknowns are skipped (their coefficients in the
// unknowns' rows are 0).
//
// k_helm_batch solves the systems of the cases of a batch in one cooperative launch: each case
// owns a contiguous range of blocks and reduces over them only, every block passes the same
// two barriers per iteration, and the launch ends when no case iterates.
#include "batch_common.cuh"

namespace ccm {

namespace {

struct HelmRows {
  const HelmCoefPtrs& h;
  int P;
  // (H x)_u at face k
  __device__ __forceinline__ double row_u(const double* U, const double* V, int k) const {
    return h.a[0][k] * U[k] + h.a[1][k] * U[k - 1] + h.a[2][k] * U[k + 1] + h.a[3][k] * U[k - P] +
           h.a[4][k] * U[k + P] + h.a[5][k] * V[k - 1] + h.a[6][k] * V[k] + h.a[7][k] * V[k + P - 1] +
           h.a[8][k] * V[k + P];
  }
  // (H x)_v at face k
  __device__ __forceinline__ double row_v(const double* U, const double* V, int k) const {
    return h.a[9][k] * V[k] + h.a[10][k] * V[k - 1] + h.a[11][k] * V[k + 1] + h.a[12][k] * V[k - P] +
           h.a[13][k] * V[k + P] + h.a[14][k] * U[k - P] + h.a[15][k] * U[k - P + 1] + h.a[16][k] * U[k] +
           h.a[17][k] * U[k + 1];
  }
};

__global__ void __launch_bounds__(kPcgThreads, 2) k_pcg_helmholtz_c(HelmCSolve a) {
  __shared__ double red[4][kPcgThreads];
  __shared__ double bsum[8];
  __shared__ double gsum[8];
  __shared__ double sc_alpha, sc_beta, sc_igamma, sc_ialpha, sc_rr, sc_bb;
  __shared__ int sc_it, sc_stop;
  unsigned int target = 0;
  const int nb = gridDim.x;
  const Geom g = a.g;
  const int P = g.pitch;
  const HelmRows H{a.h, P};
  // padded range holding every unknown face: u faces (0..nx, 0..ny-1), v faces (0..nx-1, 0..ny)
  const int T0 = (int)g.idx(0, 0), T1 = (int)g.idx(g.nx, g.ny) + 1;
  const int t0 = T0 + (int)((long long)(T1 - T0) * blockIdx.x / nb);
  const int t1 = T0 + (int)((long long)(T1 - T0) * (blockIdx.x + 1) / nb);
  const int8_t* __restrict__ ru = a.ru;
  const int8_t* __restrict__ rv = a.rv;
  // periodic sides: z, which the rows read across the side, is also written to its images
  const bool per = g.px || g.py;
  auto img = [&](double* z, int k, double val) {
    if (per) put_images(z, k % P - 1, k / P - 1, (size_t)k, val, g.nx, g.ny, (size_t)P, g.px != 0, g.py != 0);
  };

  auto reduce = [&](const double (&v)[4], int nv) {
    if (nv == 4) block_sum_warps<4>(v, red, bsum);
    else {
      const double v3[3] = {v[0], v[1], v[2]};
      block_sum_warps<3>(v3, red, bsum);
    }
    if (threadIdx.x == 0)
      for (int q = 0; q < nv; ++q) a.partials[(size_t)q * nb + blockIdx.x] = bsum[q];
  };
  // phase B: w = H z on the unknown rows; sums (r, z), (w, z), (r, r)
  auto phase_b = [&](double (&v)[4]) {
    for (int k = t0 + threadIdx.x; k < t1; k += blockDim.x) {
      if (ru[k] == R_UNKNOWN) {
        const double w = H.row_u(a.zU, a.zV, k), r = a.rU[k], z = a.zU[k];
        a.wU[k] = w;
        v[0] += r * z;
        v[1] += w * z;
        v[2] += r * r;
      }
      if (rv[k] == R_UNKNOWN) {
        const double w = H.row_v(a.zU, a.zV, k), r = a.rV[k], z = a.zV[k];
        a.wV[k] = w;
        v[0] += r * z;
        v[1] += w * z;
        v[2] += r * r;
      }
    }
  };

  // phase 0: r = b - H x, z = D^-1 r, p = s = 0, ||b||^2
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int k = t0 + threadIdx.x; k < t1; k += blockDim.x) {
    if (ru[k] == R_UNKNOWN) {
      const double b = a.bu[k], r = b - H.row_u(a.xu, a.xv, k);
      a.rU[k] = r;
      a.zU[k] = a.invu[k] * r;
      img(a.zU, k, a.zU[k]);
      a.pU[k] = 0.0;
      a.sU[k] = 0.0;
      v[3] += b * b;
    }
    if (rv[k] == R_UNKNOWN) {
      const double b = a.bv[k], r = b - H.row_v(a.xu, a.xv, k);
      a.rV[k] = r;
      a.zV[k] = a.invv[k] * r;
      img(a.zV, k, a.zV[k]);
      a.pV[k] = 0.0;
      a.sV[k] = 0.0;
      v[3] += b * b;
    }
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
      const double gamma = t[0], delta = t[1];
      sc_rr = t[2];
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
  if (ok && sc_bb == 0.0)
    for (int k = t0 + threadIdx.x; k < t1; k += blockDim.x) {
      if (ru[k] == R_UNKNOWN) a.xu[k] = 0.0;
      if (rv[k] == R_UNKNOWN) a.xv[k] = 0.0;
    }
  while (ok && sc_stop == 0) {
    {
      const double al = sc_alpha, be = sc_beta;
      for (int k = t0 + threadIdx.x; k < t1; k += blockDim.x) {
        if (ru[k] == R_UNKNOWN) {
          const double p = a.zU[k] + be * a.pU[k], s = a.wU[k] + be * a.sU[k];
          a.pU[k] = p;
          a.sU[k] = s;
          a.xu[k] += al * p;
          const double r = a.rU[k] - al * s;
          a.rU[k] = r;
          a.zU[k] = a.invu[k] * r;
          img(a.zU, k, a.zU[k]);
        }
        if (rv[k] == R_UNKNOWN) {
          const double p = a.zV[k] + be * a.pV[k], s = a.wV[k] + be * a.sV[k];
          a.pV[k] = p;
          a.sV[k] = s;
          a.xv[k] += al * p;
          const double r = a.rV[k] - al * s;
          a.rV[k] = r;
          a.zV[k] = a.invv[k] * r;
          img(a.zV, k, a.zV[k]);
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
      const double gamma = t[0], delta = t[1];
      sc_rr = t[2];
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

// ---------------------------------------------------------------------------------------
// The same solve for the cases of a batch.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kPcgThreads, 2) k_helm_batch(const HelmBatchEntry* __restrict__ cases,
                                                               const int* __restrict__ block_case, BatchControl ctl) {
  __shared__ double red[4][kPcgThreads];
  __shared__ double bsum[8];
  __shared__ double gsum[8];
  __shared__ double sc_alpha, sc_beta, sc_igamma, sc_ialpha, sc_rr, sc_bb;
  __shared__ int sc_it, sc_stop;
  __shared__ __align__(16) unsigned char s_entry[sizeof(HelmBatchEntry)];
  unsigned int target = 0;
  const int NB = gridDim.x;
  const HelmBatchEntry& E = stage_entry(cases, block_case, s_entry);
  const HelmCSolve& a = E.a;
  const Geom g = a.g;
  const HelmRows H{a.h, g.pitch};
  const int lb = blockIdx.x - E.block0, nbc = E.nblocks;
  const int T0 = (int)g.idx(0, 0), T1 = (int)g.idx(g.nx, g.ny) + 1;
  const int t0 = T0 + (int)((long long)(T1 - T0) * lb / nbc);
  const int t1 = T0 + (int)((long long)(T1 - T0) * (lb + 1) / nbc);
  const int8_t* __restrict__ ru = a.ru;
  const int8_t* __restrict__ rv = a.rv;

  auto phase_b = [&](double (&v)[4]) {
    for (int k = t0 + threadIdx.x; k < t1; k += blockDim.x) {
      if (ru[k] == R_UNKNOWN) {
        const double w = H.row_u(a.zU, a.zV, k), r = a.rU[k], z = a.zU[k];
        a.wU[k] = w;
        v[0] += r * z;
        v[1] += w * z;
        v[2] += r * r;
      }
      if (rv[k] == R_UNKNOWN) {
        const double w = H.row_v(a.zU, a.zV, k), r = a.rV[k], z = a.zV[k];
        a.wV[k] = w;
        v[0] += r * z;
        v[1] += w * z;
        v[2] += r * r;
      }
    }
  };

  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int k = t0 + threadIdx.x; k < t1; k += blockDim.x) {
    if (ru[k] == R_UNKNOWN) {
      const double b = a.bu[k], r = b - H.row_u(a.xu, a.xv, k);
      a.rU[k] = r;
      a.zU[k] = a.invu[k] * r;
      a.pU[k] = 0.0;
      a.sU[k] = 0.0;
      v[3] += b * b;
    }
    if (rv[k] == R_UNKNOWN) {
      const double b = a.bv[k], r = b - H.row_v(a.xu, a.xv, k);
      a.rV[k] = r;
      a.zV[k] = a.invv[k] * r;
      a.pV[k] = 0.0;
      a.sV[k] = 0.0;
      v[3] += b * b;
    }
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
      const double gamma = t[0], delta = t[1];
      sc_rr = t[2];
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
  if (ok && sc_bb == 0.0)
    for (int k = t0 + threadIdx.x; k < t1; k += blockDim.x) {
      if (ru[k] == R_UNKNOWN) a.xu[k] = 0.0;
      if (rv[k] == R_UNKNOWN) a.xv[k] = 0.0;
    }
  while (ok) {
    const bool run = sc_stop == 0;
    if (run) {
      const double al = sc_alpha, be = sc_beta;
      for (int k = t0 + threadIdx.x; k < t1; k += blockDim.x) {
        if (ru[k] == R_UNKNOWN) {
          const double p = a.zU[k] + be * a.pU[k], s = a.wU[k] + be * a.sU[k];
          a.pU[k] = p;
          a.sU[k] = s;
          a.xu[k] += al * p;
          const double r = a.rU[k] - al * s;
          a.rU[k] = r;
          a.zU[k] = a.invu[k] * r;
        }
        if (rv[k] == R_UNKNOWN) {
          const double p = a.zV[k] + be * a.pV[k], s = a.wV[k] + be * a.sV[k];
          a.pV[k] = p;
          a.sV[k] = s;
          a.xv[k] += al * p;
          const double r = a.rV[k] - al * s;
          a.rV[k] = r;
          a.zV[k] = a.invv[k] * r;
        }
      }
    }
    // running flags are written before the first barrier and read after it; the partials
    // before the second and after it
    if (threadIdx.x == 0) ctl.running[blockIdx.x] = run ? 1 : 0;
    if (!grid_sync(ctl.bar, target)) { ok = false; break; }
    if (!any_running(ctl.running, NB)) break;
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
        const double gamma = t[0], delta = t[1];
        sc_rr = t[2];
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

}  // namespace

cudaError_t run_helmholtz_coef(const HelmCSolve& a, cudaStream_t st) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pcg_helmholtz_c, kPcgThreads, 0);
  per = per > 2 ? 2 : (per < 1 ? 1 : per);
  cudaMemsetAsync(a.bar.count, 0, sizeof(unsigned int) * kBarWords, st);
  HelmCSolve arg = a;
  void* params[] = {&arg};
  return cudaLaunchCooperativeKernel((const void*)k_pcg_helmholtz_c, sms * per, kPcgThreads, params, 0, st);
}

}  // namespace ccm

namespace ccm {

int batch_helm_blocks() {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_helm_batch, kPcgThreads, 0);
  per = per > 2 ? 2 : (per < 1 ? 1 : per);
  return sms * per;
}

cudaError_t run_helm_batch(const HelmBatchEntry* dev_cases, const int* dev_block_case, BatchControl ctl, int blocks,
                           cudaStream_t st) {
  cudaMemsetAsync(ctl.bar.count, 0, sizeof(unsigned int) * kBarWords, st);
  void* params[] = {(void*)&dev_cases, (void*)&dev_block_case, &ctl};
  return cudaLaunchCooperativeKernel((const void*)k_helm_batch, blocks, kPcgThreads, params, 0, st);
}

}  // namespace ccm
