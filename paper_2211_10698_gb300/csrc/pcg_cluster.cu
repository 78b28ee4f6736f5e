// FP64 pressure Poisson solve (Eq. pm_poisson) for small grids: CG on the Jacobi-scaled system
// (the iteration of pcg_scaled.cu) inside ONE thread-block cluster.
//
// On a grid of a few thousand cells a grid-wide barrier and the L2 round trips of each phase
// cost several times the arithmetic.  Here the C CTAs of one cluster (C <= 16, one per SM)
// hold the whole solve in shared memory: CTA q owns a band of grid rows and keeps x~, r, p,
// s, w and the row kinds of its band; the stencil reads the neighbouring bands' edge rows
// of r through distributed shared memory; the dot products are summed per CTA and then over
// the C CTAs in rank order; the barriers are the cluster's hardware barrier.  There is no
// spin-wait: every CTA runs the same scalar recurrences on the same sums and leaves the loop
// at the same iteration.
//
// Per iteration:  A: p = r + beta p, s = w + beta s, x~ += alpha p, r -= alpha s   | cluster barrier
//                 B: w = K~ r, sums (r, r), sum (d - dreg) r^2, (w, r)             | cluster barrier
// then every CTA adds the C partial sums in the same order and forms the same scalars.
// Only nonsingular systems (an outflow side) with the Jacobi preconditioner take this path.
#include <cooperative_groups.h>

#include "pcg_common.cuh"

namespace cg = cooperative_groups;

namespace ccm {

namespace {

constexpr int kCT = 512;  // threads per CTA

// Rows [band_lo(q), band_lo(q + 1)) of the grid belong to CTA q.
__device__ __forceinline__ int band_lo(int q, int ny, int C) { return (int)((long long)ny * q / C); }

__global__ void __launch_bounds__(kCT, 1) k_pcg_poisson_cluster(ClusterSolve f) {
  __shared__ double red[4][kCT];
  __shared__ double bsum[8];
  __shared__ double part[4];  // this CTA's sums, read by every CTA of the cluster
  __shared__ double all[16][4];  // every CTA's sums, gathered
  __shared__ double sc_alpha, sc_beta, sc_igamma, sc_den, sc_rr, sc_bb;
  __shared__ double sc_igamma_next, sc_den_next;
  __shared__ int sc_it, sc_stop;
  extern __shared__ double band[];  // x~, r, p, s, w of the band (nmax each), then the kinds
  cg::cluster_group cluster = cg::this_cluster();
  const ScaledSolve& a = f.a;
  const Geom g = a.g;
  const int nx = g.nx, ny = g.ny, P = g.pitch;
  const int C = (int)cluster.num_blocks(), q = (int)cluster.block_rank();
  const int j0 = band_lo(q, ny, C), j1 = band_lo(q + 1, ny, C);
  const int ncell = (j1 - j0) * nx;
  const int nmax = f.nmax;
  double* xs = band;
  double* r = band + nmax;
  double* p = band + 2 * (size_t)nmax;
  double* s = band + 3 * (size_t)nmax;
  double* w = band + 4 * (size_t)nmax;
  int8_t* kinds = reinterpret_cast<int8_t*>(band + 5 * (size_t)nmax);
  // edge rows of the neighbouring bands: the last row of band q-1, the first of band q+1
  const double* r_below =
      q > 0 ? cluster.map_shared_rank(r, q - 1) + (size_t)(j0 - 1 - band_lo(q - 1, ny, C)) * nx : nullptr;
  const double* r_above = q < C - 1 ? cluster.map_shared_rank(r, q + 1) : nullptr;
  const KRow<double> K{a.cu, a.cv, a.dk, a.kind, a.creg_x, a.creg_y, a.dreg, (size_t)P};
  const double ax = a.ax, ay = a.ay, dreg = a.dreg;

  // B: w = K~ r on the band and the sums (as in pcg_scaled.cu); neighbours outside the domain
  // are zero (the scaled coefficients of faces to ghost cells are zero too)
  auto phase_b = [&](double (&v)[4]) {
    for (int l = threadIdx.x; l < ncell; l += kCT) {
      const int jl = l / nx, i = l - jl * nx, j = j0 + jl;
      const int8_t km = kinds[l];
      const double rc = r[l];
      const double rw = i > 0 ? r[l - 1] : 0.0;
      const double re = i < nx - 1 ? r[l + 1] : 0.0;
      const double rs = jl > 0 ? r[l - nx] : (j > 0 ? r_below[i] : 0.0);
      const double rn = l + nx < ncell ? r[l + nx] : (j < ny - 1 ? r_above[i] : 0.0);
      double wk;
      if (km == 1) {
        wk = rc - ax * (rw + re) - ay * (rs + rn);
      } else {
        const size_t k = g.idx(i, j);
        const double dk = km == 2 ? a.sd[k] * a.sd[k] : 1.0;
        wk = km == 2 ? rc - a.cus[k] * rw - a.cus[k + 1] * re - a.cvs[k] * rs - a.cvs[k + P] * rn : rc;
        v[1] += (dk - dreg) * (rc * rc);
      }
      w[l] = wk;
      v[0] += rc * rc;
      v[2] += wk * rc;
    }
  };
  // the CTA's sums into part[], then (after the cluster barrier) every CTA adds all C of them
  // in rank order
  auto publish = [&](const double (&v)[4], int nv) {
    if (nv == 4) block_sum_warps<4, kCT>(v, red, bsum);
    else {
      const double v3[3] = {v[0], v[1], v[2]};
      block_sum_warps<3, kCT>(v3, red, bsum);
    }
    if (threadIdx.x < nv) part[threadIdx.x] = bsum[threadIdx.x];
  };
  // thread rk fetches CTA rk's sums (the C remote loads overlap); threads 0 and 32 then add
  // them in rank order (call with all threads; the same sums land in t of both)
  auto gather = [&](double (&t)[4], int nv) {
    if (threadIdx.x < C) {
      const double* pr = cluster.map_shared_rank(part, (int)threadIdx.x);
      for (int m = 0; m < nv; ++m) all[threadIdx.x][m] = pr[m];
    }
    __syncthreads();
    for (int m = 0; m < nv; ++m) t[m] = 0.0;
    if (threadIdx.x == 0 || threadIdx.x == 32)
      for (int rk = 0; rk < C; ++rk)
        for (int m = 0; m < nv; ++m) t[m] += all[rk][m];
  };

  // Phase 0: x~ = D^1/2 x, r~ = D^-1/2 (b - K x), p = s = 0, the kinds, ||b||^2
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int l = threadIdx.x; l < ncell; l += kCT) {
    const int jl = l / nx, i = l - jl * nx;
    const size_t k = g.idx(i, j0 + jl);
    const double bk = a.b[k];
    const double rk = bk - K(a.x, k);
    xs[l] = a.sd[k] * a.x[k];
    r[l] = a.isd[k] * rk;
    p[l] = 0.0;
    s[l] = 0.0;
    kinds[l] = a.kinds[k];
    v[3] += bk * bk;
  }
  cluster.sync();
  phase_b(v);
  publish(v, 4);
  cluster.sync();
  double t4[4];
  gather(t4, 4);
  if (threadIdx.x == 0) {
    const double* t = t4;
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
  while (sc_stop == 0) {
    {
      const double al = sc_alpha, be = sc_beta;
      for (int l = threadIdx.x; l < ncell; l += kCT) {
        const double pk = r[l] + be * p[l];
        const double sk = w[l] + be * s[l];
        p[l] = pk;
        s[l] = sk;
        xs[l] += al * pk;
        r[l] -= al * sk;
      }
    }
    // the neighbours' new r before the stencil; every CTA has read the previous sums
    cluster.sync();
    v[0] = v[1] = v[2] = 0.0;
    phase_b(v);
    publish(v, 3);
    cluster.sync();
    double t3[4];
    gather(t3, 3);
    // beta = gamma / gamma_old; alpha = gamma / (delta - beta gamma / alpha_old).  The two
    // reciprocals are independent: 1/gamma (for the next beta) in warp 0, 1/den in warp 1,
    // which issue to different sub-partitions' FP64 pipes.
    if (threadIdx.x == 0) {
      const double gamma = t3[0];
      sc_rr = dreg * t3[0] + t3[1];
      sc_it += 1;
      sc_stop = sc_rr <= a.tol * a.tol * sc_bb ? 1 : (sc_it >= a.max_iter ? 2 : 0);
      if (sc_stop == 0) {
        sc_beta = gamma * sc_igamma;
        sc_igamma_next = recip_newton(gamma);
      }
    } else if (threadIdx.x == 32) {
      const double gamma = t3[0], delta = t3[2];
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
  // x = D^-1/2 x~ on the band
  for (int l = threadIdx.x; l < ncell; l += kCT) {
    const int jl = l / nx, i = l - jl * nx;
    const size_t k = g.idx(i, j0 + jl);
    a.x[k] = a.isd[k] * xs[l];
  }
  if (q == 0 && threadIdx.x == 0) {
    const bool conv = sc_stop == 1;
    a.out.iters[0] = sc_it;
    a.out.rr[0] = sc_rr;
    a.out.bb[0] = sc_bb;
    a.out.converged[0] = conv ? 1 : 0;
    if (a.out.total) a.out.total[0] += sc_it;
    if (!conv && a.out.nconv) a.out.nconv[0] += 1;
  }
  // no CTA leaves while another may still read its shared memory
  cluster.sync();
}

}  // namespace

size_t cluster_smem_bytes(int nx, int ny, int C) {
  const size_t nmax = (size_t)((ny + C - 1) / C) * (size_t)nx;
  return nmax * (5 * sizeof(double) + 1);
}

cudaError_t run_poisson_cluster(ClusterSolve f, int C, cudaStream_t st) {
  const Geom& g = f.a.g;
  if (C < 1 || C > 16 || C > g.ny) return cudaErrorInvalidConfiguration;
  f.nmax = (g.ny + C - 1) / C * g.nx;
  const size_t smem = cluster_smem_bytes(g.nx, g.ny, C);
  if (smem > 200 * 1024) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(k_pcg_poisson_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess && C > 8)
    e = cudaFuncSetAttribute(k_pcg_poisson_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cudaErrorInvalidConfiguration;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)C, 1, 1);
  cfg.blockDim = dim3(kCT, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, (const void*)k_pcg_poisson_cluster, &cfg) != cudaSuccess ||
      clusters < 1) {
    cudaGetLastError();
    return cudaErrorInvalidConfiguration;
  }
  return cudaLaunchKernelEx(&cfg, k_pcg_poisson_cluster, f);
}

}  // namespace ccm
