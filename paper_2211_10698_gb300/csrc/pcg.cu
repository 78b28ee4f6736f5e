// Persistent preconditioned conjugate-gradient kernels for the two linear systems of the
// PmII step (Sec. 4.6): the pressure Poisson system K Phi = rhs (Eq. pm_poisson) and the
// Crank-Nicolson Helmholtz system H U* = rhs (Eq. pm_prediction).
//
// One cooperative launch runs the whole solve: every block stays resident, device-wide
// barriers are the bounded spin barrier of ccm_internal.cuh, and the dot products are
// block partials summed by every block in one fixed order (deterministic, no atomics on
// floating point).  Standard Hestenes-Stiefel PCG with Jacobi preconditioning; the
// convergence test ||r|| <= tol ||b|| is made before every iteration.
//
// Poisson, per iteration:   A: p = z + beta p_old (recomputed for the stencil neighbours
//                              instead of a third barrier), q = K p, p.q   | barrier
//                           B: x += alpha p, r -= alpha q, z = D^-1 r, r.z, r.r | barrier
// When the Poisson system is singular (no outflow side) the preconditioned residual is
// projected onto zero-mean fields over the active cells (end of Sec. 4.6); the mean is
// carried through the reductions, so no extra barrier is needed.
//
// Helmholtz, per iteration: A: q = H p, p.q | B: x, r, z updates, r.z, r.r | C: p = z + beta p.
#include "ccm_host.h"

namespace ccm {

constexpr int kPcgThreads = 512;

__device__ __forceinline__ void publish(double* partials, int nb, const double* v, int nv) {
  if (threadIdx.x == 0)
    for (int q = 0; q < nv; ++q) partials[(size_t)q * nb + blockIdx.x] = v[q];
}

// Sum NV per-thread values over the block through shared memory; only warp 0 adds (in a
// fixed order), so the FP64 cost is per block, not per thread.  Result valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum_smem(double (&v)[NV], double (*red)[kPcgThreads]) {
#pragma unroll
  for (int q = 0; q < NV; ++q) red[q][threadIdx.x] = v[q];
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double s = 0.0;
      for (int m = lane; m < (int)blockDim.x; m += 32) s += red[q][m];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      v[q] = s;
    }
  }
}

// Cells of this block: one contiguous chunk of the row-major interior, balanced to +-1 cell
// across blocks (the FP64 pipe of each SM is the bottleneck, so per-SM work must be even).
struct Chunk {
  int t0, t1;
  __device__ Chunk(int ncell) {
    t0 = (int)((long long)ncell * blockIdx.x / gridDim.x);
    t1 = (int)((long long)ncell * (blockIdx.x + 1) / gridDim.x);
  }
};

// Walks t = first, first + stride, ... < end, keeping (i, j) of the interior cell t.
struct CellWalk {
  int t, i, j;
  const int nx, stride, end;
  __device__ CellWalk(int first, int stride_, int end_, int nx_) : t(first), nx(nx_), stride(stride_), end(end_) {
    j = first / nx;
    i = first - j * nx;
  }
  __device__ bool ok() const { return t < end; }
  __device__ void next() {
    t += stride;
    i += stride;
    while (i >= nx) { i -= nx; ++j; }
  }
};

template <class T, bool ZM>
__global__ void __launch_bounds__(kPcgThreads, 2) k_pcg_poisson(PoissonSolve<T> a) {
  __shared__ double red[5][kPcgThreads];
  __shared__ double sm[8];
  unsigned int target = 0;
  const int nb = gridDim.x;
  const Geom g = a.g;
  const int nx = g.nx;
  const Chunk ch(g.nx * g.ny);
  const int first = ch.t0 + threadIdx.x, stride = blockDim.x;
  const size_t P_ = (size_t)g.pitch;
  const T* __restrict__ cu = a.cu;
  const T* __restrict__ cv = a.cv;
  const T* __restrict__ invd = a.invd;
  const int8_t* __restrict__ act = a.act;
  T* __restrict__ x = a.x;
  T* __restrict__ r = a.r;
  T* __restrict__ z = a.z;
  T* __restrict__ q = a.q;

  // r = b - K x, z = D^-1 r
  double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (CellWalk w(first, stride, ch.t1, nx); w.ok(); w.next()) {
    const size_t k = g.idx(w.i, w.j);
    const T bk = a.b[k];
    const T rk = bk - poisson_row(cu, cv, act, g, x, k);
    const T zk = invd[k] * rk;
    r[k] = rk;
    z[k] = zk;
    a.p0[k] = (T)0;
    v[0] += (double)rk * (double)zk;
    v[1] += (double)rk * (double)rk;
    v[2] += (double)bk * (double)bk;
    if (ZM && act[k]) { v[3] += (double)zk; v[4] += (double)rk; }
  }
  block_sum_smem<5>(v, red);
  publish(a.partials, nb, v, 5);
  bool ok = grid_sync(a.bar, target);
  double s[5];
  if (ok) grid_sum<5>(a.partials, nb, s, sm);
  double zmean = (ok && ZM) ? s[3] / a.n_act : 0.0;
  double rz = ok ? s[0] - zmean * s[4] : 0.0, rr = ok ? s[1] : 0.0, bb = ok ? s[2] : 0.0;
  const double tol2 = a.tol * a.tol;
  double beta = 0.0;
  int it = 0;
  bool conv = false;
  T* pold = a.p0;
  T* pnew = a.p1;
  if (ok && bb == 0.0) {
    for (CellWalk w(first, stride, ch.t1, nx); w.ok(); w.next()) x[g.idx(w.i, w.j)] = (T)0;
    conv = true;
  }
  while (ok && !conv) {
    if (rr <= tol2 * bb) { conv = true; break; }
    if (it >= a.max_iter) break;
    const T tb = (T)beta, tzm = (T)zmean;
    // phase A: p = z + beta p_old (recomputed at the four neighbours), q = K p, p.q
    double pq[1] = {0.0};
    for (CellWalk w(first, stride, ch.t1, nx); w.ok(); w.next()) {
      const size_t k = g.idx(w.i, w.j);
      auto P = [&](size_t m) -> T {
        if (ZM) return (z[m] - (act[m] ? tzm : (T)0)) + tb * pold[m];
        return z[m] + tb * pold[m];
      };
      const T pc = P(k);
      T qk;
      if (act[k]) {
        qk = cu[k] * (pc - P(k - 1)) + cu[k + 1] * (pc - P(k + 1)) + cv[k] * (pc - P(k - P_)) +
             cv[k + P_] * (pc - P(k + P_));
      } else {
        qk = pc;
      }
      pnew[k] = pc;
      q[k] = qk;
      pq[0] += (double)pc * (double)qk;
    }
    block_sum_smem<1>(pq, red);
    publish(a.partials, nb, pq, 1);
    if (!grid_sync(a.bar, target)) { ok = false; break; }
    double spq[1];
    grid_sum<1>(a.partials, nb, spq, sm);
    const double alpha = rz / spq[0];
    const T ta = (T)alpha;
    // phase B: x += alpha p, r -= alpha q, z = D^-1 r, r.z, r.r
    double wv[4] = {0.0, 0.0, 0.0, 0.0};
    for (CellWalk w(first, stride, ch.t1, nx); w.ok(); w.next()) {
      const size_t k = g.idx(w.i, w.j);
      x[k] += ta * pnew[k];
      const T rk = r[k] - ta * q[k];
      const T zk = invd[k] * rk;
      r[k] = rk;
      z[k] = zk;
      wv[0] += (double)rk * (double)zk;
      wv[1] += (double)rk * (double)rk;
      if (ZM && act[k]) { wv[2] += (double)zk; wv[3] += (double)rk; }
    }
    double sw[4];
    if (ZM) {
      block_sum_smem<4>(wv, red);
      publish(a.partials, nb, wv, 4);
    } else {
      double w2[2] = {wv[0], wv[1]};
      block_sum_smem<2>(w2, red);
      publish(a.partials, nb, w2, 2);
    }
    if (!grid_sync(a.bar, target)) { ok = false; break; }
    if (ZM) {
      grid_sum<4>(a.partials, nb, sw, sm);
    } else {
      double s2[2];
      grid_sum<2>(a.partials, nb, s2, sm);
      sw[0] = s2[0]; sw[1] = s2[1]; sw[2] = 0.0; sw[3] = 0.0;
    }
    zmean = ZM ? sw[2] / a.n_act : 0.0;
    const double rz_new = sw[0] - zmean * sw[3];
    beta = rz_new / rz;
    rz = rz_new;
    rr = sw[1];
    T* tmp = pold; pold = pnew; pnew = tmp;
    ++it;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.out.iters[0] = it;
    a.out.rr[0] = rr;
    a.out.bb[0] = bb;
    a.out.converged[0] = conv ? 1 : 0;
    if (a.out.total) a.out.total[0] += it;
    if (!conv && a.out.nconv) a.out.nconv[0] += 1;
  }
}

// Projection of the warm start onto zero mean over active cells (singular systems only).
template <class T>
__global__ void k_zero_mean_partials(Geom g, const int8_t* act, const T* x, double* partials) {
  const int ncell = g.nx * g.ny;
  double s = 0.0;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ncell; t += gridDim.x * blockDim.x) {
    const int j = t / g.nx, i = t - j * g.nx;
    const size_t k = g.idx(i, j);
    if (act[k]) s += (double)x[k];
  }
  __shared__ double sm[32];
  double v[1] = {s};
  block_sum<1>(v, sm);
  if (threadIdx.x == 0) partials[blockIdx.x] = v[0];
}
template <class T>
__global__ void k_zero_mean_apply(Geom g, const int8_t* act, T* x, const double* partials, int nb, double n_act) {
  __shared__ double sm[32];
  double s[1];
  grid_sum<1>(partials, nb, s, sm);
  const T m = (T)(s[0] / n_act);
  const int ncell = g.nx * g.ny;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ncell; t += gridDim.x * blockDim.x) {
    const int j = t / g.nx, i = t - j * g.nx;
    const size_t k = g.idx(i, j);
    if (act[k]) x[k] -= m;
  }
}

// ---------------------------------------------------------------------------------------
// Helmholtz PCG over the velocity unknowns (u and v faces in the padded layout).
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kPcgThreads) k_pcg_helmholtz(HelmholtzSolve a) {
  __shared__ double sm[32 * 3];
  unsigned int target = 0;
  const int nb = gridDim.x;
  const Geom g = a.g;
  const Coefs& c = a.c;
  const int total = (int)g.count();
  const int t0 = blockIdx.x * blockDim.x + threadIdx.x, ts = gridDim.x * blockDim.x;
  const HomView wx{a.xu, a.xv, c.role_u, c.role_v, g, a.bc};
  const HomView wp{a.pu, a.pv, c.role_u, c.role_v, g, a.bc};
  const double mu = a.ph.mu;

  double v[3] = {0.0, 0.0, 0.0};
  for (int t = t0; t < total; t += ts) {
    const int j = t / g.pitch - 1, i = t - (j + 1) * g.pitch - 1;
    if (i > g.nx + 1) continue;
    const size_t k = (size_t)t;
    if (c.role_u[k] == R_UNKNOWN) {
      const double hx = c.massu[k] * wx.u[k] - mu * visc_u(c, g, a.bc, wx, i, j);
      const double rk = a.bu[k] - hx, zk = c.invdhu[k] * rk;
      a.ru[k] = rk; a.zu[k] = zk; a.pu[k] = zk;
      v[0] += rk * zk; v[1] += rk * rk; v[2] += a.bu[k] * a.bu[k];
    }
    if (c.role_v[k] == R_UNKNOWN) {
      const double hv = c.massv[k] * wx.v[k] - mu * visc_v(c, g, a.bc, wx, i, j);
      const double rk = a.bv[k] - hv, zk = c.invdhv[k] * rk;
      a.rv[k] = rk; a.zv[k] = zk; a.pv[k] = zk;
      v[0] += rk * zk; v[1] += rk * rk; v[2] += a.bv[k] * a.bv[k];
    }
  }
  block_sum<3>(v, sm);
  publish(a.partials, nb, v, 3);
  bool ok = grid_sync(a.bar, target);
  double s[3];
  if (ok) grid_sum<3>(a.partials, nb, s, sm);
  double rz = ok ? s[0] : 0.0, rr = ok ? s[1] : 0.0, bb = ok ? s[2] : 0.0;
  const double tol2 = a.tol * a.tol;
  int it = 0;
  bool conv = false;
  if (ok && bb == 0.0) {
    for (int t = t0; t < total; t += ts) {
      if (c.role_u[t] == R_UNKNOWN) a.xu[t] = 0.0;
      if (c.role_v[t] == R_UNKNOWN) a.xv[t] = 0.0;
    }
    conv = true;
  }
  while (ok && !conv) {
    if (rr <= tol2 * bb) { conv = true; break; }
    if (it >= a.max_iter) break;
    double pq[1] = {0.0};
    for (int t = t0; t < total; t += ts) {
      const int j = t / g.pitch - 1, i = t - (j + 1) * g.pitch - 1;
      if (i > g.nx + 1) continue;
      const size_t k = (size_t)t;
      if (c.role_u[k] == R_UNKNOWN) {
        const double qk = c.massu[k] * wp.u[k] - mu * visc_u(c, g, a.bc, wp, i, j);
        a.qu[k] = qk;
        pq[0] += a.pu[k] * qk;
      }
      if (c.role_v[k] == R_UNKNOWN) {
        const double qk = c.massv[k] * wp.v[k] - mu * visc_v(c, g, a.bc, wp, i, j);
        a.qv[k] = qk;
        pq[0] += a.pv[k] * qk;
      }
    }
    block_sum<1>(pq, sm);
    publish(a.partials, nb, pq, 1);
    if (!grid_sync(a.bar, target)) { ok = false; break; }
    double spq[1];
    grid_sum<1>(a.partials, nb, spq, sm);
    const double alpha = rz / spq[0];
    double w[2] = {0.0, 0.0};
    for (int t = t0; t < total; t += ts) {
      const size_t k = (size_t)t;
      if (c.role_u[k] == R_UNKNOWN) {
        a.xu[k] += alpha * a.pu[k];
        const double rk = a.ru[k] - alpha * a.qu[k], zk = c.invdhu[k] * rk;
        a.ru[k] = rk; a.zu[k] = zk;
        w[0] += rk * zk; w[1] += rk * rk;
      }
      if (c.role_v[k] == R_UNKNOWN) {
        a.xv[k] += alpha * a.pv[k];
        const double rk = a.rv[k] - alpha * a.qv[k], zk = c.invdhv[k] * rk;
        a.rv[k] = rk; a.zv[k] = zk;
        w[0] += rk * zk; w[1] += rk * rk;
      }
    }
    block_sum<2>(w, sm);
    publish(a.partials, nb, w, 2);
    if (!grid_sync(a.bar, target)) { ok = false; break; }
    double sw[2];
    grid_sum<2>(a.partials, nb, sw, sm);
    const double beta = sw[0] / rz;
    rz = sw[0];
    rr = sw[1];
    ++it;
    if (rr <= tol2 * bb || it >= a.max_iter) continue;  // p is not needed any more
    for (int t = t0; t < total; t += ts) {
      const size_t k = (size_t)t;
      if (c.role_u[k] == R_UNKNOWN) a.pu[k] = a.zu[k] + beta * a.pu[k];
      if (c.role_v[k] == R_UNKNOWN) a.pv[k] = a.zv[k] + beta * a.pv[k];
    }
    if (!grid_sync(a.bar, target)) { ok = false; break; }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.out.iters[0] = it;
    a.out.rr[0] = rr;
    a.out.bb[0] = bb;
    a.out.converged[0] = conv ? 1 : 0;
    if (a.out.total) a.out.total[0] += it;
    if (!conv && a.out.nconv) a.out.nconv[0] += 1;
  }
}

// ---------------------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------------------
static int coop_blocks(const void* fn, int threads, int max_per_sm) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, 0);
  if (per > max_per_sm) per = max_per_sm;
  if (per < 1) per = 1;
  return sms * per;
}

int pcg_partials_needed() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms * 4 * 8;  // blocks (at most 4 per SM) times values per reduction
}

template <class T>
cudaError_t run_poisson_pcg(PoissonSolve<T> a, cudaStream_t st) {
  const void* fn = a.zero_mean ? (const void*)k_pcg_poisson<T, true> : (const void*)k_pcg_poisson<T, false>;
  const int blocks = coop_blocks(fn, kPcgThreads, 2);
  if (a.zero_mean) {
    // singular system: warm start and right-hand side projected onto zero-mean fields
    k_zero_mean_partials<T><<<blocks, kPcgThreads, 0, st>>>(a.g, a.act, a.x, a.partials);
    k_zero_mean_apply<T><<<blocks, kPcgThreads, 0, st>>>(a.g, a.act, a.x, a.partials, blocks, a.n_act);
    k_zero_mean_partials<T><<<blocks, kPcgThreads, 0, st>>>(a.g, a.act, a.b, a.partials);
    k_zero_mean_apply<T><<<blocks, kPcgThreads, 0, st>>>(a.g, a.act, a.b, a.partials, blocks, a.n_act);
  }
  cudaMemsetAsync(a.bar.count, 0, sizeof(unsigned int), st);
  void* params[] = {&a};
  return cudaLaunchCooperativeKernel(fn, blocks, kPcgThreads, params, 0, st);
}
template cudaError_t run_poisson_pcg<double>(PoissonSolve<double>, cudaStream_t);
template cudaError_t run_poisson_pcg<float>(PoissonSolve<float>, cudaStream_t);

cudaError_t run_helmholtz_pcg(HelmholtzSolve a, cudaStream_t st) {
  const void* fn = (const void*)k_pcg_helmholtz;
  const int blocks = coop_blocks(fn, kPcgThreads, 2);
  cudaMemsetAsync(a.bar.count, 0, sizeof(unsigned int), st);
  void* params[] = {&a};
  return cudaLaunchCooperativeKernel(fn, blocks, kPcgThreads, params, 0, st);
}

}  // namespace ccm
