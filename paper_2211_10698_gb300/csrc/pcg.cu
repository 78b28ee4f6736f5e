// Persistent preconditioned conjugate-gradient kernels for the pressure Poisson system
// K Phi = rhs of the PmII step (Eq. pm_poisson) on the unscaled system: the three-phase
// kernel with the Chebyshev preconditioner, the single-reduction Jacobi kernel for singular
// systems, and their batched form.  (Nonsingular Jacobi solves use the scaled kernels of
// pcg_scaled.cu, pcg_fused.cu and pcg_mixed.cu; the Helmholtz solve is in pcg_helm.cu.)
//
// One cooperative launch runs the whole solve: every block stays resident, device-wide
// barriers are the bounded spin barrier of ccm_internal.cuh, and the dot products are
// block partials summed by every block in one fixed order (deterministic, no atomics on
// floating point).  The convergence test ||r|| <= tol ||b|| is made before every iteration.
//
// Poisson, per iteration:   A: p = z + beta p_old (recomputed for the stencil neighbours
//                              instead of a third barrier), q = K p, p.q   | barrier
//                           B: x += alpha p, r -= alpha q, z = D^-1 r, r.z, r.r | barrier
// When the Poisson system is singular (no outflow side) the preconditioned residual is
// projected onto zero-mean fields over the active cells (end of Sec. 4.6); the mean is
// carried through the reductions, so no extra barrier is needed.
#include "pcg_common.cuh"

namespace ccm {

template <class T, bool ZM, int CHEB>
__global__ void __launch_bounds__(kPcgThreads, 2) k_pcg_poisson(PoissonSolve<T> a) {
  __shared__ double red[5][kPcgThreads];
  __shared__ double sm[8];
  __shared__ PcgScalars S;
  unsigned int target = 0;
  const int nb = gridDim.x;
  const Geom g = a.g;
  const int nx = g.nx;
  const Chunk ch(g.nx * g.ny);
  const int first = ch.t0 + threadIdx.x, stride = blockDim.x;
  const KRow<T> K{a.cu, a.cv, a.dk, a.kind, (T)a.creg_x, (T)a.creg_y, (T)a.dreg, (size_t)g.pitch};
  const T* __restrict__ invd = a.invd;
  const int8_t* __restrict__ kind = a.kind;
  T* __restrict__ x = a.x;
  T* __restrict__ r = a.r;
  T* __restrict__ q = a.q;
  T* __restrict__ p = a.p0;
  T* zc = a.z;    // preconditioned residual
  T* zo = a.z2;   // Chebyshev: the other z buffer
  const T inv_theta = (T)(1.0 / ChebCoef::theta);
  const T ireg = (T)a.invd_reg;
  auto Dinv = [&](size_t k) -> T { return kind[k] == 1 ? ireg : invd[k]; };
  // periodic sides: a vector the stencil reads across the side is also written to its images
  const bool per = g.px || g.py;
  auto img = [&](T* v, const CellWalk& w, size_t k, T val) {
    if (per) put_images(v, w.i, w.j, k, val, g.nx, g.ny, (size_t)g.pitch, g.px != 0, g.py != 0);
  };

  // Chebyshev steps 1..CHEB-1 after z = w1 = D^-1 r / theta; accumulates r.z and, for
  // singular systems, the sums of z and r over active cells.
  auto cheb_rest = [&](double* acc) -> bool {
    double rho_prev = ChebCoef::delta / ChebCoef::theta;
    for (int st = 1; st < CHEB; ++st) {
      if (!grid_sync(a.bar, target)) return false;
      const double rho = 1.0 / (2.0 * ChebCoef::theta / ChebCoef::delta - rho_prev);
      const T c1 = (T)(rho * rho_prev), c2 = (T)(2.0 * rho / ChebCoef::delta);
      const bool last = st == CHEB - 1;
      for (CellWalk w(first, stride, ch.t1, nx); w.ok(); w.next()) {
        const size_t k = g.idx(w.i, w.j);
        const T sk = Dinv(k) * (r[k] - K((const T*)zc, k));
        const T w1 = c1 * a.w1[k] + c2 * sk;
        a.w1[k] = w1;
        const T zk = zc[k] + w1;
        zo[k] = zk;
        img(zo, w, k, zk);
        if (last) {
          acc[0] += (double)r[k] * (double)zk;
          if (ZM && kind[k]) { acc[2] += (double)zk; acc[3] += (double)r[k]; }
        }
      }
      T* t = zc; zc = zo; zo = t;
      rho_prev = rho;
    }
    return true;
  };

  // r = b - K x, z = M^-1 r, p = 0
  double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (CellWalk w(first, stride, ch.t1, nx); w.ok(); w.next()) {
    const size_t k = g.idx(w.i, w.j);
    const T bk = a.b[k];
    const T rk = bk - K(x, k);
    r[k] = rk;
    p[k] = (T)0;
    v[1] += (double)rk * (double)rk;
    v[2] += (double)bk * (double)bk;
    if (CHEB > 1) {
      const T w1 = Dinv(k) * rk * inv_theta;
      a.w1[k] = w1;
      zc[k] = w1;
      img(zc, w, k, w1);
    } else {
      const T zk = Dinv(k) * rk;
      zc[k] = zk;
      v[0] += (double)rk * (double)zk;
      if (ZM && kind[k]) { v[3] += (double)zk; v[4] += (double)rk; }
    }
  }
  bool ok = true;
  if (CHEB > 1) {
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    ok = cheb_rest(acc);
    v[0] = acc[0]; v[3] = acc[2]; v[4] = acc[3];
  }
  block_sum_smem<5>(v, red);
  publish(a.partials, nb, v, 5);
  ok = ok && grid_sync(a.bar, target);
  if (ok) {
    double s5[5];
    grid_sum<5>(a.partials, nb, s5, sm);
    if (threadIdx.x == 0) {
      S.zmean = ZM ? s5[3] / a.n_act : 0.0;
      S.rz = s5[0] - S.zmean * s5[4];
      S.rr = s5[1];
      S.bb = s5[2];
      S.beta = 0.0;
      S.it = 0;
      S.stop = (S.bb == 0.0 || S.rr <= a.tol * a.tol * S.bb) ? 1 : (a.max_iter <= 0 ? 2 : 0);
    }
    __syncthreads();
  }
  if (ok && S.bb == 0.0)
    for (CellWalk w(first, stride, ch.t1, nx); w.ok(); w.next()) x[g.idx(w.i, w.j)] = (T)0;
  while (ok && S.stop == 0) {
    // phase A: p = z + beta p
    {
      const T tb = (T)S.beta, tzm = (T)S.zmean;
      const T* __restrict__ z = zc;
      for (CellWalk w(first, stride, ch.t1, nx); w.ok(); w.next()) {
        const size_t k = g.idx(w.i, w.j);
        const T zk = ZM ? z[k] - (kind[k] ? tzm : (T)0) : z[k];
        const T pk = zk + tb * p[k];
        p[k] = pk;
        img(p, w, k, pk);
      }
    }
    if (!grid_sync(a.bar, target)) { ok = false; break; }
    // phase B: q = K p, p.q
    double pq[1] = {0.0};
    for (CellWalk w(first, stride, ch.t1, nx); w.ok(); w.next()) {
      const size_t k = g.idx(w.i, w.j);
      const T qk = K(p, k);
      q[k] = qk;
      pq[0] += (double)p[k] * (double)qk;
    }
    block_sum_smem<1>(pq, red);
    publish(a.partials, nb, pq, 1);
    if (!grid_sync(a.bar, target)) { ok = false; break; }
    {
      double spq[1];
      grid_sum<1>(a.partials, nb, spq, sm);
      if (threadIdx.x == 0) S.alpha = S.rz / spq[0];
      __syncthreads();
    }
    // phase C: x += alpha p, r -= alpha q, z = M^-1 r, r.z, r.r
    const T ta = (T)S.alpha;
    double wv[4] = {0.0, 0.0, 0.0, 0.0};
    for (CellWalk w(first, stride, ch.t1, nx); w.ok(); w.next()) {
      const size_t k = g.idx(w.i, w.j);
      x[k] += ta * p[k];
      const T rk = r[k] - ta * q[k];
      r[k] = rk;
      wv[1] += (double)rk * (double)rk;
      if (CHEB > 1) {
        const T w1 = Dinv(k) * rk * inv_theta;
        a.w1[k] = w1;
        zc[k] = w1;
        img(zc, w, k, w1);
      } else {
        const T zk = Dinv(k) * rk;
        zc[k] = zk;
        wv[0] += (double)rk * (double)zk;
        if (ZM && kind[k]) { wv[2] += (double)zk; wv[3] += (double)rk; }
      }
    }
    if (CHEB > 1) {
      double acc[4] = {0.0, 0.0, 0.0, 0.0};
      if (!cheb_rest(acc)) { ok = false; break; }
      wv[0] = acc[0]; wv[2] = acc[2]; wv[3] = acc[3];
    }
    double sw[4] = {0.0, 0.0, 0.0, 0.0};
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
      sw[0] = s2[0]; sw[1] = s2[1];
    }
    if (threadIdx.x == 0) {
      S.zmean = ZM ? sw[2] / a.n_act : 0.0;
      const double rz_new = sw[0] - S.zmean * sw[3];
      S.beta = rz_new / S.rz;
      S.rz = rz_new;
      S.rr = sw[1];
      S.it += 1;
      S.stop = S.rr <= a.tol * a.tol * S.bb ? 1 : (S.it >= a.max_iter ? 2 : 0);
    }
    __syncthreads();
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const bool conv = ok && S.stop == 1;
    a.out.iters[0] = ok ? S.it : 0;
    a.out.rr[0] = ok ? S.rr : 0.0;
    a.out.bb[0] = ok ? S.bb : 0.0;
    a.out.converged[0] = conv ? 1 : 0;
    if (a.out.total && ok) a.out.total[0] += S.it;
    if (!conv && a.out.nconv) a.out.nconv[0] += 1;
  }
}

// Jacobi-preconditioned CG in the single-reduction (Chronopoulos-Gear) arrangement: the
// same Krylov iterates as Hestenes-Stiefel PCG in exact arithmetic, with s = K p carried by
// recurrence so that one iteration needs one SpMV, one reduction and two barriers:
//   phase 1 (own cells): p = u + beta p, s = w + beta s, x += alpha p, r -= alpha s, u = D^-1 r
//   phase 2:             w = K u, and the sums r.u, w.u, r.r
// Singular systems (no outflow side): u is projected onto zero mean over the active cells
// lazily; since K applied to a constant vanishes on active cells, w = K u is unchanged and
// only the sums need the correction.
template <class T, bool ZM>
__global__ void __launch_bounds__(kPcgThreads, 2) k_pcg_poisson_cg(PoissonSolve<T> a) {
  __shared__ double red[6][kPcgThreads];
  __shared__ double sm[8];
  __shared__ PcgScalars S;
  __shared__ double S_alpha_prev, S_gamma;
  unsigned int target = 0;
  const int nb = gridDim.x;
  const Geom g = a.g;
  const int nx = g.nx;
  const Chunk ch(g.nx * g.ny);
  const int first = ch.t0 + threadIdx.x, stride = blockDim.x;
  const KRow<T> K{a.cu, a.cv, a.dk, a.kind, (T)a.creg_x, (T)a.creg_y, (T)a.dreg, (size_t)g.pitch};
  const T* __restrict__ invd = a.invd;
  const int8_t* __restrict__ kind = a.kind;
  T* __restrict__ x = a.x;
  T* __restrict__ r = a.r;
  T* __restrict__ u = a.z;
  T* __restrict__ w = a.q;
  T* __restrict__ p = a.p0;
  T* __restrict__ sv = a.p1;
  const T ireg = (T)a.invd_reg;
  // periodic sides: u, which the stencil reads across the side, is also written to its images
  const bool per = g.px || g.py;
  auto img = [&](T* v, const CellWalk& w, size_t k, T val) {
    if (per) put_images(v, w.i, w.j, k, val, g.nx, g.ny, (size_t)g.pitch, g.px != 0, g.py != 0);
  };

  // phase 0a: r = b - K x, u = D^-1 r, p = s = 0
  double bb_part = 0.0;
  for (CellWalk cw(first, stride, ch.t1, nx); cw.ok(); cw.next()) {
    const size_t k = g.idx(cw.i, cw.j);
    const T bk = a.b[k];
    const T rk = bk - K(x, k);
    r[k] = rk;
    u[k] = (kind[k] == 1 ? ireg : invd[k]) * rk;
    img(u, cw, k, u[k]);
    p[k] = (T)0;
    sv[k] = (T)0;
    bb_part += (double)bk * (double)bk;
  }
  bool ok = grid_sync(a.bar, target);
  // phase 0b / phase 2: w = K u and the sums
  auto phase2 = [&](double bbp) {
    double v[6] = {0.0, 0.0, 0.0, bbp, 0.0, 0.0};
    for (CellWalk cw(first, stride, ch.t1, nx); cw.ok(); cw.next()) {
      const size_t k = g.idx(cw.i, cw.j);
      const T wk = K((const T*)u, k);
      w[k] = wk;
      const double rk = (double)r[k], uk = (double)u[k];
      v[0] += rk * uk;
      v[1] += (double)wk * uk;
      v[2] += rk * rk;
      if (ZM && kind[k]) { v[4] += uk; v[5] += rk; }
    }
    // singular systems also need sum(w) over active cells: K 1 = 0 makes it zero in exact
    // arithmetic, so the correction of w.u uses sum(w) = 0 and only r.u needs sum(r)
    if (ZM) {
      block_sum_smem<6>(v, red);
      publish(a.partials, nb, v, 6);
    } else {
      double v4[4] = {v[0], v[1], v[2], v[3]};
      block_sum_smem<4>(v4, red);
      publish(a.partials, nb, v4, 4);
    }
  };
  auto finish = [&](double (&s6)[6]) {
    if (ZM) {
      grid_sum<6>(a.partials, nb, s6, sm);
    } else {
      double s4[4];
      grid_sum<4>(a.partials, nb, s4, sm);
      s6[0] = s4[0]; s6[1] = s4[1]; s6[2] = s4[2]; s6[3] = s4[3]; s6[4] = 0.0; s6[5] = 0.0;
    }
  };
  if (ok) {
    phase2(bb_part);
    ok = grid_sync(a.bar, target);
  }
  if (ok) {
    double s6[6];
    finish(s6);
    if (threadIdx.x == 0) {
      const double m = ZM ? s6[4] / a.n_act : 0.0;
      const double gamma = s6[0] - m * s6[5];
      const double delta = s6[1];  // (K u, u - m) = (K u, u) since sum over active of K u is zero
      S.zmean = m;
      S.rr = s6[2];
      S.bb = s6[3];
      S_gamma = gamma;
      S.alpha = delta != 0.0 ? gamma / delta : 0.0;
      S_alpha_prev = S.alpha;
      S.beta = 0.0;
      S.it = 0;
      S.stop = (S.bb == 0.0 || S.rr <= a.tol * a.tol * S.bb) ? 1 : (a.max_iter <= 0 ? 2 : 0);
    }
    __syncthreads();
  }
  if (ok && S.bb == 0.0)
    for (CellWalk cw(first, stride, ch.t1, nx); cw.ok(); cw.next()) x[g.idx(cw.i, cw.j)] = (T)0;
  while (ok && S.stop == 0) {
    // phase 1
    {
      const T ta = (T)S.alpha, tb = (T)S.beta, tm = (T)S.zmean;
      for (CellWalk cw(first, stride, ch.t1, nx); cw.ok(); cw.next()) {
        const size_t k = g.idx(cw.i, cw.j);
        const int8_t kk = kind[k];
        const T uk = ZM ? u[k] - (kk ? tm : (T)0) : u[k];
        const T pk = uk + tb * p[k];
        const T sk = w[k] + tb * sv[k];
        p[k] = pk;
        sv[k] = sk;
        x[k] += ta * pk;
        const T rk = r[k] - ta * sk;
        r[k] = rk;
        const T un = (kk == 1 ? ireg : invd[k]) * rk;
        u[k] = un;
        img(u, cw, k, un);
      }
    }
    if (!grid_sync(a.bar, target)) { ok = false; break; }
    phase2(0.0);
    if (!grid_sync(a.bar, target)) { ok = false; break; }
    double s6[6];
    finish(s6);
    if (threadIdx.x == 0) {
      const double m = ZM ? s6[4] / a.n_act : 0.0;
      const double gamma = s6[0] - m * s6[5];
      const double delta = s6[1];
      const double beta = gamma / S_gamma;
      const double alpha = gamma / (delta - beta * gamma / S_alpha_prev);
      S.zmean = m;
      S.beta = beta;
      S.alpha = alpha;
      S_alpha_prev = alpha;
      S_gamma = gamma;
      S.rr = s6[2];
      S.it += 1;
      S.stop = S.rr <= a.tol * a.tol * S.bb ? 1 : (S.it >= a.max_iter ? 2 : 0);
    }
    __syncthreads();
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const bool conv = ok && S.stop == 1;
    a.out.iters[0] = ok ? S.it : 0;
    a.out.rr[0] = ok ? S.rr : 0.0;
    a.out.bb[0] = ok ? S.bb : 0.0;
    a.out.converged[0] = conv ? 1 : 0;
    if (a.out.total && ok) a.out.total[0] += S.it;
    if (!conv && a.out.nconv) a.out.nconv[0] += 1;
  }
}

// ---------------------------------------------------------------------------------------
// Batched solve: the single-reduction Jacobi PCG above for many independent systems in one
// cooperative launch.  Block b serves case block_case[b] (a contiguous range of blocks per
// case, sized by the host in proportion to the expected work); each case reduces over its own
// blocks, all cases share the barriers, and a converged case's blocks idle through the
// remaining barriers.  The loop ends when no block reports a running case (a grid-wide sum
// read after a barrier, so every block takes the same decision).
// ---------------------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(kPcgThreads, 2) k_pcg_poisson_cg_batch(const BatchEntry<T>* __restrict__ cases,
                                                                        const int* __restrict__ block_case,
                                                                        BatchControl ctl) {
  __shared__ double red[6][kPcgThreads];
  __shared__ double sm[8];
  __shared__ PcgScalars S;
  __shared__ double S_alpha_prev, S_gamma;
  unsigned int target = 0;
  const int NB = gridDim.x;
  const int ci = block_case[blockIdx.x];
  const BatchEntry<T>& E = cases[ci];
  const PoissonSolve<T>& a = E.a;
  const bool ZM = a.zero_mean != 0;
  const Geom g = a.g;
  const int nx = g.nx;
  const int ncell = g.nx * g.ny;
  const int lb = blockIdx.x - E.block0, nbc = E.nblocks;
  const int t0 = (int)((long long)ncell * lb / nbc), t1 = (int)((long long)ncell * (lb + 1) / nbc);
  const int first = t0 + threadIdx.x, stride = blockDim.x;
  const KRow<T> K{a.cu, a.cv, a.dk, a.kind, (T)a.creg_x, (T)a.creg_y, (T)a.dreg, (size_t)g.pitch};
  const T* __restrict__ invd = a.invd;
  const int8_t* __restrict__ kind = a.kind;
  T* __restrict__ x = a.x;
  T* __restrict__ r = a.r;
  T* __restrict__ u = a.z;
  T* __restrict__ w = a.q;
  T* __restrict__ p = a.p0;
  T* __restrict__ sv = a.p1;
  const T ireg = (T)a.invd_reg;

  double bb_part = 0.0;
  for (CellWalk cw(first, stride, t1, nx); cw.ok(); cw.next()) {
    const size_t k = g.idx(cw.i, cw.j);
    const T bk = a.b[k];
    const T rk = bk - K(x, k);
    r[k] = rk;
    u[k] = (kind[k] == 1 ? ireg : invd[k]) * rk;
    p[k] = (T)0;
    sv[k] = (T)0;
    bb_part += (double)bk * (double)bk;
  }
  bool ok = grid_sync(ctl.bar, target);
  auto phase2 = [&](bool run, double bbp) {
    double v[6] = {0.0, 0.0, 0.0, bbp, 0.0, 0.0};
    if (run) {
      for (CellWalk cw(first, stride, t1, nx); cw.ok(); cw.next()) {
        const size_t k = g.idx(cw.i, cw.j);
        const T wk = K((const T*)u, k);
        w[k] = wk;
        const double rk = (double)r[k], uk = (double)u[k];
        v[0] += rk * uk;
        v[1] += (double)wk * uk;
        v[2] += rk * rk;
        if (ZM && kind[k]) { v[4] += uk; v[5] += rk; }
      }
    }
    block_sum_smem<6>(v, red);
    publish(ctl.partials, NB, v, 6);
  };
  if (ok) {
    phase2(true, bb_part);
    ok = grid_sync(ctl.bar, target);
  }
  if (ok) {
    double s6[6];
    range_sum<6>(ctl.partials, NB, E.block0, nbc, s6, sm);
    if (threadIdx.x == 0) {
      const double m = ZM ? s6[4] / a.n_act : 0.0;
      S.zmean = m;
      S.rr = s6[2];
      S.bb = s6[3];
      S_gamma = s6[0] - m * s6[5];
      S.alpha = s6[1] != 0.0 ? S_gamma / s6[1] : 0.0;
      S_alpha_prev = S.alpha;
      S.beta = 0.0;
      S.it = 0;
      S.stop = (S.bb == 0.0 || S.rr <= a.tol * a.tol * S.bb) ? 1 : (a.max_iter <= 0 ? 2 : 0);
    }
    __syncthreads();
  }
  if (ok && S.bb == 0.0)
    for (CellWalk cw(first, stride, t1, nx); cw.ok(); cw.next()) x[g.idx(cw.i, cw.j)] = (T)0;
  while (ok) {
    const bool run = S.stop == 0;
    if (run) {
      const T ta = (T)S.alpha, tb = (T)S.beta, tm = (T)S.zmean;
      for (CellWalk cw(first, stride, t1, nx); cw.ok(); cw.next()) {
        const size_t k = g.idx(cw.i, cw.j);
        const int8_t kk = kind[k];
        const T uk = ZM ? u[k] - (kk ? tm : (T)0) : u[k];
        const T pk = uk + tb * p[k];
        const T sk = w[k] + tb * sv[k];
        p[k] = pk;
        sv[k] = sk;
        x[k] += ta * pk;
        const T rk = r[k] - ta * sk;
        r[k] = rk;
        u[k] = (kk == 1 ? ireg : invd[k]) * rk;
      }
    }
    if (threadIdx.x == 0) ctl.running[blockIdx.x] = run ? 1 : 0;
    if (!grid_sync(ctl.bar, target)) { ok = false; break; }
    {
      // number of blocks whose case is still iterating (identical in every block)
      __shared__ int s_any;
      if (threadIdx.x < 32) {
        int c = 0;
        for (int b = threadIdx.x; b < NB; b += 32) c += __ldcg(&ctl.running[b]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
        if (threadIdx.x == 0) s_any = c;
      }
      __syncthreads();
      if (s_any == 0) break;
    }
    phase2(run, 0.0);
    if (!grid_sync(ctl.bar, target)) { ok = false; break; }
    double s6[6];
    range_sum<6>(ctl.partials, NB, E.block0, nbc, s6, sm);
    if (threadIdx.x == 0 && run) {
      const double m = ZM ? s6[4] / a.n_act : 0.0;
      const double gamma = s6[0] - m * s6[5];
      const double beta = gamma / S_gamma;
      const double alpha = gamma / (s6[1] - beta * gamma / S_alpha_prev);
      S.zmean = m;
      S.beta = beta;
      S.alpha = alpha;
      S_alpha_prev = alpha;
      S_gamma = gamma;
      S.rr = s6[2];
      S.it += 1;
      S.stop = S.rr <= a.tol * a.tol * S.bb ? 1 : (S.it >= a.max_iter ? 2 : 0);
    }
    __syncthreads();
  }
  if (lb == 0 && threadIdx.x == 0) {
    const bool conv = ok && S.stop == 1;
    a.out.iters[0] = ok ? S.it : 0;
    a.out.rr[0] = ok ? S.rr : 0.0;
    a.out.bb[0] = ok ? S.bb : 0.0;
    a.out.converged[0] = conv ? 1 : 0;
    if (a.out.total && ok) a.out.total[0] += S.it;
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
  return sms * 4 * 8 + sms * 4 * 4;  // blocks (at most 4 per SM) times values per reduction, then
                                     // the FP32 partials of the mixed solves (8 floats per block)
}
size_t pcg_float_partials_offset() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return (size_t)sms * 4 * 8;
}

template <class T, bool ZM>
static const void* poisson_kernel(int cheb) {
  switch (cheb) {
    case 2: return (const void*)k_pcg_poisson<T, ZM, 2>;
    case 3: return (const void*)k_pcg_poisson<T, ZM, 3>;
    case 4: return (const void*)k_pcg_poisson<T, ZM, 4>;
    case 5: return (const void*)k_pcg_poisson<T, ZM, 5>;
    case 6: return (const void*)k_pcg_poisson<T, ZM, 6>;
    case 8: return (const void*)k_pcg_poisson<T, ZM, 8>;
    default: return (const void*)k_pcg_poisson_cg<T, ZM>;
  }
}

bool cheb_degree_supported(int k) { return k == 1 || (k >= 2 && k <= 6) || k == 8; }

template <class T>
cudaError_t run_poisson_pcg(PoissonSolve<T> a, cudaStream_t st) {
  const int cheb = a.cheb > 1 ? a.cheb : 1;
  const void* fn = a.zero_mean ? poisson_kernel<T, true>(cheb) : poisson_kernel<T, false>(cheb);
  const int blocks = coop_blocks(fn, kPcgThreads, 2);
  if (a.zero_mean) {
    // singular system: warm start and right-hand side projected onto zero-mean fields
    k_zero_mean_partials<T><<<blocks, kPcgThreads, 0, st>>>(a.g, a.kind, a.x, a.partials);
    k_zero_mean_apply<T><<<blocks, kPcgThreads, 0, st>>>(a.g, a.kind, a.x, a.partials, blocks, a.n_act);
    k_zero_mean_partials<T><<<blocks, kPcgThreads, 0, st>>>(a.g, a.kind, a.b, a.partials);
    k_zero_mean_apply<T><<<blocks, kPcgThreads, 0, st>>>(a.g, a.kind, a.b, a.partials, blocks, a.n_act);
  }
  cudaMemsetAsync(a.bar.count, 0, sizeof(unsigned int) * kBarWords, st);
  void* params[] = {&a};
  return cudaLaunchCooperativeKernel(fn, blocks, kPcgThreads, params, 0, st);
}
template cudaError_t run_poisson_pcg<double>(PoissonSolve<double>, cudaStream_t);

int batch_blocks() { return coop_blocks((const void*)k_pcg_poisson_cg_batch<double>, kPcgThreads, 2); }

// x minus its mean over the active cells, in FP64 (the null-space projection of a singular
// system, end of Sec. 4.6); partials holds at least poisson_zero_mean_blocks() values.
int poisson_zero_mean_blocks() { return coop_blocks((const void*)k_zero_mean_partials<double>, kPcgThreads, 2); }
cudaError_t project_zero_mean(const Geom& g, const int8_t* act, double* x, double* partials, double n_act,
                              cudaStream_t st) {
  const int blocks = poisson_zero_mean_blocks();
  k_zero_mean_partials<double><<<blocks, kPcgThreads, 0, st>>>(g, act, x, partials);
  k_zero_mean_apply<double><<<blocks, kPcgThreads, 0, st>>>(g, act, x, partials, blocks, n_act);
  return cudaGetLastError();
}

// Singular systems of a batch: warm start and right-hand side projected onto zero mean
// (what run_poisson_pcg does for a single solve), then one cooperative launch for all.
template <class T>
cudaError_t run_poisson_batch(const PoissonSolve<T>* host_cases, int ncase, const BatchEntry<T>* dev_cases,
                              const int* dev_block_case, BatchControl ctl, int blocks, cudaStream_t st) {
  for (int c = 0; c < ncase; ++c) {
    const PoissonSolve<T>& a = host_cases[c];
    if (!a.zero_mean) continue;
    k_zero_mean_partials<T><<<blocks, kPcgThreads, 0, st>>>(a.g, a.kind, a.x, ctl.partials);
    k_zero_mean_apply<T><<<blocks, kPcgThreads, 0, st>>>(a.g, a.kind, a.x, ctl.partials, blocks, a.n_act);
    k_zero_mean_partials<T><<<blocks, kPcgThreads, 0, st>>>(a.g, a.kind, a.b, ctl.partials);
    k_zero_mean_apply<T><<<blocks, kPcgThreads, 0, st>>>(a.g, a.kind, a.b, ctl.partials, blocks, a.n_act);
  }
  cudaMemsetAsync(ctl.bar.count, 0, sizeof(unsigned int) * kBarWords, st);
  const void* fn = (const void*)k_pcg_poisson_cg_batch<T>;
  void* params[] = {(void*)&dev_cases, (void*)&dev_block_case, &ctl};
  return cudaLaunchCooperativeKernel(fn, blocks, kPcgThreads, params, 0, st);
}
template cudaError_t run_poisson_batch<double>(const PoissonSolve<double>*, int, const BatchEntry<double>*, const int*,
                                               BatchControl, int, cudaStream_t);
template cudaError_t run_poisson_batch<float>(const PoissonSolve<float>*, int, const BatchEntry<float>*, const int*,
                                              BatchControl, int, cudaStream_t);
template cudaError_t run_poisson_pcg<float>(PoissonSolve<float>, cudaStream_t);


}  // namespace ccm
