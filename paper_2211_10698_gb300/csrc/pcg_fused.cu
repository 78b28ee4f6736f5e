// FP64 pressure Poisson solve (Eq. pm_poisson) by CG on the Jacobi-scaled system (the
// iteration of pcg_scaled.cu) with ONE grid barrier per iteration.
//
// In pcg_scaled.cu an iteration needs two device-wide barriers: one so that the stencil
// w = K~ r sees the neighbours' new residual, one for the dot products.  Here each block
// owns a 2-D tile of cells and computes the new residual of the one-cell ring around its tile
// itself, from the previous iteration's vectors:
//     r_{i+1} = r_i - alpha_i (w_i + beta_i s_{i-1})      (= r_i - alpha_i s_i),
// so the stencil needs no other block's work of the same iteration and only the reduction
// needs a barrier.  r, w and s are double-buffered by iteration parity: iteration i reads
// buffer i%2 everywhere and writes buffer (i+1)%2 for its own cells, so the ring cells a
// neighbouring block reads are never the ones being written.
//
// Per iteration, in each block:
//   1. own cells: s_i, p_i, x~ += alpha p_i, r_{i+1} (written to the next buffers);
//      ring cells: r_{i+1} into shared memory (zero outside the domain)
//   2. block barrier; own cells: w_{i+1} = K~ r_{i+1} (neighbours inside the tile from the
//      next buffer, on the ring from shared memory), the sums; block sum; grid barrier
//   3. every block sums the partials in the same order and forms the scalars.
// With one barrier per iteration a block can publish the next iteration's partials while a
// slower block still reads this iteration's, so the partials alternate between two sets of
// rows by iteration parity.
// Tiles are TX x TY cells (TX a power of two, 32..512), one per block; the host picks the
// shape that makes the largest tile smallest.
//
// Two instantiations of the same iteration: k_pcg_poisson_f1 keeps x~, r, p, s and w in global
// memory (L2); k_pcg_poisson_f2 keeps its tile's x~, r, p, s, w and row kinds in shared memory
// for the whole solve.  Only the tile's perimeter cells are read by other blocks (for their
// ring), so f2 publishes r, w and s of its perimeter to the double-buffered global arrays once
// per iteration and touches nothing else in global memory until the final x~ -> x.  Its
// x~ += alpha p_i, which no other block reads, runs between the block's arrival at the grid
// barrier and its wait, in the time the barrier would otherwise idle.
// The sums of the iterations (reductions 1, 2, ...) are exact fixed-point sums that travel
// with the grid barrier (pcg_fixed.cuh): the block's arrival adds its digit sums to words in
// global memory and the wait on those words ends with the grid's sums in hand, so neither the
// block sum nor the grid sum is a chain of FP64 additions.  Reduction 0 (phase 0) and the
// rare reduction whose values leave the fixed-point window take the FP64 sums.
#include <algorithm>

#include "pcg_common.cuh"
#include "pcg_fixed.cuh"

namespace ccm {

namespace {

constexpr int kNT = 512;  // threads per block

// RES: the tile's vectors live in shared memory (f2); otherwise in global memory (f1).
template <bool RES>
__device__ __forceinline__ void fused_body(const FusedSolve& f) {
  __shared__ double red[4][kNT];
  __shared__ double bsum[8];
  __shared__ double gsum[8];
  __shared__ double sc_alpha, sc_beta, sc_igamma, sc_den, sc_rr, sc_bb;
  __shared__ double sc_igamma_next, sc_den_next;
  __shared__ int sc_it, sc_stop;
  __shared__ FxShared fxs;
  // dynamic shared memory: with RES x~, p, s, w of the tile (TX*TY each) and r~ of the tile in
  // a one-cell frame ((TX+2)*(TY+2), the frame holding the ring), then the ring
  // [W: TY][E: TY][S: TX][N: TX] (used without RES), then with RES the tile's row kinds, then
  // the list, then with RES and f.lcache the five scaled coefficients of the first kNT listed
  // cells (8-byte aligned: TX is a multiple of 32)
  extern __shared__ double dyn[];
  unsigned int target = 0;
  const ScaledSolve& a = f.a;
  const int nb = gridDim.x;
  const Geom g = a.g;
  const int nx = g.nx, ny = g.ny, P = g.pitch;
  const int TX = f.TX, TY = f.TY;
  const bool active = (int)blockIdx.x < f.ntiles;
  const int bx = blockIdx.x % f.nbx, by = blockIdx.x / f.nbx;
  const int i0 = bx * TX, j0 = by * TY;
  const int i1 = active ? min(i0 + TX, nx) : i0, j1 = active ? min(j0 + TY, ny) : j0;
  const int tx = threadIdx.x % TX, ty0 = threadIdx.x / TX, RP = kNT / TX;
  const int ci = i0 + tx;  // this thread's column
  const bool col = ci < i1;
  const int TXY = TX * TY;
  double* const sx = dyn;  // the RES arrays (unused otherwise)
  double* const sp = dyn + TXY;
  double* const ss = dyn + 2 * TXY;
  double* const sw = dyn + 3 * TXY;
  // RES: r~ of the tile with a one-cell frame that holds the ring, so that the stencil reads
  // every neighbour from one array without a branch
  const int TXP = TX + 2;
  double* const sr = dyn + 4 * TXY;
  double* const ring = RES ? dyn + 4 * TXY + TXP * (TY + 2) : dyn;
  int8_t* const skind = reinterpret_cast<int8_t*>(ring + 2 * (TX + TY));
  // tile-local index of own cell (i, j)
  auto lidx = [&](int i, int j) -> int { return (j - j0) * TX + (i - i0); };
  // index of cell (i, j) of the tile or its frame in the framed r~ (RES)
  auto lpad = [&](int i, int j) -> int { return (j - j0 + 1) * TXP + (i - i0 + 1); };
  // own cells on the tile's perimeter are read by the neighbouring tiles' rings
  auto perimeter = [&](int i, int j) -> bool { return i == i0 || i == i1 - 1 || j == j0 || j == j1 - 1; };
  // ring cells: W and E columns, then S and N rows, taken by threads t, t + kNT, ...
  const int nring = 2 * (j1 - j0) + 2 * (i1 - i0);
  // cell (ri, rj) of ring position t and its slot in `ring`; false outside the domain,
  // where the value is 0
  auto ring_cell = [&](int t, int& ri, int& rj, int& slot) -> bool {
    const int h = j1 - j0, w = i1 - i0;
    if (t < h) { ri = i0 - 1; rj = j0 + t; slot = t; }
    else if ((t -= h) < h) { ri = i1; rj = j0 + t; slot = TY + t; }
    else if ((t -= h) < w) { ri = i0 + t; rj = j0 - 1; slot = 2 * TY + t; }
    else { t -= w; ri = i0 + t; rj = j1; slot = 2 * TY + TX + t; }
    return ri >= 0 && ri < nx && rj >= 0 && rj < ny;
  };
  const int8_t* __restrict__ kinds = a.kinds;
  const double* __restrict__ cus = a.cus;
  const double* __restrict__ cvs = a.cvs;
  const double* __restrict__ sd = a.sd;
  const double ax = a.ax, ay = a.ay, dreg = a.dreg;
  double* __restrict__ xs = a.xs;
  double* __restrict__ p = a.p;
  const KRow<double> K{a.cu, a.cv, a.dk, a.kind, a.creg_x, a.creg_y, a.dreg, (size_t)P};

  // r~ at neighbour (i, j) of an own cell after step 1: inside the tile from the next buffer,
  // on the ring from shared memory
  auto rnb = [&](const double* rn, int i, int j) -> double {
    if constexpr (RES) return sr[lpad(i, j)];
    if (i < i0) return ring[j - j0];
    if (i >= i1) return ring[TY + (j - j0)];
    if (j < j0) return ring[2 * TY + (i - i0)];
    if (j >= j1) return ring[2 * TY + TX + (i - i0)];
    else return rn[g.idx(i, j)];
  };
  // r~ of own cell (i, j) after step 1
  auto rown = [&](const double* rn, int i, int j) -> double {
    if constexpr (RES) return sr[lpad(i, j)];
    else return rn[g.idx(i, j)];
  };
  // w~ of own cell (i, j) into the tile (RES, which also publishes the perimeter's r, w and s
  // for iteration parity `pub`) or into wn
  auto wput = [&](double* wn, int pub, int i, int j, double wk) {
    if constexpr (RES) {
      const int l = lidx(i, j);
      sw[l] = wk;
      if (perimeter(i, j)) {
        const size_t k = g.idx(i, j);
        f.R[pub][k] = sr[lpad(i, j)];
        f.W[pub][k] = wk;
        f.S[pub][k] = ss[l];
      }
    } else {
      wn[g.idx(i, j)] = wk;
    }
  };
  // Rows of cut cells and rows next to a Neumann side (kind 2) are listed per tile, in a fixed
  // order, at the start.  The stencil pass applies the constant stencil to every own cell, so
  // no warp diverges (an FP64 warp instruction costs the same however few of its lanes are
  // active); a second pass, spread densely over the threads, corrects the listed cells.
  // Inactive cells (identity rows, kind 0) get their exact solution x = b in phase 0 and zero
  // in every vector after it, so the stencil pass only has to write w = 0 there.  A tile with
  // more listed cells than the list holds takes the general row for every cell instead.
  int* const list = RES ? reinterpret_cast<int*>(skind + TXY) : reinterpret_cast<int*>(ring + 2 * (TX + TY));
  double* const lcoef = reinterpret_cast<double*>(list + TXY);  // RES: 5 x kNT
  __shared__ int s_scan[kNT / 32 + 1];
  int nlist = 0;
  bool general = false;
  {
    int mine = 0;
    if (col)
      for (int j = j0 + ty0; j < j1; j += RP) mine += kinds[g.idx(ci, j)] == 2;
    // exclusive scan of the counts over the block (thread order)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) s_scan[wid] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
      int acc = 0;
      for (int q = 0; q < kNT / 32; ++q) {
        const int c = s_scan[q];
        s_scan[q] = acc;
        acc += c;
      }
      s_scan[kNT / 32] = acc;
    }
    __syncthreads();
    nlist = s_scan[kNT / 32];
    general = nlist > f.list_cap;
    if (!general && mine > 0) {
      int at = s_scan[wid] + incl - mine;
      for (int j = j0 + ty0; j < j1; j += RP)
        if (kinds[g.idx(ci, j)] == 2) list[at++] = (j - j0) * TX + tx;
    }
    __syncthreads();
    if constexpr (RES) {
      // the first kNT listed cells' scaled coefficients, constant for the whole solve (listed
      // cell q is taken by thread kNT - 1 - q, see below)
      const int myq = kNT - 1 - (int)threadIdx.x;
      if (f.lcache && !general && myq < nlist) {
        const int q = list[myq];
        const size_t k = g.idx(i0 + q % TX, j0 + q / TX);
        lcoef[threadIdx.x] = cus[k];
        lcoef[kNT + threadIdx.x] = cus[k + 1];
        lcoef[2 * kNT + threadIdx.x] = cvs[k];
        lcoef[3 * kNT + threadIdx.x] = cvs[k + P];
        lcoef[4 * kNT + threadIdx.x] = sd[k];
      }
    }
  }
  // Listed cell q is computed by thread kNT - 1 - q (then kNT - 1 - q + kNT, ...): threads are
  // ordered by the first row they take, so the last threads have the fewest own rows (with
  // TY = 27 and 4 rows per pass, the last 128 threads take 6 rows and the others 7), and a
  // tile's listed cells fill those free slots before they lengthen any warp.  An FP64-bound
  // sub-partition's time is the sum over its warps, and the slowest tile sets every
  // iteration's barrier.
  const int myq = kNT - 1 - (int)threadIdx.x;
  // the general row at own cell (i, j) (any kind); w = K~ r and the sums of a row of kind km
  auto general_row = [&](const double* rn, int i, int j, double& rc_out) -> double {
    const size_t k = g.idx(i, j);
    const int8_t km = kinds[k];
    const double rc = rown(rn, i, j), rw = rnb(rn, i - 1, j), re = rnb(rn, i + 1, j);
    const double rs = rnb(rn, i, j - 1), rq = rnb(rn, i, j + 1);
    rc_out = rc;
    if (km == 1) return rc - ax * (rw + re) - ay * (rs + rq);
    if (km == 2) return rc - cus[k] * rw - cus[k + 1] * re - cvs[k] * rs - cvs[k + P] * rq;
    return rc;
  };
  auto diag_of = [&](int i, int j) -> double {
    const size_t k = g.idx(i, j);
    const int8_t km = kinds[k];
    return km == 1 ? dreg : (km == 2 ? sd[k] * sd[k] : 1.0);
  };
  // step 2 on own cells: w = K~ r (r in buffer rn, or the tile with RES), sums into v
  auto stencil = [&](const double* rn, double* wn, int pub, double (&v)[4]) {
    if (general) {
      if (col)
        for (int j = j0 + ty0; j < j1; j += RP) {
          double rc;
          const double wk = general_row(rn, ci, j, rc);
          wput(wn, pub, ci, j, wk);
          v[0] += rc * rc;
          v[1] += (diag_of(ci, j) - dreg) * (rc * rc);
          v[2] += wk * rc;
        }
      return;
    }
    // This thread's first listed cell: its values and coefficients are loaded before the
    // constant-stencil pass, so that their latency overlaps it.
    const int q0 = myq < nlist ? list[myq] : -1;
    int li = 0, lj = 0;
    double lr[5] = {0.0, 0.0, 0.0, 0.0, 0.0}, lc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (q0 >= 0) {
      li = i0 + q0 % TX;
      lj = j0 + q0 / TX;
      const size_t k = g.idx(li, lj);
      lr[0] = rown(rn, li, lj); lr[1] = rnb(rn, li - 1, lj); lr[2] = rnb(rn, li + 1, lj);
      lr[3] = rnb(rn, li, lj - 1); lr[4] = rnb(rn, li, lj + 1);
      if (RES && f.lcache) {
        lc[0] = lcoef[threadIdx.x]; lc[1] = lcoef[kNT + threadIdx.x]; lc[2] = lcoef[2 * kNT + threadIdx.x];
        lc[3] = lcoef[3 * kNT + threadIdx.x]; lc[4] = lcoef[4 * kNT + threadIdx.x];
      } else {
        lc[0] = cus[k]; lc[1] = cus[k + 1]; lc[2] = cvs[k]; lc[3] = cvs[k + P]; lc[4] = sd[k];
      }
    }
    // constant stencil on every own cell but the listed ones, two rows of this thread at a time
    if constexpr (RES) {
      if (col)
        for (int j = j0 + ty0; j < j1; j += RP) {
          const int l = lidx(ci, j);
          const int8_t km = skind[l];
          const double rc = sr[lpad(ci, j)], rw = rnb(rn, ci - 1, j), re = rnb(rn, ci + 1, j);
          const double rs = rnb(rn, ci, j - 1), rq = rnb(rn, ci, j + 1);
          const double wk = km == 0 ? 0.0 : rc - ax * (rw + re) - ay * (rs + rq);
          if (km != 2) {
            wput(wn, pub, ci, j, wk);
            v[0] += rc * rc;
            v[2] += wk * rc;
          }
        }
    } else {
      if (col)
        for (int j = j0 + ty0; j < j1; j += 2 * RP) {
          const bool two = j + RP < j1;
          const int jb = two ? j + RP : j;
          const size_t ka = g.idx(ci, j), kb = g.idx(ci, jb);
          const int8_t kma = kinds[ka], kmb = kinds[kb];
          const double rca = rn[ka], rwa = rnb(rn, ci - 1, j), rea = rnb(rn, ci + 1, j);
          const double rsa = rnb(rn, ci, j - 1), rqa = rnb(rn, ci, j + 1);
          const double rcb = rn[kb], rwb = rnb(rn, ci - 1, jb), reb = rnb(rn, ci + 1, jb);
          const double rsb = rnb(rn, ci, jb - 1), rqb = rnb(rn, ci, jb + 1);
          const double wa = kma == 0 ? 0.0 : rca - ax * (rwa + rea) - ay * (rsa + rqa);
          if (kma != 2) {
            wn[ka] = wa;
            v[0] += rca * rca;
            v[2] += wa * rca;
          }
          if (two) {
            const double wb = kmb == 0 ? 0.0 : rcb - ax * (rwb + reb) - ay * (rsb + rqb);
            if (kmb != 2) {
              wn[kb] = wb;
              v[0] += rcb * rcb;
              v[2] += wb * rcb;
            }
          }
        }
    }
    // the listed cells: the general row
    if (q0 >= 0) {
      const double wk = lr[0] - lc[0] * lr[1] - lc[1] * lr[2] - lc[2] * lr[3] - lc[3] * lr[4];
      wput(wn, pub, li, lj, wk);
      v[0] += lr[0] * lr[0];
      v[1] += (lc[4] * lc[4] - dreg) * (lr[0] * lr[0]);
      v[2] += wk * lr[0];
    }
    for (int q = myq + kNT; q < nlist; q += kNT) {
      const int loc = list[q];
      const int i = i0 + loc % TX, j = j0 + loc / TX;
      double rc;
      const double wk = general_row(rn, i, j, rc);
      wput(wn, pub, i, j, wk);
      v[0] += rc * rc;
      v[1] += (diag_of(i, j) - dreg) * (rc * rc);
      v[2] += wk * rc;
    }
  };
  auto reduce = [&](const double (&v)[4], int nv, double* rows) {
    if (nv == 4) block_sum_warps<4, kNT>(v, red, bsum);
    else {
      const double v3[3] = {v[0], v[1], v[2]};
      block_sum_warps<3, kNT>(v3, red, bsum);
    }
    if (threadIdx.x == 0)
      for (int q = 0; q < nv; ++q) rows[(size_t)q * nb + blockIdx.x] = bsum[q];
  };
  double* const rows0 = a.partials;              // reductions 0, 2, 4, ...
  double* const rows1 = a.partials + 4 * nb;     // reductions 1, 3, 5, ...

  // Phase 0: x~ = D^1/2 x, r_0 = D^-1/2 (b - K x) into R[0], s_{-1} = p_{-1} = 0.
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  if (col)
    for (int j = j0 + ty0; j < j1; j += RP) {
      const size_t k = g.idx(ci, j);
      const double bk = a.b[k];
      const bool inactive = kinds[k] == 0;  // identity row: x = b exactly
      const double rk = inactive ? 0.0 : bk - K(a.x, k);
      const double x0 = inactive ? bk : sd[k] * a.x[k], r0 = a.isd[k] * rk;
      if (RES) {
        const int l = lidx(ci, j);
        sx[l] = x0;
        sr[lpad(ci, j)] = r0;
        ss[l] = 0.0;
        sp[l] = 0.0;
        skind[l] = kinds[k];
        if (perimeter(ci, j)) f.R[0][k] = r0;  // the neighbours' first ring; S[0] and W[0] follow
      } else {
        xs[k] = x0;
        f.R[0][k] = r0;
        f.S[0][k] = 0.0;
        p[k] = 0.0;
      }
      v[3] += bk * bk;
    }
  // the fixed-point words start at zero (the previous launch leaves one buffer in use); the
  // barriers of phase 0 order this before their first use
  if (blockIdx.x == 0)
    for (int q = threadIdx.x; q < 3 * kFxWords; q += kNT) f.fxacc[(size_t)q * kFxStride] = 0ULL;
  bool ok = grid_sync(a.bar, target);
  if (ok) {
    // w_0 = K~ r_0: every neighbour's r_0 is complete, read through the same ring path
    for (int t = threadIdx.x; t < nring; t += kNT) {
      int ri, rj, slot;
      const bool in = ring_cell(t, ri, rj, slot);
      const double rv0 = in ? f.R[0][g.idx(ri, rj)] : 0.0;
      if constexpr (RES) sr[lpad(ri, rj)] = rv0;
      else ring[slot] = rv0;
    }
    __syncthreads();
    stencil(f.R[0], f.W[0], 0, v);
    reduce(v, 4, rows0);
    ok = grid_sync(a.bar, target);
  }
  int fx_lo = 0;  // bottom of the fixed-point window of the next reduction (same in every block)
  if (ok) {
    double t[4];
    grid_sum<4>(rows0, nb, t, gsum);
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
    fx_lo = fx_window(t[0], t[1], t[2]);
  }
  int cur = 0;
  while (ok && sc_stop == 0) {
    const int nxt = cur ^ 1;
    const double al = sc_alpha, be = sc_beta;
    const double* __restrict__ rc_ = f.R[cur];
    const double* __restrict__ wc_ = f.W[cur];
    const double* __restrict__ sc_ = f.S[cur];
    double* __restrict__ rn_ = f.R[nxt];
    double* __restrict__ sn_ = f.S[nxt];
    // this thread's first ring cell: the neighbours' iteration-i values, published before the
    // last grid barrier, are loaded now so the L2 round trip overlaps step 1
    int pf_slot = 0, pf_ri = 0, pf_rj = 0;
    bool pf_in = false;
    double pf_r = 0.0, pf_w = 0.0, pf_s = 0.0;
    if (threadIdx.x < nring) {
      int ri, rj;
      pf_in = ring_cell(threadIdx.x, ri, rj, pf_slot);
      pf_ri = ri;
      pf_rj = rj;
      if (pf_in) {
        const size_t k = g.idx(ri, rj);
        pf_r = rc_[k];
        pf_w = wc_[k];
        pf_s = sc_[k];
      }
    }
    // step 1: own cells (RES: in the tile; otherwise two rows of this thread at a time with
    // their loads in flight)
    if (RES) {
      if (col)
        for (int j = j0 + ty0; j < j1; j += RP) {
          const int l = lidx(ci, j);
          const int lp = lpad(ci, j);
          const double sk = sw[l] + be * ss[l], pk = sr[lp] + be * sp[l];
          ss[l] = sk;
          sp[l] = pk;
          sr[lp] -= al * sk;
        }
    } else if (col)
      for (int j = j0 + ty0; j < j1; j += 2 * RP) {
        const bool two = j + RP < j1;
        const size_t k0 = g.idx(ci, j), k1 = two ? g.idx(ci, j + RP) : k0;
        const double r0 = rc_[k0], w0 = wc_[k0], s0 = sc_[k0], p0 = p[k0], x0 = xs[k0];
        const double r1 = rc_[k1], w1 = wc_[k1], s1 = sc_[k1], p1 = p[k1], x1 = xs[k1];
        {
          const double sk = w0 + be * s0, pk = r0 + be * p0;
          sn_[k0] = sk;
          p[k0] = pk;
          xs[k0] = x0 + al * pk;
          rn_[k0] = r0 - al * sk;
        }
        if (two) {
          const double sk = w1 + be * s1, pk = r1 + be * p1;
          sn_[k1] = sk;
          p[k1] = pk;
          xs[k1] = x1 + al * pk;
          rn_[k1] = r1 - al * sk;
        }
      }
    // ring cells: r_{i+1} from the neighbours' iteration-i vectors
    if (threadIdx.x < nring) {
      const double rv0 = pf_in ? pf_r - al * (pf_w + be * pf_s) : 0.0;
      if constexpr (RES) sr[lpad(pf_ri, pf_rj)] = rv0;
      else ring[pf_slot] = rv0;
    }
    for (int t = threadIdx.x + kNT; t < nring; t += kNT) {
      int ri, rj, slot;
      double rv = 0.0;
      if (ring_cell(t, ri, rj, slot)) {
        const size_t k = g.idx(ri, rj);
        rv = rc_[k] - al * (wc_[k] + be * sc_[k]);
      }
      if constexpr (RES) sr[lpad(ri, rj)] = rv;
      else ring[slot] = rv;
    }
    __syncthreads();
    v[0] = v[1] = v[2] = 0.0;
    stencil(rn_, f.W[nxt], nxt, v);
    // reduction sc_it + 1 in the rotating fixed-point buffers
    const int ri = sc_it + 1, buf = ri % 3;
    fx_arrive<kNT>(v, fx_lo, f.fxacc, buf, a.bar.absent, fxs);
    if constexpr (RES) {
      // x~ += alpha p_i is read by no other block and by nothing before the end: it runs between
      // this block's arrival at the grid barrier and its wait
      if (col)
        for (int j = j0 + ty0; j < j1; j += RP) {
          const int l = lidx(ci, j);
          sx[l] += al * sp[l];
        }
    }
    if (!fx_wait(f.fxacc, buf, (ri + 2) % 3, a.bar.budget, a.bar.err, fxs)) { ok = false; break; }
    double t[3];
    // every block takes the same branch: the overflow count is the grid's, and the test hook
    // depends on the reduction index only
    const bool forced = f.fx_fallback_every > 0 && ri % f.fx_fallback_every == 0;
    if (fxs.s[kFxWords - 1] == 0 && !forced) {
      if (threadIdx.x < kFxQ) gsum[threadIdx.x] = fx_value(&fxs.s[threadIdx.x * kFxDigits], fx_lo);
      __syncthreads();
      t[0] = gsum[0];
      t[1] = gsum[1];
      t[2] = gsum[2];
    } else {
      // a value outside the window (every block sees the same count): this reduction again in
      // FP64 through the partial rows and the counter barrier
      double* const rows = (sc_it & 1) ? rows0 : rows1;
      reduce(v, 3, rows);
      if (!grid_sync(a.bar, target)) { ok = false; break; }
      grid_sum<3>(rows, nb, t, gsum);
    }
    fx_lo = fx_window(t[0], t[1], t[2]);
    // beta = gamma / gamma_old; alpha = gamma / (delta - beta gamma / alpha_old).  The two
    // reciprocals are independent: 1/gamma (for the next beta) in warp 0, 1/den in warp 1,
    // which issue to different sub-partitions' FP64 pipes.
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
    cur = nxt;
  }
  if (col)
    for (int j = j0 + ty0; j < j1; j += RP) {
      const size_t k = g.idx(ci, j);
      a.x[k] = a.isd[k] * (RES ? sx[lidx(ci, j)] : xs[k]);
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

// __grid_constant__: the body takes the parameter by reference without a local copy
__global__ void __launch_bounds__(kNT, 2) k_pcg_poisson_f1(const __grid_constant__ FusedSolve f) {
  fused_body<false>(f);
}
__global__ void __launch_bounds__(kNT, 2) k_pcg_poisson_f2(const __grid_constant__ FusedSolve f) {
  fused_body<true>(f);
}

}  // namespace

// Tile shape for at most `blocks` blocks: TX a power of two in 32..512, as many tile rows as
// the blocks allow while a tile keeps about one cell per thread; the shape with the smallest
// largest tile wins (then the shortest ring).  One block per tile.
void fused_tiles(int nx, int ny, int blocks, int* TX, int* TY, int* nbx, int* ntiles) {
  long long best = -1, best_ring = 0;
  for (int tx = 32; tx <= 512; tx *= 2) {
    const int bxn = (nx + tx - 1) / tx;
    if (bxn > blocks) continue;
    const int wx = std::min(tx, nx);
    const int min_ty = (kNT + wx - 1) / wx;
    const int byn = std::max(1, std::min(blocks / bxn, (ny + min_ty - 1) / min_ty));
    const int ty = (ny + byn - 1) / byn;
    const long long cells = (long long)wx * ty, ring = 2LL * (wx + ty);
    if (best < 0 || cells < best || (cells == best && ring < best_ring)) {
      best = cells;
      best_ring = ring;
      *TX = tx;
      *TY = ty;
      *nbx = bxn;
      *ntiles = bxn * ((ny + ty - 1) / ty);
    }
  }
}

constexpr size_t kFusedSmemMax = 64 * 1024;  // ring and list of non-uniform cells, per block

int fused_blocks() {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaFuncSetAttribute(k_pcg_poisson_f1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFusedSmemMax);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pcg_poisson_f1, kNT, kFusedSmemMax);
  per = per > 2 ? 2 : (per < 1 ? 1 : per);
  return sms * per;
}

// Dynamic shared memory of a tile with its vectors resident (f2): x~, p, s, w, r~ with its
// one-cell frame, the ring, the row kinds, a list of up to one entry per cell and, with `cache`,
// the coefficients of kNT listed cells.
size_t fused_resident_smem(int TX, int TY, bool cache) {
  const size_t txy = (size_t)TX * (size_t)TY;
  return 4 * sizeof(double) * txy + sizeof(double) * ((size_t)TX + 2) * ((size_t)TY + 2) +
         sizeof(double) * 2 * ((size_t)TX + (size_t)TY) + txy + sizeof(int) * txy +
         (cache ? 5 * sizeof(double) * kNT : 0);
}

// Whether ntiles tiles of TX x TY cells with resident vectors fit the GPU at once: with the
// coefficient cache (2), only without it (1), or not at all (0).
int fused_resident_fit(int TX, int TY, int ntiles) {
  if (fused_resident_fits(TX, TY, ntiles, true)) return 2;
  return fused_resident_fits(TX, TY, ntiles, false) ? 1 : 0;
}
bool fused_resident_ok(int TX, int TY, int ntiles) { return fused_resident_fit(TX, TY, ntiles) != 0; }

bool fused_resident_fits(int TX, int TY, int ntiles, bool cache) {
  const size_t smem = fused_resident_smem(TX, TY, cache);
  int dev = 0, sms = 0, per = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (smem > (size_t)optin ||
      cudaFuncSetAttribute(k_pcg_poisson_f2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pcg_poisson_f2, kNT, smem) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return ntiles >= 1 && ntiles <= sms * std::min(per, 2);
}

cudaError_t run_poisson_fused(FusedSolve f, cudaStream_t st) {
  const int blocks = fused_blocks();
  if (f.TX == 0) fused_tiles(f.a.g.nx, f.a.g.ny, blocks, &f.TX, &f.TY, &f.nbx, &f.ntiles);
  if (f.ntiles < 1) return cudaErrorInvalidConfiguration;
  const void* kernel = (const void*)k_pcg_poisson_f1;
  size_t smem = 0;
  if (f.resident) {
    // the tile's vectors in shared memory: as many blocks as fit must hold every tile
    const int fit = fused_resident_fit(f.TX, f.TY, f.ntiles);
    if (fit == 0) return cudaErrorInvalidConfiguration;
    f.lcache = fit == 2 ? 1 : 0;
    smem = fused_resident_smem(f.TX, f.TY, f.lcache != 0);
    f.list_cap = f.TX * f.TY;
    kernel = (const void*)k_pcg_poisson_f2;
  } else {
    const size_t ring = sizeof(double) * 2 * ((size_t)f.TX + (size_t)f.TY);
    if (ring + sizeof(int) * 256 > kFusedSmemMax || f.ntiles > blocks) return cudaErrorInvalidConfiguration;
    // the list of non-uniform cells takes what is left, up to one entry per tile cell
    f.list_cap = (int)std::min<size_t>((kFusedSmemMax - ring) / sizeof(int), (size_t)f.TX * (size_t)f.TY);
    smem = ring + sizeof(int) * (size_t)f.list_cap;
  }
  cudaMemsetAsync(f.a.bar.count, 0, sizeof(unsigned int) * kBarWords, st);
  void* params[] = {&f};
  return cudaLaunchCooperativeKernel(kernel, f.ntiles, kNT, params, smem, st);
}

}  // namespace ccm
