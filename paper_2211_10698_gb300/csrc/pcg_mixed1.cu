// Mixed-precision pressure Poisson solve (Eq. pm_poisson) with ONE grid barrier per FP32
// iteration: the reliable-update CG of pcg_mixed.cu (FP32 single-reduction CG on the
// Jacobi-scaled correction equation, FP64 residual replacements) in the tile layout of
// pcg_fused.cu, extended to the Chebyshev preconditioner.
//
// pcg_mixed.cu separates every phase that reads neighbours by a grid barrier: the vector
// update, each of the k-1 Chebyshev steps and the stencil with its sums, i.e. k+1 barriers per
// iteration.  Here each block owns a 2-D tile and a band of width k around it:
//   1. own cells: s_i = w_i + beta s_{i-1}, p_i = u_i + beta p_{i-1}, e += alpha p_i,
//      r_{i+1} = r_i - alpha s_i (stored for the neighbours);
//      band cells: r_{i+1} = r_i - alpha (w_i + beta s_{i-1}) from the neighbours' vectors of
//      the previous iteration (double-buffered by parity, so nothing read is being written);
//   2. the Chebyshev steps in shared memory on a region that shrinks by one cell per step
//      (k-1 steps leave u = M^-1 r valid on the tile and its one-cell ring);
//   3. own cells: w_{i+1} = K~ u and the sums (r, u), (w, u), (r, r);
//   4. the grid barrier, then every block sums the partials in the same order.
// The Chebyshev iteration (Saad, Chebyshev acceleration; interval of ChebCoef) keeps its
// direction implicitly: d_j = z_j - z_{j-1}, so two iterate buffers and r suffice, and z_{j+1}
// overwrites z_{j-1} in place.  A replacement (FP64 residual) is rare and takes a few extra
// barriers: fold the correction into x, the FP64 residual and its norms, the new FP32
// residual, the preconditioner and stencil on it, and, when the direction is kept, the
// formed direction and its curvature.  Sums of FP32 values are FP32 per thread and block and
// across blocks in a fixed order; every reduction alternates between two sets of partial
// rows, which are rewritten only two reductions (and so one barrier) later.
#include <algorithm>

#include "pcg_cheb.cuh"
#include "pcg_common.cuh"

namespace ccm {

namespace {

constexpr int kNT = kPcgThreads;
constexpr int kB = 4;  // cells per thread whose global loads are in flight together

// FP32 grid sum of NV quantities (rows q * nb), warp q adding quantity q; result in every thread
template <int NV>
__device__ __forceinline__ void grid_sum_f32_rows(const float* rows, int nb, float (&out)[NV], float* smem) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (w < NV) {
    const float* src = rows + (size_t)w * nb;
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

// RES: the tile's p, s, e and w stay in shared memory for the whole solve (k_pcg_poisson_m2),
// and u (Chebyshev) stays in the region's last iterate; only the frame of own cells that the
// neighbours' bands read (within h of the tile's edge) is published as r, w and s per
// iteration.  Otherwise every own-cell vector lives in global memory (k_pcg_poisson_m1).
template <bool RES>
__device__ __forceinline__ void mixed1_body(const Mixed1Solve& f) {
  __shared__ double red[3][kNT];
  __shared__ float wred[3][kNT / 32];
  __shared__ double dsum[8];
  __shared__ float fsum[8];
  __shared__ double sc_sigma, sc_rr, sc_bb, sc_rr_ref;
  __shared__ float sc_alpha, sc_beta, sc_pscale, sc_igamma, sc_ialpha, sc_gref, sc_gfresh;
  __shared__ int sc_it, sc_stop, sc_replace, sc_nrep, sc_keep, sc_restart, sc_rep_it;
  extern __shared__ float dyn1[];
  unsigned int target = 0;
  const MixedSolve& a = f.m;
  const ScaledSolve& d = a.d;
  const Geom g = d.g;
  const int nx = g.nx, ny = g.ny, P = g.pitch;
  const int nb = gridDim.x;
  const int cheb = a.cheb > 1 ? a.cheb : 1;
  const int h = cheb;  // band width
  const int TX = f.TX, TY = f.TY;
  const bool active = (int)blockIdx.x < f.ntiles;
  const int bx = blockIdx.x % f.nbx, by = blockIdx.x / f.nbx;
  const int i0 = bx * TX, j0 = by * TY;
  const int i1 = active ? min(i0 + TX, nx) : i0, j1 = active ? min(j0 + TY, ny) : j0;
  const int RX = TX + 2 * h, RN = RX * (TY + 2 * h);
  float* const sr = dyn1;                 // r_{i+1} on the region
  float* const za = dyn1 + RN;            // Chebyshev iterates (cheb > 1)
  float* const zb = dyn1 + 2 * RN;
  int8_t* const sk = reinterpret_cast<int8_t*>(dyn1 + (cheb > 1 ? 3 : 1) * RN);
  auto ridx = [&](int i, int j) -> int { return (j - j0 + h) * RX + (i - i0 + h); };
  // RES: own-cell p, s, e, w after the row kinds (16-byte aligned)
  float* const sown = dyn1 + (cheb > 1 ? 3 : 1) * RN + ((RN + 15) / 16) * 4;
  float* const sp = sown;
  float* const ss = sown + TX * TY;
  float* const se = sown + 2 * TX * TY;
  float* const sw = sown + 3 * TX * TY;
  auto lidx = [&](int i, int j) -> int { return (j - j0) * TX + (i - i0); };
  // own cells the neighbours' bands read
  auto frame = [&](int i, int j) -> bool { return i < i0 + h || i >= i1 - h || j < j0 + h || j >= j1 - h; };
  // u = M^-1 r after precond_apply: the last Chebyshev iterate, or r itself
  float* const ubuf = cheb > 1 ? ((cheb & 1) ? za : zb) : sr;
  // The band's cells inside the domain, numbered: the rows above the tile, the rows below
  // (each over the band's columns), then the columns to its left and right (over the tile's
  // rows).  band_cell(t) gives cell t; false for t >= nband.
  const int b_ia = max(i0 - h, 0), b_ib = min(i1 + h, nx), b_ja = max(j0 - h, 0), b_jb = min(j1 + h, ny);
  const int b_w = b_ib - b_ia, b_h = j1 - j0;
  const int b_nt = (j0 - b_ja) * b_w, b_nb = (b_jb - j1) * b_w, b_nl = (i0 - b_ia) * b_h;
  const int nband = active ? b_nt + b_nb + b_nl + (b_ib - i1) * b_h : 0;
  auto band_cell = [&](int t, int& bi, int& bj) -> bool {
    if (t >= nband) return false;
    if (t < b_nt) { bj = b_ja + t / b_w; bi = b_ia + t % b_w; return true; }
    t -= b_nt;
    if (t < b_nb) { bj = j1 + t / b_w; bi = b_ia + t % b_w; return true; }
    t -= b_nb;
    if (t < b_nl) { bi = b_ia + t / b_h; bj = j0 + t % b_h; return true; }
    t -= b_nl;
    bi = i1 + t / b_h;
    bj = j0 + t % b_h;
    return true;
  };
  const int8_t* __restrict__ kinds = d.kinds;
  const float* __restrict__ cus = a.cus32;
  const float* __restrict__ cvs = a.cvs32;
  const double* __restrict__ isd = d.isd;
  double* __restrict__ x = d.x;
  double* __restrict__ r64 = d.r;
  float* __restrict__ Pv = f.P;
  float* __restrict__ Uv = f.U;
  float* __restrict__ Ev = f.E;
  const float ax = (float)d.ax, ay = (float)d.ay;
  constexpr float ith = (float)(1.0 / ChebCoef::theta);
  const double tol2 = d.tol * d.tol;
  float* const fpart = a.fpartials;  // two sets of three rows of nb floats
  int nred = 0;                      // reductions so far (the same in every block)

  const int nown = TX * TY;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int kW = kNT / 32;
  auto in_dom = [&](int i, int j) -> bool { return i >= 0 && i < nx && j >= 0 && j < ny; };
  // K~ z at region cell (i, j) of kind km, z in shared memory
  auto krow = [&](const float* z, int i, int j, int8_t km) -> float {
    const int q = ridx(i, j);
    const float zc = z[q];
    if (km == 1) return zc - ax * (z[q - 1] + z[q + 1]) - ay * (z[q - RX] + z[q + RX]);
    if (km == 2) {
      const size_t k = g.idx(i, j);
      return zc - cus[k] * z[q - 1] - cus[k + 1] * z[q + 1] - cvs[k] * z[q - RX] - cvs[k + P] * z[q + RX];
    }
    return zc;
  };

  // the region's row kinds (identity outside the domain) and zero vectors
  for (int q = threadIdx.x; q < RN; q += kNT) {
    const int i = i0 - h + q % RX, j = j0 - h + q / RX;
    sk[q] = (active && in_dom(i, j) && i < i1 + h && j < j1 + h) ? kinds[g.idx(i, j)] : (int8_t)0;
    sr[q] = 0.0f;
    if (cheb > 1) { za[q] = 0.0f; zb[q] = 0.0f; }
  }
  if (threadIdx.x == 0) {
    sc_keep = 0; sc_restart = 0; sc_rep_it = -1000; sc_sigma = 0.0; sc_igamma = 1.0f; sc_pscale = 1.0f;
    sc_it = 0; sc_stop = 0; sc_nrep = 0; sc_bb = 0.0; sc_alpha = 0.0f; sc_beta = 0.0f;
  }
  // own cells: zero direction, curvature (both parities) and correction
  for (int q = threadIdx.x; q < nown; q += kNT) {
    const int i = i0 + q % TX, j = j0 + q / TX;
    if (i >= i1 || j >= j1) continue;
    const size_t k = g.idx(i, j);
    if constexpr (RES) {
      sp[q] = 0.0f; ss[q] = 0.0f; se[q] = 0.0f; sw[q] = 0.0f;
    } else {
      Pv[k] = 0.0f; Ev[k] = 0.0f;
    }
    f.S[0][k] = 0.0f; f.S[1][k] = 0.0f;
  }
  __syncthreads();

  // R2 (and the start): r64 = D^-1/2 (b - K x) on own cells; ||r64||^2, ||b - K x||^2 (||b||^2)
  auto residual64 = [&](bool with_b) -> bool {
    const KRow<double> K{d.cu, d.cv, d.dk, d.kind, d.creg_x, d.creg_y, d.dreg, (size_t)P};
    double v[3] = {0.0, 0.0, 0.0};
    for (int q = threadIdx.x; q < nown; q += kNT) {
      const int i = i0 + q % TX, j = j0 + q / TX;
      if (i >= i1 || j >= j1) continue;
      const size_t k = g.idx(i, j);
      const double bk = d.b[k];
      const double rk = bk - K(x, k);
      const double rs = isd[k] * rk;
      r64[k] = rs;
      v[0] += rs * rs;
      v[1] += rk * rk;
      v[2] += bk * bk;
    }
    block_sum_warps<3>(v, red, dsum);
    if (threadIdx.x == 0)
      for (int q = 0; q < 3; ++q) d.partials[(size_t)q * nb + blockIdx.x] = dsum[q];
    if (!grid_sync(d.bar, target)) return false;
    double t[3];
    grid_sum<3>(d.partials, nb, t, dsum);
    if (threadIdx.x == 0) {
      if (with_b) sc_bb = t[2];
      sc_rr = t[1];
      sc_rr_ref = t[1];
      const double old = sc_sigma;
      sc_sigma = t[0] > 0.0 ? 1.0 / sqrt(t[0]) : 1.0;
      const double c = old > 0.0 ? sc_sigma / old : 0.0;
      sc_pscale = (float)c;
      sc_igamma = (float)((double)sc_igamma / (c * c + (c == 0.0)));
      if (sc_bb == 0.0 || sc_rr <= tol2 * sc_bb) sc_stop = 1;
    }
    __syncthreads();
    return true;
  };

  // Chebyshev steps on the region (r in sr), then w = K~ u and the sums on own cells; stores
  // w into Wn and (cheb > 1) u into U.  v = (r, u), (w, u), (r, r).
  auto precond_apply = [&](float* Wn, float (&v)[3]) {
    const float* u = sr;
    if (cheb > 1) {
      // z1 = r / theta on the whole region (z0 = 0 in zb)
      for (int q = threadIdx.x; q < RN; q += kNT) { za[q] = ith * sr[q]; zb[q] = 0.0f; }
      __syncthreads();
      for (int js = 1; js < cheb; ++js) {
        float c1, c2;
        cheb_step_coef(js, c1, c2);
        float* zin = (js & 1) ? za : zb;   // z_j
        float* zio = (js & 1) ? zb : za;   // z_{j-1} in, z_{j+1} out
        const int m = h - js;              // the band width this step leaves valid
        // warps take rows, lanes columns (no division per cell)
        for (int j = max(j0 - m, 0) + warp; j < min(j1 + m, ny); j += kW)
          for (int i = max(i0 - m, 0) + lane; i < min(i1 + m, nx); i += 32) {
            const int q = ridx(i, j);
            const float zj = zin[q];
            const float kz = krow(zin, i, j, sk[q]);
            const float dn = c1 * (zj - zio[q]) + c2 * (sr[q] - kz);
            zio[q] = zj + dn;
          }
        __syncthreads();
      }
      u = (cheb & 1) ? za : zb;
    }
    for (int j = j0 + warp; j < j1; j += kW)
      for (int i = i0 + lane; i < i1; i += 32) {
      const int rq = ridx(i, j);
      const size_t k = g.idx(i, j);
      const float uk = u[rq], rk = sr[rq];
      const float wk = krow(u, i, j, sk[rq]);
      if constexpr (RES) {
        sw[lidx(i, j)] = wk;
        if (frame(i, j)) Wn[k] = wk;
      } else {
        Wn[k] = wk;
        if (cheb > 1) Uv[k] = uk;
      }
      v[0] += rk * uk;
      v[1] += wk * uk;
      v[2] += rk * rk;
    }
  };

  // block sums of v into the partial rows of this reduction; arrive, optional work, wait
  auto reduce_arrive = [&](const float (&v)[3], int nv) -> float* {
    float* rows = fpart + (size_t)(nred & 1) * 3 * nb;
    ++nred;
    float v3[3] = {v[0], v[1], v[2]};
    block_sum_f32<3>(v3, wred, fsum);
    if (threadIdx.x == 0)
      for (int q = 0; q < nv; ++q) rows[(size_t)q * nb + blockIdx.x] = fsum[q];
    grid_arrive(d.bar, target);
    return rows;
  };

  // scalars after the sums of an apply (fresh: on a replaced residual), as in pcg_mixed.cu
  auto scalars = [&](const float (&t)[3], bool fresh) {
    if (threadIdx.x == 0) {
      const float gamma = t[0], delta = t[1], rr32 = t[2];
      if (!fresh) {
        sc_it += 1;
        sc_pscale = 1.0f;
        sc_keep = 0;
      }
      if (fresh) sc_gref = rr32;
      // rr32 / gref <= drop^2, or the estimate rr_ref rr32 / gref of the unscaled residual
      // meets the tolerance (multiplied out: no FP64 division on the serial path)
      const double gref = sc_gref;
      sc_replace = !fresh && gref > 0.0 &&
                   ((double)rr32 <= a.drop * a.drop * gref || sc_rr_ref * (double)rr32 <= tol2 * sc_bb * gref) ? 1 : 0;
      if (!sc_replace) {
        if (fresh && sc_it == 0 && sc_nrep == 0) {
          sc_beta = 0.0f;
          sc_alpha = gamma / delta;
          sc_igamma = 1.0f / gamma;
          sc_ialpha = 1.0f / sc_alpha;
        } else if (fresh && sc_restart) {
          sc_beta = 0.0f;
          sc_alpha = gamma / delta;
          sc_igamma = 1.0f / gamma;
          sc_ialpha = 1.0f / sc_alpha;
          sc_pscale = 0.0f;
          sc_restart = 0;
        } else if (fresh) {
          sc_beta = gamma * sc_igamma;
          sc_gfresh = gamma;
          sc_keep = 1;
        } else {
          const float beta = gamma * sc_igamma;
          const float den = delta - beta * gamma * sc_ialpha;
          if (den > 0.0f && den < INFINITY) {
            sc_beta = beta;
            sc_alpha = gamma / den;
            sc_igamma = 1.0f / gamma;
            sc_ialpha = 1.0f / sc_alpha;
          } else {
            sc_replace = 1;
            sc_restart = 1;
          }
        }
      }
    }
    __syncthreads();
  };

  // a fresh residual: r = sigma r64 into Rc (own cells), barrier, the region from Rc, the
  // preconditioner and stencil into Wc, the sums and the scalars
  auto fresh_apply = [&](float* Rc, float* Wc) -> bool {
    const double sig = sc_sigma;
    for (int q = threadIdx.x; q < nown; q += kNT) {
      const int i = i0 + q % TX, j = j0 + q / TX;
      if (i >= i1 || j >= j1) continue;
      const size_t k = g.idx(i, j);
      const float rv = (float)(sig * r64[k]);
      if constexpr (RES) {
        sr[ridx(i, j)] = rv;
        if (frame(i, j)) Rc[k] = rv;
      } else {
        Rc[k] = rv;
      }
    }
    if (!grid_sync(d.bar, target)) return false;
    for (int q = threadIdx.x; q < RN; q += kNT) {
      const int i = i0 - h + q % RX, j = j0 - h + q / RX;
      const bool own = i >= i0 && i < i1 && j >= j0 && j < j1;
      if (RES && own) continue;  // already in sr
      sr[q] = (active && in_dom(i, j) && i < i1 + h && j < j1 + h) ? __ldcg(&Rc[g.idx(i, j)]) : 0.0f;
    }
    __syncthreads();
    float v[3] = {0.0f, 0.0f, 0.0f};
    precond_apply(Wc, v);
    const float* rows = reduce_arrive(v, 3);
    if (!grid_wait(d.bar, target)) return false;
    float t[3];
    grid_sum_f32_rows<3>(rows, nb, t, fsum);
    scalars(t, true);
    return true;
  };

  // phase P after a replacement: p = u + beta' p, s = w + beta' s (stored), alpha = gamma / (p, s)
  auto phase_p = [&](const float* Rc, const float* Wc, float* Sc) -> bool {
    const float be = sc_beta * sc_pscale;
    float v[3] = {0.0f, 0.0f, 0.0f};
    for (int q = threadIdx.x; q < nown; q += kNT) {
      const int i = i0 + q % TX, j = j0 + q / TX;
      if (i >= i1 || j >= j1) continue;
      const size_t k = g.idx(i, j);
      float pk, sk_;
      if constexpr (RES) {
        const int l = lidx(i, j);
        pk = ubuf[ridx(i, j)] + be * sp[l];
        sk_ = sw[l] + be * ss[l];
        sp[l] = pk;
        ss[l] = sk_;
        if (frame(i, j)) Sc[k] = sk_;
      } else {
        const float uk = cheb > 1 ? Uv[k] : Rc[k];
        pk = uk + be * Pv[k];
        sk_ = Wc[k] + be * Sc[k];
        Pv[k] = pk;
        Sc[k] = sk_;
      }
      v[0] += pk * sk_;
    }
    const float* rows = reduce_arrive(v, 1);
    if (!grid_wait(d.bar, target)) return false;
    float t[1];
    grid_sum_f32_rows<1>(rows, nb, t, fsum);
    if (threadIdx.x == 0) {
      sc_alpha = sc_gfresh / t[0];
      sc_igamma = 1.0f / sc_gfresh;
      sc_ialpha = 1.0f / sc_alpha;
    }
    __syncthreads();
    return true;
  };

  // R1: x += D^-1/2 e / sigma on own cells, e = 0 (when clear)
  auto fold = [&](bool clear) {
    const double isig = 1.0 / sc_sigma;
    for (int q = threadIdx.x; q < nown; q += kNT) {
      const int i = i0 + q % TX, j = j0 + q / TX;
      if (i >= i1 || j >= j1) continue;
      const size_t k = g.idx(i, j);
      if constexpr (RES) {
        x[k] += isd[k] * (double)se[q] * isig;
        if (clear) se[q] = 0.0f;
      } else {
        x[k] += isd[k] * (double)Ev[k] * isig;
        if (clear) Ev[k] = 0.0f;
      }
    }
  };

  int cur = 0;
  bool ok = residual64(true);
  if (ok && sc_stop == 0) ok = fresh_apply(f.R[cur], f.W[cur]);
  if (ok && sc_stop == 0 && sc_keep) ok = phase_p(f.R[cur], f.W[cur], f.S[cur]);
  bool limit = false;
  while (ok && sc_stop == 0) {
    if (sc_it >= d.max_iter) {
      limit = true;
      break;
    }
    const int nxt = cur ^ 1;
    const float al = sc_alpha, be = sc_keep ? 0.0f : sc_beta * sc_pscale;
    const bool keep = sc_keep != 0;
    const float* __restrict__ Rc = f.R[cur];
    const float* __restrict__ Wc = f.W[cur];
    const float* __restrict__ Sc = f.S[cur];
    float* __restrict__ Rn = f.R[nxt];
    float* __restrict__ Sn = f.S[nxt];
    // 1. own cells (warps take rows, lanes columns); RES: in shared memory, the frame
    // published for the neighbours' bands
    if constexpr (RES) {
      for (int j = j0 + warp; j < j1; j += kW)
        for (int i = i0 + lane; i < i1; i += 32) {
          const int q = ridx(i, j), l = lidx(i, j);
          const float rk = sr[q], uk = ubuf[q];
          const float sold = ss[l], pold = sp[l];
          const float sk_ = keep ? sold : sw[l] + be * sold;
          const float pk = keep ? pold : uk + be * pold;
          const float rn = rk - al * sk_;
          sp[l] = pk;
          ss[l] = sk_;
          se[l] += al * pk;
          sr[q] = rn;
          if (frame(i, j)) {
            const size_t k = g.idx(i, j);
            Sn[k] = sk_;
            Rn[k] = rn;
          }
        }
    } else
    // (global) kB of a lane's cells of a row at a time with all their loads issued first (one
    // L2 round trip per group instead of one per cell)
    for (int j = j0 + warp; j < j1; j += kW)
    for (int ib = i0 + lane; ib < i1; ib += 32 * kB) {
      float rk[kB], sold[kB], pold[kB], wk[kB], ek[kB], uk[kB];
      int kk[kB], rq[kB];
#pragma unroll
      for (int m = 0; m < kB; ++m) {
        const int i = ib + 32 * m;
        kk[m] = -1;
        if (i < i1) {
          const int k = (int)g.idx(i, j);
          kk[m] = k;
          rq[m] = ridx(i, j);
          rk[m] = Rc[k]; sold[m] = Sc[k]; pold[m] = Pv[k]; wk[m] = Wc[k]; ek[m] = Ev[k];
          uk[m] = cheb > 1 ? Uv[k] : rk[m];
        }
      }
#pragma unroll
      for (int m = 0; m < kB; ++m) {
        if (kk[m] < 0) continue;
        const int k = kk[m];
        const float sk_ = keep ? sold[m] : wk[m] + be * sold[m];
        const float pk = keep ? pold[m] : uk[m] + be * pold[m];
        const float rn = rk[m] - al * sk_;
        Pv[k] = pk;
        Sn[k] = sk_;
        Ev[k] = ek[m] + al * pk;
        Rn[k] = rn;
        sr[rq[m]] = rn;
      }
    }
    // band cells: r_{i+1} from the neighbours' vectors of this parity, published before the
    // last grid barrier.  (Loading them at the top of the iteration, to overlap the own-cell
    // update, gave wrong results with resident tiles for a reason not found; not used.)
    for (int t = threadIdx.x; t < nband; t += kNT) {
      int bi, bj;
      band_cell(t, bi, bj);
      const size_t k = g.idx(bi, bj);
      const float rk = __ldcg(&Rc[k]), wk = __ldcg(&Wc[k]), sold = __ldcg(&Sc[k]);
      sr[ridx(bi, bj)] = rk - al * (keep ? sold : wk + be * sold);
    }
    __syncthreads();
    // 2-3. preconditioner, w_{i+1} = K~ u_{i+1} and the sums
    float v[3] = {0.0f, 0.0f, 0.0f};
    precond_apply(f.W[nxt], v);
    const float* rows = reduce_arrive(v, 3);
    if (!grid_wait(d.bar, target)) { ok = false; break; }
    float t[3];
    grid_sum_f32_rows<3>(rows, nb, t, fsum);
    scalars(t, false);
    cur = nxt;
    if (sc_replace) {
      fold(true);
      if (threadIdx.x == 0) {
        sc_nrep += 1;
        if (sc_it - sc_rep_it < 3) sc_restart = 1;  // replacements back to back: no progress
        sc_rep_it = sc_it;
      }
      if (!grid_sync(d.bar, target)) { ok = false; break; }
      if (!residual64(false)) { ok = false; break; }
      if (sc_stop != 0) break;
      if (!fresh_apply(f.R[cur], f.W[cur])) { ok = false; break; }
      if (sc_keep && !phase_p(f.R[cur], f.W[cur], f.S[cur])) { ok = false; break; }
    }
  }
  if (ok && limit) {
    fold(false);
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

__global__ void __launch_bounds__(kNT, 1) k_pcg_poisson_m1(const __grid_constant__ Mixed1Solve f) {
  mixed1_body<false>(f);
}

__global__ void __launch_bounds__(kNT, 1) k_pcg_poisson_m2(const __grid_constant__ Mixed1Solve f) {
  mixed1_body<true>(f);
}

int mixed1_per_sm(size_t smem, int resident) {
  int dev = 0, per = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const void* kern = resident ? (const void*)k_pcg_poisson_m2 : (const void*)k_pcg_poisson_m1;
  if (smem > (size_t)optin ||
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kNT, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per;
}

}  // namespace

// r, the two Chebyshev iterates (cheb > 1) and the row kinds of a tile and its band; resident:
// then the tile's p, s, e and w
size_t mixed1_smem(int TX, int TY, int cheb, int resident) {
  const int h = cheb > 1 ? cheb : 1;
  const size_t rn = (size_t)(TX + 2 * h) * (size_t)(TY + 2 * h);
  const size_t base = (cheb > 1 ? 3 : 1) * sizeof(float) * rn;
  if (!resident) return base + rn;
  return base + ((rn + 15) / 16) * 16 + 4 * sizeof(float) * (size_t)TX * (size_t)TY;
}

bool mixed1_plan_fits(int TX, int TY, int ntiles, int cheb, int resident) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int per = mixed1_per_sm(mixed1_smem(TX, TY, cheb, resident), resident);
  return per >= 1 && ntiles >= 1 && ntiles <= sms * std::min(per, 2);
}

std::vector<TilePlan> mixed1_plan_candidates(int nx, int ny, int cheb) {
  std::vector<TilePlan> out;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  for (int resident : {1, 0})
    for (int blocks : {2 * sms, sms, sms / 2}) {
      TilePlan p{};
      fused_tiles(nx, ny, blocks, &p.TX, &p.TY, &p.nbx, &p.ntiles);
      if (p.ntiles < 1) continue;
      p.resident = resident;
      if (!mixed1_plan_fits(p.TX, p.TY, p.ntiles, cheb, resident)) continue;
      bool seen = false;
      for (const TilePlan& q : out) seen = seen || (q.TX == p.TX && q.TY == p.TY && q.resident == resident);
      if (!seen) out.push_back(p);
    }
  return out;
}

cudaError_t run_poisson_mixed1(Mixed1Solve f, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (f.TX == 0) fused_tiles(f.m.d.g.nx, f.m.d.g.ny, sms, &f.TX, &f.TY, &f.nbx, &f.ntiles);
  const int cheb = f.m.cheb > 1 ? f.m.cheb : 1;
  const size_t smem = mixed1_smem(f.TX, f.TY, cheb, f.resident);
  const int per = mixed1_per_sm(smem, f.resident);
  if (f.ntiles < 1 || per < 1 || f.ntiles > sms * std::min(per, 2)) return cudaErrorInvalidConfiguration;
  cudaMemsetAsync(f.m.d.bar.count, 0, sizeof(unsigned int) * kBarWords, st);
  void* params[] = {&f};
  const void* kern = f.resident ? (const void*)k_pcg_poisson_m2 : (const void*)k_pcg_poisson_m1;
  return cudaLaunchCooperativeKernel(kern, f.ntiles, kNT, params, smem, st);
}

}  // namespace ccm
