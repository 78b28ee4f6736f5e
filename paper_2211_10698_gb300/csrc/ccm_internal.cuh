// Internal definitions of libccm: device layout of a case, the bounded grid barrier, the
// deterministic block/grid reductions and the stencil device functions shared by the
// operator, step and PCG kernels.
//
// Layout: every array of a case is (ny + 3) rows of `pitch` elements (pitch >= nx + 3,
// rounded up to 32 elements); index (i, j), i in [-1, nx+1], j in [-1, ny+1], lives at
// (j + 1) * pitch + (i + 1).  Index (i, j) names the p-cell (i, j), the u-face at
// x0 + i*hx, the v-face at y0 + j*hy or the node (x0 + i*hx, y0 + j*hy).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ccm.h"

namespace ccm {

enum Role : int8_t { R_GHOST = 0, R_DIRICHLET = 1, R_INACTIVE = 2, R_UNKNOWN = 3 };

// Capacity slots: grid g in {0 p, 1 u, 2 v} times {V, X, Y, Ax, Ay, Wx, Wy, Bx, By}.
enum { CK_V = 0, CK_X, CK_Y, CK_AX, CK_AY, CK_WX, CK_WY, CK_BX, CK_BY };
__host__ __device__ inline int cap_slot(int g, int k) { return 9 * g + k; }

struct Geom {
  int nx, ny, pitch;
  double x0, y0, hx, hy;  // uniform spacing (a stretched mesh: its smallest spacing)
  // stretched mesh: device arrays of the face abscissas x_f, f in [-3, nx+3] (xf[f] valid for
  // those f; beyond the box the spacing mirrors the spacing inside it), or nullptr (uniform)
  const double* xf;
  const double* yf;
  int px = 0, py = 0;  // periodic in x (W with E) / in y (S with N)
  __host__ __device__ size_t idx(int i, int j) const { return (size_t)(j + 1) * pitch + (size_t)(i + 1); }
  // A cell index beyond a periodic side wrapped to its image inside the box (unchanged
  // otherwise); for the u-grid along x (or the v-grid along y) face n is face 0 as well.
  __host__ __device__ int wrap_i(int i) const { return px ? (i < 0 ? i + nx : (i >= nx ? i - nx : i)) : i; }
  __host__ __device__ int wrap_j(int j) const { return py ? (j < 0 ? j + ny : (j >= ny ? j - ny : j)) : j; }
  __host__ __device__ size_t count() const { return (size_t)(ny + 3) * pitch; }
};

// Grid lines of grid `grid` (0 p, 1 u, 2 v; Sec. 3.4), from one expression for every use so
// that neighbouring cells agree bitwise: on a uniform mesh x0 + off + i hx with the u-grid
// shifted by -hx/2; on a stretched one the face x_i, or for the u-grid the centre of pressure
// cell i-1, (x_{i-1} + x_i) / 2 (and likewise in y).
__host__ __device__ inline double grid_line(double o, double off, int i, double h, const double* f, bool stag) {
#ifdef __CUDA_ARCH__
  if (!f) return __dadd_rn(__dadd_rn(o, off), __dmul_rn((double)i, h));
  return stag ? __dmul_rn(0.5, __dadd_rn(f[i - 1], f[i])) : f[i];
#else
  if (!f) return (o + off) + (double)i * h;
  return stag ? 0.5 * (f[i - 1] + f[i]) : f[i];
#endif
}
__host__ __device__ inline double line_x(const Geom& g, int grid, int i) {
  return grid_line(g.x0, grid == 1 ? -0.5 * g.hx : 0.0, i, g.hx, g.xf, grid == 1);
}
__host__ __device__ inline double line_y(const Geom& g, int grid, int j) {
  return grid_line(g.y0, grid == 2 ? -0.5 * g.hy : 0.0, j, g.hy, g.yf, grid == 2);
}
// Area of pressure cell (i, j)
__host__ __device__ inline double cell_area(const Geom& g, int i, int j) {
  if (!g.xf && !g.yf) return g.hx * g.hy;
  return (line_x(g, 0, i + 1) - line_x(g, 0, i)) * (line_y(g, 0, j + 1) - line_y(g, 0, j));
}

struct Bc {
  int type[4];        // W E S N
  double un[4], ut[4];
  __host__ __device__ bool per_x() const { return type[0] == CCM_BC_PERIODIC; }
  __host__ __device__ bool per_y() const { return type[2] == CCM_BC_PERIODIC; }
};

// Periodic images of a position (i, j) of a cell, u- or v-face array: the copies a write must
// also make so that stencils reading across a periodic side find the value (i = 0 is also
// i = nx, i = nx-1 also i = -1; likewise j; corners in a doubly periodic box).
template <class T>
__device__ __forceinline__ void put_images(T* a, int i, int j, size_t k, T val, int nx, int ny, size_t P, bool px,
                                           bool py) {
  long long dx = 0, dy = 0;
  if (px) dx = i == 0 ? nx : (i == nx - 1 ? -nx : 0);
  if (py) dy = j == 0 ? (long long)ny * (long long)P : (j == ny - 1 ? -(long long)ny * (long long)P : 0);
  if (dx) a[(long long)k + dx] = val;
  if (dy) a[(long long)k + dy] = val;
  if (dx && dy) a[(long long)k + dx + dy] = val;
}

// Coefficients derived from the capacities, all in the padded layout.
struct Coefs {
  const int8_t* role_u;
  const int8_t* role_v;
  const int8_t* act;        // active pressure cell
  const double* ax;         // p-grid A^x at u-faces (cont, pres, conv)
  const double* ay;         // p-grid A^y at v-faces
  const double* bxx;        // B^xx at u-faces (u-grid Bx)
  const double* bxy;        // B^xy at u-faces (u-grid By)
  const double* byx;        // B^yx at v-faces (v-grid Bx)
  const double* byy;        // B^yy at v-faces (v-grid By)
  const double* wxx;        // 1/W^xx at p-cells
  const double* wyy;        // 1/W^yy at p-cells
  const double* wxa;        // node weight of the u part of S_xy
  const double* wxb;        // node weight of the v part of S_xy
  const double* cu;         // Poisson face coefficient A^2/V at u unknowns
  const double* cv;
  const double* invdk;      // 1 / diag(K) at active cells
  const double* gfu;        // (dt/rho) A / V at u unknowns (projection)
  const double* gfv;
  const double* pfac;       // (dt mu / 2 rho) / V_p at active cells
  const double* massu;      // (rho/dt) V at u unknowns
  const double* massv;
  const double* invdhu;     // 1 / diag(H) at u unknowns and inactive faces
  const double* invdhv;
  const double* liftu;      // visc(S(0, box data)) at u unknowns
  const double* liftv;
  const double* accx;       // body acceleration g at u-faces (Eq. pm_prediction's rho V g); null: g = 0
  const double* accy;       // ... at v-faces
  // the body's steady Dirichlet velocity D and its constant terms (dterms.cu); null: D = 0
  const double* dx;         // D_x per u-cell
  const double* dy;         // D_y per v-cell
  const double* hd;         // cont(0, D) at cells (zero outside the box)
  const double* sxxd;       // strain(0, D): S_xx at cells, S_yy at cells, S_xy at nodes
  const double* syyd;
  const double* sxyd;
  const double* viscdu;     // visc(S(0, D)) at u unknowns
  const double* viscdv;     // ... at v unknowns
  const float* cu32;
  const float* cv32;
  const float* invdk32;
};

struct Phys {
  double rho, mu, dt;
  // a body velocity D(t) = D0 f(t): f at the time level of the velocity a stage reads (dn) and
  // of the next level (dn1); 1 for a steady D (D = D0)
  double dn = 1.0, dn1 = 1.0;
};

// ---------------------------------------------------------------------------------------
// Bounded device-wide barrier for cooperative (co-resident) launches.  Thread 0 of each
// block arrives on a monotonically increasing counter (one release add) and polls it with
// acquire loads until all blocks of this round have arrived, giving up after `budget` clock
// cycles; on give-up it raises *err and the caller leaves the kernel (the other blocks give
// up at their own next barrier).
// ---------------------------------------------------------------------------------------
// Device-wide barrier of a cooperative launch: one arrival counter.
constexpr int kBarWords = 1;  // unsigned ints behind Barrier::count
struct Barrier {
  unsigned int* count;  // zeroed before the launch
  int* err;
  long long budget;     // clock64 cycles a block waits before it gives up
  int absent = -1;      // failure-detection tests only: this block never arrives, so every other
                        // block's wait runs out; -1 in every normal launch
};

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ bool grid_sync(const Barrier& b, unsigned int& target) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    target += gridDim.x;
    // release: the block's writes before the block barrier above become visible with the
    // arrival; the acquire loads below order what follows after every block's arrival (the
    // block barrier below carries both to the other threads of the block)
    if ((int)blockIdx.x != b.absent)
      asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(b.count), "r"(1u) : "memory");
    const long long t0 = clock64();
    while (ld_acquire_u32(b.count) < target) {
      if (clock64() - t0 > b.budget) {
        atomicExch(b.err, 1);
        ok = 0;
        break;
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// The same barrier among the n blocks that share the counter `count` (one case of a batched
// launch, whose blocks wait for each other only); err, budget and the absent block as above.
__device__ __forceinline__ bool range_sync(const Barrier& b, unsigned int* count, unsigned int n,
                                           unsigned int& target) {
  __shared__ int s_okr;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    target += n;
    if ((int)blockIdx.x != b.absent)
      asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(count), "r"(1u) : "memory");
    const long long t0 = clock64();
    while (ld_acquire_u32(count) < target) {
      if (clock64() - t0 > b.budget) {
        atomicExch(b.err, 1);
        ok = 0;
        break;
      }
    }
    s_okr = ok;
  }
  __syncthreads();
  return s_okr != 0;
}

// The same barrier in two halves, so that a block can do work that no other block reads
// between its arrival and its wait: grid_arrive (all threads), then grid_wait (all threads).
__device__ __forceinline__ void grid_arrive(const Barrier& b, unsigned int& target) {
  __syncthreads();
  if (threadIdx.x == 0) {
    target += gridDim.x;
    if ((int)blockIdx.x != b.absent)
      asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(b.count), "r"(1u) : "memory");
  }
}
__device__ __forceinline__ bool grid_wait(const Barrier& b, const unsigned int& target) {
  __shared__ int s_ok2;
  if (threadIdx.x == 0) {
    int ok = 1;
    const long long t0 = clock64();
    while (ld_acquire_u32(b.count) < target) {
      if (clock64() - t0 > b.budget) {
        atomicExch(b.err, 1);
        ok = 0;
        break;
      }
    }
    s_ok2 = ok;
  }
  __syncthreads();
  return s_ok2 != 0;
}

// Deterministic block sum of NV values (fixed shuffle tree, fixed warp order); the result
// is valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* smem /* >= 32*NV */) {
#pragma unroll
  for (int k = 0; k < NV; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) smem[k * 32 + w] = v[k];
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = lane < nw ? smem[k * 32 + lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      v[k] = s;
    }
  }
}

// Sum of the per-block partials (layout partials[k * nblocks + b]) in a fixed order; every
// block computes the identical value.  Warp k reduces quantity k: each lane first issues all
// of its loads (one L2 round trip for up to 32 * kGridSumPerLane blocks), then adds them in
// a fixed pairwise tree (four dependent adds instead of ten: the sum sits on every
// iteration's serial path), then the warp's shuffle tree finishes.  Result broadcast through
// smem.
constexpr int kGridSumPerLane = 10;
template <int NV>
__device__ __forceinline__ void grid_sum(const double* partials, int nblocks, double (&out)[NV], double* smem) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (w < NV) {
    const double* src = partials + (size_t)w * nblocks;
    double buf[kGridSumPerLane];
#pragma unroll
    for (int m = 0; m < kGridSumPerLane; ++m) {
      const int b = lane + 32 * m;
      buf[m] = b < nblocks ? __ldcg(&src[b]) : 0.0;
    }
#pragma unroll
    for (int h = 1; h < kGridSumPerLane; h <<= 1)
#pragma unroll
      for (int m = 0; m + h < kGridSumPerLane; m += 2 * h) buf[m] += buf[m + h];
    double s = buf[0];
    for (int b = lane + 32 * kGridSumPerLane; b < nblocks; b += 32) s += __ldcg(&src[b]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) smem[w] = s;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) out[k] = smem[k];
}

// ---------------------------------------------------------------------------------------
// Stencils.  Arrays are read with explicit (i, j) indices in the padded layout.
// ---------------------------------------------------------------------------------------

// Homogeneous view of a velocity-like vector: value on unknowns, zero on Dirichlet and
// inactive faces, and on ghost positions the zero-gradient copy or the reflection of the
// adjacent position according to the side's boundary type.
struct HomView {
  const double* u;
  const double* v;
  const int8_t* ru;
  const int8_t* rv;
  Geom g;
  Bc bc;
  __device__ __forceinline__ double at_u(int i, int j) const {
    double s = 1.0;
    if (g.px) i = g.wrap_i(i);
    else if (i < 0) i = 0;
    else if (i > g.nx) i = g.nx;
    if (g.py) j = g.wrap_j(j);
    else if (j < 0) { j = 0; if (bc.type[CCM_SIDE_S] == CCM_BC_DIRICHLET) s = -1.0; }
    else if (j >= g.ny) { j = g.ny - 1; if (bc.type[CCM_SIDE_N] == CCM_BC_DIRICHLET) s = -1.0; }
    size_t k = g.idx(i, j);
    return ru[k] == R_UNKNOWN ? s * u[k] : 0.0;
  }
  __device__ __forceinline__ double at_v(int i, int j) const {
    double s = 1.0;
    if (g.py) j = g.wrap_j(j);
    else if (j < 0) j = 0;
    else if (j > g.ny) j = g.ny;
    if (g.px) i = g.wrap_i(i);
    else if (i < 0) { i = 0; if (bc.type[CCM_SIDE_W] == CCM_BC_DIRICHLET) s = -1.0; }
    else if (i >= g.nx) { i = g.nx - 1; if (bc.type[CCM_SIDE_E] == CCM_BC_DIRICHLET) s = -1.0; }
    size_t k = g.idx(i, j);
    return rv[k] == R_UNKNOWN ? s * v[k] : 0.0;
  }
};

// Full view: the arrays already hold Dirichlet faces and ghosts (filled by fill_bc).
struct FullView {
  const double* u;
  const double* v;
  Geom g;
  __device__ __forceinline__ double at_u(int i, int j) const { return u[g.idx(i, j)]; }
  __device__ __forceinline__ double at_v(int i, int j) const { return v[g.idx(i, j)]; }
};

// Strain components (Eqs. diag, offdiag with D = 0).
template <class View>
__device__ __forceinline__ double strain_xx(const Coefs& c, const Geom& g, const View& w, int i, int j) {
  // p-cell (i, j): u-faces i and i+1
  return (c.bxx[g.idx(i + 1, j)] * w.at_u(i + 1, j) - c.bxx[g.idx(i, j)] * w.at_u(i, j)) * c.wxx[g.idx(i, j)];
}
template <class View>
__device__ __forceinline__ double strain_yy(const Coefs& c, const Geom& g, const View& w, int i, int j) {
  return (c.byy[g.idx(i, j + 1)] * w.at_v(i, j + 1) - c.byy[g.idx(i, j)] * w.at_v(i, j)) * c.wyy[g.idx(i, j)];
}
template <class View>
__device__ __forceinline__ double strain_xy(const Coefs& c, const Geom& g, const View& w, int i, int j) {
  // node (i, j): u-faces (i, j-1), (i, j); v-faces (i-1, j), (i, j)
  const size_t k = g.idx(i, j);
  double gu = c.bxy[k] * w.at_u(i, j) - c.bxy[g.idx(i, j - 1)] * w.at_u(i, j - 1);
  double gv = c.byx[k] * w.at_v(i, j) - c.byx[g.idx(i - 1, j)] * w.at_v(i - 1, j);
  return gu * c.wxa[k] + gv * c.wxb[k];
}

// visc_x(S) at u-face (i, j) and visc_y(S) at v-face (i, j) (Sec. 4.3), with the outflow
// rule: the tangential velocity next to an outflow side takes no shear from the nodes on
// that side.
template <class View>
__device__ __forceinline__ double visc_u(const Coefs& c, const Geom& g, const Bc& bc, const View& w, int i, int j) {
  const size_t k = g.idx(i, j);
  double sx = strain_xx(c, g, w, i, j) - strain_xx(c, g, w, i - 1, j);
  double top = (j == g.ny - 1 && bc.type[CCM_SIDE_N] == CCM_BC_OUTFLOW) ? 0.0 : strain_xy(c, g, w, i, j + 1);
  double bot = (j == 0 && bc.type[CCM_SIDE_S] == CCM_BC_OUTFLOW) ? 0.0 : strain_xy(c, g, w, i, j);
  return c.bxx[k] * sx + c.bxy[k] * (top - bot);
}
template <class View>
__device__ __forceinline__ double visc_v(const Coefs& c, const Geom& g, const Bc& bc, const View& w, int i, int j) {
  const size_t k = g.idx(i, j);
  double sy = strain_yy(c, g, w, i, j) - strain_yy(c, g, w, i, j - 1);
  double rgt = (i == g.nx - 1 && bc.type[CCM_SIDE_E] == CCM_BC_OUTFLOW) ? 0.0 : strain_xy(c, g, w, i + 1, j);
  double lft = (i == 0 && bc.type[CCM_SIDE_W] == CCM_BC_OUTFLOW) ? 0.0 : strain_xy(c, g, w, i, j);
  return c.byy[k] * sy + c.byx[k] * (rgt - lft);
}

// conv_x(U, U, 0, 0) at u-face (i, j) and conv_y at v-face (i, j) (Eq. convective, D = 0):
// divergence of the face-interpolated mass fluxes times the interpolated velocity.
__device__ __forceinline__ double conv_u(const Coefs& c, const Geom& g, const FullView& w, int i, int j) {
  const double* A = c.ax;
  const double* B = c.ay;
  double fe = 0.5 * (A[g.idx(i + 1, j)] * w.at_u(i + 1, j) + A[g.idx(i, j)] * w.at_u(i, j));
  double fw = 0.5 * (A[g.idx(i, j)] * w.at_u(i, j) + A[g.idx(i - 1, j)] * w.at_u(i - 1, j));
  double ue = 0.5 * (w.at_u(i + 1, j) + w.at_u(i, j));
  double uw = 0.5 * (w.at_u(i, j) + w.at_u(i - 1, j));
  double fn = 0.5 * (B[g.idx(i, j + 1)] * w.at_v(i, j + 1) + B[g.idx(i - 1, j + 1)] * w.at_v(i - 1, j + 1));
  double fs = 0.5 * (B[g.idx(i, j)] * w.at_v(i, j) + B[g.idx(i - 1, j)] * w.at_v(i - 1, j));
  double un = 0.5 * (w.at_u(i, j + 1) + w.at_u(i, j));
  double us = 0.5 * (w.at_u(i, j) + w.at_u(i, j - 1));
  return (fe * ue - fw * uw) + (fn * un - fs * us);
}
__device__ __forceinline__ double conv_v(const Coefs& c, const Geom& g, const FullView& w, int i, int j) {
  const double* A = c.ax;
  const double* B = c.ay;
  double fn = 0.5 * (B[g.idx(i, j + 1)] * w.at_v(i, j + 1) + B[g.idx(i, j)] * w.at_v(i, j));
  double fs = 0.5 * (B[g.idx(i, j)] * w.at_v(i, j) + B[g.idx(i, j - 1)] * w.at_v(i, j - 1));
  double vn = 0.5 * (w.at_v(i, j + 1) + w.at_v(i, j));
  double vs = 0.5 * (w.at_v(i, j) + w.at_v(i, j - 1));
  double fe = 0.5 * (A[g.idx(i + 1, j)] * w.at_u(i + 1, j) + A[g.idx(i + 1, j - 1)] * w.at_u(i + 1, j - 1));
  double fw = 0.5 * (A[g.idx(i, j)] * w.at_u(i, j) + A[g.idx(i, j - 1)] * w.at_u(i, j - 1));
  double ve = 0.5 * (w.at_v(i + 1, j) + w.at_v(i, j));
  double vw = 0.5 * (w.at_v(i, j) + w.at_v(i - 1, j));
  return (fn * vn - fs * vs) + (fe * ve - fw * vw);
}

// cont(U, 0) at p-cell (i, j) (Eq. divergence, D = 0).
template <class T>
__device__ __forceinline__ double cont_cell(const Coefs& c, const Geom& g, const T* u, const T* v, int i, int j) {
  return c.ax[g.idx(i + 1, j)] * (double)u[g.idx(i + 1, j)] - c.ax[g.idx(i, j)] * (double)u[g.idx(i, j)] +
         c.ay[g.idx(i, j + 1)] * (double)v[g.idx(i, j + 1)] - c.ay[g.idx(i, j)] * (double)v[g.idx(i, j)];
}

// K x at cell (i, j): sum over faces of c_f (x_c - x_nbr); identity on inactive cells.
// The ghost ring of x holds zeros (Dirichlet pressure on outflow sides).
template <class T, class C>
__device__ __forceinline__ T poisson_row(const C* cu, const C* cv, const int8_t* act, const Geom& g, const T* x,
                                         size_t k) {
  T xc = x[k];
  if (!act[k]) return xc;
  T cw = (T)cu[k], ce = (T)cu[k + 1], cs = (T)cv[k], cn = (T)cv[k + g.pitch];
  return cw * (xc - x[k - 1]) + ce * (xc - x[k + 1]) + cs * (xc - x[k - g.pitch]) + cn * (xc - x[k + g.pitch]);
}

}  // namespace ccm
