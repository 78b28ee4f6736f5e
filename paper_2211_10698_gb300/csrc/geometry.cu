// Capacities of the conservative cut-cell method (Sec. 3 of arXiv 2211.10698) on the GPU,
// in FP64, and the operator coefficients derived from them.
//
// Each cell of the p-, u- and v-grids (Sec. 3.4: u-grid shifted by -hx/2, v-grid by -hy/2)
// is reconstructed by marching squares with exact crossings of the boundary on its four
// edges (Sec. 3.1 allows a marching-squares reconstruction from the level set).  The fluid
// region inside a cell is then one or two convex polygons, from which
//   V, X, Y        first-kind volume and centroid          (Eqs. volumefirstkind, centroid)
//   Ax, Ay         wet length of the left / bottom edge    (Eqs. surfacefirstkindx/y)
//   Bx, By         wet length of the lines x = X, y = Y    (Eqs. surfacesecondkindx/y)
//   Wx, Wy         fluid area between the centroid of the left / lower neighbour and the
//                  cell's own centroid                     (Eqs. volumesecondkindx/y)
// follow in closed form.  One thread handles one cell of one grid and rebuilds the two
// neighbours it needs for W, so the kernel has no inter-thread dependence.
#include <math.h>

#include "ccm_internal.cuh"

namespace ccm {

struct Body {
  int kind;
  double cx, cy, r, r2;
  double ca, sa, lex, ley, ichord, t5, a4;
  double pnx, pny, poff;
};

__device__ __forceinline__ bool in_fluid(const Body& b, double x, double y) {
  if (b.kind == CCM_GEOM_CIRCLE) {
    double dx = x - b.cx, dy = y - b.cy;
    return dx * dx + dy * dy > b.r2;
  }
  if (b.kind == CCM_GEOM_HALFPLANE) return b.pnx * x + b.pny * y > b.poff;
  if (b.kind == CCM_GEOM_NACA) {
    double px = x - b.lex, py = y - b.ley;
    double xi = (px * b.ca - py * b.sa) * b.ichord;
    double eta = (px * b.sa + py * b.ca) * b.ichord;
    if (xi < 0.0 || xi > 1.0) return true;
    // NACA 4-digit symmetric half thickness, Horner form of the quartic tail
    double yt = b.t5 * (0.2969 * sqrt(xi) + xi * (-0.1260 + xi * (-0.3516 + xi * (0.2843 + xi * b.a4))));
    return fabs(eta) > yt;
  }
  return true;
}

// Position of the boundary on an axis-aligned edge whose end points differ in fluid status.
// horizontal: the edge y = c, x in [a, b]; otherwise x = c, y in [a, b].  Returns the
// distance from a.
__device__ double edge_crossing(const Body& b, bool horizontal, double c, double a, double e) {
  if (b.kind == CCM_GEOM_CIRCLE) {
    double cc = horizontal ? b.cx : b.cy;        // centre along the edge
    double co = horizontal ? c - b.cy : c - b.cx; // offset across the edge
    double d = b.r2 - co * co;
    double s = d > 0.0 ? sqrt(d) : 0.0;
    double s1 = cc - s, s2 = cc + s;
    double m = 0.5 * (a + e);
    double s0 = fabs(s1 - m) <= fabs(s2 - m) ? s1 : s2;
    s0 = fmin(fmax(s0, a), e);
    return s0 - a;
  }
  if (b.kind == CCM_GEOM_HALFPLANE) {
    double s0 = horizontal ? (b.poff - b.pny * c) / b.pnx : (b.poff - b.pnx * c) / b.pny;
    s0 = fmin(fmax(s0, a), e);
    return s0 - a;
  }
  // bisection on the fluid indicator (NACA)
  bool fa = horizontal ? in_fluid(b, a, c) : in_fluid(b, c, a);
  double lo = a, hi = e;
  for (int it = 0; it < 64; ++it) {
    double mid = 0.5 * (lo + hi);
    if (!(mid > lo && mid < hi)) break;
    bool fm = horizontal ? in_fluid(b, mid, c) : in_fluid(b, c, mid);
    if (fm == fa) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi) - a;
}

// Up to two convex pieces, in coordinates local to the cell's lower-left corner,
// counter-clockwise.  A piece has at most six vertices; clipping it by a line adds one.
struct Piece { int n; double x[8], y[8]; };
struct Cell {
  double xl, yb, w, h;
  int np;
  Piece pc[2];
  double aleft, abot;
  double V, X, Y;  // absolute centroid
};

__device__ __forceinline__ void push(Piece& p, double x, double y) {
  if (p.n < 8) { p.x[p.n] = x; p.y[p.n] = y; ++p.n; }
}

__device__ void area_moments(const Piece& p, double& a, double& mx, double& my) {
  a = 0.0; mx = 0.0; my = 0.0;
  for (int k = 0; k < p.n; ++k) {
    int q = (k + 1 == p.n) ? 0 : k + 1;
    double cr = p.x[k] * p.y[q] - p.x[q] * p.y[k];
    a += cr;
    mx += (p.x[k] + p.x[q]) * cr;
    my += (p.y[k] + p.y[q]) * cr;
  }
  a *= 0.5;
  mx *= (1.0 / 6.0);
  my *= (1.0 / 6.0);
}

__device__ void build(const Body& b, const Geom& g, int grid, int i, int j, Cell& c) {
  const double xl = line_x(g, grid, i), xr = line_x(g, grid, i + 1);
  const double yb = line_y(g, grid, j), yt = line_y(g, grid, j + 1);
  c.xl = xl; c.yb = yb; c.w = xr - xl; c.h = yt - yb;
  const double w = c.w, h = c.h;
  const bool f0 = in_fluid(b, xl, yb), f1 = in_fluid(b, xr, yb), f2 = in_fluid(b, xr, yt), f3 = in_fluid(b, xl, yt);
  // local crossing positions: bottom, right, top, left
  const double cb = (f0 != f1) ? edge_crossing(b, true, yb, xl, xr) : 0.0;
  const double cr = (f1 != f2) ? edge_crossing(b, false, xr, yb, yt) : 0.0;
  const double ct = (f3 != f2) ? edge_crossing(b, true, yt, xl, xr) : 0.0;
  const double cl = (f0 != f3) ? edge_crossing(b, false, xl, yb, yt) : 0.0;
  c.aleft = f0 ? (f3 ? h : cl) : (f3 ? h - cl : 0.0);
  c.abot = f0 ? (f1 ? w : cb) : (f1 ? w - cb : 0.0);
  c.np = 0;
  const int code = (int)f0 | ((int)f1 << 1) | ((int)f2 << 2) | ((int)f3 << 3);
  if (code != 0) {
    // vertices around the cell: corner k then the crossing on the edge leaving corner k
    const double vx[4] = {0.0, w, w, 0.0}, vy[4] = {0.0, 0.0, h, h};
    const double ex[4] = {cb, w, ct, 0.0}, ey[4] = {0.0, cr, h, cl};
    const bool fl[4] = {f0, f1, f2, f3};
    const bool saddle = (code == 5 || code == 10);
    if (saddle && !in_fluid(b, xl + 0.5 * w, yb + 0.5 * h)) {
      // disconnected: a triangle at each fluid corner
      c.np = 2;
      c.pc[0].n = 0; c.pc[1].n = 0;
      const int k0 = f0 ? 0 : 1;  // first fluid corner
      for (int s = 0; s < 2; ++s) {
        int k = k0 + 2 * s, km = (k + 3) & 3;
        Piece& p = c.pc[s];
        push(p, ex[km], ey[km]);
        push(p, vx[k], vy[k]);
        push(p, ex[k], ey[k]);
      }
    } else {
      c.np = 1;
      Piece& p = c.pc[0];
      p.n = 0;
      for (int k = 0; k < 4; ++k) {
        if (fl[k]) push(p, vx[k], vy[k]);
        if (fl[k] != fl[(k + 1) & 3]) push(p, ex[k], ey[k]);
      }
    }
  }
  double A = 0.0, MX = 0.0, MY = 0.0;
  for (int s = 0; s < c.np; ++s) {
    double a, mx, my;
    area_moments(c.pc[s], a, mx, my);
    A += a; MX += mx; MY += my;
  }
  c.V = A;
  if (A > 0.0) { c.X = xl + MX / A; c.Y = yb + MY / A; }
  else { c.X = xl + 0.5 * w; c.Y = yb + 0.5 * h; }
}

// Area of the part of a convex piece on one side of an axis-aligned line.
__device__ double side_area(const Piece& p, bool xaxis, double s, bool above) {
  Piece q;
  q.n = 0;
  for (int k = 0; k < p.n; ++k) {
    int n = (k + 1 == p.n) ? 0 : k + 1;
    double a = xaxis ? p.x[k] : p.y[k], e = xaxis ? p.x[n] : p.y[n];
    bool ia = above ? a >= s : a <= s, ie = above ? e >= s : e <= s;
    if (ia) push(q, p.x[k], p.y[k]);
    if (ia != ie) {
      double t = (s - a) / (e - a);
      if (xaxis) push(q, s, p.y[k] + t * (p.y[n] - p.y[k]));
      else push(q, p.x[k] + t * (p.x[n] - p.x[k]), s);
    }
  }
  if (q.n < 3) return 0.0;
  double a, mx, my;
  area_moments(q, a, mx, my);
  return a;
}

// Length of the intersection of a convex piece with an axis-aligned line.
__device__ double chord(const Piece& p, bool xaxis, double s) {
  double lo = INFINITY, hi = -INFINITY;
  for (int k = 0; k < p.n; ++k) {
    int n = (k + 1 == p.n) ? 0 : k + 1;
    double a = xaxis ? p.x[k] : p.y[k], e = xaxis ? p.x[n] : p.y[n];
    double qa = xaxis ? p.y[k] : p.x[k], qe = xaxis ? p.y[n] : p.x[n];
    if ((a - s) * (e - s) > 0.0) continue;
    if (a == e) {
      lo = fmin(lo, fmin(qa, qe));
      hi = fmax(hi, fmax(qa, qe));
    } else {
      double q = qa + (s - a) / (e - a) * (qe - qa);
      lo = fmin(lo, q);
      hi = fmax(hi, q);
    }
  }
  return hi >= lo ? hi - lo : 0.0;
}

__global__ void k_capacities(Body b, Geom g, int grid, double* const* caps) {
  const int i = (int)(blockIdx.x * blockDim.x + threadIdx.x) - 1;
  const int j = (int)blockIdx.y - 1;
  if (i > g.nx + 1 || j > g.ny + 1) return;
  Cell c, cw, cs;
  build(b, g, grid, i, j, c);
  build(b, g, grid, i - 1, j, cw);
  build(b, g, grid, i, j - 1, cs);
  double bx = 0.0, by = 0.0, wx = 0.0, wy = 0.0;
  for (int s = 0; s < c.np; ++s) {
    bx += chord(c.pc[s], true, c.X - c.xl);
    by += chord(c.pc[s], false, c.Y - c.yb);
    wx += side_area(c.pc[s], true, c.X - c.xl, false);
    wy += side_area(c.pc[s], false, c.Y - c.yb, false);
  }
  for (int s = 0; s < cw.np; ++s) wx += side_area(cw.pc[s], true, cw.X - cw.xl, true);
  for (int s = 0; s < cs.np; ++s) wy += side_area(cs.pc[s], false, cs.Y - cs.yb, true);
  const size_t k = g.idx(i, j);
  caps[cap_slot(grid, CK_V)][k] = c.V;
  caps[cap_slot(grid, CK_X)][k] = c.X;
  caps[cap_slot(grid, CK_Y)][k] = c.Y;
  caps[cap_slot(grid, CK_AX)][k] = c.aleft;
  caps[cap_slot(grid, CK_AY)][k] = c.abot;
  caps[cap_slot(grid, CK_WX)][k] = wx;
  caps[cap_slot(grid, CK_WY)][k] = wy;
  caps[cap_slot(grid, CK_BX)][k] = bx;
  caps[cap_slot(grid, CK_BY)][k] = by;
}

// Host launcher: fills the 27 capacity arrays.
cudaError_t launch_capacities(const ccm_geometry& geo, const Geom& g, double* const* caps_dev, cudaStream_t st) {
  Body b{};
  b.kind = geo.kind;
  b.cx = geo.cx; b.cy = geo.cy; b.r = geo.r; b.r2 = geo.r * geo.r;
  double a = geo.aoa_deg * (M_PI / 180.0);
  b.ca = cos(a); b.sa = sin(a);
  b.lex = geo.le_x; b.ley = geo.le_y;
  b.ichord = geo.chord > 0 ? 1.0 / geo.chord : 1.0;
  b.t5 = 5.0 * geo.naca_tt / 100.0;
  b.a4 = geo.closed_te ? -0.1036 : -0.1015;
  b.pnx = geo.hp_nx; b.pny = geo.hp_ny; b.poff = geo.hp_off;
  dim3 blk(128, 1), grd((g.nx + 3 + 127) / 128, g.ny + 3);
  for (int grid = 0; grid < 3; ++grid) k_capacities<<<grd, blk, 0, st>>>(b, g, grid, caps_dev);
  return cudaGetLastError();
}

}  // namespace ccm
