/*
 * FP64 CPU oracle for the conservative Cartesian cut-cell method on staggered (MAC) grids
 * of Quiros Rodriguez, Fullana, Le Chenadec and Sayadi (arXiv 2211.10698).
 *
 * TEST INFRASTRUCTURE.  This file is the plain, slow statement of what the
 * GPU library must compute.  Only the tests, the package's smoke check and the bench's CPU
 * baseline call it; the library never does.  It shares no code, header or table with the
 * CUDA sources.
 *
 * Layout: every array is padded to (ny+3) x (nx+3), x fastest; index (i, j) with
 * i in [-1, nx+1], j in [-1, ny+1] lives at (j+1)*(nx+3) + (i+1).  (i, j) denotes the
 * pressure cell i,j, the x-face x0+i*hx (u), the y-face y0+j*hy (v) or the node
 * (x0+i*hx, y0+j*hy), depending on the array.
 *
 * Capacities (Sec. 3, Eqs. volumefirstkind..surfacesecondkindy) are stored per grid
 * g in {p, u, v} (Sec. 3.4: u-grid shifted by -hx/2, v-grid by -hy/2), nine arrays per
 * grid in the order V, X, Y, Ax, Ay, Wx, Wy, Bx, By, each indexed by the grid cell's own
 * (i, j).  Ax/Wx belong to the cell's left face, Ay/Wy to its bottom face, so that
 *   p-grid: Ax(i,j) = A^x at u-face (i,j), Ay(i,j) = A^y at v-face (i,j),
 *           Wx(i,j) = W^x at u-face (i,j), Wy(i,j) = W^y at v-face (i,j);
 *   u-grid: Ax(i+1,j) = A^xx and Wx(i+1,j) = W^xx at p-cell (i,j),
 *           Ay(i,j) = A^xy and Wy(i,j) = W^xy at node (i,j), Bx = B^xx, By = B^xy at u-face;
 *   v-grid: Ax(i,j) = A^yx and Wx(i,j) = W^yx at node (i,j),
 *           Ay(i,j+1) = A^yy and Wy(i,j+1) = W^yy at p-cell (i,j), Bx = B^yx, By = B^yy.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Loops over cells or vector elements whose iterations write distinct outputs may run on
 * several threads (OpenMP, when built with it); the results do not depend on the thread count.
 * Sums (dot products, means) are taken in a fixed order: serially within fixed blocks of
 * DOT_BLOCK elements, then over the blocks in order. */
#ifdef _OPENMP
#define PAR_FOR _Pragma("omp parallel for schedule(static)")
#else
#define PAR_FOR
#endif
#define DOT_BLOCK 4096

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct {
  int nx, ny;
  double x0, y0, hx, hy;
  double rho, mu, dt;
  int bc_type[4];          /* W, E, S, N: 0 Dirichlet, 1 outflow, 2 periodic (W with E, S with N) */
  double bc_un[4];         /* Dirichlet normal velocity component (u on W/E, v on S/N) */
  double bc_ut[4];         /* Dirichlet tangential component (v on W/E, u on S/N) */
  int geom_kind;           /* 0 none, 1 circle, 2 NACA 00tt, 3 half plane */
  double cx, cy, r;
  int naca_tt, closed_te;
  double chord, aoa_deg, le_x, le_y;
  double hp_nx, hp_ny, hp_off;
  int literal_offdiag;     /* 1: Eq. offdiag with separate W^xy, W^yx */
  int pressure_update;     /* volume dividing the viscous correction of Eq. pm_update:
                              0 the full cell's area, 1 the cell's fluid volume V_p, 2 none */
  int precond;             /* 0 Jacobi, 1 Chebyshev */
  int cheb_degree;
  double tol_p, tol_h;
  int max_iter_p, max_iter_h;
  /* Rectilinear, possibly stretched mesh (Sec. 3.1): the face abscissas x_0 = x0 < x_1 < ...
   * < x_nx and y_0 < ... < y_ny, or NULL for the uniform spacing hx, hy.  With a stretched
   * mesh hx and hy hold the smallest spacing (used for thresholds only). */
  const double* xf;
  const double* yf;
} orc_case;

typedef struct {
  int iters_h, iters_p;
  double res_h, res_p;
  double max_div, kinetic;
  int conv_h, conv_p;
} orc_stats;

enum { G_P = 0, G_U = 1, G_V = 2 };
enum { K_V = 0, K_X, K_Y, K_AX, K_AY, K_WX, K_WY, K_BX, K_BY };
enum { W_SIDE = 0, E_SIDE = 1, S_SIDE = 2, N_SIDE = 3 };
#define BC_DIR 0
#define BC_OUT 1
#define BC_PER 2
/* periodic in x (W and E) or y (S and N): face nx is face 0 and cell -1 is cell nx-1 */
#define PER_X(c) ((c)->bc_type[W_SIDE] == BC_PER)
#define PER_Y(c) ((c)->bc_type[S_SIDE] == BC_PER)

#define PITCH(c) ((c)->nx + 3)
#define SIZE(c) ((size_t)((c)->nx + 3) * (size_t)((c)->ny + 3))
#define AT(c, a, i, j) ((a)[(size_t)((j) + 1) * PITCH(c) + (size_t)((i) + 1)])
#define CAP(c, caps, g, k) ((caps) + ((size_t)(g) * 9 + (size_t)(k)) * SIZE(c))

size_t orc_size(const orc_case* c) { return SIZE(c); }

/* Threads for the parallel loops (n < 1: all); returns the number in use.  1 without OpenMP. */
int orc_set_threads(int n) {
#ifdef _OPENMP
  if (n >= 1) omp_set_num_threads(n);
  else omp_set_num_threads(omp_get_num_procs());
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

static void zero_fill(double* a, size_t n) {
  PAR_FOR
  for (size_t k = 0; k < n; ++k) a[k] = 0.0;
}

static double* zalloc(size_t n) {
  double* a = malloc(n * sizeof(double));
  zero_fill(a, n);
  return a;
}

/* ------------------------------------------------------------------------------------------
 * Geometry input (Sec. 3.1): the fluid characteristic function H^f of Eq. characteristic,
 * given by the sign of a level set; points on the boundary count as solid.
 * ---------------------------------------------------------------------------------------- */

static double naca_half_thickness(const orc_case* c, double xi) {
  /* Standard NACA 4-digit symmetric thickness law (not given in the paper, which only names
   * the NACA 0010 section); closed trailing edge uses -0.1036 for the quartic term. */
  double t = c->naca_tt / 100.0;
  double a4 = c->closed_te ? -0.1036 : -0.1015;
  return 5.0 * t * (0.2969 * sqrt(xi) - 0.1260 * xi - 0.3516 * xi * xi + 0.2843 * xi * xi * xi +
                    a4 * xi * xi * xi * xi);
}

static int is_fluid(const orc_case* c, double x, double y) {
  switch (c->geom_kind) {
    case 1: {
      double dx = x - c->cx, dy = y - c->cy;
      return dx * dx + dy * dy > c->r * c->r;
    }
    case 2: {
      double a = c->aoa_deg * M_PI / 180.0;
      double px = x - c->le_x, py = y - c->le_y;
      double xi = (px * cos(a) - py * sin(a)) / c->chord;
      double eta = (px * sin(a) + py * cos(a)) / c->chord;
      if (xi < 0.0 || xi > 1.0) return 1;
      return fabs(eta) > naca_half_thickness(c, xi);
    }
    case 3:
      return c->hp_nx * x + c->hp_ny * y > c->hp_off;
    default:
      return 1;
  }
}

/* Boundary crossing on the segment (xa,ya)->(xb,yb), whose end points differ in fluid
 * status.  Returns the parameter t in [0,1].  Circle: root of the quadratic; half plane: the
 * linear root; NACA: bisection on the fluid indicator. */
static double crossing_t(const orc_case* c, double xa, double ya, double xb, double yb) {
  double dx = xb - xa, dy = yb - ya;
  if (c->geom_kind == 1) {
    double fx = xa - c->cx, fy = ya - c->cy;
    double qa = dx * dx + dy * dy;
    double qb = fx * dx + fy * dy;
    double qc = fx * fx + fy * fy - c->r * c->r;
    double disc = qb * qb - qa * qc;
    if (disc < 0.0) disc = 0.0;
    double sq = sqrt(disc);
    double t1 = (-qb - sq) / qa, t2 = (-qb + sq) / qa;
    double best = t1, d1 = 0.0, d2 = 0.0;
    if (t1 < 0.0) d1 = -t1; else if (t1 > 1.0) d1 = t1 - 1.0;
    if (t2 < 0.0) d2 = -t2; else if (t2 > 1.0) d2 = t2 - 1.0;
    if (d2 < d1) best = t2;
    if (best < 0.0) best = 0.0;
    if (best > 1.0) best = 1.0;
    return best;
  }
  if (c->geom_kind == 3) {
    double fa = c->hp_nx * xa + c->hp_ny * ya - c->hp_off;
    double fb = c->hp_nx * xb + c->hp_ny * yb - c->hp_off;
    double t = fa / (fa - fb);
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
    return t;
  }
  {
    int fa = is_fluid(c, xa, ya);
    double lo = 0.0, hi = 1.0;
    for (int k = 0; k < 64; ++k) {
      double m = 0.5 * (lo + hi);
      if (m <= lo || m >= hi) break;
      if (is_fluid(c, xa + m * dx, ya + m * dy) == fa) lo = m; else hi = m;
    }
    return 0.5 * (lo + hi);
  }
}

/* ------------------------------------------------------------------------------------------
 * Capacities (Sec. 3.2-3.4) by marching squares with exact edge crossings (Sec. 3.1 allows a
 * marching-squares reconstruction): the fluid part of a cell is the polygon bounded by the
 * wet parts of its edges and the straight segments joining the crossings.  Ambiguous
 * (saddle) cells are resolved by the fluid status of the cell centre.  Crossings are always
 * computed on edges oriented towards +x or +y so that neighbouring cells agree.
 * Coordinates are taken relative to the cell's lower-left corner.
 * ---------------------------------------------------------------------------------------- */

typedef struct { int n; double x[8], y[8]; int cross[8]; } polygon;

typedef struct {
  int npoly;
  polygon P[2];
  double xl, yb, hx, hy;      /* lower-left corner (absolute) and size */
  double ax_left, ay_bottom;  /* wet length of the left and bottom edges */
} cell_geom;

static void poly_add(polygon* p, double x, double y) { p->x[p->n] = x; p->y[p->n] = y; p->cross[p->n] = 0; p->n++; }
static void poly_add_cross(polygon* p, double x, double y) { poly_add(p, x, y); p->cross[p->n - 1] = 1; }

static void build_cell(const orc_case* c, double xl, double xr, double yb, double yt, cell_geom* g) {
  double hx = xr - xl, hy = yt - yb;
  g->xl = xl; g->yb = yb; g->hx = hx; g->hy = hy;
  g->npoly = 0;
  int f0 = is_fluid(c, xl, yb), f1 = is_fluid(c, xr, yb), f2 = is_fluid(c, xr, yt), f3 = is_fluid(c, xl, yt);
  /* crossings in local coordinates */
  double e0x = 0, e1y = 0, e2x = 0, e3y = 0;
  if (f0 != f1) e0x = crossing_t(c, xl, yb, xr, yb) * hx;
  if (f1 != f2) e1y = crossing_t(c, xr, yb, xr, yt) * hy;
  if (f3 != f2) e2x = crossing_t(c, xl, yt, xr, yt) * hx;
  if (f0 != f3) e3y = crossing_t(c, xl, yb, xl, yt) * hy;
  /* wet length of the left edge (x = xl) and bottom edge (y = yb) */
  if (f0 && f3) g->ax_left = hy; else if (!f0 && !f3) g->ax_left = 0.0; else if (f0) g->ax_left = e3y; else g->ax_left = hy - e3y;
  if (f0 && f1) g->ay_bottom = hx; else if (!f0 && !f1) g->ay_bottom = 0.0; else if (f0) g->ay_bottom = e0x; else g->ay_bottom = hx - e0x;

  int nf = f0 + f1 + f2 + f3;
  if (nf == 0) return;
  double cxs[4] = {0.0, hx, hx, 0.0}, cys[4] = {0.0, 0.0, hy, hy};
  double ex[4] = {e0x, hx, e2x, 0.0}, ey[4] = {0.0, e1y, hy, e3y};
  int f[4] = {f0, f1, f2, f3};
  int saddle = (f0 == f2) && (f1 == f3) && (f0 != f1);
  if (saddle && !is_fluid(c, xl + 0.5 * hx, yb + 0.5 * hy)) {
    /* separated: one triangle around each fluid corner */
    g->npoly = 2;
    polygon* a = &g->P[0];
    polygon* b = &g->P[1];
    a->n = 0; b->n = 0;
    if (f0) {
      poly_add(a, cxs[0], cys[0]); poly_add_cross(a, ex[0], ey[0]); poly_add_cross(a, ex[3], ey[3]);
      poly_add_cross(b, ex[1], ey[1]); poly_add(b, cxs[2], cys[2]); poly_add_cross(b, ex[2], ey[2]);
    } else {
      poly_add_cross(a, ex[0], ey[0]); poly_add(a, cxs[1], cys[1]); poly_add_cross(a, ex[1], ey[1]);
      poly_add_cross(b, ex[2], ey[2]); poly_add(b, cxs[3], cys[3]); poly_add_cross(b, ex[3], ey[3]);
    }
    return;
  }
  g->npoly = 1;
  polygon* p = &g->P[0];
  p->n = 0;
  for (int k = 0; k < 4; ++k) {
    int kn = (k + 1) & 3;
    if (f[k]) poly_add(p, cxs[k], cys[k]);
    if (f[k] != f[kn]) poly_add_cross(p, ex[k], ey[k]);
  }
}

static void poly_area_centroid(const polygon* p, double* area, double* mx, double* my) {
  /* shoelace area and first moments */
  double a = 0.0, sx = 0.0, sy = 0.0;
  for (int k = 0; k < p->n; ++k) {
    int kn = (k + 1) % p->n;
    double cr = p->x[k] * p->y[kn] - p->x[kn] * p->y[k];
    a += cr;
    sx += (p->x[k] + p->x[kn]) * cr;
    sy += (p->y[k] + p->y[kn]) * cr;
  }
  *area = 0.5 * a;
  *mx = sx / 6.0;  /* = integral of x over the polygon */
  *my = sy / 6.0;
}

/* Area of the part of a convex polygon with (coordinate >= s) if keep_above, else (<= s);
 * axis 0 clips on x, axis 1 on y (one Sutherland-Hodgman stage). */
static double clipped_area(const polygon* p, int axis, double s, int keep_above) {
  polygon q;
  q.n = 0;
  for (int k = 0; k < p->n; ++k) {
    int kn = (k + 1) % p->n;
    double pa = axis == 0 ? p->x[k] : p->y[k];
    double pb = axis == 0 ? p->x[kn] : p->y[kn];
    int ina = keep_above ? (pa >= s) : (pa <= s);
    int inb = keep_above ? (pb >= s) : (pb <= s);
    if (ina) poly_add(&q, p->x[k], p->y[k]);
    if (ina != inb) {
      double t = (s - pa) / (pb - pa);
      if (axis == 0) poly_add(&q, s, p->y[k] + t * (p->y[kn] - p->y[k]));
      else poly_add(&q, p->x[k] + t * (p->x[kn] - p->x[k]), s);
    }
  }
  if (q.n < 3) return 0.0;
  double a, mx, my;
  poly_area_centroid(&q, &a, &mx, &my);
  return a;
}

/* Length of the intersection of a convex polygon with the line (axis coordinate == s). */
static double line_length(const polygon* p, int axis, double s) {
  double lo = 1e300, hi = -1e300;
  int hit = 0;
  for (int k = 0; k < p->n; ++k) {
    int kn = (k + 1) % p->n;
    double pa = axis == 0 ? p->x[k] : p->y[k];
    double pb = axis == 0 ? p->x[kn] : p->y[kn];
    double qa = axis == 0 ? p->y[k] : p->x[k];
    double qb = axis == 0 ? p->y[kn] : p->x[kn];
    if ((pa - s) * (pb - s) > 0.0) continue;
    if (pa == pb) {
      /* edge lies on the line */
      if (qa < lo) lo = qa;
      if (qa > hi) hi = qa;
      if (qb < lo) lo = qb;
      if (qb > hi) hi = qb;
      hit = 1;
      continue;
    }
    double t = (s - pa) / (pb - pa);
    double q = qa + t * (qb - qa);
    if (q < lo) lo = q;
    if (q > hi) hi = q;
    hit = 1;
  }
  return hit ? hi - lo : 0.0;
}

typedef struct {
  cell_geom geo;
  double V, X, Y;   /* absolute centroid */
} cell_moments;

static void grid_offsets(const orc_case* c, int g, double* ox, double* oy) {
  *ox = (g == G_U) ? -0.5 * c->hx : 0.0;
  *oy = (g == G_V) ? -0.5 * c->hy : 0.0;
}

/* Face abscissa f of a stretched mesh for f in [-n, 2n]: beyond the box the spacing mirrors
 * the spacing inside it (x_{-k} = 2 x_0 - x_k), written as a sum and a difference so that no
 * compiler contracts it into a fused multiply-add. */
static double face_at(const double* a, int n, int f) {
  if (f < 0) return (a[0] + a[0]) - a[-f];
  if (f > n) return (a[n] + a[n]) - a[2 * n - f];
  return a[f];
}

/* Grid line abscissas: one expression for every use, so that cells sharing an edge or a
 * corner see bitwise identical coordinates.  Line i of the p- and v-grids in x is face x_i;
 * the u-grid's cells are centred on the faces (Sec. 3.4), so its line i is the centre of
 * p-cell i-1, (x_{i-1} + x_i) / 2 (on a uniform mesh, x0 + i hx - hx/2).  Likewise in y. */
static double line_x(const orc_case* c, int g, int i) {
  if (!c->xf) {
    double ox, oy;
    grid_offsets(c, g, &ox, &oy);
    return c->x0 + ox + i * c->hx;
  }
  if (g == G_U) return 0.5 * (face_at(c->xf, c->nx, i - 1) + face_at(c->xf, c->nx, i));
  return face_at(c->xf, c->nx, i);
}
static double line_y(const orc_case* c, int g, int j) {
  if (!c->yf) {
    double ox, oy;
    grid_offsets(c, g, &ox, &oy);
    return c->y0 + oy + j * c->hy;
  }
  if (g == G_V) return 0.5 * (face_at(c->yf, c->ny, j - 1) + face_at(c->yf, c->ny, j));
  return face_at(c->yf, c->ny, j);
}

/* Area of p-cell (i, j). */
static double cell_area(const orc_case* c, int i, int j) {
  if (!c->xf && !c->yf) return c->hx * c->hy;
  return (line_x(c, G_P, i + 1) - line_x(c, G_P, i)) * (line_y(c, G_P, j + 1) - line_y(c, G_P, j));
}

/* First-kind volume capacity and centroid of cell (i, j) of grid g (Eqs. volumefirstkind,
 * centroid).  An empty cell gets the cell centre as its centroid. */
static void moments(const orc_case* c, int g, int i, int j, cell_moments* m) {
  double xl = line_x(c, g, i), xr = line_x(c, g, i + 1);
  double yb = line_y(c, g, j), yt = line_y(c, g, j + 1);
  build_cell(c, xl, xr, yb, yt, &m->geo);
  double V = 0.0, MX = 0.0, MY = 0.0;
  for (int k = 0; k < m->geo.npoly; ++k) {
    double a, mx, my;
    poly_area_centroid(&m->geo.P[k], &a, &mx, &my);
    V += a; MX += mx; MY += my;
  }
  m->V = V;
  if (V > 0.0) {
    m->X = xl + MX / V;
    m->Y = yb + MY / V;
  } else {
    m->X = xl + 0.5 * m->geo.hx;
    m->Y = yb + 0.5 * m->geo.hy;
  }
}

/* Second-kind surface capacity (Eqs. surfacesecondkindx/y): wet length of the grid line
 * x = X (axis 0) or y = Y (axis 1) inside the cell. */
static double second_kind_surface(const cell_moments* m, int axis) {
  double s = axis == 0 ? m->X - m->geo.xl : m->Y - m->geo.yb;
  double L = 0.0;
  for (int k = 0; k < m->geo.npoly; ++k) L += line_length(&m->geo.P[k], axis, s);
  return L;
}

/* Second-kind volume capacity (Eqs. volumesecondkindx/y) at the left (axis 0) or bottom
 * (axis 1) face of cell (i, j): fluid area between the centroid of the neighbour
 * (i-1, j) or (i, j-1) and the centroid of (i, j). */
static double second_kind_volume(const orc_case* c, int g, int i, int j, int axis) {
  cell_moments a, b;
  if (axis == 0) moments(c, g, i - 1, j, &a); else moments(c, g, i, j - 1, &a);
  moments(c, g, i, j, &b);
  double W = 0.0;
  double sa = axis == 0 ? a.X - a.geo.xl : a.Y - a.geo.yb;
  double sb = axis == 0 ? b.X - b.geo.xl : b.Y - b.geo.yb;
  for (int k = 0; k < a.geo.npoly; ++k) W += clipped_area(&a.geo.P[k], axis, sa, 1);
  for (int k = 0; k < b.geo.npoly; ++k) W += clipped_area(&b.geo.P[k], axis, sb, 0);
  return W;
}

void orc_capacities(const orc_case* c, double* caps) {
  size_t S = SIZE(c);
  zero_fill(caps, 27 * S);
  for (int g = 0; g < 3; ++g) {
    PAR_FOR
    for (int j = -1; j <= c->ny + 1; ++j)
      for (int i = -1; i <= c->nx + 1; ++i) {
        cell_moments m;
        moments(c, g, i, j, &m);
        AT(c, CAP(c, caps, g, K_V), i, j) = m.V;
        AT(c, CAP(c, caps, g, K_X), i, j) = m.X;
        AT(c, CAP(c, caps, g, K_Y), i, j) = m.Y;
        AT(c, CAP(c, caps, g, K_AX), i, j) = m.geo.ax_left;
        AT(c, CAP(c, caps, g, K_AY), i, j) = m.geo.ay_bottom;
        AT(c, CAP(c, caps, g, K_BX), i, j) = second_kind_surface(&m, 0);
        AT(c, CAP(c, caps, g, K_BY), i, j) = second_kind_surface(&m, 1);
        AT(c, CAP(c, caps, g, K_WX), i, j) = second_kind_volume(c, g, i, j, 0);
        AT(c, CAP(c, caps, g, K_WY), i, j) = second_kind_volume(c, g, i, j, 1);
      }
  }
}

/* Boundary segment(s) of a cell: total length and the x component of the outward (from the
 * fluid) normal integrated over them, for the Surface Conservation Law of Eq. approximate.
 * Returns sum over segments of n_x |segment| and n_y |segment|, where n is the normal of
 * the boundary pointing out of the fluid region. */
void orc_cell_boundary(const orc_case* c, int g, int i, int j, double* nx_len, double* ny_len) {
  cell_moments m;
  moments(c, g, i, j, &m);
  double sx = 0.0, sy = 0.0;
  for (int k = 0; k < m.geo.npoly; ++k) {
    const polygon* p = &m.geo.P[k];
    for (int e = 0; e < p->n; ++e) {
      int en = (e + 1) % p->n;
      double ax = p->x[e], ay = p->y[e], bx = p->x[en], by = p->y[en];
      /* the boundary segments join two crossings; other edges are wet cell edges */
      if (!(p->cross[e] && p->cross[en])) continue;
      /* counter-clockwise polygon: outward normal of edge (dx, dy) is (dy, -dx) */
      sx += (by - ay);
      sy += -(bx - ax);
    }
  }
  *nx_len = sx;
  *ny_len = sy;
}

/* ------------------------------------------------------------------------------------------
 * Discrete operators (Sec. 4.1-4.4) in raw stencil form.  Face values (including ghost
 * layers) are taken as given; Dirichlet data D (the boundary value of the velocity on the
 * immersed boundary) may be NULL, meaning zero (no-slip, fixed body).
 * Notation: delta is the unit-spacing difference (Eq. differentiation), the bar the
 * two-point average (Eq. interpolation).
 * ---------------------------------------------------------------------------------------- */

static double dval(const orc_case* c, const double* D, int i, int j) { return D ? AT(c, D, i, j) : 0.0; }

static int in_pad(const orc_case* c, int i, int j) { return i >= -1 && i <= c->nx + 1 && j >= -1 && j <= c->ny + 1; }

/* Eq. divergence: volume-integrated velocity divergence at p-cells, with the heterogeneous
 * (immersed-boundary) terms built from the p-grid B and the Dirichlet data D. */
void orc_cont(const orc_case* c, const double* caps, const double* u, const double* v, const double* Dx,
              const double* Dy, double* out) {
  const double* Ax = CAP(c, caps, G_P, K_AX);
  const double* Ay = CAP(c, caps, G_P, K_AY);
  const double* Bx = CAP(c, caps, G_P, K_BX);
  const double* By = CAP(c, caps, G_P, K_BY);
  zero_fill(out, SIZE(c));
  PAR_FOR
  for (int j = 0; j < c->ny; ++j)
    for (int i = 0; i < c->nx; ++i) {
      double hom = AT(c, Ax, i + 1, j) * AT(c, u, i + 1, j) - AT(c, Ax, i, j) * AT(c, u, i, j) +
                   AT(c, Ay, i, j + 1) * AT(c, v, i, j + 1) - AT(c, Ay, i, j) * AT(c, v, i, j);
      /* x part: delta_x((bar B_x^x - A_x) D_x) - bar(delta_x B_x D_x)^x */
      double Er = (0.5 * (AT(c, Bx, i + 1, j) + AT(c, Bx, i, j)) - AT(c, Ax, i + 1, j)) * dval(c, Dx, i + 1, j);
      double El = (0.5 * (AT(c, Bx, i, j) + AT(c, Bx, i - 1, j)) - AT(c, Ax, i, j)) * dval(c, Dx, i, j);
      double Fr = (AT(c, Bx, i + 1, j) - AT(c, Bx, i, j)) * dval(c, Dx, i + 1, j);
      double Fl = (AT(c, Bx, i, j) - AT(c, Bx, i - 1, j)) * dval(c, Dx, i, j);
      double hx_ = (Er - El) - 0.5 * (Fr + Fl);
      double Et = (0.5 * (AT(c, By, i, j + 1) + AT(c, By, i, j)) - AT(c, Ay, i, j + 1)) * dval(c, Dy, i, j + 1);
      double Eb = (0.5 * (AT(c, By, i, j) + AT(c, By, i, j - 1)) - AT(c, Ay, i, j)) * dval(c, Dy, i, j);
      double Ft = (AT(c, By, i, j + 1) - AT(c, By, i, j)) * dval(c, Dy, i, j + 1);
      double Fb = (AT(c, By, i, j) - AT(c, By, i, j - 1)) * dval(c, Dy, i, j);
      double hy_ = (Et - Eb) - 0.5 * (Ft + Fb);
      AT(c, out, i, j) = hom + hx_ + hy_;
    }
}

/* Pressure gradient pres_alpha(P) = A_alpha delta_alpha P (Sec. 4.1), at u-faces
 * i in [0,nx], j in [0,ny) and v-faces i in [0,nx), j in [0,ny]. */
void orc_pres(const orc_case* c, const double* caps, const double* p, double* ou, double* ov) {
  const double* Ax = CAP(c, caps, G_P, K_AX);
  const double* Ay = CAP(c, caps, G_P, K_AY);
  zero_fill(ou, SIZE(c));
  zero_fill(ov, SIZE(c));
  PAR_FOR
  for (int j = 0; j < c->ny; ++j)
    for (int i = 0; i <= c->nx; ++i) AT(c, ou, i, j) = AT(c, Ax, i, j) * (AT(c, p, i, j) - AT(c, p, i - 1, j));
  PAR_FOR
  for (int j = 0; j <= c->ny; ++j)
    for (int i = 0; i < c->nx; ++i) AT(c, ov, i, j) = AT(c, Ay, i, j) * (AT(c, p, i, j) - AT(c, p, i, j - 1));
}

static double winv(const orc_case* c, double W) { return W > 1e-12 * c->hx * c->hy ? 1.0 / W : 0.0; }

/* Strain-rate tensor (Eqs. diag and offdiag).  S_xx at p-cells i in [-1,nx], j in [0,ny);
 * S_yy at p-cells i in [0,nx), j in [-1,ny]; S_xy at nodes i in [0,nx], j in [0,ny].
 * The off-diagonal weight is W^xy and W^yx separately when literal_offdiag is set and
 * their average (W^xy + W^yx)/2 for both halves otherwise.  Immersed-boundary terms whose
 * stencil leaves the padded range are dropped (the body stays two cells from the box). */
void orc_strain(const orc_case* c, const double* caps, const double* u, const double* v, const double* Dx,
                const double* Dy, double* sxx, double* syy, double* sxy) {
  const double* AxU = CAP(c, caps, G_U, K_AX);
  const double* AyU = CAP(c, caps, G_U, K_AY);
  const double* BxU = CAP(c, caps, G_U, K_BX);
  const double* ByU = CAP(c, caps, G_U, K_BY);
  const double* WxU = CAP(c, caps, G_U, K_WX);
  const double* WyU = CAP(c, caps, G_U, K_WY);
  const double* AxV = CAP(c, caps, G_V, K_AX);
  const double* AyV = CAP(c, caps, G_V, K_AY);
  const double* BxV = CAP(c, caps, G_V, K_BX);
  const double* ByV = CAP(c, caps, G_V, K_BY);
  const double* WxV = CAP(c, caps, G_V, K_WX);
  const double* WyV = CAP(c, caps, G_V, K_WY);
  zero_fill(sxx, SIZE(c));
  zero_fill(syy, SIZE(c));
  zero_fill(sxy, SIZE(c));
  /* S_xx at p-cell (i,j): u-faces i and i+1; A^xx at p-cell k is AxU(k+1) */
  PAR_FOR
  for (int j = 0; j < c->ny; ++j)
    for (int i = -1; i <= c->nx; ++i) {
      double g = AT(c, BxU, i + 1, j) * AT(c, u, i + 1, j) - AT(c, BxU, i, j) * AT(c, u, i, j);
      if (in_pad(c, i + 2, j)) {
        /* face f: (bar A^xx^x - B^xx) D_x, with bar A^xx at u-face f = (AxU(f+1) + AxU(f))/2 */
        double Er = (0.5 * (AT(c, AxU, i + 2, j) + AT(c, AxU, i + 1, j)) - AT(c, BxU, i + 1, j)) * dval(c, Dx, i + 1, j);
        double El = (0.5 * (AT(c, AxU, i + 1, j) + AT(c, AxU, i, j)) - AT(c, BxU, i, j)) * dval(c, Dx, i, j);
        double Fr = (AT(c, AxU, i + 2, j) - AT(c, AxU, i + 1, j)) * dval(c, Dx, i + 1, j);
        double Fl = (AT(c, AxU, i + 1, j) - AT(c, AxU, i, j)) * dval(c, Dx, i, j);
        g += (Er - El) - 0.5 * (Fr + Fl);
      }
      AT(c, sxx, i, j) = g * winv(c, AT(c, WxU, i + 1, j));
    }
  PAR_FOR
  for (int j = -1; j <= c->ny; ++j)
    for (int i = 0; i < c->nx; ++i) {
      double g = AT(c, ByV, i, j + 1) * AT(c, v, i, j + 1) - AT(c, ByV, i, j) * AT(c, v, i, j);
      if (in_pad(c, i, j + 2)) {
        double Et = (0.5 * (AT(c, AyV, i, j + 2) + AT(c, AyV, i, j + 1)) - AT(c, ByV, i, j + 1)) * dval(c, Dy, i, j + 1);
        double Eb = (0.5 * (AT(c, AyV, i, j + 1) + AT(c, AyV, i, j)) - AT(c, ByV, i, j)) * dval(c, Dy, i, j);
        double Ft = (AT(c, AyV, i, j + 2) - AT(c, AyV, i, j + 1)) * dval(c, Dy, i, j + 1);
        double Fb = (AT(c, AyV, i, j + 1) - AT(c, AyV, i, j)) * dval(c, Dy, i, j);
        g += (Et - Eb) - 0.5 * (Ft + Fb);
      }
      AT(c, syy, i, j) = g * winv(c, AT(c, WyV, i, j + 1));
    }
  /* S_xy at node (i,j) */
  PAR_FOR
  for (int j = 0; j <= c->ny; ++j)
    for (int i = 0; i <= c->nx; ++i) {
      /* alpha = x, beta = y on the u-grid: B^xy at u-faces (i,j-1),(i,j); A^xy at nodes = AyU */
      double gx = AT(c, ByU, i, j) * AT(c, u, i, j) - AT(c, ByU, i, j - 1) * AT(c, u, i, j - 1);
      {
        double Et = (0.5 * (AT(c, AyU, i, j + 1) + AT(c, AyU, i, j)) - AT(c, ByU, i, j)) * dval(c, Dx, i, j);
        double Eb = (0.5 * (AT(c, AyU, i, j) + AT(c, AyU, i, j - 1)) - AT(c, ByU, i, j - 1)) * dval(c, Dx, i, j - 1);
        double Ft = (AT(c, AyU, i, j + 1) - AT(c, AyU, i, j)) * dval(c, Dx, i, j);
        double Fb = (AT(c, AyU, i, j) - AT(c, AyU, i, j - 1)) * dval(c, Dx, i, j - 1);
        gx += (Et - Eb) - 0.5 * (Ft + Fb);
      }
      /* alpha = y, beta = x on the v-grid: B^yx at v-faces (i-1,j),(i,j); A^yx at nodes = AxV */
      double gy = AT(c, BxV, i, j) * AT(c, v, i, j) - AT(c, BxV, i - 1, j) * AT(c, v, i - 1, j);
      {
        double Er = (0.5 * (AT(c, AxV, i + 1, j) + AT(c, AxV, i, j)) - AT(c, BxV, i, j)) * dval(c, Dy, i, j);
        double El = (0.5 * (AT(c, AxV, i, j) + AT(c, AxV, i - 1, j)) - AT(c, BxV, i - 1, j)) * dval(c, Dy, i - 1, j);
        double Fr = (AT(c, AxV, i + 1, j) - AT(c, AxV, i, j)) * dval(c, Dy, i, j);
        double Fl = (AT(c, AxV, i, j) - AT(c, AxV, i - 1, j)) * dval(c, Dy, i - 1, j);
        gy += (Er - El) - 0.5 * (Fr + Fl);
      }
      double wxy = AT(c, WyU, i, j), wyx = AT(c, WxV, i, j);
      if (c->literal_offdiag)
        AT(c, sxy, i, j) = 0.5 * gx * winv(c, wxy) + 0.5 * gy * winv(c, wyx);
      else
        AT(c, sxy, i, j) = 0.5 * (gx + gy) * winv(c, 0.5 * (wxy + wyx));
    }
}

/* Viscous transport visc_alpha(S) = sum_beta B_alpha_beta delta_beta S_alpha_beta
 * (Sec. 4.3), at u-faces i in [0,nx], j in [0,ny) and v-faces i in [0,nx), j in [0,ny]. */
void orc_visc(const orc_case* c, const double* caps, const double* sxx, const double* syy, const double* sxy,
              double* ou, double* ov) {
  const double* BxU = CAP(c, caps, G_U, K_BX);
  const double* ByU = CAP(c, caps, G_U, K_BY);
  const double* BxV = CAP(c, caps, G_V, K_BX);
  const double* ByV = CAP(c, caps, G_V, K_BY);
  zero_fill(ou, SIZE(c));
  zero_fill(ov, SIZE(c));
  PAR_FOR
  for (int j = 0; j < c->ny; ++j)
    for (int i = 0; i <= c->nx; ++i)
      AT(c, ou, i, j) = AT(c, BxU, i, j) * (AT(c, sxx, i, j) - AT(c, sxx, i - 1, j)) +
                        AT(c, ByU, i, j) * (AT(c, sxy, i, j + 1) - AT(c, sxy, i, j));
  PAR_FOR
  for (int j = 0; j <= c->ny; ++j)
    for (int i = 0; i < c->nx; ++i)
      AT(c, ov, i, j) = AT(c, ByV, i, j) * (AT(c, syy, i, j) - AT(c, syy, i, j - 1)) +
                        AT(c, BxV, i, j) * (AT(c, sxy, i + 1, j) - AT(c, sxy, i, j));
}

/* Convective transport, Eq. convective, conv_alpha(U, U', D, D') at u-faces
 * i in [0,nx], j in [0,ny) and v-faces i in [0,nx), j in [0,ny].  The mass fluxes use the
 * p-grid surface capacities A_beta; the bracket uses the p-grid B_beta and D_beta. */
void orc_conv(const orc_case* c, const double* caps, const double* u, const double* v, const double* ut,
              const double* vt, const double* Dx, const double* Dy, const double* Dxt, const double* Dyt,
              double* ou, double* ov) {
  const double* Ax = CAP(c, caps, G_P, K_AX);
  const double* Ay = CAP(c, caps, G_P, K_AY);
  const double* Bx = CAP(c, caps, G_P, K_BX);
  const double* By = CAP(c, caps, G_P, K_BY);
  zero_fill(ou, SIZE(c));
  zero_fill(ov, SIZE(c));
#define EX(i, j) ((0.5 * (AT(c, Bx, (i), (j)) + AT(c, Bx, (i) - 1, (j))) - AT(c, Ax, (i), (j))) * dval(c, Dx, (i), (j)))
#define FX(i, j) ((AT(c, Bx, (i), (j)) - AT(c, Bx, (i) - 1, (j))) * dval(c, Dx, (i), (j)))
#define EY(i, j) ((0.5 * (AT(c, By, (i), (j)) + AT(c, By, (i), (j) - 1)) - AT(c, Ay, (i), (j))) * dval(c, Dy, (i), (j)))
#define FY(i, j) ((AT(c, By, (i), (j)) - AT(c, By, (i), (j) - 1)) * dval(c, Dy, (i), (j)))
  PAR_FOR
  for (int j = 0; j < c->ny; ++j)
    for (int i = 0; i <= c->nx; ++i) {
      /* beta = x: mass flux bar(A_x U_x)^x and bar(U'_x)^x at p-cells i-1 and i */
      double Fr = 0.5 * (AT(c, Ax, i + 1, j) * AT(c, u, i + 1, j) + AT(c, Ax, i, j) * AT(c, u, i, j));
      double Fl = 0.5 * (AT(c, Ax, i, j) * AT(c, u, i, j) + AT(c, Ax, i - 1, j) * AT(c, u, i - 1, j));
      double ur = 0.5 * (AT(c, ut, i + 1, j) + AT(c, ut, i, j));
      double ul = 0.5 * (AT(c, ut, i, j) + AT(c, ut, i - 1, j));
      double cx_ = Fr * ur - Fl * ul;
      /* beta = y: bar(A_y U_y)^x and bar(U'_x)^y at nodes (i,j+1) and (i,j) */
      double Gt = 0.5 * (AT(c, Ay, i, j + 1) * AT(c, v, i, j + 1) + AT(c, Ay, i - 1, j + 1) * AT(c, v, i - 1, j + 1));
      double Gb = 0.5 * (AT(c, Ay, i, j) * AT(c, v, i, j) + AT(c, Ay, i - 1, j) * AT(c, v, i - 1, j));
      double ut_t = 0.5 * (AT(c, ut, i, j + 1) + AT(c, ut, i, j));
      double ut_b = 0.5 * (AT(c, ut, i, j) + AT(c, ut, i, j - 1));
      double cy_ = Gt * ut_t - Gb * ut_b;
      /* bracket: delta_beta(bar((bar B_beta^beta - A_beta) D_beta)^x) - bar(bar(delta_beta B_beta D_beta)^beta)^x */
      double br = 0.0;
      if (in_pad(c, i + 2, j) && in_pad(c, i - 2, j)) {
        double ebar_r = 0.5 * (EX(i + 1, j) + EX(i, j)); /* p-cell i */
        double ebar_l = 0.5 * (EX(i, j) + EX(i - 1, j)); /* p-cell i-1 */
        double fbar_r = 0.5 * (FX(i + 1, j) + FX(i, j));
        double fbar_l = 0.5 * (FX(i, j) + FX(i - 1, j));
        br += (ebar_r - ebar_l) - 0.5 * (fbar_r + fbar_l);
      }
      if (in_pad(c, i - 1, j + 2) && in_pad(c, i, j - 1)) {
        double eyt = 0.5 * (EY(i, j + 1) + EY(i - 1, j + 1)); /* node (i,j+1) */
        double eyb = 0.5 * (EY(i, j) + EY(i - 1, j));         /* node (i,j) */
        double fy_r = 0.5 * (FY(i, j + 1) + FY(i, j));         /* p-cell (i,j) */
        double fy_l = 0.5 * (FY(i - 1, j + 1) + FY(i - 1, j)); /* p-cell (i-1,j) */
        br += (eyt - eyb) - 0.5 * (fy_r + fy_l);
      }
      AT(c, ou, i, j) = cx_ + cy_ + br * 0.5 * (AT(c, ut, i, j) + dval(c, Dxt, i, j));
    }
  PAR_FOR
  for (int j = 0; j <= c->ny; ++j)
    for (int i = 0; i < c->nx; ++i) {
      /* beta = y: bar(A_y U_y)^y and bar(U'_y)^y at p-cells j-1 and j */
      double Ht = 0.5 * (AT(c, Ay, i, j + 1) * AT(c, v, i, j + 1) + AT(c, Ay, i, j) * AT(c, v, i, j));
      double Hb = 0.5 * (AT(c, Ay, i, j) * AT(c, v, i, j) + AT(c, Ay, i, j - 1) * AT(c, v, i, j - 1));
      double vt_t = 0.5 * (AT(c, vt, i, j + 1) + AT(c, vt, i, j));
      double vt_b = 0.5 * (AT(c, vt, i, j) + AT(c, vt, i, j - 1));
      double cy_ = Ht * vt_t - Hb * vt_b;
      /* beta = x: bar(A_x U_x)^y and bar(U'_y)^x at nodes (i+1,j) and (i,j) */
      double Kr = 0.5 * (AT(c, Ax, i + 1, j) * AT(c, u, i + 1, j) + AT(c, Ax, i + 1, j - 1) * AT(c, u, i + 1, j - 1));
      double Kl = 0.5 * (AT(c, Ax, i, j) * AT(c, u, i, j) + AT(c, Ax, i, j - 1) * AT(c, u, i, j - 1));
      double vr = 0.5 * (AT(c, vt, i + 1, j) + AT(c, vt, i, j));
      double vl = 0.5 * (AT(c, vt, i, j) + AT(c, vt, i - 1, j));
      double cx_ = Kr * vr - Kl * vl;
      double br = 0.0;
      if (in_pad(c, i, j + 2) && in_pad(c, i, j - 2)) {
        double ebar_t = 0.5 * (EY(i, j + 1) + EY(i, j));
        double ebar_b = 0.5 * (EY(i, j) + EY(i, j - 1));
        double fbar_t = 0.5 * (FY(i, j + 1) + FY(i, j));
        double fbar_b = 0.5 * (FY(i, j) + FY(i, j - 1));
        br += (ebar_t - ebar_b) - 0.5 * (fbar_t + fbar_b);
      }
      if (in_pad(c, i + 2, j - 1) && in_pad(c, i - 1, j)) {
        double exr = 0.5 * (EX(i + 1, j) + EX(i + 1, j - 1)); /* node (i+1,j) */
        double exl = 0.5 * (EX(i, j) + EX(i, j - 1));         /* node (i,j) */
        double fx_t = 0.5 * (FX(i + 1, j) + FX(i, j));         /* p-cell (i,j) */
        double fx_b = 0.5 * (FX(i + 1, j - 1) + FX(i, j - 1)); /* p-cell (i,j-1) */
        br += (exr - exl) - 0.5 * (fx_t + fx_b);
      }
      AT(c, ov, i, j) = cy_ + cx_ + br * 0.5 * (AT(c, vt, i, j) + dval(c, Dyt, i, j));
    }
#undef EX
#undef FX
#undef EY
#undef FY
}

/* ------------------------------------------------------------------------------------------
 * Box boundary conditions (Sec. 4.6 and Sec. 5.1: velocity Dirichlet on the inflow side,
 * zero-gradient velocity with zero pressure on outflow sides; the discrete form is not
 * spelled out in the paper).  Dirichlet sides fix the normal face velocity and reflect the
 * tangential component about the prescribed value; outflow sides copy the adjacent value
 * into the ghost layer.
 * ---------------------------------------------------------------------------------------- */

static int is_dir_u(const orc_case* c, int i) {
  return (i == 0 && c->bc_type[W_SIDE] == BC_DIR) || (i == c->nx && c->bc_type[E_SIDE] == BC_DIR);
}
static int is_dir_v(const orc_case* c, int j) {
  return (j == 0 && c->bc_type[S_SIDE] == BC_DIR) || (j == c->ny && c->bc_type[N_SIDE] == BC_DIR);
}

static double epsV(const orc_case* c) { return 1e-12 * c->hx * c->hy; }

/* role of a u-face: 0 not a velocity position (ghost), 1 Dirichlet box face, 2 inactive
 * (no fluid in its control volume, held at zero), 3 unknown */
static int role_u(const orc_case* c, const double* caps, int i, int j) {
  if (i < 0 || i > c->nx || j < 0 || j >= c->ny) return 0;
  if (PER_X(c) && i == c->nx) return 0;  /* the image of face 0 */
  if (is_dir_u(c, i)) return 1;
  return AT(c, CAP(c, caps, G_U, K_V), i, j) > epsV(c) ? 3 : 2;
}
static int role_v(const orc_case* c, const double* caps, int i, int j) {
  if (i < 0 || i >= c->nx || j < 0 || j > c->ny) return 0;
  if (PER_Y(c) && j == c->ny) return 0;
  if (is_dir_v(c, j)) return 1;
  return AT(c, CAP(c, caps, G_V, K_V), i, j) > epsV(c) ? 3 : 2;
}

int orc_role_u(const orc_case* c, const double* caps, int i, int j) { return role_u(c, caps, i, j); }
int orc_role_v(const orc_case* c, const double* caps, int i, int j) { return role_v(c, caps, i, j); }

/* Periodic sides: every position beyond the box takes the value of its image inside it,
 * face nx that of face 0 (x first over all rows, then y over all columns, so that the corners
 * are consistent). */
static void wrap_faces(const orc_case* c, double* u, double* v) {
  int nx = c->nx, ny = c->ny;
  if (PER_X(c))
    for (int j = -1; j <= ny + 1; ++j) {
      if (u) { AT(c, u, -1, j) = AT(c, u, nx - 1, j); AT(c, u, nx, j) = AT(c, u, 0, j); AT(c, u, nx + 1, j) = AT(c, u, 1, j); }
      if (v) { AT(c, v, -1, j) = AT(c, v, nx - 1, j); AT(c, v, nx, j) = AT(c, v, 0, j); AT(c, v, nx + 1, j) = AT(c, v, 1, j); }
    }
  if (PER_Y(c))
    for (int i = -1; i <= nx + 1; ++i) {
      if (u) { AT(c, u, i, -1) = AT(c, u, i, ny - 1); AT(c, u, i, ny) = AT(c, u, i, 0); AT(c, u, i, ny + 1) = AT(c, u, i, 1); }
      if (v) { AT(c, v, i, -1) = AT(c, v, i, ny - 1); AT(c, v, i, ny) = AT(c, v, i, 0); AT(c, v, i, ny + 1) = AT(c, v, i, 1); }
    }
}

/* Cell fields on periodic sides: cell -1 takes cell nx-1, cell nx cell 0 (and y likewise). */
static void wrap_cells(const orc_case* c, double* p) {
  int nx = c->nx, ny = c->ny;
  if (PER_X(c))
    for (int j = -1; j <= ny + 1; ++j) { AT(c, p, -1, j) = AT(c, p, nx - 1, j); AT(c, p, nx, j) = AT(c, p, 0, j); }
  if (PER_Y(c))
    for (int i = -1; i <= nx + 1; ++i) { AT(c, p, i, -1) = AT(c, p, i, ny - 1); AT(c, p, i, ny) = AT(c, p, i, 0); }
}

/* Set the Dirichlet box faces to their values (scaled by `scale`, 0 for the homogeneous
 * part) and fill the ghost layer. */
static void fill_bc(const orc_case* c, double* u, double* v, double scale) {
  int nx = c->nx, ny = c->ny;
  for (int j = 0; j < ny; ++j) {
    if (c->bc_type[W_SIDE] == BC_DIR) AT(c, u, 0, j) = scale * c->bc_un[W_SIDE];
    if (c->bc_type[E_SIDE] == BC_DIR) AT(c, u, nx, j) = scale * c->bc_un[E_SIDE];
  }
  for (int i = 0; i < nx; ++i) {
    if (c->bc_type[S_SIDE] == BC_DIR) AT(c, v, i, 0) = scale * c->bc_un[S_SIDE];
    if (c->bc_type[N_SIDE] == BC_DIR) AT(c, v, i, ny) = scale * c->bc_un[N_SIDE];
  }
  /* normal-component ghosts beyond W/E (u) and S/N (v): copies */
  for (int j = 0; j < ny; ++j) {
    AT(c, u, -1, j) = AT(c, u, 0, j);
    AT(c, u, nx + 1, j) = AT(c, u, nx, j);
  }
  for (int i = 0; i < nx; ++i) {
    AT(c, v, i, -1) = AT(c, v, i, 0);
    AT(c, v, i, ny + 1) = AT(c, v, i, ny);
  }
  /* tangential ghosts: u below S / above N, v left of W / right of E */
  for (int i = 0; i <= nx; ++i) {
    AT(c, u, i, -1) = c->bc_type[S_SIDE] == BC_DIR ? 2.0 * scale * c->bc_ut[S_SIDE] - AT(c, u, i, 0) : AT(c, u, i, 0);
    AT(c, u, i, ny) = c->bc_type[N_SIDE] == BC_DIR ? 2.0 * scale * c->bc_ut[N_SIDE] - AT(c, u, i, ny - 1) : AT(c, u, i, ny - 1);
  }
  for (int j = 0; j <= ny; ++j) {
    AT(c, v, -1, j) = c->bc_type[W_SIDE] == BC_DIR ? 2.0 * scale * c->bc_ut[W_SIDE] - AT(c, v, 0, j) : AT(c, v, 0, j);
    AT(c, v, nx, j) = c->bc_type[E_SIDE] == BC_DIR ? 2.0 * scale * c->bc_ut[E_SIDE] - AT(c, v, nx - 1, j) : AT(c, v, nx - 1, j);
  }
  wrap_faces(c, u, v);
}

void orc_fill_ghosts(const orc_case* c, double* u, double* v) { fill_bc(c, u, v, 1.0); }

/* Viscous operator with the box boundary rules, visc(S(U)) on ghost-filled U, restricted
 * to the velocity unknowns.  On an outflow side the tangential velocity next to the side
 * does not receive the shear stress at the boundary nodes: with zero-gradient ghosts its
 * total coefficient in that stress vanishes, so dropping it keeps the operator symmetric. */
static void visc_bc(const orc_case* c, const double* caps, const double* u, const double* v, const double* Dx,
                    const double* Dy, double* ou, double* ov) {
  size_t S = SIZE(c);
  double* sxx = malloc(S * sizeof(double));
  double* syy = malloc(S * sizeof(double));
  double* sxy = malloc(S * sizeof(double));
  orc_strain(c, caps, u, v, Dx, Dy, sxx, syy, sxy);
  orc_visc(c, caps, sxx, syy, sxy, ou, ov);
  const double* ByU = CAP(c, caps, G_U, K_BY);
  const double* BxV = CAP(c, caps, G_V, K_BX);
  int nx = c->nx, ny = c->ny;
  if (c->bc_type[E_SIDE] == BC_OUT)
    for (int j = 0; j <= ny; ++j) AT(c, ov, nx - 1, j) -= AT(c, BxV, nx - 1, j) * AT(c, sxy, nx, j);
  if (c->bc_type[W_SIDE] == BC_OUT)
    for (int j = 0; j <= ny; ++j) AT(c, ov, 0, j) += AT(c, BxV, 0, j) * AT(c, sxy, 0, j);
  if (c->bc_type[N_SIDE] == BC_OUT)
    for (int i = 0; i <= nx; ++i) AT(c, ou, i, ny - 1) -= AT(c, ByU, i, ny - 1) * AT(c, sxy, i, ny);
  if (c->bc_type[S_SIDE] == BC_OUT)
    for (int i = 0; i <= nx; ++i) AT(c, ou, i, 0) += AT(c, ByU, i, 0) * AT(c, sxy, i, 0);
  PAR_FOR
  for (int j = -1; j <= ny + 1; ++j)
    for (int i = -1; i <= nx + 1; ++i) {
      if (role_u(c, caps, i, j) != 3) AT(c, ou, i, j) = 0.0;
      if (role_v(c, caps, i, j) != 3) AT(c, ov, i, j) = 0.0;
    }
  free(sxx); free(syy); free(sxy);
}

/* visc with box rules applied to a velocity field whose Dirichlet faces and ghosts are
 * filled here (affine in the boundary values). */
void orc_visc_bc(const orc_case* c, const double* caps, const double* u_in, const double* v_in, double* ou,
                 double* ov) {
  size_t S = SIZE(c);
  double* u = malloc(S * sizeof(double));
  double* v = malloc(S * sizeof(double));
  memcpy(u, u_in, S * sizeof(double));
  memcpy(v, v_in, S * sizeof(double));
  fill_bc(c, u, v, 1.0);
  visc_bc(c, caps, u, v, NULL, NULL, ou, ov);
  free(u); free(v);
}

/* conv(U, U, D, D) on ghost-filled U, restricted to the velocity unknowns (D may be NULL). */
static void conv_bc(const orc_case* c, const double* caps, const double* u_in, const double* v_in,
                    const double* Dx, const double* Dy, double* ou, double* ov) {
  size_t S = SIZE(c);
  double* u = malloc(S * sizeof(double));
  double* v = malloc(S * sizeof(double));
  memcpy(u, u_in, S * sizeof(double));
  memcpy(v, v_in, S * sizeof(double));
  fill_bc(c, u, v, 1.0);
  orc_conv(c, caps, u, v, u, v, Dx, Dy, Dx, Dy, ou, ov);
  PAR_FOR
  for (int j = -1; j <= c->ny + 1; ++j)
    for (int i = -1; i <= c->nx + 1; ++i) {
      if (role_u(c, caps, i, j) != 3) AT(c, ou, i, j) = 0.0;
      if (role_v(c, caps, i, j) != 3) AT(c, ov, i, j) = 0.0;
    }
  free(u); free(v);
}

/* conv(U, U, 0, 0) on ghost-filled U, restricted to the velocity unknowns. */
void orc_conv_bc(const orc_case* c, const double* caps, const double* u_in, const double* v_in, double* ou,
                 double* ov) {
  conv_bc(c, caps, u_in, v_in, NULL, NULL, ou, ov);
}

/* pres(P) restricted to the velocity unknowns; the ghost ring of P is read as zero
 * (Dirichlet pressure on outflow sides). */
void orc_pres_bc(const orc_case* c, const double* caps, const double* p_in, double* ou, double* ov) {
  size_t S = SIZE(c);
  double* p = zalloc(S);
  PAR_FOR
  for (int j = 0; j < c->ny; ++j)
    for (int i = 0; i < c->nx; ++i) AT(c, p, i, j) = AT(c, p_in, i, j);
  wrap_cells(c, p);  /* periodic sides: the image cells; otherwise zero (Dirichlet) */
  orc_pres(c, caps, p, ou, ov);
  PAR_FOR
  for (int j = -1; j <= c->ny + 1; ++j)
    for (int i = -1; i <= c->nx + 1; ++i) {
      if (role_u(c, caps, i, j) != 3) AT(c, ou, i, j) = 0.0;
      if (role_v(c, caps, i, j) != 3) AT(c, ov, i, j) = 0.0;
    }
  free(p);
}

/* ------------------------------------------------------------------------------------------
 * Implicit operators of the projection step (Sec. 4.6).
 * Helmholtz: H U = (rho/dt) M U - mu visc(S_hom(U)) on the velocity unknowns, identity on
 * inactive faces (Eq. pm_prediction, Crank-Nicolson half of the viscous term).
 * Poisson:  K Phi = -cont(M^-1 pres(Phi), 0) on active cells, identity on inactive cells
 * (Eq. pm_poisson with the mass matrix of Eq. semidiscrete).
 * ---------------------------------------------------------------------------------------- */

void orc_helmholtz(const orc_case* c, const double* caps, const double* u_in, const double* v_in, double* ou,
                   double* ov) {
  size_t S = SIZE(c);
  double* u = zalloc(S);
  double* v = zalloc(S);
  PAR_FOR
  for (int j = -1; j <= c->ny + 1; ++j)
    for (int i = -1; i <= c->nx + 1; ++i) {
      if (role_u(c, caps, i, j) == 3) AT(c, u, i, j) = AT(c, u_in, i, j);
      if (role_v(c, caps, i, j) == 3) AT(c, v, i, j) = AT(c, v_in, i, j);
    }
  fill_bc(c, u, v, 0.0);
  visc_bc(c, caps, u, v, NULL, NULL, ou, ov);
  const double* Vu = CAP(c, caps, G_U, K_V);
  const double* Vv = CAP(c, caps, G_V, K_V);
  double s = c->rho / c->dt;
  PAR_FOR
  for (int j = -1; j <= c->ny + 1; ++j)
    for (int i = -1; i <= c->nx + 1; ++i) {
      int ru = role_u(c, caps, i, j), rv = role_v(c, caps, i, j);
      if (ru == 3) AT(c, ou, i, j) = s * AT(c, Vu, i, j) * AT(c, u, i, j) - c->mu * AT(c, ou, i, j);
      else AT(c, ou, i, j) = (ru == 2) ? AT(c, u_in, i, j) : 0.0;
      if (rv == 3) AT(c, ov, i, j) = s * AT(c, Vv, i, j) * AT(c, v, i, j) - c->mu * AT(c, ov, i, j);
      else AT(c, ov, i, j) = (rv == 2) ? AT(c, v_in, i, j) : 0.0;
    }
  free(u); free(v);
}

/* Poisson face coefficient A_f^2 / V_f of an unknown face, zero otherwise. */
static double coef_u(const orc_case* c, const double* caps, int i, int j) {
  if (PER_X(c) && i == c->nx) i = 0;
  if (role_u(c, caps, i, j) != 3) return 0.0;
  double A = AT(c, CAP(c, caps, G_P, K_AX), i, j);
  return A * A * winv(c, AT(c, CAP(c, caps, G_U, K_V), i, j));
}
static double coef_v(const orc_case* c, const double* caps, int i, int j) {
  if (PER_Y(c) && j == c->ny) j = 0;
  if (role_v(c, caps, i, j) != 3) return 0.0;
  double A = AT(c, CAP(c, caps, G_P, K_AY), i, j);
  return A * A * winv(c, AT(c, CAP(c, caps, G_V, K_V), i, j));
}

static int cell_active(const orc_case* c, const double* caps, int i, int j) {
  if (i < 0 || i >= c->nx || j < 0 || j >= c->ny) return 0;
  return coef_u(c, caps, i, j) + coef_u(c, caps, i + 1, j) + coef_v(c, caps, i, j) + coef_v(c, caps, i, j + 1) > 0.0;
}
int orc_cell_active(const orc_case* c, const double* caps, int i, int j) { return cell_active(c, caps, i, j); }

/* Role arrays over the padded layout: u/v roles (0 ghost, 1 Dirichlet, 2 inactive,
 * 3 unknown) and active pressure cells (1/0). */
void orc_roles(const orc_case* c, const double* caps, int* ru, int* rv, int* act) {
  for (int j = -1; j <= c->ny + 1; ++j)
    for (int i = -1; i <= c->nx + 1; ++i) {
      size_t k = (size_t)(j + 1) * PITCH(c) + (size_t)(i + 1);
      ru[k] = role_u(c, caps, i, j);
      rv[k] = role_v(c, caps, i, j);
      act[k] = cell_active(c, caps, i, j);
    }
}

void orc_poisson(const orc_case* c, const double* caps, const double* phi_in, double* out) {
  size_t S = SIZE(c);
  double* phi = zalloc(S);
  double* gu = malloc(S * sizeof(double));
  double* gv = malloc(S * sizeof(double));
  PAR_FOR
  for (int j = 0; j < c->ny; ++j)
    for (int i = 0; i < c->nx; ++i)
      if (cell_active(c, caps, i, j)) AT(c, phi, i, j) = AT(c, phi_in, i, j);
  /* pres(Phi) on unknown faces, then M^-1 */
  orc_pres_bc(c, caps, phi, gu, gv);
  const double* Vu = CAP(c, caps, G_U, K_V);
  const double* Vv = CAP(c, caps, G_V, K_V);
  PAR_FOR
  for (size_t k = 0; k < S; ++k) {
    gu[k] *= winv(c, Vu[k]);
    gv[k] *= winv(c, Vv[k]);
  }
  wrap_faces(c, gu, gv);  /* periodic: the flux through face nx is the flux through face 0 */
  orc_cont(c, caps, gu, gv, NULL, NULL, out);
  PAR_FOR
  for (int j = -1; j <= c->ny + 1; ++j)
    for (int i = -1; i <= c->nx + 1; ++i) {
      if (cell_active(c, caps, i, j)) AT(c, out, i, j) = -AT(c, out, i, j);
      else if (i >= 0 && i < c->nx && j >= 0 && j < c->ny) AT(c, out, i, j) = AT(c, phi_in, i, j);
      else AT(c, out, i, j) = 0.0;
    }
  free(phi); free(gu); free(gv);
}

/* Diagonals by probing: apply the operator to the sum of unit vectors of one colour class
 * (positions congruent mod 3 in both directions); the operators couple only positions at
 * distance <= 1, so each probe returns the diagonal entries of its class. */
void orc_poisson_diag(const orc_case* c, const double* caps, double* diag) {
  size_t S = SIZE(c);
  double* e = malloc(S * sizeof(double));
  double* o = malloc(S * sizeof(double));
  memset(diag, 0, S * sizeof(double));
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      zero_fill(e, S);
      PAR_FOR
      for (int j = 0; j < c->ny; ++j)
        for (int i = 0; i < c->nx; ++i)
          if (i % 3 == a && j % 3 == b) AT(c, e, i, j) = 1.0;
      orc_poisson(c, caps, e, o);
      PAR_FOR
      for (int j = 0; j < c->ny; ++j)
        for (int i = 0; i < c->nx; ++i)
          if (i % 3 == a && j % 3 == b) AT(c, diag, i, j) = AT(c, o, i, j);
    }
  free(e); free(o);
}

void orc_helmholtz_diag(const orc_case* c, const double* caps, double* du, double* dv) {
  size_t S = SIZE(c);
  double* eu = malloc(S * sizeof(double));
  double* ev = malloc(S * sizeof(double));
  double* ou = malloc(S * sizeof(double));
  double* ov = malloc(S * sizeof(double));
  memset(du, 0, S * sizeof(double));
  memset(dv, 0, S * sizeof(double));
  for (int comp = 0; comp < 2; ++comp)
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        memset(eu, 0, S * sizeof(double));
        memset(ev, 0, S * sizeof(double));
        for (int j = -1; j <= c->ny + 1; ++j)
          for (int i = -1; i <= c->nx + 1; ++i) {
            if (((i + 3) % 3) != a || ((j + 3) % 3) != b) continue;
            if (comp == 0 && role_u(c, caps, i, j) >= 2) AT(c, eu, i, j) = 1.0;
            if (comp == 1 && role_v(c, caps, i, j) >= 2) AT(c, ev, i, j) = 1.0;
          }
        orc_helmholtz(c, caps, eu, ev, ou, ov);
        for (int j = -1; j <= c->ny + 1; ++j)
          for (int i = -1; i <= c->nx + 1; ++i) {
            if (((i + 3) % 3) != a || ((j + 3) % 3) != b) continue;
            if (comp == 0 && role_u(c, caps, i, j) >= 2) AT(c, du, i, j) = AT(c, ou, i, j);
            if (comp == 1 && role_v(c, caps, i, j) >= 2) AT(c, dv, i, j) = AT(c, ov, i, j);
          }
      }
  free(eu); free(ev); free(ou); free(ov);
}

/* ------------------------------------------------------------------------------------------
 * Preconditioned conjugate gradients (Hestenes-Stiefel).  The paper only states that the
 * Poisson equation is solved iteratively and that, when the pressure is determined up to a
 * constant, the updates are projected onto zero-mean fields (end of Sec. 4.6).
 * Convergence: ||r||_2 <= tol * ||b||_2, checked before every iteration.
 * Preconditioners: Jacobi, or for the Poisson system the k-step Chebyshev iteration from
 * zero on the Jacobi-scaled operator over [lmax/30, lmax], lmax = 2 (Saad, Iterative
 * Methods for Sparse Linear Systems, Chebyshev acceleration).
 * ---------------------------------------------------------------------------------------- */

typedef void (*apply_fn)(const orc_case*, const double*, const double*, double*);

typedef struct {
  const orc_case* c;
  const double* caps;
  int system;            /* 0 Poisson (n = S), 1 Helmholtz (n = 2S, u then v) */
  const double* diag;    /* length n; zero marks positions outside the system */
  const double* mask;    /* zero-mean mask (active cells) or NULL */
  int precond;
  int cheb_degree;
} pcg_ctx;

static void op_apply(const pcg_ctx* k, const double* x, double* y) {
  size_t S = SIZE(k->c);
  if (k->system == 0) orc_poisson(k->c, k->caps, x, y);
  else orc_helmholtz(k->c, k->caps, x, x + S, y, y + S);
}

static size_t op_n(const pcg_ctx* k) { return (k->system == 0 ? 1 : 2) * SIZE(k->c); }

/* sum of a[i] * b[i] (b NULL: of a[i]) over the i with mask[i] != 0 (mask NULL: all), in
 * the fixed blocked order */
static double block_sum(const double* a, const double* b, const double* mask, size_t n) {
  size_t nb = (n + DOT_BLOCK - 1) / DOT_BLOCK;
  double* part = malloc((nb ? nb : 1) * sizeof(double));
  PAR_FOR
  for (size_t q = 0; q < nb; ++q) {
    size_t e = (q + 1) * DOT_BLOCK < n ? (q + 1) * DOT_BLOCK : n;
    double s = 0.0;
    for (size_t i = q * DOT_BLOCK; i < e; ++i)
      if (!mask || mask[i] != 0.0) s += b ? a[i] * b[i] : a[i];
    part[q] = s;
  }
  double s = 0.0;
  for (size_t q = 0; q < nb; ++q) s += part[q];
  free(part);
  return s;
}

static double dot(const double* a, const double* b, size_t n) { return block_sum(a, b, NULL, n); }

static void zero_mean(const pcg_ctx* k, double* x) {
  if (!k->mask) return;
  size_t n = op_n(k);
  double s = block_sum(x, NULL, k->mask, n), m = block_sum(k->mask, NULL, k->mask, n);
  if (m == 0.0) return;
  s /= m;
  PAR_FOR
  for (size_t i = 0; i < n; ++i) if (k->mask[i] != 0.0) x[i] -= s;
}

static void precondition(const pcg_ctx* k, const double* r, double* z, double* w1, double* w2, double* w3) {
  size_t n = op_n(k);
  if (k->precond == 0 || k->system != 0) {
    PAR_FOR
    for (size_t i = 0; i < n; ++i) z[i] = k->diag[i] != 0.0 ? r[i] / k->diag[i] : 0.0;
  } else {
    /* Chebyshev iteration for K z = r from z = 0, Jacobi-scaled, eigenvalue interval
     * [a, b] = [2/30, 2]; w1 = search increment d, w2 = residual, w3 = K z */
    double b = 2.0, a = b / 30.0;
    double theta = 0.5 * (b + a), delta = 0.5 * (b - a), sigma = theta / delta;
    double rho_prev = 1.0 / sigma;
    PAR_FOR
    for (size_t i = 0; i < n; ++i) {
      double s = k->diag[i] != 0.0 ? r[i] / k->diag[i] : 0.0;
      w1[i] = s / theta;
      z[i] = w1[i];
    }
    for (int it = 1; it < k->cheb_degree; ++it) {
      op_apply(k, z, w3);
      double rho = 1.0 / (2.0 * sigma - rho_prev);
      PAR_FOR
      for (size_t i = 0; i < n; ++i) {
        w2[i] = r[i] - w3[i];
        double s = k->diag[i] != 0.0 ? w2[i] / k->diag[i] : 0.0;
        w1[i] = rho * rho_prev * w1[i] + (2.0 * rho / delta) * s;
        z[i] += w1[i];
      }
      rho_prev = rho;
    }
  }
  zero_mean(k, z);
}

/* Solve A x = b; x holds the initial guess.  Returns 1 if converged. */
static int pcg(const pcg_ctx* k, const double* b, double* x, double tol, int max_iter, int* iters, double* relres) {
  size_t n = op_n(k);
  double* r = malloc(n * sizeof(double));
  double* z = malloc(n * sizeof(double));
  double* p = malloc(n * sizeof(double));
  double* q = malloc(n * sizeof(double));
  double* w1 = malloc(n * sizeof(double));
  double* w2 = malloc(n * sizeof(double));
  double* w3 = malloc(n * sizeof(double));
  double bn = sqrt(dot(b, b, n));
  int conv = 0, it = 0;
  *relres = 0.0;
  if (bn == 0.0) {
    memset(x, 0, n * sizeof(double));
    *iters = 0;
    free(r); free(z); free(p); free(q); free(w1); free(w2); free(w3);
    return 1;
  }
  zero_mean(k, x);
  op_apply(k, x, q);
  PAR_FOR
  for (size_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
  precondition(k, r, z, w1, w2, w3);
  memcpy(p, z, n * sizeof(double));
  double rz = dot(r, z, n);
  for (;;) {
    double rn = sqrt(dot(r, r, n));
    *relres = rn / bn;
    if (rn <= tol * bn) { conv = 1; break; }
    if (it >= max_iter) break;
    op_apply(k, p, q);
    double alpha = rz / dot(p, q, n);
    PAR_FOR
    for (size_t i = 0; i < n; ++i) {
      x[i] += alpha * p[i];
      r[i] -= alpha * q[i];
    }
    precondition(k, r, z, w1, w2, w3);
    double rz_new = dot(r, z, n);
    double beta = rz_new / rz;
    rz = rz_new;
    PAR_FOR
    for (size_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    ++it;
  }
  *iters = it;
  free(r); free(z); free(p); free(q); free(w1); free(w2); free(w3);
  return conv;
}

static int has_outflow(const orc_case* c) {
  for (int s = 0; s < 4; ++s) if (c->bc_type[s] == BC_OUT) return 1;
  return 0;
}

static void poisson_ctx(const orc_case* c, const double* caps, pcg_ctx* k, double* diag, double* mask) {
  size_t S = SIZE(c);
  orc_poisson_diag(c, caps, diag);
  for (int j = -1; j <= c->ny + 1; ++j)
    for (int i = -1; i <= c->nx + 1; ++i) {
      int act = cell_active(c, caps, i, j);
      int dom = i >= 0 && i < c->nx && j >= 0 && j < c->ny;
      if (!dom) AT(c, diag, i, j) = 0.0;
      AT(c, mask, i, j) = act ? 1.0 : 0.0;
    }
  (void)S;
  k->c = c; k->caps = caps; k->system = 0; k->diag = diag;
  k->mask = has_outflow(c) ? NULL : mask;
  k->precond = c->precond; k->cheb_degree = c->cheb_degree > 0 ? c->cheb_degree : 1;
}

/* Solve K Phi = rhs (active cells) with the case's preconditioner; phi is the warm start. */
int orc_solve_poisson(const orc_case* c, const double* caps, const double* rhs_in, double* phi, double tol,
                      int max_iter, int* iters, double* relres) {
  size_t S = SIZE(c);
  double* diag = malloc(S * sizeof(double));
  double* mask = malloc(S * sizeof(double));
  double* rhs = malloc(S * sizeof(double));
  pcg_ctx k;
  poisson_ctx(c, caps, &k, diag, mask);
  for (size_t i = 0; i < S; ++i) rhs[i] = mask[i] != 0.0 ? rhs_in[i] : 0.0;
  for (size_t i = 0; i < S; ++i) if (diag[i] == 0.0 || mask[i] == 0.0) phi[i] = 0.0;
  if (k.mask) {
    /* singular (all-Dirichlet velocity box): keep the right-hand side in the range */
    double s = 0.0, m = 0.0;
    for (size_t i = 0; i < S; ++i) if (mask[i] != 0.0) { s += rhs[i]; m += 1.0; }
    if (m > 0.0) for (size_t i = 0; i < S; ++i) if (mask[i] != 0.0) rhs[i] -= s / m;
  }
  int ok = pcg(&k, rhs, phi, tol, max_iter, iters, relres);
  free(diag); free(mask); free(rhs);
  return ok;
}

/* The Poisson PCG's preconditioner applied once, z = M^-1 r, with the case's choice (Jacobi,
 * or the k-step Chebyshev iteration over [2/30, 2] on the Jacobi-scaled operator); r and z
 * are padded cell arrays.  Exported so that tests can check it against its closed form. */
void orc_poisson_precondition(const orc_case* c, const double* caps, const double* r, double* z) {
  size_t S = SIZE(c);
  double* diag = malloc(S * sizeof(double));
  double* mask = malloc(S * sizeof(double));
  double* w = malloc(3 * S * sizeof(double));
  pcg_ctx k;
  poisson_ctx(c, caps, &k, diag, mask);
  precondition(&k, r, z, w, w + S, w + 2 * S);
  free(diag); free(mask); free(w);
}

int orc_solve_helmholtz(const orc_case* c, const double* caps, const double* rhs_u, const double* rhs_v,
                        double* xu, double* xv, double tol, int max_iter, int* iters, double* relres) {
  size_t S = SIZE(c);
  double* diag = malloc(2 * S * sizeof(double));
  double* b = malloc(2 * S * sizeof(double));
  double* x = malloc(2 * S * sizeof(double));
  orc_helmholtz_diag(c, caps, diag, diag + S);
  PAR_FOR
  for (int j = -1; j <= c->ny + 1; ++j)
    for (int i = -1; i <= c->nx + 1; ++i) {
      size_t k = (size_t)(j + 1) * PITCH(c) + (size_t)(i + 1);
      int ru = role_u(c, caps, i, j), rv = role_v(c, caps, i, j);
      b[k] = ru == 3 ? rhs_u[k] : 0.0;
      b[S + k] = rv == 3 ? rhs_v[k] : 0.0;
      x[k] = ru == 3 ? xu[k] : 0.0;
      x[S + k] = rv == 3 ? xv[k] : 0.0;
    }
  pcg_ctx kx;
  kx.c = c; kx.caps = caps; kx.system = 1; kx.diag = diag; kx.mask = NULL; kx.precond = 0; kx.cheb_degree = 1;
  int ok = pcg(&kx, b, x, tol, max_iter, iters, relres);
  memcpy(xu, x, S * sizeof(double));
  memcpy(xv, x + S, S * sizeof(double));
  free(diag); free(b); free(x);
  return ok;
}

/* ------------------------------------------------------------------------------------------
 * Diagnostics: discrete kinetic energy (Sec. 4.4, sum over faces of V_alpha U_alpha^2 / 2
 * over the velocity positions inside the box) and max |cont(U, 0)| over active cells.
 * ---------------------------------------------------------------------------------------- */

double orc_kinetic(const orc_case* c, const double* caps, const double* u, const double* v) {
  const double* Vu = CAP(c, caps, G_U, K_V);
  const double* Vv = CAP(c, caps, G_V, K_V);
  double k = 0.0;
  int iu = PER_X(c) ? c->nx - 1 : c->nx, jv = PER_Y(c) ? c->ny - 1 : c->ny;  /* last face of its own */
  for (int j = 0; j < c->ny; ++j)
    for (int i = 0; i <= iu; ++i) k += 0.5 * AT(c, Vu, i, j) * AT(c, u, i, j) * AT(c, u, i, j);
  for (int j = 0; j <= jv; ++j)
    for (int i = 0; i < c->nx; ++i) k += 0.5 * AT(c, Vv, i, j) * AT(c, v, i, j) * AT(c, v, i, j);
  return k;
}

static double max_div_d(const orc_case* c, const double* caps, const double* u, const double* v, const double* Dx,
                        const double* Dy) {
  size_t S = SIZE(c);
  double* d = malloc(S * sizeof(double));
  orc_cont(c, caps, u, v, Dx, Dy, d);
  double m = 0.0;
  for (int j = 0; j < c->ny; ++j)
    for (int i = 0; i < c->nx; ++i)
      if (cell_active(c, caps, i, j) && fabs(AT(c, d, i, j)) > m) m = fabs(AT(c, d, i, j));
  free(d);
  return m;
}

/* Conservation sums (the momentum and mass sums of the diagnostics): out[0] = sum of
 * cont(U, D) over the box cells (Eq. divergence; it telescopes to the net flux through the box
 * and the body), out[1] = sum of V^x u over the u-positions in the box, out[2] = sum of V^y v
 * over the v-positions (the discrete momentum per unit density), on the ranges of the kinetic
 * energy.  D may be NULL. */
void orc_conservation(const orc_case* c, const double* caps, const double* u, const double* v, const double* Dx,
                      const double* Dy, double* out) {
  const double* Vu = CAP(c, caps, G_U, K_V);
  const double* Vv = CAP(c, caps, G_V, K_V);
  size_t S = SIZE(c);
  double* d = malloc(S * sizeof(double));
  orc_cont(c, caps, u, v, Dx, Dy, d);
  double m = 0.0, px = 0.0, py = 0.0;
  for (int j = 0; j < c->ny; ++j)
    for (int i = 0; i < c->nx; ++i) m += AT(c, d, i, j);
  int iu = PER_X(c) ? c->nx - 1 : c->nx, jv = PER_Y(c) ? c->ny - 1 : c->ny;
  for (int j = 0; j < c->ny; ++j)
    for (int i = 0; i <= iu; ++i) px += AT(c, Vu, i, j) * AT(c, u, i, j);
  for (int j = 0; j <= jv; ++j)
    for (int i = 0; i < c->nx; ++i) py += AT(c, Vv, i, j) * AT(c, v, i, j);
  out[0] = m;
  out[1] = px;
  out[2] = py;
  free(d);
}

double orc_max_div(const orc_case* c, const double* caps, const double* u, const double* v) {
  return max_div_d(c, caps, u, v, NULL, NULL);
}

/* ------------------------------------------------------------------------------------------
 * Force on the body (the paper reports drag and lift, Sec. 5, but defines no discrete force).
 * Reading: the force the fluid exerts on the body is minus the body's share of the momentum
 * the pressure and viscous terms of Eq. pm_prediction give the fluid.  Summing pres_alpha(P)
 * and visc_alpha(2 mu S) over the velocity positions of the box and moving the difference
 * operators onto the capacities (summation by parts) leaves box-boundary fluxes plus terms in
 * the differences of A and B across cells, which vanish wherever the grid is uncut; those
 * terms are the body's share.  Per component, with F = (Fp_x, Fp_y, Fv_x, Fv_y):
 *   Fp_x = sum_cells P (A^x_left - A^x_right)        (= sum P n_x |Gamma| by Eq. approximate,
 *   Fp_y = sum_cells P (A^y_bottom - A^y_top)           the surface conservation law: the
 *                                                       normal pointing out of the fluid)
 *   Fv_x = -2 mu [ sum_cells S_xx (B^xx_left - B^xx_right) + sum_nodes S_xy (B^xy_below - B^xy_above) ]
 *   Fv_y = -2 mu [ sum_cells S_yy (B^yy_below - B^yy_above) + sum_nodes S_xy (B^yx_left - B^yx_right) ]
 * over p-cells i in [0,nx), j in [0,ny); the S_xy sums run over the nodes whose two u-faces
 * (i in [0,nx], j in [1,ny)) or two v-faces (i in [1,nx), j in [0,ny]) lie in the box.
 * S is the strain of Eqs. diag and offdiag with the body's Dirichlet data D (orc_body_force:
 * D = 0, a no-slip body).  The convective term has no share for a body whose D has no normal
 * component (no flux through the boundary).
 * ---------------------------------------------------------------------------------------- */
void orc_body_force_d(const orc_case* c, const double* caps, const double* u, const double* v, const double* p,
                      const double* Dx, const double* Dy, double* force) {
  const double* Ax = CAP(c, caps, G_P, K_AX);
  const double* Ay = CAP(c, caps, G_P, K_AY);
  const double* BxU = CAP(c, caps, G_U, K_BX);
  const double* ByU = CAP(c, caps, G_U, K_BY);
  const double* BxV = CAP(c, caps, G_V, K_BX);
  const double* ByV = CAP(c, caps, G_V, K_BY);
  size_t S = SIZE(c);
  double* sxx = malloc(S * sizeof(double));
  double* syy = malloc(S * sizeof(double));
  double* sxy = malloc(S * sizeof(double));
  orc_strain(c, caps, u, v, Dx, Dy, sxx, syy, sxy);
  double fpx = 0.0, fpy = 0.0, gx = 0.0, gy = 0.0;
  for (int j = 0; j < c->ny; ++j)
    for (int i = 0; i < c->nx; ++i) {
      fpx += AT(c, p, i, j) * (AT(c, Ax, i, j) - AT(c, Ax, i + 1, j));
      fpy += AT(c, p, i, j) * (AT(c, Ay, i, j) - AT(c, Ay, i, j + 1));
      gx += AT(c, sxx, i, j) * (AT(c, BxU, i, j) - AT(c, BxU, i + 1, j));
      gy += AT(c, syy, i, j) * (AT(c, ByV, i, j) - AT(c, ByV, i, j + 1));
    }
  for (int j = 1; j < c->ny; ++j)
    for (int i = 0; i <= c->nx; ++i) gx += AT(c, sxy, i, j) * (AT(c, ByU, i, j - 1) - AT(c, ByU, i, j));
  for (int j = 0; j <= c->ny; ++j)
    for (int i = 1; i < c->nx; ++i) gy += AT(c, sxy, i, j) * (AT(c, BxV, i - 1, j) - AT(c, BxV, i, j));
  force[0] = fpx;
  force[1] = fpy;
  force[2] = -2.0 * c->mu * gx;
  force[3] = -2.0 * c->mu * gy;
  free(sxx);
  free(syy);
  free(sxy);
}

void orc_body_force(const orc_case* c, const double* caps, const double* u, const double* v, const double* p,
                    double* force) {
  orc_body_force_d(c, caps, u, v, p, NULL, NULL, force);
}

/* ------------------------------------------------------------------------------------------
 * Initial velocity: u = bc_un[W] (the inflow speed) on every u-position whose control
 * volume holds fluid, v = 0; then the seeded perturbation (may be NULL) on the unknowns;
 * then the Dirichlet faces and ghosts.
 * ---------------------------------------------------------------------------------------- */

void orc_init_velocity(const orc_case* c, const double* caps, double u0, double v0, const double* pu,
                       const double* pv, double* u, double* v) {
  size_t S = SIZE(c);
  memset(u, 0, S * sizeof(double));
  memset(v, 0, S * sizeof(double));
  for (int j = -1; j <= c->ny + 1; ++j)
    for (int i = -1; i <= c->nx + 1; ++i) {
      int ru = role_u(c, caps, i, j), rv = role_v(c, caps, i, j);
      if (ru == 3) AT(c, u, i, j) = u0 + (pu ? AT(c, pu, i, j) : 0.0);
      if (rv == 3) AT(c, v, i, j) = v0 + (pv ? AT(c, pv, i, j) : 0.0);
    }
  fill_bc(c, u, v, 1.0);
}

/* ------------------------------------------------------------------------------------------
 * One PmII projection step (Sec. 4.6, Eqs. pm_prediction, pm_poisson, pm_projection,
 * pm_update), with the mass matrix and density placed as in the semi-discrete system
 * (Eq. semidiscrete):
 *   (rho/dt) M U* - visc(mu S_hom(U*)) = (rho/dt) M U^n - 3/2 rho conv^n + 1/2 rho conv^{n-1}
 *                                        - pres(P^{n-1/2}) + visc(mu S(U^n)) + visc(mu S_D)
 *   (dt/rho) cont(M^-1 pres Phi, 0) = cont(U*, D)      i.e.  K Phi = -(rho/dt) cont(U*, D)
 *   U^{n+1} = U* - (dt/rho) M^-1 pres(Phi)
 *   P^{n+1/2} = P^{n-1/2} + Phi - (dt mu / 2 rho) V^-1 cont(M^-1 pres Phi, 0)
 * where V, the volume that turns the volume-integrated Laplacian into a point value, is the
 * full cell's area by default (pressure_update = 0): dividing by the fluid volume V_p of a
 * small cut cell (pressure_update = 1) makes the correction an unbounded gain there and the
 * step unstable (the paper does not say which volume).
 * The first step uses conv^{-1} = conv^0; P^{-1/2} = 0; the body is fixed, the box boundary
 * data are steady.  orc_step is the no-slip body (D = 0) without body acceleration; orc_step_g
 * adds g, orc_step_gd a steady D and orc_step_gdt a D given at both time levels.
 * State arrays: u, v, p (P^{n-1/2}), phi (Phi^n, the warm start), cu, cv (conv^{n-1}).
 * `first` is 1 for the first step.  Intermediate results may be returned through
 * ustar/vstar and bdiv when not NULL.
 * ---------------------------------------------------------------------------------------- */

/* Right-hand side of Eq. pm_prediction on the velocity unknowns (u, v: U^n, ghosts filled
 * here; p: P^{n-1/2}; cu, cv: conv^{n-1}, replaced by conv^0 when first is set).  Returns
 * conv^n in cnu, cnv. */
/* The same with the body-force term rho V_alpha g_alpha of Eq. pm_prediction; gx at u-faces and
 * gy at v-faces (accelerations, padded layout) may be NULL (g = 0). */
/* The body velocity may change in time: D^n (Dxn, Dyn) enters conv^n and the explicit half
 * visc(mu S^n), S^n = strain(U^n, D^n); D^{n+1} (Dx1, Dy1) enters the implicit half through its
 * lifting, S* = strain(U*, D^{n+1}) (Sec. 4.6: the boundary data of U* are those of the next
 * time level).  conv^{n-1} (cu, cv) was formed in the previous step with D^{n-1}. */
void orc_predictor_rhs_gdt(const orc_case* c, const double* caps, double* u, double* v, const double* p,
                           const double* cu, const double* cv, int first, const double* gx, const double* gy,
                           const double* Dxn, const double* Dyn, const double* Dx1, const double* Dy1, double* ru,
                           double* rv, double* cnu, double* cnv) {
  size_t S = SIZE(c);
  double* gu = malloc(S * sizeof(double));
  double* gv = malloc(S * sizeof(double));
  double* vu = malloc(S * sizeof(double));
  double* vv = malloc(S * sizeof(double));
  double* lu = malloc(S * sizeof(double));
  double* lv = malloc(S * sizeof(double));
  const double* Vu = CAP(c, caps, G_U, K_V);
  const double* Vv = CAP(c, caps, G_V, K_V);
  double rho = c->rho, dt = c->dt, mu = c->mu;
  fill_bc(c, u, v, 1.0);
  conv_bc(c, caps, u, v, Dxn, Dyn, cnu, cnv);
  const double* pu = first ? cnu : cu;
  const double* pv = first ? cnv : cv;
  orc_pres_bc(c, caps, p, gu, gv);
  visc_bc(c, caps, u, v, Dxn, Dyn, vu, vv);
  /* lifting of the implicit half: visc(mu S(0, D^{n+1})) from the box boundary values and the
   * body's Dirichlet data of the next time level */
  {
    double* zu = calloc(S, sizeof(double));
    double* zv = calloc(S, sizeof(double));
    fill_bc(c, zu, zv, 1.0);
    visc_bc(c, caps, zu, zv, Dx1, Dy1, lu, lv);
    free(zu); free(zv);
  }
  PAR_FOR
  for (size_t k = 0; k < S; ++k) {
    ru[k] = (rho / dt) * Vu[k] * u[k] - 1.5 * rho * cnu[k] + 0.5 * rho * pu[k] - gu[k] + mu * vu[k] + mu * lu[k];
    rv[k] = (rho / dt) * Vv[k] * v[k] - 1.5 * rho * cnv[k] + 0.5 * rho * pv[k] - gv[k] + mu * vv[k] + mu * lv[k];
    if (gx) ru[k] += rho * Vu[k] * gx[k];
    if (gy) rv[k] += rho * Vv[k] * gy[k];
  }
  PAR_FOR
  for (int j = -1; j <= c->ny + 1; ++j)
    for (int i = -1; i <= c->nx + 1; ++i) {
      if (role_u(c, caps, i, j) != 3) AT(c, ru, i, j) = 0.0;
      if (role_v(c, caps, i, j) != 3) AT(c, rv, i, j) = 0.0;
    }
  free(gu); free(gv); free(vu); free(vv); free(lu); free(lv);
}

void orc_predictor_rhs_gd(const orc_case* c, const double* caps, double* u, double* v, const double* p,
                          const double* cu, const double* cv, int first, const double* gx, const double* gy,
                          const double* Dx, const double* Dy, double* ru, double* rv, double* cnu, double* cnv) {
  orc_predictor_rhs_gdt(c, caps, u, v, p, cu, cv, first, gx, gy, Dx, Dy, Dx, Dy, ru, rv, cnu, cnv);
}

void orc_predictor_rhs_g(const orc_case* c, const double* caps, double* u, double* v, const double* p,
                         const double* cu, const double* cv, int first, const double* gx, const double* gy,
                         double* ru, double* rv, double* cnu, double* cnv) {
  orc_predictor_rhs_gd(c, caps, u, v, p, cu, cv, first, gx, gy, NULL, NULL, ru, rv, cnu, cnv);
}

void orc_predictor_rhs(const orc_case* c, const double* caps, double* u, double* v, const double* p, const double* cu,
                       const double* cv, int first, double* ru, double* rv, double* cnu, double* cnv) {
  orc_predictor_rhs_gd(c, caps, u, v, p, cu, cv, first, NULL, NULL, NULL, NULL, ru, rv, cnu, cnv);
}

/* One PmII step with the body acceleration g (gx at u-faces, gy at v-faces; NULL: g = 0) and
 * the body's Dirichlet velocity D (per u-cell and per v-cell; NULL: no-slip, D = 0) in Eqs.
 * divergence, diag/offdiag (through visc) and convective, at two time levels: D^n (Dxn, Dyn)
 * in conv^n and S^n, D^{n+1} (Dx1, Dy1) in S*, on the faces of U* whose control volume holds
 * no fluid, in cont(U*, D^{n+1}) (Eq. pm_poisson) and in the reported max |cont(U^{n+1},
 * D^{n+1})|. */
int orc_step_gdt(const orc_case* c, const double* caps, double* u, double* v, double* p, double* phi, double* cu,
                 double* cv, int first, const double* gx, const double* gy, const double* Dxn, const double* Dyn,
                 const double* Dx1, const double* Dy1, double* ustar, double* vstar, double* bdiv, orc_stats* st) {
  size_t S = SIZE(c);
  double* cnu = malloc(S * sizeof(double));
  double* cnv = malloc(S * sizeof(double));
  double* gu = malloc(S * sizeof(double));
  double* gv = malloc(S * sizeof(double));
  double* ru = malloc(S * sizeof(double));
  double* rv = malloc(S * sizeof(double));
  double* xu = malloc(S * sizeof(double));
  double* xv = malloc(S * sizeof(double));
  double* b = malloc(S * sizeof(double));
  double* kp = malloc(S * sizeof(double));
  const double* Vu = CAP(c, caps, G_U, K_V);
  const double* Vv = CAP(c, caps, G_V, K_V);
  const double* Vp = CAP(c, caps, G_P, K_V);
  double rho = c->rho, dt = c->dt, mu = c->mu;

  orc_predictor_rhs_gdt(c, caps, u, v, p, cu, cv, first, gx, gy, Dxn, Dyn, Dx1, Dy1, ru, rv, cnu, cnv);
  for (size_t k = 0; k < S; ++k) {
    xu[k] = u[k];
    xv[k] = v[k];
  }
  int ok_h = orc_solve_helmholtz(c, caps, ru, rv, xu, xv, c->tol_h, c->max_iter_h, &st->iters_h, &st->res_h);
  /* U*: unknowns from the solve, Dirichlet faces keep their values, inactive faces (no fluid in
   * their control volume) the body's velocity D (0 for a no-slip body) */
  PAR_FOR
  for (int j = -1; j <= c->ny + 1; ++j)
    for (int i = -1; i <= c->nx + 1; ++i) {
      size_t k = (size_t)(j + 1) * PITCH(c) + (size_t)(i + 1);
      int r_u = role_u(c, caps, i, j), r_v = role_v(c, caps, i, j);
      if (r_u == 3) u[k] = xu[k]; else if (r_u == 2) u[k] = Dx1 ? Dx1[k] : 0.0;
      if (r_v == 3) v[k] = xv[k]; else if (r_v == 2) v[k] = Dy1 ? Dy1[k] : 0.0;
    }
  fill_bc(c, u, v, 1.0);
  if (ustar) memcpy(ustar, u, S * sizeof(double));
  if (vstar) memcpy(vstar, v, S * sizeof(double));
  orc_cont(c, caps, u, v, Dx1, Dy1, b);
  if (bdiv) memcpy(bdiv, b, S * sizeof(double));
  double* rhs = malloc(S * sizeof(double));
  for (size_t k = 0; k < S; ++k) rhs[k] = -(rho / dt) * b[k];
  int ok_p = orc_solve_poisson(c, caps, rhs, phi, c->tol_p, c->max_iter_p, &st->iters_p, &st->res_p);
  free(rhs);
  /* projection */
  orc_pres_bc(c, caps, phi, gu, gv);
  PAR_FOR
  for (size_t k = 0; k < S; ++k) {
    u[k] -= (dt / rho) * winv(c, Vu[k]) * gu[k];
    v[k] -= (dt / rho) * winv(c, Vv[k]) * gv[k];
  }
  fill_bc(c, u, v, 1.0);
  /* pressure update: -cont(M^-1 pres Phi, 0) = K Phi on active cells */
  orc_poisson(c, caps, phi, kp);
  PAR_FOR
  for (int j = 0; j < c->ny; ++j)
    for (int i = 0; i < c->nx; ++i)
      if (cell_active(c, caps, i, j)) {
        double iv = c->pressure_update == 0 ? 1.0 / cell_area(c, i, j)
                    : c->pressure_update == 1 ? winv(c, AT(c, Vp, i, j)) : 0.0;
        AT(c, p, i, j) += AT(c, phi, i, j) + (dt * mu / (2.0 * rho)) * iv * AT(c, kp, i, j);
      }
  memcpy(cu, cnu, S * sizeof(double));
  memcpy(cv, cnv, S * sizeof(double));
  st->conv_h = ok_h;
  st->conv_p = ok_p;
  st->max_div = max_div_d(c, caps, u, v, Dx1, Dy1);
  st->kinetic = orc_kinetic(c, caps, u, v);
  free(cnu); free(cnv); free(gu); free(gv);
  free(ru); free(rv); free(xu); free(xv); free(b); free(kp);
  return ok_h && ok_p;
}

/* The same with a steady body velocity D (both time levels the same). */
int orc_step_gd(const orc_case* c, const double* caps, double* u, double* v, double* p, double* phi, double* cu,
                double* cv, int first, const double* gx, const double* gy, const double* Dx, const double* Dy,
                double* ustar, double* vstar, double* bdiv, orc_stats* st) {
  return orc_step_gdt(c, caps, u, v, p, phi, cu, cv, first, gx, gy, Dx, Dy, Dx, Dy, ustar, vstar, bdiv, st);
}

int orc_step_g(const orc_case* c, const double* caps, double* u, double* v, double* p, double* phi, double* cu,
               double* cv, int first, const double* gx, const double* gy, double* ustar, double* vstar, double* bdiv,
               orc_stats* st) {
  return orc_step_gd(c, caps, u, v, p, phi, cu, cv, first, gx, gy, NULL, NULL, ustar, vstar, bdiv, st);
}

int orc_step(const orc_case* c, const double* caps, double* u, double* v, double* p, double* phi, double* cu,
             double* cv, int first, double* ustar, double* vstar, double* bdiv, orc_stats* st) {
  return orc_step_gd(c, caps, u, v, p, phi, cu, cv, first, NULL, NULL, NULL, NULL, ustar, vstar, bdiv, st);
}
