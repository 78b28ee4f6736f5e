// The body's Dirichlet velocity D in the step (the heterogeneous terms of Eqs. divergence,
// diag/offdiag and convective), for a steady D on a fixed body: every D-term is then constant
// in time and computed once, when D is set.
//
//   h      = cont(0, D) at cells: per direction, the difference of (mean of B over the face's
//            two cells - A) D across the cell minus the cell mean of (B-difference across
//            the face) D (Eq. divergence);
//   S_D    = strain(0, D): the same construction on the u- and v-grids' capacities (A and B
//            exchange roles, Eqs. diag and offdiag), divided by the strain's volume weights;
//   visc_D = visc(S_D) at the velocity unknowns, with the outflow rule of visc_u / visc_v.
//
// In the step, cont(U, D) = cont(U, 0) + h; visc(S(U, D)) = visc(S(U, 0)) + visc_D for both the
// explicit half and the implicit half's lift; conv(U, U, D, D) adds, at a face, the mean of h
// over the face's two cells times (U + D)/2 (Eq. convective: the bracket is the face mean of
// h, since difference and mean commute).  The D-terms whose stencil leaves the padded range are
// dropped, as for a body that stays two cells from the box.
#include "ccm_host.h"

namespace ccm {

namespace {

#define DT_IJ(g)                                                    \
  const int i = (int)(blockIdx.x * blockDim.x + threadIdx.x) - 1;   \
  const int j = (int)(blockIdx.y * blockDim.y + threadIdx.y) - 1;   \
  if (i > (g).nx + 1 || j > (g).ny + 1) return;                     \
  const size_t k = (g).idx(i, j);

__device__ __forceinline__ bool in_box_cell(const Geom& g, int i, int j) {
  return i >= 0 && i < g.nx && j >= 0 && j < g.ny;
}

// One heterogeneous term of Eq. divergence (or diag) along one direction: with the face
// values e_f = (mean B over the face's two cells - A_f) D_f and f_f = (B-difference across the
// face) D_f, the term at the cell between faces lo and hi is (e_hi - e_lo) - (f_hi + f_lo)/2.
__device__ __forceinline__ double het(double e_lo, double e_hi, double f_lo, double f_hi) {
  return (e_hi - e_lo) - 0.5 * (f_hi + f_lo);
}

__global__ void k_dterms_cells(Geom g, CapPtrs cp, Coefs c, const double* Dx, const double* Dy, double* hd,
                               double* sxxd, double* syyd) {
  DT_IJ(g)
  const size_t P = g.pitch;
  // h at box cells: p-grid A (faces) and B (cells)
  if (in_box_cell(g, i, j)) {
    const double* A = cp.a[cap_slot(0, CK_AX)];
    const double* B = cp.a[cap_slot(0, CK_BX)];
    auto ex = [&](size_t f) { return (0.5 * (B[f] + B[f - 1]) - A[f]) * Dx[f]; };
    auto fx = [&](size_t f) { return (B[f] - B[f - 1]) * Dx[f]; };
    const double* Ay = cp.a[cap_slot(0, CK_AY)];
    const double* By = cp.a[cap_slot(0, CK_BY)];
    auto ey = [&](size_t f) { return (0.5 * (By[f] + By[f - P]) - Ay[f]) * Dy[f]; };
    auto fy = [&](size_t f) { return (By[f] - By[f - P]) * Dy[f]; };
    hd[k] = het(ex(k), ex(k + 1), fx(k), fx(k + 1)) + het(ey(k), ey(k + P), fy(k), fy(k + P));
  } else {
    hd[k] = 0.0;
  }
  // S_xx at cells i in [-1, nx], j in [0, ny): the u-grid's A^xx sits at the edge between
  // u-cells (index f + 1 for the edge right of u-face f), B^xx at the u-faces
  double sx = 0.0;
  if (i >= -1 && i <= g.nx - 1 && j >= 0 && j < g.ny) {
    const double* A = cp.a[cap_slot(1, CK_AX)];
    const double* B = cp.a[cap_slot(1, CK_BX)];
    auto e = [&](size_t f) { return (0.5 * (A[f + 1] + A[f]) - B[f]) * Dx[f]; };
    auto f_ = [&](size_t f) { return (A[f + 1] - A[f]) * Dx[f]; };
    sx = het(e(k), e(k + 1), f_(k), f_(k + 1)) * c.wxx[k];
  }
  sxxd[k] = sx;
  double sy = 0.0;
  if (j >= -1 && j <= g.ny - 1 && i >= 0 && i < g.nx) {
    const double* A = cp.a[cap_slot(2, CK_AY)];
    const double* B = cp.a[cap_slot(2, CK_BY)];
    auto e = [&](size_t f) { return (0.5 * (A[f + P] + A[f]) - B[f]) * Dy[f]; };
    auto f_ = [&](size_t f) { return (A[f + P] - A[f]) * Dy[f]; };
    sy = het(e(k), e(k + P), f_(k), f_(k + P)) * c.wyy[k];
  }
  syyd[k] = sy;
}

// S_xy at nodes i in [0, nx], j in [0, ny]: the u part along y (u-grid A^xy at the u-cells'
// bottom edges, B^xy at the u-faces) and the v part along x (v-grid A^yx, B^yx), with the
// same weights as the homogeneous part.
__global__ void k_dterms_nodes(Geom g, CapPtrs cp, Coefs c, const double* Dx, const double* Dy, double* sxyd) {
  DT_IJ(g)
  const size_t P = g.pitch;
  double s = 0.0;
  if (i >= 0 && i <= g.nx && j >= 0 && j <= g.ny) {
    const double* Au = cp.a[cap_slot(1, CK_AY)];
    const double* Bu = cp.a[cap_slot(1, CK_BY)];
    auto eu = [&](size_t f) { return (0.5 * (Au[f + P] + Au[f]) - Bu[f]) * Dx[f]; };
    auto fu = [&](size_t f) { return (Au[f + P] - Au[f]) * Dx[f]; };
    const double* Av = cp.a[cap_slot(2, CK_AX)];
    const double* Bv = cp.a[cap_slot(2, CK_BX)];
    auto ev = [&](size_t f) { return (0.5 * (Av[f + 1] + Av[f]) - Bv[f]) * Dy[f]; };
    auto fv = [&](size_t f) { return (Av[f + 1] - Av[f]) * Dy[f]; };
    const double gu = het(eu(k - P), eu(k), fu(k - P), fu(k));
    const double gv = het(ev(k - 1), ev(k), fv(k - 1), fv(k));
    s = gu * c.wxa[k] + gv * c.wxb[k];
  }
  sxyd[k] = s;
}

// visc(S_D) at the velocity unknowns (zero elsewhere), with the outflow rule.
__global__ void k_dterms_visc(Geom g, Bc bc, Coefs c, const double* sxxd, const double* syyd, const double* sxyd,
                              double* vu, double* vv) {
  DT_IJ(g)
  const size_t P = g.pitch;
  double a = 0.0, b = 0.0;
  if (c.role_u[k] == R_UNKNOWN) {
    const double top = (j == g.ny - 1 && bc.type[CCM_SIDE_N] == CCM_BC_OUTFLOW) ? 0.0 : sxyd[k + P];
    const double bot = (j == 0 && bc.type[CCM_SIDE_S] == CCM_BC_OUTFLOW) ? 0.0 : sxyd[k];
    a = c.bxx[k] * (sxxd[k] - sxxd[k - 1]) + c.bxy[k] * (top - bot);
  }
  if (c.role_v[k] == R_UNKNOWN) {
    const double rgt = (i == g.nx - 1 && bc.type[CCM_SIDE_E] == CCM_BC_OUTFLOW) ? 0.0 : sxyd[k + 1];
    const double lft = (i == 0 && bc.type[CCM_SIDE_W] == CCM_BC_OUTFLOW) ? 0.0 : sxyd[k];
    b = c.byy[k] * (syyd[k] - syyd[k - P]) + c.byx[k] * (rgt - lft);
  }
  vu[k] = a;
  vv[k] = b;
}

// Faces whose control volume holds no fluid carry the body's velocity f D0.
__global__ void k_inactive_to_body(Geom g, const int8_t* ru, const int8_t* rv, const double* Dx, const double* Dy,
                                   double f, double* u, double* v) {
  DT_IJ(g)
  if (ru[k] == R_INACTIVE) u[k] = Dx ? f * Dx[k] : 0.0;
  if (rv[k] == R_INACTIVE) v[k] = Dy ? f * Dy[k] : 0.0;
}

}  // namespace

void launch_body_dterms(const Geom& g, const Bc& bc, const CapPtrs& cp, const Coefs& c, const double* Dx,
                        const double* Dy, double* hd, double* sxxd, double* syyd, double* sxyd, double* vu,
                        double* vv, cudaStream_t st) {
  const dim3 b(64, 4);
  const dim3 gr((g.nx + 3 + b.x - 1) / b.x, (g.ny + 3 + b.y - 1) / b.y);
  k_dterms_cells<<<gr, b, 0, st>>>(g, cp, c, Dx, Dy, hd, sxxd, syyd);
  k_dterms_nodes<<<gr, b, 0, st>>>(g, cp, c, Dx, Dy, sxyd);
  k_dterms_visc<<<gr, b, 0, st>>>(g, bc, c, sxxd, syyd, sxyd, vu, vv);
}

void launch_inactive_to_body(const Geom& g, const int8_t* ru, const int8_t* rv, const double* Dx, const double* Dy,
                             double* u, double* v, cudaStream_t st, double f) {
  const dim3 b(64, 4);
  const dim3 gr((g.nx + 3 + b.x - 1) / b.x, (g.ny + 3 + b.y - 1) / b.y);
  k_inactive_to_body<<<gr, b, 0, st>>>(g, ru, rv, Dx, Dy, f, u, v);
}

}  // namespace ccm
