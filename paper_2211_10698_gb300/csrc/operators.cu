// Operator kernels of libccm: coefficient derivation, box boundary fill, the discrete
// operators of Sec. 4 (cont, pres, conv, visc, the Helmholtz and Poisson operators of the
// projection step) and the explicit stages of one PmII step (Sec. 4.6).
//
// Kernels that touch staggered data run one thread per padded index (i, j) and handle
// the u-face, v-face and p-cell that carry that index.
#include "ccm_host.h"

namespace ccm {

#define PAD_IJ(g)                                                        \
  const int i = (int)(blockIdx.x * blockDim.x + threadIdx.x) - 1;       \
  const int j = (int)(blockIdx.y * blockDim.y + threadIdx.y) - 1;       \
  if (i > (g).nx + 1 || j > (g).ny + 1) return;                         \
  const size_t k = (g).idx(i, j);

dim3 pad_grid(const Geom& g, dim3 blk) { return dim3((g.nx + 3 + blk.x - 1) / blk.x, (g.ny + 3 + blk.y - 1) / blk.y); }
static const dim3 kBlk(64, 4);

__device__ __forceinline__ double inv_or_zero(double w, double eps) { return w > eps ? 1.0 / w : 0.0; }

// ---------------------------------------------------------------------------------------
// Coefficients derived from the capacities.
// ---------------------------------------------------------------------------------------
__global__ void k_derive1(Geom g, Bc bc, Phys ph, int literal, CapPtrs cp, CoefPtrs o) {
  PAD_IJ(g)
  const double eps = 1e-12 * g.hx * g.hy;
  // on a periodic axis face n is the image of face 0: not a position of its own, but its
  // Poisson coefficient couples cell n-1 with cell 0 (through the ghost image)
  const bool uimg = g.px && i == g.nx && j >= 0 && j < g.ny;
  const bool vimg = g.py && j == g.ny && i >= 0 && i < g.nx;
  const bool udom = i >= 0 && i <= g.nx && j >= 0 && j < g.ny && !uimg;
  const bool vdom = i >= 0 && i < g.nx && j >= 0 && j <= g.ny && !vimg;
  const bool udir = udom && ((i == 0 && bc.type[CCM_SIDE_W] == CCM_BC_DIRICHLET) ||
                             (i == g.nx && bc.type[CCM_SIDE_E] == CCM_BC_DIRICHLET));
  const bool vdir = vdom && ((j == 0 && bc.type[CCM_SIDE_S] == CCM_BC_DIRICHLET) ||
                             (j == g.ny && bc.type[CCM_SIDE_N] == CCM_BC_DIRICHLET));
  const double Vu = cp.a[cap_slot(1, CK_V)][k], Vv = cp.a[cap_slot(2, CK_V)][k];
  const int8_t ru = !udom ? R_GHOST : udir ? R_DIRICHLET : (Vu > eps ? R_UNKNOWN : R_INACTIVE);
  const int8_t rv = !vdom ? R_GHOST : vdir ? R_DIRICHLET : (Vv > eps ? R_UNKNOWN : R_INACTIVE);
  o.role_u[k] = ru;
  o.role_v[k] = rv;
  const double Ax = cp.a[cap_slot(0, CK_AX)][k], Ay = cp.a[cap_slot(0, CK_AY)][k];
  const double ivu = inv_or_zero(Vu, eps), ivv = inv_or_zero(Vv, eps);
  o.cu[k] = (ru == R_UNKNOWN || (uimg && Vu > eps)) ? Ax * Ax * ivu : 0.0;
  o.cv[k] = (rv == R_UNKNOWN || (vimg && Vv > eps)) ? Ay * Ay * ivv : 0.0;
  o.gfu[k] = ru == R_UNKNOWN ? (ph.dt / ph.rho) * Ax * ivu : 0.0;
  o.gfv[k] = rv == R_UNKNOWN ? (ph.dt / ph.rho) * Ay * ivv : 0.0;
  o.massu[k] = ru == R_UNKNOWN ? (ph.rho / ph.dt) * Vu : 0.0;
  o.massv[k] = rv == R_UNKNOWN ? (ph.rho / ph.dt) * Vv : 0.0;
  // 1/W^xx at p-cell (i, j) is the u-grid Wx at u-cell i+1; 1/W^yy likewise
  o.wxx[k] = (i + 1 <= g.nx + 1) ? inv_or_zero(cp.a[cap_slot(1, CK_WX)][g.idx(i + 1, j)], eps) : 0.0;
  o.wyy[k] = (j + 1 <= g.ny + 1) ? inv_or_zero(cp.a[cap_slot(2, CK_WY)][g.idx(i, j + 1)], eps) : 0.0;
  const double wxy = cp.a[cap_slot(1, CK_WY)][k], wyx = cp.a[cap_slot(2, CK_WX)][k];
  if (literal) {
    o.wxa[k] = 0.5 * inv_or_zero(wxy, eps);
    o.wxb[k] = 0.5 * inv_or_zero(wyx, eps);
  } else {
    const double wb = 0.5 * inv_or_zero(0.5 * (wxy + wyx), eps);
    o.wxa[k] = wb;
    o.wxb[k] = wb;
  }
}

__global__ void k_derive2(Geom g, Phys ph, int pupdate, CapPtrs cp, CoefPtrs o) {
  PAD_IJ(g)
  const bool dom = i >= 0 && i < g.nx && j >= 0 && j < g.ny;
  double s = 0.0;
  if (dom) s = o.cu[k] + o.cu[k + 1] + o.cv[k] + o.cv[k + g.pitch];
  const bool a = dom && s > 0.0;
  o.act[k] = a ? 1 : 0;
  o.invdk[k] = a ? 1.0 / s : (dom ? 1.0 : 0.0);
  o.diagk[k] = a ? s : (dom ? 1.0 : 0.0);
  const double eps = 1e-12 * g.hx * g.hy;
  const double Vp = cp.a[cap_slot(0, CK_V)][k];
  // volume that turns the volume-integrated Laplacian of Eq. pm_update into a point value
  const double iv = pupdate == 0 ? 1.0 / cell_area(g, i, j) : (pupdate == 1 ? inv_or_zero(Vp, eps) : 0.0);
  o.pfac[k] = a ? (ph.dt * ph.mu / (2.0 * ph.rho)) * iv : 0.0;
  o.cu32[k] = (float)o.cu[k];
  o.cv32[k] = (float)o.cv[k];
  o.invdk32[k] = (float)o.invdk[k];
  o.diagk32[k] = (float)o.diagk[k];
  // row kind for the PCG: uncut rows (all four faces full) use the uniform-grid constants
  int8_t kind = 0;
  if (a) {
    const double cx = g.hy / g.hx, cy = g.hx / g.hy, e = 1e-14;
    const bool full = fabs(o.cu[k] - cx) <= e * cx && fabs(o.cu[k + 1] - cx) <= e * cx &&
                      fabs(o.cv[k] - cy) <= e * cy && fabs(o.cv[k + g.pitch] - cy) <= e * cy;
    kind = full ? 1 : 2;
  }
  o.kind[k] = kind;
}

// ---------------------------------------------------------------------------------------
// Box boundary data: Dirichlet faces get scale * bc_un, ghosts the zero-gradient copy
// (outflow and normal components) or the reflection 2 scale bc_ut - interior (tangential
// components on Dirichlet sides).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void fill_bc_at(const Geom& g, const Bc& bc, double* u, double* v, double scale, int i,
                                           int j, size_t k) {
  const int nx = g.nx, ny = g.ny;
  const bool wd = bc.type[CCM_SIDE_W] == CCM_BC_DIRICHLET, ed = bc.type[CCM_SIDE_E] == CCM_BC_DIRICHLET;
  const bool sd = bc.type[CCM_SIDE_S] == CCM_BC_DIRICHLET, nd = bc.type[CCM_SIDE_N] == CCM_BC_DIRICHLET;
  auto uval = [&](int a, int b) {
    if (a == 0 && wd) return scale * bc.un[CCM_SIDE_W];
    if (a == nx && ed) return scale * bc.un[CCM_SIDE_E];
    return u[g.idx(a, b)];
  };
  auto vval = [&](int a, int b) {
    if (b == 0 && sd) return scale * bc.un[CCM_SIDE_S];
    if (b == ny && nd) return scale * bc.un[CCM_SIDE_N];
    return v[g.idx(a, b)];
  };
  // u
  if (j >= 0 && j < ny) {
    if ((i == 0 && wd) || (i == nx && ed)) u[k] = uval(i, j);
    else if (i == -1) u[k] = uval(0, j);
    else if (i == nx + 1) u[k] = uval(nx, j);
  } else if (i >= 0 && i <= nx) {
    if (j == -1) u[k] = sd ? 2.0 * scale * bc.ut[CCM_SIDE_S] - uval(i, 0) : uval(i, 0);
    else if (j == ny) u[k] = nd ? 2.0 * scale * bc.ut[CCM_SIDE_N] - uval(i, ny - 1) : uval(i, ny - 1);
  }
  // v
  if (i >= 0 && i < nx) {
    if ((j == 0 && sd) || (j == ny && nd)) v[k] = vval(i, j);
    else if (j == -1) v[k] = vval(i, 0);
    else if (j == ny + 1) v[k] = vval(i, ny);
  } else if (j >= 0 && j <= ny) {
    if (i == -1) v[k] = wd ? 2.0 * scale * bc.ut[CCM_SIDE_W] - vval(0, j) : vval(0, j);
    else if (i == nx) v[k] = ed ? 2.0 * scale * bc.ut[CCM_SIDE_E] - vval(nx - 1, j) : vval(nx - 1, j);
  }
}
__global__ void k_fill_bc(Geom g, Bc bc, double* u, double* v, double scale) {
  PAD_IJ(g)
  fill_bc_at(g, bc, u, v, scale, i, j, k);
}

// Periodic sides, after the box rules of the other sides: every position beyond a periodic
// side (and face n along it) takes the value of its image inside the box.  A source is never
// a target, so one launch suffices.
__global__ void k_wrap_faces(Geom g, double* u, double* v) {
  PAD_IJ(g)
  const int iu = g.px ? (i >= g.nx ? i - g.nx : (i < 0 ? i + g.nx : i)) : i;
  const int jc = g.wrap_j(j);
  if (u && (iu != i || jc != j)) u[k] = u[g.idx(iu, jc)];
  const int ic = g.wrap_i(i);
  const int jv = g.py ? (j >= g.ny ? j - g.ny : (j < 0 ? j + g.ny : j)) : j;
  if (v && (ic != i || jv != j)) v[k] = v[g.idx(ic, jv)];
}
__global__ void k_wrap_cells(Geom g, double* p) {
  PAD_IJ(g)
  const int ic = g.wrap_i(i), jc = g.wrap_j(j);
  if (ic != i || jc != j) p[k] = p[g.idx(ic, jc)];
}

// ---------------------------------------------------------------------------------------
// Operators (used by ccm_apply_op and by set-up).
// ---------------------------------------------------------------------------------------
__global__ void k_cont(Coefs c, Geom g, const double* u, const double* v, double* out) {
  PAD_IJ(g)
  const bool dom = i >= 0 && i < g.nx && j >= 0 && j < g.ny;
  out[k] = dom ? cont_cell(c, g, u, v, i, j) : 0.0;
}

// pres(P) on velocity unknowns; cells outside the box read as zero (their images on a
// periodic side).
__global__ void k_pres(Coefs c, Geom g, const double* p, double* ou, double* ov) {
  PAD_IJ(g)
  auto P = [&](int a, int b) {
    a = g.wrap_i(a);
    b = g.wrap_j(b);
    return (a >= 0 && a < g.nx && b >= 0 && b < g.ny) ? p[g.idx(a, b)] : 0.0;
  };
  ou[k] = c.role_u[k] == R_UNKNOWN ? c.ax[k] * (P(i, j) - P(i - 1, j)) : 0.0;
  ov[k] = c.role_v[k] == R_UNKNOWN ? c.ay[k] * (P(i, j) - P(i, j - 1)) : 0.0;
}

__global__ void k_conv(Coefs c, Geom g, FullView w, double* ou, double* ov) {
  PAD_IJ(g)
  ou[k] = c.role_u[k] == R_UNKNOWN ? conv_u(c, g, w, i, j) : 0.0;
  ov[k] = c.role_v[k] == R_UNKNOWN ? conv_v(c, g, w, i, j) : 0.0;
}

__global__ void k_visc(Coefs c, Geom g, Bc bc, FullView w, double* ou, double* ov) {
  PAD_IJ(g)
  ou[k] = c.role_u[k] == R_UNKNOWN ? visc_u(c, g, bc, w, i, j) : 0.0;
  ov[k] = c.role_v[k] == R_UNKNOWN ? visc_v(c, g, bc, w, i, j) : 0.0;
}

// Helmholtz operator (rho/dt) M U - mu visc(S_hom(U)); identity on inactive faces.
__global__ void k_helmholtz(Coefs c, Geom g, Bc bc, Phys ph, HomView w, double* ou, double* ov) {
  PAD_IJ(g)
  const int8_t ru = c.role_u[k], rv = c.role_v[k];
  ou[k] = ru == R_UNKNOWN ? c.massu[k] * w.u[k] - ph.mu * visc_u(c, g, bc, w, i, j) : (ru == R_INACTIVE ? w.u[k] : 0.0);
  ov[k] = rv == R_UNKNOWN ? c.massv[k] * w.v[k] - ph.mu * visc_v(c, g, bc, w, i, j) : (rv == R_INACTIVE ? w.v[k] : 0.0);
}

// Poisson operator K = -cont(M^-1 pres(.), 0); identity on inactive cells.  The input is
// read through a copy whose ghost ring is zero.
__global__ void k_poisson(Coefs c, Geom g, const double* x, double* out) {
  PAD_IJ(g)
  const bool dom = i >= 0 && i < g.nx && j >= 0 && j < g.ny;
  out[k] = dom ? poisson_row(c.cu, c.cv, c.act, g, x, k) : 0.0;
}

__global__ void k_copy_interior_cells(Geom g, const double* in, double* out) {
  PAD_IJ(g)
  const bool dom = i >= 0 && i < g.nx && j >= 0 && j < g.ny;
  out[k] = dom ? in[k] : 0.0;
}

// Probe vectors for diag(H): ones on the unknown and inactive positions of one component
// whose indices are congruent to (a, b) mod 3 (H couples positions at distance <= 1).
__global__ void k_probe_set(Coefs c, Geom g, int comp, int a, int b, double* eu, double* ev) {
  PAD_IJ(g)
  const bool col = ((i + 3) % 3 == a) && ((j + 3) % 3 == b);
  eu[k] = (comp == 0 && col && c.role_u[k] >= R_INACTIVE) ? 1.0 : 0.0;
  ev[k] = (comp == 1 && col && c.role_v[k] >= R_INACTIVE) ? 1.0 : 0.0;
}
__global__ void k_probe_get(Coefs c, Geom g, int comp, int a, int b, const double* ou, const double* ov, double* du,
                            double* dv) {
  PAD_IJ(g)
  const bool col = ((i + 3) % 3 == a) && ((j + 3) % 3 == b);
  if (comp == 0 && col && c.role_u[k] >= R_INACTIVE) du[k] = ou[k];
  if (comp == 1 && col && c.role_v[k] >= R_INACTIVE) dv[k] = ov[k];
}
// Coefficient extraction: after applying the operator to the unit vector of colour (a, b) of
// component comp, row (i, j) sees exactly one unit inside its 3x3 neighbourhood, at the offset
// (di, dj) with i + di = a, j + dj = b (mod 3); its response is the coefficient of that
// neighbour.  A response at an offset outside the row's pattern is flagged in *bad.
__global__ void k_probe_coef(Coefs c, Geom g, int comp, int a, int b, const double* ou, const double* ov,
                             HelmCoefPtrs h, int* bad) {
  PAD_IJ(g)
  auto off = [](int want, int at) {
    const int d = ((want - at) % 3 + 3) % 3;
    return d == 2 ? -1 : d;
  };
  const int di = off(a, i), dj = off(b, j);
  if (c.role_u[k] == R_UNKNOWN) {
    int slot = -1;
    if (comp == 0)
      slot = (di == 0 && dj == 0) ? 0 : (di == -1 && dj == 0) ? 1 : (di == 1 && dj == 0) ? 2
           : (di == 0 && dj == -1) ? 3 : (di == 0 && dj == 1) ? 4 : -1;
    else
      slot = (di == -1 && dj == 0) ? 5 : (di == 0 && dj == 0) ? 6 : (di == -1 && dj == 1) ? 7
           : (di == 0 && dj == 1) ? 8 : -1;
    if (slot >= 0) h.a[slot][k] = ou[k];
    else if (ou[k] != 0.0) atomicOr(bad, 1);
  }
  if (c.role_v[k] == R_UNKNOWN) {
    int slot = -1;
    if (comp == 1)
      slot = (di == 0 && dj == 0) ? 9 : (di == -1 && dj == 0) ? 10 : (di == 1 && dj == 0) ? 11
           : (di == 0 && dj == -1) ? 12 : (di == 0 && dj == 1) ? 13 : -1;
    else
      slot = (di == 0 && dj == -1) ? 14 : (di == 1 && dj == -1) ? 15 : (di == 0 && dj == 0) ? 16
           : (di == 1 && dj == 0) ? 17 : -1;
    if (slot >= 0) h.a[slot][k] = ov[k];
    else if (ov[k] != 0.0) atomicOr(bad, 1);
  }
}
__global__ void k_invert_diag(Geom g, const double* du, const double* dv, double* iu, double* iv) {
  PAD_IJ(g)
  iu[k] = du[k] != 0.0 ? 1.0 / du[k] : 0.0;
  iv[k] = dv[k] != 0.0 ? 1.0 / dv[k] : 0.0;
}

// ---------------------------------------------------------------------------------------
// Explicit stages of the PmII step (Eq. pm_prediction right-hand side, Eq. pm_poisson
// right-hand side, Eqs. pm_projection and pm_update).
// ---------------------------------------------------------------------------------------
// EXTRA: the case may have a body acceleration g or a body velocity D (their terms are compiled
// in only then, so the common case keeps the plain kernel's registers and instructions)
template <bool EXTRA>
__device__ __forceinline__ void predictor_rhs_at(const Coefs& c, const Geom& g, const Bc& bc, const Phys& ph,
                                                 const FullView& w, const double* p, const double* cpu,
                                                 const double* cpv, double* cnu, double* cnv, double* ru_, double* rv_,
                                                 int first, int i, int j, size_t k) {
  auto P = [&](int a, int b) {
    a = g.wrap_i(a);
    b = g.wrap_j(b);
    return (a >= 0 && a < g.nx && b >= 0 && b < g.ny) ? p[g.idx(a, b)] : 0.0;
  };
  if (c.role_u[k] == R_UNKNOWN) {
    double cn = conv_u(c, g, w, i, j);
    // conv(U, U, D, D): the face mean of h = cont(0, D) times (U + D)/2 (Eq. convective)
    // with D = f D0 the bracket is the steady one scaled by f (h) and f (D); f = 1 is exact
    if (EXTRA && c.hd)
      cn += 0.5 * (ph.dn * c.hd[k] + ph.dn * c.hd[k - 1]) * 0.5 * (w.u[k] + ph.dn * c.dx[k]);
    const double cp = first ? cn : cpu[k];
    const double gp = c.ax[k] * (P(i, j) - P(i - 1, j));
    const double vs = visc_u(c, g, bc, w, i, j);
    double r = c.massu[k] * w.u[k] - 1.5 * ph.rho * cn + 0.5 * ph.rho * cp - gp + ph.mu * vs + ph.mu * c.liftu[k];
    if (EXTRA && c.accx) r += c.massu[k] * ph.dt * c.accx[k];  // rho V g
    // visc(S(0, D)): explicit half (D^n) and the implicit half's lift (D^{n+1})
    if (EXTRA && c.viscdu) r += (ph.dn + ph.dn1) * ph.mu * c.viscdu[k];
    ru_[k] = r;
    cnu[k] = cn;
  } else {
    ru_[k] = 0.0;
    cnu[k] = 0.0;
  }
  if (c.role_v[k] == R_UNKNOWN) {
    double cn = conv_v(c, g, w, i, j);
    if (EXTRA && c.hd)
      cn += 0.5 * (ph.dn * c.hd[k] + ph.dn * c.hd[k - g.pitch]) * 0.5 * (w.v[k] + ph.dn * c.dy[k]);
    const double cp = first ? cn : cpv[k];
    const double gp = c.ay[k] * (P(i, j) - P(i, j - 1));
    const double vs = visc_v(c, g, bc, w, i, j);
    double r = c.massv[k] * w.v[k] - 1.5 * ph.rho * cn + 0.5 * ph.rho * cp - gp + ph.mu * vs + ph.mu * c.liftv[k];
    if (EXTRA && c.accy) r += c.massv[k] * ph.dt * c.accy[k];
    if (EXTRA && c.viscdv) r += (ph.dn + ph.dn1) * ph.mu * c.viscdv[k];
    rv_[k] = r;
    cnv[k] = cn;
  } else {
    rv_[k] = 0.0;
    cnv[k] = 0.0;
  }
}
template <bool EXTRA>
__global__ void k_predictor_rhs(Coefs c, Geom g, Bc bc, Phys ph, FullView w, const double* p, const double* cpu,
                                const double* cpv, double* cnu, double* cnv, double* ru_, double* rv_, int first) {
  PAD_IJ(g)
  predictor_rhs_at<EXTRA>(c, g, bc, ph, w, p, cpu, cpv, cnu, cnv, ru_, rv_, first, i, j, k);
}

// b = cont(U*, D^{n+1}) on cells; Poisson right-hand side -(rho/dt) b on active cells.
__device__ __forceinline__ void divergence_at(const Coefs& c, const Geom& g, const Phys& ph, const double* u,
                                              const double* v, double* b, double* rhs, int i, int j, size_t k) {
  const bool dom = i >= 0 && i < g.nx && j >= 0 && j < g.ny;
  const double d = dom ? cont_cell(c, g, u, v, i, j) + (c.hd ? ph.dn1 * c.hd[k] : 0.0) : 0.0;
  b[k] = d;
  rhs[k] = c.act[k] ? -(ph.rho / ph.dt) * d : 0.0;
}
__global__ void k_divergence(Coefs c, Geom g, Phys ph, const double* u, const double* v, double* b, double* rhs) {
  PAD_IJ(g)
  divergence_at(c, g, ph, u, v, b, rhs, i, j, k);
}

// U^{n+1} = U* - (dt/rho) M^-1 pres(Phi); P^{n+1/2} = P^{n-1/2} + Phi + (dt mu / 2 rho)
// V_p^-1 K Phi.  Phi's ghost ring is zero.
__device__ __forceinline__ void project_at(const Coefs& c, const Geom& g, const double* phi, double* u, double* v,
                                           double* p, int i, int j, size_t k) {
  if (c.role_u[k] == R_UNKNOWN) u[k] -= c.gfu[k] * (phi[k] - phi[k - 1]);
  if (c.role_v[k] == R_UNKNOWN) v[k] -= c.gfv[k] * (phi[k] - phi[k - g.pitch]);
  if (c.act[k]) p[k] += phi[k] + c.pfac[k] * poisson_row(c.cu, c.cv, c.act, g, phi, k);
}
__global__ void k_project(Coefs c, Geom g, const double* phi, double* u, double* v, double* p) {
  PAD_IJ(g)
  project_at(c, g, phi, u, v, p, i, j, k);
}

// ---------------------------------------------------------------------------------------
// The explicit stages for the cases of a batch, one launch per stage: the blocks of case c
// are starts[c] .. starts[c+1]-1 and tile its padded rows, pitch included, in rows of gx
// blocks (kBlk), so each thread runs the same per-point body as the single-case kernel.  The divergence stage
// also takes the copies U* of the predicted velocity (the whole padded arrays, pitch included,
// as the single-case step copies them).
// ---------------------------------------------------------------------------------------
template <int KIND, bool EXTRA = false>
__global__ void __launch_bounds__(256) k_stage_batch(const StageCase* __restrict__ cases,
                                                     const int* __restrict__ starts, int n) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (starts[mid] <= (int)blockIdx.x) lo = mid;
    else hi = mid - 1;
  }
  const StageCase& S = cases[lo];
  const int lb = (int)blockIdx.x - starts[lo];
  const int bx = lb % S.gx, by = lb / S.gx;
  const int i = bx * (int)blockDim.x + (int)threadIdx.x - 1;
  const int j = by * (int)blockDim.y + (int)threadIdx.y - 1;
  const Geom& g = S.g;
  if (j > g.ny + 1) return;
  const size_t k = g.idx(i, j);
  if (KIND == STAGE_DIVERGENCE && i <= g.pitch - 2) {
    S.ustar[k] = S.u[k];
    S.vstar[k] = S.v[k];
  }
  if (i > g.nx + 1) return;
  if (KIND == STAGE_FILL_BC) fill_bc_at(g, S.bc, S.u, S.v, 1.0, i, j, k);
  if (KIND == STAGE_PREDICT)
    predictor_rhs_at<EXTRA>(S.c, g, S.bc, S.ph, FullView{S.u, S.v, g}, S.p, S.cpu, S.cpv, S.cnu, S.cnv, S.ru, S.rv,
                            S.first, i, j, k);
  if (KIND == STAGE_DIVERGENCE) divergence_at(S.c, g, S.ph, S.u, S.v, S.div, S.rhs, i, j, k);
  if (KIND == STAGE_PROJECT) project_at(S.c, g, S.phi, S.u, S.v, S.p, i, j, k);
}

// Diagnostics: per-block max |cont(U, D)| over active cells, sum of V U^2 / 2 over velocity
// positions inside the box, a non-finite flag, and the conservation sums: cont(U, D) over the
// box cells (mass), V u and V v over the velocity positions inside the box (momentum).
__global__ void k_diagnostics(Coefs c, Geom g, const double* Vu, const double* Vv, const double* u, const double* v,
                              double fd, double* partials) {
  const int i = (int)(blockIdx.x * blockDim.x + threadIdx.x) - 1;
  const int j = (int)(blockIdx.y * blockDim.y + threadIdx.y) - 1;
  double dmax = 0.0, ke = 0.0, bad = 0.0, mass = 0.0, mx = 0.0, my = 0.0;
  if (i <= g.nx + 1 && j <= g.ny + 1) {
    const size_t k = g.idx(i, j);
    if (i >= 0 && i < g.nx && j >= 0 && j < g.ny) {
      const double d = cont_cell(c, g, u, v, i, j) + (c.hd ? fd * c.hd[k] : 0.0);
      mass = d;
      if (c.act[k]) dmax = fabs(d);
    }
    if (i >= 0 && i <= g.nx - g.px && j >= 0 && j < g.ny) {  // face nx of a periodic x is face 0
      ke += 0.5 * Vu[k] * u[k] * u[k];
      mx = Vu[k] * u[k];
      if (!isfinite(u[k])) bad = 1.0;
    }
    if (i >= 0 && i < g.nx && j >= 0 && j <= g.ny - g.py) {
      ke += 0.5 * Vv[k] * v[k] * v[k];
      my = Vv[k] * v[k];
      if (!isfinite(v[k])) bad = 1.0;
    }
  }
  __shared__ double sm[6][256];
  const int t = threadIdx.y * blockDim.x + threadIdx.x;
  sm[0][t] = dmax; sm[1][t] = ke; sm[2][t] = bad; sm[3][t] = mass; sm[4][t] = mx; sm[5][t] = my;
  __syncthreads();
  for (int s = (blockDim.x * blockDim.y) / 2; s > 0; s >>= 1) {
    if (t < s) {
      sm[0][t] = fmax(sm[0][t], sm[0][t + s]);
      sm[1][t] += sm[1][t + s];
      sm[2][t] = fmax(sm[2][t], sm[2][t + s]);
      sm[3][t] += sm[3][t + s];
      sm[4][t] += sm[4][t + s];
      sm[5][t] += sm[5][t + s];
    }
    __syncthreads();
  }
  if (t == 0) {
    const size_t b = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
    const size_t nb = (size_t)gridDim.x * gridDim.y;
    for (int q = 0; q < 6; ++q) partials[q * nb + b] = sm[q][0];
  }
}

// out = (max |cont|, kinetic energy, non-finite flag, mass, momentum x, momentum y)
__global__ void k_diagnostics_final(const double* partials, int nb, double* out) {
  __shared__ double sm[6][256];
  const int t = threadIdx.x;
  double m = 0.0, bad = 0.0, s[4] = {0.0, 0.0, 0.0, 0.0};
  for (int b = t; b < nb; b += blockDim.x) {
    m = fmax(m, partials[b]);
    s[0] += partials[nb + b];
    bad = fmax(bad, partials[2 * nb + b]);
    s[1] += partials[3 * (size_t)nb + b];
    s[2] += partials[4 * (size_t)nb + b];
    s[3] += partials[5 * (size_t)nb + b];
  }
  sm[0][t] = m; sm[1][t] = s[0]; sm[2][t] = bad; sm[3][t] = s[1]; sm[4][t] = s[2]; sm[5][t] = s[3];
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (t < st) {
      sm[0][t] = fmax(sm[0][t], sm[0][t + st]);
      sm[2][t] = fmax(sm[2][t], sm[2][t + st]);
      sm[1][t] += sm[1][t + st];
      sm[3][t] += sm[3][t + st];
      sm[4][t] += sm[4][t + st];
      sm[5][t] += sm[5][t + st];
    }
    __syncthreads();
  }
  if (t == 0)
    for (int q = 0; q < 6; ++q) out[q] = sm[q][0];
}

// Force of the fluid on the body: the body's share of the momentum that pres(P) and
// visc(2 mu S) give the fluid (the paper reports drag and lift, Sec. 5, without a discrete
// force).  Moving the differences of pres and visc onto the capacities (summation by parts)
// leaves, besides box-boundary fluxes, terms in the differences of A and B across cells, which
// vanish wherever the grid is uncut:
//   Fp_x = sum_cells P (A^x_left - A^x_right),  Fp_y = sum_cells P (A^y_bottom - A^y_top),
//   Fv_x = -2 mu [sum_cells S_xx (B^xx_left - B^xx_right) + sum_nodes S_xy (B^xy_below - B^xy_above)],
//   Fv_y = -2 mu [sum_cells S_yy (B^yy_below - B^yy_above) + sum_nodes S_xy (B^yx_left - B^yx_right)],
// cells i in [0,nx), j in [0,ny); the S_xy sums over the nodes whose two u-faces (i in [0,nx],
// j in [1,ny)) or two v-faces (i in [1,nx), j in [0,ny]) lie in the box.  One thread per
// (i, j) in [0,nx] x [0,ny] takes the cell and the node of that index; the strain is evaluated
// only where its B-difference is nonzero (0 * S adds nothing).  Per-block partials of the four
// sums (before the factor -2 mu), in a fixed tree order.
__global__ void k_body_force(Coefs c, Geom g, FullView w, const double* p, double fd, double* partials) {
  const int i = (int)(blockIdx.x * blockDim.x + threadIdx.x) - 1;
  const int j = (int)(blockIdx.y * blockDim.y + threadIdx.y) - 1;
  double f[4] = {0.0, 0.0, 0.0, 0.0};
  if (i >= 0 && j >= 0 && i <= g.nx && j <= g.ny) {
    const size_t k = g.idx(i, j);
    if (i < g.nx && j < g.ny) {
      const double pk = p[k];
      f[0] = pk * (c.ax[k] - c.ax[k + 1]);
      f[1] = pk * (c.ay[k] - c.ay[k + g.pitch]);
      const double dbx = c.bxx[k] - c.bxx[k + 1];
      if (dbx != 0.0) f[2] = (strain_xx(c, g, w, i, j) + (c.sxxd ? fd * c.sxxd[k] : 0.0)) * dbx;
      const double dby = c.byy[k] - c.byy[k + g.pitch];
      if (dby != 0.0) f[3] = (strain_yy(c, g, w, i, j) + (c.syyd ? fd * c.syyd[k] : 0.0)) * dby;
    }
    const double dnx = (j >= 1 && j < g.ny) ? c.bxy[k - g.pitch] - c.bxy[k] : 0.0;
    const double dny = (i >= 1 && i < g.nx) ? c.byx[k - 1] - c.byx[k] : 0.0;
    if (dnx != 0.0 || dny != 0.0) {
      const double sxy = strain_xy(c, g, w, i, j) + (c.sxyd ? fd * c.sxyd[k] : 0.0);
      f[2] += sxy * dnx;
      f[3] += sxy * dny;
    }
  }
  __shared__ double sm[4][256];
  const int t = threadIdx.y * blockDim.x + threadIdx.x;
#pragma unroll
  for (int q = 0; q < 4; ++q) sm[q][t] = f[q];
  __syncthreads();
  for (int s = (blockDim.x * blockDim.y) / 2; s > 0; s >>= 1) {
    if (t < s)
#pragma unroll
      for (int q = 0; q < 4; ++q) sm[q][t] += sm[q][t + s];
    __syncthreads();
  }
  if (t == 0) {
    const size_t b = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
    const size_t nb = (size_t)gridDim.x * gridDim.y;
#pragma unroll
    for (int q = 0; q < 4; ++q) partials[q * nb + b] = sm[q][0];
  }
}

// The four sums over the blocks in a fixed order; out = (Fp_x, Fp_y, Fv_x, Fv_y).
__global__ void k_body_force_final(const double* partials, int nb, double mu, double* out) {
  __shared__ double sm[4][256];
  const int t = threadIdx.x;
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (int b = t; b < nb; b += blockDim.x)
#pragma unroll
    for (int q = 0; q < 4; ++q) s[q] += partials[(size_t)q * nb + b];
#pragma unroll
  for (int q = 0; q < 4; ++q) sm[q][t] = s[q];
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (t < st)
#pragma unroll
      for (int q = 0; q < 4; ++q) sm[q][t] += sm[q][t + st];
    __syncthreads();
  }
  if (t == 0) {
    out[0] = sm[0][0];
    out[1] = sm[1][0];
    out[2] = -2.0 * mu * sm[2][0];
    out[3] = -2.0 * mu * sm[3][0];
  }
}

// ---------------------------------------------------------------------------------------
// Mixed-precision refinement of the Poisson solve: FP64 residual r = b - K x (stored to
// FP32 for the inner solve) with per-block sums of r.r and b.b, and x += d.
// ---------------------------------------------------------------------------------------
__global__ void k_residual64(Coefs c, Geom g, const double* x, const double* b, float* r32, double* partials) {
  const int i = (int)(blockIdx.x * blockDim.x + threadIdx.x) - 1;
  const int j = (int)(blockIdx.y * blockDim.y + threadIdx.y) - 1;
  double rr = 0.0, bb = 0.0;
  if (i <= g.nx + 1 && j <= g.ny + 1) {
    const size_t k = g.idx(i, j);
    float rk32 = 0.0f;
    if (c.act[k]) {
      const double rk = b[k] - poisson_row(c.cu, c.cv, c.act, g, x, k);
      rk32 = (float)rk;
      rr = rk * rk;
      bb = b[k] * b[k];
    }
    r32[k] = rk32;
  }
  __shared__ double sm[2][256];
  const int t = threadIdx.y * blockDim.x + threadIdx.x;
  sm[0][t] = rr;
  sm[1][t] = bb;
  __syncthreads();
  for (int s = (blockDim.x * blockDim.y) / 2; s > 0; s >>= 1) {
    if (t < s) { sm[0][t] += sm[0][t + s]; sm[1][t] += sm[1][t + s]; }
    __syncthreads();
  }
  if (t == 0) {
    const size_t bi = (size_t)blockIdx.y * gridDim.x + blockIdx.x, nb = (size_t)gridDim.x * gridDim.y;
    partials[bi] = sm[0][0];
    partials[nb + bi] = sm[1][0];
  }
}

__global__ void k_sum2(const double* partials, int nb, double* out) {
  __shared__ double sm[2][256];
  const int t = threadIdx.x;
  double a = 0.0, b = 0.0;
  for (int k = t; k < nb; k += blockDim.x) { a += partials[k]; b += partials[nb + k]; }
  sm[0][t] = a; sm[1][t] = b;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (t < s) { sm[0][t] += sm[0][t + s]; sm[1][t] += sm[1][t + s]; }
    __syncthreads();
  }
  if (t == 0) { out[0] = sm[0][0]; out[1] = sm[1][0]; }
}

__global__ void k_add_correction(Geom g, const int8_t* act, double* x, const float* d) {
  PAD_IJ(g)
  if (act[k]) x[k] += (double)d[k];
}

// ---------------------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------------------
void launch_residual64(const Coefs& c, const Geom& g, const double* x, const double* b, float* r32, double* partials,
                       double* out2, cudaStream_t st) {
  dim3 gr = pad_grid(g, kBlk);
  k_residual64<<<gr, kBlk, 0, st>>>(c, g, x, b, r32, partials);
  k_sum2<<<1, 256, 0, st>>>(partials, (int)(gr.x * gr.y), out2);
}
void launch_add_correction(const Geom& g, const int8_t* act, double* x, const float* d, cudaStream_t st) {
  k_add_correction<<<pad_grid(g, kBlk), kBlk, 0, st>>>(g, act, x, d);
}
void launch_derive(const Geom& g, const Bc& bc, const Phys& ph, int literal, int pupdate, const CapPtrs& cp,
                   const CoefPtrs& o, cudaStream_t st) {
  k_derive1<<<pad_grid(g, kBlk), kBlk, 0, st>>>(g, bc, ph, literal, cp, o);
  k_derive2<<<pad_grid(g, kBlk), kBlk, 0, st>>>(g, ph, pupdate, cp, o);
}
void launch_fill_bc(const Geom& g, const Bc& bc, double* u, double* v, double scale, cudaStream_t st) {
  k_fill_bc<<<pad_grid(g, kBlk), kBlk, 0, st>>>(g, bc, u, v, scale);
  if (g.px || g.py) k_wrap_faces<<<pad_grid(g, kBlk), kBlk, 0, st>>>(g, u, v);
}
void launch_wrap_cells(const Geom& g, double* p, cudaStream_t st) {
  if (g.px || g.py) k_wrap_cells<<<pad_grid(g, kBlk), kBlk, 0, st>>>(g, p);
}
void launch_cont(const Coefs& c, const Geom& g, const double* u, const double* v, double* out, cudaStream_t st) {
  k_cont<<<pad_grid(g, kBlk), kBlk, 0, st>>>(c, g, u, v, out);
}
void launch_pres(const Coefs& c, const Geom& g, const double* p, double* ou, double* ov, cudaStream_t st) {
  k_pres<<<pad_grid(g, kBlk), kBlk, 0, st>>>(c, g, p, ou, ov);
}
void launch_conv(const Coefs& c, const Geom& g, const double* u, const double* v, double* ou, double* ov,
                 cudaStream_t st) {
  k_conv<<<pad_grid(g, kBlk), kBlk, 0, st>>>(c, g, FullView{u, v, g}, ou, ov);
}
void launch_visc(const Coefs& c, const Geom& g, const Bc& bc, const double* u, const double* v, double* ou, double* ov,
                 cudaStream_t st) {
  k_visc<<<pad_grid(g, kBlk), kBlk, 0, st>>>(c, g, bc, FullView{u, v, g}, ou, ov);
}
void launch_helmholtz(const Coefs& c, const Geom& g, const Bc& bc, const Phys& ph, const double* u, const double* v,
                      double* ou, double* ov, cudaStream_t st) {
  HomView w{u, v, c.role_u, c.role_v, g, bc};
  k_helmholtz<<<pad_grid(g, kBlk), kBlk, 0, st>>>(c, g, bc, ph, w, ou, ov);
}
void launch_poisson(const Coefs& c, const Geom& g, const double* x, double* out, double* tmp, cudaStream_t st) {
  k_copy_interior_cells<<<pad_grid(g, kBlk), kBlk, 0, st>>>(g, x, tmp);
  if (g.px || g.py) k_wrap_cells<<<pad_grid(g, kBlk), kBlk, 0, st>>>(g, tmp);
  k_poisson<<<pad_grid(g, kBlk), kBlk, 0, st>>>(c, g, tmp, out);
}
void launch_helmholtz_diag(const Coefs& c, const Geom& g, const Bc& bc, const Phys& ph, double* eu, double* ev,
                           double* ou, double* ov, double* du, double* dv, double* iu, double* iv, cudaStream_t st) {
  cudaMemsetAsync(du, 0, g.count() * sizeof(double), st);
  cudaMemsetAsync(dv, 0, g.count() * sizeof(double), st);
  for (int comp = 0; comp < 2; ++comp)
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        k_probe_set<<<pad_grid(g, kBlk), kBlk, 0, st>>>(c, g, comp, a, b, eu, ev);
        launch_helmholtz(c, g, bc, ph, eu, ev, ou, ov, st);
        k_probe_get<<<pad_grid(g, kBlk), kBlk, 0, st>>>(c, g, comp, a, b, ou, ov, du, dv);
      }
  if (iu) k_invert_diag<<<pad_grid(g, kBlk), kBlk, 0, st>>>(g, du, dv, iu, iv);
}
void launch_helmholtz_coefs(const Coefs& c, const Geom& g, const Bc& bc, const Phys& ph, double* eu, double* ev,
                            double* ou, double* ov, const HelmCoefPtrs& h, int* bad, cudaStream_t st) {
  for (int q = 0; q < 18; ++q) cudaMemsetAsync(h.a[q], 0, g.count() * sizeof(double), st);
  cudaMemsetAsync(bad, 0, sizeof(int), st);
  for (int comp = 0; comp < 2; ++comp)
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        k_probe_set<<<pad_grid(g, kBlk), kBlk, 0, st>>>(c, g, comp, a, b, eu, ev);
        launch_helmholtz(c, g, bc, ph, eu, ev, ou, ov, st);
        k_probe_coef<<<pad_grid(g, kBlk), kBlk, 0, st>>>(c, g, comp, a, b, ou, ov, h, bad);
      }
}
void launch_predictor_rhs(const Coefs& c, const Geom& g, const Bc& bc, const Phys& ph, const double* u, const double* v,
                          const double* p, const double* cpu, const double* cpv, double* cnu, double* cnv, double* ru,
                          double* rv, int first, cudaStream_t st) {
  if (c.accx || c.viscdu || c.hd)
    k_predictor_rhs<true><<<pad_grid(g, kBlk), kBlk, 0, st>>>(c, g, bc, ph, FullView{u, v, g}, p, cpu, cpv, cnu, cnv,
                                                             ru, rv, first);
  else
    k_predictor_rhs<false><<<pad_grid(g, kBlk), kBlk, 0, st>>>(c, g, bc, ph, FullView{u, v, g}, p, cpu, cpv, cnu, cnv,
                                                              ru, rv, first);
}
void launch_divergence(const Coefs& c, const Geom& g, const Phys& ph, const double* u, const double* v, double* b,
                       double* rhs, cudaStream_t st) {
  k_divergence<<<pad_grid(g, kBlk), kBlk, 0, st>>>(c, g, ph, u, v, b, rhs);
}
void launch_project(const Coefs& c, const Geom& g, const double* phi, double* u, double* v, double* p,
                    cudaStream_t st) {
  k_project<<<pad_grid(g, kBlk), kBlk, 0, st>>>(c, g, phi, u, v, p);
}
int stage_case_blocks(const Geom& g, int* gx) {
  *gx = (g.pitch + (int)kBlk.x - 1) / (int)kBlk.x;
  return *gx * (int)((g.ny + 3 + kBlk.y - 1) / kBlk.y);
}
cudaError_t launch_stage_batch(int kind, const StageCase* dev_cases, const int* dev_starts, int n, int blocks,
                               cudaStream_t st, bool extra) {
  if (n <= 0 || blocks <= 0) return cudaSuccess;
  switch (kind) {
    case STAGE_FILL_BC: k_stage_batch<STAGE_FILL_BC><<<blocks, kBlk, 0, st>>>(dev_cases, dev_starts, n); break;
    case STAGE_PREDICT:
      if (extra) k_stage_batch<STAGE_PREDICT, true><<<blocks, kBlk, 0, st>>>(dev_cases, dev_starts, n);
      else k_stage_batch<STAGE_PREDICT, false><<<blocks, kBlk, 0, st>>>(dev_cases, dev_starts, n);
      break;
    case STAGE_DIVERGENCE: k_stage_batch<STAGE_DIVERGENCE><<<blocks, kBlk, 0, st>>>(dev_cases, dev_starts, n); break;
    case STAGE_PROJECT: k_stage_batch<STAGE_PROJECT><<<blocks, kBlk, 0, st>>>(dev_cases, dev_starts, n); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}
int body_force_partials(const Geom& g) {
  dim3 gr = pad_grid(g, kBlk);
  return 4 * (int)(gr.x * gr.y);
}
void launch_body_force(const Coefs& c, const Geom& g, const Phys& ph, const double* u, const double* v,
                       const double* p, double* partials, double* out, cudaStream_t st) {
  dim3 gr = pad_grid(g, kBlk);
  k_body_force<<<gr, kBlk, 0, st>>>(c, g, FullView{u, v, g}, p, ph.dn, partials);
  k_body_force_final<<<1, 256, 0, st>>>(partials, (int)(gr.x * gr.y), ph.mu, out);
}
int diagnostics_partials(const Geom& g) {
  dim3 gr = pad_grid(g, kBlk);
  return (int)(gr.x * gr.y);
}
void launch_diagnostics(const Coefs& c, const Geom& g, const double* Vu, const double* Vv, const double* u,
                        const double* v, double* partials, double* out, cudaStream_t st, double fd) {
  dim3 gr = pad_grid(g, kBlk);
  k_diagnostics<<<gr, kBlk, 0, st>>>(c, g, Vu, Vv, u, v, fd, partials);
  k_diagnostics_final<<<1, 256, 0, st>>>(partials, (int)(gr.x * gr.y), out);
}

}  // namespace ccm
