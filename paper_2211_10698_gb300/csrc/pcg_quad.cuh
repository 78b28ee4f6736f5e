// FP32 phases of the mixed-precision Poisson solve (Eq. pm_poisson, FP32 CG on the Jacobi-
// scaled system K~ = D^-1/2 K D^-1/2) on aligned quads of the padded arrays: padded indices
// k0 .. k0+3 with k0 a multiple of 4 (the pitch is a multiple of 32, so every row starts a
// quad).  A row's quads span its interior cells plus the ghost and padding slots beside them;
// those slots hold zero in every FP32 vector and stay zero (their inputs are zero and their
// row kind is the identity), so quads are processed whole.  Used by the single-case solve
// (pcg_mixed.cu) and the batched one (pcg_batch.cu).
#pragma once
#include "pcg_cheb.cuh"
#include "pcg_common.cuh"

namespace ccm {

__device__ __forceinline__ float4 ld4(const float* a, int k) { return *reinterpret_cast<const float4*>(a + k); }
__device__ __forceinline__ void st4(float* a, int k, float4 v) { *reinterpret_cast<float4*>(a + k) = v; }
// (float) (sig * a[k .. k+3]) for an FP64 array (k even: two 16-byte loads)
__device__ __forceinline__ float4 ld4_scaled(const double* a, int k, double sig) {
  const double2 lo = *reinterpret_cast<const double2*>(a + k);
  const double2 hi = *reinterpret_cast<const double2*>(a + k + 2);
  return make_float4((float)(sig * lo.x), (float)(sig * lo.y), (float)(sig * hi.x), (float)(sig * hi.y));
}
__device__ __forceinline__ float at(const float4& v, int m) { return m == 0 ? v.x : m == 1 ? v.y : m == 2 ? v.z : v.w; }
__device__ __forceinline__ void put(float4& v, int m, float x) {
  if (m == 0) v.x = x; else if (m == 1) v.y = x; else if (m == 2) v.z = x; else v.w = x;
}
__device__ __forceinline__ float4 axpy4(float a, const float4& x, const float4& y) {
  return make_float4(a * x.x + y.x, a * x.y + y.y, a * x.z + y.z, a * x.w + y.w);
}
__device__ __forceinline__ float dot4(const float4& a, const float4& b) {
  return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
}

// Quads of a grid: nq per row, row j starting at padded index (j+1) pitch (the ghost slot of
// i = -1); quad u of the row-major enumeration starts at k(u).
struct Quads {
  int nq, nquad, P;
  __device__ Quads(const Geom& g) : nq(g.nx / 4 + 1), nquad(g.ny * (g.nx / 4 + 1)), P(g.pitch) {}
  __device__ int k(int u) const {
    const int j = u / nq;
    return (j + 1) * P + 4 * (u - j * nq);
  }
};

struct QuadOpsF32 {
  const int8_t* kinds;
  const float* cus;
  const float* cvs;
  float ax, ay;
  int P;

  // Scaled face coefficients of the quad (W faces, E face of the last cell, S faces, N faces).
  // Only rows of kind 2 (cut) use them, so a quad without one loads none: on the uniform
  // part of the grid the stencil reads its vector and the kinds only.
  __device__ __forceinline__ void coefs(int k0, const char4& km, float4& cw, float& ce4, float4& cs, float4& cn) const {
    cw = cs = cn = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    ce4 = 0.0f;
    if (km.x == 2 || km.y == 2 || km.z == 2 || km.w == 2) {
      cw = ld4(cus, k0);
      cs = ld4(cvs, k0);
      cn = ld4(cvs, k0 + P);
      ce4 = cus[k0 + 4];
    }
  }
  // (K~ z) on the quad from z at the quad (zc), its W/E cells and S/N quads
  __device__ __forceinline__ float4 row(const char4& km, const float4& zc, float zw, float ze, const float4& zs,
                                        const float4& zq, const float4& cw, float ce4, const float4& cs,
                                        const float4& cn) const {
    float4 out;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int8_t kk = m == 0 ? km.x : m == 1 ? km.y : m == 2 ? km.z : km.w;
      const float c = at(zc, m);
      const float l = m == 0 ? zw : at(zc, m - 1);
      const float rr = m == 3 ? ze : at(zc, m + 1);
      const float sv = at(zs, m), nv = at(zq, m);
      const float ce = m == 3 ? ce4 : at(cw, m + 1);
      const float wu = c - ax * (l + rr) - ay * (sv + nv);
      const float wg = c - at(cw, m) * l - ce * rr - at(cs, m) * sv - at(cn, m) * nv;
      put(out, m, kk == 1 ? wu : (kk == 2 ? wg : c));
    }
    return out;
  }

  // vector update: p = r + be p, s = w + be s (or p, s as stored when keep), e += al p,
  // r -= al s
  __device__ __forceinline__ void update(float* p, float* r, const float* w, float* s, float* e, int k0, float al,
                                         float be, bool keep) const {
    const float4 pm = ld4(p, k0), rm = ld4(r, k0), wm = ld4(w, k0), sm = ld4(s, k0);
    float4 em = pm;
    if (e) em = ld4(e, k0);
    float4 pk = pm, sk = sm;
    if (!keep) {
      pk = axpy4(be, pm, rm);
      sk = axpy4(be, sm, wm);
      st4(p, k0, pk);
      st4(s, k0, sk);
    }
    if (e) st4(e, k0, axpy4(al, pk, em));
    st4(r, k0, axpy4(-al, sk, rm));
  }
  // e += al p on the quad (the correction's update, when it runs apart from phase A)
  __device__ __forceinline__ void add_e(float* e, const float* p, int k0, float al) const {
    st4(e, k0, axpy4(al, ld4(p, k0), ld4(e, k0)));
  }
  // the same update with the preconditioned residual u: p = u + be p, s = w + be s
  __device__ __forceinline__ void update_u(float* p, const float* u, float* r, const float* w, float* s, float* e,
                                           int k0, float al, float be, bool keep) const {
    const float4 pm = ld4(p, k0), um = ld4(u, k0), wm = ld4(w, k0), sm = ld4(s, k0), em = ld4(e, k0);
    const float4 rm = ld4(r, k0);
    float4 pk = pm, sk = sm;
    if (!keep) {
      pk = axpy4(be, pm, um);
      sk = axpy4(be, sm, wm);
      st4(p, k0, pk);
      st4(s, k0, sk);
    }
    st4(e, k0, axpy4(al, pk, em));
    st4(r, k0, axpy4(-al, sk, rm));
  }
  // w = K~ r on the quad and the sums (r, r), (w, r) into v.  With r64 given, r is first set
  // from sig * r64 (read the same way at the neighbours).  The vector loads are issued
  // together; cut quads then load their coefficients.
  __device__ __forceinline__ void stencil(float* r, float* w, const double* r64, double sig, int k0,
                                          float (&v)[2]) const {
    const char4 km = *reinterpret_cast<const char4*>(kinds + k0);
    float4 rc, rs, rq;
    float rw, re;
    if (r64) {
      rc = ld4_scaled(r64, k0, sig);
      rs = ld4_scaled(r64, k0 - P, sig);
      rq = ld4_scaled(r64, k0 + P, sig);
      rw = (float)(sig * r64[k0 - 1]);
      re = (float)(sig * r64[k0 + 4]);
    } else {
      rc = ld4(r, k0);
      rs = ld4(r, k0 - P);
      rq = ld4(r, k0 + P);
      rw = r[k0 - 1];
      re = r[k0 + 4];
    }
    float4 cw, cs, cn;
    float ce4;
    coefs(k0, km, cw, ce4, cs, cn);
    const float4 wq = row(km, rc, rw, re, rs, rq, cw, ce4, cs, cn);
    v[0] += dot4(rc, rc);
    v[1] += dot4(wq, rc);
    if (r64) st4(r, k0, rc);
    st4(w, k0, wq);
  }
  // K~ z on the quad (z at the quad returned in zc)
  __device__ __forceinline__ float4 apply(const float* z, int k0, float4& zc) const {
    const char4 km = *reinterpret_cast<const char4*>(kinds + k0);
    zc = ld4(z, k0);
    const float4 zs = ld4(z, k0 - P), zq = ld4(z, k0 + P);
    const float zw = z[k0 - 1], ze = z[k0 + 4];
    float4 cw, cs, cn;
    float ce4;
    coefs(k0, km, cw, ce4, cs, cn);
    return row(km, zc, zw, ze, zs, zq, cw, ce4, cs, cn);
  }
  // w = K~ u and the sums (r, u), (w, u), (r, r) into v
  __device__ __forceinline__ void apply_sums(const float* u, const float* r, float* w, int k0, float (&v)[3]) const {
    float4 uc;
    const float4 wq = apply(u, k0, uc);
    const float4 rq = ld4(r, k0);
    st4(w, k0, wq);
    v[0] += dot4(rq, uc);
    v[1] += dot4(wq, uc);
    v[2] += dot4(rq, rq);
  }
  // Chebyshev step 1 taken from r itself (z1 = d1 = ith r, not stored):
  // d2 = c1 d1 + c2 (r - K~ z1), z2 = z1 + d2 into d and zout
  __device__ __forceinline__ void cheb_first(const float* r, float* d, float* zout, int k0, float ith, float c1,
                                             float c2) const {
    float4 rc;
    const float4 kr = apply(r, k0, rc);
    float4 dn, zn;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const float z1 = ith * at(rc, m);
      const float dv = c1 * z1 + c2 * (at(rc, m) - ith * at(kr, m));
      put(dn, m, dv);
      put(zn, m, z1 + dv);
    }
    st4(d, k0, dn);
    st4(zout, k0, zn);
  }
  // Chebyshev step j >= 2: d = c1 d + c2 (r - K~ zin), zout = zin + d
  __device__ __forceinline__ void cheb_step(const float* zin, const float* r, float* d, float* zout, int k0, float c1,
                                            float c2) const {
    float4 zc;
    const float4 kz = apply(zin, k0, zc);
    const float4 rq = ld4(r, k0), dq = ld4(d, k0);
    const float4 dn = make_float4(c1 * dq.x + c2 * (rq.x - kz.x), c1 * dq.y + c2 * (rq.y - kz.y),
                                  c1 * dq.z + c2 * (rq.z - kz.z), c1 * dq.w + c2 * (rq.w - kz.w));
    st4(d, k0, dn);
    st4(zout, k0, make_float4(zc.x + dn.x, zc.y + dn.y, zc.z + dn.z, zc.w + dn.w));
  }
  // the direction after a replacement: p = u + be p, s = w + be s stored; returns (p, s) on
  // the quad
  __device__ __forceinline__ float form(float* p, const float* u, const float* w, float* s, int k0, float be) const {
    const float4 pm = ld4(p, k0), um = ld4(u, k0), wm = ld4(w, k0), sm = ld4(s, k0);
    const float4 pk = axpy4(be, pm, um);
    const float4 sk = axpy4(be, sm, wm);
    st4(p, k0, pk);
    st4(s, k0, sk);
    return dot4(pk, sk);
  }
};

// x += D^-1/2 e * isig on the quad (1/sqrt(d) is 0 on ghost and padding slots, so x changes on
// interior cells only); e = 0 when asked
__device__ __forceinline__ void quad_fold(double* x, const double* isd, float* e, int k0, double isig, bool clear) {
  const float4 em = ld4(e, k0);
  x[k0] += isd[k0] * (double)em.x * isig;
  x[k0 + 1] += isd[k0 + 1] * (double)em.y * isig;
  x[k0 + 2] += isd[k0 + 2] * (double)em.z * isig;
  x[k0 + 3] += isd[k0 + 3] * (double)em.w * isig;
  if (clear) st4(e, k0, make_float4(0.0f, 0.0f, 0.0f, 0.0f));
}

}  // namespace ccm
