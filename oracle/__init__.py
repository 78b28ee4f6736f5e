"""FP64 CPU oracle for the cut-cell MAC projection step (arXiv 2211.10698).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference legs of ``bench.py`` may import this package.  It wraps ``ccm_oracle.c`` (plain C,
FP64, optional OpenMP loops, no code shared with the CUDA library) through ctypes and adds numpy
helpers that build dense matrices by applying the oracle's operators to unit vectors.

Every array is a padded ``(ny + 3, nx + 3)`` float64 array (see
``paper_2211_10698_gb300.inputs`` for the index convention).

Parity status: every function here is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` (closed forms, the paper's worked example, identities of the
discrete calculus, brute-force dense solves); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
from ctypes import POINTER, c_double, c_int, c_size_t

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ccm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, so x86 and Arm agree), with OpenMP for
    its cell loops when the compiler has it (the results do not depend on the thread count)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
        if r.returncode != 0:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


def set_threads(n: int = 0) -> int:
    """Threads for the oracle's parallel loops (0: all of this machine's); returns the count in
    use (1 when built without OpenMP)."""
    return int(_load().orc_set_threads(int(n)))


class OrcCase(ctypes.Structure):
    _fields_ = [("nx", c_int), ("ny", c_int),
                ("x0", c_double), ("y0", c_double), ("hx", c_double), ("hy", c_double),
                ("rho", c_double), ("mu", c_double), ("dt", c_double),
                ("bc_type", c_int * 4), ("bc_un", c_double * 4), ("bc_ut", c_double * 4),
                ("geom_kind", c_int), ("cx", c_double), ("cy", c_double), ("r", c_double),
                ("naca_tt", c_int), ("closed_te", c_int),
                ("chord", c_double), ("aoa_deg", c_double), ("le_x", c_double), ("le_y", c_double),
                ("hp_nx", c_double), ("hp_ny", c_double), ("hp_off", c_double),
                ("literal_offdiag", c_int), ("pressure_update", c_int), ("precond", c_int), ("cheb_degree", c_int),
                ("tol_p", c_double), ("tol_h", c_double),
                ("max_iter_p", c_int), ("max_iter_h", c_int),
                ("xf", POINTER(c_double)), ("yf", POINTER(c_double))]


class OrcStats(ctypes.Structure):
    _fields_ = [("iters_h", c_int), ("iters_p", c_int), ("res_h", c_double), ("res_p", c_double),
                ("max_div", c_double), ("kinetic", c_double), ("conv_h", c_int), ("conv_p", c_int)]


_lib = None
_DP = POINTER(c_double)


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        cp = POINTER(OrcCase)
        ip = POINTER(c_int)
        sig = {
            "orc_size": (c_size_t, [cp]),
            "orc_capacities": (None, [cp, _DP]),
            "orc_cell_boundary": (None, [cp, c_int, c_int, c_int, _DP, _DP]),
            "orc_cont": (None, [cp, _DP, _DP, _DP, _DP, _DP, _DP]),
            "orc_pres": (None, [cp, _DP, _DP, _DP, _DP]),
            "orc_strain": (None, [cp, _DP, _DP, _DP, _DP, _DP, _DP, _DP, _DP]),
            "orc_visc": (None, [cp, _DP, _DP, _DP, _DP, _DP, _DP]),
            "orc_conv": (None, [cp, _DP, _DP, _DP, _DP, _DP, _DP, _DP, _DP, _DP, _DP, _DP]),
            "orc_fill_ghosts": (None, [cp, _DP, _DP]),
            "orc_visc_bc": (None, [cp, _DP, _DP, _DP, _DP, _DP]),
            "orc_conv_bc": (None, [cp, _DP, _DP, _DP, _DP, _DP]),
            "orc_pres_bc": (None, [cp, _DP, _DP, _DP, _DP]),
            "orc_helmholtz": (None, [cp, _DP, _DP, _DP, _DP, _DP]),
            "orc_poisson": (None, [cp, _DP, _DP, _DP]),
            "orc_poisson_diag": (None, [cp, _DP, _DP]),
            "orc_helmholtz_diag": (None, [cp, _DP, _DP, _DP]),
            "orc_solve_poisson": (c_int, [cp, _DP, _DP, _DP, c_double, c_int, ip, _DP]),
            "orc_solve_helmholtz": (c_int, [cp, _DP, _DP, _DP, _DP, _DP, c_double, c_int, ip, _DP]),
            "orc_kinetic": (c_double, [cp, _DP, _DP, _DP]),
            "orc_max_div": (c_double, [cp, _DP, _DP, _DP]),
            "orc_body_force": (None, [cp, _DP, _DP, _DP, _DP, _DP]),
            "orc_init_velocity": (None, [cp, _DP, c_double, c_double, _DP, _DP, _DP, _DP]),
            "orc_step": (c_int, [cp, _DP, _DP, _DP, _DP, _DP, _DP, _DP, c_int, _DP, _DP, _DP,
                                 POINTER(OrcStats)]),
            "orc_roles": (None, [cp, _DP, ip, ip, ip]),
            "orc_predictor_rhs": (None, [cp, _DP, _DP, _DP, _DP, _DP, _DP, c_int, _DP, _DP, _DP, _DP]),
            "orc_predictor_rhs_g": (None, [cp, _DP, _DP, _DP, _DP, _DP, _DP, c_int, _DP, _DP, _DP, _DP, _DP,
                                           _DP]),
            "orc_step_g": (c_int, [cp, _DP, _DP, _DP, _DP, _DP, _DP, _DP, c_int, _DP, _DP, _DP, _DP, _DP,
                                   POINTER(OrcStats)]),
            "orc_step_gd": (c_int, [cp, _DP, _DP, _DP, _DP, _DP, _DP, _DP, c_int, _DP, _DP, _DP, _DP, _DP, _DP, _DP,
                                    POINTER(OrcStats)]),
            "orc_step_gdt": (c_int, [cp, _DP, _DP, _DP, _DP, _DP, _DP, _DP, c_int, _DP, _DP, _DP, _DP, _DP, _DP,
                                     _DP, _DP, _DP, POINTER(OrcStats)]),
            "orc_body_force_d": (None, [cp, _DP, _DP, _DP, _DP, _DP, _DP, _DP]),
            "orc_conservation": (None, [cp, _DP, _DP, _DP, _DP, _DP, _DP]),
            "orc_poisson_precondition": (None, [cp, _DP, _DP, _DP]),
            "orc_set_threads": (c_int, [c_int]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], "oracle arrays are C-contiguous float64"
    return a.ctypes.data_as(_DP)


def case_struct(case, precond=None) -> OrcCase:
    g = case.geom
    s = OrcCase()
    s.nx, s.ny = case.nx, case.ny
    s.x0, s.y0 = case.x0, case.y0
    s.hx, s.hy = case.hx, case.hy
    s.rho, s.mu, s.dt = case.rho, case.mu, case.dt
    for k in range(4):
        s.bc_type[k] = int(case.bc_type[k])
        s.bc_un[k] = float(case.bc_un[k])
        s.bc_ut[k] = float(case.bc_ut[k])
    s.geom_kind = g.kind
    s.cx, s.cy, s.r = g.cx, g.cy, g.r
    s.naca_tt, s.closed_te = g.naca_tt, g.closed_te
    s.chord, s.aoa_deg, s.le_x, s.le_y = g.chord, g.aoa_deg, g.le_x, g.le_y
    s.hp_nx, s.hp_ny, s.hp_off = g.hp_nx, g.hp_ny, g.hp_off
    s.literal_offdiag = int(case.literal_offdiag)
    s.pressure_update = int(case.pressure_update)
    pc = precond if precond is not None else case.precond
    s.precond = 1 if pc == "chebyshev" else 0
    s.cheb_degree = case.cheb_degree
    s.tol_p, s.tol_h = case.tol_p, case.tol_h
    s.max_iter_p, s.max_iter_h = case.max_iter_p, case.max_iter_h
    # stretched mesh: face abscissas (the arrays are kept alive by the caller, see Oracle)
    s.xf = _p(case.faces_x()) if case.stretched else None
    s.yf = _p(case.faces_y()) if case.stretched else None
    return s


CAP_NAMES = ("V", "X", "Y", "AX", "AY", "WX", "WY", "BX", "BY")
GRIDS = ("p", "u", "v")


class Oracle:
    """The oracle bound to one case; capacities are computed at construction."""

    def __init__(self, case, precond=None):
        self.lib = _load()
        self.case = case
        self._faces = (case.faces_x(), case.faces_y()) if case.stretched else None
        self.s = case_struct(case, precond)
        if self._faces is not None:
            self.s.xf, self.s.yf = _p(self._faces[0]), _p(self._faces[1])
        self.shape = case.shape
        self.S = case.shape[0] * case.shape[1]
        self.caps = np.zeros((3, 9) + self.shape)
        self.lib.orc_capacities(ctypes.byref(self.s), _p(self.caps))
        ru = np.zeros(self.shape, dtype=np.int32)
        rv = np.zeros(self.shape, dtype=np.int32)
        act = np.zeros(self.shape, dtype=np.int32)
        ip = POINTER(c_int)
        self.lib.orc_roles(ctypes.byref(self.s), _p(self.caps), ru.ctypes.data_as(ip),
                           rv.ctypes.data_as(ip), act.ctypes.data_as(ip))
        self.role_u, self.role_v, self.active = ru, rv, act.astype(bool)

    # -- helpers ---------------------------------------------------------------------------
    def z(self):
        return np.zeros(self.shape)

    def cap(self, grid: str, name: str) -> np.ndarray:
        return self.caps[GRIDS.index(grid), CAP_NAMES.index(name)]

    def at(self, a, i, j):
        return a[j + 1, i + 1]

    def _c(self, a):
        return None if a is None else np.ascontiguousarray(a, dtype=np.float64)

    # -- raw operators ---------------------------------------------------------------------
    def cont(self, u, v, Dx=None, Dy=None):
        o = self.z()
        u, v, Dx, Dy = map(self._c, (u, v, Dx, Dy))
        self.lib.orc_cont(ctypes.byref(self.s), _p(self.caps), _p(u), _p(v), _p(Dx), _p(Dy), _p(o))
        return o

    def pres(self, p):
        ou, ov = self.z(), self.z()
        self.lib.orc_pres(ctypes.byref(self.s), _p(self.caps), _p(self._c(p)), _p(ou), _p(ov))
        return ou, ov

    def strain(self, u, v, Dx=None, Dy=None):
        a, b, c = self.z(), self.z(), self.z()
        u, v, Dx, Dy = map(self._c, (u, v, Dx, Dy))
        self.lib.orc_strain(ctypes.byref(self.s), _p(self.caps), _p(u), _p(v), _p(Dx), _p(Dy),
                            _p(a), _p(b), _p(c))
        return a, b, c

    def visc(self, sxx, syy, sxy):
        ou, ov = self.z(), self.z()
        sxx, syy, sxy = map(self._c, (sxx, syy, sxy))
        self.lib.orc_visc(ctypes.byref(self.s), _p(self.caps), _p(sxx), _p(syy), _p(sxy), _p(ou), _p(ov))
        return ou, ov

    def conv(self, u, v, ut=None, vt=None, Dx=None, Dy=None, Dxt=None, Dyt=None):
        ut = u if ut is None else ut
        vt = v if vt is None else vt
        ou, ov = self.z(), self.z()
        args = list(map(self._c, (u, v, ut, vt, Dx, Dy, Dxt, Dyt)))
        self.lib.orc_conv(ctypes.byref(self.s), _p(self.caps), *[_p(a) for a in args], _p(ou), _p(ov))
        return ou, ov

    # -- operators with the box boundary rules ------------------------------------------------
    def fill_ghosts(self, u, v):
        u = np.array(u, dtype=np.float64, order="C")
        v = np.array(v, dtype=np.float64, order="C")
        self.lib.orc_fill_ghosts(ctypes.byref(self.s), _p(u), _p(v))
        return u, v

    def visc_bc(self, u, v):
        ou, ov = self.z(), self.z()
        self.lib.orc_visc_bc(ctypes.byref(self.s), _p(self.caps), _p(self._c(u)), _p(self._c(v)), _p(ou), _p(ov))
        return ou, ov

    def conv_bc(self, u, v):
        ou, ov = self.z(), self.z()
        self.lib.orc_conv_bc(ctypes.byref(self.s), _p(self.caps), _p(self._c(u)), _p(self._c(v)), _p(ou), _p(ov))
        return ou, ov

    def pres_bc(self, p):
        ou, ov = self.z(), self.z()
        self.lib.orc_pres_bc(ctypes.byref(self.s), _p(self.caps), _p(self._c(p)), _p(ou), _p(ov))
        return ou, ov

    def helmholtz(self, u, v):
        ou, ov = self.z(), self.z()
        self.lib.orc_helmholtz(ctypes.byref(self.s), _p(self.caps), _p(self._c(u)), _p(self._c(v)), _p(ou), _p(ov))
        return ou, ov

    def poisson(self, phi):
        o = self.z()
        self.lib.orc_poisson(ctypes.byref(self.s), _p(self.caps), _p(self._c(phi)), _p(o))
        return o

    def poisson_diag(self):
        d = self.z()
        self.lib.orc_poisson_diag(ctypes.byref(self.s), _p(self.caps), _p(d))
        return d

    def helmholtz_diag(self):
        du, dv = self.z(), self.z()
        self.lib.orc_helmholtz_diag(ctypes.byref(self.s), _p(self.caps), _p(du), _p(dv))
        return du, dv

    def poisson_precondition(self, r):
        """z = M^-1 r with the Poisson PCG's preconditioner (Jacobi or k-step Chebyshev)."""
        z = self.z()
        self.lib.orc_poisson_precondition(ctypes.byref(self.s), _p(self.caps), _p(self._c(r)), _p(z))
        return z

    def solve_poisson(self, rhs, phi0=None, tol=None, max_iter=None):
        phi = self.z() if phi0 is None else np.array(phi0, dtype=np.float64, order="C")
        it = c_int(0)
        rr = c_double(0.0)
        ok = self.lib.orc_solve_poisson(ctypes.byref(self.s), _p(self.caps), _p(self._c(rhs)), _p(phi),
                                        self.case.tol_p if tol is None else tol,
                                        self.case.max_iter_p if max_iter is None else max_iter,
                                        ctypes.byref(it), ctypes.byref(rr))
        return phi, dict(converged=bool(ok), iters=it.value, rel_res=rr.value)

    def solve_helmholtz(self, ru, rv, u0=None, v0=None, tol=None, max_iter=None):
        xu = self.z() if u0 is None else np.array(u0, dtype=np.float64, order="C")
        xv = self.z() if v0 is None else np.array(v0, dtype=np.float64, order="C")
        it = c_int(0)
        rr = c_double(0.0)
        ok = self.lib.orc_solve_helmholtz(ctypes.byref(self.s), _p(self.caps), _p(self._c(ru)), _p(self._c(rv)),
                                          _p(xu), _p(xv), self.case.tol_h if tol is None else tol,
                                          self.case.max_iter_h if max_iter is None else max_iter,
                                          ctypes.byref(it), ctypes.byref(rr))
        return xu, xv, dict(converged=bool(ok), iters=it.value, rel_res=rr.value)

    def kinetic(self, u, v):
        return self.lib.orc_kinetic(ctypes.byref(self.s), _p(self.caps), _p(self._c(u)), _p(self._c(v)))

    def max_div(self, u, v):
        return self.lib.orc_max_div(ctypes.byref(self.s), _p(self.caps), _p(self._c(u)), _p(self._c(v)))

    def body_force(self, u, v, p, Dx=None, Dy=None):
        """(Fp_x, Fp_y, Fv_x, Fv_y): pressure and viscous force of the fluid on the body (whose
        Dirichlet velocity is D, zero when not given)."""
        f = np.zeros(4)
        self.lib.orc_body_force_d(ctypes.byref(self.s), _p(self.caps), _p(self._c(u)), _p(self._c(v)),
                                  _p(self._c(p)), _p(self._c(Dx)), _p(self._c(Dy)), _p(f))
        return f

    def conservation(self, u, v, Dx=None, Dy=None):
        """(sum of cont(U, D) over the box cells, sum V^x u, sum V^y v)."""
        out = np.zeros(3)
        self.lib.orc_conservation(ctypes.byref(self.s), _p(self.caps), _p(self._c(u)), _p(self._c(v)),
                                  _p(self._c(Dx)), _p(self._c(Dy)), _p(out))
        return out

    def cell_boundary(self, grid, i, j):
        a, b = c_double(0.0), c_double(0.0)
        self.lib.orc_cell_boundary(ctypes.byref(self.s), GRIDS.index(grid), i, j, ctypes.byref(a), ctypes.byref(b))
        return a.value, b.value

    def predictor_rhs(self, u, v, p, cu=None, cv=None, first=True):
        """Right-hand side of Eq. pm_prediction and conv^n from U^n (ghosts filled here)."""
        u = np.array(u, dtype=np.float64, order="C")
        v = np.array(v, dtype=np.float64, order="C")
        cu = self.z() if cu is None else self._c(cu)
        cv = self.z() if cv is None else self._c(cv)
        ru, rv, cnu, cnv = self.z(), self.z(), self.z(), self.z()
        self.lib.orc_predictor_rhs(ctypes.byref(self.s), _p(self.caps), _p(u), _p(v), _p(self._c(p)), _p(cu),
                                   _p(cv), 1 if first else 0, _p(ru), _p(rv), _p(cnu), _p(cnv))
        return ru, rv, cnu, cnv

    # -- time stepping ---------------------------------------------------------------------
    def init_state(self, pu=None, pv=None, u0=None, v0=0.0):
        u, v = self.z(), self.z()
        u0 = self.case.bc_un[0] if u0 is None else u0
        self.lib.orc_init_velocity(ctypes.byref(self.s), _p(self.caps), u0, v0, _p(self._c(pu)),
                                   _p(self._c(pv)), _p(u), _p(v))
        return dict(u=u, v=v, p=self.z(), phi=self.z(), cu=self.z(), cv=self.z(), n=0)

    def step(self, st, nsteps=1, keep=False):
        stats = OrcStats()
        extra = None
        hist = []
        for _ in range(nsteps):
            us, vs, bd = (self.z(), self.z(), self.z()) if keep else (None, None, None)
            # st may carry a body acceleration "gx" (u-faces), "gy" (v-faces), Eq. pm_prediction's rho V g,
            # and the body's Dirichlet velocity "Dx" (per u-cell), "Dy" (per v-cell); with "motion"
            # (a0, a1, omega, phase) the body velocity at step n is D0 times the factor
            # inputs.body_motion_factor gives for t = n dt (D0 = Dx, Dy), else it is steady
            gx, gy = st.get("gx"), st.get("gy")
            Dx, Dy = self._c(st.get("Dx")), self._c(st.get("Dy"))
            motion = st.get("motion")
            if motion is None or Dx is None:
                Dxn, Dyn, Dx1, Dy1 = Dx, Dy, Dx, Dy
            else:
                from paper_2211_10698_gb300.inputs import body_motion_factor
                fn = body_motion_factor(motion, st["n"], self.case.dt)
                f1 = body_motion_factor(motion, st["n"] + 1, self.case.dt)
                Dxn, Dyn, Dx1, Dy1 = fn * Dx, fn * Dy, f1 * Dx, f1 * Dy
            ok = self.lib.orc_step_gdt(ctypes.byref(self.s), _p(self.caps), _p(st["u"]), _p(st["v"]), _p(st["p"]),
                                       _p(st["phi"]), _p(st["cu"]), _p(st["cv"]), 1 if st["n"] == 0 else 0,
                                       _p(self._c(gx)), _p(self._c(gy)), _p(Dxn), _p(Dyn), _p(Dx1), _p(Dy1),
                                       _p(us), _p(vs), _p(bd), ctypes.byref(stats))
            st["n"] += 1
            hist.append(dict(iters_h=stats.iters_h, iters_p=stats.iters_p, res_h=stats.res_h,
                             res_p=stats.res_p, max_div=stats.max_div, kinetic=stats.kinetic,
                             ok=bool(ok)))
            if keep:
                extra = dict(ustar=us, vstar=vs, b=bd)
        return hist, extra


def dense(apply, n_in_shape, mask_in, mask_out):
    """Matrix of a linear map restricted to masked positions, by unit vectors (small grids)."""
    idx_in = [tuple(ix) for ix in np.argwhere(mask_in)]
    idx_out = [tuple(ix) for ix in np.argwhere(mask_out)]
    M = np.zeros((len(idx_out), len(idx_in)))
    for col, ix in enumerate(idx_in):
        e = np.zeros(mask_in.shape)
        e[ix] = 1.0
        y = apply(e)
        M[:, col] = [y[o] for o in idx_out]
    return M
