"""ctypes binding of libccm (include/ccm.h).  Argument marshalling only: every step of the
computation runs in the CUDA library, and importing this module fails loudly when the
library has not been built.

The functions keep the C names (``ccm_create_case``, ``ccm_step``, ...).  ``Case`` is a
small owner object that builds a ``ccm_config`` from a ``paper_2211_10698_gb300.inputs.Case``
and releases the library case when it goes away.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import CFUNCTYPE, POINTER, Structure, c_double, c_int, c_longlong, c_size_t, c_void_p

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libccm.so")

CCM_OK, CCM_E_INVALID, CCM_E_OOM, CCM_E_CUDA, CCM_E_NOT_CONVERGED, CCM_E_NONFINITE, CCM_E_TIMEOUT, CCM_E_STATE = range(8)
STATUS_NAMES = ["CCM_OK", "CCM_E_INVALID", "CCM_E_OOM", "CCM_E_CUDA", "CCM_E_NOT_CONVERGED", "CCM_E_NONFINITE",
                "CCM_E_TIMEOUT", "CCM_E_STATE"]
CCM_BC_DIRICHLET, CCM_BC_OUTFLOW, CCM_BC_PERIODIC = 0, 1, 2
CCM_FP64, CCM_MIXED = 0, 1
CCM_JACOBI, CCM_CHEBYSHEV = 0, 1
CCM_F_U, CCM_F_V, CCM_F_P, CCM_F_PHI, CCM_F_CONV_U, CCM_F_CONV_V, CCM_F_USTAR, CCM_F_VSTAR, CCM_F_DIV, CCM_F_STEP = range(10)
CCM_F_GX, CCM_F_GY = 10, 11   # body acceleration g at u- and v-faces (rho V g in the predictor)
CCM_F_DX, CCM_F_DY = 12, 13   # the body's steady Dirichlet velocity D per u- and v-cell
CCM_F_CAP = 16
(CCM_OP_CONT, CCM_OP_PRES, CCM_OP_CONV, CCM_OP_VISC, CCM_OP_HELMHOLTZ, CCM_OP_POISSON, CCM_OP_POISSON_DIAG,
 CCM_OP_HELMHOLTZ_DIAG) = range(8)
CAP_NAMES = ("V", "X", "Y", "AX", "AY", "WX", "WY", "BX", "BY")
GRIDS = ("p", "u", "v")

ccm_alloc_fn = CFUNCTYPE(c_void_p, c_size_t, c_void_p)
ccm_free_fn = CFUNCTYPE(None, c_void_p, c_void_p)


class ccm_config(Structure):
    _fields_ = [("nx", c_int), ("ny", c_int),
                ("x0", c_double), ("x1", c_double), ("y0", c_double), ("y1", c_double),
                ("rho", c_double), ("mu", c_double), ("dt", c_double),
                ("bc_type", c_int * 4), ("bc_un", c_double * 4), ("bc_ut", c_double * 4),
                ("precision", c_int), ("precond", c_int), ("cheb_degree", c_int),
                ("tol_p", c_double), ("tol_h", c_double), ("tol_inner", c_double),
                ("max_iter_p", c_int), ("max_iter_h", c_int), ("literal_offdiag", c_int), ("pressure_update", c_int),
                ("replace_drop", c_double), ("autotune", c_int),
                ("alloc", ccm_alloc_fn), ("free", ccm_free_fn), ("alloc_ctx", c_void_p),
                ("stream", c_void_p), ("xf", POINTER(c_double)), ("yf", POINTER(c_double)),
                ("guess_history", c_int)]


class ccm_geometry(Structure):
    _fields_ = [("kind", c_int), ("cx", c_double), ("cy", c_double), ("r", c_double),
                ("naca_tt", c_int), ("closed_te", c_int),
                ("chord", c_double), ("aoa_deg", c_double), ("le_x", c_double), ("le_y", c_double),
                ("hp_nx", c_double), ("hp_ny", c_double), ("hp_off", c_double)]


class ccm_solve_stats(Structure):
    _fields_ = [("iters", c_int), ("outer", c_int), ("rel_res", c_double), ("converged", c_int)]


class ccm_step_stats(Structure):
    _fields_ = [("steps", c_int), ("iters_p", c_longlong), ("iters_h", c_longlong),
                ("last_iters_p", c_int), ("last_iters_h", c_int),
                ("last_res_p", c_double), ("last_res_h", c_double),
                ("max_div", c_double), ("kinetic", c_double), ("converged", c_int),
                ("mass", c_double), ("momentum_x", c_double), ("momentum_y", c_double)]


class CcmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


_lib = None
_DP = POINTER(c_double)


def lib():
    """Load libccm.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise ImportError(f"libccm.so is not built ({_LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(_LIB_PATH)
        cp = c_void_p
        sigs = {
            "ccm_version": (c_int, []),
            "ccm_last_error": (ctypes.c_char_p, []),
            "ccm_create_case": (c_int, [POINTER(ccm_config), POINTER(c_void_p)]),
            "ccm_destroy_case": (c_int, [cp]),
            "ccm_set_geometry": (c_int, [cp, POINTER(ccm_geometry)]),
            "ccm_set_field": (c_int, [cp, c_int, _DP, c_size_t]),
            "ccm_get_field": (c_int, [cp, c_int, _DP, c_size_t]),
            "ccm_field_device_ptr": (c_int, [cp, c_int, POINTER(c_void_p), POINTER(c_int)]),
            "ccm_apply_op": (c_int, [cp, c_int, _DP, _DP, _DP, _DP]),
            "ccm_step": (c_int, [cp, c_int, POINTER(ccm_step_stats)]),
            "ccm_solve_pressure": (c_int, [cp, _DP, POINTER(ccm_solve_stats)]),
            "ccm_step_async": (c_int, [cp, c_int]),
            "ccm_read_stats": (c_int, [cp, POINTER(ccm_step_stats)]),
            "ccm_body_force": (c_int, [cp, _DP]),
            "ccm_set_force_history": (c_int, [cp, c_int]),
            "ccm_get_force_history": (c_int, [cp, _DP, c_int, POINTER(c_int), POINTER(c_longlong)]),
            "ccm_enable_kernel_timing": (c_int, [cp, c_int]),
            "ccm_kernel_timing": (c_int, [cp, POINTER(c_double), POINTER(c_longlong), POINTER(c_longlong),
                                          POINTER(c_longlong)]),
            "ccm_solve_pressure_noalloc": (c_int, [cp, c_void_p, c_void_p, POINTER(ccm_solve_stats)]),
            "ccm_set_barrier_fault": (c_int, [cp, c_longlong, c_int]),
            "ccm_set_body_motion": (c_int, [cp, c_double, c_double, c_double, c_double]),
            "ccm_set_sum_fallback": (c_int, [cp, c_int]),
            "ccm_measure_fp64_rate": (c_int, [_DP]),
            "ccm_batch_create": (c_int, [c_int, c_void_p, POINTER(c_void_p)]),
            "ccm_batch_destroy": (c_int, [cp]),
            "ccm_batch_add": (c_int, [cp, cp]),
            "ccm_batch_remove": (c_int, [cp, cp]),
            "ccm_batch_size": (c_int, [cp]),
            "ccm_batch_step": (c_int, [cp, c_int, POINTER(ccm_step_stats)]),
            "ccm_batch_set_graphs": (c_int, [cp, c_int]),
            "ccm_batch_graph_steps": (c_int, [cp, POINTER(c_longlong)]),
            "ccm_batch_set_tuning": (c_int, [cp, c_int]),
            "ccm_batch_split": (c_int, [cp, POINTER(c_double), POINTER(c_int)]),
            "ccm_case_bytes": (c_int, [POINTER(ccm_config), POINTER(c_size_t)]),
            "ccm_launch_plan": (c_int, [c_void_p, POINTER(c_int)]),
            "ccm_set_launch_plan": (c_int, [c_void_p, POINTER(c_int)]),
            "ccm_server_create": (c_int, [c_size_t, c_int, c_int, c_void_p, POINTER(c_void_p)]),
            "ccm_server_destroy": (c_int, [cp]),
            "ccm_server_submit": (c_int, [cp, POINTER(ccm_config), POINTER(ccm_geometry), c_int, POINTER(c_longlong)]),
            "ccm_server_run": (c_int, [cp, c_int, POINTER(c_int)]),
            "ccm_server_poll": (c_int, [cp, c_longlong, POINTER(c_int), POINTER(c_double), POINTER(ccm_step_stats)]),
            "ccm_server_get_field": (c_int, [cp, c_longlong, c_int, _DP, c_size_t]),
            "ccm_server_release": (c_int, [cp, c_longlong]),
            "ccm_server_bytes_in_use": (c_size_t, [cp]),
        }
        for name, (res, args) in sigs.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status, allow=()):
    if status != CCM_OK and status not in allow:
        raise CcmError(status, lib().ccm_last_error().decode())
    return status


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_DP)


def make_config(case, precision=None, precond=None, stream=None) -> ccm_config:
    cfg = ccm_config()
    cfg.nx, cfg.ny = case.nx, case.ny
    cfg.x0, cfg.x1, cfg.y0, cfg.y1 = case.x0, case.x1, case.y0, case.y1
    cfg.rho, cfg.mu, cfg.dt = case.rho, case.mu, case.dt
    for s in range(4):
        cfg.bc_type[s] = int(case.bc_type[s])
        cfg.bc_un[s] = float(case.bc_un[s])
        cfg.bc_ut[s] = float(case.bc_ut[s])
    prec = precision if precision is not None else case.precision
    cfg.precision = CCM_MIXED if prec == "mixed" else CCM_FP64
    pc = precond if precond is not None else case.precond
    cfg.precond = CCM_CHEBYSHEV if pc == "chebyshev" else CCM_JACOBI
    cfg.cheb_degree = case.cheb_degree
    cfg.tol_p, cfg.tol_h, cfg.tol_inner = case.tol_p, case.tol_h, case.tol_inner
    cfg.max_iter_p, cfg.max_iter_h = case.max_iter_p, case.max_iter_h
    cfg.literal_offdiag = int(case.literal_offdiag)
    cfg.pressure_update = int(getattr(case, "pressure_update", 0))
    cfg.replace_drop = float(getattr(case, "replace_drop", 0.0))
    cfg.autotune = int(getattr(case, "autotune", 0))
    cfg.guess_history = int(getattr(case, "guess_history", 0))
    cfg.stream = stream
    if getattr(case, "stretched", False):
        # the arrays must outlive the call that reads them: kept on the structure
        cfg._faces = (case.faces_x(), case.faces_y())
        cfg.xf = cfg._faces[0].ctypes.data_as(_DP)
        cfg.yf = cfg._faces[1].ctypes.data_as(_DP)
    return cfg


def make_geometry(geom) -> ccm_geometry:
    g = ccm_geometry()
    g.kind = geom.kind
    g.cx, g.cy, g.r = geom.cx, geom.cy, geom.r
    g.naca_tt, g.closed_te = geom.naca_tt, geom.closed_te
    g.chord, g.aoa_deg, g.le_x, g.le_y = geom.chord, geom.aoa_deg, geom.le_x, geom.le_y
    g.hp_nx, g.hp_ny, g.hp_off = geom.hp_nx, geom.hp_ny, geom.hp_off
    return g


class TorchAllocator:
    """Device memory for cases from PyTorch's caching allocator (through the ccm_config
    allocator hooks)."""

    def __init__(self):
        import torch
        self._torch = torch

        def _alloc(nbytes, ctx):
            return int(torch.cuda.caching_allocator_alloc(int(nbytes)))

        def _free(ptr, ctx):
            torch.cuda.caching_allocator_delete(int(ptr))

        self.alloc = ccm_alloc_fn(_alloc)
        self.free = ccm_free_fn(_free)


class Case:
    """A library case built from an ``inputs.Case``; geometry is set at construction."""

    def __init__(self, case, precision=None, precond=None, stream=None, allocator=None, set_geometry=True):
        self.spec = case
        self.shape = case.shape
        self.n = case.shape[0] * case.shape[1]
        self.cfg = make_config(case, precision, precond, stream)
        self._allocator = allocator
        if allocator is not None:
            self.cfg.alloc = allocator.alloc
            self.cfg.free = allocator.free
        h = c_void_p()
        _check(lib().ccm_create_case(ctypes.byref(self.cfg), ctypes.byref(h)))
        self.h = h
        if set_geometry:
            self.set_geometry(case.geom)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().ccm_destroy_case(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_geometry(self, geom):
        g = make_geometry(geom)
        _check(lib().ccm_set_geometry(self.h, ctypes.byref(g)))

    def set_field(self, field, arr):
        a = np.ascontiguousarray(arr, dtype=np.float64)
        assert a.shape == self.shape
        _check(lib().ccm_set_field(self.h, field, _ptr(a), a.size))

    def get_field(self, field, out=None):
        a = np.empty(self.shape) if out is None else out
        assert a.shape == self.shape and a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
        _check(lib().ccm_get_field(self.h, field, _ptr(a), a.size))
        return a

    def cap(self, grid, name):
        return self.get_field(CCM_F_CAP + 9 * GRIDS.index(grid) + CAP_NAMES.index(name))

    def apply(self, op, in0=None, in1=None, nout=2):
        i0 = None if in0 is None else np.ascontiguousarray(in0, dtype=np.float64)
        i1 = None if in1 is None else np.ascontiguousarray(in1, dtype=np.float64)
        o0 = np.zeros(self.shape)
        o1 = np.zeros(self.shape) if nout > 1 else None
        _check(lib().ccm_apply_op(self.h, op, _ptr(i0), _ptr(i1), _ptr(o0), _ptr(o1)))
        return (o0, o1) if nout > 1 else o0

    def step(self, n=1, allow_not_converged=False):
        st = ccm_step_stats()
        allow = (CCM_E_NOT_CONVERGED,) if allow_not_converged else ()
        _check(lib().ccm_step(self.h, n, ctypes.byref(st)), allow)
        return {f: getattr(st, f) for f, _ in ccm_step_stats._fields_}

    def launch_plan(self):
        """(tile width, tile height, tiles per row, tiles, mixed blocks, cluster CTAs, resident
        tiles) of the single-case Poisson solve; zeros where the built-in shape is used."""
        plan = (c_int * 7)()
        _check(lib().ccm_launch_plan(self.h, plan))
        return tuple(plan)

    def set_launch_plan(self, plan):
        plan = tuple(plan) + (0,) * (7 - len(plan))
        arr = (c_int * 7)(*plan)
        _check(lib().ccm_set_launch_plan(self.h, arr))

    def step_async(self, n=1):
        _check(lib().ccm_step_async(self.h, n))

    def read_stats(self, allow_not_converged=False):
        st = ccm_step_stats()
        allow = (CCM_E_NOT_CONVERGED,) if allow_not_converged else ()
        _check(lib().ccm_read_stats(self.h, ctypes.byref(st)), allow)
        return {f: getattr(st, f) for f, _ in ccm_step_stats._fields_}

    def set_body_motion(self, a0, a1, omega, phase):
        """Body velocity D(t) = (a0 + a1 sin(omega t + phase)) D0 from the next step on, with D0
        the field set through CCM_F_DX / CCM_F_DY and t = n dt at step n."""
        _check(lib().ccm_set_body_motion(self.h, float(a0), float(a1), float(omega), float(phase)))

    def body_force(self):
        """(Fp_x, Fp_y, Fv_x, Fv_y): pressure and viscous force of the fluid on the body at the
        current state."""
        f = np.zeros(4)
        _check(lib().ccm_body_force(self.h, _ptr(f)))
        return f

    def set_force_history(self, capacity):
        """Record the body force after every step (newest ``capacity`` steps kept)."""
        _check(lib().ccm_set_force_history(self.h, int(capacity)))
        self._force_capacity = int(capacity)

    def force_history(self, max_rows=None):
        """(rows x 4 array of recorded forces, oldest first; steps recorded in total)."""
        n = c_int()
        tot = c_longlong()
        _check(lib().ccm_get_force_history(self.h, None, 0, ctypes.byref(n), ctypes.byref(tot)))
        kept = min(tot.value, getattr(self, "_force_capacity", 0))
        cap = kept if max_rows is None else int(max_rows)
        out = np.zeros((max(cap, 0), 4))
        _check(lib().ccm_get_force_history(self.h, _ptr(out) if cap > 0 else None, cap, ctypes.byref(n),
                                           ctypes.byref(tot)))
        return out[:n.value], tot.value

    def enable_kernel_timing(self, on=True):
        _check(lib().ccm_enable_kernel_timing(self.h, 1 if on else 0))

    def kernel_timing(self):
        ms, nl, it, kl = c_double(), c_longlong(), c_longlong(), c_longlong()
        _check(lib().ccm_kernel_timing(self.h, ctypes.byref(ms), ctypes.byref(nl), ctypes.byref(it), ctypes.byref(kl)))
        return dict(poisson_ms=ms.value, poisson_launches=nl.value, poisson_iters=it.value, kernel_launches=kl.value)

    def solve_pressure(self, rhs):
        r = np.ascontiguousarray(rhs, dtype=np.float64)
        st = ccm_solve_stats()
        _check(lib().ccm_solve_pressure(self.h, _ptr(r), ctypes.byref(st)), (CCM_E_NOT_CONVERGED,))
        return {f: getattr(st, f) for f, _ in ccm_solve_stats._fields_}

    def device_ptr(self, field):
        p = c_void_p()
        pitch = c_int()
        _check(lib().ccm_field_device_ptr(self.h, field, ctypes.byref(p), ctypes.byref(pitch)))
        return p.value, pitch.value


class Batch:
    """Cases advanced together (one batched Poisson solve per step)."""

    def __init__(self, max_cases, stream=None):
        h = c_void_p()
        _check(lib().ccm_batch_create(max_cases, stream, ctypes.byref(h)))
        self.h = h
        self.cases = []

    def add(self, case):
        _check(lib().ccm_batch_add(self.h, case.h))
        self.cases.append(case)

    def remove(self, case):
        _check(lib().ccm_batch_remove(self.h, case.h))
        self.cases.remove(case)

    def step(self, n=1, allow_not_converged=False):
        arr = (ccm_step_stats * max(len(self.cases), 1))()
        allow = (CCM_E_NOT_CONVERGED,) if allow_not_converged else ()
        _check(lib().ccm_batch_step(self.h, n, arr), allow)
        return [{f: getattr(arr[i], f) for f, _ in ccm_step_stats._fields_} for i in range(len(self.cases))]

    def set_graphs(self, enable=True):
        _check(lib().ccm_batch_set_graphs(self.h, 1 if enable else 0))

    def set_tuning(self, enable=True):
        _check(lib().ccm_batch_set_tuning(self.h, 1 if enable else 0))

    def split(self):
        """(exponent a of the Poisson split cells x nx^a, whether the tuning has finished)"""
        a, t = c_double(), c_int()
        _check(lib().ccm_batch_split(self.h, ctypes.byref(a), ctypes.byref(t)))
        return a.value, bool(t.value)

    def graph_steps(self):
        n = c_longlong()
        _check(lib().ccm_batch_graph_steps(self.h, ctypes.byref(n)))
        return n.value

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().ccm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def case_bytes(case, precision=None, precond=None):
    """Device bytes a case of this description holds (ccm_case_bytes; allocates nothing)."""
    cfg = make_config(case, precision, precond)
    n = c_size_t()
    _check(lib().ccm_case_bytes(ctypes.byref(cfg), ctypes.byref(n)))
    return n.value


class Server:
    """Request loop: submit flow-past-body requests, run rounds, poll for completion."""

    STATES = ("queued", "running", "done", "failed")

    def __init__(self, hbm_budget_bytes, max_batch=64, chunk_steps=10, stream=None):
        h = c_void_p()
        _check(lib().ccm_server_create(int(hbm_budget_bytes), max_batch, chunk_steps, stream, ctypes.byref(h)))
        self.h = h

    def submit(self, case, nsteps=None, precision=None, precond=None):
        cfg = make_config(case, precision, precond)
        geo = make_geometry(case.geom)
        rid = c_longlong()
        _check(lib().ccm_server_submit(self.h, ctypes.byref(cfg), ctypes.byref(geo),
                                       case.steps if nsteps is None else nsteps, ctypes.byref(rid)))
        return rid.value

    def run(self, rounds=1):
        active = c_int()
        _check(lib().ccm_server_run(self.h, rounds, ctypes.byref(active)), (CCM_E_NOT_CONVERGED,))
        return active.value

    def poll(self, rid):
        state = c_int()
        times = (c_double * 3)()
        st = ccm_step_stats()
        _check(lib().ccm_server_poll(self.h, rid, ctypes.byref(state), times, ctypes.byref(st)))
        return dict(state=self.STATES[state.value], t_submit=times[0], t_admit=times[1], t_done=times[2],
                    **{f: getattr(st, f) for f, _ in ccm_step_stats._fields_})

    def get_field(self, rid, field, shape):
        a = np.empty(shape)
        _check(lib().ccm_server_get_field(self.h, rid, field, _ptr(a), a.size))
        return a

    def release(self, rid):
        _check(lib().ccm_server_release(self.h, rid))

    def bytes_in_use(self):
        return lib().ccm_server_bytes_in_use(self.h)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().ccm_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
