"""The C ABI library builds, loads without a GPU and exports every function that
include/ccm.h declares; the Python binding uses the same names."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ccm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ccm_[a-z_0-9]+)\s*\(", src)) - {"ccm_alloc_fn", "ccm_free_fn"})


@pytest.fixture(scope="module")
def libccm():
    from paper_2211_10698_gb300 import build

    build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("ccm_create_case", "ccm_set_geometry", "ccm_step", "ccm_solve_pressure",
                     "ccm_get_field", "ccm_set_field", "ccm_apply_op", "ccm_destroy_case", "ccm_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(libccm):
    for name in _declared():
        assert hasattr(libccm, name), name


def test_binding_uses_the_same_names(libccm):
    from paper_2211_10698_gb300 import ccm

    L = ccm.lib()
    for name in _declared():
        assert getattr(L, name) is not None
    assert L.ccm_version() == 1


def test_errors_without_gpu_work(libccm):
    """Argument validation happens on the host, before any device call."""
    from paper_2211_10698_gb300 import ccm, inputs

    case = inputs.small_cylinder()
    cfg = ccm.make_config(case)
    cfg.nx = 2
    h = ctypes.c_void_p()
    assert ccm.lib().ccm_create_case(ctypes.byref(cfg), ctypes.byref(h)) == ccm.CCM_E_INVALID
    assert b"nx" in ccm.lib().ccm_last_error()
    assert ccm.lib().ccm_create_case(None, ctypes.byref(h)) == ccm.CCM_E_INVALID
    assert ccm.lib().ccm_step(None, 1, None) == ccm.CCM_E_INVALID


def test_force_and_body_fields_validate_on_the_host(libccm):
    """The force, force-record and body-field entry points reject bad arguments before any
    device work."""
    import ctypes

    from paper_2211_10698_gb300 import ccm

    L = ccm.lib()
    f = (ctypes.c_double * 4)()
    assert L.ccm_body_force(None, f) == ccm.CCM_E_INVALID
    assert L.ccm_set_force_history(None, 4) == ccm.CCM_E_INVALID
    n, tot = ctypes.c_int(), ctypes.c_longlong()
    assert L.ccm_get_force_history(None, None, 0, ctypes.byref(n), ctypes.byref(tot)) == ccm.CCM_E_INVALID
    buf = (ctypes.c_double * 8)()
    for field in (ccm.CCM_F_GX, ccm.CCM_F_GY, ccm.CCM_F_DX, ccm.CCM_F_DY):
        assert L.ccm_set_field(None, field, buf, 8) == ccm.CCM_E_INVALID


def test_allocator_hook_failure_is_out_of_memory(libccm):
    """An allocator hook that returns NULL makes ccm_create_case fail with CCM_E_OOM and no case
    (the hook is the first device-memory request, so this runs without a GPU)."""
    from paper_2211_10698_gb300 import ccm, inputs

    calls = []

    def _alloc(nbytes, ctx):
        calls.append(int(nbytes))
        return None

    def _free(ptr, ctx):
        raise AssertionError("nothing was allocated")

    cfg = ccm.make_config(inputs.small_cylinder())
    cfg.alloc, cfg.free = ccm.ccm_alloc_fn(_alloc), ccm.ccm_free_fn(_free)
    h = ctypes.c_void_p()
    assert ccm.lib().ccm_create_case(ctypes.byref(cfg), ctypes.byref(h)) == ccm.CCM_E_OOM
    assert b"allocator hook" in ccm.lib().ccm_last_error()
    assert h.value is None and len(calls) == 1
    need = ctypes.c_size_t()
    assert ccm.lib().ccm_case_bytes(ctypes.byref(cfg), ctypes.byref(need)) == ccm.CCM_OK
    assert calls[0] >= need.value > 0


def test_barrier_fault_hook_validates_on_the_host(libccm):
    from paper_2211_10698_gb300 import ccm

    L = ccm.lib()
    assert L.ccm_set_barrier_fault(None, 0, -1) == ccm.CCM_E_INVALID


def test_body_motion_validates_on_the_host(libccm):
    from paper_2211_10698_gb300 import ccm

    L = ccm.lib()
    assert L.ccm_set_body_motion(None, 1.0, 0.0, 0.0, 0.0) == ccm.CCM_E_INVALID


def test_stretched_faces_validate_on_the_host(libccm):
    """Face abscissas of a stretched mesh must increase strictly from x0 to x1 (y0 to y1)."""
    import numpy as np

    from paper_2211_10698_gb300 import ccm, inputs

    case = inputs.stretched_cylinder()
    for bad in ("order", "end"):
        cfg = ccm.make_config(case)
        xf = case.faces_x().copy()
        if bad == "order":
            xf[5], xf[6] = xf[6], xf[5]
        else:
            xf[-1] += 1e-9
        keep = np.ascontiguousarray(xf)
        cfg.xf = keep.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        h = ctypes.c_void_p()
        assert ccm.lib().ccm_create_case(ctypes.byref(cfg), ctypes.byref(h)) == ccm.CCM_E_INVALID
        assert b"abscissas" in ccm.lib().ccm_last_error()


def test_guess_history_validates_on_the_host(libccm):
    from paper_2211_10698_gb300 import ccm, inputs

    case = inputs.cylinder_re40_128x64()
    case.guess_history = 33
    cfg = ccm.make_config(case)
    h = ctypes.c_void_p()
    assert ccm.lib().ccm_create_case(ctypes.byref(cfg), ctypes.byref(h)) == ccm.CCM_E_INVALID
    assert b"guess_history" in ccm.lib().ccm_last_error()


def test_periodic_sides_validate_on_the_host(libccm):
    """Periodic sides come in pairs, on a uniform axis with a multiple of 3 cells."""
    from paper_2211_10698_gb300 import ccm, inputs

    L = ccm.lib()
    h = ctypes.c_void_p()
    cfg = ccm.make_config(inputs.taylor_green(24))
    cfg.bc_type[1] = ccm.CCM_BC_OUTFLOW
    assert L.ccm_create_case(ctypes.byref(cfg), ctypes.byref(h)) == ccm.CCM_E_INVALID
    assert b"pairs" in L.ccm_last_error()
    cfg = ccm.make_config(inputs.taylor_green(25 - 1))
    cfg.nx = 25
    assert L.ccm_create_case(ctypes.byref(cfg), ctypes.byref(h)) == ccm.CCM_E_INVALID
    assert b"multiple of 3" in L.ccm_last_error()
