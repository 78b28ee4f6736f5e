"""Failure detection through the C ABI, in forms that fault, trap or hang no GPU.

* A device-wide barrier that runs out: one block of every cooperative launch skips its
  arrivals (ccm_set_barrier_fault), so every other block's bounded wait gives up after a short
  budget; ccm_step must return CCM_E_TIMEOUT, and the same case must step on normally once the
  fault is cleared and a checkpoint restored.
* Non-finite fields set from the host: ccm_step must return CCM_E_NONFINITE.
* Checkpoint and restore through ccm_get_field / ccm_set_field: a fresh case restored from the
  state after k steps must continue bit for bit like the uninterrupted run.
(The allocator hook that returns NULL is checked on the CPU in test_abi.py.)"""
import ctypes
import time

import numpy as np
import pytest

from paper_2211_10698_gb300 import ccm, inputs as I

pytestmark = pytest.mark.gpu

STATE = (ccm.CCM_F_U, ccm.CCM_F_V, ccm.CCM_F_P, ccm.CCM_F_PHI, ccm.CCM_F_CONV_U, ccm.CCM_F_CONV_V,
         ccm.CCM_F_STEP)


def _case(precision="fp64", precond="jacobi", nx=256):
    case = I.small_cylinder(nx=nx, ny=nx // 2, box=(-2.0, 6.0, -2.0, 2.0), r=0.5, cx=0.0, cy=0.0)
    case.precision, case.precond, case.cheb_degree = precision, precond, 3
    case.autotune = 0  # the built-in launch shape, the same in every process
    return case


def _checkpoint(g):
    return {f: g.get_field(f).copy() for f in STATE}


def _restore(g, ck):
    for f in STATE:
        g.set_field(f, ck[f])


def _status(g, n):
    st = ccm.ccm_step_stats()
    return ccm.lib().ccm_step(g.h, n, ctypes.byref(st)), st


@pytest.mark.parametrize("precision,precond,plan", [("fp64", "jacobi", None), ("mixed", "jacobi", None),
                                                    ("mixed", "chebyshev", None),
                                                    ("mixed", "chebyshev", (64, 16, 4, 32, 0, 0, 0))])
def test_barrier_timeout_is_reported_and_the_case_recovers(precision, precond, plan):
    """plan: a mixed tile plan selects the solve with one barrier per iteration."""
    case = _case(precision, precond)
    g = ccm.Case(case)
    if plan:
        g.set_launch_plan(plan)
    assert g.launch_plan()[5] == 0, "the single-cluster solve has no spin barrier to run out"
    g.step(2)
    ck = _checkpoint(g)
    L = ccm.lib()
    assert L.ccm_set_barrier_fault(g.h, 1_000_000, 0) == ccm.CCM_OK  # ~0.5 ms per wait, block 0 absent
    t0 = time.time()
    status, _ = _status(g, 1)
    assert status == ccm.CCM_E_TIMEOUT, (ccm.STATUS_NAMES[status], L.ccm_last_error())
    assert b"barrier" in L.ccm_last_error()
    assert time.time() - t0 < 60.0
    # the context is usable: clear the fault, restore the checkpoint and step on
    assert L.ccm_set_barrier_fault(g.h, 0, -1) == ccm.CCM_OK
    _restore(g, ck)
    st = g.step(2)
    assert st["converged"] and st["steps"] == 2
    ref = ccm.Case(case)
    if plan:
        ref.set_launch_plan(plan)
    ref.step(4)
    for f in (ccm.CCM_F_U, ccm.CCM_F_V, ccm.CCM_F_P, ccm.CCM_F_PHI):
        assert np.array_equal(g.get_field(f), ref.get_field(f)), f
    g.close()
    ref.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_nonfinite_velocity_is_reported(precision):
    case = _case(precision, nx=128)  # a NaN residual never meets the tolerance: the solves
    g = ccm.Case(case)                # run to their iteration limits (bounded)
    g.step(1)
    u = g.get_field(ccm.CCM_F_U)
    u[20, 30] = np.nan  # a fluid u-face upstream of the body
    g.set_field(ccm.CCM_F_U, u)
    status, _ = _status(g, 1)
    assert status == ccm.CCM_E_NONFINITE, (ccm.STATUS_NAMES[status], ccm.lib().ccm_last_error())
    # restoring a finite state clears it
    g2 = ccm.Case(case)
    g2.step(1)
    _restore(g, _checkpoint(g2))
    status, _ = _status(g, 1)
    assert status == ccm.CCM_OK, ccm.lib().ccm_last_error()
    g.close()
    g2.close()


@pytest.mark.parametrize("precision,precond", [("fp64", "jacobi"), ("mixed", "chebyshev")])
def test_checkpoint_restore_continues_bitwise(precision, precond):
    case = _case(precision, precond, nx=192)
    case.perturb_sigma = 1e-3
    k, m = 5, 4
    ref = ccm.Case(case)
    pu, pv = I.perturbation(case)
    u0 = ref.get_field(ccm.CCM_F_U) + pu * (ref.cap("u", "V") > 0)
    v0 = ref.get_field(ccm.CCM_F_V) + pv * (ref.cap("v", "V") > 0)
    ref.set_field(ccm.CCM_F_U, u0)
    ref.set_field(ccm.CCM_F_V, v0)
    ref.step(k)
    ck = _checkpoint(ref)
    assert ck[ccm.CCM_F_STEP][0, 0] == k
    ref.step(m)
    g = ccm.Case(case)
    _restore(g, ck)
    g.step(m)
    for f in (ccm.CCM_F_U, ccm.CCM_F_V, ccm.CCM_F_P, ccm.CCM_F_PHI, ccm.CCM_F_CONV_U, ccm.CCM_F_CONV_V):
        assert np.array_equal(g.get_field(f), ref.get_field(f)), f
    assert g.get_field(ccm.CCM_F_STEP)[0, 0] == k + m
    g.close()
    ref.close()


@pytest.mark.parametrize("plan", [(128, 27, 8, 152, 0, 0, 1), (64, 27, 16, 304, 0, 0, 0)])
def test_fixed_point_sums_fallback_path(plan):
    """The FP64 one-barrier CG sums its dot products as exact fixed-point digits and falls back
    to FP64 partials and a counter barrier when a value leaves the digits' window (a sum that
    grew 2^20-fold in one iteration).  The test hook forces that fallback on every third
    reduction: the steps converge, and the fields equal those of the normal path to the solver
    tolerance (resident and global-memory tiles, 1024x512 cylinder)."""
    def run(every):
        case = I.cylinder_re100_1024x512()
        case.autotune = 0
        g = ccm.Case(case)
        g.set_launch_plan(plan)
        assert ccm.lib().ccm_set_sum_fallback(g.h, every) == ccm.CCM_OK
        st = g.step(3)
        out = {f: g.get_field(f) for f in (ccm.CCM_F_U, ccm.CCM_F_V, ccm.CCM_F_P)}
        g.close()
        return st, out

    s0, f0 = run(0)
    s3, f3 = run(3)
    assert s0["converged"] and s3["converged"]
    assert abs(s3["iters_p"] - s0["iters_p"]) <= 0.02 * s0["iters_p"] + 3
    for f in f0:
        assert np.linalg.norm(f3[f] - f0[f]) / np.linalg.norm(f0[f]) < 1e-9, f
    assert ccm.lib().ccm_set_sum_fallback(None, 1) == ccm.CCM_E_INVALID
