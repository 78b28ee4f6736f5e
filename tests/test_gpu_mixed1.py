"""The mixed-precision Poisson solve with one grid barrier per iteration (pcg_mixed1.cu), forced
through a mixed tile plan, the tile's vectors in global or in shared memory: FP32 CG on the
Jacobi-scaled system (Jacobi or Chebyshev of degree k, the band of width k recomputed per
tile) with FP64 residual replacements.

Checked through the C ABI against the oracle (Eq. pm_poisson): the solution's residual under
the oracle's FP64 operator meets the tolerance, the solution agrees with the oracle's tight
solve to the conditioning of the system, the iteration count stays close to the other mixed
kernel's, and steps agree with the FP64 oracle to 1e-8 (the mixed-path tolerance).  Ragged
grids make tiles that the grid clips."""
import copy

import numpy as np
import pytest

from paper_2211_10698_gb300 import ccm, inputs as I

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _plan(nx, ny, tx, ty, resident=0):
    nbx = -(-nx // tx)
    return (tx, ty, nbx, nbx * -(-ny // ty), 0, 0, resident)


def _case(nx, ny, precond, degree, tol=1e-10):
    c = I.small_cylinder(nx=nx, ny=ny, box=(-2.0, 6.0, -2.0, 2.0), r=0.5, cx=0.1, cy=-0.05, re=100.0)
    c.precision, c.precond, c.cheb_degree, c.tol_p = "mixed", precond, degree, tol
    c.autotune = 0
    return c


GRIDS = [(128, 64, 64, 8), (53, 31, 32, 8), (256, 128, 64, 16)]
PRECS = [("jacobi", 1), ("chebyshev", 2), ("chebyshev", 3), ("chebyshev", 4)]


@pytest.mark.parametrize("resident", [0, 1])
@pytest.mark.parametrize("nx,ny,tx,ty", GRIDS)
@pytest.mark.parametrize("precond,degree", PRECS)
def test_one_barrier_mixed_solve_against_oracle(orc, nx, ny, tx, ty, precond, degree, resident):
    case = _case(nx, ny, precond, degree)
    g = ccm.Case(case)
    g.set_launch_plan(_plan(nx, ny, tx, ty, resident))
    assert g.launch_plan() == _plan(nx, ny, tx, ty, resident)
    o = orc.Oracle(case)
    rhs = np.random.default_rng(11).standard_normal(case.shape) * o.active
    st = g.solve_pressure(rhs)
    assert st["converged"] and st["rel_res"] <= case.tol_p, st
    phi = g.get_field(ccm.CCM_F_PHI)
    # the residual under the oracle's FP64 operator
    res = rhs - o.poisson(phi)
    res[~o.active] = 0.0
    assert np.linalg.norm(res) <= 1.05 * case.tol_p * np.linalg.norm(rhs)
    ref, info = o.solve_poisson(rhs, tol=1e-13, max_iter=50000)
    assert info["converged"]
    assert _rel(phi[o.active], ref[o.active]) < 1e-6
    # the kernel with k + 1 barriers per iteration on the same system
    g2 = ccm.Case(case)
    st2 = g2.solve_pressure(rhs)
    assert st2["converged"]
    assert abs(st["iters"] - st2["iters"]) <= 0.1 * st2["iters"] + 10, (st, st2)
    g.close()
    g2.close()


@pytest.mark.parametrize("resident", [0, 1])
@pytest.mark.parametrize("precond,degree", [("jacobi", 1), ("chebyshev", 3)])
def test_one_barrier_mixed_steps_against_oracle(orc, precond, degree, resident):
    """Six projection steps of a 128x64 cylinder: mixed precision with the one-barrier solve
    against the FP64 oracle with tight tolerances, 1e-8 on u, v and P."""
    case = _case(128, 64, precond, degree)
    g = ccm.Case(case)
    g.set_launch_plan(_plan(128, 64, 64, 8, resident))
    st = g.step(6)
    assert st["converged"]
    ocase = copy.deepcopy(case)
    ocase.tol_p = ocase.tol_h = 1e-13
    o = orc.Oracle(ocase)
    s = o.init_state()
    o.step(s, 6)
    for f, key in ((ccm.CCM_F_U, "u"), (ccm.CCM_F_V, "v"), (ccm.CCM_F_P, "p")):
        e = _rel(g.get_field(f), s[key])
        assert e < 1e-8, (key, e)
    g.close()


def test_one_barrier_mixed_plan_validation():
    case = _case(128, 64, "jacobi", 1)
    g = ccm.Case(case)
    with pytest.raises(ccm.CcmError):
        g.set_launch_plan((48, 8, 3, 24, 0, 0, 0))  # width not a power of two
    with pytest.raises(ccm.CcmError):
        g.set_launch_plan(_plan(128, 64, 64, 8)[:4] + (0, 0, 2))  # resident is 0 or 1
    with pytest.raises(ccm.CcmError):
        g.set_launch_plan(_plan(128, 64, 64, 8)[:4] + (0, 4, 0))  # tiles exclude a cluster
    with pytest.raises(ccm.CcmError):
        g.set_launch_plan((512, 512, 1, 1, 0, 0, 1))  # a 512x512 resident tile does not fit
    g.close()


@pytest.mark.parametrize("precond,degree", [("jacobi", 1), ("chebyshev", 3)])
def test_resident_tiles_match_global_tiles(precond, degree):
    """The same tiles with their vectors in shared memory (k_pcg_poisson_m2) and in global
    memory (k_pcg_poisson_m1) run the same arithmetic in the same order: equal iteration
    counts and fields to rounding."""
    case = _case(256, 128, precond, degree)
    res = ccm.Case(case)
    res.set_launch_plan(_plan(256, 128, 64, 16, 1))
    glob = ccm.Case(case)
    glob.set_launch_plan(_plan(256, 128, 64, 16, 0))
    st_r = res.step(3)
    st_g = glob.step(3)
    assert st_r["converged"] and st_g["converged"]
    assert st_r["iters_p"] == st_g["iters_p"]
    for f in (ccm.CCM_F_U, ccm.CCM_F_V, ccm.CCM_F_P):
        assert _rel(res.get_field(f), glob.get_field(f)) < 1e-12, f
    res.close()
    glob.close()
