"""One-launch mixed-precision Poisson solve (FP32 CG on the Jacobi-scaled system with FP64
residual replacements) and the FP64 solve on the scaled system: FP64 residual target met,
iteration counts close to FP64 Jacobi-PCG, independence from the scale of the right-hand
side, warm starts, and the iteration limit."""
import numpy as np
import pytest

from paper_2211_10698_gb300 import ccm, inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2211_10698_gb300 import build

    build.build()


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _case(nx=256, ny=128, precision="mixed", tol=1e-10):
    c = I.small_cylinder(nx=nx, ny=ny, box=(-2.0, 6.0, -2.0, 2.0), r=0.5, cx=0.0, cy=0.0, re=40.0)
    c.precision = precision
    c.precond = "jacobi"
    c.tol_p = tol
    return c


@pytest.mark.parametrize("nx,ny", [(128, 64), (512, 256)])
def test_mixed_iterations_close_to_fp64(nx, ny):
    c64 = _case(nx, ny, "fp64")
    cmx = _case(nx, ny, "mixed")
    rhs = np.random.default_rng(3).standard_normal(c64.shape)
    g64 = ccm.Case(c64)
    gmx = ccm.Case(cmx)
    s64 = g64.solve_pressure(rhs)
    smx = gmx.solve_pressure(rhs)
    assert s64["converged"] and smx["converged"]
    assert smx["rel_res"] <= 1e-10 and s64["rel_res"] <= 1e-10
    assert smx["outer"] >= 2  # FP64 residual replacements
    assert smx["iters"] <= 1.6 * s64["iters"] + 20, (smx, s64)
    # both solutions satisfy the same system to the tolerance: cond(K) * 1e-10 apart at most
    assert _rel(gmx.get_field(ccm.CCM_F_PHI), g64.get_field(ccm.CCM_F_PHI)) < 1e-5


@pytest.mark.parametrize("scale", [2.0 ** -100, 2.0 ** 100])
def test_mixed_scale_of_rhs_exact(scale):
    """FP32 values are normalised at every replacement: scaling the right-hand side by a power
    of two changes no FP32 value, so the iteration is the same and the solution scales
    exactly, whatever the magnitude."""
    c = _case(128, 64)
    rhs = np.random.default_rng(4).standard_normal(c.shape)
    g1 = ccm.Case(c)
    s1 = g1.solve_pressure(rhs)
    g2 = ccm.Case(c)
    s2 = g2.solve_pressure(rhs * scale)
    assert s1["converged"] and s2["converged"]
    assert s1["iters"] == s2["iters"] and s1["outer"] == s2["outer"]
    assert np.array_equal(g2.get_field(ccm.CCM_F_PHI), g1.get_field(ccm.CCM_F_PHI) * scale)


@pytest.mark.parametrize("scale", [1e-30, 1e30])
def test_mixed_scale_of_rhs(scale):
    """Far outside FP32's range the solve converges the same way; rounding of the scaled
    values changes the FP32 trajectory, so the iteration count may differ a little."""
    c = _case(128, 64)
    rhs = np.random.default_rng(4).standard_normal(c.shape)
    g1 = ccm.Case(c)
    s1 = g1.solve_pressure(rhs)
    g2 = ccm.Case(c)
    s2 = g2.solve_pressure(rhs * scale)
    assert s1["converged"] and s2["converged"] and s2["rel_res"] <= 1e-10
    assert abs(s1["iters"] - s2["iters"]) <= 0.15 * s1["iters"]
    assert _rel(g2.get_field(ccm.CCM_F_PHI) / scale, g1.get_field(ccm.CCM_F_PHI)) < 1e-8


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_warm_start(precision):
    c = _case(128, 64, precision)
    rhs = np.random.default_rng(5).standard_normal(c.shape)
    g = ccm.Case(c)
    s1 = g.solve_pressure(rhs)
    phi = g.get_field(ccm.CCM_F_PHI)
    s2 = g.solve_pressure(rhs)  # starts from the converged solution
    assert s1["converged"] and s2["converged"]
    assert s2["iters"] <= 2
    assert _rel(g.get_field(ccm.CCM_F_PHI), phi) < 1e-9


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_iteration_limit(precision):
    c = _case(128, 64, precision)
    c.max_iter_p = 25
    rhs = np.random.default_rng(6).standard_normal(c.shape)
    g = ccm.Case(c)
    st = g.solve_pressure(rhs)
    assert not st["converged"] and st["iters"] == 25
    assert 0.0 < st["rel_res"] < 1.0  # progress kept, state usable
    c.max_iter_p = 20000
    g2 = ccm.Case(c)
    g2.set_field(ccm.CCM_F_PHI, g.get_field(ccm.CCM_F_PHI))
    st2 = g2.solve_pressure(rhs)
    assert st2["converged"]
