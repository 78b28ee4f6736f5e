"""The body-force term rho V g of Eq. pm_prediction through the C ABI: forced steps equal the
oracle's forced steps, and on the manufactured steady solution in a closed no-slip box the
library's steady state converges to the exact fields at second order (FP64 and mixed)."""
import numpy as np
import pytest

import oracle as O
from paper_2211_10698_gb300 import ccm, inputs as I

pytestmark = pytest.mark.gpu

STEP_TOL = 1e-9


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2211_10698_gb300 import build

    build.build()


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("name,precision", [("cylinder", "fp64"), ("mms", "fp64"), ("cylinder", "mixed")])
def test_forced_steps_match_oracle(name, precision):
    if name == "cylinder":
        case = I.small_cylinder(nx=64, ny=32, box=(-2.0, 6.0, -2.0, 2.0), r=0.5, cx=0.0, cy=0.1, re=60.0)
        rng = np.random.default_rng(17)
        gx, gy = 0.3 * rng.standard_normal(case.shape), 0.3 * rng.standard_normal(case.shape)
    else:
        case = I.mms_box(48)
        _, _, _, gx, gy = I.mms_fields(case)
    case.tol_p = case.tol_h = 1e-13
    case.precision = precision
    o = O.Oracle(case)
    g = ccm.Case(case)
    s = o.init_state(u0=case.bc_un[0])
    if name == "mms":
        g.set_field(ccm.CCM_F_U, s["u"])
    s["gx"], s["gy"] = gx, gy
    g.set_field(ccm.CCM_F_GX, gx)
    g.set_field(ccm.CCM_F_GY, gy)
    assert np.array_equal(g.get_field(ccm.CCM_F_GX), gx)
    gs = g.step(4)
    o.step(s, 4)
    assert gs["converged"]
    tol = STEP_TOL if precision == "fp64" else 1e-8
    for f, ref in ((ccm.CCM_F_U, s["u"]), (ccm.CCM_F_V, s["v"]), (ccm.CCM_F_P, s["p"])):
        assert rel(g.get_field(f), ref) < tol, f


def _steady(n, precision="fp64", T=2.5):
    case = I.mms_box(n)
    case.precision = precision
    g = ccm.Case(case)
    ue, ve, pe, gx, gy = I.mms_fields(case)
    g.set_field(ccm.CCM_F_U, ue)
    g.set_field(ccm.CCM_F_V, ve)
    g.set_field(ccm.CCM_F_P, pe)
    g.set_field(ccm.CCM_F_GX, gx)
    g.set_field(ccm.CCM_F_GY, gy)
    nsteps = int(round(T / case.dt))
    g.step(nsteps - 1)
    u_prev = g.get_field(ccm.CCM_F_U)
    st = g.step(1)
    assert st["converged"]
    u, v, p = (g.get_field(f) for f in (ccm.CCM_F_U, ccm.CCM_F_V, ccm.CCM_F_P))
    o = O.Oracle(case)
    act = o.active
    p = p - p[act].mean()
    pe = pe - pe[act].mean()
    return dict(du=np.abs(u - u_prev).max(), eu=np.abs(u - ue)[o.role_u == 3].max(),
                ev=np.abs(v - ve)[o.role_v == 3].max(), ep=np.abs(p - pe)[act].max(), u=u, v=v, p=p)


def test_manufactured_solution_second_order_on_the_device():
    """Steady states at 32, 64 and 128 cells: the error falls by 4 per halving of h, and the
    32-cell state is the oracle's (same discrete steady equations)."""
    r = [_steady(n) for n in (32, 64, 128)]
    for x in r:
        assert x["du"] < 1e-9
    for a, b in zip(r, r[1:]):
        assert 3.6 < a["eu"] / b["eu"] < 4.4
        assert 3.6 < a["ev"] / b["ev"] < 4.4
        assert 3.4 < a["ep"] / b["ep"] < 4.6
    assert r[0]["eu"] == pytest.approx(3.194e-3, rel=2e-3)   # the oracle's steady error at 32 cells


def test_manufactured_solution_mixed_precision():
    """The mixed-precision step (FP32 CG with FP64 residual replacements to the same 1e-10)
    reaches the FP64 step's steady state."""
    a, b = _steady(64, "fp64"), _steady(64, "mixed")
    assert b["du"] < 1e-8
    assert rel(b["u"], a["u"]) < 1e-8 and rel(b["v"], a["v"]) < 1e-8
    assert abs(b["eu"] - a["eu"]) < 1e-3 * a["eu"]
