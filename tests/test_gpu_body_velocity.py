"""The body's steady Dirichlet velocity D through the C ABI (Eqs. divergence, diag/offdiag and
convective with D): steps equal the oracle's, a body moving with the stream leaves it
undisturbed, the force includes D's strain, and the vortex around a rotating cylinder is
reached at first order."""
import numpy as np
import pytest

import oracle as O
from paper_2211_10698_gb300 import ccm, inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2211_10698_gb300 import build

    build.build()


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _cyl():
    return I.small_cylinder(nx=64, ny=32, box=(-2.0, 6.0, -2.0, 2.0), r=0.5, cx=0.03, cy=0.02, re=80.0)


def _rotation(o, case, omega):
    """D = omega x (x - c) at the boundary points of the u- and v-control volumes."""
    g = case.geom
    xu, yu = I.circle_boundary_points(o.cap("u", "X"), o.cap("u", "Y"), g.cx, g.cy, g.r)
    xv, yv = I.circle_boundary_points(o.cap("v", "X"), o.cap("v", "Y"), g.cx, g.cy, g.r)
    return -omega * (yu - g.cy), omega * (xv - g.cx)


def test_body_moving_with_the_stream_on_the_device():
    case = _cyl()
    g = ccm.Case(case)
    g.set_field(ccm.CCM_F_DX, np.full(case.shape, case.u_inf))
    g.set_field(ccm.CCM_F_DY, np.zeros(case.shape))
    g.step(3)
    o = O.Oracle(case)
    u, v, p = (g.get_field(f) for f in (ccm.CCM_F_U, ccm.CCM_F_V, ccm.CCM_F_P))
    assert np.abs(u - case.u_inf)[o.role_u == 3].max() < 1e-12
    assert np.abs(v)[o.role_v == 3].max() < 1e-12
    assert np.abs(p).max() < 1e-12


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_rotating_cylinder_steps_match_oracle(precision):
    case = _cyl()
    case.tol_p = case.tol_h = 1e-13
    case.precision = precision
    o = O.Oracle(case)
    Dx, Dy = _rotation(o, case, 1.5)
    g = ccm.Case(case)
    g.set_field(ccm.CCM_F_DX, Dx)
    g.set_field(ccm.CCM_F_DY, Dy)
    assert np.array_equal(g.get_field(ccm.CCM_F_DX), Dx)
    s = o.init_state()
    s["Dx"], s["Dy"] = Dx, Dy
    s["u"][o.role_u == 2] = Dx[o.role_u == 2]
    s["v"][o.role_v == 2] = Dy[o.role_v == 2]
    gs = g.step(4)
    hist, extra = o.step(s, 4, keep=True)
    assert gs["converged"]
    tol = 1e-9 if precision == "fp64" else 1e-8
    for f, ref in ((ccm.CCM_F_U, s["u"]), (ccm.CCM_F_V, s["v"]), (ccm.CCM_F_P, s["p"]),
                   (ccm.CCM_F_USTAR, extra["ustar"]), (ccm.CCM_F_DIV, extra["b"])):
        assert rel(g.get_field(f), ref) < tol, f
    assert gs["max_div"] == pytest.approx(hist[-1]["max_div"], rel=1e-3, abs=1e-12)
    # the force includes the strain of D; it matches the oracle's on the device's state
    u, v, p = (g.get_field(f) for f in (ccm.CCM_F_U, ccm.CCM_F_V, ccm.CCM_F_P))
    want = o.body_force(u, v, p, Dx, Dy)
    got = g.body_force()
    assert np.abs(got - want).max() < 1e-11 * np.abs(want).max()
    assert abs(o.body_force(u, v, p)[2] - want[2]) > 1e-3 * abs(want[2])   # D's strain matters


def _vortex(n):
    case = I.vortex_box(n)
    g = ccm.Case(case)
    ue, ve, gx, gy = I.vortex_fields(case)
    Dx, Dy = I.vortex_body_velocity(case, g.cap("u", "X"), g.cap("u", "Y"), g.cap("v", "X"), g.cap("v", "Y"))
    g.set_field(ccm.CCM_F_DX, Dx)
    g.set_field(ccm.CCM_F_DY, Dy)
    g.set_field(ccm.CCM_F_U, ue)
    g.set_field(ccm.CCM_F_V, ve)
    g.set_field(ccm.CCM_F_GX, gx)
    g.set_field(ccm.CCM_F_GY, gy)
    st = g.step(int(round(2.5 / case.dt)))
    assert st["converged"]
    o = O.Oracle(case)
    u, v = g.get_field(ccm.CCM_F_U), g.get_field(ccm.CCM_F_V)
    return np.abs(u - ue)[o.role_u == 3].max(), np.abs(v - ve)[o.role_v == 3].max()


def test_rotating_cylinder_vortex_first_order_on_the_device():
    """The oracle's error at 32 cells (1.030e-2) and first-order decay up to 128 cells."""
    e = [_vortex(n) for n in (32, 64, 128)]
    assert e[0][0] == pytest.approx(1.030e-2, rel=5e-3)
    for a, b in zip(e, e[1:]):
        assert a[0] / b[0] > 1.6 and a[1] / b[1] > 1.6
