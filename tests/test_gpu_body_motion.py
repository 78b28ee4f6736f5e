"""A body velocity that changes in time, through the C ABI (ccm_set_body_motion, Sec. 4.6: D^n in
conv^n and S^n, D^{n+1} in S* and in cont(U*, D^{n+1})): steps from rest equal the oracle's two-
level steps, a constant factor equals the steady D, the velocity is second order in time, and
batches refuse such a case."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2211_10698_gb300 import ccm, inputs as I

pytestmark = pytest.mark.gpu

MOTION = (0.5, 0.5, 4.0 * math.pi, -0.5 * math.pi)  # f = (1 - cos(omega t)) / 2: from rest


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2211_10698_gb300 import build

    build.build()


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _case(nsub, T=0.5, precision="fp64"):
    case = I.small_cylinder(nx=32, ny=32, box=(-1.0, 1.0, -1.0, 1.0), r=0.37, cx=0.03, cy=-0.02,
                            re=50.0, bc=I.flow_past_body_bc(0.0))
    case.mu = 0.02
    case.dt = T / nsub
    case.tol_p = case.tol_h = 1e-13
    case.autotune = 0
    case.precision = precision
    return case


def _d0(o):
    case = o.case
    args = (o.cap("u", "X"), o.cap("u", "Y"), o.cap("v", "X"), o.cap("v", "Y"), case.geom.cx, case.geom.cy,
            case.geom.r)
    ax, ay = I.rotation_velocity(*args, omega=2.0)
    bx, by = I.transpiration_velocity(*args, w=0.3)
    return ax + bx, ay + by


def _device(case, Dx, Dy, motion=MOTION):
    g = ccm.Case(case)
    g.set_field(ccm.CCM_F_U, np.zeros(case.shape))
    g.set_field(ccm.CCM_F_V, np.zeros(case.shape))
    g.set_field(ccm.CCM_F_DX, Dx)
    g.set_field(ccm.CCM_F_DY, Dy)
    if motion is not None:
        g.set_body_motion(*motion)
    return g


def _oracle_start(o, Dx, Dy, motion=MOTION):
    st = o.init_state(u0=0.0)
    st["Dx"], st["Dy"], st["motion"] = Dx, Dy, motion
    f0 = I.body_motion_factor(motion, 0, o.case.dt)
    st["u"][o.role_u == 2] = f0 * Dx[o.role_u == 2]
    st["v"][o.role_v == 2] = f0 * Dy[o.role_v == 2]
    return st


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_moving_wall_steps_match_oracle(precision):
    """12 steps of a cylinder wall that turns and blows with a factor ramping from rest: U, V, P,
    U* and cont(U*, D^{n+1}) equal the oracle's two-level steps (1e-9 FP64, 1e-8 mixed), the
    reported max |cont(U^{n+1}, D^{n+1})| is the oracle's, and the force includes the strain of
    the present level's D."""
    case = _case(40, precision=precision)
    o = O.Oracle(case)
    Dx, Dy = _d0(o)
    g = _device(case, Dx, Dy)
    s = _oracle_start(o, Dx, Dy)
    gs = g.step(12)
    hist, extra = o.step(s, 12, keep=True)
    assert gs["converged"] and all(h["ok"] for h in hist)
    tol = 1e-9 if precision == "fp64" else 1e-8
    for f, ref in ((ccm.CCM_F_U, s["u"]), (ccm.CCM_F_V, s["v"]), (ccm.CCM_F_P, s["p"]),
                   (ccm.CCM_F_USTAR, extra["ustar"]), (ccm.CCM_F_DIV, extra["b"])):
        assert rel(g.get_field(f), ref) < tol, f
    assert gs["max_div"] < 1e-10 and hist[-1]["max_div"] < 1e-10
    f1 = I.body_motion_factor(MOTION, 12, case.dt)
    u, v, p = (g.get_field(f) for f in (ccm.CCM_F_U, ccm.CCM_F_V, ccm.CCM_F_P))
    want = o.body_force(u, v, p, f1 * Dx, f1 * Dy)
    got = g.body_force()
    assert np.abs(got - want).max() < 1e-11 * np.abs(want).max()
    g.close()


def test_constant_factor_equals_steady_body_velocity():
    """f = a0 with a1 = 0 is D = a0 D0 bit for bit; a0 = 1, a1 = 0 is the steady path itself."""
    case = _case(40)
    o = O.Oracle(case)
    Dx, Dy = _d0(o)
    a = _device(case, Dx, Dy, motion=(0.6, 0.0, 1.0, 0.3))
    b = _device(case, 0.6 * Dx, 0.6 * Dy, motion=None)
    c = _device(case, Dx, Dy, motion=(1.0, 0.0, 5.0, 0.0))
    d = _device(case, Dx, Dy, motion=None)
    for h in (a, b, c, d):
        h.step(5)
    for f in (ccm.CCM_F_U, ccm.CCM_F_V, ccm.CCM_F_P):
        assert rel(a.get_field(f), b.get_field(f)) < 1e-13, f
        assert np.array_equal(c.get_field(f), d.get_field(f)), f
    for h in (a, b, c, d):
        h.close()


def test_moving_wall_second_order_in_time_on_the_device():
    """The device's velocity at T = 0.5 converges at second order in dt (ratio > 3.2 per halving)."""
    res = {}
    for n in (20, 40, 80, 160):
        case = _case(n)
        o = O.Oracle(case)
        Dx, Dy = _d0(o)
        g = _device(case, Dx, Dy)
        assert g.step(n)["converged"]
        res[n] = (g.get_field(ccm.CCM_F_U), g.get_field(ccm.CCM_F_V))
        g.close()
    mu_, mv_ = o.role_u == 3, o.role_v == 3
    for comp, m in ((0, mu_), (1, mv_)):
        e = [np.sqrt(np.mean((res[a][comp] - res[b][comp])[m] ** 2)) for a, b in ((20, 40), (40, 80), (80, 160))]
        assert e[0] / e[1] > 3.2 and e[1] / e[2] > 3.2, (comp, e)


def test_batch_refuses_a_moving_body():
    case = _case(40)
    o = O.Oracle(case)
    Dx, Dy = _d0(o)
    g = _device(case, Dx, Dy)
    b = ccm.Batch(4)
    with pytest.raises(ccm.CcmError, match="not batched"):
        b.add(g)
    b.close()
    g.close()
