"""Periodic box sides on the GPU (through the C ABI) against the oracle: the doubly periodic
Taylor-Green box and an x-periodic channel with a cylinder between no-slip walls.  Both have a
singular Poisson system (no outflow side), kept at zero mean (end of Sec. 4.6); face nx is
face 0 and the cells beyond a periodic side are the cells at the other end."""
import copy

import numpy as np
import pytest

from paper_2211_10698_gb300 import ccm, inputs as I

pytestmark = pytest.mark.gpu

OP_TOL = 1e-11


def _rel(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def _channel():
    return I.small_cylinder(nx=48, ny=24, box=(-2.0, 2.0, -1.0, 1.0), r=0.35, cx=0.1, cy=0.05,
                            bc=I.periodic_bc(True, False), re=50.0)


CASES = {"taylor_green": lambda: I.taylor_green(24), "channel": _channel}


@pytest.mark.parametrize("name", list(CASES))
def test_periodic_operators(orc, name):
    case = CASES[name]()
    o = orc.Oracle(case)
    g = ccm.Case(case)
    rng = np.random.default_rng(21)
    u, v, p = (rng.standard_normal(o.shape) for _ in range(3))
    assert _rel(g.apply(ccm.CCM_OP_CONT, *o.fill_ghosts(u, v), nout=1), o.cont(*o.fill_ghosts(u, v))) < OP_TOL
    gu, gv = g.apply(ccm.CCM_OP_PRES, p)
    ru, rv = o.pres_bc(p)
    assert _rel(gu, ru) < OP_TOL and _rel(gv, rv) < OP_TOL
    for op, ref in ((ccm.CCM_OP_CONV, o.conv_bc), (ccm.CCM_OP_VISC, o.visc_bc), (ccm.CCM_OP_HELMHOLTZ, o.helmholtz)):
        gu, gv = g.apply(op, u, v)
        ru, rv = ref(u, v)
        assert _rel(gu, ru) < OP_TOL and _rel(gv, rv) < OP_TOL, op
    assert _rel(g.apply(ccm.CCM_OP_POISSON, p, nout=1), o.poisson(p)) < OP_TOL
    assert _rel(g.apply(ccm.CCM_OP_POISSON_DIAG, nout=1), o.poisson_diag()) < 1e-12
    gu, gv = g.apply(ccm.CCM_OP_HELMHOLTZ_DIAG)
    du, dv = o.helmholtz_diag()
    assert _rel(gu, du) < 1e-12 and _rel(gv, dv) < 1e-12
    g.close()


def _start(o, g, case, name):
    if name == "taylor_green":
        u0, v0, _ = I.taylor_green_exact(case, 0.0)
    else:
        rng = np.random.default_rng(3)
        u0 = 0.3 + 0.1 * rng.standard_normal(o.shape)
        v0 = 0.1 * rng.standard_normal(o.shape)
    s = o.init_state(u0=0.0)
    s["u"], s["v"] = o.fill_ghosts(np.where(o.role_u == 3, u0, 0.0), np.where(o.role_v == 3, v0, 0.0))
    g.set_field(ccm.CCM_F_U, s["u"])
    g.set_field(ccm.CCM_F_V, s["v"])
    return s


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_periodic_steps(orc, name, precision):
    case = CASES[name]()
    case.tol_p = 1e-12 if precision == "mixed" else 1e-13
    case.tol_h = 1e-13
    case.precision = precision
    ocase = copy.deepcopy(case)
    ocase.tol_p = ocase.tol_h = 1e-13
    o = orc.Oracle(ocase)
    g = ccm.Case(case)
    s = _start(o, g, case, name)
    st = g.step(5)
    assert st["converged"]
    hist, _ = o.step(s, 5)
    tol = 1e-9 if precision == "fp64" else 1e-8
    # the library keeps P's periodic images in its ghost ring; the oracle's P carries none
    act = o.active
    for f, key, m in ((ccm.CCM_F_U, "u", np.ones(o.shape, bool)), (ccm.CCM_F_V, "v", np.ones(o.shape, bool)),
                      (ccm.CCM_F_P, "p", act)):
        e = _rel(g.get_field(f)[m], s[key][m])
        assert e < tol, (key, e)
    assert st["kinetic"] == pytest.approx(hist[-1]["kinetic"], rel=1e-10)
    g.close()


def test_periodic_momentum_conserved():
    """No wall in the doubly periodic box: the momentum sums stay at their initial values."""
    case = I.taylor_green(24)
    case.tol_p = case.tol_h = 1e-13
    g = ccm.Case(case)
    u0, v0, _ = I.taylor_green_exact(case, 0.0)
    g.set_field(ccm.CCM_F_U, u0 + 0.25)
    g.set_field(ccm.CCM_F_V, v0 - 0.1)
    a = g.step(1)
    b = g.step(10)
    assert abs(b["momentum_x"] - a["momentum_x"]) < 1e-11 * abs(a["momentum_x"])
    assert abs(b["momentum_y"] - a["momentum_y"]) < 1e-11 * abs(a["momentum_y"])
    assert abs(b["mass"]) < 1e-11 and b["max_div"] < 1e-10
    g.close()


def test_taylor_green_on_gpu(orc):
    """The Taylor-Green vortex to t = 1: the GPU's error against the exact solution equals the
    oracle's (same discretisation), and halves twice per halving of h."""
    errs = []
    for n in (24, 48):
        case = I.taylor_green(n)
        case.tol_p = case.tol_h = 1e-12
        g = ccm.Case(case)
        u0, v0, _ = I.taylor_green_exact(case, 0.0)
        g.set_field(ccm.CCM_F_U, u0)
        g.set_field(ccm.CCM_F_V, v0)
        nsteps = int(round(1.0 / case.dt))
        assert g.step(nsteps)["converged"]
        ue, ve, _ = I.taylor_green_exact(case, nsteps * case.dt)
        o = orc.Oracle(case)
        eu = np.abs(g.get_field(ccm.CCM_F_U) - ue)[o.role_u == 3].max()
        errs.append(eu)
        g.close()
    assert errs[0] / errs[1] > 3.3, errs
