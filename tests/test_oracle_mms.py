"""Step accuracy of the oracle on a manufactured steady solution (body free, closed no-slip
box), driven by the body-force term rho V g of Eq. pm_prediction: the steady state the PmII
step relaxes to converges to the exact velocity and pressure at second order.  The forcing's
hand-derived derivatives are checked against finite differences first.  CPU only."""
import numpy as np
import pytest

from paper_2211_10698_gb300 import inputs as I


def test_manufactured_forcing_matches_finite_differences():
    """g = (U.grad)U + grad p / rho - nu lap U, with every derivative checked by central
    differences of the exact fields; U is divergence free."""
    rng = np.random.default_rng(3)
    x, y = rng.uniform(0.05, 0.95, 50), rng.uniform(0.05, 0.95, 50)
    rho, mu, e = 1.3, 0.2, 1e-4
    f = lambda a, b: I.mms_exact(a, b, rho, mu)
    u, v, p, gx, gy = f(x, y)
    d = lambda k, dx, dy: (f(x + dx, y + dy)[k] - f(x - dx, y - dy)[k]) / (2 * max(dx, dy))
    dd = lambda k, dx, dy: (f(x + dx, y + dy)[k] - 2 * f(x, y)[k] + f(x - dx, y - dy)[k]) / max(dx, dy) ** 2
    ux, uy, vx, vy = d(0, e, 0), d(0, 0, e), d(1, e, 0), d(1, 0, e)
    px, py = d(2, e, 0), d(2, 0, e)
    lu = dd(0, 1e-3, 0) + dd(0, 0, 1e-3)
    lv = dd(1, 1e-3, 0) + dd(1, 0, 1e-3)
    nu = mu / rho
    assert np.abs(ux + vy).max() < 1e-7
    assert np.abs(gx - (u * ux + v * uy + px / rho - nu * lu)).max() < 1e-4
    assert np.abs(gy - (u * vx + v * vy + py / rho - nu * lv)).max() < 1e-4


def _steady_error(orc, n, T=2.5):
    case = I.mms_box(n)
    o = orc.Oracle(case)
    ue, ve, pe, gx, gy = I.mms_fields(case)
    st = o.init_state(u0=0.0)
    st["u"][:] = np.where(o.role_u == 3, ue, 0.0)
    st["v"][:] = np.where(o.role_v == 3, ve, 0.0)
    st["p"][:] = np.where(o.active, pe, 0.0)
    st["gx"], st["gy"] = gx, gy
    nsteps = int(round(T / case.dt))
    o.step(st, nsteps - 1)
    u_prev = st["u"].copy()
    hist, _ = o.step(st, 1)
    assert hist[-1]["ok"]
    act = o.active
    p = st["p"] - st["p"][act].mean()
    pe = pe - pe[act].mean()
    return dict(du=np.abs(st["u"] - u_prev).max(),
                eu=np.abs(st["u"] - ue)[o.role_u == 3].max(),
                ev=np.abs(st["v"] - ve)[o.role_v == 3].max(),
                ep=np.abs(p - pe)[act].max())


def test_manufactured_solution_converges_at_second_order(orc):
    """Body free, the discrete operators are the textbook MAC ones (second order), so the steady
    state's error falls by 4 per halving of h in velocity and pressure (measured: 3.95 and 3.85
    from 16 to 32 cells, 3.99 and 3.96 from 32 to 64)."""
    a, b = _steady_error(orc, 16), _steady_error(orc, 32)
    for r in (a, b):
        assert r["du"] < 1e-9                      # steady
    assert b["eu"] < 4e-3 and b["ev"] < 4e-3 and b["ep"] < 5e-3
    assert 3.6 < a["eu"] / b["eu"] < 4.4
    assert 3.6 < a["ev"] / b["ev"] < 4.4
    assert 3.4 < a["ep"] / b["ep"] < 4.6


def test_forcing_enters_as_rho_V_g(orc):
    """The predictor right-hand side with g differs from the one without by rho V g exactly, on
    the velocity unknowns only."""
    case = I.small_cylinder(nx=24, ny=12, rho=1.7)
    o = orc.Oracle(case)
    st = o.init_state()
    rng = np.random.default_rng(9)
    gx, gy = rng.standard_normal(o.shape), rng.standard_normal(o.shape)
    import ctypes
    from oracle import _p
    outs = []
    for g in ((None, None), (gx, gy)):
        ru, rv, cu, cv = o.z(), o.z(), o.z(), o.z()
        o.lib.orc_predictor_rhs_g(ctypes.byref(o.s), _p(o.caps), _p(st["u"].copy()), _p(st["v"].copy()),
                                  _p(st["p"]), _p(o.z()), _p(o.z()), 1, _p(g[0]), _p(g[1]), _p(ru), _p(rv),
                                  _p(cu), _p(cv))
        outs.append((ru, rv))
    du = outs[1][0] - outs[0][0]
    dv = outs[1][1] - outs[0][1]
    want_u = np.where(o.role_u == 3, case.rho * o.cap("u", "V") * gx, 0.0)
    want_v = np.where(o.role_v == 3, case.rho * o.cap("v", "V") * gy, 0.0)
    assert np.allclose(du, want_u, rtol=1e-12, atol=1e-14)
    assert np.allclose(dv, want_v, rtol=1e-12, atol=1e-14)
