"""Pins for the oracle with periodic box sides (the all-periodic or periodic-and-wall boxes whose
Poisson system is singular, end of Sec. 4.6: the constants are its null space and the iterates
are kept at zero mean).  Face nx is face 0 and the cells beyond a periodic side are the cells
at the other end.  CPU only."""
import copy
import math

import numpy as np
import pytest

import oracle as O
from paper_2211_10698_gb300 import inputs as I


def _tg(n, nu=0.05):
    return I.taylor_green(n, nu=nu)


def _divfree(o, rng, scale=1.0):
    """A discretely divergence-free periodic field from a random periodic streamfunction at the
    nodes: u = delta_y psi, v = -delta_x psi (uniform square cells, no body)."""
    n, m = o.case.nx, o.case.ny
    psi = rng.standard_normal((m, n)) * scale
    u, v = o.z(), o.z()
    for j in range(m):
        for i in range(n):
            o.at(u, i, j)  # index check
            u[j + 1, i + 1] = psi[(j + 1) % m, i] - psi[j, i]
            v[j + 1, i + 1] = -(psi[j, (i + 1) % n] - psi[j, i])
    return o.fill_ghosts(u, v)


def test_periodic_operators_structure(orc):
    """G = -D^T bitwise (Eq. compatibility), K symmetric positive semidefinite with exactly the
    constants as null space, the probed diagonals equal the dense ones, the Helmholtz operator
    symmetric positive definite, on a doubly periodic box and an x-periodic channel with a
    cylinder."""
    for case in (_tg(12), I.small_cylinder(nx=24, ny=12, box=(-2.0, 2.0, -1.0, 1.0), r=0.35, cx=0.1,
                                           bc=I.periodic_bc(True, False))):
        o = orc.Oracle(case)
        act = o.active
        ru, rv = o.role_u == 3, o.role_v == 3
        Dm_u = O.dense(lambda u: o.cont(*o.fill_ghosts(u, o.z())), o.shape, ru, act)
        Dm_v = O.dense(lambda v: o.cont(*o.fill_ghosts(o.z(), v)), o.shape, rv, act)
        Gu = O.dense(lambda p: o.pres_bc(p)[0], o.shape, act, ru)
        Gv = O.dense(lambda p: o.pres_bc(p)[1], o.shape, act, rv)
        assert np.array_equal(Gu, -Dm_u.T) and np.array_equal(Gv, -Dm_v.T)
        K = O.dense(o.poisson, o.shape, act, act)
        assert np.abs(K - K.T).max() <= 1e-14 * np.abs(K).max()
        w = np.linalg.eigvalsh(K)
        assert abs(w[0]) < 1e-12 * w[-1] and w[1] > 1e-6 * w[-1]
        assert np.abs(K @ np.ones(K.shape[0])).max() < 1e-12 * np.abs(K).max()
        assert np.abs(np.diag(K) - o.poisson_diag()[act]).max() < 1e-14 * np.abs(K).max()
        mask = np.concatenate([ru.ravel(), rv.ravel()])
        N = o.shape[0] * o.shape[1]

        def helm(x):
            a, b = o.helmholtz(x[:N].reshape(o.shape), x[N:].reshape(o.shape))
            return np.concatenate([a.ravel(), b.ravel()])

        H = O.dense(helm, (2 * N,), mask, mask)
        assert np.abs(H - H.T).max() <= 1e-12 * np.abs(H).max()
        assert np.linalg.eigvalsh(H).min() > 0
        du, dv = o.helmholtz_diag()
        assert np.abs(np.diag(H) - np.concatenate([du.ravel(), dv.ravel()])[mask]).max() < 1e-12 * np.abs(H).max()


def test_periodic_convection_conserves_energy(orc):
    """For a discretely divergence-free U in the doubly periodic box, U^T conv(U) = 0 (Eqs.
    u-dot-qdm and kinetic: the convective term neither creates nor destroys kinetic energy)."""
    case = _tg(12)
    o = orc.Oracle(case)
    rng = np.random.default_rng(3)
    u, v = _divfree(o, rng)
    assert np.abs(o.cont(u, v)[o.active]).max() < 1e-13
    cu, cv = o.conv_bc(u, v)
    ru, rv = o.role_u == 3, o.role_v == 3
    e = (u[ru] * cu[ru]).sum() + (v[rv] * cv[rv]).sum()
    scale = np.abs(u[ru] * cu[ru]).sum() + np.abs(v[rv] * cv[rv]).sum()
    assert abs(e) < 1e-13 * scale


def test_periodic_steps_conserve_mass_and_momentum(orc):
    """Steps of a random divergence-free flow in the doubly periodic box: every cell divergence
    stays at the solver tolerance and the momentum sums stay at their initial values (no wall
    takes momentum; convection, pressure and viscosity telescope)."""
    case = _tg(12, nu=0.02)
    case.tol_p = case.tol_h = 1e-13
    o = orc.Oracle(case)
    rng = np.random.default_rng(5)
    u, v = _divfree(o, rng, 0.3)
    u += 0.4 * (o.role_u == 3)  # a mean flow
    u, v = o.fill_ghosts(u, v)
    st = o.init_state(u0=0.0)
    st["u"], st["v"] = u, v
    m0 = o.conservation(u, v)
    hist, _ = o.step(st, 8)
    assert all(h["ok"] for h in hist)
    m1 = o.conservation(st["u"], st["v"])
    assert abs(m1[0]) < 1e-12
    assert abs(m1[1] - m0[1]) < 1e-12 * abs(m0[1]) and abs(m1[2] - m0[2]) < 1e-11
    assert hist[-1]["max_div"] < 1e-11


def _tg_error(orc, n, T=1.0):
    case = _tg(n)
    case.tol_p = case.tol_h = 1e-12
    o = orc.Oracle(case)
    u0, v0, _ = I.taylor_green_exact(case, 0.0)
    st = o.init_state(u0=0.0)
    st["u"], st["v"] = o.fill_ghosts(np.where(o.role_u == 3, u0, 0.0), np.where(o.role_v == 3, v0, 0.0))
    nsteps = int(round(T / case.dt))
    hist, _ = o.step(st, nsteps)
    assert all(h["ok"] for h in hist)
    t = nsteps * case.dt
    ue, ve, pe = I.taylor_green_exact(case, t)
    act = o.active
    p = st["p"] - st["p"][act].mean()
    return (np.abs(st["u"] - ue)[o.role_u == 3].max(), np.abs(st["v"] - ve)[o.role_v == 3].max(),
            np.abs(p - (pe - pe[act].mean()))[act].max())


def test_taylor_green_second_order(orc):
    """The Taylor-Green vortex (an exact solution) decays at the right rate: the error of u and
    v at t = 1 falls by about four per halving of h (dt in proportion)."""
    a, b = _tg_error(orc, 12), _tg_error(orc, 24)
    assert b[0] < 5e-3 and b[1] < 5e-3
    assert a[0] / b[0] > 3.3 and a[1] / b[1] > 3.3
