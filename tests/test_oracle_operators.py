"""Pins for the oracle's discrete operators (Sec. 4.1-4.4) against identities of the
discrete calculus, the classical MAC formulas they reduce to away from the body, and
truncation order.  CPU only."""
import numpy as np
import pytest

import oracle as O
from paper_2211_10698_gb300 import inputs as I


def _cyl(nx=16, ny=8, bc=None, **kw):
    return I.small_cylinder(nx=nx, ny=ny, bc=bc, **kw)


def _closed(nx=12, ny=8, **kw):
    return I.small_cylinder(nx=nx, ny=ny, box=(-1.5, 1.5, -1.0, 1.0), r=0.41, cx=0.07, cy=-0.05,
                            bc=I.closed_box_bc(), **kw)


def _const(o, c):
    return np.full(o.shape, float(c))


@pytest.mark.parametrize("geom", ["circle", "naca"])
def test_free_stream_preserved(orc, geom):
    """Constant states are preserved near the boundary and away from it (Sec. 1, Sec. 2.1):
    cont(c, c) = 0, strain(c, c) = 0 and conv(c, c, c, c) = 0 for any geometry."""
    if geom == "circle":
        case = _cyl(24, 12)
    else:
        case = I.make_case("naca", 40, 20, (-0.5, 1.5, -0.5, 0.5),
                           I.Geometry(kind=I.GEOM_NACA, naca_tt=12, aoa_deg=9.0), re=100,
                           cfl=0.5, lref=1.0)
    o = orc.Oracle(case)
    cx, cy = 0.73, -0.41
    U, V = _const(o, cx), _const(o, cy)
    scale = max(case.hx, case.hy) * (abs(cx) + abs(cy))
    d = o.cont(U, V, U, V)
    assert np.abs(d).max() < 1e-14 * scale
    sxx, syy, sxy = o.strain(U, V, U, V)
    assert max(np.abs(sxx).max(), np.abs(syy).max(), np.abs(sxy).max()) < 1e-12 * (abs(cx) + abs(cy)) / min(case.hx, case.hy)
    cu, cv = o.conv(U, V, U, V, U, V, U, V)
    assert max(np.abs(cu).max(), np.abs(cv).max()) < 1e-14 * scale * (abs(cx) + abs(cy))
    # and the homogeneous part alone is NOT zero near the body (the D terms matter)
    assert np.abs(o.cont(U, V)).max() > 1e-3 * scale


def test_gradient_is_negative_transpose_of_divergence(orc):
    """Eq. compatibility: pres = -(d cont / d U)^T on the velocity unknowns, exactly."""
    case = _cyl(10, 6)
    o = orc.Oracle(case)
    unk = np.stack([o.role_u == 3, o.role_v == 3])
    cells = np.zeros(o.shape, bool)
    cells[1:-2, 1:-2] = True
    Dm = O.dense(lambda e: o.cont(e[0], e[1]), unk.shape, unk, cells)
    Gm = O.dense(lambda e: np.stack(o.pres_bc(e)), cells.shape, cells, unk)
    assert np.array_equal(Gm, -Dm.T)


def _div_free(o, seed):
    """A random velocity field made discretely divergence-free by the exact projection."""
    rng = np.random.default_rng(seed)
    u = rng.standard_normal(o.shape) * (o.role_u == 3)
    v = rng.standard_normal(o.shape) * (o.role_v == 3)
    act = o.active
    K = O.dense(o.poisson, o.shape, act, act)
    b = o.cont(u, v)[act]
    phi = np.zeros(o.shape)
    phi[act] = np.linalg.lstsq(K, -b, rcond=None)[0]
    gu, gv = o.pres_bc(phi)
    Vu, Vv = o.cap("u", "V"), o.cap("v", "V")
    u = u - np.where(Vu > 0, gu / np.where(Vu > 0, Vu, 1), 0)
    v = v - np.where(Vv > 0, gv / np.where(Vv > 0, Vv, 1), 0)
    u, v = o.fill_ghosts(u, v)
    assert np.abs(o.cont(u, v)).max() < 1e-12
    return u, v


def test_convection_skew_symmetric_for_divergence_free_field(orc):
    """Eqs. u-dot-qdm and kinetic: for a divergence-free U and no flux through the boundary
    (closed box, D = 0), w -> conv(U, w, 0, 0) is skew-symmetric on the velocity unknowns,
    so U^T conv(U, U) = 0."""
    case = _closed()
    o = orc.Oracle(case)
    u, v = _div_free(o, 3)
    unk = np.stack([o.role_u == 3, o.role_v == 3])

    def conv_w(e):
        wu, wv = e[0].copy(), e[1].copy()
        # homogeneous velocity boundary data for the transported field
        wu, wv = o.fill_ghosts(wu, wv)
        return np.stack(o.conv(u, v, wu, wv))

    C = O.dense(conv_w, unk.shape, unk, unk)
    assert np.abs(C + C.T).max() < 1e-13 * np.abs(C).max()
    cu, cv = o.conv(u, v)
    e = (u * cu * (o.role_u == 3)).sum() + (v * cv * (o.role_v == 3)).sum()
    assert abs(e) < 1e-13 * np.abs(C).max() * (u ** 2 + v ** 2).sum()


@pytest.mark.parametrize("bc", ["flow", "closed"])
def test_viscous_operator_symmetric_negative_semidefinite(orc, bc):
    """Sec. 4.3 / Sec. 1: the viscous operator visc(S(U)) is symmetric and dissipative.
    With one weight (W^xy + W^yx)/2 for both halves of Eq. offdiag (the reading used
    throughout) it is symmetric for any geometry, including the outflow box rules."""
    case = _cyl(12, 8) if bc == "flow" else _closed()
    o = orc.Oracle(case)
    unk = np.stack([o.role_u == 3, o.role_v == 3])
    H = O.dense(lambda e: np.stack(o.helmholtz(e[0], e[1])), unk.shape, unk, unk)
    M = np.diag(np.concatenate([o.cap("u", "V")[unk[0]], o.cap("v", "V")[unk[1]]]))
    L = ((case.rho / case.dt) * M - H) / case.mu
    assert np.abs(L - L.T).max() < 1e-12 * np.abs(L).max()
    w = np.linalg.eigvalsh(0.5 * (L + L.T))
    assert w.max() < 1e-12 * np.abs(w).max()
    assert np.linalg.eigvalsh(0.5 * (H + H.T)).min() > 0


def test_literal_offdiag_weights_are_not_symmetric_on_cut_cells(orc):
    """Eq. offdiag read literally (W^xy and W^yx separately) is symmetric only where the two
    weights agree; on a cut circle they differ, which is why the averaged weight is used."""
    case = _closed()
    case.literal_offdiag = 1
    o = orc.Oracle(case)
    unk = np.stack([o.role_u == 3, o.role_v == 3])
    H = O.dense(lambda e: np.stack(o.helmholtz(e[0], e[1])), unk.shape, unk, unk)
    asym = np.abs(H - H.T).max() / np.abs(H).max()
    assert asym > 1e-8
    Wxy, Wyx = o.cap("u", "WY"), o.cap("v", "WX")
    assert np.abs(Wxy - Wyx).max() > 1e-6


def _free(nx=10, ny=7, bc=None):
    return I.make_case("free", nx, ny, (0.0, 1.3, 0.0, 0.8), I.Geometry(), re=10, cfl=0.5,
                       lref=1.0, bc=bc)


def test_body_free_operators_are_classical_mac(orc):
    """Away from boundaries the cut-cell operators revert to the classical formulas
    (Sec. 2.3): cont = h_y d_x u + h_x d_y v, pres = A d P, conv = the Harlow-Welch
    divergence form, and 2 visc(S(U)) = vector Laplacian + d_x(cont)/h_x."""
    case = _free()
    o = orc.Oracle(case)
    hx, hy = case.hx, case.hy
    rng = np.random.default_rng(5)
    u, v = rng.standard_normal(o.shape), rng.standard_normal(o.shape)
    P = rng.standard_normal(o.shape)
    nx, ny = case.nx, case.ny
    U = lambda i, j: u[j + 1, i + 1]
    W = lambda i, j: v[j + 1, i + 1]
    d = o.cont(u, v)
    pu, pv = o.pres(P)
    cu, cv = o.conv(u, v)
    sxx, syy, sxy = o.strain(u, v)
    vu, vv = o.visc(sxx, syy, sxy)
    for j in range(ny):
        for i in range(nx):
            ref = hy * (U(i + 1, j) - U(i, j)) + hx * (W(i, j + 1) - W(i, j))
            assert o.at(d, i, j) == pytest.approx(ref, abs=1e-14)
    for j in range(ny):
        for i in range(nx + 1):
            assert o.at(pu, i, j) == pytest.approx(hy * (P[j + 1, i + 1] - P[j + 1, i]), abs=1e-14)
    for j in range(1, ny - 1):
        for i in range(1, nx):
            ue, uw = 0.5 * (U(i + 1, j) + U(i, j)), 0.5 * (U(i, j) + U(i - 1, j))
            vn, vs = 0.5 * (W(i, j + 1) + W(i - 1, j + 1)), 0.5 * (W(i, j) + W(i - 1, j))
            un, us = 0.5 * (U(i, j + 1) + U(i, j)), 0.5 * (U(i, j) + U(i, j - 1))
            ref = hy * (ue * ue - uw * uw) + hx * (vn * un - vs * us)
            assert o.at(cu, i, j) == pytest.approx(ref, abs=1e-13)
            lap = (hy / hx) * (U(i + 1, j) - 2 * U(i, j) + U(i - 1, j)) + \
                  (hx / hy) * (U(i, j + 1) - 2 * U(i, j) + U(i, j - 1))
            grad_div = (o.at(d, i, j) - o.at(d, i - 1, j)) / hx
            assert 2 * o.at(vu, i, j) == pytest.approx(lap + grad_div, abs=1e-12)
    for j in range(1, ny):
        for i in range(1, nx - 1):
            lap = (hy / hx) * (W(i + 1, j) - 2 * W(i, j) + W(i - 1, j)) + \
                  (hx / hy) * (W(i, j + 1) - 2 * W(i, j) + W(i, j - 1))
            grad_div = (o.at(d, i, j) - o.at(d, i, j - 1)) / hy
            assert 2 * o.at(vv, i, j) == pytest.approx(lap + grad_div, abs=1e-12)


def test_body_free_poisson_is_five_point(orc):
    """-cont(M^-1 pres Phi) on a body-free grid is the classical 5-point operator with
    homogeneous Neumann data on the inflow side and Dirichlet data on outflow sides
    (Sec. 4.6)."""
    case = _free()
    o = orc.Oracle(case)
    hx, hy = case.hx, case.hy
    phi = np.random.default_rng(2).standard_normal(o.shape)
    K = o.poisson(phi)
    nx, ny = case.nx, case.ny
    f = lambda i, j: phi[j + 1, i + 1] if (0 <= i < nx and 0 <= j < ny) else 0.0
    for j in range(ny):
        for i in range(nx):
            ax = hy / hx
            ay = hx / hy
            w = 0.0 if i == 0 else ax * (f(i, j) - f(i - 1, j))  # west inflow: no flux
            ref = ax * (f(i, j) - f(i + 1, j)) + w + ay * (2 * f(i, j) - f(i, j + 1) - f(i, j - 1))
            assert o.at(K, i, j) == pytest.approx(ref, abs=1e-13)


def _sample_velocity(case, fu, fv):
    """Point values of a smooth field at the u- and v-face centres (padded layout)."""
    ii = np.arange(-1, case.nx + 2)
    jj = np.arange(-1, case.ny + 2)
    xu = case.x0 + ii * case.hx
    yu = case.y0 + (jj + 0.5) * case.hy
    xv = case.x0 + (ii + 0.5) * case.hx
    yv = case.y0 + jj * case.hy
    Xu, Yu = np.meshgrid(xu, yu)
    Xv, Yv = np.meshgrid(xv, yv)
    return fu(Xu, Yu), fv(Xv, Yv), (Xu, Yu, Xv, Yv)


def test_body_free_second_order_truncation(orc):
    """On a uniform body-free grid, conv / V and visc(2S) / V approximate div(u u) and
    div(2 s) at second order (the classical second-order formulas, Sec. 1)."""
    k = 2.0
    fu = lambda x, y: np.sin(k * x) * np.cos(y)
    fv = lambda x, y: np.cos(x) * np.sin(k * y) + 0.3
    # exact: d(uu)/dx + d(uv)/dy at u-faces; lap u + d/dx(div) for div(2s)
    ux = lambda x, y: k * np.cos(k * x) * np.cos(y)
    uy = lambda x, y: -np.sin(k * x) * np.sin(y)
    vx = lambda x, y: -np.sin(x) * np.sin(k * y)
    vy = lambda x, y: k * np.cos(x) * np.cos(k * y)
    conv_x = lambda x, y: 2 * fu(x, y) * ux(x, y) + uy(x, y) * fv(x, y) + fu(x, y) * vy(x, y)
    # div(2s)_x = 2 u_xx + u_yy + v_xy
    divs_x = lambda x, y: 2 * (-k * k * np.sin(k * x) * np.cos(y)) + (-np.sin(k * x) * np.cos(y)) + \
        (-k * np.sin(x) * np.cos(k * y))
    errs_c, errs_v = [], []
    for n in (16, 32, 64):
        case = I.make_case("free", n, n, (0.0, 1.0, 0.0, 1.0), I.Geometry(), re=10, cfl=0.5, lref=1.0)
        o = orc.Oracle(case)
        u, v, (Xu, Yu, _, _) = _sample_velocity(case, fu, fv)
        cu, _ = o.conv(u, v)
        sxx, syy, sxy = o.strain(u, v)
        vu, _ = o.visc(sxx, syy, sxy)
        A = case.hx * case.hy
        sl = (slice(3, -3), slice(3, -3))
        errs_c.append(np.abs(cu[sl] / A - conv_x(Xu, Yu)[sl]).max())
        errs_v.append(np.abs(2 * vu[sl] / A - divs_x(Xu, Yu)[sl]).max())
    for e in (errs_c, errs_v):
        assert 3.5 < e[0] / e[1] < 4.5 and 3.5 < e[1] / e[2] < 4.5, e
