"""Pins for the oracle on stretched rectilinear meshes (Sec. 3.1: arbitrary abscissas
x_0 < ... < x_nx; the paper's grids G1-G3 are stretched).  The staggered grids of Sec. 3.4
have their cells centred on the faces, so the u-grid's x-lines are the centres of the
pressure cells; beyond the box the spacing mirrors the spacing inside it.  CPU only."""
import copy
import math

import numpy as np
import pytest

import oracle as O
from paper_2211_10698_gb300 import inputs as I

from tests.test_oracle_capacities import _clip_rect, _wet_interval


def _random_faces(rng, n, a, b, spread=0.6):
    h = rng.uniform(1.0 - spread, 1.0 + spread, n)
    x = a + np.concatenate([[0.0], np.cumsum(h)]) * (b - a) / h.sum()
    x[-1] = b
    return x


def _lines(f, staggered):
    """Grid lines -1 .. n+2 of a grid, built here independently of the oracle: faces mirrored
    beyond both ends, or (staggered) the midpoints of consecutive faces."""
    n = len(f) - 1
    ext = np.concatenate([2 * f[0] - f[2:0:-1], f, 2 * f[-1] - f[-2:-4:-1]])  # faces -2 .. n+2
    face = lambda k: ext[k + 2]
    if staggered:
        return {i: 0.5 * (face(i - 1) + face(i)) for i in range(-1, n + 3)}
    return {i: face(i) for i in range(-1, n + 3)}


@pytest.mark.parametrize("seed", range(4))
def test_stretched_halfplane_closed_form(orc, seed):
    """A straight boundary on a randomly stretched mesh: every capacity of Sec. 3 equals its
    definition evaluated in closed form on the cell's own lines, on all three grids."""
    rng = np.random.default_rng(2000 + seed)
    th = rng.uniform(0, 2 * np.pi)
    n = (math.cos(th), math.sin(th))
    nx, ny = 7, 6
    box = (-1.0, 1.2, -0.7, 0.9)
    xf, yf = _random_faces(rng, nx, box[0], box[1]), _random_faces(rng, ny, box[2], box[3])
    off = n[0] * 0.1 + n[1] * 0.1 + rng.uniform(-0.3, 0.3)
    g = I.Geometry(kind=I.GEOM_HALFPLANE, hp_nx=n[0], hp_ny=n[1], hp_off=off)
    case = I.make_case("hp_s", nx, ny, box, g, re=10, cfl=0.5, lref=1.0, xf=xf, yf=yf)
    o = orc.Oracle(case)
    hmax = max(np.diff(xf).max(), np.diff(yf).max())
    tol_a, tol_l = 1e-13 * hmax * hmax, 1e-13 * hmax
    for grid in "puv":
        Lx, Ly = _lines(xf, grid == "u"), _lines(yf, grid == "v")

        def cell(i, j):
            return Lx[i], Lx[i + 1], Ly[j], Ly[j + 1]

        def centroid(i, j):
            xl, xr, yb, yt = cell(i, j)
            a, c = _clip_rect(xl, xr, yb, yt, n, off)
            return (a, c) if a > 0 else (0.0, (0.5 * (xl + xr), 0.5 * (yb + yt)))

        for j in range(0, ny + 2):
            for i in range(0, nx + 2):
                xl, xr, yb, yt = cell(i, j)
                V, (X, Y) = centroid(i, j)
                kap = max(1.0, (xr - xl) * (yt - yb) / V) if V > 0 else 1.0
                Vl, (Xl, _) = centroid(i - 1, j)
                Vb, (_, Yb) = centroid(i, j - 1)
                kapw = max(kap, hmax * hmax / Vl if Vl > 0 else 1.0, hmax * hmax / Vb if Vb > 0 else 1.0)
                assert abs(o.at(o.cap(grid, "V"), i, j) - V) <= tol_a, (grid, i, j)
                assert abs(o.at(o.cap(grid, "X"), i, j) - X) <= tol_l * kap
                assert abs(o.at(o.cap(grid, "Y"), i, j) - Y) <= tol_l * kap
                assert abs(o.at(o.cap(grid, "AX"), i, j) - _wet_interval(yb, yt, xl, 0, n, off)) <= tol_l
                assert abs(o.at(o.cap(grid, "AY"), i, j) - _wet_interval(xl, xr, yb, 1, n, off)) <= tol_l
                Bx = _wet_interval(yb, yt, X, 0, n, off) if V > 0 else 0.0
                By = _wet_interval(xl, xr, Y, 1, n, off) if V > 0 else 0.0
                assert abs(o.at(o.cap(grid, "BX"), i, j) - Bx) <= tol_l * kap
                assert abs(o.at(o.cap(grid, "BY"), i, j) - By) <= tol_l * kap
                Wx, _ = _clip_rect(Xl, X, yb, yt, n, off)
                Wy, _ = _clip_rect(xl, xr, Yb, Y, n, off)
                assert abs(o.at(o.cap(grid, "WX"), i, j) - Wx) <= tol_a * kapw, (grid, i, j)
                assert abs(o.at(o.cap(grid, "WY"), i, j) - Wy) <= tol_a * kapw, (grid, i, j)


def test_stretched_worked_example(orc):
    """The worked example of Sec. 2.3 with unequal cells: a mesh-aligned wall inside cell 1 at
    distance 2f from its right face, cells of widths h_1, h_2, h_3.  Capacities V_1 = 2 f h_y,
    W_{1/2} = f h_y, W_{3/2} = g h_y with g = f + h_2/2, W_{5/2} = (h_2 + h_3)/2 h_y, and the
    gradients Q_{1/2} = (T_1 - D_1)/f, Q_{3/2} = (T_2 - T_1)/g, Q_{5/2} = (T_3 - T_2)/((h_2+h_3)/2)
    on the u-grid (whose cells are centred on the faces)."""
    hy, f = 0.7, 0.23
    xf = np.array([0.0, 0.9, 1.7, 2.8, 3.4, 4.6, 5.1])
    # the u-grid's cell k+1 spans the centres of p-cells k and k+1; the wall sits in u-cell 2
    Lx = _lines(xf, True)
    xw = Lx[3] - 2 * f
    assert Lx[2] < xw < Lx[3]
    g_ = I.Geometry(kind=I.GEOM_HALFPLANE, hp_nx=1.0, hp_ny=0.0, hp_off=xw)
    case = I.make_case("worked_s", 6, 4, (0.0, 5.1, 0.0, 4 * hy), g_, re=10, cfl=0.5, lref=1.0, xf=xf,
                       yf=hy * np.arange(5.0))
    o = orc.Oracle(case)
    h = {k: Lx[k + 2] - Lx[k + 1] for k in (1, 2, 3)}  # paper cell k = u-cell k+1
    gg = f + 0.5 * h[2]
    at = lambda name, k: o.at(o.cap("u", name), k + 1, 1)
    assert at("V", 0) == 0.0
    assert at("V", 1) == pytest.approx(2 * f * hy, rel=1e-13)
    assert at("V", 2) == pytest.approx(h[2] * hy, rel=1e-13)
    assert at("WX", 1) == pytest.approx(f * hy, rel=1e-13)
    assert at("WX", 2) == pytest.approx(gg * hy, rel=1e-13)
    assert at("WX", 3) == pytest.approx(0.5 * (h[2] + h[3]) * hy, rel=1e-13)
    rng = np.random.default_rng(8)
    T = rng.standard_normal(case.nx + 3)
    D = rng.standard_normal(case.nx + 3)
    u = np.tile(T, (case.ny + 3, 1))
    Dx = np.tile(D, (case.ny + 3, 1))
    z = o.z()
    sxx, _, _ = o.strain(u, z, Dx, z)
    t = lambda k: T[k + 2]
    d = lambda k: D[k + 2]
    assert o.at(sxx, 1, 1) == pytest.approx((t(1) - d(1)) / f, rel=1e-12)
    assert o.at(sxx, 2, 1) == pytest.approx((t(2) - t(1)) / gg, rel=1e-12)
    assert o.at(sxx, 3, 1) == pytest.approx((t(3) - t(2)) / (0.5 * (h[2] + h[3])), rel=1e-12)


def test_stretched_volume_sum_equals_box_minus_polygon(orc):
    """A circle on a stretched mesh: the fluid volume over the interior cells is the box minus
    the polygon through the circle's crossings with the grid lines (exact for marching squares
    when no cell holds more than one boundary segment)."""
    case = I.stretched_cylinder(nx=40, ny=30, box=(-3.0, 5.0, -3.0, 3.0), fine=(16, 16), h_fine=0.1, ratio=1.1)
    o = orc.Oracle(case)
    xf, yf = case.faces_x(), case.faces_y()
    r = case.geom.r
    pts = []
    for x in xf:
        if abs(x) < r:
            s = math.sqrt(r * r - x * x)
            pts += [(x, s), (x, -s)]
    for y in yf:
        if abs(y) < r:
            s = math.sqrt(r * r - y * y)
            pts += [(s, y), (-s, y)]
    pts.sort(key=lambda p: math.atan2(p[1], p[0]))
    P = np.array(pts)
    poly = 0.5 * abs(np.sum(P[:, 0] * np.roll(P[:, 1], -1) - np.roll(P[:, 0], -1) * P[:, 1]))
    V = o.cap("p", "V")[1:-2, 1:-2].sum()
    box = (xf[-1] - xf[0]) * (yf[-1] - yf[0])
    assert abs(V - (box - poly)) <= 1e-12 * box
    assert abs(poly - math.pi * r * r) < 0.02 * math.pi * r * r


def test_stretched_uniform_spacing_reproduces_the_uniform_mesh(orc):
    """Abscissas that happen to be equally spaced give the uniform mesh's capacities (to the
    rounding of the line coordinates)."""
    case = I.small_cylinder(nx=16, ny=8)
    s = copy.deepcopy(case)
    s.xf, s.yf = case.faces_x(), case.faces_y()
    a, b = orc.Oracle(case), orc.Oracle(s)
    assert np.abs(a.caps - b.caps).max() < 1e-13


def _stretched_small():
    return I.stretched_cylinder(nx=14, ny=10, box=(-2.0, 3.0, -1.6, 1.6), fine=(6, 4), h_fine=0.2, ratio=1.15,
                                r=0.37)


def test_stretched_compatibility_and_symmetry(orc):
    """G = -D^T bitwise (Eq. compatibility), K symmetric positive definite and the Helmholtz
    operator symmetric on a stretched mesh with a cut circle."""
    case = _stretched_small()
    o = orc.Oracle(case)
    act = o.active
    ru, rv = o.role_u == 3, o.role_v == 3
    Dm_u = O.dense(lambda u: o.cont(u, o.z()), o.shape, ru, act)
    Dm_v = O.dense(lambda v: o.cont(o.z(), v), o.shape, rv, act)
    Gu = O.dense(lambda p: o.pres(p)[0], o.shape, act, ru)
    Gv = O.dense(lambda p: o.pres(p)[1], o.shape, act, rv)
    assert np.array_equal(Gu, -Dm_u.T) and np.array_equal(Gv, -Dm_v.T)
    K = O.dense(o.poisson, o.shape, act, act)
    assert np.abs(K - K.T).max() <= 1e-14 * np.abs(K).max()
    assert np.linalg.eigvalsh(K).min() > 0
    mask = np.concatenate([ru.ravel(), rv.ravel()])

    def helm(x):
        n = o.shape[0] * o.shape[1]
        a, b = o.helmholtz(x[:n].reshape(o.shape), x[n:].reshape(o.shape))
        return np.concatenate([a.ravel(), b.ravel()])

    H = O.dense(helm, (2 * o.shape[0] * o.shape[1],), mask, mask)
    assert np.abs(H - H.T).max() <= 1e-12 * np.abs(H).max()


def test_stretched_free_stream_preserved(orc):
    """A constant state with D = that constant leaves cont, strain and conv at zero
    (free-stream preservation) on a stretched mesh with a body."""
    case = _stretched_small()
    o = orc.Oracle(case)
    c = np.full(o.shape, 0.8)
    d = np.full(o.shape, -0.3)
    assert np.abs(o.cont(c, d, c, d)).max() < 1e-13
    sxx, syy, sxy = o.strain(c, d, c, d)
    assert max(np.abs(sxx).max(), np.abs(syy).max(), np.abs(sxy).max()) < 1e-12
    cu, cv = o.conv(c, d, c, d, c, d, c, d)
    assert max(np.abs(cu).max(), np.abs(cv).max()) < 1e-12


def test_body_free_stretched_poisson_is_five_point(orc):
    """Without a body the Poisson rows are the textbook five-point operator of a non-uniform
    MAC mesh: sum over the faces of (face length / distance between the two centres) times
    the difference of the values (Eq. pm_poisson with the mass matrix of Eq. semidiscrete)."""
    rng = np.random.default_rng(4)
    nx, ny = 9, 7
    xf, yf = _random_faces(rng, nx, 0.0, 1.3), _random_faces(rng, ny, -0.2, 0.8)
    case = I.make_case("bf_s", nx, ny, (0.0, 1.3, -0.2, 0.8), I.Geometry(kind=I.GEOM_NONE), re=10, cfl=0.5,
                       lref=1.0, xf=xf, yf=yf, bc=I.closed_box_bc())
    o = orc.Oracle(case)
    phi = rng.standard_normal(o.shape)
    Kp = o.poisson(phi)
    xc, yc = 0.5 * (xf[1:] + xf[:-1]), 0.5 * (yf[1:] + yf[:-1])
    hx, hy = np.diff(xf), np.diff(yf)
    for j in range(ny):
        for i in range(nx):
            s = 0.0
            P = lambda a, b: phi[b + 1, a + 1]
            if i > 0:
                s += hy[j] / (xc[i] - xc[i - 1]) * (P(i, j) - P(i - 1, j))
            if i < nx - 1:
                s += hy[j] / (xc[i + 1] - xc[i]) * (P(i, j) - P(i + 1, j))
            if j > 0:
                s += hx[i] / (yc[j] - yc[j - 1]) * (P(i, j) - P(i, j - 1))
            if j < ny - 1:
                s += hx[i] / (yc[j + 1] - yc[j]) * (P(i, j) - P(i, j + 1))
            assert o.at(Kp, i, j) == pytest.approx(s, rel=1e-12, abs=1e-12)


def _smooth_faces(n, eps=0.35):
    xi = np.linspace(0.0, 1.0, n + 1)
    return xi - eps / (2 * np.pi) * np.sin(2 * np.pi * xi)


def _mms_stretched_error(orc, n, T=2.5):
    case = I.mms_box(n)
    case.xf, case.yf = _smooth_faces(n), _smooth_faces(n)
    case.dt = 0.5 * case.hx
    o = orc.Oracle(case)
    ue, ve, pe, gx, gy = I.mms_fields(case)
    st = o.init_state(u0=0.0)
    st["u"][:] = np.where(o.role_u == 3, ue, 0.0)
    st["v"][:] = np.where(o.role_v == 3, ve, 0.0)
    st["gx"], st["gy"] = gx, gy
    nsteps = int(round(T / case.dt))
    hist, _ = o.step(st, nsteps)
    assert hist[-1]["ok"]
    act = o.active
    p = st["p"] - st["p"][act].mean()
    pe = pe - pe[act].mean()
    return dict(eu=np.abs(st["u"] - ue)[o.role_u == 3].max(), ev=np.abs(st["v"] - ve)[o.role_v == 3].max(),
                ep=np.abs(p - pe)[act].max())


def test_manufactured_solution_on_smoothly_stretched_mesh(orc):
    """The manufactured steady solution of the closed box on a smoothly stretched mesh (spacing
    ratio about 2 between the coarsest and finest cells): second order (measured error ratios
    3.99 in u and v, 3.65 in P from 16 to 32 cells; 3.99 and 3.91 from 32 to 64)."""
    a, b = _mms_stretched_error(orc, 16), _mms_stretched_error(orc, 32)
    assert b["eu"] < 5e-3 and b["ev"] < 5e-3 and b["ep"] < 1.5e-2
    assert a["eu"] / b["eu"] > 3.6 and a["ev"] / b["ev"] > 3.6
    assert a["ep"] / b["ep"] > 3.3
