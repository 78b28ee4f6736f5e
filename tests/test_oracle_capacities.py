"""Pins for the oracle's capacities (Sec. 3) against closed forms, the paper's worked example
(Sec. 2.3) and geometric invariants.  CPU only."""
import math

import numpy as np
import pytest

from paper_2211_10698_gb300 import inputs as I


def _clip_rect(xl, xr, yb, yt, n, off):
    """Independent reference: the part of the rectangle where n.x > off, by clipping the
    four corners against the line (a general convex clip, not marching squares)."""
    pts = [(xl, yb), (xr, yb), (xr, yt), (xl, yt)]
    out = []
    f = lambda p: n[0] * p[0] + n[1] * p[1] - off
    for k in range(4):
        a, b = pts[k], pts[(k + 1) % 4]
        fa, fb = f(a), f(b)
        if fa > 0:
            out.append(a)
        if (fa > 0) != (fb > 0):
            t = fa / (fa - fb)
            out.append((a[0] + t * (b[0] - a[0]), a[1] + t * (b[1] - a[1])))
    if len(out) < 3:
        return 0.0, None
    x = np.array([p[0] for p in out])
    y = np.array([p[1] for p in out])
    cr = x * np.roll(y, -1) - np.roll(x, -1) * y
    area = 0.5 * cr.sum()
    if area <= 0:
        return 0.0, None
    cx = ((x + np.roll(x, -1)) * cr).sum() / (6 * area)
    cy = ((y + np.roll(y, -1)) * cr).sum() / (6 * area)
    return area, (cx, cy)


def _wet_interval(a, b, fixed, axis, n, off):
    """Length of {s in [a,b] : n.x > off} on the line x = fixed (axis 0) or y = fixed."""
    if axis == 0:
        c0, c1 = n[0] * fixed - off, n[1]
    else:
        c0, c1 = n[1] * fixed - off, n[0]
    # c0 + c1 * s > 0
    if c1 == 0:
        return (b - a) if c0 > 0 else 0.0
    s0 = -c0 / c1
    if c1 > 0:
        lo = max(a, s0)
        return max(0.0, b - lo)
    hi = min(b, s0)
    return max(0.0, hi - a)


@pytest.mark.parametrize("seed", range(6))
def test_halfplane_closed_form(orc, seed):
    """Marching squares is exact for a straight boundary: every capacity of Sec. 3 equals
    its definition evaluated in closed form (Eqs. volumefirstkind, centroid,
    surfacefirstkindx/y, volumesecondkindx/y, surfacesecondkindx/y)."""
    rng = np.random.default_rng(1000 + seed)
    th = rng.uniform(0, 2 * np.pi)
    n = (math.cos(th), math.sin(th))
    nx, ny = 7, 5
    box = (-1.0, 1.0 + 0.17 * seed, -0.6, 0.9)
    cx, cy = 0.5 * (box[0] + box[1]), 0.5 * (box[2] + box[3])
    off = n[0] * cx + n[1] * cy + rng.uniform(-0.3, 0.3)
    g = I.Geometry(kind=I.GEOM_HALFPLANE, hp_nx=n[0], hp_ny=n[1], hp_off=off)
    case = I.make_case("hp", nx, ny, box, g, re=10, cfl=0.5, lref=1.0)
    o = orc.Oracle(case)
    hx, hy = case.hx, case.hy
    tol_a = 1e-13 * hx * hy
    tol_l = 1e-13 * max(hx, hy)
    for gi, grid in enumerate("puv"):
        ox = -0.5 * hx if grid == "u" else 0.0
        oy = -0.5 * hy if grid == "v" else 0.0

        def cell(i, j):
            xl = case.x0 + ox + i * hx
            yb = case.y0 + oy + j * hy
            return xl, xl + hx, yb, yb + hy

        def centroid(i, j):
            xl, xr, yb, yt = cell(i, j)
            a, c = _clip_rect(xl, xr, yb, yt, n, off)
            return (a, c) if a > 0 else (0.0, (0.5 * (xl + xr), 0.5 * (yb + yt)))

        for j in range(-1, ny + 2):
            for i in range(-1, nx + 2):
                xl, xr, yb, yt = cell(i, j)
                V, (X, Y) = centroid(i, j)
                # a sliver's centroid carries a rounding error ~ eps h^3 / V
                kap = max(1.0, hx * hy / V) if V > 0 else 1.0
                _, (Xl, _) = centroid(i - 1, j)
                _, (_, Yb) = centroid(i, j - 1)
                Vl, Vb = centroid(i - 1, j)[0], centroid(i, j - 1)[0]
                kapw = max(kap, hx * hy / Vl if Vl > 0 else 1.0, hx * hy / Vb if Vb > 0 else 1.0)
                assert abs(o.at(o.cap(grid, "V"), i, j) - V) <= tol_a
                assert abs(o.at(o.cap(grid, "X"), i, j) - X) <= tol_l * kap
                assert abs(o.at(o.cap(grid, "Y"), i, j) - Y) <= tol_l * kap
                assert abs(o.at(o.cap(grid, "AX"), i, j) - _wet_interval(yb, yt, xl, 0, n, off)) <= tol_l
                assert abs(o.at(o.cap(grid, "AY"), i, j) - _wet_interval(xl, xr, yb, 1, n, off)) <= tol_l
                Bx = _wet_interval(yb, yt, X, 0, n, off) if V > 0 else 0.0
                By = _wet_interval(xl, xr, Y, 1, n, off) if V > 0 else 0.0
                assert abs(o.at(o.cap(grid, "BX"), i, j) - Bx) <= tol_l * kap
                assert abs(o.at(o.cap(grid, "BY"), i, j) - By) <= tol_l * kap
                # second-kind volumes: fluid between neighbouring centroids
                Wx, _ = _clip_rect(Xl, X, yb, yt, n, off)
                Wy, _ = _clip_rect(xl, xr, Yb, Y, n, off)
                assert abs(o.at(o.cap(grid, "WX"), i, j) - Wx) <= tol_a * kapw, (grid, i, j)
                assert abs(o.at(o.cap(grid, "WY"), i, j) - Wy) <= tol_a * kapw, (grid, i, j)


def _worked_example_case(hx=1.0, hy=0.7, f=0.3, grid="p"):
    """Sec. 2.3 configuration: a mesh-aligned wall inside cell 1 with fluid to the right,
    V_1 = 2 f h_y.  For grid 'p' cell k is p-cell k; for grid 'u' it is u-cell k+1."""
    shift = 0.0 if grid == "p" else 0.5 * hx
    x_w = 2 * hx - 2 * f + shift
    g = I.Geometry(kind=I.GEOM_HALFPLANE, hp_nx=1.0, hp_ny=0.0, hp_off=x_w)
    return I.make_case("worked", 6, 4, (0.0, 6 * hx, 0.0, 4 * hy), g, re=10, cfl=0.5, lref=1.0), x_w


def test_worked_example_capacities(orc):
    """The capacities listed for the worked example (Sec. 2.3): V_0=0, V_1=2f h_y,
    V_2=h_x h_y, A_{-1/2}=A_{1/2}=0, A_{3/2}=A_{5/2}=h_y, B_0=0, B_1=B_2=h_y, W_{-1/2}=0,
    W_{1/2}=f h_y, W_{3/2}=g h_y, W_{5/2}=h_x h_y, with g the distance between the
    centroids of cells 1 and 2."""
    hx, hy, f = 1.0, 0.7, 0.3
    g = hx / 2 + f
    for grid, k0 in (("p", 0), ("u", 1)):
        case, _ = _worked_example_case(hx, hy, f, grid)
        o = orc.Oracle(case)
        V, A, B, W = (o.cap(grid, n) for n in ("V", "AX", "BX", "WX"))
        j = 1
        at = lambda a, k: o.at(a, k0 + k, j)
        assert at(V, 0) == 0.0
        assert at(V, 1) == pytest.approx(2 * f * hy, abs=1e-15)
        assert at(V, 2) == pytest.approx(hx * hy, abs=1e-15)
        assert at(A, 0) == 0.0 and at(A, 1) == 0.0          # A_{-1/2}, A_{1/2}
        assert at(A, 2) == pytest.approx(hy) and at(A, 3) == pytest.approx(hy)
        assert at(B, 0) == 0.0
        assert at(B, 1) == pytest.approx(hy) and at(B, 2) == pytest.approx(hy)
        assert at(W, 0) == 0.0                              # W_{-1/2}
        assert at(W, 1) == pytest.approx(f * hy, abs=1e-15)  # W_{1/2}
        assert at(W, 2) == pytest.approx(g * hy, abs=1e-15)  # W_{3/2}
        assert at(W, 3) == pytest.approx(hx * hy, abs=1e-15)  # W_{5/2}


def test_worked_example_gradient_and_poisson_rows(orc):
    """Eq. gradD reproduces Q_{1/2}=(T_1-D_1)/f, Q_{3/2}=(T_2-T_1)/g, Q_{5/2}=(T_3-T_2)/h_x,
    and div(Q,Q) = sum B delta Q (Eq. divD) the Poisson rows 0=0,
    h_y((T_2-T_1)/g-(T_1-D)/f) and h_y((T_3-T_2)/h_x-(T_2-T_1)/g) (Sec. 2.3).
    Checked on the u-grid, where the strain operator (Eq. diag) is Eq. gradD and the
    viscous operator (Sec. 4.3) is Eq. divD."""
    hx, hy, f = 1.0, 0.7, 0.3
    g = hx / 2 + f
    case, _ = _worked_example_case(hx, hy, f, "u")
    o = orc.Oracle(case)
    rng = np.random.default_rng(7)
    T = rng.standard_normal(case.nx + 3)
    D = rng.standard_normal(case.nx + 3)
    u = np.tile(T, (case.ny + 3, 1))
    Dx = np.tile(D, (case.ny + 3, 1))
    z = o.z()
    sxx, syy, sxy = o.strain(u, z, Dx, z)
    t = lambda k: T[(k + 1) + 1]  # paper cell k = u-face k+1 -> array column k+2
    d = lambda k: D[(k + 1) + 1]
    for j in range(case.ny):
        # S_xx at p-cell k+1 is the paper's Q_{k+1/2}
        assert o.at(sxx, 1, j) == pytest.approx((t(1) - d(1)) / f, rel=1e-13)
        assert o.at(sxx, 2, j) == pytest.approx((t(2) - t(1)) / g, rel=1e-13)
        assert o.at(sxx, 3, j) == pytest.approx((t(3) - t(2)) / hx, rel=1e-13)
    assert np.abs(sxy).max() < 1e-12 * np.abs(sxx).max()
    vu, _ = o.visc(sxx, syy, sxy)
    for j in range(case.ny):
        assert o.at(vu, 1, j) == 0.0
        assert o.at(vu, 2, j) == pytest.approx(hy * ((t(2) - t(1)) / g - (t(1) - d(1)) / f), rel=1e-12)
        assert o.at(vu, 3, j) == pytest.approx(hy * ((t(3) - t(2)) / hx - (t(2) - t(1)) / g), rel=1e-12)


def _circle_crossings(case, ox, oy):
    """All intersections of the circle with the lines of the grid shifted by (ox, oy), for
    edges whose end points differ in fluid status; asserts that no edge is crossed twice."""
    g = case.geom
    r2 = g.r ** 2
    fl = lambda x, y: (x - g.cx) ** 2 + (y - g.cy) ** 2 > r2
    pts = []
    xs = [case.x0 + ox + i * case.hx for i in range(-1, case.nx + 3)]
    ys = [case.y0 + oy + j * case.hy for j in range(-1, case.ny + 3)]
    for x in xs:
        d = r2 - (x - g.cx) ** 2
        if d <= 0:
            continue
        for y in (g.cy - math.sqrt(d), g.cy + math.sqrt(d)):
            k = math.floor((y - ys[0]) / case.hy)
            ya, yb = ys[k], ys[k + 1]
            assert fl(x, ya) != fl(x, yb), "edge crossed twice; choose other parameters"
            pts.append((x, y))
    for y in ys:
        d = r2 - (y - g.cy) ** 2
        if d <= 0:
            continue
        for x in (g.cx - math.sqrt(d), g.cx + math.sqrt(d)):
            k = math.floor((x - xs[0]) / case.hx)
            xa, xb = xs[k], xs[k + 1]
            assert fl(xa, y) != fl(xb, y), "edge crossed twice; choose other parameters"
            pts.append((x, y))
    return np.array(pts)


@pytest.mark.parametrize("grid", ["p", "u", "v"])
def test_circle_volume_is_box_minus_inscribed_polygon(orc, grid):
    """Sum of V over the padded grid = padded-box area - area of the polygon through the
    boundary crossings taken in angular order (marching squares joins consecutive
    crossings by straight segments)."""
    case = I.small_cylinder(nx=32, ny=16, r=0.6, cx=0.031, cy=-0.047)
    o = orc.Oracle(case)
    ox = -0.5 * case.hx if grid == "u" else 0.0
    oy = -0.5 * case.hy if grid == "v" else 0.0
    P = _circle_crossings(case, ox, oy)
    ang = np.arctan2(P[:, 1] - case.geom.cy, P[:, 0] - case.geom.cx)
    P = P[np.argsort(ang)]
    x, y = P[:, 0], P[:, 1]
    poly = 0.5 * (x * np.roll(y, -1) - np.roll(x, -1) * y).sum()
    box = (case.nx + 3) * case.hx * (case.ny + 3) * case.hy
    assert o.cap(grid, "V").sum() == pytest.approx(box - poly, rel=0, abs=1e-12)


def test_circle_area_second_order(orc):
    """The solid area seen by the capacities converges to pi r^2 at second order."""
    errs = []
    for n in (32, 64, 128):
        case = I.small_cylinder(nx=n, ny=n // 2, r=0.61, cx=0.031, cy=-0.047)
        o = orc.Oracle(case)
        box = (case.nx + 3) * case.hx * (case.ny + 3) * case.hy
        errs.append(abs(box - o.cap("p", "V").sum() - math.pi * 0.61 ** 2))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.0 < r1 < 5.5 and 3.0 < r2 < 5.5, errs


@pytest.mark.parametrize("geom", ["circle", "naca"])
def test_surface_conservation_law(orc, geom):
    """Eq. approximate: A^+ - A^- = -n_x |Gamma| (and the same in y) in every cell."""
    if geom == "circle":
        case = I.small_cylinder(nx=24, ny=12)
    else:
        case = I.make_case("naca", 40, 20, (-0.5, 1.5, -0.5, 0.5),
                           I.Geometry(kind=I.GEOM_NACA, naca_tt=12, aoa_deg=7.0), re=100, cfl=0.5,
                           lref=1.0)
    o = orc.Oracle(case)
    for grid in "puv":
        Ax, Ay = o.cap(grid, "AX"), o.cap(grid, "AY")
        for j in range(-1, case.ny + 1):
            for i in range(-1, case.nx + 1):
                nxl, nyl = o.cell_boundary(grid, i, j)
                assert o.at(Ax, i + 1, j) - o.at(Ax, i, j) == pytest.approx(-nxl, abs=1e-14)
                assert o.at(Ay, i, j + 1) - o.at(Ay, i, j) == pytest.approx(-nyl, abs=1e-14)


def test_naca_area_converges(orc):
    """The solid area of a NACA00tt section approaches 10 t c^2 * integral of the thickness
    polynomial (closed trailing edge)."""
    t = 0.12
    integral = 0.2969 * 2 / 3 - 0.1260 / 2 - 0.3516 / 3 + 0.2843 / 4 - 0.1036 / 5
    exact = 10 * t * integral
    errs = []
    for n in (64, 128, 256):
        case = I.make_case("naca", n, n // 2, (-0.5, 1.5, -0.5, 0.5),
                           I.Geometry(kind=I.GEOM_NACA, naca_tt=12, aoa_deg=4.0), re=100, cfl=0.5,
                           lref=1.0)
        o = orc.Oracle(case)
        box = (case.nx + 3) * case.hx * (case.ny + 3) * case.hy
        errs.append(abs(box - o.cap("p", "V").sum() - exact) / exact)
    assert errs[2] < errs[1] < errs[0] and errs[2] < 2e-3, errs


def test_capacity_bounds_and_full_cells(orc):
    """0 <= capacities <= full values; cells away from the body have the full values."""
    case = I.small_cylinder(nx=24, ny=12)
    o = orc.Oracle(case)
    hx, hy = case.hx, case.hy
    for grid in "puv":
        # cell edges come from the grid-line formula, so widths match hx, hy to a few ulps
        assert (o.cap(grid, "V") >= 0).all() and (o.cap(grid, "V") <= hx * hy * (1 + 1e-13)).all()
        for nm, full in (("AX", hy), ("BX", hy), ("AY", hx), ("BY", hx)):
            a = o.cap(grid, nm)
            assert (a >= 0).all() and (a <= full * (1 + 1e-13)).all()
        # ring of cells two away from the box edge: full
        V = o.cap(grid, "V")
        assert np.allclose(V[:3, :], hx * hy, rtol=1e-13, atol=0)
        assert np.allclose(V[-3:, :], hx * hy, rtol=1e-13, atol=0)
