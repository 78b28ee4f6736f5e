"""Pins for the oracle's force on the body.  The paper reports drag and lift (Sec. 5) without
a discrete definition; the oracle takes the body's share of the momentum that pres(P) and
visc(2 mu S) give the fluid.  These checks tie that definition to closed forms (a closed body
under uniform pressure, a linear pressure field, plane Couette flow over a mesh-aligned wall)
and to the discrete operators themselves (for fields that vanish near the box, the force is
the sum of pres and visc over every velocity position).  CPU only."""
import math

import numpy as np
import pytest

from paper_2211_10698_gb300 import inputs as I


def _cyl(nx, ny, r=0.5, **kw):
    return I.make_case("cyl", nx, ny, (-2.0, 2.0, -1.5, 1.5),
                       I.Geometry(kind=I.GEOM_CIRCLE, cx=0.031, cy=-0.047, r=r), re=100.0, cfl=0.5,
                       lref=2 * r, **kw)


def _naca(nx, ny, **kw):
    return I.make_case("naca", nx, ny, (-0.5, 1.5, -0.6, 0.6),
                       I.Geometry(kind=I.GEOM_NACA, naca_tt=12, aoa_deg=7.0), re=500.0, cfl=0.5,
                       lref=1.0, **kw)


def _wall(nx=12, ny=8, jw=3):
    """Fluid above the mesh-aligned horizontal wall y = y0 + jw hy."""
    box = (0.0, 1.5, 0.0, 1.0)
    yw = box[2] + jw * (box[3] - box[2]) / ny
    g = I.Geometry(kind=I.GEOM_HALFPLANE, hp_nx=0.0, hp_ny=1.0, hp_off=yw)
    return I.make_case("wall", nx, ny, box, g, re=20.0, cfl=0.5, lref=1.0), yw


def _centres(case):
    """Cell-centre abscissas and ordinates on the padded layout (index i+1, j+1)."""
    i = np.arange(-1, case.nx + 2)
    j = np.arange(-1, case.ny + 2)
    xc = case.x0 + (i + 0.5) * case.hx
    yc = case.y0 + (j + 0.5) * case.hy
    return np.broadcast_to(xc[None, :], case.shape).copy(), np.broadcast_to(yc[:, None], case.shape).copy()


def test_uniform_pressure_on_closed_body_gives_no_force(orc):
    """A closed body under uniform pressure feels no net force: every row and column of
    A-differences telescopes to the wet box faces at both ends."""
    case = _cyl(48, 36)
    o = orc.Oracle(case)
    p0 = 3.7
    f = o.body_force(o.z(), o.z(), np.full(o.shape, p0))
    assert np.abs(f).max() < 1e-13 * p0 * case.ny * case.hy


@pytest.mark.parametrize("nx,ny", [(48, 36), (96, 72)])
def test_linear_pressure_gives_the_face_sampled_body_area(orc, nx, ny):
    """P = x gives Fp_x = -h_x * (dry length of the interior x-faces), exactly (summation by
    parts of the force sum), and that tends to minus the body area pi r^2 (the integral of
    grad P over the body, with the normal pointing out of the fluid).  P = y likewise in y.
    The cross components vanish (rows and columns telescope)."""
    case = _cyl(nx, ny)
    o = orc.Oracle(case)
    xc, yc = _centres(case)
    Ax, Ay = o.cap("p", "AX"), o.cap("p", "AY")
    dry_x = (case.hy - Ax[1:-2, 2:-2]).sum()          # x-faces i in [1, nx), j in [0, ny)
    dry_y = (case.hx - Ay[2:-2, 1:-2]).sum()          # y-faces j in [1, ny), i in [0, nx)
    fx = o.body_force(o.z(), o.z(), xc)
    fy = o.body_force(o.z(), o.z(), yc)
    area = math.pi * 0.5 ** 2
    assert fx[0] == pytest.approx(-case.hx * dry_x, rel=1e-12)
    assert fy[1] == pytest.approx(-case.hy * dry_y, rel=1e-12)
    assert abs(fx[1]) < 1e-12 and abs(fy[0]) < 1e-12
    assert np.abs(fx[2:]).max() == 0.0 and np.abs(fy[2:]).max() == 0.0
    assert abs(fx[0] + area) < case.hx ** 1.5 and abs(fy[1] + area) < case.hy ** 1.5


def test_linear_pressure_area_converges(orc):
    """The face-sampled area is a sum of exact chord lengths at the face abscissas: a
    midpoint-type rule for a chord with square-root ends, so its error is O(h^1.5) (not
    monotone in h: it depends on where the faces fall near the body's ends)."""
    for n in (32, 64, 128, 256):
        case = _cyl(n, 3 * n // 4)
        o = orc.Oracle(case)
        xc, _ = _centres(case)
        err = abs(o.body_force(o.z(), o.z(), xc)[0] + math.pi * 0.25)
        assert err < case.hx ** 1.5, (n, err)


def test_uniform_pressure_on_mesh_aligned_wall(orc):
    """Pressure P0 above a horizontal wall spanning the box pushes it down with P0 per unit
    length: Fp = (0, -P0 L)."""
    case, _ = _wall()
    o = orc.Oracle(case)
    p0 = 2.5
    f = o.body_force(o.z(), o.z(), np.full(o.shape, p0))
    L = case.nx * case.hx
    assert f[0] == pytest.approx(0.0, abs=1e-14)
    assert f[1] == pytest.approx(-p0 * L, rel=1e-14)


def test_couette_shear_on_mesh_aligned_wall(orc):
    """Plane Couette flow u = gamma (y - y_w), v = 0 over a no-slip wall: the wall shear stress
    is mu gamma, and the discrete strain at the wall nodes is exactly gamma / 2 (Eq. offdiag
    with the half-cell weight W = h_x h_y / 2).  The wall row has nx + 1 nodes of spacing h_x,
    so Fv = (mu gamma h_x (nx + 1), 0)."""
    case, yw = _wall(nx=10, ny=8, jw=3)
    o = orc.Oracle(case)
    gamma = 1.7
    _, yc = _centres(case)
    Vu = o.cap("u", "V")
    u = np.where(Vu > 0, gamma * (yc - yw), 0.0)
    f = o.body_force(u, o.z(), o.z())
    assert f[2] == pytest.approx(case.mu * gamma * case.hx * (case.nx + 1), rel=1e-13)
    assert abs(f[3]) < 1e-14 and f[0] == 0.0 and f[1] == 0.0
    # the strain itself is the constant gamma / 2 on every node of the fluid (the closed form)
    sxx, syy, sxy = o.strain(u, o.z())
    jw = 3
    assert np.allclose(sxy[jw + 1:case.ny + 1, 1:case.nx + 2], gamma / 2, rtol=1e-13)


@pytest.mark.parametrize("geom,literal", [("circle", 0), ("naca", 0), ("circle", 1)])
def test_force_is_the_operator_sum_for_fields_vanishing_near_the_box(orc, geom, literal):
    """With U and P zero within a few cells of the box, the box-boundary fluxes vanish, so the
    pressure force equals the sum of pres(P) over every velocity position and the viscous
    force minus the sum of visc(2 mu S(U)) (the momentum the body takes from the fluid)."""
    case = _cyl(40, 30, literal_offdiag=literal) if geom == "circle" else _naca(48, 28, literal_offdiag=literal)
    o = orc.Oracle(case)
    rng = np.random.default_rng(11)
    bump = np.zeros(o.shape)
    bump[5:-6, 5:-6] = 1.0
    u = rng.standard_normal(o.shape) * bump * (o.cap("u", "V") > 0)
    v = rng.standard_normal(o.shape) * bump * (o.cap("v", "V") > 0)
    p = rng.standard_normal(o.shape) * bump
    f = o.body_force(u, v, p)
    pu, pv = o.pres(p)
    sxx, syy, sxy = o.strain(u, v)
    vu, vv = o.visc(sxx, syy, sxy)
    mu = case.mu
    scale_p = np.abs(pu).sum() + np.abs(pv).sum()
    scale_v = 2 * mu * (np.abs(vu).sum() + np.abs(vv).sum())
    assert f[0] == pytest.approx(pu.sum(), abs=1e-13 * scale_p)
    assert f[1] == pytest.approx(pv.sum(), abs=1e-13 * scale_p)
    assert f[2] == pytest.approx(-2 * mu * vu.sum(), abs=1e-13 * scale_v)
    assert f[3] == pytest.approx(-2 * mu * vv.sum(), abs=1e-13 * scale_v)
    # and the force is not trivially small for these fields
    assert np.abs(f[:2]).max() > 1e-3 * scale_p / o.S ** 0.5
    assert np.abs(f[2:]).max() > 1e-3 * scale_v / o.S ** 0.5
