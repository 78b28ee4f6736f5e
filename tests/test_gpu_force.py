"""Force on the body through the C ABI: the device reduction gives the oracle's force on the
same fields (the library's own state after some steps), the closed forms the oracle is pinned
to, and the per-step record equals the force read after each step."""
import numpy as np
import pytest

from paper_2211_10698_gb300 import ccm, forces, inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2211_10698_gb300 import build

    build.build()


def _abs_scale(o, u, v, p):
    """Sum of the absolute values of every term of the force sums (the rounding scale)."""
    Ax, Ay = o.cap("p", "AX"), o.cap("p", "AY")
    Bxx, Bxy, Byx, Byy = o.cap("u", "BX"), o.cap("u", "BY"), o.cap("v", "BX"), o.cap("v", "BY")
    sxx, syy, sxy = o.strain(u, v)
    c = (slice(1, -2), slice(1, -2))            # cells i in [0, nx), j in [0, ny)
    sp = (np.abs(p[c]) * (np.abs(np.diff(Ax[1:-2, 1:-1], axis=1)) + np.abs(np.diff(Ay[1:-1, 1:-2], axis=0)))).sum()
    sv = (np.abs(sxx[c]) * np.abs(np.diff(Bxx[1:-2, 1:-1], axis=1))).sum()
    sv += (np.abs(syy[c]) * np.abs(np.diff(Byy[1:-1, 1:-2], axis=0))).sum()
    sv += (np.abs(sxy[1:-1, 1:-1]) * (np.abs(np.diff(Bxy[0:-1, 1:-1], axis=0)) +
                                      np.abs(np.diff(Byx[1:-1, 0:-1], axis=1)))).sum()
    return sp, 2 * o.case.mu * sv


@pytest.mark.parametrize("which", ["c1", "naca", "mixed"])
def test_body_force_matches_oracle_on_the_library_state(orc, which):
    if which == "naca":
        case = I.make_case("naca_small", 160, 80, (-1.0, 3.0, -1.0, 1.0),
                           I.Geometry(kind=I.GEOM_NACA, naca_tt=12, aoa_deg=8.0), re=500.0, cfl=0.5, lref=1.0)
    else:
        case = I.cylinder_re40_128x64()
    if which == "mixed":
        case.precision = "mixed"
    g = ccm.Case(case)
    g.step(6)
    u, v, p = (g.get_field(f) for f in (ccm.CCM_F_U, ccm.CCM_F_V, ccm.CCM_F_P))
    o = orc.Oracle(case)
    want = o.body_force(u, v, p)
    got = g.body_force()
    sp, sv = _abs_scale(o, u, v, p)
    assert np.abs(got[:2] - want[:2]).max() <= 1e-13 * sp, (got, want, sp)
    assert np.abs(got[2:] - want[2:]).max() <= 1e-13 * sv, (got, want, sv)
    # a body in a uniform stream is dragged downstream
    assert got[0] + got[2] > 0


def test_symmetric_cylinder_has_no_lift():
    """The Re 40 cylinder on [-2,6]x[-2,2] sits on the grid's symmetry line: after some steps
    the lift vanishes to rounding, the drag does not."""
    g = ccm.Case(I.cylinder_re40_128x64())
    g.step(10)
    f = g.body_force()
    assert abs(f[1] + f[3]) < 1e-9 * abs(f[0] + f[2])


def _wall_case(nx=64, ny=32, jw=9):
    box = (0.0, 2.0, 0.0, 1.0)
    yw = box[2] + jw * (box[3] - box[2]) / ny
    g = I.Geometry(kind=I.GEOM_HALFPLANE, hp_nx=0.0, hp_ny=1.0, hp_off=yw)
    # outflow west and east: the end faces are velocity unknowns and keep the profile
    bc = ((I.BC_OUTFLOW, I.BC_OUTFLOW, I.BC_DIRICHLET, I.BC_DIRICHLET), (0.0,) * 4, (0.0,) * 4)
    case = I.make_case("wall", nx, ny, box, g, re=20.0, cfl=0.5, lref=1.0, bc=bc)
    case.autotune = 0
    return case, yw


def test_couette_and_uniform_pressure_on_a_wall():
    """Closed forms on the device: Couette flow u = gamma (y - y_w) over a mesh-aligned wall
    gives Fv_x = mu gamma h_x (nx + 1) (nx + 1 wall nodes, shear stress mu gamma); a uniform
    pressure P0 gives Fp_y = -P0 L."""
    case, yw = _wall_case()
    g = ccm.Case(case)
    gamma, p0 = 1.3, 0.75
    yc = case.y0 + (np.arange(-1, case.ny + 2) + 0.5) * case.hy
    Vu = g.cap("u", "V")
    u = np.where(Vu > 0, gamma * (yc[:, None] - yw), 0.0)
    g.set_field(ccm.CCM_F_U, u)
    g.set_field(ccm.CCM_F_V, np.zeros(case.shape))
    g.set_field(ccm.CCM_F_P, np.full(case.shape, p0))
    f = g.body_force()
    L = case.nx * case.hx
    assert f[2] == pytest.approx(case.mu * gamma * case.hx * (case.nx + 1), rel=1e-13)
    assert f[1] == pytest.approx(-p0 * L, rel=1e-13)
    assert abs(f[0]) < 1e-13 * p0 * L and abs(f[3]) < 1e-13 * case.mu * gamma * L


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_force_record_equals_force_after_each_step(precision):
    case = I.cylinder_re40_128x64()
    case.precision = precision
    g = ccm.Case(case)
    g.set_force_history(4)
    after = []
    for _ in range(6):
        g.step(1)
        after.append(g.body_force())
    rows, total = g.force_history()
    assert total == 6 and rows.shape == (4, 4)
    assert np.array_equal(rows, np.array(after[2:]))
    # fewer rows on request, still the newest, oldest first
    rows2, _ = g.force_history(max_rows=2)
    assert np.array_equal(rows2, np.array(after[4:]))
    # async steps record the same way; a new capacity clears the record
    g.set_force_history(10)
    g.step_async(3)
    g.read_stats()
    rows3, total3 = g.force_history()
    assert total3 == 3 and rows3.shape == (3, 4)
    assert np.array_equal(rows3[-1], g.body_force())
    g.set_force_history(0)
    assert g.force_history()[1] == 0


def test_step_filtered_drag_of_the_record():
    """The viscous force of the state alternates in sign from step to step (the Crank-Nicolson
    mode of the small cut cells); filtered over consecutive steps the drag coefficient is
    positive and of the size a confined cylinder at Re 40 has, and the alternating part is far
    larger than the filtered one (the reason for the filter)."""
    case = I.cylinder_re40_128x64()
    g = ccm.Case(case)
    g.set_force_history(12)
    g.step(30)
    rows, total = g.force_history()
    assert total == 30 and rows.shape == (12, 4)
    cdl = forces.coefficients(forces.step_filter(rows), case.rho, case.u_inf, 1.0)
    assert ((cdl[:, 0] > 0.5) & (cdl[:, 0] < 10.0)).all(), cdl
    alt = np.abs(np.diff(rows[:, 2])).min()
    assert alt > 5 * np.abs(forces.step_filter(rows)[:, 2]).max()
