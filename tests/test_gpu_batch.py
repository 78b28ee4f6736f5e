"""Batched stepping: cases of different sizes and geometries advanced together (one batched
Poisson solve per step) give the same fields as each case advanced alone, within the
solver tolerances, in FP64 and in the mixed-precision setting; bookkeeping and errors."""
import numpy as np
import pytest

from paper_2211_10698_gb300 import ccm, inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2211_10698_gb300 import build

    build.build()


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _field(case, spec, f):
    """Field f; in a closed box the pressure up to its mean over fluid cells (an all-Dirichlet
    box fixes the pressure only up to a constant, Sec. 4.6 null space)."""
    x = case.get_field(f)
    if f == ccm.CCM_F_P and tuple(spec.bc_type) == I.closed_box_bc()[0]:
        fluid = case.cap("p", "V") > 0
        x = np.where(fluid, x - x[fluid].mean(), 0.0)
    return x


def _mix(precision):
    cs = [
        I.small_cylinder(nx=48, ny=24, box=(-2.0, 4.0, -1.5, 1.5), r=0.5, cx=0.0, cy=0.0),
        I.small_cylinder(nx=96, ny=40, box=(-2.0, 4.0, -1.25, 1.25), r=0.43, cx=0.1, cy=-0.05),
        I.make_case("naca", 96, 48, (-0.5, 1.5, -0.5, 0.5),
                    I.Geometry(kind=I.GEOM_NACA, naca_tt=12, aoa_deg=7.0), re=200.0, cfl=0.5, lref=1.0),
        I.small_cylinder(nx=37, ny=23, box=(-1.5, 1.5, -1.0, 1.0), r=0.41, cx=0.07, cy=-0.05,
                         bc=I.closed_box_bc(lid=1.0), re=50.0),
        I.make_case("channel", 64, 16, (0.0, 4.0, 0.0, 1.0), I.Geometry(), re=20.0, cfl=0.5, lref=1.0,
                    bc=((I.BC_DIRICHLET, I.BC_OUTFLOW, I.BC_DIRICHLET, I.BC_DIRICHLET), (1.0, 0, 0, 0), (0, 0, 0, 0))),
    ]
    for c in cs:
        c.precision = precision
        c.tol_p = 1e-12 if precision == "mixed" else 1e-13
        c.tol_h = 1e-13
    return cs


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("mixed", 1e-8)])
@pytest.mark.parametrize("with_closed", [True, False])
def test_batch_equals_alone(precision, tol, with_closed):
    """With a closed box (a singular system) in the batch, the unscaled batched PCG and the
    host-driven refinement run; without, the scaled FP64 and the one-launch mixed batches."""
    specs = _mix(precision)
    if not with_closed:
        specs = [c for c in specs if tuple(c.bc_type) != I.closed_box_bc()[0]]
        assert len(specs) == 4
    alone = [ccm.Case(c) for c in specs]
    for a in alone:
        a.step(4)
    mixed = [ccm.Case(c) for c in specs]
    b = ccm.Batch(8)
    for m in mixed:
        b.add(m)
    stats = b.step(4)
    assert len(stats) == len(specs)
    for a, m, st, sp in zip(alone, mixed, stats, specs):
        assert st["converged"] and st["steps"] == 4
        for f in (ccm.CCM_F_U, ccm.CCM_F_V, ccm.CCM_F_P):
            assert _rel(_field(m, sp, f), _field(a, sp, f)) < tol, (m.spec.name, f)
    b.close()


@pytest.mark.parametrize("pcs", [("chebyshev", 4), ("alternate", 4), ("chebyshev", 3), ("degrees", 0)])
def test_mixed_batch_chebyshev_equals_alone(pcs):
    """The batched mixed solve with the Chebyshev preconditioner: every case of the batch, of
    any size, preconditioner and degree, gives the fields of the same case advanced alone
    (one-launch mixed solve with its own preconditioner)."""
    kind, degree = pcs
    specs = [c for c in _mix("mixed") if tuple(c.bc_type) != I.closed_box_bc()[0]]
    for k, c in enumerate(specs):
        if kind == "chebyshev":
            c.precond, c.cheb_degree = "chebyshev", degree
        elif kind == "alternate":
            c.precond, c.cheb_degree = ("chebyshev" if k % 2 == 0 else "jacobi"), degree
        else:
            c.precond, c.cheb_degree = "chebyshev", 2 + k
    alone = [ccm.Case(c) for c in specs]
    for a in alone:
        a.step(4)
    mixed = [ccm.Case(c) for c in specs]
    b = ccm.Batch(8)
    for m in mixed:
        b.add(m)
    stats = b.step(4)
    for a, m, st in zip(alone, mixed, stats):
        assert st["converged"] and st["steps"] == 4
        for f in (ccm.CCM_F_U, ccm.CCM_F_V, ccm.CCM_F_P):
            assert _rel(m.get_field(f), a.get_field(f)) < 1e-8, (m.spec.name, f)
    b.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_replay_equals_eager(precision):
    """Steps replayed from the captured graphs give the fields of steps that issue every
    launch, bit for bit; a case stepped on its own in between makes the batch recapture."""
    specs = [c for c in _mix(precision) if tuple(c.bc_type) != I.closed_box_bc()[0]]
    for c in specs:
        c.precond = "chebyshev"

    def run(graphs):
        cs = [ccm.Case(c) for c in specs]
        b = ccm.Batch(8)
        b.set_graphs(graphs)
        b.set_tuning(False)  # the same block split in both batches: bitwise comparable
        for c in cs:
            b.add(c)
        st = b.step(4)
        why = ccm.lib().ccm_last_error().decode()
        cs[1].step(1)
        st += b.step(2)
        return cs, b, st, why

    cg, bg, sg, why = run(True)
    ce, be, se, _ = run(False)
    assert bg.graph_steps() == 5, why  # 3 + 2: each case's first step runs without a graph
    assert be.graph_steps() == 0
    assert all(s["converged"] for s in sg + se)
    for a, m in zip(cg, ce):
        for f in (ccm.CCM_F_U, ccm.CCM_F_V, ccm.CCM_F_P):
            np.testing.assert_array_equal(a.get_field(f), m.get_field(f))
    bg.close()
    be.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("mixed", 1e-8)])
def test_split_tuning(precision, tol):
    """The three steps after the first try one block split of the Poisson launch each and keep
    one of the candidates; the fields match a batch that does not tune."""
    specs = [c for c in _mix(precision) if tuple(c.bc_type) != I.closed_box_bc()[0]]
    tuned = [ccm.Case(c) for c in specs]
    plain = [ccm.Case(c) for c in specs]
    bt, bp = ccm.Batch(8), ccm.Batch(8)
    bp.set_tuning(False)
    for a, m in zip(tuned, plain):
        bt.add(a)
        bp.add(m)
    assert bt.split() == (0.0, False)
    st = bt.step(6)
    sp = bp.step(6)
    a, done = bt.split()
    assert done and a in (0.0, 0.5, 1.0)
    assert bp.split() == (0.0, False)
    assert bt.graph_steps() == 2 and bp.graph_steps() == 5
    assert all(s["converged"] for s in st + sp)
    for x, y in zip(tuned, plain):
        for f in (ccm.CCM_F_U, ccm.CCM_F_V, ccm.CCM_F_P):
            assert _rel(x.get_field(f), y.get_field(f)) < tol, f
    bt.close()
    bp.close()


def test_cases_join_and_leave_between_steps():
    specs = _mix("fp64")[:3]
    ref = [ccm.Case(c) for c in specs]
    for r in ref:
        r.step(3)
    cs = [ccm.Case(c) for c in specs]
    b = ccm.Batch(4)
    b.add(cs[0])
    b.add(cs[1])
    b.step(1)
    b.add(cs[2])
    cs[2].step(1)  # the late case catches up alone
    b.step(1)
    b.remove(cs[0])
    cs[0].step(1)
    b.step(1)
    for r, c in zip(ref, cs):
        assert _rel(c.get_field(ccm.CCM_F_U), r.get_field(ccm.CCM_F_U)) < 1e-9
    b.close()


def test_batch_errors():
    specs = _mix("fp64")
    a = ccm.Case(specs[0])
    b = ccm.Batch(1)
    b.add(a)
    with pytest.raises(ccm.CcmError):
        b.add(ccm.Case(specs[1]))  # full
    with pytest.raises(ccm.CcmError):
        b.add(a)
    m = specs[1]
    m.precision = "mixed"
    b2 = ccm.Batch(2)
    b2.add(ccm.Case(specs[2]))
    with pytest.raises(ccm.CcmError):
        b2.add(ccm.Case(m))  # precision differs
    b.close()
    b2.close()


def _rotation(case, g, omega):
    """The velocity omega x (x - c) of a rotating cylinder at the u- and v-control volumes'
    boundary points (the body's D)."""
    geo = case.geom
    xu, yu = I.circle_boundary_points(g.cap("u", "X"), g.cap("u", "Y"), geo.cx, geo.cy, geo.r)
    xv, yv = I.circle_boundary_points(g.cap("v", "X"), g.cap("v", "Y"), geo.cx, geo.cy, geo.r)
    return -omega * (yu - geo.cy), omega * (xv - geo.cx)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("mixed", 1e-8)])
def test_batch_with_body_velocity_and_forcing_equals_alone(precision, tol):
    """A case with a rotating body (its D-terms) and a case with a body acceleration g, batched
    with plain cases, give the fields of the same cases advanced alone: the batched stages read
    the same per-case terms as the single-case ones."""
    specs = [c for c in _mix(precision) if tuple(c.bc_type) != I.closed_box_bc()[0]]
    rng = np.random.default_rng(21)
    gx = 0.2 * rng.standard_normal(specs[2].shape)
    gy = 0.2 * rng.standard_normal(specs[2].shape)

    def make():
        cases = [ccm.Case(c) for c in specs]
        dx, dy = _rotation(specs[1], cases[1], 1.2)
        cases[1].set_field(ccm.CCM_F_DX, dx)
        cases[1].set_field(ccm.CCM_F_DY, dy)
        cases[2].set_field(ccm.CCM_F_GX, gx)
        cases[2].set_field(ccm.CCM_F_GY, gy)
        return cases

    alone = make()
    for a in alone:
        a.step(4)
    together = make()
    b = ccm.Batch(8)
    for m in together:
        b.add(m)
    stats = b.step(4)
    for a, m, st, sp in zip(alone, together, stats, specs):
        assert st["converged"] and st["steps"] == 4
        for f in (ccm.CCM_F_U, ccm.CCM_F_V, ccm.CCM_F_P):
            assert _rel(_field(m, sp, f), _field(a, sp, f)) < tol, (m.spec.name, f)
    b.close()
