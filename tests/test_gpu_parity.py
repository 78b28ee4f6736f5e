"""Parity of the CUDA path (through the C ABI) with the FP64 oracle: capacities, every
operator, the diagonals, the Poisson solve and whole projection steps, on small cases that
span several tiles with ragged edges, the C1 configuration, and full-size C2/C3 grids
checked stage by stage with the oracle's operators."""
import numpy as np
import pytest

import oracle as O
from paper_2211_10698_gb300 import ccm, inputs as I

pytestmark = pytest.mark.gpu

OP_TOL = 1e-11     # relative L2 per operator apply (FP64)
STEP_TOL = 1e-9    # relative L2 on velocity and pressure after the steps (FP64)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2211_10698_gb300 import build

    build.build()
    O.build()


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _naca_small():
    return I.make_case("naca_small", 96, 48, (-0.5, 1.5, -0.5, 0.5),
                       I.Geometry(kind=I.GEOM_NACA, naca_tt=12, aoa_deg=7.0), re=200.0, cfl=0.5, lref=1.0)


def _closed_cyl():
    return I.small_cylinder(nx=37, ny=23, box=(-1.5, 1.5, -1.0, 1.0), r=0.41, cx=0.07, cy=-0.05,
                            bc=I.closed_box_bc(), re=50.0)


def _cavity():
    return I.make_case("cavity", 33, 29, (0.0, 1.0, 0.0, 1.0), I.Geometry(), re=100.0, cfl=0.5, lref=1.0,
                       bc=I.closed_box_bc(lid=1.0), u_inf=1.0)


def _ragged():
    return I.small_cylinder(nx=53, ny=31, box=(-2.0, 3.0, -1.4, 1.5), r=0.45, cx=0.11, cy=0.04)


def _stretched():
    return I.stretched_cylinder(nx=64, ny=48, box=(-3.0, 7.0, -3.0, 3.0), fine=(24, 24), h_fine=0.08, ratio=1.08)


def _stretched_naca():
    """NACA 0012 at 6 degrees on a mesh refined around the section (Sec. 3.1, stretched)."""
    xf = I.stretched_faces(96, -1.5, 2.5, 40, 0.03, 1.05)
    yf = I.stretched_faces(50, -1.0, 1.0, 20, 0.03, 1.08)
    return I.make_case("stretched_naca", 96, 50, (-1.5, 2.5, -1.0, 1.0),
                       I.Geometry(kind=I.GEOM_NACA, naca_tt=12, aoa_deg=6.0, le_x=-0.5), re=200.0, cfl=0.5,
                       lref=1.0, xf=xf, yf=yf)


CASES = {
    "cylinder": lambda: I.small_cylinder(nx=48, ny=24, box=(-2.0, 4.0, -1.5, 1.5), r=0.5, cx=0.0, cy=0.0),
    "ragged": _ragged,
    "naca": _naca_small,
    "closed": _closed_cyl,
    "cavity": _cavity,
    "stretched": _stretched,
    "stretched_naca": _stretched_naca,
}


def _sliver_scale(o, grid):
    hx, hy = o.case.hx, o.case.hy
    V = o.cap(grid, "V")
    kap = np.where(V > 0, np.maximum(1.0, hx * hy / np.where(V > 0, V, 1.0)), 1.0)
    # second-kind quantities also depend on the neighbours' centroids
    k2 = kap.copy()
    k2[:, 1:] = np.maximum(k2[:, 1:], kap[:, :-1])
    k2[1:, :] = np.maximum(k2[1:, :], kap[:-1, :])
    return k2


@pytest.mark.parametrize("name", list(CASES))
def test_capacities(name):
    case = CASES[name]()
    o = O.Oracle(case)
    g = ccm.Case(case)
    hx, hy = case.hx, case.hy
    for grid in "puv":
        kap = _sliver_scale(o, grid)
        for nm in O.CAP_NAMES:
            ref = o.cap(grid, nm)
            got = g.cap(grid, nm)
            unit = hx * hy if nm in ("V", "WX", "WY") else max(hx, hy)
            scale = kap if nm not in ("V", "AX", "AY") else 1.0
            if nm in ("X", "Y"):
                err = np.abs(got - ref) / (unit * scale)
            else:
                err = np.abs(got - ref) / (unit * scale)
            assert err.max() < 1e-12, (grid, nm, err.max(), np.unravel_index(err.argmax(), err.shape))


def _inputs(o, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(o.shape), rng.standard_normal(o.shape), rng.standard_normal(o.shape)


@pytest.mark.parametrize("name", list(CASES))
def test_operators(name):
    case = CASES[name]()
    o = O.Oracle(case)
    g = ccm.Case(case)
    u, v, p = _inputs(o, 17)
    assert rel(g.apply(ccm.CCM_OP_CONT, u, v, nout=1), o.cont(u, v)) < OP_TOL
    gu, gv = g.apply(ccm.CCM_OP_PRES, p)
    ru, rv = o.pres_bc(p)
    assert rel(gu, ru) < OP_TOL and rel(gv, rv) < OP_TOL
    gu, gv = g.apply(ccm.CCM_OP_CONV, u, v)
    ru, rv = o.conv_bc(u, v)
    assert rel(gu, ru) < OP_TOL and rel(gv, rv) < OP_TOL
    gu, gv = g.apply(ccm.CCM_OP_VISC, u, v)
    ru, rv = o.visc_bc(u, v)
    assert rel(gu, ru) < OP_TOL and rel(gv, rv) < OP_TOL
    gu, gv = g.apply(ccm.CCM_OP_HELMHOLTZ, u, v)
    ru, rv = o.helmholtz(u, v)
    assert rel(gu, ru) < OP_TOL and rel(gv, rv) < OP_TOL
    assert rel(g.apply(ccm.CCM_OP_POISSON, p, nout=1), o.poisson(p)) < OP_TOL
    # the diagonals by probing: sums of many terms, whose rounding grows with the spread of the
    # capacities (small cut cells on a fine part of a stretched mesh)
    assert rel(g.apply(ccm.CCM_OP_POISSON_DIAG, nout=1), o.poisson_diag()) < 1e-12
    gu, gv = g.apply(ccm.CCM_OP_HELMHOLTZ_DIAG)
    du, dv = o.helmholtz_diag()
    assert rel(gu, du) < 1e-12 and rel(gv, dv) < 1e-12


def test_literal_offdiag_operator():
    case = _closed_cyl()
    case.literal_offdiag = 1
    o = O.Oracle(case)
    g = ccm.Case(case)
    u, v, _ = _inputs(o, 23)
    gu, gv = g.apply(ccm.CCM_OP_HELMHOLTZ, u, v)
    ru, rv = o.helmholtz(u, v)
    assert rel(gu, ru) < OP_TOL and rel(gv, rv) < OP_TOL


@pytest.mark.parametrize("name", ["cylinder", "ragged", "naca", "closed", "stretched", "stretched_naca"])
def test_poisson_solve(name):
    case = CASES[name]()
    case.tol_p = 1e-13
    o = O.Oracle(case)
    g = ccm.Case(case)
    rhs = np.random.default_rng(5).standard_normal(o.shape) * o.active
    if name == "closed":
        rhs[o.active] -= rhs[o.active].mean()
    st = g.solve_pressure(rhs)
    assert st["converged"]
    phi_g = g.get_field(ccm.CCM_F_PHI)
    phi_o, info = o.solve_poisson(rhs, tol=1e-13)
    assert rel(phi_g, phi_o) < 1e-9
    assert abs(st["iters"] - info["iters"]) <= max(3, 0.05 * info["iters"])
    # the GPU solution satisfies the oracle's system
    assert rel(o.poisson(phi_g)[o.active], rhs[o.active]) < 2e-13


@pytest.mark.parametrize("nx,ny", [(5, 4), (61, 7), (300, 4), (9, 211), (130, 66)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_poisson_solve_tile_shapes(nx, ny, precision):
    """The FP64 solve tiles the grid (tile widths 32..512, one block per tile, the ring of each
    tile recomputed by its block): grids narrower than a tile, very flat and very tall grids
    agree with the oracle, and so does the mixed solve on the same grids."""
    box = (0.0, nx / 8.0, 0.0, ny / 8.0)
    geom = I.Geometry(kind=I.GEOM_CIRCLE, cx=box[1] * 0.4, cy=box[3] * 0.5, r=0.3) if min(nx, ny) >= 12 else I.Geometry()
    case = I.make_case(f"tiles_{nx}x{ny}", nx, ny, box, geom, re=50.0, cfl=0.5, lref=1.0)
    case.tol_p = 1e-12
    case.precision = precision
    o = O.Oracle(case)
    g = ccm.Case(case)
    rhs = np.random.default_rng(nx * 1000 + ny).standard_normal(o.shape) * o.active
    st = g.solve_pressure(rhs)
    assert st["converged"]
    phi_g = g.get_field(ccm.CCM_F_PHI)
    phi_o, _ = o.solve_poisson(rhs, tol=1e-13)
    assert rel(phi_g, phi_o) < (1e-9 if precision == "fp64" else 1e-7)
    assert rel(o.poisson(phi_g)[o.active], rhs[o.active]) < 1.01e-12


@pytest.mark.parametrize("name", ["cylinder", "naca", "closed", "stretched"])
@pytest.mark.parametrize("degree", [2, 4])
def test_chebyshev_poisson_solve(name, degree):
    """Chebyshev-preconditioned PCG (k-step Chebyshev iteration on the Jacobi-scaled
    operator) agrees with the oracle's, solution and iteration count."""
    case = CASES[name]()
    case.tol_p = 1e-13
    case.precond = "chebyshev"
    case.cheb_degree = degree
    o = O.Oracle(case)
    g = ccm.Case(case)
    rhs = np.random.default_rng(8).standard_normal(o.shape) * o.active
    if name == "closed":
        rhs[o.active] -= rhs[o.active].mean()
    st = g.solve_pressure(rhs)
    phi_o, info = o.solve_poisson(rhs, tol=1e-13)
    assert st["converged"]
    assert rel(g.get_field(ccm.CCM_F_PHI), phi_o) < 1e-9
    assert abs(st["iters"] - info["iters"]) <= max(3, 0.05 * info["iters"])


@pytest.mark.parametrize("name", ["cylinder", "naca", "closed"])
@pytest.mark.parametrize("precond", ["jacobi", "chebyshev"])
def test_mixed_precision_poisson_solve(name, precond):
    """FP32 inner PCG with FP64 residual refinement reaches the FP64 residual target and
    the FP64 oracle's solution."""
    case = CASES[name]()
    case.tol_p = 1e-12
    case.precision = "mixed"
    case.precond = precond
    o = O.Oracle(case)
    g = ccm.Case(case)
    rhs = np.random.default_rng(9).standard_normal(o.shape) * o.active
    if name == "closed":
        rhs[o.active] -= rhs[o.active].mean()
    st = g.solve_pressure(rhs)
    assert st["converged"] and st["outer"] >= 2 and st["rel_res"] <= 1e-12
    phi_g = g.get_field(ccm.CCM_F_PHI)
    assert rel(o.poisson(phi_g)[o.active], rhs[o.active]) < 1.01e-12
    phi_o, _ = o.solve_poisson(rhs, tol=1e-13)
    # the residual target bounds the solution error by cond(K) * 1e-12 (cond ~ 1e4 here)
    assert rel(phi_g, phi_o) < 1e-7


@pytest.mark.parametrize("name", ["cylinder", "naca", "closed", "stretched"])
@pytest.mark.parametrize("precond", ["jacobi", "chebyshev"])
def test_mixed_precision_steps(name, precond):
    """Steps with the mixed-precision Poisson solve refined to an FP64 residual of 1e-12
    stay within 1e-8 of the FP64 oracle (the closed box: a singular system, whose pressure
    increment is kept at zero mean in FP64)."""
    case = CASES[name]()
    case.tol_p, case.tol_h = 1e-12, 1e-13
    case.precision = "mixed"
    case.precond = precond
    o = O.Oracle(case)
    g = ccm.Case(case)
    if name == "closed":
        rng = np.random.default_rng(3)
        u0 = rng.standard_normal(o.shape) * (o.role_u == 3)
        v0 = rng.standard_normal(o.shape) * (o.role_v == 3)
        s = o.init_state(u0=0.0)
        s["u"], s["v"] = o.fill_ghosts(u0, v0)
        g.set_field(ccm.CCM_F_U, s["u"])
        g.set_field(ccm.CCM_F_V, s["v"])
    else:
        s = o.init_state()
    o.step(s, 4)
    gs = g.step(4)
    assert gs["converged"]
    for f, ref in ((ccm.CCM_F_U, s["u"]), (ccm.CCM_F_V, s["v"]), (ccm.CCM_F_P, s["p"])):
        assert rel(g.get_field(f), ref) < 1e-8, f


@pytest.mark.parametrize("name,nsteps", [("cylinder", 5), ("ragged", 4), ("naca", 3), ("closed", 4), ("cavity", 4),
                                         ("stretched", 4), ("stretched_naca", 3)])
def test_steps(name, nsteps):
    case = CASES[name]()
    case.tol_p = case.tol_h = 1e-13
    o = O.Oracle(case)
    g = ccm.Case(case)
    if name in ("closed",):
        # start from a random field (no inflow drives the closed box)
        rng = np.random.default_rng(3)
        u0 = rng.standard_normal(o.shape) * (o.role_u == 3)
        v0 = rng.standard_normal(o.shape) * (o.role_v == 3)
        s = o.init_state(u0=0.0)
        s["u"], s["v"] = o.fill_ghosts(u0, v0)
        g.set_field(ccm.CCM_F_U, s["u"])
        g.set_field(ccm.CCM_F_V, s["v"])
    else:
        s = o.init_state(u0=case.bc_un[0] if name != "cavity" else 0.0)
        if name == "cavity":
            g.set_field(ccm.CCM_F_U, s["u"])
    gs = g.step(nsteps)
    hist, extra = o.step(s, nsteps, keep=True)
    assert gs["converged"]
    for f, ref in ((ccm.CCM_F_U, s["u"]), (ccm.CCM_F_V, s["v"]), (ccm.CCM_F_P, s["p"]),
                   (ccm.CCM_F_PHI, s["phi"]), (ccm.CCM_F_USTAR, extra["ustar"]), (ccm.CCM_F_VSTAR, extra["vstar"])):
        assert rel(g.get_field(f), ref) < STEP_TOL, f
    assert gs["kinetic"] == pytest.approx(hist[-1]["kinetic"], rel=1e-10)
    assert gs["max_div"] < 1e-10 * max(1.0, np.abs(extra["b"]).max())


@pytest.mark.parametrize("pupdate", [0, 1, 2])
def test_pressure_update_volume_options(pupdate):
    """The three readings of the volume in the correction of Eq. pm_update agree with the
    oracle (0: full cell, the default, 1: fluid volume V_p, 2: no correction)."""
    case = CASES["ragged"]()
    case.tol_p = case.tol_h = 1e-13
    case.pressure_update = pupdate
    o = O.Oracle(case)
    g = ccm.Case(case)
    s = o.init_state()
    o.step(s, 3)
    g.step(3)
    for f, ref in ((ccm.CCM_F_U, s["u"]), (ccm.CCM_F_P, s["p"])):
        assert rel(g.get_field(f), ref) < STEP_TOL, f


def test_c1_cylinder_re40_100_steps():
    """The 128x64 Re 40 cylinder configuration, 100 steps; CG tolerances tightened to 1e-13
    on both sides so that the comparison measures the discretisation, not the stopping
    point of two CG runs."""
    case = I.cylinder_re40_128x64()
    case.tol_p = case.tol_h = 1e-13
    o = O.Oracle(case)
    g = ccm.Case(case)
    s = o.init_state()
    o.step(s, case.steps)
    gs = g.step(case.steps)
    assert gs["converged"]
    for f, ref in ((ccm.CCM_F_U, s["u"]), (ccm.CCM_F_V, s["v"]), (ccm.CCM_F_P, s["p"])):
        assert rel(g.get_field(f), ref) < STEP_TOL, f


def test_c1_at_config_tolerance():
    """At the configuration's own tolerance (1e-10) the two stopping points differ; the
    fields still agree to the accuracy the solves guarantee."""
    case = I.cylinder_re40_128x64()
    o = O.Oracle(case)
    g = ccm.Case(case)
    s = o.init_state()
    o.step(s, 20)
    g.step(20)
    assert rel(g.get_field(ccm.CCM_F_U), s["u"]) < 1e-7
    assert rel(g.get_field(ccm.CCM_F_P), s["p"]) < 1e-5


@pytest.mark.parametrize("which", ["c2", "c3"])
def test_full_size_one_step_stagewise(which):
    """Full-size grids (1024x512 cylinder with the seeded perturbation, 2048x1024 NACA0012):
    capacities and operators against the oracle, then one GPU step checked stage by stage
    with the oracle's operators: the predictor equation, the divergence, the Poisson
    equation, the projection and the pressure update."""
    case = I.cylinder_re100_1024x512() if which == "c2" else I.naca0012_re1000_2048x1024()
    case.precision = "fp64"
    case.precond = "jacobi"
    o = O.Oracle(case)
    g = ccm.Case(case)
    h = max(case.hx, case.hy)
    for grid in "puv":
        kap = _sliver_scale(o, grid)
        for nm in ("V", "AX", "AY", "WX", "BY"):
            unit = h * h if nm in ("V", "WX") else h
            scale = kap if nm in ("WX", "BY") else 1.0
            assert (np.abs(g.cap(grid, nm) - o.cap(grid, nm)) / (unit * scale)).max() < 1e-12, (grid, nm)
    u0, v0, p0 = _inputs(o, 29)
    assert rel(g.apply(ccm.CCM_OP_POISSON, p0, nout=1), o.poisson(p0)) < OP_TOL
    gu, gv = g.apply(ccm.CCM_OP_HELMHOLTZ, u0, v0)
    ru, rv = o.helmholtz(u0, v0)
    assert rel(gu, ru) < OP_TOL and rel(gv, rv) < OP_TOL
    # initial state (with the seeded perturbation for the shedding case)
    pu, pv = I.perturbation(case)
    s = o.init_state(pu=pu if case.perturb_sigma > 0 else None, pv=pv if case.perturb_sigma > 0 else None)
    g.set_field(ccm.CCM_F_U, s["u"])
    g.set_field(ccm.CCM_F_V, s["v"])
    un, vn = s["u"].copy(), s["v"].copy()
    gs = g.step(1)
    assert gs["converged"]
    us, vs = g.get_field(ccm.CCM_F_USTAR), g.get_field(ccm.CCM_F_VSTAR)
    u1, v1 = g.get_field(ccm.CCM_F_U), g.get_field(ccm.CCM_F_V)
    phi, P = g.get_field(ccm.CCM_F_PHI), g.get_field(ccm.CCM_F_P)
    # predictor: H U* = rhs(U^n)
    rhs_u, rhs_v, _, _ = o.predictor_rhs(un, vn, np.zeros(o.shape))
    hu, hv = o.helmholtz(us, vs)
    r = np.concatenate([(hu - rhs_u).ravel(), (hv - rhs_v).ravel()])
    b = np.concatenate([rhs_u.ravel(), rhs_v.ravel()])
    assert np.linalg.norm(r) <= 1.01 * case.tol_h * np.linalg.norm(b)
    # divergence and Poisson
    div = o.cont(us, vs)
    assert rel(g.get_field(ccm.CCM_F_DIV), div) < 1e-12
    rhs_p = -(case.rho / case.dt) * div * o.active
    kphi = o.poisson(phi)
    assert np.linalg.norm((kphi - rhs_p)[o.active]) <= 1.01 * case.tol_p * np.linalg.norm(rhs_p[o.active])
    # projection and pressure update
    gu_, gv_ = o.pres_bc(phi)
    Vu, Vv, Vp = o.cap("u", "V"), o.cap("v", "V"), o.cap("p", "V")
    fu = (case.dt / case.rho) * np.where(Vu > 1e-12 * case.hx * case.hy, 1.0 / np.where(Vu > 0, Vu, 1.0), 0.0)
    fv = (case.dt / case.rho) * np.where(Vv > 1e-12 * case.hx * case.hy, 1.0 / np.where(Vv > 0, Vv, 1.0), 0.0)
    unk_u, unk_v = o.role_u == 3, o.role_v == 3
    assert np.abs((u1 - (us - fu * gu_))[unk_u]).max() < 1e-12 * np.abs(us).max()
    assert np.abs((v1 - (vs - fv * gv_))[unk_v]).max() < 1e-12 * max(np.abs(vs).max(), 1e-30)
    pfac = (case.dt * case.mu / (2 * case.rho)) / (case.hx * case.hy)  # default volume: the full cell
    pref = (phi + pfac * kphi) * o.active
    assert rel(P, pref) < 1e-12


def test_determinism():
    case = _ragged()
    a, b = ccm.Case(case), ccm.Case(case)
    a.step(3)
    b.step(3)
    for f in (ccm.CCM_F_U, ccm.CCM_F_V, ccm.CCM_F_P, ccm.CCM_F_PHI):
        assert np.array_equal(a.get_field(f), b.get_field(f))


def test_torch_allocator_hook():
    torch = pytest.importorskip("torch")
    case = _ragged()
    a = ccm.Case(case, allocator=ccm.TorchAllocator())
    b = ccm.Case(case)
    a.step(2)
    b.step(2)
    assert np.array_equal(a.get_field(ccm.CCM_F_U), b.get_field(ccm.CCM_F_U))
    before = torch.cuda.memory_allocated()
    a.close()
    assert torch.cuda.memory_allocated() < before


def test_error_paths():
    case = _ragged()
    g = ccm.Case(case, set_geometry=False)
    with pytest.raises(ccm.CcmError) as e:
        g.step(1)
    assert e.value.status == ccm.CCM_E_STATE
    bad = I.small_cylinder(nx=16, ny=8, box=(-1.0, 1.0, -1.0, 1.0), r=0.8)
    g2 = ccm.Case(bad, set_geometry=False)
    with pytest.raises(ccm.CcmError) as e:
        g2.set_geometry(bad.geom)
    assert e.value.status == ccm.CCM_E_INVALID
    g3 = ccm.Case(case)
    small = np.zeros(9)
    assert ccm.lib().ccm_set_field(g3.h, ccm.CCM_F_U, small.ctypes.data_as(ccm._DP), 9) == ccm.CCM_E_INVALID
    assert ccm.lib().ccm_set_field(g3.h, ccm.CCM_F_USTAR, small.ctypes.data_as(ccm._DP), 9) == ccm.CCM_E_INVALID
    case.max_iter_p = 2
    g4 = ccm.Case(case)
    st = g4.step(1, allow_not_converged=True)
    assert not st["converged"] and st["last_iters_p"] == 2
    # the case stays usable
    case.max_iter_p = 20000
    g5 = ccm.Case(case)
    assert g5.step(1)["converged"]


@pytest.mark.parametrize("name", ["cylinder", "closed"])
def test_conservation_sums_match_oracle(name):
    """The step statistics' mass and momentum sums (the diagnostics) equal the oracle's on the
    library's own fields; in the closed box the net flux through the walls is zero, so the mass
    sum is at the solver's tolerance."""
    case = CASES[name]()
    case.tol_p = case.tol_h = 1e-13
    g = ccm.Case(case)
    o = O.Oracle(case)
    if name == "closed":
        rng = np.random.default_rng(3)
        u0 = rng.standard_normal(o.shape) * (o.role_u == 3)
        v0 = rng.standard_normal(o.shape) * (o.role_v == 3)
        s0 = o.init_state(u0=0.0)
        s0["u"], s0["v"] = o.fill_ghosts(u0, v0)
        g.set_field(ccm.CCM_F_U, s0["u"])
        g.set_field(ccm.CCM_F_V, s0["v"])
    st = g.step(3)
    u, v = g.get_field(ccm.CCM_F_U), g.get_field(ccm.CCM_F_V)
    m, px, py = o.conservation(u, v)
    scale = np.abs(o.cap("u", "V") * u).sum() + np.abs(o.cap("v", "V") * v).sum()
    assert st["momentum_x"] == pytest.approx(px, abs=1e-13 * scale)
    assert st["momentum_y"] == pytest.approx(py, abs=1e-13 * scale)
    assert st["mass"] == pytest.approx(m, abs=1e-13 * scale)
    if name == "closed":
        assert abs(st["mass"]) < 1e-9 * scale
