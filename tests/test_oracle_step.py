"""Pins for the oracle's linear solvers and its PmII step (Sec. 4.6): brute-force dense
solves, operator structure, and physical solutions the step must reproduce.  CPU only."""
import numpy as np
import pytest

import oracle as O
from paper_2211_10698_gb300 import inputs as I


def _cyl(nx=16, ny=8, **kw):
    return I.small_cylinder(nx=nx, ny=ny, **kw)


@pytest.mark.parametrize("precond", ["jacobi", "chebyshev"])
def test_poisson_pcg_matches_dense_solve(orc, precond):
    """PCG on K Phi = b agrees with a dense LU solve (brute force, 16x8 with a circle)."""
    case = _cyl()
    o = orc.Oracle(case, precond=precond)
    act = o.active
    K = O.dense(o.poisson, o.shape, act, act)
    assert np.abs(K - K.T).max() < 1e-14 * np.abs(K).max()
    assert np.linalg.eigvalsh(K).min() > 0
    b = np.random.default_rng(1).standard_normal(o.shape) * act
    phi, info = o.solve_poisson(b, tol=1e-14, max_iter=5000)
    assert info["converged"]
    ref = np.linalg.solve(K, b[act])
    assert np.abs(phi[act] - ref).max() < 1e-10 * np.abs(ref).max()
    assert np.all(phi[~act] == 0)


def test_chebyshev_cuts_iterations(orc):
    case = _cyl(32, 16)
    b = None
    its = {}
    for pc in ("jacobi", "chebyshev"):
        o = orc.Oracle(case, precond=pc)
        if b is None:
            b = np.random.default_rng(4).standard_normal(o.shape) * o.active
        _, info = o.solve_poisson(b, tol=1e-10)
        its[pc] = info["iters"]
    assert its["chebyshev"] < 0.6 * its["jacobi"], its


def _chebyshev_q(k, a, b):
    """q_k(lam) = (1 - T_k((theta - lam)/delta) / T_k(theta/delta)) / lam, theta = (a+b)/2,
    delta = (b-a)/2: the polynomial that k steps of Chebyshev acceleration from zero apply to
    the residual (Saad, Iterative Methods for Sparse Linear Systems, Chebyshev acceleration).
    Built from numpy's Chebyshev-to-power conversion and composed exactly."""
    from numpy.polynomial import Polynomial, chebyshev as C
    theta, delta = 0.5 * (b + a), 0.5 * (b - a)
    tk = Polynomial(C.cheb2poly([0.0] * k + [1.0]))
    p = tk(Polynomial([theta / delta, -1.0 / delta])) / tk(theta / delta)
    q, rem = divmod(1.0 - p, Polynomial([0.0, 1.0]))
    assert np.abs(rem.coef).max() < 1e-12
    return q


@pytest.mark.parametrize("degree", [1, 2, 3, 4])
def test_chebyshev_preconditioner_closed_form(orc, degree):
    """The Chebyshev preconditioner is z = D^-1/2 q_k(K~) D^-1/2 r with K~ = D^-1/2 K D^-1/2
    the Jacobi-scaled operator on [a, b] = [2/30, 2]: on each eigenvector v of K~ (eigenvalue
    lam), r = D^1/2 v gives z = q_k(lam) D^-1/2 v.  Dense eigenpairs on a 16x8 cut circle."""
    case = _cyl()
    case.precond, case.cheb_degree = "chebyshev", degree
    o = orc.Oracle(case)
    dom = np.zeros(o.shape, dtype=bool)
    dom[1:-2, 1:-2] = True
    K = O.dense(o.poisson, o.shape, dom, dom)
    d = o.poisson_diag()[dom]
    assert np.all(d > 0)
    Ks = K / np.sqrt(np.outer(d, d))
    lam, V = np.linalg.eigh(Ks)
    q = _chebyshev_q(degree, 2.0 / 30.0, 2.0)
    qmax = np.abs(q(lam)).max()     # the scale of z: rounding is relative to it, not to q(lam)
    for col in range(V.shape[1]):
        r = np.zeros(o.shape)
        r[dom] = np.sqrt(d) * V[:, col]
        z = o.poisson_precondition(r)
        want = q(lam[col]) * V[:, col] / np.sqrt(d)
        assert np.abs(z[dom] - want).max() <= 1e-13 * qmax * np.abs(V[:, col] / np.sqrt(d)).max(), \
            (col, lam[col])
        assert np.all(z[~dom] == 0)
    # a random residual: the same polynomial of the whole operator
    r = np.random.default_rng(5).standard_normal(o.shape) * dom
    z = o.poisson_precondition(r)
    want = (V * q(lam)) @ (V.T @ (r[dom] / np.sqrt(d))) / np.sqrt(d)
    assert np.abs(z[dom] - want).max() <= 1e-13 * np.abs(want).max()


def test_singular_poisson_zero_mean(orc):
    """All-Dirichlet velocity box: K is singular with the constants as null space; the
    iterates are kept zero-mean (end of Sec. 4.6)."""
    case = I.small_cylinder(nx=12, ny=8, box=(-1.5, 1.5, -1.0, 1.0), r=0.41, bc=I.closed_box_bc())
    o = orc.Oracle(case)
    act = o.active
    K = O.dense(o.poisson, o.shape, act, act)
    w = np.linalg.eigvalsh(K)
    assert abs(w[0]) < 1e-12 * w[-1] and w[1] > 1e-6 * w[-1]
    b = np.random.default_rng(2).standard_normal(o.shape) * act
    b[act] -= b[act].mean()
    phi, info = o.solve_poisson(b, tol=1e-13, max_iter=5000)
    assert info["converged"]
    assert abs(phi[act].mean()) < 1e-12
    ref = np.linalg.lstsq(K, b[act], rcond=None)[0]
    ref -= ref.mean()
    assert np.abs(phi[act] - ref).max() < 1e-9 * np.abs(ref).max()


def test_helmholtz_pcg_matches_dense_solve(orc):
    case = _cyl()
    o = orc.Oracle(case)
    unk = np.stack([o.role_u == 3, o.role_v == 3])
    H = O.dense(lambda e: np.stack(o.helmholtz(e[0], e[1])), unk.shape, unk, unk)
    rng = np.random.default_rng(3)
    ru = rng.standard_normal(o.shape) * unk[0]
    rv = rng.standard_normal(o.shape) * unk[1]
    xu, xv, info = o.solve_helmholtz(ru, rv, tol=1e-14, max_iter=2000)
    assert info["converged"]
    ref = np.linalg.solve(H, np.concatenate([ru[unk[0]], rv[unk[1]]]))
    got = np.concatenate([xu[unk[0]], xv[unk[1]]])
    assert np.abs(got - ref).max() < 1e-11 * np.abs(ref).max()


def test_diagonal_probes_match_dense_diagonals(orc):
    case = _cyl(12, 8)
    o = orc.Oracle(case)
    act = o.active
    K = O.dense(o.poisson, o.shape, act, act)
    assert np.array_equal(o.poisson_diag()[act], np.diag(K))
    unk = np.stack([o.role_u == 3, o.role_v == 3])
    H = O.dense(lambda e: np.stack(o.helmholtz(e[0], e[1])), unk.shape, unk, unk)
    du, dv = o.helmholtz_diag()
    np.testing.assert_allclose(np.concatenate([du[unk[0]], dv[unk[1]]]), np.diag(H), rtol=1e-14)
    # inactive faces are identity rows
    assert np.all(du[o.role_u == 2] == 1.0) and np.all(dv[o.role_v == 2] == 1.0)


def test_uniform_flow_is_steady_without_body(orc):
    """With no body, u = U_inf, v = 0 satisfies every equation of the step exactly."""
    case = I.make_case("free", 16, 8, (0.0, 2.0, -0.5, 0.5), I.Geometry(), re=50, cfl=0.5, lref=1.0)
    o = orc.Oracle(case)
    st = o.init_state()
    hist, _ = o.step(st, 3)
    assert np.abs(st["u"][1:-1, 1:-1] - 1.0).max() < 1e-13
    assert np.abs(st["v"]).max() < 1e-13 and np.abs(st["p"]).max() < 1e-12


def test_step_projects_to_divergence_free(orc):
    case = _cyl(32, 16)
    case.tol_p = 1e-12
    o = orc.Oracle(case)
    st = o.init_state()
    hist, extra = o.step(st, 2, keep=True)
    b = extra["b"]
    assert o.max_div(st["u"], st["v"]) < 1e-10 * np.abs(b[o.active]).max()
    # mass: the sum of cont over all cells is the net flux through the box sides
    d = o.cont(st["u"], st["v"])
    Ax, Ay = o.cap("p", "AX"), o.cap("p", "AY")
    nx, ny = case.nx, case.ny
    u, v = st["u"], st["v"]
    flux = sum(o.at(Ax, nx, j) * o.at(u, nx, j) - o.at(Ax, 0, j) * o.at(u, 0, j) for j in range(ny)) + \
        sum(o.at(Ay, i, ny) * o.at(v, i, ny) - o.at(Ay, i, 0) * o.at(v, i, 0) for i in range(nx))
    assert d[1:-2, 1:-2].sum() == pytest.approx(flux, abs=1e-13)


def test_poiseuille_channel(orc):
    """Plane channel (no-slip walls on S and N, uniform inflow on W, outflow on E): the
    developed flow is the Poiseuille profile, u_max = 3/2 U_mean, with the pressure
    gradient dP/dx = -12 mu U_mean / H^2 (Sec. 4.6 step with the viscous and pressure
    operators at their physical scale)."""
    H = 1.0
    bc = ((I.BC_DIRICHLET, I.BC_OUTFLOW, I.BC_DIRICHLET, I.BC_DIRICHLET),
          (1.0, 0.0, 0.0, 0.0), (0.0, 0.0, 0.0, 0.0))
    case = I.make_case("chan", 48, 12, (0.0, 4.0, 0.0, H), I.Geometry(), re=1.0, cfl=0.5, lref=1.0,
                       bc=bc)
    case.tol_p = case.tol_h = 1e-12
    o = orc.Oracle(case)
    st = o.init_state()
    o.step(st, 120)
    u = st["u"]
    ny = case.ny
    i = 3 * case.nx // 4
    prof = np.array([o.at(u, i, j) for j in range(ny)])
    y = (np.arange(ny) + 0.5) * case.hy
    # discrete Poiseuille with no-slip at the walls, normalised to the mean flow
    exact = 6.0 * y * (H - y) / H ** 2
    assert np.abs(prof - exact).max() < 2e-2 * 1.5
    P = st["p"]
    j0 = ny // 2
    dpdx = (o.at(P, i + 1, j0) - o.at(P, i - 1, j0)) / (2 * case.hx)
    assert dpdx == pytest.approx(-12.0 * case.mu * 1.0 / H ** 2, rel=3e-2)


def test_kinetic_energy_decays_in_closed_box(orc):
    """Closed box, no inflow: viscous dissipation (Sec. 4.3) makes the discrete kinetic
    energy (Sec. 4.4) decrease monotonically from a divergence-free start."""
    case = I.small_cylinder(nx=16, ny=12, box=(-1.5, 1.5, -1.0, 1.0), r=0.41, bc=I.closed_box_bc(),
                            re=20.0, cfl=0.2)
    case.tol_p = case.tol_h = 1e-12
    o = orc.Oracle(case)
    rng = np.random.default_rng(11)
    st = o.init_state(u0=0.0)
    st["u"] = rng.standard_normal(o.shape) * (o.role_u == 3)
    st["v"] = rng.standard_normal(o.shape) * (o.role_v == 3)
    hist, _ = o.step(st, 1)
    ke = [h["kinetic"] for h in o.step(st, 15)[0]]
    assert all(b < a for a, b in zip(ke, ke[1:])), ke


def test_semidiscrete_energy_budget(orc):
    """For a divergence-free U with D = 0, U^T(-conv(U) + visc(2 mu S(U))) <= 0: convection
    exchanges no energy (Eq. kinetic) and viscosity dissipates (Sec. 1)."""
    case = I.small_cylinder(nx=12, ny=8, box=(-1.5, 1.5, -1.0, 1.0), r=0.41, bc=I.closed_box_bc())
    o = orc.Oracle(case)
    from tests.test_oracle_operators import _div_free
    u, v = _div_free(o, 9)
    cu, cv = o.conv(u, v)
    vu, vv = o.visc_bc(u, v)
    mu_ = o.role_u == 3
    mv_ = o.role_v == 3
    e_conv = (u * cu * mu_).sum() + (v * cv * mv_).sum()
    e_visc = (u * vu * mu_).sum() + (v * vv * mv_).sum()
    assert abs(e_conv) < 1e-12 * (abs(e_visc) + 1)
    assert e_visc < 0


def test_conservation_sums(orc):
    """The mass sum of the diagnostics telescopes: the sum of cont(U, 0) over the box cells is the
    net flux A u through the box's faces (Eq. divergence, interior faces cancel; the body's
    faces are dry); the momentum sums are the volume-weighted velocity sums."""
    import numpy as np

    from paper_2211_10698_gb300 import inputs as I

    case = I.small_cylinder(nx=40, ny=20, box=(-2.0, 4.0, -1.5, 1.5), r=0.45, cx=0.1, cy=0.05)
    o = orc.Oracle(case)
    rng = np.random.default_rng(4)
    u = rng.standard_normal(o.shape) * (o.cap("u", "V") > 0)
    v = rng.standard_normal(o.shape) * (o.cap("v", "V") > 0)
    m, px, py = o.conservation(u, v)
    Ax, Ay = o.cap("p", "AX"), o.cap("p", "AY")
    nx, ny = case.nx, case.ny
    flux = ((Ax[1:ny + 1, nx + 1] * u[1:ny + 1, nx + 1]).sum() - (Ax[1:ny + 1, 1] * u[1:ny + 1, 1]).sum()
            + (Ay[ny + 1, 1:nx + 1] * v[ny + 1, 1:nx + 1]).sum() - (Ay[1, 1:nx + 1] * v[1, 1:nx + 1]).sum())
    assert m == pytest.approx(flux, abs=1e-12 * np.abs(u).sum())
    assert abs(m) > 1e-3                     # not trivially zero for a random field
    assert px == pytest.approx((o.cap("u", "V") * u)[1:ny + 1, 1:nx + 2].sum(), rel=1e-13)
    assert py == pytest.approx((o.cap("v", "V") * v)[1:ny + 2, 1:nx + 1].sum(), rel=1e-13)


def test_oracle_threads_bitwise(orc):
    """The oracle's sums run over fixed blocks in a fixed order, so a run on one thread and a run
    on four give the same fields bit for bit (the grid spans several summation blocks)."""
    case = I.small_cylinder(nx=160, ny=80, box=(-2.0, 6.0, -2.0, 2.0), r=0.5)
    out = []
    for t in (1, 4):
        prev = O.set_threads(t)
        try:
            o = orc.Oracle(case)
            s = o.init_state()
            hist, _ = o.step(s, 3)
        finally:
            O.set_threads(0)
        assert all(h["ok"] for h in hist) and prev >= 1
        out.append((s["u"].copy(), s["v"].copy(), s["p"].copy(), [h["iters_p"] for h in hist]))
    for a, b in zip(out[0][:3], out[1][:3]):
        assert np.array_equal(a, b)
    assert out[0][3] == out[1][3]
