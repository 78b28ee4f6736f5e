"""Seeded synthetic inputs for the cut-cell MAC projection step.

This module describes *problems*, never how they are solved: grid sizes, the box, the
immersed body, the physical constants, the box boundary types, solver settings, and the
random draws (initial velocity perturbations, the mixes of cases used for batched and
served runs).  Both the CUDA library's tests/bench and the FP64 oracle read their inputs
from here; neither the capacities, nor the operators, nor the time step live here.

Conventions shared by every consumer:

* A case has ``nx x ny`` pressure cells on ``[x0, x1] x [y0, y1]``.
* Every field is exchanged as a padded array of shape ``(ny + 3, nx + 3)`` (x fastest):
  array element ``[j + 1, i + 1]`` holds index ``(i, j)`` with ``i`` in ``[-1, nx + 1]`` and
  ``j`` in ``[-1, ny + 1]``.  Index ``(i, j)`` means the pressure cell ``i, j``, the x-face
  ``x0 + i*hx`` (u), the y-face ``y0 + j*hy`` (v) or the node ``(x0 + i*hx, y0 + j*hy)``
  depending on the field.
* Box sides are numbered W=0, E=1, S=2, N=3.  A side is ``DIRICHLET`` (prescribed
  normal component ``bc_un`` and tangential component ``bc_ut``; an inflow is a Dirichlet
  side with ``bc_un = U_inf``), ``OUTFLOW`` (zero-gradient velocity, pressure zero) or
  ``PERIODIC`` (W with E, S with N: face nx is face 0; on a uniform mesh whose cell count
  along that axis is a multiple of 3).
* The time step is ``dt = CFL * min(hx, hy) / U_inf`` and the viscosity
  ``mu = rho * U_inf * L / Re`` with ``L`` the cylinder diameter or the airfoil chord.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

SEED = 2211106980

SIDE_W, SIDE_E, SIDE_S, SIDE_N = 0, 1, 2, 3
BC_DIRICHLET, BC_OUTFLOW, BC_PERIODIC = 0, 1, 2

GEOM_NONE, GEOM_CIRCLE, GEOM_NACA, GEOM_HALFPLANE = 0, 1, 2, 3


@dataclasses.dataclass
class Geometry:
    kind: int = GEOM_NONE
    # circle: fluid where |x - c| > r
    cx: float = 0.0
    cy: float = 0.0
    r: float = 0.0
    # symmetric NACA 4-digit 00tt: leading edge at (le_x, le_y), chord, angle of attack
    naca_tt: int = 12
    chord: float = 1.0
    aoa_deg: float = 0.0
    le_x: float = 0.0
    le_y: float = 0.0
    closed_te: int = 1
    # half plane: fluid where hp_nx * x + hp_ny * y > hp_off
    hp_nx: float = 1.0
    hp_ny: float = 0.0
    hp_off: float = 0.0


@dataclasses.dataclass
class Case:
    name: str
    nx: int
    ny: int
    x0: float
    x1: float
    y0: float
    y1: float
    rho: float
    mu: float
    dt: float
    u_inf: float
    bc_type: Tuple[int, int, int, int]
    bc_un: Tuple[float, float, float, float]
    bc_ut: Tuple[float, float, float, float]
    geom: Geometry
    steps: int = 1
    precision: str = "fp64"        # "fp64" or "mixed"
    precond: str = "jacobi"        # "jacobi" or "chebyshev"
    cheb_degree: int = 4
    tol_p: float = 1e-10
    tol_h: float = 1e-10
    tol_inner: float = 1e-5
    max_iter_p: int = 20000
    max_iter_h: int = 2000
    perturb_sigma: float = 0.0
    seed: int = SEED
    literal_offdiag: int = 0
    pressure_update: int = 0       # volume in the pressure-update correction: 0 hx*hy, 1 V_p, 2 none
    replace_drop: float = 0.5      # mixed one-launch solve: FP32 residual drop per FP64 replacement
    autotune: int = 1              # time launch shapes of the single-case Poisson solve at set-up
    # stretched mesh (Sec. 3.1): face abscissas x_0 = x0 < ... < x_nx = x1 and y_0 < ... < y_ny,
    # or None for the uniform spacing
    xf: Optional[np.ndarray] = None
    yf: Optional[np.ndarray] = None
    # Poisson initial guess: 0 the previous Phi, L > 0 the projection onto the last L solutions
    guess_history: int = 0

    @property
    def stretched(self) -> bool:
        return self.xf is not None or self.yf is not None

    def faces_x(self) -> np.ndarray:
        if self.xf is not None:
            return np.ascontiguousarray(self.xf, dtype=np.float64)
        return self.x0 + np.arange(self.nx + 1) * ((self.x1 - self.x0) / self.nx)

    def faces_y(self) -> np.ndarray:
        if self.yf is not None:
            return np.ascontiguousarray(self.yf, dtype=np.float64)
        return self.y0 + np.arange(self.ny + 1) * ((self.y1 - self.y0) / self.ny)

    @property
    def hx(self) -> float:
        """The uniform spacing, or the smallest spacing of a stretched mesh."""
        if self.stretched:
            return float(np.diff(self.faces_x()).min())
        return (self.x1 - self.x0) / self.nx

    @property
    def hy(self) -> float:
        if self.stretched:
            return float(np.diff(self.faces_y()).min())
        return (self.y1 - self.y0) / self.ny

    @property
    def shape(self) -> Tuple[int, int]:
        return (self.ny + 3, self.nx + 3)

    @property
    def cells(self) -> int:
        return self.nx * self.ny


def flow_past_body_bc(u_inf: float = 1.0):
    """West inflow (u = U_inf, v = 0), outflow on east, south and north."""
    return ((BC_DIRICHLET, BC_OUTFLOW, BC_OUTFLOW, BC_OUTFLOW),
            (u_inf, 0.0, 0.0, 0.0), (0.0, 0.0, 0.0, 0.0))


def closed_box_bc(lid: float = 0.0):
    """Four no-slip walls; the north wall slides with tangential speed ``lid``."""
    return ((BC_DIRICHLET,) * 4, (0.0, 0.0, 0.0, 0.0), (0.0, 0.0, 0.0, lid))


def periodic_bc(x: bool = True, y: bool = True):
    """Periodic W/E (x) and S/N (y) pairs; the other pair no-slip walls."""
    t = (BC_PERIODIC, BC_PERIODIC) if x else (BC_DIRICHLET, BC_DIRICHLET)
    t2 = (BC_PERIODIC, BC_PERIODIC) if y else (BC_DIRICHLET, BC_DIRICHLET)
    return (t + t2, (0.0, 0.0, 0.0, 0.0), (0.0, 0.0, 0.0, 0.0))


def make_case(name, nx, ny, box, geom, re, cfl, lref, *, u_inf=1.0, rho=1.0, bc=None,
              **kw) -> Case:
    x0, x1, y0, y1 = box
    hx, hy = (x1 - x0) / nx, (y1 - y0) / ny
    if kw.get("xf") is not None:
        hx = float(np.diff(kw["xf"]).min())
    if kw.get("yf") is not None:
        hy = float(np.diff(kw["yf"]).min())
    dt = cfl * min(hx, hy) / u_inf
    mu = rho * u_inf * lref / re
    bt, bn, bu = bc if bc is not None else flow_past_body_bc(u_inf)
    return Case(name=name, nx=nx, ny=ny, x0=x0, x1=x1, y0=y0, y1=y1, rho=rho, mu=mu, dt=dt,
                u_inf=u_inf, bc_type=tuple(bt), bc_un=tuple(bn), bc_ut=tuple(bu), geom=geom, **kw)


def cylinder_re40_128x64() -> Case:
    """FP64 single case: 128x64 on [-2,6]x[-2,2], circle D=1 at the origin, Re 40, CFL 0.5,
    100 steps, Jacobi-PCG to 1e-10."""
    return make_case("cylinder_re40_128x64", 128, 64, (-2.0, 6.0, -2.0, 2.0),
                     Geometry(kind=GEOM_CIRCLE, cx=0.0, cy=0.0, r=0.5), re=40.0, cfl=0.5,
                     lref=1.0, steps=100)


def cylinder_re100_1024x512() -> Case:
    """FP64 vortex-shedding case: 1024x512 on [-4,12]x[-4,4], circle D=1, Re 100, CFL 0.5,
    2000 steps, N(0, 1e-3) velocity perturbation, Jacobi-PCG to 1e-10."""
    return make_case("cylinder_re100_1024x512", 1024, 512, (-4.0, 12.0, -4.0, 4.0),
                     Geometry(kind=GEOM_CIRCLE, cx=0.0, cy=0.0, r=0.5), re=100.0, cfl=0.5,
                     lref=1.0, steps=2000, perturb_sigma=1e-3)


def naca0012_re1000_2048x1024() -> Case:
    """Mixed-precision airfoil: NACA0012, chord 1, 4 deg, leading edge at the origin,
    Re 1000, 2048x1024 on [-2,6]x[-2,2], 1000 steps, Chebyshev-PCG FP32 inner with FP64
    refinement to 1e-10.  Degree 3: on this grid degrees 3, 4, 6 and 8 took 105, 111, 126
    and 145 ms per step (the one-launch solve is bound by its barriers, and the iteration
    count falls more slowly than the barriers per iteration rise)."""
    return make_case("naca0012_re1000_2048x1024", 2048, 1024, (-2.0, 6.0, -2.0, 2.0),
                     Geometry(kind=GEOM_NACA, naca_tt=12, chord=1.0, aoa_deg=4.0),
                     re=1000.0, cfl=0.5, lref=1.0, steps=1000, precision="mixed",
                     precond="chebyshev", cheb_degree=3)


def batch_cases(n: int = 64, seed: int = SEED, steps: int = 500,
                nx_range=(256, 1024)) -> List[Case]:
    """Batched mix: half cylinders (D ~ U[0.5,1.5], centre ~ U[-0.5,0.5]^2), half NACA00tt
    (tt uniform in 08..18, AoA ~ U[0,10] deg); nx log-uniform in ``nx_range`` rounded to a
    multiple of 16, ny = nx/2, box [-2,6]x[-2,2]; Re ~ U[40,1000]; mixed precision.  In a
    batch an FP64 residual replacement holds up every case for its slots, so these cases
    replace after a fourfold FP32 residual drop (0.25) instead of twofold."""
    out = []
    for k in range(n):
        rng = np.random.default_rng(seed + k)
        nx = int(round(math.exp(rng.uniform(math.log(nx_range[0]), math.log(nx_range[1]))) / 16.0)) * 16
        nx = max(nx, 16)
        ny = nx // 2
        re = float(rng.uniform(40.0, 1000.0))
        if k % 2 == 0:
            d = float(rng.uniform(0.5, 1.5))
            c = rng.uniform(-0.5, 0.5, size=2)
            geom = Geometry(kind=GEOM_CIRCLE, cx=float(c[0]), cy=float(c[1]), r=0.5 * d)
            lref = d
        else:
            tt = int(rng.integers(8, 19))
            aoa = float(rng.uniform(0.0, 10.0))
            geom = Geometry(kind=GEOM_NACA, naca_tt=tt, chord=1.0, aoa_deg=aoa)
            lref = 1.0
        out.append(make_case(f"batch{k:03d}", nx, ny, (-2.0, 6.0, -2.0, 2.0), geom, re=re,
                             cfl=0.5, lref=lref, steps=steps, precision="mixed",
                             precond="chebyshev", seed=seed + k, autotune=0, replace_drop=0.25))
    return out


def serving_requests(n: int = 1000, lam: float = 20.0, seed: int = SEED,
                     nx_range=(128, 2048), steps_range=(200, 5000)):
    """Request stream: exponential inter-arrival times with rate ``lam`` per second;
    geometry and Re drawn like ``batch_cases``; nx log-uniform in ``nx_range``; steps
    uniform in ``steps_range``.  Returns a list of (arrival_time_s, Case)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / lam, size=n)
    t = np.cumsum(gaps)
    reqs = []
    for k in range(n):
        c = batch_cases(1, seed=seed + 100000 + k, nx_range=nx_range)[0]
        r2 = np.random.default_rng(seed + 200000 + k)
        c.steps = int(r2.integers(steps_range[0], steps_range[1] + 1))
        c.name = f"req{k:04d}"
        reqs.append((float(t[k]), c))
    return reqs


def perturbation(case: Case) -> Tuple[np.ndarray, np.ndarray]:
    """Seeded N(0, sigma^2) draws for the u and v arrays (padded shape).  Consumers add them
    on the velocity unknowns whose staggered control volume holds fluid."""
    rng = np.random.default_rng(case.seed)
    pu = rng.standard_normal(case.shape) * case.perturb_sigma
    pv = rng.standard_normal(case.shape) * case.perturb_sigma
    return pu, pv


def random_field(case: Case, seed: int, scale: float = 1.0) -> np.ndarray:
    """A seeded N(0, scale^2) padded array, for operator parity inputs."""
    return np.random.default_rng(seed).standard_normal(case.shape) * scale


def stretched_faces(n: int, a: float, b: float, nfine: int, h: float, ratio: float) -> np.ndarray:
    """Face abscissas of a mesh on [a, b] with ``nfine`` cells of size h centred on 0 and cells
    growing by ``ratio`` per cell outwards; each side's growing cells are scaled together so
    that the faces end at a and b.  Returns n + 1 increasing values, x_0 = a, x_n = b."""
    ns = n - nfine
    nl = int(round(ns * (0.0 - a) / (b - a)))
    nr = ns - nl
    f0, f1 = -0.5 * nfine * h, 0.5 * nfine * h
    assert a < f0 and f1 < b and nl >= 1 and nr >= 1
    gl = h * ratio ** np.arange(1, nl + 1)
    gr = h * ratio ** np.arange(1, nr + 1)
    gl *= (f0 - a) / gl.sum()
    gr *= (b - f1) / gr.sum()
    x = np.concatenate([(f0 - np.cumsum(gl))[::-1], f0 + h * np.arange(nfine + 1), f1 + np.cumsum(gr)])
    x[0], x[-1] = a, b
    return x


def stretched_cylinder(nx=64, ny=48, box=(-3.0, 7.0, -3.0, 3.0), r=0.5, fine=(24, 24), h_fine=0.08,
                       ratio=1.08, re=100.0, cfl=0.5, **kw) -> Case:
    """A cylinder at the origin on a mesh that is uniform (spacing ``h_fine``) over ``fine``
    cells around the body and stretched geometrically towards the box (Sec. 3.1; the paper's
    grids G1-G3 are of this kind, their stretching laws not given)."""
    xf = stretched_faces(nx, box[0], box[1], fine[0], h_fine, ratio)
    yf = stretched_faces(ny, box[2], box[3], fine[1], h_fine, ratio)
    return make_case(f"stretched_cyl_{nx}x{ny}", nx, ny, box, Geometry(kind=GEOM_CIRCLE, r=r), re=re, cfl=cfl,
                     lref=2 * r, xf=xf, yf=yf, **kw)


# ---------------------------------------------------------------------------------------------
# Taylor-Green vortex in the doubly periodic box [0, 2 pi]^2 (rho = 1): an exact solution of the
# incompressible Navier-Stokes equations,
#   u = -cos x sin y F(t),  v = sin x cos y F(t),  p = -(cos 2x + cos 2y) F(t)^2 / 4,
#   F(t) = exp(-2 nu t).
# ---------------------------------------------------------------------------------------------
def taylor_green(n: int, nu: float = 0.05, cfl: float = 0.25, u_ref: float = 1.0) -> Case:
    """The doubly periodic Taylor-Green box with n x n cells (n a multiple of 3)."""
    L = 2.0 * math.pi
    case = make_case(f"taylor_green_{n}", n, n, (0.0, L, 0.0, L), Geometry(kind=GEOM_NONE), re=1.0, cfl=cfl,
                     lref=1.0, u_inf=u_ref, bc=periodic_bc(True, True))
    case.mu = nu * case.rho
    case.autotune = 0
    return case


def taylor_green_exact(case: Case, t: float):
    """Padded arrays of the exact u (u-faces), v (v-faces) and p (cell centres) at time t."""
    xf, xc, yf, yc = mesh_positions(case)
    F = math.exp(-2.0 * case.mu / case.rho * t)
    XU, YU = np.meshgrid(xf, yc)
    XV, YV = np.meshgrid(xc, yf)
    XP, YP = np.meshgrid(xc, yc)
    u = -np.cos(XU) * np.sin(YU) * F
    v = np.sin(XV) * np.cos(YV) * F
    p = -(np.cos(2 * XP) + np.cos(2 * YP)) * F * F / 4.0
    return u, v, p


def small_cylinder(nx=16, ny=8, box=(-2.0, 2.0, -1.0, 1.0), r=0.37, cx=0.05, cy=-0.03,
                   re=40.0, cfl=0.5, bc=None, **kw) -> Case:
    """A small off-centre cylinder case for dense and brute-force tests."""
    return make_case(f"small_cyl_{nx}x{ny}", nx, ny, box,
                     Geometry(kind=GEOM_CIRCLE, cx=cx, cy=cy, r=r), re=re, cfl=cfl,
                     lref=2 * r, bc=bc, **kw)


# ---------------------------------------------------------------------------------------------
# Manufactured steady solution in a closed no-slip box (body free): the body acceleration g of
# Eq. pm_prediction that makes
#   u = sin^2(pi x) sin(2 pi y),  v = -sin(2 pi x) sin^2(pi y),  p = cos(pi x) cos(pi y)
# a steady solution of rho (U.grad) U + grad p - mu lap U = rho g on [0,1]^2.  U is divergence
# free and vanishes on the walls; p has mean zero.
# ---------------------------------------------------------------------------------------------
def mms_box(n: int, mu: float = 0.2, cfl: float = 0.5) -> Case:
    case = make_case(f"mms_box_{n}", n, n, (0.0, 1.0, 0.0, 1.0), Geometry(kind=GEOM_NONE), re=1.0, cfl=cfl,
                     lref=1.0, bc=closed_box_bc())
    case.mu = mu
    case.autotune = 0
    return case


def mms_exact(x, y, rho: float, mu: float):
    """(u, v, p, g_x, g_y) of the manufactured solution at points (x, y)."""
    pi = np.pi
    s1, c1 = np.sin(pi * x), np.cos(pi * x)
    s1y, c1y = np.sin(pi * y), np.cos(pi * y)
    s2x, c2x = np.sin(2 * pi * x), np.cos(2 * pi * x)
    s2y, c2y = np.sin(2 * pi * y), np.cos(2 * pi * y)
    u = s1 ** 2 * s2y
    v = -s2x * s1y ** 2
    p = c1 * c1y
    ux, uy = pi * s2x * s2y, 2 * pi * s1 ** 2 * c2y
    vx, vy = -2 * pi * c2x * s1y ** 2, -pi * s2x * s2y
    lap_u = 2 * pi ** 2 * c2x * s2y - 4 * pi ** 2 * s1 ** 2 * s2y
    lap_v = 4 * pi ** 2 * s2x * s1y ** 2 - 2 * pi ** 2 * s2x * c2y
    px, py = -pi * s1 * c1y, -pi * c1 * s1y
    nu = mu / rho
    gx = u * ux + v * uy + px / rho - nu * lap_u
    gy = u * vx + v * vy + py / rho - nu * lap_v
    return u, v, p, gx, gy


def mesh_positions(case: Case):
    """Face and centre coordinates for index i in [-1, nx+1] (and j likewise): the face x_i and
    the centre of pressure cell i.  On a stretched mesh the spacing beyond the box mirrors the
    spacing inside it."""
    if not case.stretched:
        i = np.arange(-1, case.nx + 2, dtype=np.float64)
        j = np.arange(-1, case.ny + 2, dtype=np.float64)
        return (case.x0 + i * case.hx, case.x0 + (i + 0.5) * case.hx,
                case.y0 + j * case.hy, case.y0 + (j + 0.5) * case.hy)

    def ext(f):  # faces -1 .. n+2
        return np.concatenate([[2 * f[0] - f[1]], f, [2 * f[-1] - f[-2], 2 * f[-1] - f[-3]]])

    fx, fy = ext(case.faces_x()), ext(case.faces_y())
    return fx[:-1], 0.5 * (fx[:-1] + fx[1:]), fy[:-1], 0.5 * (fy[:-1] + fy[1:])


def mms_fields(case: Case):
    """Padded arrays of the manufactured solution: u and g_x at u-faces, v and g_y at v-faces,
    p at cell centres, for index i in [-1, nx+1]."""
    xf, xc, yf, yc = mesh_positions(case)
    XU, YU = np.meshgrid(xf, yc)
    XV, YV = np.meshgrid(xc, yf)
    XP, YP = np.meshgrid(xc, yc)
    u, _, _, gx, _ = mms_exact(XU, YU, case.rho, case.mu)
    _, v, _, _, gy = mms_exact(XV, YV, case.rho, case.mu)
    _, _, p, _, _ = mms_exact(XP, YP, case.rho, case.mu)
    return u, v, p, gx, gy


# ---------------------------------------------------------------------------------------------
# Manufactured steady solution around a rotating cylinder: a compactly supported vortex
#   u_theta(r) = A r (1 - r^2/R^2)^3 (r < R), 0 beyond,  p = 0,
# centred on the cylinder (radius r0 < R) in the closed no-slip unit box.  Its streamlines are
# circles, so the body's velocity D = u_theta(r0) e_theta has no normal component.  The body
# acceleration g = (U.grad)U - nu lap U (azimuthal part 24 nu A r q (1 - 2 r^2/R^2) / R^2,
# radial part -u_theta^2 / r, q = 1 - r^2/R^2) makes it a steady solution.
# ---------------------------------------------------------------------------------------------
VORTEX = dict(A=2.0, R=0.45, cx=0.5, cy=0.5, r0=0.2)


def vortex_box(n: int, mu: float = 0.2) -> Case:
    case = mms_box(n, mu)
    case.name = f"vortex_box_{n}"
    case.geom = Geometry(kind=GEOM_CIRCLE, cx=VORTEX["cx"], cy=VORTEX["cy"], r=VORTEX["r0"])
    return case


def vortex_exact(x, y, rho: float, mu: float):
    """(u, v, g_x, g_y) of the vortex at points (x, y)."""
    A, R = VORTEX["A"], VORTEX["R"]
    dx, dy = x - VORTEX["cx"], y - VORTEX["cy"]
    r2 = dx * dx + dy * dy
    q = np.where(r2 < R * R, 1.0 - r2 / R ** 2, 0.0)
    nu = mu / rho
    k = 24.0 * nu * A * q * (1.0 - 2.0 * r2 / R ** 2) / R ** 2
    return (-A * dy * q ** 3, A * dx * q ** 3,
            -A ** 2 * q ** 6 * dx - k * dy, -A ** 2 * q ** 6 * dy + k * dx)


def vortex_fields(case: Case):
    """Padded arrays: u, g_x at u-faces; v, g_y at v-faces."""
    i = np.arange(-1, case.nx + 2, dtype=np.float64)
    j = np.arange(-1, case.ny + 2, dtype=np.float64)
    XU, YU = np.meshgrid(case.x0 + i * case.hx, case.y0 + (j + 0.5) * case.hy)
    XV, YV = np.meshgrid(case.x0 + (i + 0.5) * case.hx, case.y0 + j * case.hy)
    u, _, gx, _ = vortex_exact(XU, YU, case.rho, case.mu)
    _, v, _, gy = vortex_exact(XV, YV, case.rho, case.mu)
    return u, v, gx, gy


def circle_boundary_points(X, Y, cx: float, cy: float, r: float):
    """Where the boundary of a circular body meets the ray from its centre through each control
    volume's fluid centroid (X, Y): the point at which a body velocity is sampled for D."""
    dx, dy = X - cx, Y - cy
    d = np.hypot(dx, dy)
    d = np.where(d > 0, d, 1.0)
    return cx + r * dx / d, cy + r * dy / d


def body_motion_factor(motion, n: int, dt: float) -> float:
    """The prescribed time law of a body velocity D(t) = D0 f(t): with motion = (a0, a1, omega,
    phase), f = a0 + a1 sin(omega t + phase) at t = n dt (the time of step n).  Boundary data,
    evaluated the same way by the library (ccm_set_body_motion)."""
    a0, a1, omega, phase = motion
    t = float(n) * dt
    return a0 + a1 * math.sin(omega * t + phase)


def rotation_velocity(Xu, Yu, Xv, Yv, cx: float, cy: float, r: float, omega: float = 1.0):
    """(Dx per u-cell, Dy per v-cell) of a circle of radius r about (cx, cy) turning at the
    angular velocity omega, sampled at the boundary points of the control volumes whose fluid
    centroids are (Xu, Yu), (Xv, Yv)."""
    xu, yu = circle_boundary_points(Xu, Yu, cx, cy, r)
    xv, yv = circle_boundary_points(Xv, Yv, cx, cy, r)
    return -omega * (yu - cy), omega * (xv - cx)


def transpiration_velocity(Xu, Yu, Xv, Yv, cx: float, cy: float, r: float, w: float = 1.0):
    """(Dx, Dy) of a porous circle that blows out (w > 0) or sucks in at the normal speed w,
    sampled like rotation_velocity."""
    xu, yu = circle_boundary_points(Xu, Yu, cx, cy, r)
    xv, yv = circle_boundary_points(Xv, Yv, cx, cy, r)
    return w * (xu - cx) / r, w * (yv - cy) / r


def vortex_body_velocity(case: Case, Xu, Yu, Xv, Yv):
    """(Dx per u-cell, Dy per v-cell): the vortex's velocity on the cylinder, sampled at the
    boundary points of the u- and v-control volumes whose centroids are (Xu, Yu), (Xv, Yv)."""
    c = VORTEX
    xu, yu = circle_boundary_points(Xu, Yu, c["cx"], c["cy"], c["r0"])
    xv, yv = circle_boundary_points(Xv, Yv, c["cx"], c["cy"], c["r0"])
    return vortex_exact(xu, yu, case.rho, case.mu)[0], vortex_exact(xv, yv, case.rho, case.mu)[1]
