"""Pins for the oracle's step with a body velocity that changes in time (Sec. 4.6): D^n enters
conv^n and S^n = strain(U^n, D^n), D^{n+1} enters S* = strain(U*, D^{n+1}) and the Poisson
right-hand side cont(U*, D^{n+1}) (Eqs. pm_prediction and pm_poisson), and conv^{n-1} keeps
the D^{n-1} it was formed with.  The body is fixed; its wall turns and blows with the factor
f(t) = a0 + a1 sin(omega t + phase) of a fixed velocity field D0.  CPU only.

What fixes the time levels:
* PmII is second order in time for the velocity, so on a fixed mesh the difference between
  runs at dt and dt/2 falls by about four per halving.  Taking any one of the D-terms at the
  other time level leaves an O(dt) error per unit time, and the ratio falls to about two
  (measured on this case: every such single-term change, and the whole step at one level,
  gives ratios of 2.0 to 2.9 against 3.3 to 4.7).
* After each step the velocity satisfies the constraint of the new level,
  cont(U^{n+1}, D^{n+1}) = 0 to the solver's tolerance, which the old level does not.
* A constant factor reduces the step to the steady-D step exactly."""
import math

import numpy as np
import pytest

from paper_2211_10698_gb300 import inputs as I

# the wall speed ramps up smoothly from rest: f = (1 - cos(omega t)) / 2, two periods per unit time
MOTION = (0.5, 0.5, 4.0 * math.pi, -0.5 * math.pi)


def _case(nsub, T=0.5):
    case = I.small_cylinder(nx=32, ny=32, box=(-1.0, 1.0, -1.0, 1.0), r=0.37, cx=0.03, cy=-0.02,
                            re=50.0, bc=I.flow_past_body_bc(0.0))
    case.mu = 0.02
    case.dt = T / nsub
    case.tol_p = case.tol_h = 1e-13
    case.autotune = 0
    return case


def _d0(o):
    """A turning (omega 2) and blowing (normal speed 0.3) cylinder wall."""
    case = o.case
    args = (o.cap("u", "X"), o.cap("u", "Y"), o.cap("v", "X"), o.cap("v", "Y"), case.geom.cx, case.geom.cy,
            case.geom.r)
    ax, ay = I.rotation_velocity(*args, omega=2.0)
    bx, by = I.transpiration_velocity(*args, w=0.3)
    return ax + bx, ay + by


def _start(orc, case, motion=MOTION):
    """Fluid at rest with the wall at rest (f(0) = 0): a smooth start."""
    o = orc.Oracle(case)
    Dx, Dy = _d0(o)
    st = o.init_state(u0=0.0)
    st["Dx"], st["Dy"], st["motion"] = Dx, Dy, motion
    f0 = I.body_motion_factor(motion, 0, case.dt)
    st["u"][o.role_u == 2] = f0 * Dx[o.role_u == 2]
    st["v"][o.role_v == 2] = f0 * Dy[o.role_v == 2]
    return o, st


def test_moving_wall_velocity_is_second_order_in_time(orc):
    """Self-convergence in time at T = 0.5 on a fixed 32x32 mesh, dt = T/20 .. T/160: each
    halving of dt cuts the change of u and v by more than 3.2 (PmII's second order)."""
    runs = {}
    for n in (20, 40, 80, 160):
        o, st = _start(orc, _case(n))
        hist, _ = o.step(st, n)
        assert all(h["ok"] for h in hist)
        runs[n] = (o, st)
    o = runs[20][0]
    for key, mask in (("u", o.role_u == 3), ("v", o.role_v == 3)):
        e = [np.sqrt(np.mean((runs[a][1][key] - runs[b][1][key])[mask] ** 2))
             for a, b in ((20, 40), (40, 80), (80, 160))]
        assert e[0] / e[1] > 3.2 and e[1] / e[2] > 3.2, (key, e)
        assert e[2] < 4e-5, (key, e)


def test_new_velocity_meets_the_new_level_constraint(orc):
    """cont(U^{n+1}, D^{n+1}) = 0 at every active cell to rounding after each step, while the
    wall's blowing changes between levels, so cont(U^{n+1}, D^n) is of the size of that change;
    the faces whose control volume holds no fluid carry D^{n+1}."""
    case = _case(40)
    o, st = _start(orc, case)
    act = o.cap("p", "V") > 0
    for n in range(1, 6):
        o.step(st, 1)
        f1 = I.body_motion_factor(MOTION, n, case.dt)
        fn = I.body_motion_factor(MOTION, n - 1, case.dt)
        d1 = o.cont(st["u"], st["v"], f1 * st["Dx"], f1 * st["Dy"])
        dn = o.cont(st["u"], st["v"], fn * st["Dx"], fn * st["Dy"])
        assert np.abs(d1[act]).max() < 1e-14
        assert np.abs(dn[act]).max() > 1e3 * max(np.abs(d1[act]).max(), 1e-18)
        assert np.array_equal(st["u"][o.role_u == 2], (f1 * st["Dx"])[o.role_u == 2])
        assert np.array_equal(st["v"][o.role_v == 2], (f1 * st["Dy"])[o.role_v == 2])


def test_constant_factor_is_the_steady_step(orc):
    """f = a0 (a1 = 0) gives bit for bit the step with the steady D = a0 D0."""
    case = _case(40)
    o, st = _start(orc, case, motion=(0.7, 0.0, 3.0, 0.2))
    ref = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in st.items()}
    ref["Dx"], ref["Dy"] = 0.7 * st["Dx"], 0.7 * st["Dy"]
    del ref["motion"]
    o.step(st, 4)
    o.step(ref, 4)
    for k in ("u", "v", "p", "phi", "cu", "cv"):
        assert np.array_equal(st[k], ref[k]), k
