"""Drag, lift and Strouhal number from the force on the body.

Sec. 5 of the paper reports, for the cylinder at Re 100, the Strouhal number, the r.m.s. lift
coefficient and the mean drag coefficient (and for the NACA 0010 at Re 500 the Strouhal number
and the mean coefficients).  The library returns the force per step (``Case.body_force`` or the
per-step record of ``Case.set_force_history``); this module turns a record into those numbers:

- step filter: the viscous force of a state alternates in sign from one step to the next in
  cut cells of small volume (their viscous modes are stiff, and the Crank-Nicolson factor of a
  stiff mode is close to -1), so the record is filtered with the weights (1, 2, 1) / 4 over
  consecutive steps, which removes a mode alternating with the step even when its amplitude
  drifts linearly, and scales a frequency f by cos^2(pi f dt) (1 - 3e-4 for the cylinder's
  shedding at dt = 1/32);
- coefficients: C = F / (rho U^2 L / 2) with F the pressure plus viscous force;
- Strouhal number St = f L / U, f the lift's dominant frequency, estimated from the upward
  crossings of the lift's mean (linear interpolation between steps), averaged over the whole
  periods in the window.

``python -m paper_2211_10698_gb300.forces`` runs a cylinder in uniform flow until shedding
settles and prints these numbers as one JSON line (a GPU run).
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np


def coefficients(force, rho: float, u_inf: float, lref: float) -> np.ndarray:
    """(C_d, C_l) per row of ``force`` (rows of Fp_x, Fp_y, Fv_x, Fv_y)."""
    f = np.atleast_2d(np.asarray(force, dtype=np.float64))
    q = 0.5 * rho * u_inf ** 2 * lref
    return np.stack([(f[:, 0] + f[:, 2]) / q, (f[:, 1] + f[:, 3]) / q], axis=1)


def step_filter(rows) -> np.ndarray:
    """(1, 2, 1) / 4 over consecutive rows (steps); two rows shorter than the input."""
    r = np.asarray(rows, dtype=np.float64)
    if r.shape[0] < 3:
        raise ValueError("the step filter needs three rows")
    return 0.25 * r[:-2] + 0.5 * r[1:-1] + 0.25 * r[2:]


def mean_up_crossings(signal, dt: float) -> np.ndarray:
    """Times at which ``signal`` (sampled every dt from t = 0) crosses its mean upwards."""
    x = np.asarray(signal, dtype=np.float64)
    x = x - x.mean()
    k = np.nonzero((x[:-1] < 0.0) & (x[1:] >= 0.0))[0]
    return (k + (-x[k]) / (x[k + 1] - x[k])) * dt


def strouhal(lift, dt: float, lref: float, u_inf: float):
    """(St, whole periods used) from a lift record sampled every dt.  Raises ValueError when
    the record holds fewer than two upward crossings of its mean."""
    t = mean_up_crossings(lift, dt)
    if len(t) < 2:
        raise ValueError("the lift record holds less than one period")
    f = (len(t) - 1) / (t[-1] - t[0])
    return f * lref / u_inf, len(t) - 1


def rms(x) -> float:
    x = np.asarray(x, dtype=np.float64)
    return float(np.sqrt(np.mean((x - x.mean()) ** 2)))


def shedding(case, t_end: float, t_avg: float, chunk: int = 200, perturb: bool = True):
    """Advance ``case`` (an ``inputs.Case`` with a body) to t_end recording the force every step;
    returns the statistics over the last t_avg time units and the run's throughput."""
    from . import ccm, inputs

    steps = int(round(t_end / case.dt))
    keep = int(round(t_avg / case.dt))
    if perturb and case.perturb_sigma == 0.0:
        case.perturb_sigma = 1e-3
    c = ccm.Case(case)
    if case.perturb_sigma > 0.0:
        pu, pv = inputs.perturbation(case)
        c.set_field(ccm.CCM_F_U, c.get_field(ccm.CCM_F_U) + pu)
        c.set_field(ccm.CCM_F_V, c.get_field(ccm.CCM_F_V) + pv)
    c.set_force_history(keep)
    t0 = time.perf_counter()
    done, iters_p = 0, 0
    while done < steps:
        n = min(chunk, steps - done)
        st = c.step(n)
        iters_p += st["iters_p"]
        done += n
    wall = time.perf_counter() - t0
    hist, total = c.force_history()
    lref = 2.0 * case.geom.r if case.geom.kind == inputs.GEOM_CIRCLE else case.geom.chord
    hist = step_filter(hist)
    cdl = coefficients(hist, case.rho, case.u_inf, lref)
    st_num, periods = strouhal(cdl[:, 1], case.dt, lref, case.u_inf)
    return dict(steps=steps, t_end=steps * case.dt, t_avg=len(hist) * case.dt, strouhal=st_num, periods=periods,
                cd_mean=float(cdl[:, 0].mean()), cd_amp=float(0.5 * (cdl[:, 0].max() - cdl[:, 0].min())),
                cl_rms=rms(cdl[:, 1]), cl_mean=float(cdl[:, 1].mean()),
                cd_pressure=float(np.mean(hist[:, 0]) / (0.5 * case.rho * case.u_inf ** 2 * lref)),
                wall_s=wall, cell_steps_per_s=case.cells * steps / wall, poisson_iters_per_step=iters_p / steps)


def _main():
    from . import inputs

    ap = argparse.ArgumentParser(description="cylinder in uniform flow: drag, lift and Strouhal number")
    ap.add_argument("--nx", type=int, default=512)
    ap.add_argument("--ny", type=int, default=256)
    ap.add_argument("--box", default="-8,24,-8,8")
    ap.add_argument("--re", type=float, default=100.0)
    ap.add_argument("--cfl", type=float, default=0.5)
    ap.add_argument("--t-end", type=float, default=150.0)
    ap.add_argument("--t-avg", type=float, default=50.0)
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    args = ap.parse_args()
    box = tuple(float(v) for v in args.box.split(","))
    case = inputs.make_case(f"cylinder_re{args.re:g}_{args.nx}x{args.ny}", args.nx, args.ny, box,
                            inputs.Geometry(kind=inputs.GEOM_CIRCLE, cx=0.0, cy=0.0, r=0.5), re=args.re,
                            cfl=args.cfl, lref=1.0)
    case.precision = args.precision
    if args.precision == "mixed":
        case.precond = "chebyshev"
        case.cheb_degree = 3
    out = shedding(case, args.t_end, args.t_avg)
    out.update(workload=case.name, box=list(box), h=case.hx, dt=case.dt, precision=args.precision,
               cells_per_diameter=round(1.0 / case.hx, 3))
    print(json.dumps(out))


if __name__ == "__main__":
    _main()
