"""Writes c2_trajectory.json: samples of the FP64 oracle's trajectory of the 1024x512 Re 100
cylinder (seeded N(0, 1e-3) perturbation, Jacobi-PCG) over its first 20 steps, with both CG
tolerances tightened to 1e-13, for the GPU's trajectory parity test.

Calls only the oracle (and the seeded inputs).  The file records a hash of the case manifest;
the test refuses a file whose hash no longer matches the inputs.  Norms and sums are taken over
the velocity unknowns and the active cells.

    python tests/golden/make_c2_trajectory.py
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2211_10698_gb300 import inputs  # noqa: E402

STEPS = 20
CHECKPOINTS = (10, 20)
SAMPLES = 512
TOL = 1e-13


def trajectory_case():
    case = inputs.cylinder_re100_1024x512()
    case.tol_p = case.tol_h = TOL
    return case


def manifest(case) -> dict:
    """Everything that defines the trajectory: the case description and the step count."""
    g = case.geom
    return dict(nx=case.nx, ny=case.ny, box=[case.x0, case.x1, case.y0, case.y1], rho=case.rho, mu=case.mu,
                dt=case.dt, bc_type=list(case.bc_type), bc_un=list(case.bc_un), bc_ut=list(case.bc_ut),
                geom=dict(kind=g.kind, cx=g.cx, cy=g.cy, r=g.r), tol_p=case.tol_p, tol_h=case.tol_h,
                perturb_sigma=case.perturb_sigma, seed=case.seed, pressure_update=case.pressure_update,
                literal_offdiag=case.literal_offdiag, steps=STEPS)


def manifest_hash(case) -> str:
    return hashlib.sha256(json.dumps(manifest(case), sort_keys=True).encode()).hexdigest()[:16]


def sample_positions(o, seed=7):
    """Seeded positions (padded row, column) of velocity unknowns and active cells."""
    rng = np.random.default_rng(seed)
    out = {}
    for name, mask in (("u", o.role_u == 3), ("v", o.role_v == 3), ("p", o.active)):
        idx = np.argwhere(mask)
        pick = idx[rng.choice(len(idx), size=SAMPLES, replace=False)]
        out[name] = pick.tolist()
    return out


def main():
    oracle.set_threads(0)
    case = trajectory_case()
    o = oracle.Oracle(case)
    pu, pv = inputs.perturbation(case)
    st = o.init_state(pu, pv)
    pos = sample_positions(o)
    rec = dict(manifest=manifest(case), manifest_hash=manifest_hash(case), samples=SAMPLES, positions=pos,
               checkpoints={}, iters_p=[], iters_h=[])
    t0 = time.time()
    for n in range(1, STEPS + 1):
        hist, _ = o.step(st, 1)
        rec["iters_p"].append(hist[0]["iters_p"])
        rec["iters_h"].append(hist[0]["iters_h"])
        if n in CHECKPOINTS:
            cp = {}
            for name, mask in (("u", o.role_u == 3), ("v", o.role_v == 3), ("p", o.active)):
                a = st[name]
                # norms over the unknowns only: ghost and corner slots carry no solution
                cp[name] = dict(values=[float(a[j, i]) for j, i in pos[name]],
                                l2=float(np.linalg.norm(a[mask])), sum=float(a[mask].sum()))
            cp["kinetic"] = hist[0]["kinetic"]
            rec["checkpoints"][str(n)] = cp
        print(f"step {n}: {hist[0]['iters_p']} Poisson iterations, {time.time() - t0:.0f} s", flush=True)
    with open(os.path.join(HERE, "c2_trajectory.json"), "w") as f:
        json.dump(rec, f, indent=0)


if __name__ == "__main__":
    main()
