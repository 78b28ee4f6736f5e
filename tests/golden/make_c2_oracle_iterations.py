"""Writes c2_oracle_iterations.json: the FP64 oracle's PCG iteration counts and the
invariants of the first steps of the 1024x512 Re 100 cylinder workload (seeded
perturbation, tolerances 1e-10).  Calls only oracle/ and the input generator; the bench's
CPU baseline uses the iteration counts to scale its bounded oracle sample to whole steps.

    python tests/golden/make_c2_oracle_iterations.py [nsteps]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2211_10698_gb300 import inputs  # noqa: E402


def main(nsteps=8):
    case = inputs.cylinder_re100_1024x512()
    o = oracle.Oracle(case)
    pu, pv = inputs.perturbation(case)
    st = o.init_state(pu=pu, pv=pv)
    rows = []
    for n in range(nsteps):
        t0 = time.perf_counter()
        hist, _ = o.step(st, 1)
        h = hist[0]
        h["seconds"] = time.perf_counter() - t0
        h["step"] = n + 1
        rows.append(h)
        print(json.dumps(h), flush=True)
    out = dict(workload=case.name, nx=case.nx, ny=case.ny, tol_p=case.tol_p, tol_h=case.tol_h,
               seed=case.seed, perturb_sigma=case.perturb_sigma, steps=rows,
               note="oracle (oracle/ccm_oracle.c), single thread; seconds are this machine's and informative only")
    with open(os.path.join(HERE, "c2_oracle_iterations.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 8)
