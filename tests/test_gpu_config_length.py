"""Parity with the FP64 oracle over each configuration's own length (one PmII step, Sec. 4.6,
Eqs. pm_prediction to pm_update, repeated).

Two correct CG solves stop at different iterates (relative residual <= tol), and the shedding
cylinder amplifies such differences over thousands of steps, so long runs are compared in two
ways:
* per step from shared states: the GPU runs the configuration for its full step count; at
  several steps its whole state (U, V, P, Phi, conv^{n-1}) is loaded into the oracle, and one
  more step is taken on both sides from that state;
* a 20-step trajectory of the 1024x512 cylinder with both CG tolerances tightened to 1e-13,
  against samples of the oracle's trajectory in tests/golden/c2_trajectory.json (written by
  tests/golden/make_c2_trajectory.py, which calls only the oracle).
Tolerances (relative L2 on U, V and P): 1e-9 for the FP64 path, 1e-8 for the mixed path
refined to a 1e-10 Poisson residual."""
import copy
import json
import os

import numpy as np
import pytest

from paper_2211_10698_gb300 import ccm, inputs as I

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
FIELDS = (("u", ccm.CCM_F_U), ("v", ccm.CCM_F_V), ("p", ccm.CCM_F_P))


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _perturbed(case):
    g = ccm.Case(case)
    pu, pv = I.perturbation(case)
    g.set_field(ccm.CCM_F_U, g.get_field(ccm.CCM_F_U) + pu)
    g.set_field(ccm.CCM_F_V, g.get_field(ccm.CCM_F_V) + pv)
    return g


def _state(g):
    """The GPU state as the oracle's state dictionary (the same padded layout)."""
    get = g.get_field
    return dict(u=get(ccm.CCM_F_U).copy(), v=get(ccm.CCM_F_V).copy(), p=get(ccm.CCM_F_P).copy(),
                phi=get(ccm.CCM_F_PHI).copy(), cu=get(ccm.CCM_F_CONV_U).copy(), cv=get(ccm.CCM_F_CONV_V).copy(),
                n=int(get(ccm.CCM_F_STEP)[0, 0]))


def _gpu_step_from(case, st):
    g = ccm.Case(case)
    for key, f in (("u", ccm.CCM_F_U), ("v", ccm.CCM_F_V), ("p", ccm.CCM_F_P), ("phi", ccm.CCM_F_PHI),
                   ("cu", ccm.CCM_F_CONV_U), ("cv", ccm.CCM_F_CONV_V)):
        g.set_field(f, st[key])
    g.set_field(ccm.CCM_F_STEP, np.full(case.shape, float(st["n"])))
    stats = g.step(1)
    out = {name: g.get_field(f).copy() for name, f in FIELDS}
    g.close()
    return out, stats


def _oracle_step_from(orc, case, st):
    import oracle

    oracle.set_threads(0)
    o = orc.Oracle(case)
    s = {k: (np.array(v, order="C") if isinstance(v, np.ndarray) else v) for k, v in st.items()}
    hist, _ = o.step(s, 1)
    return {name: s[name] for name, _ in FIELDS}, hist[0]


def test_c2_per_step_parity_over_2000_steps(orc):
    """1024x512 Re 100 shedding cylinder, FP64 Jacobi: states at steps 500, 1000 and 2000 of the
    GPU run (1e-10 tolerances as configured); the step from each with both CG tolerances at
    1e-13 on both sides agrees to 1e-9."""
    case = I.cylinder_re100_1024x512()
    tight = copy.deepcopy(case)
    tight.tol_p = tight.tol_h = 1e-13
    g = _perturbed(case)
    done = 0
    for k in (500, 1000, 2000):
        st = g.step(k - done)
        assert st["converged"]
        done = k
        state = _state(g)
        got, _ = _gpu_step_from(tight, state)
        want, oh = _oracle_step_from(orc, tight, state)
        assert oh["ok"]
        for name, _ in FIELDS:
            e = _rel(got[name], want[name])
            assert e < 1e-9, (k, name, e)
    g.close()


def test_c3_mixed_step_parity_after_1000_steps(orc):
    """2048x1024 NACA0012 at 4 degrees, Re 1000, mixed precision with Chebyshev degree 3 as
    configured: the state after the GPU's 1000 steps; one more mixed step (FP32 inner CG, FP64
    residual to 1e-10) against one FP64 oracle step at 1e-13 agrees to 1e-8."""
    case = I.naca0012_re1000_2048x1024()
    g = ccm.Case(case)
    st = g.step(case.steps)
    assert st["converged"]
    state = _state(g)
    g.close()
    assert state["n"] == case.steps
    got, stats = _gpu_step_from(case, state)
    assert stats["converged"] and stats["last_res_p"] <= case.tol_p
    ocase = copy.deepcopy(case)
    ocase.tol_p = ocase.tol_h = 1e-13
    want, oh = _oracle_step_from(orc, ocase, state)
    assert oh["ok"]
    for name, _ in FIELDS:
        e = _rel(got[name], want[name])
        assert e < 1e-8, (name, e)


def test_c2_trajectory_matches_cached_oracle(orc):
    """The first 20 steps of the 1024x512 cylinder with both CG tolerances at 1e-13: the GPU's
    u, v and P at steps 10 and 20 agree with the oracle's samples to 1e-9 (relative L2 over the
    samples) and their norms over the unknowns to 1e-9."""
    import importlib.util

    path = os.path.join(HERE, "golden", "c2_trajectory.json")
    spec = importlib.util.spec_from_file_location("make_c2", os.path.join(HERE, "golden", "make_c2_trajectory.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    with open(path) as f:
        ref = json.load(f)
    case = mk.trajectory_case()
    assert ref["manifest_hash"] == mk.manifest_hash(case), "stale golden file: rerun make_c2_trajectory.py"
    o = orc.Oracle(case)  # the roles of the positions (unknowns, active cells)
    masks = dict(u=o.role_u == 3, v=o.role_v == 3, p=o.active)
    g = _perturbed(case)
    done = 0
    for k in sorted(int(x) for x in ref["checkpoints"]):
        st = g.step(k - done)
        assert st["converged"]
        done = k
        cp = ref["checkpoints"][str(k)]
        for name, f in FIELDS:
            a = g.get_field(f)
            pos = ref["positions"][name]
            got = np.array([a[j, i] for j, i in pos])
            want = np.array(cp[name]["values"])
            assert _rel(got, want) < 1e-9, (k, name, _rel(got, want))
            assert abs(np.linalg.norm(a[masks[name]]) - cp[name]["l2"]) <= 1e-9 * cp[name]["l2"], (k, name)
    g.close()
