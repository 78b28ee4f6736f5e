"""The projected initial guess of the Poisson solve (guess.cu): each step starts its PCG from the
K-orthogonal projection of the new solution onto the span of the previous solutions instead of
the previous Phi.  The stopping test is the same, so the fields agree with the oracle (which
starts from the previous Phi) to the solver tolerance, and a smoothly evolving flow needs fewer
iterations."""
import copy

import numpy as np
import pytest

from paper_2211_10698_gb300 import ccm, inputs as I

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("mixed", 1e-8)])
def test_projected_guess_steps_match_oracle(orc, precision, tol):
    case = I.cylinder_re40_128x64()
    case.tol_p = 1e-12 if precision == "mixed" else 1e-13
    case.tol_h = 1e-13
    case.precision = precision
    case.guess_history = 6  # restarts twice over the 20 steps
    g = ccm.Case(case)
    st = g.step(20)
    assert st["converged"]
    ocase = copy.deepcopy(case)
    ocase.tol_p = ocase.tol_h = 1e-13
    o = orc.Oracle(ocase)
    s = o.init_state()
    o.step(s, 20)
    for f, key in ((ccm.CCM_F_U, "u"), (ccm.CCM_F_V, "v"), (ccm.CCM_F_P, "p")):
        e = _rel(g.get_field(f), s[key])
        assert e < tol, (key, e)
    g.close()


def test_projected_guess_lowers_iterations():
    """The 128x64 Re 40 cylinder from rest: over steps 21-60 the projection onto the last 16
    solutions needs fewer Poisson iterations than the previous Phi, at the same tolerance."""
    its = {}
    for L in (0, 16):
        case = I.cylinder_re40_128x64()
        case.guess_history = L
        g = ccm.Case(case)
        g.step(20)
        st = g.step(40)
        assert st["converged"]
        its[L] = st["iters_p"] / 40
        g.close()
    assert its[16] < 0.9 * its[0], its


def test_history_is_cleared_by_a_new_state():
    """Restoring a state starts a new history: the restored run matches a fresh run from the
    same state bit for bit."""
    case = I.cylinder_re40_128x64()
    case.guess_history = 8
    case.autotune = 0
    g = ccm.Case(case)
    g.step(5)
    snap = {f: g.get_field(f).copy() for f in (ccm.CCM_F_U, ccm.CCM_F_V, ccm.CCM_F_P, ccm.CCM_F_PHI,
                                               ccm.CCM_F_CONV_U, ccm.CCM_F_CONV_V, ccm.CCM_F_STEP)}
    g.step(3)
    for f, a in snap.items():
        g.set_field(f, a)
    g.step(4)
    h = ccm.Case(case)
    for f, a in snap.items():
        h.set_field(f, a)
    h.step(4)
    for f in (ccm.CCM_F_U, ccm.CCM_F_V, ccm.CCM_F_P):
        assert np.array_equal(g.get_field(f), h.get_field(f)), f
    g.close()
    h.close()


def test_history_survives_a_velocity_and_pressure_upload():
    """Uploading U, V and P (the end-to-end loop's host round trip) keeps the history: the
    steps continue with the same iteration counts and fields as without the round trip."""
    case = I.cylinder_re40_128x64()
    case.guess_history = 8
    case.autotune = 0
    a, b = ccm.Case(case), ccm.Case(case)
    a.step(6)
    b.step(6)
    ia, ib = [], []
    for _ in range(4):
        for f in (ccm.CCM_F_U, ccm.CCM_F_V, ccm.CCM_F_P):
            b.set_field(f, b.get_field(f))
        ia.append(a.step(1)["iters_p"])
        ib.append(b.step(1)["iters_p"])
    assert ia == ib
    for f in (ccm.CCM_F_U, ccm.CCM_F_V, ccm.CCM_F_P, ccm.CCM_F_PHI):
        assert np.array_equal(a.get_field(f), b.get_field(f)), f
    a.close()
    b.close()
