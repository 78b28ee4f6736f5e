"""Host-side post-processing of the force record (CPU): coefficients and the Strouhal number
from the lift's upward mean crossings, checked on signals with a known frequency."""
import math

import numpy as np
import pytest

from paper_2211_10698_gb300 import forces


@pytest.mark.parametrize("f0,phase", [(0.167, 0.3), (0.36, 2.1), (0.0891, -1.0)])
def test_strouhal_of_a_sampled_periodic_signal(f0, phase):
    """A lift record of a known frequency (with a second harmonic, a slow drift-free offset and
    a little noise) gives St = f L / U to a small fraction of the sampling step."""
    dt = 1.0 / 128
    t = np.arange(0, 60.0, dt)
    rng = np.random.default_rng(5)
    lift = 0.6 * np.sin(2 * math.pi * f0 * t + phase) + 0.15 * np.sin(4 * math.pi * f0 * t + 0.4) + 0.05
    lift += 1e-4 * rng.standard_normal(t.size)
    st, periods = forces.strouhal(lift, dt, lref=2.0, u_inf=1.5)
    assert periods >= int(60 * f0) - 1
    assert st == pytest.approx(f0 * 2.0 / 1.5, rel=2e-4)


def test_mean_crossings_interpolate_between_samples():
    """Three whole periods sampled uniformly have mean zero, so the crossings are the sine's
    own, 0.033 + 4 k; linear interpolation across a zero of a sine is accurate to third order
    in the step."""
    dt = 0.1
    t = np.arange(0, 12, dt)
    x = np.sin(2 * math.pi * 0.25 * (t - 0.033))
    c = forces.mean_up_crossings(x, dt)
    assert len(c) == 3
    assert np.abs(c - (0.033 + 4 * np.arange(3))).max() < 1e-4


def test_strouhal_needs_a_period():
    with pytest.raises(ValueError):
        forces.strouhal(np.linspace(0, 1, 50), 0.1, 1.0, 1.0)


def test_coefficients_and_rms():
    f = np.array([[1.0, 0.2, 0.5, -0.1], [2.0, -0.4, 0.1, 0.0]])
    c = forces.coefficients(f, rho=2.0, u_inf=0.5, lref=4.0)
    q = 0.5 * 2.0 * 0.25 * 4.0
    assert np.allclose(c, [[1.5 / q, 0.1 / q], [2.1 / q, -0.4 / q]], rtol=1e-15)
    assert forces.rms([1.0, -1.0, 1.0, -1.0]) == pytest.approx(1.0)
    assert forces.rms(np.sin(np.linspace(0, 2 * math.pi, 100001))) == pytest.approx(1 / math.sqrt(2), rel=1e-4)


def test_step_filter_removes_the_alternating_mode_and_keeps_trends():
    """(1, 2, 1) / 4 annihilates (-1)^k (a + b k) exactly and reproduces a + b k exactly."""
    k = np.arange(40, dtype=np.float64)
    trend = 0.7 + 0.01 * k
    alt = (-1.0) ** k * (13.0 + 0.02 * k)
    rows = np.stack([trend + alt, -trend, alt, trend], axis=1)
    f = forces.step_filter(rows)
    assert f.shape == (38, 4)
    assert np.allclose(f[:, 0], trend[1:-1], rtol=0, atol=1e-13)
    assert np.allclose(f[:, 1], -trend[1:-1], rtol=0, atol=1e-15)
    assert np.abs(f[:, 2]).max() < 1e-13
    with pytest.raises(ValueError):
        forces.step_filter(rows[:2])
