"""Pins for the closed forms themselves: limits that the integrals must reach."""
import math

import numpy as np
import pytest
from scipy import special

from oracle import analytic


def test_lambda_small_T_limit():
    # T -> 0: T ~ 1 / (2 lambda^2)
    for T in (1e-4, 1e-3):
        assert analytic.lambda_of_T(T) == pytest.approx(1 / math.sqrt(2 * T), rel=2e-3)


def test_lambda_large_T_limit():
    # lambda -> 0: E1(x) ~ -gamma - ln x, and int_0^1 s ln s / sqrt(1-s^2) ds = ln 2 - 1
    lam = 1e-4
    expect = -np.euler_gamma - 2 * math.log(lam) - 2 * (math.log(2) - 1)
    assert analytic.T_of_lambda(lam) == pytest.approx(expect, rel=1e-6)
    assert analytic.T_of_lambda(analytic.lambda_of_T(4.0)) == pytest.approx(4.0, rel=1e-10)


def test_terzaghi_series_limits():
    p0, cv = 1.0, 1.0
    z = np.linspace(0, 0.9, 10)
    assert np.allclose(analytic.terzaghi_pressure(z, 1e-7, 1.0, p0, cv, terms=20000), 1.0, atol=2e-2)
    assert abs(analytic.terzaghi_pressure(np.array([1.0]), 0.1, 1.0, p0, cv)[0]) < 1e-12
    # late time: single mode decay
    t = 1.0
    first = 4 / math.pi * math.exp(-math.pi ** 2 * t / 4)
    assert analytic.terzaghi_pressure(np.array([0.0]), t, 1.0, p0, cv)[0] == pytest.approx(first, rel=1e-8)


def test_theis_scale():
    assert analytic.theis_dpstar(1e-6, 0.89e-3, 1e-15) == pytest.approx(70823.95, rel=1e-6)
    # stress-injection parameter of the paper's marginally pressurised case: T = 4
    T = analytic.stress_injection_parameter(47.830e6, 0.6, 80e6, 1e-6, 0.89e-3, 1e-15)
    assert T == pytest.approx(4.0, rel=2e-3)
