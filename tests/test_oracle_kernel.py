"""Pins of the oracle's smoothing kernel (Sec. 3.2; h = 4r, Sec. 5).

The paper gives no kernel formula; the cubic spline is the reading.  These tests pin the
oracle to facts that hold for any correct implementation of that spline: hand-worked
values, unit normalisation, the gradient being the derivative of W, antisymmetry and
compact support.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "cubic_spline.txt")


def _golden():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        q, w = line.split()
        rows.append((float(q), float(w)))
    return rows


@pytest.mark.parametrize("h", [0.04, 1.0, 0.02])
def test_hand_worked_values(oracle_lib, h):
    sigma = 8.0 / (math.pi * h ** 3)
    for q, w in _golden():
        assert oracle_lib.W(q * h, h) == pytest.approx(w * sigma, rel=1e-14, abs=1e-300)


@pytest.mark.parametrize("h", [0.04, 0.02, 1.0])
def test_unit_integral(oracle_lib, h):
    val, _ = integrate.quad(lambda r: 4.0 * math.pi * r * r * oracle_lib.W(r, h), 0.0, h,
                            points=[0.5 * h], epsabs=1e-13, epsrel=1e-13)
    assert val == pytest.approx(1.0, abs=1e-10)


def test_gradient_is_derivative(oracle_lib):
    h = 0.04
    rng = np.random.default_rng(7)
    for _ in range(200):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        r = rng.uniform(0.01, 0.999) * h
        x = d * r
        g = oracle_lib.gradW(x, h)
        e = 1e-7 * h
        dW = (oracle_lib.W(r + e, h) - oracle_lib.W(r - e, h)) / (2 * e)
        np.testing.assert_allclose(g, dW * d, rtol=1e-6, atol=1e-9 * abs(dW) + 1e-12)


def test_gradient_antisymmetric_and_support(oracle_lib):
    h = 0.04
    rng = np.random.default_rng(3)
    for _ in range(100):
        x = rng.uniform(-h, h, size=3)
        np.testing.assert_array_equal(oracle_lib.gradW(-x, h), -oracle_lib.gradW(x, h))
    np.testing.assert_array_equal(oracle_lib.gradW(np.zeros(3), h), np.zeros(3))
    for r in [h, 1.0001 * h, 2 * h]:
        assert oracle_lib.W(r, h) == 0.0
        np.testing.assert_array_equal(oracle_lib.gradW(np.array([r, 0, 0]), h), np.zeros(3))
    # gradient points towards the origin (W decreases outwards)
    g = oracle_lib.gradW(np.array([0.3 * h, 0, 0]), h)
    assert g[0] < 0 and g[1] == 0 and g[2] == 0


def test_continuity_at_half(oracle_lib):
    h = 1.0
    a = oracle_lib.W(0.5 - 1e-12, h)
    b = oracle_lib.W(0.5 + 1e-12, h)
    assert a == pytest.approx(b, rel=1e-9)
    ga = oracle_lib.gradW(np.array([0.5 - 1e-12, 0, 0]), h)
    gb = oracle_lib.gradW(np.array([0.5 + 1e-12, 0, 0]), h)
    np.testing.assert_allclose(ga, gb, rtol=1e-9)
