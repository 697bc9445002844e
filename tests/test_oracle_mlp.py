"""Pins of the oracle's warm-start network (a learned component the paper does not have).

Forward: a special case that reduces to the GELU definition.  Backward: central finite
differences.  Adam: the closed form of the first step.  Training: a small set is fit.
"""
import math

import numpy as np
import pytest


def _rand_w(oracle_lib, rng, scale=0.3):
    return rng.normal(scale=scale, size=oracle_lib.mlp_nweights())


def test_forward_special_case(oracle_lib):
    rng = np.random.default_rng(0)
    w = _rand_w(oracle_lib, rng)
    H, F = 64, 4
    W2 = w[H * F + H: H * F + H + H * H]
    W2[:] = 0.0                                   # second layer sees only its bias
    b2 = w[H * F + H + H * H: H * F + H + H * H + H]
    W3 = w[H * F + 2 * H + H * H: H * F + 3 * H + H * H]
    b3 = w[-1]
    f = rng.normal(size=(50, 4))
    y = oracle_lib.mlp_forward(w, f)
    gelu = np.array([0.5 * b * (1.0 + math.erf(b / math.sqrt(2.0))) for b in b2])
    np.testing.assert_allclose(y, np.full(50, W3 @ gelu + b3), rtol=1e-13)


def test_gradient_finite_differences(oracle_lib):
    rng = np.random.default_rng(1)
    w = _rand_w(oracle_lib, rng)
    f = rng.normal(size=(16, 4))
    t = rng.normal(size=16)
    loss, g = oracle_lib.mlp_loss_grad(w, f, t)
    y = oracle_lib.mlp_forward(w, f)
    assert loss == pytest.approx(np.mean((y - t) ** 2), rel=1e-13)
    idx = rng.choice(len(w), size=120, replace=False)
    idx = np.concatenate([idx, [len(w) - 1, 0, 300]])
    e = 1e-6
    for k in idx:
        wp = w.copy(); wp[k] += e
        wm = w.copy(); wm[k] -= e
        fd = (oracle_lib.mlp_loss_grad(wp, f, t)[0] - oracle_lib.mlp_loss_grad(wm, f, t)[0]) / (2 * e)
        assert g[k] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_adam_first_step_closed_form(oracle_lib):
    rng = np.random.default_rng(2)
    n = 40
    w = rng.normal(size=n)
    g = rng.normal(size=n)
    m = np.zeros(n)
    v = np.zeros(n)
    w0 = w.copy()
    oracle_lib.adam_step(w, m, v, g, 1, lr=1e-3, eps=1e-8)
    # bias-corrected moments equal g and g^2 after one step
    np.testing.assert_allclose(w, w0 - 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_overfit_small_set(oracle_lib):
    rng = np.random.default_rng(3)
    f = rng.normal(size=(256, 4))
    t = np.sin(f[:, 0]) + 0.5 * f[:, 1] * f[:, 2] - 0.3 * f[:, 3]
    w = _rand_w(oracle_lib, rng, 0.2)
    m = np.zeros_like(w)
    v = np.zeros_like(w)
    l0 = oracle_lib.mlp_loss_grad(w, f, t)[0]
    for it in range(1, 1501):
        loss, g = oracle_lib.mlp_loss_grad(w, f, t)
        oracle_lib.adam_step(w, m, v, g, it, lr=3e-3)
    assert loss < 0.02 * l0
