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


def test_learned_fraction_scales_kappa0():
    """The learned warm start applies a fraction of the network's stiffness: kappa0 at a
    fraction f is f times kappa0 at f = 1, the default fraction is 0.6, and at f = 1 kappa0
    is the network's de-standardised output (9.81 h units) on the gated particles."""
    import oracle
    from paper_2403_11156_gb300 import scenes
    rng = np.random.default_rng(7)
    nw = oracle.mlp_nweights()
    p = np.zeros(oracle.mlp_nparam())
    p[:nw] = rng.normal(scale=0.3, size=nw)
    p[nw:nw + 4] = (0.0, 0.0, 1.0, 1.0)          # feature means
    p[nw + 4:nw + 8] = (1e-3, 1e-3, 0.1, 1.0)    # feature stds
    p[nw + 8], p[nw + 9] = 1.0, 0.5               # label mean, std (kappa0 mostly > 0)
    base = oracle.Scene(scenes.dam_break_small(n=(8, 8, 8)))
    for _ in range(3):
        base.step(4e-4)
    x, v = base.get(oracle.X), base.get(oracle.V)
    k0 = {}
    for f in (1.0, 0.3, 0.0):
        d = scenes.dam_break_small(n=(8, 8, 8), warm_start=scenes.WARM_LEARNED, learned_fraction=f)
        o = oracle.Scene(d)
        o.set_mlp(p)
        o.set_state(x, v)                          # the same state for every fraction
        o.step(4e-4)
        k0[f] = o.get(oracle.KAPPA0)
        if f == 1.0:
            feat = o.get(oracle.FEAT)
            h = 4.0 * d["radius"]
    on = k0[1.0] > 0
    assert on.sum() >= 10
    np.testing.assert_allclose(k0[0.3], 0.3 * k0[1.0], rtol=1e-12, atol=0)
    np.testing.assert_allclose(k0[0.0], 0.6 * k0[1.0], rtol=1e-12, atol=0)
    y = oracle.mlp_forward(p, (feat - p[nw:nw + 4]) / p[nw + 4:nw + 8])
    want = (y * p[nw + 9] + p[nw + 8]) * 9.81 * h
    np.testing.assert_allclose(k0[1.0][on], want[on], rtol=1e-12)
