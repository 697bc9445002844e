"""Pins of the oracle's implicit viscosity (Sec. 3.6.2): the operator is symmetric, has
translations and rotations in its null space, I - dt A is positive definite, the CG
solve reaches its tolerance, and for a small step the implicit update agrees with the
explicit Laplacian of Sec. 3.6.1 Eq. lap (which Sec. 3.6.2 discretises)."""
import numpy as np
import pytest

from paper_2403_11156_gb300 import scenes


def _scene(oracle_lib, nu=0.1):
    d = scenes.dam_break_small(seed=8, n=(8, 8, 8), box=0.3, viscosity=nu, viscosity_mode=3,
                               max_iter_density=0, max_iter_divergence=0, warm_start=0,
                               divergence_solve=0, gravity=(0.0, 0.0, 0.0))
    s = oracle_lib.Scene(d)
    s.prepare()
    return d, s


def test_operator_symmetric_and_definite(oracle_lib):
    d, s = _scene(oracle_lib)
    rng = np.random.default_rng(0)
    n = len(d["fluid_x"])
    dt = 1e-3
    for _ in range(3):
        u = rng.normal(size=(n, 3))
        v = rng.normal(size=(n, 3))
        Mu = s.visc_operator(dt, u)
        Mv = s.visc_operator(dt, v)
        a, b = np.sum(u * Mv), np.sum(v * Mu)
        assert a == pytest.approx(b, rel=1e-12)
        assert np.sum(u * Mu) > np.sum(u * u)      # I - dt A with A negative semidefinite
        assert np.sum(u * Mu) - np.sum(u * u) > 1e-6 * np.sum(u * u)


def test_operator_null_space(oracle_lib):
    d, s = _scene(oracle_lib)
    x = d["fluid_x"].astype(np.float64)
    for v in (np.tile([1.0, -2.0, 0.5], (len(x), 1)), np.cross([0.3, 1.0, -0.7], x - 0.15)):
        Mv = s.visc_operator(1e-2, v)
        np.testing.assert_allclose(Mv, v, rtol=0, atol=1e-12 * np.abs(v).max())


def test_cg_solves(oracle_lib):
    d, s = _scene(oracle_lib, nu=0.1)
    rng = np.random.default_rng(1)
    b = rng.normal(size=(len(d["fluid_x"]), 3))
    x, it = s.visc_solve(1e-3, b)
    r = s.visc_operator(1e-3, x) - b
    assert it > 1
    assert np.linalg.norm(r) <= 1e-4 * np.linalg.norm(b) * 1.0001


def test_small_step_matches_explicit(oracle_lib):
    # (I - dt A)^-1 v = v + dt A v + O(dt^2), and dt A v is the explicit step of Eq. lap
    nu = 0.1
    dt = 1e-8
    rng = np.random.default_rng(2)
    d = scenes.dam_break_small(seed=8, n=(8, 8, 8), box=0.3, viscosity=nu,
                               max_iter_density=0, max_iter_divergence=0, warm_start=0,
                               divergence_solve=0, gravity=(0.0, 0.0, 0.0), cg_tol=1e-12)
    d["fluid_v"] = rng.normal(size=d["fluid_x"].shape).astype(np.float32)
    out = {}
    for mode in (1, 3):
        dd = dict(d)
        dd["viscosity_mode"] = mode
        s = oracle_lib.Scene(dd)
        s.step(dt)
        out[mode] = s.get(oracle_lib.V_NONP) - d["fluid_v"].astype(np.float64)
    assert np.abs(out[1]).max() > 0
    np.testing.assert_allclose(out[3], out[1], rtol=0, atol=1e-4 * np.abs(out[1]).max())
