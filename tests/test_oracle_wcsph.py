"""Pins of the oracle's WCSPH step (Sec. 3.4.1 equation of state inside Alg.
general_algorithm, Eq. pressure_acceleration): the
closed-form density and symmetry of a compressed 3 x 3 x 3 cluster with every velocity
checked against an all-pairs restatement without grid or lists, momentum conservation of
the pressure forces, the zero-pressure clamp, and a short stable dam break."""
import math

import numpy as np
import pytest

import oracle
from paper_2403_11156_gb300 import scenes


def _w(q):
    return np.where(q <= 0.5, 6 * q ** 3 - 6 * q ** 2 + 1, np.where(q <= 1.0, 2 * (1 - q) ** 3, 0.0))


def _dw(q):
    return np.where(q <= 0.5, q * (3 * q - 2), np.where(q <= 1.0, -(1 - q) ** 2, 0.0))


@pytest.mark.parametrize("gamma", [1.0, 7.0])
def test_cluster_against_all_pairs_and_closed_form(gamma):
    # a 3 x 3 x 3 cube at spacing a = 1.75 r (the centre sees all 26 others within h = 4r),
    # compressed in its middle; r and a are powers of two times small integers, so the
    # float positions are exact and the cube exactly symmetric
    r, rho0, k, dt = 2.0 ** -7, 1000.0, 3.0e4, 1e-4
    h, a = 4 * r, 1.75 * r
    g = np.arange(3) * a
    x = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3) + 0.25
    x = x.astype(np.float32)
    desc = scenes.random_cloud(1, radius=r, extent=0.6, gravity=(0, 0, 0), viscosity=0.0,
                               viscosity_mode=scenes.VISC_NONE, **scenes.wcsph_parameters(0.2, r))
    desc.update(fluid_x=x, fluid_v=np.zeros_like(x), eos_stiffness=k, eos_exponent=gamma)
    o = oracle.Scene(desc)
    o.step(dt)
    m = rho0 * (2 * r) ** 3
    sigma = 8.0 / (math.pi * h ** 3)
    # closed form of the centre's density: itself, 6 face, 12 edge and 8 corner neighbours
    s3 = [1.0, 0.4375, 0.4375 * math.sqrt(2.0), 0.4375 * math.sqrt(3.0)]
    rho_c = m * sigma * (1 + 6 * float(_w(s3[1])) + 12 * float(_w(s3[2])) + 8 * float(_w(s3[3])))
    c = 13                                  # centre of the 3 x 3 x 3 cube
    assert o.get(oracle.RHO)[c] == pytest.approx(rho_c, rel=1e-12)
    # all pairs, no grid: density, equation of state, Eq. pressure_acceleration
    X = x.astype(np.float64)
    D = X[:, None, :] - X[None, :, :]
    R = np.linalg.norm(D, axis=-1)
    rho = m * sigma * _w(R / h).sum(axis=1)
    p = np.maximum(k * ((rho / rho0) ** gamma - 1.0), 0.0)
    with np.errstate(invalid="ignore", divide="ignore"):
        gradW = (48.0 / (math.pi * h ** 4) * _dw(R / h) / R)[..., None] * D
    gradW[np.arange(27), np.arange(27)] = 0.0
    acc = -(m * (p / rho ** 2)[:, None] + m * (p / rho ** 2)[None, :])[..., None] * gradW
    v_ref = dt * acc.sum(axis=1)
    assert p.max() > 0 and np.any(p == 0)      # the corners stay below rest density
    np.testing.assert_allclose(o.get(oracle.RHO), rho, rtol=1e-12)
    np.testing.assert_allclose(o.get(oracle.PRESSURE), p, rtol=1e-10, atol=0)
    v = o.get(oracle.V)
    np.testing.assert_allclose(v, v_ref, rtol=1e-10, atol=1e-12 * np.abs(v_ref).max())
    # symmetry: the centre stays at rest, mirror particles move oppositely
    assert np.abs(v[c]).max() <= 1e-6 * np.abs(v).max()
    np.testing.assert_allclose(v[::-1], -v, rtol=0, atol=1e-9 * np.abs(v).max())
    np.testing.assert_allclose(o.get(oracle.X), X + dt * v, rtol=0, atol=1e-9)


def test_isolated_pair_is_clamped():
    # two particles are far below rest density: the clamp leaves them at rest
    r = 0.01
    x = np.array([[0.3, 0.3, 0.3], [0.32, 0.3, 0.3]], np.float32)
    desc = scenes.random_cloud(2, radius=r, extent=0.6, gravity=(0, 0, 0), viscosity=0.0,
                               viscosity_mode=scenes.VISC_NONE, **scenes.wcsph_parameters(0.2, r))
    desc.update(fluid_x=x, fluid_v=np.zeros_like(x))
    o = oracle.Scene(desc)
    o.step(1e-4)
    assert np.all(o.get(oracle.PRESSURE) == 0.0) and np.all(o.get(oracle.V) == 0.0)


def test_pressure_forces_conserve_momentum():
    r = 0.01
    rng = np.random.default_rng(4)
    x = scenes.lattice_block((8, 8, 8), 1.8 * r, (0.2, 0.2, 0.2), 2e-4, rng)   # compressed
    desc = scenes.random_cloud(1, radius=r, extent=0.6, gravity=(0, 0, 0), viscosity=0.0,
                               viscosity_mode=scenes.VISC_NONE, **scenes.wcsph_parameters(0.2, r))
    v0 = (0.05 * rng.normal(size=x.shape)).astype(np.float32)
    desc.update(fluid_x=x, fluid_v=v0)
    o = oracle.Scene(desc)
    o.step(2e-4)
    p = o.get(oracle.PRESSURE)
    v = o.get(oracle.V)
    assert p.max() > 0
    # all particles have the same mass: total momentum is the sum of velocities
    dv = v.sum(axis=0) - v0.astype(np.float64).sum(axis=0)
    assert np.abs(dv).max() <= 1e-12 * np.abs(v - v0).sum()
    # the compressed block expands: velocity changes point away from the centre
    c = x.mean(axis=0)
    assert np.sum((x - c) * (v - v0)) > 0


def test_expanded_lattice_has_no_pressure():
    r = 0.01
    x = scenes.lattice_block((6, 6, 6), 2.2 * r, (0.2, 0.2, 0.2))
    desc = scenes.random_cloud(1, radius=r, extent=0.6, gravity=(0, 0, 0), viscosity=0.0,
                               viscosity_mode=scenes.VISC_NONE, **scenes.wcsph_parameters(0.2, r))
    v0 = np.full(x.shape, 0.1, np.float32)
    desc.update(fluid_x=x, fluid_v=v0)
    o = oracle.Scene(desc)
    o.step(1e-4)
    assert np.all(o.get(oracle.PRESSURE) == 0.0)
    np.testing.assert_allclose(o.get(oracle.V), v0.astype(np.float64), rtol=0, atol=0)
    st = o.stats()
    assert st["dens_iters"] == 0 and st["div_iters"] == 0


def test_dam_break_steps_stay_bounded():
    d = scenes.dam_break_wcsph(n=(8, 8, 8), box=0.3)
    o = oracle.Scene(d)
    for _ in range(20):
        o.step(0.0)
    x, v, rho = o.get(oracle.X), o.get(oracle.V), o.get(oracle.RHO)
    assert np.all(np.isfinite(x)) and np.all(np.isfinite(v))
    assert np.abs(v).max() < 2.0
    assert rho.max() < 1.05 * d["rest_density"]           # weakly compressible: ~1 %
