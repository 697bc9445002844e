"""Pins of the oracle's PCISPH solve (an iterative PPE solver of Alg. ppe_solver, the
predictive-corrective form the paper cites): the prototype stiffness against a direct
lattice sum, its closed form, and half the DFSPH factor of the prototype particle, monotone convergence with the iteration count, the 0.1 % tolerance over a dam
break, momentum conservation of the pressure forces, and hydrostatic equilibrium (the
walls carry the fluid's weight)."""
import math

import numpy as np
import pytest

import oracle
from paper_2403_11156_gb300 import scenes


def test_prototype_factor_lattice_sum():
    r = 0.01
    d = scenes.dam_break_pcisph(n=(4, 4, 4), box=0.3, radius=r)
    o = oracle.Scene(d)
    h, s = 4 * r, 2 * r
    # sum of |grad W|^2 over the full lattice neighbourhood, from dW/dr = 48/(pi h^4) g(q)
    tot = 0.0
    for a in range(-3, 4):
        for b in range(-3, 4):
            for c in range(-3, 4):
                q = math.sqrt(a * a + b * b + c * c) * s / h
                if 0 < q <= 1.0:
                    g = q * (3 * q - 2) if q <= 0.5 else -(1 - q) ** 2
                    tot += (48.0 / (math.pi * h ** 4) * g) ** 2
    m_over_rho0 = s ** 3
    want = 1.0 / (2.0 * m_over_rho0 ** 2 * tot)
    assert o.pcisph_factor() == pytest.approx(want, rel=1e-12)
    # closed form: the shells of the lattice at q = 1/2 (6, g = -1/4), sqrt2/2 (12) and
    # sqrt3/2 (8, g = -(1 - q)^2); the six at q = 1 have g = 0 and sum grad W = 0 by symmetry
    G = 6 / 16 + 12 * (1 - math.sqrt(2) / 2) ** 4 + 8 * (1 - math.sqrt(3) / 2) ** 4
    closed = 1.0 / (2.0 * s ** 6 * (48.0 / (math.pi * h ** 4)) ** 2 * G)
    assert o.pcisph_factor() == pytest.approx(closed, rel=1e-12)


def test_prototype_factor_is_half_the_dfsph_factor_of_the_prototype(oracle_lib):
    # PCISPH's stiffness assumes every neighbour carries the same pressure correction, so its
    # update moves the prototype particle twice as far as DFSPH's exact one-particle factor:
    # p = delta (rho* - rho0)/dt^2 and kappa = alpha (rho* - rho0)/dt^2 with p = kappa rho give
    # delta = alpha rho0^2 / (2 rho) on the interior of the full lattice (alpha pinned in
    # test_oracle_alpha.py)
    r = 2.0 ** -7
    x = scenes.lattice_block((9, 9, 9), 2 * r, (0.25, 0.25, 0.25))
    d = scenes.random_cloud(1, radius=r, extent=0.6, max_iter_density=0, max_iter_divergence=0,
                            warm_start=0, divergence_solve=0, viscosity_mode=0, gravity=(0.0, 0.0, 0.0))
    d["fluid_x"], d["fluid_v"] = x, np.zeros_like(x)
    o = oracle_lib.Scene(d)
    o.step(1e-4)
    centre = 4 + 9 * (4 + 9 * 4)
    alpha, rho = o.get(oracle_lib.ALPHA)[centre], o.get(oracle_lib.RHO)[centre]
    assert o.pcisph_factor() == pytest.approx(alpha * 1000.0 ** 2 / (2.0 * rho), rel=1e-12)


def test_pcisph_converges_with_iterations():
    errs = []
    for iters in (1, 3, 10, 40):
        d = scenes.dam_break_pcisph(seed=3, n=(10, 10, 10), box=0.4, min_iter_density=iters,
                                    max_iter_density=iters, eta_density=0.0)
        s = oracle.Scene(d)
        s.step(4e-4)
        errs.append(s.stats()["dens_err"])
    assert all(a > b for a, b in zip(errs, errs[1:]))


def test_pcisph_reaches_tolerance():
    d = scenes.dam_break_pcisph(seed=2, n=(10, 10, 10), box=0.4)
    s = oracle.Scene(d)
    for _ in range(20):
        s.step(0.0)
        st = s.stats()
        assert st["dens_err"] <= 1e-3 or st["dens_iters"] == 100
        assert st["dens_iters"] >= 3 and st["div_iters"] == 0
    assert np.all(np.isfinite(s.get(oracle.X)))
    assert np.all(s.get(oracle.PRESSURE) >= 0.0)


def test_pcisph_pressure_conserves_momentum():
    r = 0.01
    rng = np.random.default_rng(5)
    x = scenes.lattice_block((8, 8, 8), 1.9 * r, (0.2, 0.2, 0.2), 2e-4, rng)
    desc = scenes.random_cloud(1, radius=r, extent=0.6, gravity=(0, 0, 0), viscosity=0.0,
                               viscosity_mode=scenes.VISC_NONE, pressure_solver=scenes.SOLVER_PCISPH,
                               warm_start=0, divergence_solve=0, min_iter_density=5,
                               max_iter_density=5)
    v0 = (0.05 * rng.normal(size=x.shape)).astype(np.float32)
    desc.update(fluid_x=x, fluid_v=v0)
    o = oracle.Scene(desc)
    o.step(4e-4)
    v = o.get(oracle.V)
    assert o.get(oracle.PRESSURE).max() > 0
    dv = v.sum(axis=0) - v0.astype(np.float64).sum(axis=0)
    assert np.abs(dv).max() <= 1e-12 * np.abs(v - v0).sum()


def test_pcisph_hydrostatic_equilibrium():
    d = scenes.resting_tank(n=(8, 8, 12), dt_max=1e-3, viscosity=0.05,
                            pressure_solver=scenes.SOLVER_PCISPH, warm_start=0, divergence_solve=0,
                            min_iter_density=3)
    s = oracle.Scene(d)
    for _ in range(300):
        s.step(0.0)
    F = np.zeros(3)
    K = 200
    for _ in range(K):
        s.step(0.0)
        F += s.get(oracle.FB_IMPULSE).sum(0) / s.stats()["dt"]
    F /= K
    weight = s.mass * len(d["fluid_x"]) * 9.81
    assert F[2] / weight == pytest.approx(1.0, abs=0.01)
    assert abs(F[0]) < 0.01 * weight and abs(F[1]) < 0.01 * weight
