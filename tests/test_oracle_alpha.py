"""Pins of the oracle's DFSPH factor alpha (Sec. 3.4.2, Alg. ppe_solver with the cited
DFSPH stiffness kappa_i = alpha_i e_i / dt^2) against what the mathematics fixes.

alpha_i = rho_i / (|S1_i|^2 + S2_i) with S1_i = sum_j m grad W_ij + sum_b Psi_b grad W_ib
and S2_i = sum_j |m grad W_ij|^2 is the factor that makes one Jacobi update cancel a lone
particle's predicted density error exactly, so two independent checks pin it:

* closed form: on an exact lattice of spacing h/2 the interior particle has S1 = 0 by
  symmetry, and S2 is a three-shell sum worked by hand;
* the defining property, with a wall: a single compressed particle next to the floor,
  among uncompressed fluid, gets kappa_i = alpha_i (rho_i - rho0)/dt^2 from the solver;
  the update of Eq. pressure_acceleration (with the Sec. 3.5 boundary term) then changes
  its predicted density by -dt^2 kappa_i / alpha_i, which brings rho*_i to rho0 to
  rounding.  The test recomputes rho*_i from the oracle's output velocities with
  brute-force neighbours (Eq. density_source with the SPH divergence), so a wrong alpha
  (a dropped S2, Psi moved into S2 or left out of S1, m squared once too often) leaves a
  residual of the same order as the initial error;
* the same property in the divergence-free solve (Eq. velocity_source): one particle moving
  towards the floor among resting fluid gets kappa_v = alpha D rho/Dt / dt, and one update
  brings its D rho/Dt to zero to rounding.
"""
import math

import numpy as np
import pytest

from paper_2403_11156_gb300 import scenes


def _quiet(**kw):
    base = dict(max_iter_density=0, max_iter_divergence=0, warm_start=0, divergence_solve=0,
                viscosity_mode=0, gravity=(0.0, 0.0, 0.0))
    base.update(kw)
    return base


def test_alpha_closed_form_on_lattice(oracle_lib):
    # exact lattice at spacing h/2, interior particle: neighbour shells at q = 1/2 (6),
    # sqrt2/2 (12), sqrt3/2 (8); |grad W| = 48/(pi h^4) |g(q)| with g(1/2) = -1/4 and
    # g(q) = -(1-q)^2 above 1/2.  With m = rho0 (h/2)^3 and rho = rho0 S/pi,
    #   alpha = rho / (m^2 (48/(pi h^4))^2 G) = S pi h^2 / (36 rho0 G),
    #   G = 6/16 + 12 (1 - sqrt2/2)^4 + 8 (1 - sqrt3/2)^4.
    r = 2.0 ** -7                           # lattice exact in float
    h = 4 * r
    x = scenes.lattice_block((9, 9, 9), 2 * r, (0.25, 0.25, 0.25))
    d = scenes.random_cloud(1, radius=r, extent=0.6, **_quiet())
    d["fluid_x"], d["fluid_v"] = x, np.zeros_like(x)
    s = oracle_lib.Scene(d)
    s.step(1e-4)
    S = 1 + 6 * 0.25 + 12 * 2 * (1 - math.sqrt(2) / 2) ** 3 + 8 * 2 * (1 - math.sqrt(3) / 2) ** 3
    G = 6 / 16 + 12 * (1 - math.sqrt(2) / 2) ** 4 + 8 * (1 - math.sqrt(3) / 2) ** 4
    want = S * math.pi * h * h / (36 * 1000.0 * G)
    centre = 4 + 9 * (4 + 9 * 4)
    assert s.get(oracle_lib.ALPHA)[centre] == pytest.approx(want, rel=1e-12)


def _rho_star(oracle_lib, xf, v, rho, psi, xb, i, dt, h, m):
    """Eq. density_source with the SPH divergence of Sec. 3.2 and the Sec. 3.5 boundary
    term (walls at rest), for particle i; neighbours by brute force under the float
    predicate d2 < h^2."""
    h2 = np.float32(h) * np.float32(h)

    def within(Y):
        dd = (xf[i][None, :] - Y).astype(np.float32)
        d2 = (dd[:, 0] * dd[:, 0] + dd[:, 1] * dd[:, 1]) + dd[:, 2] * dd[:, 2]
        return np.nonzero(d2 < h2)[0]

    xi = xf[i].astype(np.float64)
    div, s1f, s1b = 0.0, np.zeros(3), np.zeros(3)
    for j in within(xf):
        if j == i:
            continue
        g = oracle_lib.gradW(xi - xf[j].astype(np.float64), h)
        div += m * np.dot(v[i] - v[j], g)
        s1f += m * g
    for b in within(xb):
        g = oracle_lib.gradW(xi - xb[b].astype(np.float64), h)
        div += psi[b] * np.dot(v[i], g)
        s1b += psi[b] * g
    return rho[i] + dt * div, s1f, s1b


@pytest.mark.parametrize("drop", [0.008, 0.010])
def test_alpha_cancels_a_lone_compression_next_to_a_wall(oracle_lib, drop):
    rr, dt = 0.01, 4e-4
    # stretched lattice (uncompressed everywhere) above the floor of a closed box; one
    # particle of the bottom layer is pushed towards the floor wall
    x = scenes.lattice_block((6, 6, 4), 2 * rr * 1.06, (0.05, 0.05, scenes.WALL_GAP * 2 * rr))
    x = x.astype(np.float64)
    i = 2 + 6 * 2
    x[i, 2] -= drop
    x[i, 0] += 0.0013
    x = x.astype(np.float32)
    d = scenes.dam_break_small(seed=1, n=(2, 2, 2), box=0.3,
                               **_quiet(min_iter_density=1, max_iter_density=1))
    d["fluid_x"], d["fluid_v"] = x, np.zeros_like(x)
    s = oracle_lib.Scene(d)
    s.step(dt)
    rho = s.get(oracle_lib.RHO)
    # only particle i is compressed, so only its kappa is non-zero in the one iteration
    assert list(np.nonzero(rho > 1000.0)[0]) == [i]
    assert s.stats()["dens_iters"] == 1
    e0 = rho[i] - 1000.0
    rs, s1f, s1b = _rho_star(oracle_lib, x, s.get(oracle_lib.V), rho, s.get(oracle_lib.PSI),
                             d["boundary_x"], i, dt, 4 * rr, s.mass)
    # the wall is a large part of S1 (so the pin covers the boundary reading of alpha)
    assert np.linalg.norm(s1b) > 0.3 * np.linalg.norm(s1f + s1b)
    assert abs(rs - 1000.0) <= 1e-9 * e0


def _drho_dt(oracle_lib, xf, v, psi, xb, i, h, m):
    """SPH rate of density change (continuity equation with the Sec. 3.2 divergence and the
    Sec. 3.5 boundary term, walls at rest) of particle i, brute-force neighbours."""
    h2 = np.float32(h) * np.float32(h)

    def within(Y):
        dd = (xf[i][None, :] - Y).astype(np.float32)
        d2 = (dd[:, 0] * dd[:, 0] + dd[:, 1] * dd[:, 1]) + dd[:, 2] * dd[:, 2]
        return np.nonzero(d2 < h2)[0]

    xi = xf[i].astype(np.float64)
    s = 0.0
    for j in within(xf):
        if j != i:
            s += m * np.dot(v[i] - v[j], oracle_lib.gradW(xi - xf[j].astype(np.float64), h))
    for b in within(xb):
        s += psi[b] * np.dot(v[i], oracle_lib.gradW(xi - xb[b].astype(np.float64), h))
    return s


def test_alpha_cancels_a_lone_divergence_next_to_a_wall(oracle_lib):
    # the divergence-free solve (Eq. velocity_source) uses the same factor: with one particle
    # moving towards the floor among resting fluid, kappa_v = alpha D rho/Dt / dt, and one
    # update of Eq. pressure_acceleration brings its D rho/Dt to zero to rounding
    rr, dt = 0.01, 4e-4
    x = scenes.lattice_block((6, 6, 4), 2 * rr * 1.06, (0.05, 0.05, scenes.WALL_GAP * 2 * rr))
    i = 2 + 6 * 2
    v = np.zeros_like(x)
    v[i] = (0.0, 0.0, -0.5)
    d = scenes.dam_break_small(seed=1, n=(2, 2, 2), box=0.3,
                               **_quiet(divergence_solve=1, min_iter_divergence=1, max_iter_divergence=1))
    d["fluid_x"], d["fluid_v"] = x, v
    s = oracle_lib.Scene(d)
    s.step(dt)
    psi, xb, m = s.get(oracle_lib.PSI), d["boundary_x"], s.mass
    v0 = v.astype(np.float64)
    # only particle i converges on its neighbours, so only its kappa_v is non-zero
    rates = [_drho_dt(oracle_lib, x, v0, psi, xb, k, 4 * rr, m) for k in range(len(x))]
    assert [k for k, r in enumerate(rates) if r > 0.0] == [i]
    assert s.stats()["div_iters"] == 1
    after = _drho_dt(oracle_lib, x, s.get(oracle_lib.V_DIV), psi, xb, i, 4 * rr, m)
    assert abs(after) <= 1e-9 * rates[i]
