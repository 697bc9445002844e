"""Pins of the oracle's rigid-body integration and two-way coupling (Sec. 3.5; weak
coupling as in Sec. 2.2/6): symplectic-Euler free fall in closed form, the exact per-step
rotation angle of the normalised first-order quaternion update, conservation of the
total fluid + body momentum under the symmetric pressure forces of Eq.
rigid_pressure_symmetric, and the depth-independent buoyancy of a submerged body (Archimedes)."""
import math

import numpy as np
import pytest

from paper_2403_11156_gb300 import scenes


def _body_scene(fluid_x, center=(0.5, 0.5, 0.5), omega=(0.0, 0.0, 0.0), gravity=(0, 0, -9.81),
                **kw):
    pts, body = scenes.cube_body(center, 0.1, 0.02, 500.0)
    body["omega"] = omega
    p = scenes.params(radius=0.01, domain_min=(0, 0, 0), domain_max=(1, 1, 1),
                      gravity=gravity, **kw)
    d = dict(p)
    d["fluid_x"] = np.asarray(fluid_x, np.float32).reshape(-1, 3)
    d["fluid_v"] = np.zeros_like(d["fluid_x"])
    d["boundary_x"] = pts
    d["boundary_body"] = np.zeros(len(pts), np.int32)
    d["bodies"] = [body]
    return d


def test_free_fall_closed_form(oracle_lib):
    d = _body_scene([[0.05, 0.05, 0.05]], center=(0.5, 0.5, 0.8))
    s = oracle_lib.Scene(d)
    dt = 1e-3
    for n in range(1, 51):
        s.step(dt)
        com = s.bodies()[0, 0:3]
        vel = s.bodies()[0, 7:10]
        assert vel[2] == pytest.approx(-9.81 * dt * n, rel=1e-12)
        assert com[2] == pytest.approx(0.8 - 9.81 * dt * dt * n * (n + 1) / 2, rel=1e-12)


def test_torque_free_spin_angle(oracle_lib):
    w = np.array([0.0, 0.0, 3.0])
    d = _body_scene([[0.05, 0.05, 0.05]], omega=tuple(w), gravity=(0, 0, 0))
    s = oracle_lib.Scene(d)
    dt = 1e-2
    n = 40
    for _ in range(n):
        s.step(dt)
    q = s.bodies()[0, 3:7]
    np.testing.assert_allclose(s.bodies()[0, 10:13], w, rtol=1e-12)
    # each step multiplies q by (1, dt w/2) and renormalises: a rotation by 2 atan(|w| dt/2)
    angle = n * 2.0 * math.atan(3.0 * dt / 2.0)
    np.testing.assert_allclose(q, [math.cos(angle / 2), 0, 0, math.sin(angle / 2)], atol=1e-12)


def test_fluid_body_momentum_conserved(oracle_lib):
    # fluid packed tightly around a free cube, no gravity, no walls: the pressure pushes
    # both, and the total momentum of fluid plus body stays zero
    rng = np.random.default_rng(0)
    x = scenes.lattice_block((12, 12, 12), 0.018, (0.39, 0.39, 0.39), 2e-4, rng)
    c = np.array([0.5, 0.5, 0.5])
    keep = np.max(np.abs(x - c), axis=1) > 0.062
    d = _body_scene(x[keep], center=tuple(c + [0.01, 0.0, -0.005]), gravity=(0, 0, 0),
                    viscosity_mode=0)
    s = oracle_lib.Scene(d)
    M = d["bodies"][0]["mass"]
    for _ in range(3):
        s.step(2e-4)
        pf = s.mass * s.get(oracle_lib.V).sum(0)
        pb = M * s.bodies()[0, 7:10]
        assert np.abs(pb).max() > 1e-6
        np.testing.assert_allclose(pf + pb, 0.0, atol=1e-10 * np.abs(pb).max())


def test_resume_from_state_and_bodies(oracle_lib):
    # a scene given another run's fluid state and rigid state continues exactly as that run
    # does: the setters copy state and place the body's boundary particles at its pose
    d = scenes.body_in_fluid(gravity=(0.0, 0.0, -9.81), warm_start=scenes.WARM_ZERO)
    dt = 4e-4
    a = oracle_lib.Scene(d)
    for _ in range(3):
        a.step(dt)
    assert np.abs(a.bodies()[0, 7:13]).max() > 0          # the body moves
    b = oracle_lib.Scene(d)
    b.set_state(a.get(oracle_lib.X), a.get(oracle_lib.V))
    b.set_bodies(a.bodies())
    np.testing.assert_array_equal(b.get(oracle_lib.XB), a.get(oracle_lib.XB))
    a.step(dt)
    b.step(dt)
    np.testing.assert_array_equal(b.get(oracle_lib.X), a.get(oracle_lib.X))
    np.testing.assert_array_equal(b.get(oracle_lib.V), a.get(oracle_lib.V))
    np.testing.assert_array_equal(b.bodies(), a.bodies())


def _held_box_in_tank(oracle_lib, centre_layers, steps=300, avg=100):
    """Mean fluid force on a 0.12 m surface-sampled box (6 spacings, 218 particles) held
    at rest with its centre `centre_layers` spacings above the first fluid layer of a
    16 x 16 x 18 resting block; the fluid overlapping the box is left out.  The body is
    put back to its pose with zero velocity before every step (a held body; gravity on
    the body does not enter the fluid's force)."""
    r = 0.01
    s = 2 * r
    g = scenes.WALL_GAP * s
    tank = (15 * s + 2 * g, 15 * s + 2 * g, 27 * s)
    fx = scenes.lattice_block((16, 16, 18), s, (g, g, g))
    walls = scenes.tank_walls(tank, s)
    L = 6 * s
    c = (0.5 * tank[0], 0.5 * tank[1], g + centre_layers * s)
    pts, body = scenes.cube_body(c, L, s, 500.0)
    keep = np.any(np.abs(fx - np.array(c)) > 0.5 * L + scenes.WALL_GAP * s, axis=1)
    d = dict(scenes.params(radius=r, domain_min=(0, 0, 0), domain_max=tank, viscosity=0.05,
                           dt_max=1e-3))
    d["fluid_x"] = np.ascontiguousarray(fx[keep])
    d["fluid_v"] = np.zeros_like(d["fluid_x"])
    d["boundary_x"] = np.concatenate([walls, pts]).astype(np.float32)
    d["boundary_body"] = np.concatenate([np.full(len(walls), -1, np.int32),
                                         np.zeros(len(pts), np.int32)])
    d["bodies"] = [body]
    o = oracle_lib.Scene(d)
    b0 = o.bodies().copy()
    F = np.zeros(3)
    for k in range(steps + avg):
        o.set_bodies(b0)
        o.step(0.0)
        if k >= steps:
            F += o.bodies()[0][13:16]
    return F / avg, L, r, o.get(oracle_lib.X)[:, 2].max() - (c[2] + 0.5 * L)


def test_submerged_box_buoyancy(oracle_lib):
    # Archimedes (Sec. 3.5 coupling, Eq. rigid_pressure_symmetric summed over the body):
    # a fully submerged body feels rho0 g V_eff upward whatever its depth.  The box's
    # one-layer particle surface keeps the fluid about one spacing away, so V_eff lies
    # between the particle-surface volume L^3 and that volume grown by r on every side.
    F1, L, r, top1 = _held_box_in_tank(oracle_lib, 7.0)
    F2, _, _, top2 = _held_box_in_tank(oracle_lib, 9.0)
    assert top1 > 4 * r and top2 > 4 * r            # fluid above the box: submerged
    for F in (F1, F2):
        assert abs(F[0]) < 0.02 * F[2] and abs(F[1]) < 0.02 * F[2]
        v_eff = F[2] / (1000.0 * 9.81)
        assert L ** 3 < v_eff < (L + 2 * r) ** 3
    assert F2[2] == pytest.approx(F1[2], rel=0.05)    # independent of depth
