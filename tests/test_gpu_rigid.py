"""GPU parity of the two-way rigid coupling (Sec. 3.5 Eqs. rigid_pressure and
rigid_pressure_symmetric, weak coupling) against the oracle: moving-body pseudo-masses,
the fluid's force and torque on each body, and the body's update, from one step off the
same state with forced iteration counts."""
import numpy as np
import pytest

import oracle
from paper_2403_11156_gb300 import scenes, sph

from gpu_util import assert_rel, forced, gpu_ctx

pytestmark = pytest.mark.gpu


def _scene():
    # a small rigid dam break: 30 x 22 x 22 fluid (1.1-spacing wall gaps on every side of
    # the 0.25 m cross-section), three boxes in air, r = 0.005
    return scenes.dam_break_rigid(seed=9, n=(30, 22, 22), tank=(0.5, 0.25, 0.35), box_edge=0.04)


def _submerged(lanes=1):
    """The small scene with its boxes moved into the fluid block (fluid particles inside
    a box, or within one spacing of its surface, removed) so the coupling is active."""
    d = forced(_scene(), 2, 3)
    d["lanes_per_particle"] = lanes
    bx = d["boundary_x"].copy()
    keep = np.ones(len(d["fluid_x"]), bool)
    for k, b in enumerate(d["bodies"]):
        new = np.array([0.06 + 0.09 * k, 0.125, 0.12])
        sel = d["boundary_body"] == k
        bx[sel] += (new - np.array(b["com"])).astype(np.float32)
        b["com"] = tuple(new)
        inside = np.all(np.abs(d["fluid_x"] - new) < 0.02 + 0.01, axis=1)
        keep &= ~inside
    d["boundary_x"] = bx
    d["fluid_x"] = d["fluid_x"][keep]
    d["fluid_v"] = d["fluid_v"][keep]
    return d


@pytest.mark.parametrize("lanes", [1, 2, 4, 8])
def test_body_force_and_update(lanes):
    d = _submerged(lanes)
    dt = 5e-4
    g = gpu_ctx(d)
    o = oracle.Scene(d)
    q0 = np.array([b["quat"] for b in d["bodies"]])
    g.sph_step(dt)
    g.sph_synchronize(raise_on_error=False)
    o.step(dt)
    gb, ob = g.sph_read_bodies(), o.bodies()
    assert np.abs(ob[:, 13:16]).max() > 1e-4          # the fluid pushes the boxes
    assert_rel(g.sph_read_field(sph.FIELD_PSI), o.get(oracle.PSI), 1e-5, what="psi")
    for k in range(len(gb)):
        F, T = ob[k, 13:16], ob[k, 16:19]
        np.testing.assert_allclose(gb[k, 13:16], F, rtol=0, atol=2e-4 * np.abs(F).max() + 1e-9)
        np.testing.assert_allclose(gb[k, 16:19], T, rtol=0, atol=2e-4 * np.abs(T).max() + 1e-12)
        np.testing.assert_allclose(gb[k, 0:3], ob[k, 0:3], rtol=0, atol=1e-9)
        # the rotation of one step is ~1e-5: compare the change of the quaternion
        dq = np.abs(ob[k, 3:7] - q0[k]).max()
        np.testing.assert_allclose(gb[k, 3:7], ob[k, 3:7], rtol=0, atol=1e-3 * dq + 1e-12)
        np.testing.assert_allclose(gb[k, 7:10], ob[k, 7:10], rtol=1e-4, atol=1e-7)


def test_boxes_fall_then_stay_bounded():
    # the boxes start in air: symplectic free fall until the fluid reaches them, and the
    # coupled motion afterwards stays finite and inside the tank
    d = _scene()
    g = gpu_ctx(d)
    z0 = g.sph_read_bodies()[:, 2].copy()
    dt = 5e-4
    n = 20
    g.sph_steps(n, dt)
    b = g.sph_read_bodies()
    np.testing.assert_allclose(b[:, 9], -9.81 * dt * n, rtol=1e-5)
    np.testing.assert_allclose(b[:, 2], z0 - 9.81 * dt * dt * n * (n + 1) / 2, rtol=0, atol=1e-6)
    g.sph_steps(300, 0.0)
    assert g.sph_synchronize(raise_on_error=False) in (sph.SPH_OK, sph.SPH_ENOCONVERGE)
    x, v, rho, p = g.sph_read_state()
    assert np.all(np.isfinite(x)) and np.all(np.isfinite(v))
    b = g.sph_read_bodies()
    assert np.all(np.isfinite(b))
    lo, hi = np.array(d["domain_min"]), np.array(d["domain_max"])
    assert np.all(b[:, 0:3] > lo - 1e-9) and np.all(b[:, 0:3] < hi + 1e-9)


def test_batch_with_static_scene_matches_single():
    # a scene with moving bodies makes the context re-sort every scene's boundary each step;
    # a static-walled scene batched beside it keeps its wall pseudo-masses and steps
    # bit-identically to itself alone, and so does the rigid scene
    # (both at one thread per particle: alone, the small scene would pick 8 lanes by size,
    # which changes its FP32 summation order)
    ds = [_submerged(), scenes.dam_break_small(seed=7, n=(9, 11, 13), box=0.4, lanes_per_particle=1)]
    done = (sph.SPH_OK, sph.SPH_ENOCONVERGE)     # forced counts may stop above tolerance
    batch = gpu_ctx(ds)
    batch.sph_steps(4, 4e-4)
    assert batch.sph_synchronize(raise_on_error=False) in done
    for k, d in enumerate(ds):
        single = gpu_ctx(d)
        single.sph_steps(4, 4e-4)
        assert single.sph_synchronize(raise_on_error=False) in done
        for u, w in zip(batch.sph_read_state(k), single.sph_read_state()):
            np.testing.assert_array_equal(u, w)
        np.testing.assert_array_equal(batch.sph_read_field(sph.FIELD_PSI, k), single.sph_read_field(sph.FIELD_PSI))
        np.testing.assert_array_equal(batch.sph_read_bodies(k), single.sph_read_bodies())


def test_checkpoint_resume_with_bodies_bit_exact():
    # fluid state, solver memory (sph_write_state) and rigid state (sph_write_bodies) taken
    # from a run with the boxes in the fluid resume it exactly
    d = _submerged()
    a = gpu_ctx(d)
    a.sph_steps(5, 4e-4)
    a.sph_synchronize(raise_on_error=False)
    x, v, _, _ = a.sph_read_state()
    kp, kvp = a.sph_read_field(sph.FIELD_KAPPA_PREV), a.sph_read_field(sph.FIELD_KAPPA_V_PREV)
    bodies = a.sph_read_bodies()
    assert np.abs(bodies[:, 7:13]).max() > 0            # the boxes move
    b = gpu_ctx(d)
    b.sph_write_state(0, x, v, kp, kvp)
    b.sph_write_bodies(0, bodies)
    for g in (a, b):
        g.sph_steps(3, 4e-4)
        g.sph_synchronize(raise_on_error=False)
    for u, w in zip(a.sph_read_state(), b.sph_read_state()):
        np.testing.assert_array_equal(u, w)
    np.testing.assert_array_equal(a.sph_read_bodies(), b.sph_read_bodies())
    # malformed rigid state is refused and leaves the bodies as they were
    before = b.sph_read_bodies()
    for bad in (np.zeros_like(bodies), np.where(np.arange(19) == 0, np.nan, bodies)):
        with pytest.raises(sph.SphError) as e:
            b.sph_write_bodies(0, bad)
        assert e.value.status == sph.SPH_EINVAL
    np.testing.assert_array_equal(b.sph_read_bodies(), before)
