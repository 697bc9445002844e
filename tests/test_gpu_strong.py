"""GPU parity of the strong rigid-fluid coupling against the oracle from identical states
with the iteration counts forced equal: the body's force, torque and velocities after the
step (force and torque within 2e-4 of their magnitude, as for the weak coupling; the
velocity change within 2e-4 of itself), the fluid's velocities within the DFSPH velocity
bound; and on the GPU alone: the immovable-body limit equals the weak coupling, and the
coupled rigid dam break runs stably."""
import numpy as np
import pytest

import oracle
from paper_2403_11156_gb300 import scenes, sph

from gpu_util import forced, gpu_ctx

pytestmark = pytest.mark.gpu

DT = 4e-4


@pytest.mark.parametrize("lanes", [1, 4, 8])
def test_one_step_parity(lanes):
    d = forced(scenes.body_in_fluid(rigid_coupling=1, density=200.0, lanes_per_particle=lanes), 2, 3)
    g = gpu_ctx(d)
    o = oracle.Scene(d)
    b0 = np.array(d["bodies"][0]["vel"])
    g.sph_step(DT)
    g.sph_synchronize(raise_on_error=False)
    o.step(DT)
    gb, ob = g.sph_read_bodies()[0], o.bodies()[0]
    F, T = ob[13:16], ob[16:19]
    assert np.abs(F).max() > 0
    np.testing.assert_allclose(gb[13:16], F, rtol=0, atol=2e-4 * np.abs(F).max() + 1e-9)
    np.testing.assert_allclose(gb[16:19], T, rtol=0, atol=2e-4 * np.abs(T).max() + 1e-12)
    dv = ob[7:10] - b0
    np.testing.assert_allclose(gb[7:10], ob[7:10], rtol=0, atol=2e-4 * np.abs(dv).max() + 1e-9)
    np.testing.assert_allclose(gb[10:13], ob[10:13], rtol=0, atol=2e-4 * np.abs(ob[10:13]).max() + 1e-9)
    v = g.sph_read_state()[1]
    vo = o.get(oracle.V)
    dvf = vo - o.get(oracle.V_NONP)
    assert np.abs(v - vo).max() <= 1e-3 * np.abs(dvf).max() + 1e-5 * np.abs(vo).max()


def test_immovable_body_matches_weak():
    out = []
    for coupling in (0, 1):
        d = forced(scenes.body_in_fluid(rigid_coupling=coupling), 2, 3)
        b = d["bodies"][0]
        b["mass"] *= 1e12
        b["inertia"] = tuple(1e12 * i for i in b["inertia"])
        g = gpu_ctx(d)
        g.sph_step(DT)
        g.sph_synchronize(raise_on_error=False)
        out.append((g.sph_read_state()[1], g.sph_read_bodies()[0]))
    (v0, b0), (v1, b1) = out
    np.testing.assert_allclose(v1, v0, rtol=0, atol=1e-6 * np.abs(v0).max())
    np.testing.assert_allclose(b1[13:19], b0[13:19], rtol=1e-5, atol=1e-5 * np.abs(b0[13:19]).max())


def test_strongly_coupled_dam_break_runs():
    d = scenes.dam_break_rigid(seed=9, n=(30, 22, 22), tank=(0.5, 0.25, 0.35), box_edge=0.04,
                               rigid_coupling=1)
    g = gpu_ctx(d)
    z0 = g.sph_read_bodies()[:, 2].copy()
    g.sph_steps(150, 0.0)
    assert g.sph_synchronize(raise_on_error=False) in (sph.SPH_OK, sph.SPH_ENOCONVERGE)
    x, v, _, _ = g.sph_read_state()
    b = g.sph_read_bodies()
    assert np.all(np.isfinite(x)) and np.all(np.isfinite(b))
    assert np.all(b[:, 2] < z0)                        # the boxes fell
    assert np.abs(v).max() < 5.0


def test_batch_with_longer_solve_matches_single():
    # a strongly coupled scene batched beside a scene whose solves run longer: the batch's
    # extra Jacobi iterations must not push the converged scene's body again (its solver is
    # inactive there, so its pass B and its body update both skip); both scenes step
    # bit-identically to each alone
    strong = forced(scenes.body_in_fluid(rigid_coupling=1, density=200.0), 2, 3)
    other = forced(scenes.dam_break_small(seed=7, n=(9, 11, 13), box=0.4), 3, 6)
    # (forced counts may stop a solve above its tolerance: SPH_ENOCONVERGE, state advanced)
    done = (sph.SPH_OK, sph.SPH_ENOCONVERGE)
    batch = gpu_ctx([strong, other])
    batch.sph_steps(3, DT)
    assert batch.sph_synchronize(raise_on_error=False) in done
    for k, d in enumerate((strong, other)):
        single = gpu_ctx(d)
        single.sph_steps(3, DT)
        assert single.sph_synchronize(raise_on_error=False) in done
        for u, w in zip(batch.sph_read_state(k), single.sph_read_state()):
            np.testing.assert_array_equal(u, w)
        np.testing.assert_array_equal(batch.sph_read_bodies(k), single.sph_read_bodies())


def test_batch_with_warm_started_scene_matches_single():
    # a strongly coupled scene without a warm start beside a scene with the previous-step
    # warm start: the batch runs the warm-start passes, and their body update must leave
    # the first scene's body alone (its warm pass applied nothing); both scenes step
    # bit-identically to each alone
    strong = scenes.body_in_fluid(rigid_coupling=1, density=200.0, warm_start=scenes.WARM_ZERO)
    other = scenes.dam_break_small(seed=7, n=(9, 11, 13), box=0.4)
    done = (sph.SPH_OK, sph.SPH_ENOCONVERGE)
    batch = gpu_ctx([strong, other])
    batch.sph_steps(4, DT)
    assert batch.sph_synchronize(raise_on_error=False) in done
    for k, d in enumerate((strong, other)):
        single = gpu_ctx(d)
        single.sph_steps(4, DT)
        assert single.sph_synchronize(raise_on_error=False) in done
        for u, w in zip(batch.sph_read_state(k), single.sph_read_state()):
            np.testing.assert_array_equal(u, w)
        np.testing.assert_array_equal(batch.sph_read_bodies(k), single.sph_read_bodies())
