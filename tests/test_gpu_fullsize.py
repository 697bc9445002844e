"""Full-size checks in the benchmark's configuration (1,200,500 fluid particles, rigid
boxes, CUDA-graph steps): grid keys and sort order bit-exact against the oracle's
contracts, neighbour counts bit-exact on a sample against brute force over all
particles, density / alpha / Psi of every particle against the oracle (prepared on the
full scene), one solver step's fields of every particle against the oracle (counts forced
equal, the tolerances of the small-scene parity tests), the learned warm start's kappa0 of
every particle against the oracle's FP64 network, and solver invariants over 20 steps.  The
64-scene batch (5.07M particles in one context) and the 250k-particle implicit-viscosity
column are checked in their benchmark configurations too: the batch's smallest and largest
scenes field by field, the column's CG velocity against the oracle's FP64 system.  WCSPH,
PCISPH and strong coupling each take one step on the 1.2M dam break from the GPU's state,
compared with the oracle field by field."""
import numpy as np
import pytest

import oracle
from paper_2403_11156_gb300 import scenes, sph

from gpu_util import assert_abs, assert_rel, field_tolerances, forced, gpu_ctx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c2():
    d = scenes.dam_break_rigid()
    g = gpu_ctx(d)
    g.sph_step(0.0)
    g.sph_synchronize()
    return d, g


def test_keys_order_counts(c2):
    d, g = c2
    x = d["fluid_x"]
    cell = oracle.default_cell_size(d["radius"])
    keys = oracle.cell_keys(x, d["domain_min"], d["domain_max"], cell)
    np.testing.assert_array_equal(g.sph_read_field(sph.FIELD_CELL_KEY), keys)
    np.testing.assert_array_equal(g.sph_read_field(sph.FIELD_SORTED_ID), oracle.sort_order(keys))
    rng = np.random.default_rng(0)
    idx = rng.choice(len(x), size=1500, replace=False)
    h = np.float32(4 * d["radius"])
    nn = g.sph_read_field(sph.FIELD_NN_FLUID)
    np.testing.assert_array_equal(nn[idx], oracle.neighbor_counts_brute(x[idx], x, h, False) - 1)
    nb = g.sph_read_field(sph.FIELD_NN_BOUNDARY)
    np.testing.assert_array_equal(nb[idx], oracle.neighbor_counts_brute(x[idx], d["boundary_x"], h, False))


def test_density_alpha_psi_full(c2):
    d, g = c2
    o = oracle.Scene(d)
    o.prepare()
    assert_rel(g.sph_read_field(sph.FIELD_RHO), o.get(oracle.RHO), 1e-5, what="rho")
    assert_rel(g.sph_read_field(sph.FIELD_ALPHA), o.get(oracle.ALPHA), 1e-5, what="alpha")
    assert_rel(g.sph_read_field(sph.FIELD_PSI), o.get(oracle.PSI), 1e-5, what="psi")
    np.testing.assert_array_equal(g.sph_read_field(sph.FIELD_NN_FLUID), o.get(oracle.NN_F).astype(np.int32))


def test_twenty_steps_invariants(c2):
    d, g = c2
    g.sph_steps(20, 0.0)
    assert g.sph_synchronize(raise_on_error=False) == sph.SPH_OK
    st = g.sph_get_stats()
    assert st["dens_err"] <= 1e-3 and st["div_err"] <= 1e-3
    assert st["flags"] == 0 and st["steps"] == 21
    x, v, rho, p = g.sph_read_state()
    assert len(x) == 1200500 and np.all(np.isfinite(x)) and np.all(np.isfinite(v))
    assert np.all(x >= -0.01) and np.all(x[:, 0] <= 2.01)


def test_batch_of_64_scenes():
    # 64 dam breaks of 20k-200k particles (5.07M total) in one context
    ds = scenes.batch_dam_break()
    g = gpu_ctx(ds)
    g.sph_steps(10, 0.0)
    assert g.sph_synchronize(raise_on_error=False) == sph.SPH_OK
    for k in (0, 17, 63):
        st = g.sph_get_stats(k)
        assert st["steps"] == 10 and st["flags"] == 0 and st["dens_err"] <= 1e-3
        x, v, _, _ = g.sph_read_state(k)
        assert len(x) == len(ds[k]["fluid_x"]) and np.all(np.isfinite(x))


DT = 1e-3   # the scene's CFL step at rest (dt_max)


def _stepped_pair(d):
    """GPU context and oracle scene on the GPU's state after a first step (warm-start
    memory included), both then stepped once."""
    g = gpu_ctx(d)
    g.sph_step(DT)
    x, v, _, _ = g.sph_read_state()
    o = oracle.Scene(d)
    o.set_state(x, v, g.sph_read_field(sph.FIELD_KAPPA_PREV), g.sph_read_field(sph.FIELD_KAPPA_V_PREV))
    g.sph_step(DT)
    g.sph_synchronize(raise_on_error=False)
    o.step(DT)
    return g, o


def test_one_step_fields_full():
    # zero warm start: no decision of the step depends on a float comparison with a jump
    # (the warm-start gates open or close a whole stiffness), so every field compares
    # element by element; 2 divergence and 3 density iterations
    d = forced(scenes.dam_break_rigid(warm_start=scenes.WARM_ZERO), 2, 3)
    g, o = _stepped_pair(d)
    k_scale, v_tol = field_tolerances(o, d, DT)
    assert_rel(g.sph_read_field(sph.FIELD_RHO), o.get(oracle.RHO), 1e-5, what="rho")
    assert_abs(g.sph_read_field(sph.FIELD_KAPPA_V), o.get(oracle.KAPPA_V), 1e-5 * k_scale, "kappa_v")
    assert_abs(g.sph_read_field(sph.FIELD_KAPPA), o.get(oracle.KAPPA), 1e-5 * k_scale, "kappa")
    x2, v2, _, p2 = g.sph_read_state()
    assert_abs(v2, o.get(oracle.V), v_tol, "v")
    assert_abs(x2, o.get(oracle.X), v_tol * DT, "x")
    assert_abs(p2, o.get(oracle.PRESSURE), 1e-5 * k_scale * o.get(oracle.RHO), "pressure")
    gs, os_ = g.sph_get_stats(), o.stats()
    assert gs["dens_err"] == pytest.approx(os_["dens_err"], rel=1e-3, abs=1e-7)
    assert gs["div_err"] == pytest.approx(os_["div_err"], rel=1e-3, abs=1e-7)


def test_previous_step_warm_start_full():
    # the warm start's gate rho* > rho0 is decided in FP32 on the GPU and in FP64 in the
    # oracle; at 1.2M particles a few sit within rounding of rho0 and may decide apart.
    # Where both open it, kappa0 agrees within 1e-5 of its scale; flips are rare.
    d = forced(scenes.dam_break_rigid(), 2, 3)
    g, o = _stepped_pair(d)
    k_scale, _ = field_tolerances(o, d, DT)
    kg = g.sph_read_field(sph.FIELD_KAPPA0).astype(np.float64)
    ko = o.get(oracle.KAPPA0)
    gate_g, gate_o = kg > 0, ko > 0
    assert np.sum(gate_g != gate_o) <= 1e-4 * len(kg)
    both = gate_g & gate_o
    assert both.sum() > 100_000
    assert_abs(kg[both], ko[both], 1e-5 * k_scale[both], "kappa0")
    # the divergence solve's stiffness sum includes its own warm start, gated on D rho/Dt > 0
    # at the step's start (the same kind of float decision): all but a 1e-4 fraction of the
    # particles agree within the one-step tolerance
    kvg = g.sph_read_field(sph.FIELD_KAPPA_V).astype(np.float64)
    kvo = o.get(oracle.KAPPA_V)
    bad = np.abs(kvg - kvo) > 1e-5 * k_scale + 1e-5 * np.abs(kvo).max()
    assert np.sum(bad) <= 1e-4 * len(kvg)
    assert np.sum(kvo > 0) > 100_000


def test_learned_kappa0_full():
    # a network trained briefly on the solver's own states of a 200k-particle dam break;
    # the full scene's kappa0 against the oracle's FP64 network with the same weights
    from paper_2403_11156_gb300 import warmstart
    f, y = warmstart.generate_dataset(20_000, 20, n_scenes=1, size_range=(2e5, 2e5))
    params, _ = warmstart.train(f, y, epochs=10)
    d = forced(scenes.dam_break_rigid(warm_start=scenes.WARM_LEARNED), 1, 2)
    g = gpu_ctx(d)
    g.sph_set_mlp(params)
    for _ in range(3):
        g.sph_step(DT)
    x, v, _, _ = g.sph_read_state()
    o = oracle.Scene(d)
    o.set_mlp(params.astype(np.float64))
    o.set_state(x, v, g.sph_read_field(sph.FIELD_KAPPA_PREV), g.sph_read_field(sph.FIELD_KAPPA_V_PREV))
    g.sph_step(DT)
    g.sph_synchronize(raise_on_error=False)
    o.step(DT)
    kg = g.sph_read_field(sph.FIELD_KAPPA0).astype(np.float64)
    ko = o.get(oracle.KAPPA0)
    gate_g, gate_o = kg > 0, ko > 0
    assert np.mean(gate_g != gate_o) < 0.01
    both = gate_g & gate_o
    assert both.sum() > 10_000
    # BF16 layers: normwise 3e-2 of the FP64 network's kappa0
    assert np.linalg.norm(kg[both] - ko[both]) <= 3e-2 * np.linalg.norm(ko[both])


def test_batch_fields_full():
    # the 64-scene batch in one context (the bench's batched configuration): the smallest and
    # the largest scene against the oracle on its own, after the first step's sweep --
    # keys, order and neighbour counts bit-exact, density and alpha within 1e-5
    ds = scenes.batch_dam_break()
    g = gpu_ctx(ds)
    g.sph_step(0.0)
    assert g.sph_synchronize(raise_on_error=False) == sph.SPH_OK
    sizes = [len(d["fluid_x"]) for d in ds]
    for k in (int(np.argmin(sizes)), int(np.argmax(sizes))):
        d = ds[k]
        keys = oracle.cell_keys(d["fluid_x"], d["domain_min"], d["domain_max"],
                                oracle.default_cell_size(d["radius"]))
        np.testing.assert_array_equal(g.sph_read_field(sph.FIELD_CELL_KEY, k), keys)
        np.testing.assert_array_equal(g.sph_read_field(sph.FIELD_SORTED_ID, k), oracle.sort_order(keys))
        o = oracle.Scene(d)
        o.prepare()
        np.testing.assert_array_equal(g.sph_read_field(sph.FIELD_NN_FLUID, k), o.get(oracle.NN_F).astype(np.int32))
        assert_rel(g.sph_read_field(sph.FIELD_RHO, k), o.get(oracle.RHO), 1e-5, what="rho scene %d" % k)
        assert_rel(g.sph_read_field(sph.FIELD_ALPHA, k), o.get(oracle.ALPHA), 1e-5, what="alpha scene %d" % k)


def test_viscous_column_cg_full():
    # the 250k-particle column of the viscosity benchmark, 200 CFL steps in (after its
    # impact on the plane), then one step with the pressure solves off so that the velocity
    # is the implicit viscosity solve's v*: it solves the oracle's FP64 system
    # (I - dt A) v* = v + dt g to the CG tolerance plus the FP32 operator floor, and agrees
    # with the oracle's own CG solution
    d = scenes.viscous_column()
    g = gpu_ctx(d)
    g.sph_steps(200, 0.0)
    assert g.sph_synchronize(raise_on_error=False) == sph.SPH_OK
    x, v, _, _ = g.sph_read_state()
    d1 = dict(d, fluid_x=x, fluid_v=v, max_iter_density=0, min_iter_density=0, warm_start=0,
              divergence_solve=0)
    h = gpu_ctx(d1)
    h.sph_step(DT)
    assert h.sph_synchronize(raise_on_error=False) == sph.SPH_OK
    st = h.sph_get_stats()
    tol = d["cg_tol"]
    assert st["cg_iters"] > 5 and st["cg_residual"] <= tol * 1.0001
    v_gpu = h.sph_read_state()[1].astype(np.float64)
    o = oracle.Scene(d1)
    o.prepare()
    b = v.astype(np.float64) + DT * np.array(d["gravity"])
    res = o.visc_operator(DT, v_gpu) - b
    assert np.linalg.norm(res) <= (tol + 1e-5) * np.linalg.norm(b)
    o.step(DT)
    assert np.abs(v_gpu - o.get(oracle.V)).max() <= 20 * (tol + 1e-5) * np.abs(b).max()


def test_wcsph_step_full():
    # the bench's WCSPH workload (the 1.2M dam break without boxes at its acoustic step):
    # 20 steps build a compressed state, then one step from the GPU's state on both sides,
    # with the tolerances of the small-scene WCSPH parity test
    d = scenes.dam_break_rigid(n_boxes=0)
    d.update(scenes.wcsph_parameters(98 * 2 * d["radius"], d["radius"]))
    dt = d["dt_max"]
    g = gpu_ctx(d)
    g.sph_steps(20, dt)
    x, v, _, _ = g.sph_read_state()
    o = oracle.Scene(d)
    o.set_state(x, v, np.zeros(len(x), np.float32), np.zeros(len(x), np.float32))
    g.sph_step(dt)
    assert g.sph_synchronize(raise_on_error=False) == sph.SPH_OK
    o.step(dt)
    k, gamma = d["eos_stiffness"], d["eos_exponent"]
    assert_rel(g.sph_read_field(sph.FIELD_RHO), o.get(oracle.RHO), 1e-5, what="rho")
    x2, v2, _, p2 = g.sph_read_state()
    p_ref = o.get(oracle.PRESSURE)
    assert p_ref.max() > 0
    assert np.abs(p2 - p_ref).max() <= 1e-5 * gamma * k + 1e-5 * np.abs(p_ref).max()
    dv = o.get(oracle.V) - o.get(oracle.V_NONP)
    tol = 1e-3 * np.abs(dv).max() + 1e-5 * np.abs(o.get(oracle.V)).max()
    assert np.abs(v2 - o.get(oracle.V)).max() <= tol
    assert np.abs(x2 - o.get(oracle.X)).max() <= tol * dt + 1e-6


def test_pcisph_step_full():
    # the 1.2M dam break (no boxes) under PCISPH: 10 steps build a compressed state, then one
    # step from the GPU's state on both sides with three refinements forced, at the
    # tolerances of the small-scene PCISPH parity test (pressure: 3 refinements of delta times
    # the FP32 density resolution 1e-5 rho0; velocities: 2e-3 of the pressure velocity change)
    d = forced(scenes.dam_break_rigid(n_boxes=0, pressure_solver=scenes.SOLVER_PCISPH,
                                      warm_start=scenes.WARM_ZERO, divergence_solve=0), 0, 3)
    g = gpu_ctx(d)
    g.sph_steps(10, DT)
    x, v, _, _ = g.sph_read_state()
    o = oracle.Scene(d)
    z = np.zeros(len(x), np.float32)
    o.set_state(x, v, z, z)
    g.sph_step(DT)
    g.sph_synchronize(raise_on_error=False)
    o.step(DT)
    assert_rel(g.sph_read_field(sph.FIELD_RHO), o.get(oracle.RHO), 1e-5, what="rho")
    x2, v2, _, p2 = g.sph_read_state()
    p_ref = o.get(oracle.PRESSURE)
    delta = o.pcisph_factor() / DT ** 2
    assert p_ref.max() > 0
    assert np.abs(p2 - p_ref).max() <= 3 * delta * 1e-5 * d["rest_density"] + 1e-5 * np.abs(p_ref).max()
    dv = o.get(oracle.V) - o.get(oracle.V_NONP)
    tol = 2e-3 * np.abs(dv).max() + 1e-5 * np.abs(o.get(oracle.V)).max()
    assert np.abs(v2 - o.get(oracle.V)).max() <= tol
    assert np.abs(x2 - o.get(oracle.X)).max() <= tol * DT + 1e-6
    gs, os_ = g.sph_get_stats(), o.stats()
    assert gs["dens_iters"] == os_["dens_iters"] == 3 and gs["div_iters"] == 0
    assert gs["dens_err"] == pytest.approx(os_["dens_err"], rel=2e-3, abs=1e-7)


def test_strong_coupling_step_full():
    # the bench's strongly coupled 1.2M dam break (zero warm start, so that no warm-start gate
    # decides apart between FP32 and FP64), 500 CFL steps in, with the boxes in the flow: the
    # oracle resumes from the GPU's fluid and rigid state and takes the GPU's next step at the
    # GPU's iteration counts.  Each body's force within 2e-4 of its magnitude (as in the
    # small-scene strong test); torque and velocities within what that force error implies:
    # the lever arm (the cube's half-diagonal) times it for the torque, dt / mass and
    # dt r / I for the linear and angular velocity (the torque sums r x f over the surface
    # and cancels, so its own magnitude is not the scale).  Fluid velocities within the
    # DFSPH velocity bound of the full-size field test.
    d = scenes.dam_break_rigid(rigid_coupling=scenes.COUPLING_STRONG, warm_start=scenes.WARM_ZERO)
    g = gpu_ctx(d)
    g.sph_steps(500, 0.0)
    assert g.sph_synchronize(raise_on_error=False) == sph.SPH_OK
    x, v, _, _ = g.sph_read_state()
    b0 = g.sph_read_bodies()
    g.sph_step(DT)
    assert g.sph_synchronize(raise_on_error=False) == sph.SPH_OK
    st = g.sph_get_stats()
    o = oracle.Scene(forced(d, int(st["div_iters"]), int(st["dens_iters"])))
    o.set_state(x, v)
    o.set_bodies(b0)
    o.step(DT)
    gb, ob = g.sph_read_bodies(), o.bodies()
    for k, body in enumerate(d["bodies"]):
        F, T = ob[k, 13:16], ob[k, 16:19]
        assert np.abs(F).max() > 0                      # the box is in the fluid
        f_tol = 2e-4 * np.abs(F).max()
        edge = np.sqrt(6.0 * body["inertia"][0] / body["mass"])   # solid cube: I = m e^2 / 6
        arm = 0.5 * np.sqrt(3.0) * edge
        np.testing.assert_allclose(gb[k, 13:16], F, rtol=0, atol=f_tol)
        np.testing.assert_allclose(gb[k, 16:19], T, rtol=0, atol=arm * f_tol)
        np.testing.assert_allclose(gb[k, 7:10], ob[k, 7:10], rtol=0, atol=DT * f_tol / body["mass"] + 1e-9)
        np.testing.assert_allclose(gb[k, 10:13], ob[k, 10:13], rtol=0,
                                   atol=DT * arm * f_tol / body["inertia"][0] + 1e-9)
    _, v_tol = field_tolerances(o, d, DT)
    assert_abs(g.sph_read_state()[1], o.get(oracle.V), v_tol, "v")
