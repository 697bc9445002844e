"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same
seeded inputs.

Bit-exact: cell keys, (key, id) sort order, fluid and boundary neighbour counts.
Every check runs with 1, 2, 4 and 8 threads per particle in the neighbour sweeps (the
neighbour sets are the same; only the FP32 summation order changes).
FP32 vs FP64 fields from one step off identical states with the iteration counts forced
equal: density, Psi and alpha within 1e-5 relative (alpha with a floor of 1e-3 rms for
free-surface particles whose factor is tiny); the stiffnesses kappa within 1e-5 of their
natural scale alpha_i rho0 / dt^2 (kappa turns a density deviation into a velocity
change, so that scale corresponds to a 1e-5 rho0 error in rho*, the quantity FP32 can
resolve; rho* - rho0 itself cancels to ~1e-2 of rho in FP32); velocities and positions
within the velocity change that such a density error implies, v_tol = 1e-5 rho0
sqrt(alpha/rho) / dt per particle (plus 1e-5 relative).
"""
import numpy as np
import pytest

import oracle
from paper_2403_11156_gb300 import scenes, sph

from gpu_util import assert_abs as _assert_abs, assert_rel, field_tolerances as _field_tolerances, forced, gpu_ctx, oracle_step

pytestmark = pytest.mark.gpu

DT = 4e-4


def _c1(**kw):
    return scenes.dam_break_small(**kw)


def _small(**kw):
    # several tiles of 128 particles plus a ragged tail (9 x 11 x 13 = 1287)
    return scenes.dam_break_small(seed=7, n=(9, 11, 13), box=0.4, **kw)


LANES = [1, 2, 4, 8]


@pytest.mark.parametrize("lanes", LANES)
@pytest.mark.parametrize("make", [_small, _c1])
def test_neighbor_structures_bit_exact(make, lanes):
    d = forced(make(lanes_per_particle=lanes), 1, 2)
    g = gpu_ctx(d)
    g.sph_step(DT)
    g.sph_synchronize(raise_on_error=False)
    x = d["fluid_x"]
    cell = oracle.default_cell_size(d["radius"])
    keys = oracle.cell_keys(x, d["domain_min"], d["domain_max"], cell)
    np.testing.assert_array_equal(g.sph_read_field(sph.FIELD_CELL_KEY), keys)
    np.testing.assert_array_equal(g.sph_read_field(sph.FIELD_SORTED_ID), oracle.sort_order(keys))
    bkeys = oracle.cell_keys(d["boundary_x"], d["domain_min"], d["domain_max"], cell)
    np.testing.assert_array_equal(g.sph_read_field(sph.FIELD_BOUNDARY_CELL_KEY), bkeys)
    np.testing.assert_array_equal(g.sph_read_field(sph.FIELD_BOUNDARY_SORTED_ID),
                                  oracle.sort_order(bkeys))
    h = np.float32(4 * d["radius"])
    np.testing.assert_array_equal(g.sph_read_field(sph.FIELD_NN_FLUID),
                                  oracle.neighbor_counts_brute(x, x, h, True))
    np.testing.assert_array_equal(g.sph_read_field(sph.FIELD_NN_BOUNDARY),
                                  oracle.neighbor_counts_brute(x, d["boundary_x"], h, False))


@pytest.mark.parametrize("lanes", LANES)
def test_exact_lattice_ties(lanes):
    # positions exact in float, spacing h/2: pairs at exactly h are excluded by '<'
    r = 2.0 ** -7
    x = scenes.lattice_block((10, 10, 10), 2 * r, (0.25, 0.25, 0.25))
    d = scenes.random_cloud(1, radius=r, extent=0.6, gravity=(0, 0, 0), warm_start=0,
                            max_iter_density=0, max_iter_divergence=0, lanes_per_particle=lanes)
    d["fluid_x"], d["fluid_v"] = x, np.zeros_like(x)
    g = gpu_ctx(d)
    g.sph_step(DT)
    nn = g.sph_read_field(sph.FIELD_NN_FLUID)
    np.testing.assert_array_equal(nn, oracle.neighbor_counts_brute(x, x, np.float32(4 * r), True))
    assert nn[5 + 10 * (5 + 10 * 5)] == 26


@pytest.mark.parametrize("cell_factor", [1.00390625, 0.501953125])
@pytest.mark.parametrize("lanes", LANES)
def test_counts_with_particles_outside_domain(lanes, cell_factor):
    # particles beyond the domain are clamped into the edge cells; the stencil culling of
    # the density sweep must still find exactly the brute-force neighbours
    rng = np.random.default_rng(11)
    r = 0.01
    x = rng.uniform(-0.06, 0.26, size=(3000, 3)).astype(np.float32)
    d = scenes.random_cloud(1, radius=r, extent=0.2, gravity=(0, 0, 0), warm_start=0,
                            max_iter_density=0, max_iter_divergence=0, lanes_per_particle=lanes,
                            max_fluid_neighbors=400)
    d["fluid_x"], d["fluid_v"] = x, np.zeros_like(x)
    h = np.float32(4 * r)
    d["cell_size"] = float(h * np.float32(cell_factor))
    g = gpu_ctx(d)
    g.sph_step(DT)
    g.sph_synchronize(raise_on_error=False)
    np.testing.assert_array_equal(g.sph_read_field(sph.FIELD_NN_FLUID),
                                  oracle.neighbor_counts_brute(x, x, h, True))


@pytest.mark.parametrize("lanes", LANES)
@pytest.mark.parametrize("make", [_small, _c1])
def test_density_alpha_psi(make, lanes):
    d = forced(make(lanes_per_particle=lanes), 1, 2)
    g = gpu_ctx(d)
    g.sph_step(DT)
    o = oracle_step(d, DT)
    assert_rel(g.sph_read_field(sph.FIELD_PSI), o.get(oracle.PSI), 1e-5, what="psi")
    assert_rel(g.sph_read_field(sph.FIELD_RHO), o.get(oracle.RHO), 1e-5, what="rho")
    assert_rel(g.sph_read_field(sph.FIELD_ALPHA), o.get(oracle.ALPHA), 1e-5, what="alpha")


@pytest.mark.parametrize("lanes", LANES)
@pytest.mark.parametrize("make,warm,visc", [
    (_small, 0, 1), (_small, 1, 1), (_c1, 1, 1), (_small, 1, 2), (_small, 1, 0)])
def test_one_step_fields(make, warm, visc, lanes):
    d = forced(make(warm_start=warm, viscosity_mode=visc, xsph_c=0.05, lanes_per_particle=lanes), 2, 3)
    g = gpu_ctx(d)
    o = oracle.Scene(d)
    # a first step builds the warm-start memory on both sides from the same input; the
    # second step starts from the GPU's state (fed to the oracle) so both start equal
    g.sph_step(DT)
    x, v, _, _ = g.sph_read_state()
    kp = g.sph_read_field(sph.FIELD_KAPPA_PREV)
    kvp = g.sph_read_field(sph.FIELD_KAPPA_V_PREV)
    o.set_state(x, v, kp, kvp)
    g.sph_step(DT)
    g.sph_synchronize(raise_on_error=False)
    o.step(DT)
    k_scale, v_tol = _field_tolerances(o, d, DT)
    assert_rel(g.sph_read_field(sph.FIELD_RHO), o.get(oracle.RHO), 1e-5, what="rho")
    _assert_abs(g.sph_read_field(sph.FIELD_KAPPA_V), o.get(oracle.KAPPA_V), 1e-5 * k_scale, "kappa_v")
    _assert_abs(g.sph_read_field(sph.FIELD_KAPPA), o.get(oracle.KAPPA), 1e-5 * k_scale, "kappa")
    _assert_abs(g.sph_read_field(sph.FIELD_V_DIV), o.get(oracle.V_DIV), v_tol, "v after divergence solve")
    x2, v2, rho2, p2 = g.sph_read_state()
    _assert_abs(v2, o.get(oracle.V), v_tol, "v")
    _assert_abs(x2, o.get(oracle.X), v_tol * DT, "x")
    _assert_abs(p2, o.get(oracle.PRESSURE), 1e-5 * k_scale * o.get(oracle.RHO), "pressure")
    gs, os_ = g.sph_get_stats(), o.stats()
    assert gs["div_iters"] == os_["div_iters"] == 2 and gs["dens_iters"] == os_["dens_iters"] == 3
    assert gs["dens_err"] == pytest.approx(os_["dens_err"], rel=1e-3, abs=1e-7)
    assert gs["div_err"] == pytest.approx(os_["div_err"], rel=1e-3, abs=1e-7)


def test_warm_start_fraction_parity():
    # a non-default warm-start fraction enters both warm starts the same way on both sides
    d = forced(_small(warm_start=1, warm_start_fraction=0.75), 2, 3)
    g = gpu_ctx(d)
    o = oracle.Scene(d)
    g.sph_step(DT)
    x, v, _, _ = g.sph_read_state()
    o.set_state(x, v, g.sph_read_field(sph.FIELD_KAPPA_PREV), g.sph_read_field(sph.FIELD_KAPPA_V_PREV))
    g.sph_step(DT)
    g.sph_synchronize(raise_on_error=False)
    o.step(DT)
    k_scale, v_tol = _field_tolerances(o, d, DT)
    _assert_abs(g.sph_read_field(sph.FIELD_KAPPA0), o.get(oracle.KAPPA0), 1e-5 * k_scale, "kappa0")
    _assert_abs(g.sph_read_field(sph.FIELD_KAPPA), o.get(oracle.KAPPA), 1e-5 * k_scale, "kappa")
    _assert_abs(g.sph_read_state()[1], o.get(oracle.V), v_tol, "v")


def test_iteration_counts_track_oracle():
    d = _c1()
    g = gpu_ctx(d)
    o = oracle.Scene(d)
    for k in range(10):
        x, v, _, _ = g.sph_read_state()
        if k:
            o.set_state(x, v, g.sph_read_field(sph.FIELD_KAPPA_PREV), g.sph_read_field(sph.FIELD_KAPPA_V_PREV))
        g.sph_step(DT)
        o.step(DT)
        gs, os_ = g.sph_get_stats(), o.stats()
        assert abs(gs["div_iters"] - os_["div_iters"]) <= 1
        assert abs(gs["dens_iters"] - os_["dens_iters"]) <= 1


def test_hundred_steps_invariants():
    d = _c1()
    g = gpu_ctx(d)
    for k in range(100):
        g.sph_step(0.0)
        if k % 10 == 9:
            st = g.sph_get_stats()
            assert st["dens_err"] <= d["eta_density"] or st["dens_iters"] == d["max_iter_density"]
            assert st["div_err"] <= d["eta_divergence"] or st["div_iters"] == d["max_iter_divergence"]
    assert g.sph_synchronize() == sph.SPH_OK
    x, v, rho, p = g.sph_read_state()
    assert np.all(np.isfinite(x)) and np.all(np.isfinite(v))
    assert len(x) == 8000
    st = g.sph_get_stats()
    assert st["steps"] == 100 and st["flags"] == 0
    assert st["total_dens_iters"] >= 200 and st["total_div_iters"] >= 100
