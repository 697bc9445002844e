"""GPU edge cases against the oracle: the degenerate scenes of the method.

- One particle, no boundary: no neighbour, so alpha = 0 (the DFSPH factor's denominator
  vanishes), both solves apply nothing, and the particle falls freely; its density is the
  self term m W(0).
- A sparse cloud in which most particles have no neighbour and a few have one to three:
  neighbour counts bit-exact, density within 1e-5, one step's velocities within the DFSPH
  velocity bound.  alpha = rho / (|sum m grad W|^2 + sum |m grad W|^2) of a particle with
  one or two neighbours cannot average rounding over a full neighbourhood: near the edge of
  the support the spline gradient goes as (1 - q)^2, FP32 gives 1 - q to about 3 eps
  absolute (q = r / h through a rounded sum of squares, rsqrt and product), so alpha,
  inversely quadratic in the gradients, carries a relative error up to 12 eps / (1 - q).
  Its bound is 1e-5 plus that for the particle's outermost neighbour (measured 1.45e-5, a
  quarter of its bound, on a particle whose outermost pair sits at q = 0.97).
- A one-particle scene batched beside a lattice scene steps bit-identically to each alone
  (a scene smaller than a warp shares no block with its neighbour in the batch)."""
import numpy as np
import pytest

import oracle
from paper_2403_11156_gb300 import scenes, sph

from gpu_util import assert_abs, assert_rel, field_tolerances, forced, gpu_ctx

pytestmark = pytest.mark.gpu

DT = 4e-4


@pytest.mark.parametrize("lanes", [1, 8])
def test_single_particle_falls_freely(lanes):
    d = scenes.random_cloud(1, seed=2, extent=0.5, lanes_per_particle=lanes)
    g = gpu_ctx(d)
    o = oracle.Scene(d)
    for _ in range(10):
        g.sph_step(DT)
        o.step(DT)
    assert g.sph_synchronize(raise_on_error=False) == sph.SPH_OK
    x, v, rho, _ = g.sph_read_state()
    assert g.sph_read_field(sph.FIELD_NN_FLUID)[0] == 0
    assert g.sph_read_field(sph.FIELD_ALPHA)[0] == 0.0
    np.testing.assert_allclose(rho, o.get(oracle.RHO), rtol=1e-6)
    # gravity alone: v = g t (FP32 sums of dt g against the oracle's FP64)
    np.testing.assert_allclose(v, o.get(oracle.V), rtol=1e-5, atol=0)
    assert v[0, 2] == pytest.approx(-9.81 * 10 * DT, rel=1e-5)
    np.testing.assert_allclose(x, o.get(oracle.X), rtol=0, atol=1e-6)


@pytest.mark.parametrize("lanes", [1, 8])
def test_sparse_cloud_fields(lanes):
    # 300 particles in a 0.5 m cube (mean spacing 7.5 cm against h = 4 cm): mostly
    # isolated, some pairs and triples
    d = forced(scenes.random_cloud(300, seed=9, extent=0.5, lanes_per_particle=lanes), 1, 2)
    g = gpu_ctx(d)
    g.sph_step(DT)
    assert g.sph_synchronize(raise_on_error=False) == sph.SPH_OK
    o = oracle.Scene(d)
    o.step(DT)
    nn = g.sph_read_field(sph.FIELD_NN_FLUID)
    np.testing.assert_array_equal(nn, o.get(oracle.NN_F).astype(np.int32))
    assert (nn == 0).sum() > 100 and nn.max() >= 1
    assert_rel(g.sph_read_field(sph.FIELD_RHO), o.get(oracle.RHO), 1e-5, what="rho")
    # per particle: 1e-5 + 12 eps32 / (1 - q) of its outermost neighbour (q = r / h)
    x = d["fluid_x"].astype(np.float64)
    h = 4.0 * d["radius"]
    q = np.sqrt(((x[:, None, :] - x[None, :, :]) ** 2).sum(-1)) / h
    q[(q >= 1.0) | (q == 0.0)] = 0.0
    bound = 1e-5 + 12 * np.finfo(np.float32).eps / (1.0 - q.max(axis=1))
    a_g = g.sph_read_field(sph.FIELD_ALPHA).astype(np.float64)
    a_o = o.get(oracle.ALPHA)
    np.testing.assert_array_equal(a_g == 0, a_o == 0)
    e = np.abs(a_g - a_o) / np.maximum(np.abs(a_o), 1e-30)
    assert np.all(e <= bound), (e.max(), bound[np.argmax(e / bound)])
    _, v_tol = field_tolerances(o, d, DT)
    assert_abs(g.sph_read_state()[1], o.get(oracle.V), v_tol, "v")


def test_one_particle_scene_in_a_batch():
    ds = [scenes.random_cloud(1, seed=4, extent=0.3),
          scenes.dam_break_small(seed=7, n=(9, 11, 13), box=0.4),
          scenes.random_cloud(1, seed=5, extent=0.3)]
    batch = gpu_ctx(ds)
    batch.sph_steps(5, DT)
    assert batch.sph_synchronize(raise_on_error=False) == sph.SPH_OK
    for k, d in enumerate(ds):
        single = gpu_ctx(d)
        single.sph_steps(5, DT)
        for u, w in zip(batch.sph_read_state(k), single.sph_read_state()):
            np.testing.assert_array_equal(u, w)


@pytest.mark.parametrize("lanes", [1, 8])
def test_crowded_cells_keep_the_grid_order(lanes):
    # 1,500 fluid particles squeezed into a few cells (plus a regular block) and 600
    # boundary points outside the domain, clamped into its edge cells: cells of hundreds of
    # particles go through the block-sorted path of the grid order, which must still give
    # the (cell key, id) order bit for bit
    rng = np.random.default_rng(11)
    d = scenes.dam_break_small(seed=2, n=(8, 8, 8), box=0.4, lanes_per_particle=lanes,
                               max_iter_density=1, min_iter_density=1, max_iter_divergence=1)
    crowd = (0.2 + 0.03 * rng.random((1500, 3))).astype(np.float32)
    x = np.concatenate([d["fluid_x"], crowd]).astype(np.float32)
    d["fluid_x"], d["fluid_v"] = x, np.zeros_like(x)
    out = (np.array([0.9, 0.1, -0.5]) + 0.01 * rng.random((600, 3))).astype(np.float32)
    bx = np.concatenate([d["boundary_x"], out]).astype(np.float32)
    d["boundary_x"] = bx
    d["boundary_body"] = np.full(len(bx), -1, np.int32)
    g = gpu_ctx(d)
    g.sph_step(DT)
    g.sph_synchronize(raise_on_error=False)           # the crowd overflows the lists
    cell = oracle.default_cell_size(d["radius"])
    keys = oracle.cell_keys(x, d["domain_min"], d["domain_max"], cell)
    assert np.bincount(keys).max() > 200               # crowded cells were exercised
    np.testing.assert_array_equal(g.sph_read_field(sph.FIELD_SORTED_ID), oracle.sort_order(keys))
    bkeys = oracle.cell_keys(bx, d["domain_min"], d["domain_max"], cell)
    assert np.bincount(bkeys).max() > 200
    np.testing.assert_array_equal(g.sph_read_field(sph.FIELD_BOUNDARY_SORTED_ID), oracle.sort_order(bkeys))
