"""Pins of the oracle's neighbour-search contracts (Sec. 5.6 prefix-sum grid).

The float cell key, the (key, id) sort order and the strict float predicate are this
project's bit-exact contracts.  The oracle's internal cell-bucket lists are checked
against O(n^2) brute force on random, exact-lattice and jittered-lattice inputs.
"""
import numpy as np
import pytest

from paper_2403_11156_gb300 import scenes


def _lists_counts(oracle_lib, desc):
    d = dict(desc)
    d.update(max_iter_density=0, max_iter_divergence=0, warm_start=0, viscosity_mode=0)
    s = oracle_lib.Scene(d)
    s.step(1e-4)
    return s.get(oracle_lib.NN_F).astype(np.int32), s.get(oracle_lib.NN_B).astype(np.int32)


@pytest.mark.parametrize("kind", ["random", "lattice", "jitter"])
def test_lists_equal_brute_force(oracle_lib, kind):
    r = 0.01
    h = np.float32(4 * r)
    if kind == "random":
        d = scenes.random_cloud(1500, seed=11, radius=r, extent=0.25)
    else:
        d = scenes.dam_break_small(seed=5, n=(11, 11, 11), radius=r, box=0.3,
                                   jitter=(1e-4 if kind == "jitter" else 0.0))
    nf, nb = _lists_counts(oracle_lib, d)
    bf = oracle_lib.neighbor_counts_brute(d["fluid_x"], d["fluid_x"], h, True)
    np.testing.assert_array_equal(nf, bf)
    if len(d["boundary_x"]):
        bb = oracle_lib.neighbor_counts_brute(d["fluid_x"], d["boundary_x"], h, False)
        np.testing.assert_array_equal(nb, bb)


def test_exact_lattice_strict_tie(oracle_lib):
    # spacing 2^-6 (exact in float): axis neighbours at exactly h are excluded by '<'
    r = 2.0 ** -7
    s = 2 * r
    x = scenes.lattice_block((7, 7, 7), s, (0.25, 0.25, 0.25))
    c = oracle_lib.neighbor_counts_brute(x, x, np.float32(4 * r), True)
    centre = 3 + 7 * (3 + 7 * 3)
    assert c[centre] == 26
    # with the tie included (slightly larger h) the 6 axis neighbours at distance h join
    c2 = oracle_lib.neighbor_counts_brute(x, x, np.float32(4 * r) * np.float32(1.0001), True)
    assert c2[centre] == 32


def test_cell_keys_contract(oracle_lib):
    rng = np.random.default_rng(1)
    dmin = np.array([0.0, -0.5, 0.1], np.float32)
    dmax = np.array([1.0, 0.5, 0.7], np.float32)
    c = oracle_lib.default_cell_size(0.01)
    assert c > np.float32(0.04)
    x = rng.uniform(-0.2, 1.2, size=(5000, 3)).astype(np.float32)
    keys = oracle_lib.cell_keys(x, dmin, dmax, c)
    dims, org = oracle_lib.grid_dims(dmin, dmax, c)
    # independent restatement in numpy float32 arithmetic
    cf = np.float32(c)
    o = (dmin - cf).astype(np.float32)
    np.testing.assert_array_equal(org, o)
    n = (np.ceil((dmax - dmin) / cf).astype(np.int32) + 2)
    np.testing.assert_array_equal(dims, n)
    t = ((x - o) / cf).astype(np.float32)
    idx = np.floor(t).astype(np.int64)
    idx = np.clip(idx, 0, n - 1)
    exp = idx[:, 0] + n[0] * (idx[:, 1] + n[1] * idx[:, 2])
    np.testing.assert_array_equal(keys.astype(np.int64), exp)
    # every pair within h lies in adjacent cells
    i = idx
    xx = x[:400]
    d2 = ((xx[:, None, :] - xx[None, :, :]) ** 2).sum(-1)
    close = d2 < np.float32(0.04) ** 2
    a, b = np.nonzero(close)
    assert np.all(np.abs(i[a] - i[b]) <= 1)


def test_sort_order_lexicographic(oracle_lib):
    rng = np.random.default_rng(2)
    keys = rng.integers(0, 50, size=3000).astype(np.uint32)
    order = oracle_lib.sort_order(keys)
    exp = np.lexsort((np.arange(len(keys)), keys))
    np.testing.assert_array_equal(order, exp)
