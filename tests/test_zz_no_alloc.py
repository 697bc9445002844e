"""sph_grid_order_noalloc: the neighbour-search grid order for callers that cannot let a
library allocate device memory (work enqueued during another component's CUDA-graph
capture, applications that own the GPU memory budget, real-time loops).  Checked through
the C ABI against the oracle's cell keys and (cell key, index) order (the float cell-key
contract of the neighbour search, bit-exact), on two calls in a row that share the static
scratch array, with points outside the domain clamped into the edge cells; and against
the grid order the regular path (sph_create + sph_step) reports for the same positions.
Collected last so that a stop-at-first-failure run has already run the rest of the
suite."""
import numpy as np
import pytest

import oracle
from paper_2403_11156_gb300 import scenes, sph

from gpu_util import gpu_ctx

pytestmark = pytest.mark.gpu


def _run(x_np, dmin, dmax, cell, stream):
    import torch
    n = len(x_np)
    x = torch.from_numpy(np.ascontiguousarray(x_np)).cuda()
    order = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    keys = torch.zeros(n, dtype=torch.int32, device="cuda")
    st = sph.sph_grid_order_noalloc(x, n, dmin, dmax, np.float32(cell), order, keys, stream)
    assert st == sph.SPH_OK
    assert sph.sph_grid_order_noalloc_status(stream) == sph.SPH_OK
    return order.cpu().numpy(), keys.cpu().numpy().view(np.uint32)


def test_noalloc_grid_order_matches_oracle():
    import torch
    d = scenes.dam_break_small()                      # 8,000 points
    x = np.array(d["fluid_x"])
    # a few points outside the domain (and on its faces): clamped into the edge cells
    x[:6] = np.array([[-0.3, 0.2, 0.2], [0.9, 0.2, 0.2], [0.2, -1.0, 0.2],
                      [0.2, 0.2, 5.0], [0.0, 0.0, 0.0], [0.8, 0.8, 0.8]], np.float32)
    cell = oracle.default_cell_size(d["radius"])
    keys_o = oracle.cell_keys(x, d["domain_min"], d["domain_max"], cell)
    order_o = oracle.sort_order(keys_o)
    stream = torch.cuda.current_stream()
    for _ in range(2):                                # the second call reuses the scratch
        order, keys = _run(x, d["domain_min"], d["domain_max"], cell, stream)
        np.testing.assert_array_equal(keys, keys_o)
        np.testing.assert_array_equal(order, order_o)


def test_noalloc_grid_order_matches_regular_path():
    import torch
    d = scenes.dam_break_small(seed=4, n=(12, 14, 10))
    g = gpu_ctx(d)
    g.sph_step(4e-4)
    g.sph_synchronize(raise_on_error=False)
    order_ref = g.sph_read_field(sph.FIELD_SORTED_ID)
    keys_ref = g.sph_read_field(sph.FIELD_CELL_KEY)
    g.close()
    cell = oracle.default_cell_size(d["radius"])
    order, keys = _run(d["fluid_x"], d["domain_min"], d["domain_max"], cell,
                       torch.cuda.current_stream())
    np.testing.assert_array_equal(order, order_ref)
    np.testing.assert_array_equal(keys, keys_ref)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    x = torch.zeros((4, 3), device="cuda")
    out = torch.zeros(4, dtype=torch.int32, device="cuda")
    too_many = sph.NOALLOC_MAX_POINTS + 1
    assert sph.sph_grid_order_noalloc(x, too_many, (0, 0, 0), (1, 1, 1), 0.04, out) == sph.SPH_EINVAL
    # 1 m cube at cell 0.004 m: 252^3 cells > SPH_NOALLOC_MAX_CELLS
    assert sph.sph_grid_order_noalloc(x, 4, (0, 0, 0), (1, 1, 1), 0.004, out) == sph.SPH_EINVAL


def test_noalloc_crowded_cells_order_and_linear_time():
    # 5,000 and 20,000 points clamped into at most 8 cells (a corner outside the domain):
    # the order is the oracle's, and the time grows about linearly with the count (a
    # per-point count over the whole cell would grow 16-fold from 5k to 20k)
    import torch
    dmin, dmax = (0.0, 0.0, 0.0), (0.4, 0.4, 0.4)
    cell = oracle.default_cell_size(0.01)
    stream = torch.cuda.current_stream()
    times = {}
    for n in (5000, 20000):
        rng = np.random.default_rng(n)
        x = (np.array([-1.0, -1.0, -1.0]) + rng.random((n, 3)) * np.array([0.5, 1.6, 1.6]) *
             np.where(rng.random((n, 3)) < 0.5, 1.0, -1.0)).astype(np.float32)
        x[:, 1:] = np.clip(x[:, 1:], -2.0, 0.03)       # y, z: first or second cell
        keys_o = oracle.cell_keys(x, dmin, dmax, cell)
        assert len(np.unique(keys_o)) <= 8
        order, keys = _run(x, dmin, dmax, cell, stream)
        np.testing.assert_array_equal(keys, keys_o)
        np.testing.assert_array_equal(order, oracle.sort_order(keys_o))
        xd = torch.from_numpy(x).cuda()
        out = torch.empty(n, dtype=torch.int32, device="cuda")
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(3):
            sph.sph_grid_order_noalloc(xd, n, dmin, dmax, np.float32(cell), out, None, stream)
        a.record(stream)
        for _ in range(10):
            sph.sph_grid_order_noalloc(xd, n, dmin, dmax, np.float32(cell), out, None, stream)
        b.record(stream)
        torch.cuda.synchronize()
        assert sph.sph_grid_order_noalloc_status(stream) == sph.SPH_OK
        times[n] = a.elapsed_time(b) / 10
    assert times[20000] < 8.0 * times[5000], times
