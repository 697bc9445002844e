"""sph_grid_order_noalloc: the neighbour-search grid order for callers that cannot let a
library allocate device memory (work enqueued during another component's CUDA-graph
capture, applications that own the GPU memory budget, real-time loops).  Checked through
the C ABI against the grid order and cell keys that the regular path (sph_create +
sph_step) reports for the same positions, on two calls in a row that share the static
scratch array.  Collected last so that a stop-at-first-failure run has already run the
rest of the suite."""
import numpy as np
import pytest

from paper_2403_11156_gb300 import scenes, sph

from gpu_util import gpu_ctx

pytestmark = pytest.mark.gpu


def _reference(d):
    g = gpu_ctx(d)
    g.sph_step(4e-4)
    g.sph_synchronize(raise_on_error=False)
    order = g.sph_read_field(sph.FIELD_SORTED_ID)
    keys = g.sph_read_field(sph.FIELD_CELL_KEY)
    g.close()
    return order, keys


def test_noalloc_grid_order_matches_regular_path():
    import torch
    d = scenes.dam_break_small()                      # 8,000 points
    order_ref, keys_ref = _reference(d)
    cell = np.float32(np.float32(4.0) * np.float32(d["radius"])) * np.float32(1.00390625)
    x = torch.from_numpy(np.ascontiguousarray(d["fluid_x"])).cuda()
    n = len(d["fluid_x"])
    stream = torch.cuda.current_stream()
    for _ in range(2):                                # the second call reuses the scratch
        order = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        keys = torch.zeros(n, dtype=torch.int32, device="cuda")
        st = sph.sph_grid_order_noalloc(x, n, d["domain_min"], d["domain_max"], np.float32(cell),
                                        order, keys, stream)
        assert st == sph.SPH_OK
        torch.cuda.synchronize()
        np.testing.assert_array_equal(order.cpu().numpy(), order_ref)
        np.testing.assert_array_equal(keys.cpu().numpy().view(np.uint32), keys_ref)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    x = torch.zeros((4, 3), device="cuda")
    out = torch.zeros(4, dtype=torch.int32, device="cuda")
    too_many = sph.NOALLOC_MAX_POINTS + 1
    assert sph.sph_grid_order_noalloc(x, too_many, (0, 0, 0), (1, 1, 1), 0.04, out) == sph.SPH_EINVAL
    # 1 m cube at cell 0.004 m: 252^3 cells > SPH_NOALLOC_MAX_CELLS
    assert sph.sph_grid_order_noalloc(x, 4, (0, 0, 0), (1, 1, 1), 0.004, out) == sph.SPH_EINVAL
