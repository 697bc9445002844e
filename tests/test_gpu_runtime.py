"""GPU runtime behaviour: status codes, checkpoint/resume, graph vs eager replay, batched
scenes vs single scenes, launch counting."""
import numpy as np
import pytest

from paper_2403_11156_gb300 import scenes, sph

from gpu_util import gpu_ctx

pytestmark = pytest.mark.gpu
DT = 4e-4


def _small(seed=7, **kw):
    return scenes.dam_break_small(seed=seed, n=(9, 11, 13), box=0.4, **kw)


def test_noconverge_reported_and_state_advances():
    d = _small(max_iter_density=1, min_iter_density=1, eta_density=1e-12)
    g = gpu_ctx(d)
    x0 = g.sph_read_state()[0]
    g.sph_step(DT)
    assert g.sph_synchronize(raise_on_error=False) == sph.SPH_ENOCONVERGE
    st = g.sph_get_stats()
    assert st["dens_iters"] == 1 and st["flags"] & 2
    assert not np.array_equal(g.sph_read_state()[0], x0)
    g.sph_step(DT)                                     # context still usable
    assert g.sph_synchronize(raise_on_error=False) == sph.SPH_OK   # already reported


@pytest.mark.parametrize("lanes", [1, 2, 4, 8])
def test_overflow_reported(lanes):
    g = gpu_ctx(_small(max_fluid_neighbors=8, lanes_per_particle=lanes))
    g.sph_step(DT)
    assert g.sph_synchronize(raise_on_error=False) == sph.SPH_EOVERFLOW
    assert g.sph_get_stats()["max_fluid_nbrs"] > 8


def test_lanes_default_by_size():
    assert gpu_ctx(_small()).sph_get_tuning()["lanes"] == 8            # 1,287 particles
    mid = scenes.dam_break_small(n=(40, 40, 30), box=1.0)               # 48,000
    assert gpu_ctx(mid).sph_get_tuning()["lanes"] == 4
    big = scenes.dam_break_small(n=(60, 40, 40), box=1.4)               # 96,000
    assert gpu_ctx(big).sph_get_tuning()["lanes"] == 2
    assert gpu_ctx(dict(big, lanes_per_particle=1)).sph_get_tuning()["lanes"] == 1


@pytest.mark.parametrize("lanes", [4, 8])
def test_lanes_change_only_rounding(lanes):
    # the same 10 steps with 1 and 4 (8) threads per particle: identical neighbour counts,
    # iteration counts equal or off by one, positions within FP32 rounding growth
    a, b = gpu_ctx(_small(lanes_per_particle=1)), gpu_ctx(_small(lanes_per_particle=lanes))
    for g in (a, b):
        g.sph_steps(10, DT)
    np.testing.assert_array_equal(a.sph_read_field(sph.FIELD_NN_FLUID), b.sph_read_field(sph.FIELD_NN_FLUID))
    sa, sb = a.sph_get_stats(), b.sph_get_stats()
    assert abs(sa["total_dens_iters"] - sb["total_dens_iters"]) <= 2
    np.testing.assert_allclose(a.sph_read_state()[0], b.sph_read_state()[0], rtol=0, atol=1e-5)


def test_checkpoint_resume_bit_exact():
    d = _small()
    a = gpu_ctx(d)
    a.sph_steps(6, DT)
    x, v, _, _ = a.sph_read_state()
    kp = a.sph_read_field(sph.FIELD_KAPPA_PREV)
    kvp = a.sph_read_field(sph.FIELD_KAPPA_V_PREV)
    b = gpu_ctx(d)
    b.sph_write_state(0, x, v, kp, kvp)
    for ctx in (a, b):
        ctx.sph_steps(3, DT)
    xa, va, ra, pa = a.sph_read_state()
    xb, vb, rb, pb = b.sph_read_state()
    np.testing.assert_array_equal(xa, xb)
    np.testing.assert_array_equal(va, vb)
    np.testing.assert_array_equal(ra, rb)
    np.testing.assert_array_equal(pa, pb)


def test_graph_and_eager_identical():
    d = _small(cfl=0.4, dt_max=1e-3)
    a = gpu_ctx(d)
    b = gpu_ctx(d)
    b.sph_set_mode(graph=False, timing=True)
    for ctx in (a, b):
        ctx.sph_steps(8, 0.0)
    for u, w in zip(a.sph_read_state(), b.sph_read_state()):
        np.testing.assert_array_equal(u, w)
    assert a.sph_get_stats()["total_dens_iters"] == b.sph_get_stats()["total_dens_iters"]
    assert a.sph_launch_count() == b.sph_launch_count()
    kt = b.sph_kernel_times()
    assert kt["density_alpha"][0] == 8 and kt["advect"][0] == 8


def test_batch_equals_single():
    ds = [_small(seed=3), scenes.dam_break_small(seed=4, n=(17, 5, 9), box=0.5, warm_start=0),
          _small(seed=5, viscosity_mode=2, xsph_c=0.1)]
    batch = gpu_ctx(ds)
    batch.sph_steps(6, DT)
    for k, d in enumerate(ds):
        single = gpu_ctx(d)
        single.sph_steps(6, DT)
        for u, w in zip(batch.sph_read_state(k), single.sph_read_state()):
            np.testing.assert_array_equal(u, w)
        assert batch.sph_get_stats(k)["total_dens_iters"] == single.sph_get_stats()["total_dens_iters"]


def test_read_state_device_matches_host():
    import torch
    d = _small()
    g = gpu_ctx(d)
    g.sph_steps(2, DT)
    n = len(d["fluid_x"])
    x = torch.empty((n, 3), device="cuda")
    p = torch.empty(n, device="cuda")
    g.sph_read_state_device(0, x=x, pressure=p)
    hx, _, _, hp = g.sph_read_state()
    np.testing.assert_array_equal(x.cpu().numpy(), hx)
    np.testing.assert_array_equal(p.cpu().numpy(), hp)


def test_enqueue_only_read_matches_synchronous_read():
    import torch
    d = _small()
    g = gpu_ctx(d)
    g.sph_steps(3, DT)
    n = len(d["fluid_x"])
    x = torch.empty((n, 3), device="cuda")
    g.sph_read_state_device(0, x=x, sync=False)
    g.sph_synchronize()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(x.cpu().numpy(), g.sph_read_state()[0])



def test_bounded_wait_that_runs_out_reports_timeout():
    """A device wait that runs out (the probe waits on a flag that nothing sets, about 200 us)
    is reported as SPH_ETIMEOUT and poisons the context; the GPU stays usable for a new one.
    No kernel faults, traps or hangs."""
    d = _small()
    g = gpu_ctx(d)
    g.sph_step(DT)
    assert g.sph_synchronize(raise_on_error=False) == sph.SPH_OK
    assert g.sph_probe_wait_timeout(200) == sph.SPH_OK
    assert g.sph_synchronize(raise_on_error=False) == sph.SPH_ETIMEOUT
    with pytest.raises(sph.SphError):
        g.sph_step(DT)
    g.close()
    h = gpu_ctx(d)
    h.sph_step(DT)
    assert h.sph_synchronize(raise_on_error=False) == sph.SPH_OK


def test_nonfinite_state_reported():
    # a NaN velocity written into the state (host-side injection) is caught after the step
    d = _small()
    g = gpu_ctx(d)
    g.sph_step(DT)
    _, v, _, _ = g.sph_read_state()
    v = v.copy()
    v[5] = np.nan
    g.sph_write_state(v=v)
    g.sph_step(DT)
    assert g.sph_synchronize(raise_on_error=False) == sph.SPH_ENUMERIC


def test_large_batch_equals_single():
    """More scenes than one warp of the convergence check's block handles at once and an
    implicit-viscosity scene: every reduction order depends on the scene alone, so each scene
    of the batch steps bit-identically to the scene alone."""
    ds = [scenes.dam_break_small(seed=11 + k, n=(6 + k, 7, 5 + 2 * k), box=0.4) for k in range(5)]
    ds.append(_small(seed=17, viscosity=0.05, viscosity_mode=scenes.VISC_IMPLICIT))
    batch = gpu_ctx(ds)
    batch.sph_steps(5, DT)
    for k, d in enumerate(ds):
        single = gpu_ctx(d)
        single.sph_steps(5, DT)
        for u, w in zip(batch.sph_read_state(k), single.sph_read_state()):
            np.testing.assert_array_equal(u, w)
        sb, ss = batch.sph_get_stats(k), single.sph_get_stats()
        assert sb["total_dens_iters"] == ss["total_dens_iters"]
        assert sb["total_div_iters"] == ss["total_div_iters"]
        assert sb["cg_iters"] == ss["cg_iters"]


def test_every_kind_batched_matches_single():
    # one context holding a scene of every kind: DFSPH, PCISPH, WCSPH, a strongly coupled
    # body (moving boundary), an implicit-viscosity column, and a DFSPH scene without the
    # divergence solve or warm start and with XSPH.  Every kernel a kind needs runs over the
    # whole batch and must leave the other kinds untouched: each scene steps bit-identically
    # to itself alone (one thread per particle everywhere, so the summation orders match)
    one = dict(lanes_per_particle=1)
    ds = [scenes.dam_break_small(seed=4, n=(9, 11, 13), box=0.4, **one),
          scenes.dam_break_pcisph(seed=7, n=(9, 11, 13), box=0.4, **one),
          scenes.dam_break_wcsph(seed=7, n=(9, 11, 13), box=0.4, **one),
          scenes.body_in_fluid(rigid_coupling=1, density=200.0, **one),
          scenes.viscous_column(n=(8, 8, 16), plane_size=0.15, **one),
          scenes.dam_break_small(seed=6, n=(7, 9, 8), box=0.3, divergence_solve=0, warm_start=0,
                                 viscosity_mode=2, xsph_c=0.1, **one)]
    dt = 2e-4
    done = (sph.SPH_OK, sph.SPH_ENOCONVERGE)
    batch = gpu_ctx(ds)
    batch.sph_steps(5, dt)
    assert batch.sph_synchronize(raise_on_error=False) in done
    for k, d in enumerate(ds):
        single = gpu_ctx(d)
        single.sph_steps(5, dt)
        assert single.sph_synchronize(raise_on_error=False) in done
        for u, w in zip(batch.sph_read_state(k), single.sph_read_state()):
            np.testing.assert_array_equal(u, w, err_msg="scene %d" % k)
        np.testing.assert_array_equal(batch.sph_read_bodies(k), single.sph_read_bodies())
        bs, ss = batch.sph_get_stats(k), single.sph_get_stats()
        for key in ("total_dens_iters", "total_div_iters", "cg_iters"):
            assert bs[key] == ss[key], (k, key)


def test_checkpoint_resume_inside_a_batch():
    # the state of one scene of a batch (fluid, solver memory, bodies) written into the same
    # scene of a fresh batch context resumes it exactly, and the other scenes are untouched
    ds = [_small(seed=3, lanes_per_particle=1),
          scenes.body_in_fluid(rigid_coupling=1, density=200.0, lanes_per_particle=1)]
    a = gpu_ctx(ds)
    a.sph_steps(4, DT)
    a.sph_synchronize(raise_on_error=False)
    b = gpu_ctx(ds)
    x, v, _, _ = a.sph_read_state(1)
    b.sph_write_state(1, x, v, a.sph_read_field(sph.FIELD_KAPPA_PREV, 1), a.sph_read_field(sph.FIELD_KAPPA_V_PREV, 1))
    b.sph_write_bodies(1, a.sph_read_bodies(1))
    x0 = b.sph_read_state(0)[0].copy()
    np.testing.assert_array_equal(x0, ds[0]["fluid_x"])     # scene 0 still at its start
    for g in (a, b):
        g.sph_steps(2, DT)
        g.sph_synchronize(raise_on_error=False)
    for u, w in zip(a.sph_read_state(1), b.sph_read_state(1)):
        np.testing.assert_array_equal(u, w)
    np.testing.assert_array_equal(a.sph_read_bodies(1), b.sph_read_bodies(1))


def test_read_state_enqueued_into_host_memory():
    # on_device = 3: the read is only enqueued (unpermute on the context stream, copy on the
    # library's copy stream); once sph_read_wait says so, the page-locked host buffers hold
    # what the synchronous read returns.  Reads stay in flight across the next step: the
    # buffers of step k are checked after step k + 1 was enqueued (keep = 1 each step).
    import torch
    stream = torch.cuda.Stream()
    g = gpu_ctx(_small(), stream=stream)
    n = g.n_fluid[0]
    bufs = [(torch.full((n, 3), float("nan"), pin_memory=True), torch.full((n,), float("nan"), pin_memory=True))
            for _ in range(2)]
    ref = []
    with sph.Context(_small(), stream=torch.cuda.Stream()) as h:
        for _ in range(4):
            h.sph_step(DT)
            xs, _, rs, _ = h.sph_read_state()
            ref.append((xs, rs))
    for k in range(4):
        g.sph_step(DT)
        x, rho = bufs[k % 2]
        g.sph_read_state_host(0, x=x, rho=rho, sync=False)
        g.sph_read_wait(1)                            # step k - 1's read is on the host
        if k >= 1:
            xp, rp = bufs[(k - 1) % 2]
            np.testing.assert_array_equal(xp.numpy(), ref[k - 1][0])
            np.testing.assert_array_equal(rp.numpy(), ref[k - 1][1])
    g.sph_read_wait(0)
    np.testing.assert_array_equal(bufs[1][0].numpy(), ref[3][0])
    np.testing.assert_array_equal(bufs[1][1].numpy(), ref[3][1])
    # an unknown mode and a keep beyond the ring are refused
    st = sph.load().sph_read_state(g.ctx, 0, bufs[0][0].data_ptr(), None, None, None, 4)
    assert st == sph.SPH_EINVAL
    assert sph.load().sph_read_wait(g.ctx, 8) == sph.SPH_EINVAL
