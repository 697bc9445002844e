"""The C-ABI library builds, loads and exports every symbol include/sph.h declares, and
rejects malformed scene descriptors before touching the GPU (no compute calls here)."""
import os
import re

import numpy as np
import pytest

from paper_2403_11156_gb300 import build, scenes, sph

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return sph.load()


def _declared():
    text = open(os.path.join(ROOT, "include", "sph.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sph_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert "sph_create" in names and "sph_step" in names and "sph_read_state" in names
    for n in names:
        assert hasattr(lib, n), n
    assert lib.sph_abi_version() == 2


def test_status_strings(lib):
    for k in range(8):
        assert lib.sph_status_string(k)


def _bad(**kw):
    d = scenes.dam_break_small(n=(4, 4, 4), box=0.2)
    d.update(kw)
    return d


@pytest.mark.parametrize("kw", [
    dict(radius=0.0), dict(rest_density=-1.0), dict(domain_max=(0.0, 0.2, 0.2)),
    dict(min_iter_density=-1), dict(max_iter_divergence=-3), dict(viscosity_mode=7), dict(warm_start=9),
    dict(dt_max=0.0), dict(max_fluid_neighbors=5000), dict(cell_size=0.01),
    dict(lanes_per_particle=3), dict(lanes_per_particle=-1), dict(lanes_per_particle=16),
    dict(warm_start_fraction=1.5), dict(warm_start_fraction=-0.1), dict(learned_fraction=1.01),
    dict(learned_fraction=-1.0), dict(pressure_solver=3),
    dict(pressure_solver=1, eos_stiffness=0.0),
    dict(fluid_x=np.full((3, 3), np.nan, np.float32)),
    dict(fluid_x=np.zeros((0, 3), np.float32)),
])
def test_rejects_bad_descriptors(lib, kw):
    d = _bad(**kw)
    if "fluid_x" in kw:
        d["fluid_v"] = np.zeros_like(d["fluid_x"])
    with pytest.raises(sph.SphError) as e:
        sph.Context(d, torch_allocator=False)
    assert e.value.status == sph.SPH_EINVAL


@pytest.mark.parametrize("lanes", [0, 1, 2, 4, 8])
def test_accepts_good_descriptors(lib, lanes):
    # without a GPU a valid scene passes validation and fails at the first CUDA call
    import torch
    if torch.cuda.is_available():
        pytest.skip("host-only check")
    d = _bad(lanes_per_particle=lanes, max_fluid_neighbors=1024 if lanes == 4 else 0)
    with pytest.raises(sph.SphError) as e:
        sph.Context(d, torch_allocator=False)
    assert e.value.status == sph.SPH_ECUDA


def test_rejects_bad_body_index(lib):
    d = _bad()
    d["boundary_body"] = np.full(len(d["boundary_x"]), 3, np.int32)
    with pytest.raises(sph.SphError) as e:
        sph.Context(d, torch_allocator=False)
    assert e.value.status == sph.SPH_EINVAL


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(sph, "_lib", None)
    monkeypatch.setattr(sph, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(ImportError):
        sph.load()


def test_trace_kernel_ids_match_header():
    # the binding names trace entries by the header's SPH_KID_* values
    text = open(os.path.join(ROOT, "include", "sph.h")).read()
    ids = {int(v): k for k, v in re.findall(r"#define SPH_(KID_\w+) (\d+)", text)}
    assert sorted(ids) == list(range(1, len(ids) + 1))
    assert sorted(sph.KERNEL_IDS) == sorted(ids)
