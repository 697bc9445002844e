"""Thin ctypes binding of the C ABI in include/sph.h (argument marshalling only).

Every function here has the C function's name and forwards to libsph.so; all compute
runs in that library's CUDA kernels.  There is no CPU fallback: loading fails loudly when
the library is missing, and the calls fail when no GPU is present.  PyTorch, when
available, provides device memory (its caching allocator is passed to sph_create) and
streams.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsph.so")

SPH_OK, SPH_EINVAL, SPH_ENOMEM, SPH_ECUDA, SPH_ENOCONVERGE, SPH_ETIMEOUT, SPH_ENUMERIC, \
    SPH_EOVERFLOW = range(8)
STATUS_NAMES = ["SPH_OK", "SPH_EINVAL", "SPH_ENOMEM", "SPH_ECUDA", "SPH_ENOCONVERGE",
                "SPH_ETIMEOUT", "SPH_ENUMERIC", "SPH_EOVERFLOW"]

FIELD_RHO, FIELD_ALPHA, FIELD_KAPPA, FIELD_KAPPA_V, FIELD_NN_FLUID, FIELD_NN_BOUNDARY, \
    FIELD_V_DIV, FIELD_KAPPA_PREV, FIELD_KAPPA_V_PREV, FIELD_CELL_KEY, FIELD_SORTED_ID, \
    FIELD_PSI, FIELD_BOUNDARY_SORTED_ID, FIELD_BOUNDARY_CELL_KEY, FIELD_FEATURES, \
    FIELD_KAPPA0 = range(16)

# (dtype, width, boundary?) of each field
FIELD_LAYOUT = {
    FIELD_RHO: (np.float32, 1, False), FIELD_ALPHA: (np.float32, 1, False),
    FIELD_KAPPA: (np.float32, 1, False), FIELD_KAPPA_V: (np.float32, 1, False),
    FIELD_NN_FLUID: (np.int32, 1, False), FIELD_NN_BOUNDARY: (np.int32, 1, False),
    FIELD_V_DIV: (np.float32, 3, False), FIELD_KAPPA_PREV: (np.float32, 1, False),
    FIELD_KAPPA_V_PREV: (np.float32, 1, False), FIELD_CELL_KEY: (np.uint32, 1, False),
    FIELD_SORTED_ID: (np.int32, 1, False), FIELD_PSI: (np.float32, 1, True),
    FIELD_BOUNDARY_SORTED_ID: (np.int32, 1, True), FIELD_BOUNDARY_CELL_KEY: (np.uint32, 1, True),
    FIELD_FEATURES: (np.float32, 4, False), FIELD_KAPPA0: (np.float32, 1, False),
}


KERNEL_IDS = {i + 1: n for i, n in enumerate([
    "step_begin", "key_hist_fluid", "key_hist_boundary", "scan", "scatter_fluid", "scatter_boundary",
    "rank_gather_fluid", "rank_gather_boundary", "density_alpha", "div_pass_a", "dens_pass_a",
    "div_pass_b", "dens_pass_b", "div_warm_pass_b", "dens_warm_pass_b", "nonpressure", "warm_density",
    "advect", "step_end", "set_dt", "boundary_update", "boundary_psi", "body_force", "body_reduce",
    "cg_init", "cg_ap", "cg_xr", "cg_p", "mlp_warm", "body_force_inc", "body_apply",
    "boundary_vel", "div_check", "dens_check", "cg_alpha", "cg_beta", "body_touch",
    "rank_large_fluid", "rank_large_boundary"])}


class SphError(RuntimeError):
    def __init__(self, status, msg):
        self.status = status
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < 8 else status, msg))


class RigidDesc(C.Structure):
    _fields_ = [("mass", C.c_double), ("inertia", C.c_double * 3), ("com", C.c_double * 3),
                ("quat", C.c_double * 4), ("vel", C.c_double * 3), ("omega", C.c_double * 3)]


class SceneDesc(C.Structure):
    _fields_ = [
        ("n_fluid", C.c_int64), ("fluid_x", C.POINTER(C.c_float)),
        ("fluid_v", C.POINTER(C.c_float)),
        ("n_boundary", C.c_int64), ("boundary_x", C.POINTER(C.c_float)),
        ("boundary_body", C.POINTER(C.c_int32)),
        ("n_bodies", C.c_int32), ("bodies", C.POINTER(RigidDesc)),
        ("radius", C.c_float), ("rest_density", C.c_float), ("viscosity", C.c_float),
        ("xsph_c", C.c_float), ("gravity", C.c_float * 3),
        ("domain_min", C.c_float * 3), ("domain_max", C.c_float * 3),
        ("cell_size", C.c_float), ("eta_density", C.c_float), ("eta_divergence", C.c_float),
        ("dt_max", C.c_float), ("cfl", C.c_float),
        ("min_iter_density", C.c_int32), ("max_iter_density", C.c_int32),
        ("min_iter_divergence", C.c_int32), ("max_iter_divergence", C.c_int32),
        ("viscosity_mode", C.c_int32), ("warm_start", C.c_int32),
        ("divergence_solve", C.c_int32), ("max_fluid_neighbors", C.c_int32),
        ("max_boundary_neighbors", C.c_int32), ("cg_tol", C.c_float), ("cg_max_iter", C.c_int32),
        ("lanes_per_particle", C.c_int32), ("pressure_solver", C.c_int32),
        ("eos_stiffness", C.c_float), ("eos_exponent", C.c_float),
        ("warm_start_fraction", C.c_float), ("rigid_coupling", C.c_int32),
        ("learned_fraction", C.c_float), ("learned_gate", C.c_int32),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("steps", C.c_int64), ("div_iters", C.c_int32), ("dens_iters", C.c_int32),
        ("div_err", C.c_double), ("dens_err", C.c_double), ("div_err0", C.c_double),
        ("dens_err0", C.c_double), ("dt", C.c_float), ("dt_next", C.c_float),
        ("max_speed", C.c_float), ("max_fluid_nbrs", C.c_int32),
        ("max_boundary_nbrs", C.c_int32), ("cg_iters", C.c_int32), ("cg_residual", C.c_float),
        ("clamps", C.c_int32), ("flags", C.c_int32), ("total_div_iters", C.c_int64),
        ("total_dens_iters", C.c_int64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Tuning(C.Structure):
    _fields_ = [("tuned", C.c_int32), ("from_cache", C.c_int32), ("gather_batch", C.c_int32),
                ("cell_factor", C.c_float), ("n_trials", C.c_int32),
                ("trial_cell_factor", C.c_float * 8), ("trial_batch", C.c_int32 * 8),
                ("trial_ms", C.c_float * 8), ("lanes", C.c_int32), ("trial_lanes", C.c_int32 * 8)]

    def as_dict(self):
        n = self.n_trials
        return {"tuned": self.tuned, "from_cache": self.from_cache, "gather_batch": self.gather_batch,
                "cell_factor": self.cell_factor, "lanes": self.lanes,
                "trials": [{"cell_factor": self.trial_cell_factor[k], "gather_batch": self.trial_batch[k],
                            "lanes": self.trial_lanes[k], "ms_per_step": self.trial_ms[k]}
                           for k in range(n)]}


class KernelTime(C.Structure):
    _fields_ = [("name", C.c_char * 64), ("launches", C.c_int64), ("total_ms", C.c_double)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)


class Allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", C.c_void_p)]


_lib = None


def load():
    """Load libsph.so (built by paper_2403_11156_gb300.build); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libsph.so not built (%s); run __graft_entry__.build()" % LIB_PATH)
    L = C.CDLL(LIB_PATH)
    vp, ip, fp, dp = C.c_void_p, C.c_int32, C.POINTER(C.c_float), C.POINTER(C.c_double)
    L.sph_abi_version.restype = C.c_int32
    L.sph_create.argtypes = [C.POINTER(SceneDesc), C.POINTER(Allocator), vp, C.POINTER(vp)]
    L.sph_create_batch.argtypes = [C.POINTER(SceneDesc), ip, C.POINTER(Allocator), vp, C.POINTER(vp)]
    L.sph_step.argtypes = [vp, C.c_float]
    L.sph_steps.argtypes = [vp, ip, C.c_float]
    L.sph_synchronize.argtypes = [vp]
    L.sph_read_state.argtypes = [vp, ip, vp, vp, vp, vp, ip]
    L.sph_write_state.argtypes = [vp, ip, vp, vp, vp, vp, ip]
    L.sph_probe_wait_timeout.argtypes = [vp, ip]
    L.sph_read_field.argtypes = [vp, ip, ip, vp, ip]
    L.sph_get_stats.argtypes = [vp, ip, C.POINTER(Stats)]
    L.sph_read_bodies.argtypes = [vp, ip, dp]
    L.sph_write_bodies.argtypes = [vp, ip, dp]
    L.sph_set_mode.argtypes = [vp, ip, ip]
    L.sph_kernel_times.argtypes = [vp, C.POINTER(KernelTime), ip, C.POINTER(C.c_int32), ip]
    L.sph_launch_count.argtypes = [vp, C.POINTER(C.c_int64)]
    L.sph_status_string.restype = C.c_char_p
    L.sph_status_string.argtypes = [ip]
    L.sph_last_error.restype = C.c_char_p
    L.sph_last_error.argtypes = [vp]
    L.sph_destroy.argtypes = [vp]
    L.sph_grid_order_noalloc.argtypes = [vp, C.c_int64, fp, fp, C.c_float, vp, vp, vp]
    L.sph_grid_order_noalloc_status.argtypes = [vp]
    L.sph_read_wait.argtypes = [vp, ip]
    L.sph_set_mlp.argtypes = [vp, fp, C.c_int64]
    L.sph_get_tuning.argtypes = [vp, C.POINTER(Tuning)]
    L.sph_set_trace.argtypes = [vp, ip]
    L.sph_read_trace.argtypes = [vp, vp, ip, C.POINTER(C.c_int32), ip]
    L.sph_mlp_forward.argtypes = [vp, vp, C.c_int64, vp, vp, vp]
    L.sph_mlp_grad.argtypes = [vp, vp, vp, C.c_int64, vp, vp, vp, vp]
    L.sph_mlp_train.argtypes = [vp, vp, C.c_int64, vp, vp, ip, ip, C.c_float, C.c_uint64, vp, vp, vp]
    L.sph_surface_field.argtypes = [vp, ip, fp, C.c_float, C.POINTER(C.c_int32), vp]
    L.sph_surface_mesh.argtypes = [vp, C.POINTER(C.c_int32), fp, C.c_float, C.c_float, vp, C.c_int64,
                                   C.POINTER(C.c_int64), vp]
    L.sph_render_heightmap.argtypes = [vp, ip, fp, fp, ip, ip, C.c_float, vp]
    for name in ("sph_create", "sph_create_batch", "sph_step", "sph_steps", "sph_synchronize",
                 "sph_read_state", "sph_write_state", "sph_read_field", "sph_get_stats", "sph_probe_wait_timeout",
                 "sph_read_bodies", "sph_set_mode", "sph_kernel_times", "sph_launch_count",
                 "sph_grid_order_noalloc", "sph_grid_order_noalloc_status", "sph_read_wait", "sph_set_mlp", "sph_mlp_forward", "sph_mlp_grad", "sph_mlp_train", "sph_get_tuning", "sph_set_trace",
                 "sph_read_trace", "sph_surface_field", "sph_surface_mesh", "sph_render_heightmap"):
        getattr(L, name).restype = C.c_int32
    _lib = L
    return L


def _check(ctx, status):
    if status != SPH_OK:
        msg = load().sph_last_error(ctx).decode() if ctx else ""
        raise SphError(status, msg)
    return status


def _fptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


class _TorchAllocator:
    """Routes the library's device allocations through torch's caching allocator."""

    def __init__(self):
        import torch
        self.torch = torch

        def _alloc(user, nbytes, stream):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), stream=stream or 0)
            except Exception:
                return None

        def _free(user, ptr, nbytes, stream):
            torch.cuda.caching_allocator_delete(ptr)

        self._a = ALLOC_FN(_alloc)
        self._f = FREE_FN(_free)
        self.struct = Allocator(self._a, self._f, None)


def _make_desc(d, keep):
    fx = np.ascontiguousarray(d["fluid_x"], dtype=np.float32).reshape(-1, 3)
    fv = np.ascontiguousarray(d.get("fluid_v", np.zeros_like(fx)), dtype=np.float32).reshape(-1, 3)
    bx = np.ascontiguousarray(d.get("boundary_x", np.zeros((0, 3))), dtype=np.float32).reshape(-1, 3)
    bb = np.ascontiguousarray(d.get("boundary_body", np.full(len(bx), -1)), dtype=np.int32)
    bodies = d.get("bodies", [])
    rb = (RigidDesc * max(len(bodies), 1))()
    for k, b in enumerate(bodies):
        rb[k].mass = b["mass"]
        for a in range(3):
            rb[k].inertia[a] = b["inertia"][a]
            rb[k].com[a] = b["com"][a]
            rb[k].vel[a] = b["vel"][a]
            rb[k].omega[a] = b["omega"][a]
        for a in range(4):
            rb[k].quat[a] = b["quat"][a]
    keep += [fx, fv, bx, bb, rb]
    s = SceneDesc()
    s.n_fluid = len(fx)
    s.fluid_x = _fptr(fx)
    s.fluid_v = _fptr(fv)
    s.n_boundary = len(bx)
    s.boundary_x = _fptr(bx)
    s.boundary_body = bb.ctypes.data_as(C.POINTER(C.c_int32))
    s.n_bodies = len(bodies)
    s.bodies = C.cast(rb, C.POINTER(RigidDesc))
    s.radius = d["radius"]
    s.rest_density = d["rest_density"]
    s.viscosity = d["viscosity"]
    s.xsph_c = d.get("xsph_c", 0.0)
    for a in range(3):
        s.gravity[a] = d["gravity"][a]
        s.domain_min[a] = d["domain_min"][a]
        s.domain_max[a] = d["domain_max"][a]
    s.cell_size = d.get("cell_size", 0.0)
    s.eta_density = d["eta_density"]
    s.eta_divergence = d["eta_divergence"]
    s.dt_max = d["dt_max"]
    s.cfl = d["cfl"]
    s.min_iter_density = d["min_iter_density"]
    s.max_iter_density = d["max_iter_density"]
    s.min_iter_divergence = d["min_iter_divergence"]
    s.max_iter_divergence = d["max_iter_divergence"]
    s.viscosity_mode = d["viscosity_mode"]
    s.warm_start = d["warm_start"]
    s.divergence_solve = d["divergence_solve"]
    s.max_fluid_neighbors = d.get("max_fluid_neighbors", 0)
    s.max_boundary_neighbors = d.get("max_boundary_neighbors", 0)
    s.cg_tol = d.get("cg_tol", 1e-4)
    s.cg_max_iter = d.get("cg_max_iter", 500)
    s.lanes_per_particle = d.get("lanes_per_particle", 0)
    s.pressure_solver = d.get("pressure_solver", 0)
    s.eos_stiffness = d.get("eos_stiffness", 0.0)
    s.eos_exponent = d.get("eos_exponent", 7.0)
    s.warm_start_fraction = d.get("warm_start_fraction", 0.0)
    s.learned_fraction = d.get("learned_fraction", 0.0)
    s.learned_gate = d.get("learned_gate", 0)
    s.rigid_coupling = d.get("rigid_coupling", 0)
    return s


class Context:
    """Owns one sph_ctx (one or several scenes).  Scene dicts come from ``scenes``."""

    def __init__(self, scene_descs, stream=None, torch_allocator=True, autotune=False):
        L = load()
        if isinstance(scene_descs, dict):
            scene_descs = [scene_descs]
        self.descs = list(scene_descs)
        if autotune:
            self.descs = [dict(d, cell_size=-1.0) for d in self.descs]
        self._keep = []
        arr = (SceneDesc * len(self.descs))()
        for k, d in enumerate(self.descs):
            arr[k] = _make_desc(d, self._keep)
        self._alloc = _TorchAllocator() if torch_allocator else None
        handle = C.c_void_p()
        st_ptr = None
        if stream is not None:
            st_ptr = C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        self.stream = stream
        status = L.sph_create_batch(arr, len(self.descs),
                                    C.byref(self._alloc.struct) if self._alloc else None,
                                    st_ptr, C.byref(handle))
        if status != SPH_OK:
            raise SphError(status, "sph_create failed")
        self.ctx = handle.value
        self.n_fluid = [len(d["fluid_x"]) for d in self.descs]
        self.n_boundary = [len(d.get("boundary_x", [])) for d in self.descs]

    # --------------------------------------------------------------------------- lifecycle
    def close(self):
        if getattr(self, "ctx", None):
            load().sph_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ------------------------------------------------------------------------------- calls
    def sph_step(self, dt=0.0):
        return _check(self.ctx, load().sph_step(self.ctx, float(dt)))

    def sph_steps(self, n, dt=0.0):
        return _check(self.ctx, load().sph_steps(self.ctx, int(n), float(dt)))

    def sph_synchronize(self, raise_on_error=True):
        st = load().sph_synchronize(self.ctx)
        if raise_on_error:
            _check(self.ctx, st)
        return st

    def sph_read_state(self, scene=0):
        n = self.n_fluid[scene]
        x = np.zeros((n, 3), np.float32)
        v = np.zeros((n, 3), np.float32)
        rho = np.zeros(n, np.float32)
        p = np.zeros(n, np.float32)
        _check(self.ctx, load().sph_read_state(self.ctx, scene, x.ctypes.data, v.ctypes.data,
                                               rho.ctypes.data, p.ctypes.data, 0))
        return x, v, rho, p

    def sph_read_state_device(self, scene, x=None, v=None, rho=None, pressure=None, sync=True):
        """Write into caller-owned device buffers (torch tensors or raw pointers); with
        sync=False the copy is only enqueued on the context's stream."""
        def ptr(t):
            return None if t is None else (t.data_ptr() if hasattr(t, "data_ptr") else int(t))
        _check(self.ctx, load().sph_read_state(self.ctx, scene, ptr(x), ptr(v), ptr(rho),
                                               ptr(pressure), 1 if sync else 2))

    def sph_read_wait(self, keep=0):
        """Wait until at most `keep` enqueued host reads are still in flight."""
        _check(self.ctx, load().sph_read_wait(self.ctx, int(keep)))

    def sph_read_state_host(self, scene, x=None, v=None, rho=None, pressure=None, sync=True):
        """Write into caller-owned host buffers (page-locked torch CPU tensors, numpy arrays
        or raw pointers); with sync=False the read is only enqueued (on_device = 3) and its
        data is there once sph_read_wait says so."""
        def ptr(t):
            if t is None:
                return None
            if hasattr(t, "data_ptr"):
                return t.data_ptr()
            return t.ctypes.data if hasattr(t, "ctypes") else int(t)
        _check(self.ctx, load().sph_read_state(self.ctx, scene, ptr(x), ptr(v), ptr(rho),
                                               ptr(pressure), 0 if sync else 3))

    def sph_write_state(self, scene=0, x=None, v=None, kappa_prev=None, kappa_v_prev=None):
        def arr(a, shape):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=np.float32).reshape(shape)
            self._keep.append(a)
            return a.ctypes.data
        n = self.n_fluid[scene]
        _check(self.ctx, load().sph_write_state(self.ctx, scene, arr(x, (n, 3)), arr(v, (n, 3)),
                                                arr(kappa_prev, (n,)), arr(kappa_v_prev, (n,)), 0))

    def sph_read_field_device(self, field, out, scene=0):
        """Write a per-particle field into a caller-owned device buffer (tensor or pointer)."""
        _check(self.ctx, load().sph_read_field(self.ctx, scene, field, _dptr(out), 1))
        return out

    def sph_read_field(self, field, scene=0):
        dt, w, boundary = FIELD_LAYOUT[field]
        n = self.n_boundary[scene] if boundary else self.n_fluid[scene]
        out = np.zeros((n, w) if w > 1 else n, dtype=dt)
        _check(self.ctx, load().sph_read_field(self.ctx, scene, field, out.ctypes.data, 0))
        return out

    def sph_get_stats(self, scene=0):
        s = Stats()
        _check(self.ctx, load().sph_get_stats(self.ctx, scene, C.byref(s)))
        return s.as_dict()

    def sph_read_bodies(self, scene=0):
        nb = len(self.descs[scene].get("bodies", []))
        out = np.zeros((max(nb, 1), 19))
        _check(self.ctx, load().sph_read_bodies(self.ctx, scene,
                                                out.ctypes.data_as(C.POINTER(C.c_double))))
        return out[:nb]

    def sph_write_bodies(self, scene, bodies):
        """Rigid state from rows of sph_read_bodies' layout (com, quat, vel, omega; the
        force and torque columns are ignored)."""
        nb = len(self.descs[scene].get("bodies", []))
        b = np.ascontiguousarray(bodies, dtype=np.float64).reshape(-1, 19)
        if len(b) != nb:
            raise ValueError("scene %d has %d bodies, got %d rows" % (scene, nb, len(b)))
        _check(self.ctx, load().sph_write_bodies(self.ctx, scene,
                                                 b.ctypes.data_as(C.POINTER(C.c_double))))

    def sph_probe_wait_timeout(self, spin_limit=1000):
        """Enqueue a bounded wait that runs out (the device error path); returns the status
        of the enqueue, the next synchronize reports SPH_ETIMEOUT."""
        return load().sph_probe_wait_timeout(self.ctx, int(spin_limit))

    def sph_set_mode(self, graph=True, timing=False):
        _check(self.ctx, load().sph_set_mode(self.ctx, int(graph), int(timing)))

    def sph_kernel_times(self, reset=False):
        cap = 128
        arr = (KernelTime * cap)()
        n = C.c_int32()
        _check(self.ctx, load().sph_kernel_times(self.ctx, arr, cap, C.byref(n), int(reset)))
        return {arr[k].name.decode(): (arr[k].launches, arr[k].total_ms) for k in range(min(n.value, cap))}

    def sph_set_mlp(self, params):
        a = np.ascontiguousarray(params, dtype=np.float32)
        _check(self.ctx, load().sph_set_mlp(self.ctx, _fptr(a), a.size))

    def sph_get_tuning(self):
        t = Tuning()
        _check(self.ctx, load().sph_get_tuning(self.ctx, C.byref(t)))
        return t.as_dict()

    def sph_set_trace(self, capacity):
        _check(self.ctx, load().sph_set_trace(self.ctx, int(capacity)))

    def sph_read_trace(self, cap=1 << 20, reset=True):
        """Returns (kernel names, start times in ns) of the traced launches in order."""
        buf = np.zeros(cap, dtype=np.uint64)
        n = C.c_int32()
        _check(self.ctx, load().sph_read_trace(self.ctx, buf.ctypes.data, cap, C.byref(n), int(reset)))
        k = min(n.value, cap)
        raw = buf[:k]
        return [KERNEL_IDS.get(int(r & 0xFF), "?") for r in raw], (raw >> np.uint64(8)).astype(np.int64)

    def sph_launch_count(self):
        n = C.c_int64()
        _check(self.ctx, load().sph_launch_count(self.ctx, C.byref(n)))
        return n.value

    def sph_surface_field(self, origin, spacing, dims, scene=0, out=None):
        """Volume-fraction field on the grid (device tensor [dims[2]][dims[1]][dims[0]])."""
        import torch
        dims = [int(d) for d in dims]
        if out is None:
            out = torch.empty((dims[2], dims[1], dims[0]), dtype=torch.float32, device="cuda")
        o = (C.c_float * 3)(*origin)
        d = (C.c_int32 * 3)(*dims)
        _check(self.ctx, load().sph_surface_field(self.ctx, scene, o, float(spacing), d, out.data_ptr()))
        return out

    def sph_render_heightmap(self, lo, hi, width, height, radius, scene=0, out=None):
        """Height map viewed down -z (device tensor [height][width], NaN where empty)."""
        import torch
        if out is None:
            out = torch.empty((int(height), int(width)), dtype=torch.float32, device="cuda")
        a, b = (C.c_float * 2)(*lo), (C.c_float * 2)(*hi)
        _check(self.ctx, load().sph_render_heightmap(self.ctx, scene, a, b, int(width), int(height),
                                                     float(radius), out.data_ptr()))
        return out


NOALLOC_MAX_POINTS = 262144
NOALLOC_MAX_CELLS = 1048576


def sph_grid_order_noalloc(x, n, domain_min, domain_max, cell_size, order, keys=None, stream=None):
    """Marshal sph_grid_order_noalloc: x, order, keys are device pointers (ints or tensors
    with data_ptr()); domain bounds are 3-sequences; returns the status code."""
    def ptr(t):
        return None if t is None else (t.data_ptr() if hasattr(t, "data_ptr") else int(t))
    lo = (C.c_float * 3)(*domain_min)
    hi = (C.c_float * 3)(*domain_max)
    st = None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    return load().sph_grid_order_noalloc(ptr(x), int(n), lo, hi, float(cell_size), ptr(order),
                                         ptr(keys), st)


def sph_grid_order_noalloc_status(stream=None):
    """Marshal sph_grid_order_noalloc_status: SPH_OK once the last call's work on `stream`
    completed with its prefix scan, SPH_ETIMEOUT if a wait of that scan ran out."""
    st = None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    return load().sph_grid_order_noalloc_status(st)


def sph_surface_mesh(field, origin, spacing, iso=0.5, cap=None, stream=None):
    """Marshal sph_surface_mesh on a device field tensor [nz][ny][nx]: returns the device
    tensor of triangles [n][3][3] (grown and rerun once if the first capacity is short)."""
    import torch
    nz, ny, nx = (int(d) for d in field.shape)
    dims = (C.c_int32 * 3)(nx, ny, nz)
    o = (C.c_float * 3)(*origin)
    st = None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    if st is None:
        st = torch.cuda.current_stream().cuda_stream
    cap = int(cap) if cap is not None else max(1024, 4 * nx * ny)
    for _ in range(2):
        tris = torch.empty((cap, 3, 3), dtype=torch.float32, device=field.device)
        n = C.c_int64()
        status = load().sph_surface_mesh(field.data_ptr(), dims, o, float(spacing), float(iso),
                                          tris.data_ptr(), cap, C.byref(n), st)
        if status == SPH_EOVERFLOW:
            cap = int(n.value)
            continue
        _check(None, status)
        return tris[:n.value]
    raise SphError(SPH_EOVERFLOW, "triangle count changed between runs")


MLP_PARAMS = 4555
MLP_WEIGHTS = 4545


def sph_mlp_forward(params, features, n, y, error, stream=None):
    """Marshal sph_mlp_forward: device pointers (ints or tensors); returns the status."""
    def ptr(t):
        return None if t is None else (t.data_ptr() if hasattr(t, "data_ptr") else int(t))
    st = None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    return load().sph_mlp_forward(ptr(params), ptr(features), int(n), ptr(y), ptr(error), st)


def _dptr(t):
    return None if t is None else (t.data_ptr() if hasattr(t, "data_ptr") else int(t))


def _sptr(stream):
    return None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def sph_mlp_grad(params, features, labels, n, grad, loss, error, stream=None):
    """Marshal sph_mlp_grad (device pointers or tensors); returns the status."""
    return load().sph_mlp_grad(_dptr(params), _dptr(features), _dptr(labels), int(n), _dptr(grad),
                               _dptr(loss), _dptr(error), _sptr(stream))


def sph_mlp_train(features, labels, n, params, adam_state, epochs, batch, lr, seed, loss_history,
                  error, stream=None):
    """Marshal sph_mlp_train (device pointers or tensors); returns the status."""
    return load().sph_mlp_train(_dptr(features), _dptr(labels), int(n), _dptr(params),
                                _dptr(adam_state), int(epochs), int(batch), float(lr), int(seed),
                                _dptr(loss_history), _dptr(error), _sptr(stream))
