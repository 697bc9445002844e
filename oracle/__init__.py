"""FP64 CPU oracle of the per-step DFSPH particle pipeline (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import this package.  It loads ``liboracle.so`` (built from ``dfsph_oracle.c`` by
:func:`build`) through ctypes and shares nothing with the CUDA library.

Parity unpinned: the absolute multi-step trajectories (splash shapes) of the dam-break
scenes; the paper prints no numeric example of them.  The per-step functions are pinned
by closed forms, invariants or brute force in ``tests/test_oracle_*.py``: among them the
DFSPH factor alpha (``test_oracle_alpha.py``: the lattice closed form, and one Jacobi
update cancelling a lone compression next to a wall exactly), the hydrostatic pressure
gradient within 5 % and the depth-independent buoyancy of a submerged body.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dfsph_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

# field ids (mirror the enum in dfsph_oracle.c)
X, V, RHO, ALPHA, KAPPA, KAPPA_V, PRESSURE, NN_F, NN_B = range(9)
V_DIV, V_NONP, PSI, XB, VB, KAPPA0, FEAT, DIV_ERR_I, DENS_ERR_I, FB_IMPULSE = range(9, 19)

STAT_NAMES = ["div_iters", "dens_iters", "div_err", "dens_err", "dt", "dt_next", "max_v",
              "clamps", "cg_iters", "cg_res", "div_err0", "dens_err0", "steps"]


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (FP64, no FMA contraction, OpenMP)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-fopenmp", _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [
        ("radius", C.c_double), ("rest_density", C.c_double), ("viscosity", C.c_double),
        ("gravity", C.c_double * 3),
        ("eta_density", C.c_double), ("eta_divergence", C.c_double),
        ("dt_max", C.c_double), ("cfl", C.c_double),
        ("min_iter_density", C.c_int32), ("max_iter_density", C.c_int32),
        ("min_iter_divergence", C.c_int32), ("max_iter_divergence", C.c_int32),
        ("viscosity_mode", C.c_int32), ("warm_start", C.c_int32),
        ("divergence_solve", C.c_int32),
        ("domain_min", C.c_float * 3), ("domain_max", C.c_float * 3),
        ("xsph_c", C.c_double), ("cg_tol", C.c_double),
        ("cg_max_iter", C.c_int32), ("pad_", C.c_int32),
        ("pressure_solver", C.c_int32), ("pad2_", C.c_int32),
        ("eos_stiffness", C.c_double), ("eos_exponent", C.c_double),
        ("warm_start_fraction", C.c_double),
        ("rigid_coupling", C.c_int32), ("pad3_", C.c_int32),
        ("learned_fraction", C.c_double),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        dp, fp, ip, up, lp = (C.POINTER(C.c_double), C.POINTER(C.c_float),
                              C.POINTER(C.c_int32), C.POINTER(C.c_uint32),
                              C.POINTER(C.c_int64))
        L.or_W.restype = C.c_double
        L.or_W.argtypes = [C.c_double, C.c_double]
        L.or_gradW.argtypes = [dp, C.c_double, dp]
        L.or_default_cell_size.restype = C.c_float
        L.or_default_cell_size.argtypes = [C.c_float]
        L.or_grid_dims.argtypes = [fp, fp, C.c_float, ip, fp]
        L.or_cell_keys.argtypes = [C.c_int64, fp, fp, fp, C.c_float, up]
        L.or_sort_order.argtypes = [C.c_int64, up, lp]
        L.or_neighbor_counts_brute.argtypes = [C.c_int64, fp, C.c_int64, fp, C.c_float,
                                               C.c_int, ip]
        L.or_mlp_nparam.restype = C.c_int64
        L.or_mlp_nweights.restype = C.c_int64
        L.or_mlp_forward.argtypes = [dp, C.c_int64, dp, dp]
        L.or_mlp_loss_grad.restype = C.c_double
        L.or_mlp_loss_grad.argtypes = [dp, C.c_int64, dp, dp, dp]
        L.or_adam_step.argtypes = [dp, dp, dp, dp, C.c_int64, C.c_int64, C.c_double,
                                   C.c_double, C.c_double, C.c_double]
        L.or_create.restype = C.c_void_p
        L.or_create.argtypes = [C.POINTER(Params), C.c_int64, fp, fp, C.c_int64, fp, ip,
                                C.c_int32, dp]
        L.or_destroy.argtypes = [C.c_void_p]
        L.or_set_mlp.argtypes = [C.c_void_p, dp]
        L.or_set_state.argtypes = [C.c_void_p, dp, dp, dp, dp]
        L.or_set_bodies.argtypes = [C.c_void_p, dp]
        L.or_step.argtypes = [C.c_void_p, C.c_double]
        L.or_field_width.restype = C.c_int64
        L.or_field_width.argtypes = [C.c_int32]
        L.or_get.restype = C.c_int64
        L.or_get.argtypes = [C.c_void_p, C.c_int32, dp]
        L.or_get_stats.argtypes = [C.c_void_p, dp]
        L.or_get_bodies.argtypes = [C.c_void_p, dp]
        L.or_visc_operator.argtypes = [C.c_void_p, C.c_double, dp, dp]
        L.or_prepare.argtypes = [C.c_void_p]
        L.or_pcisph_factor.argtypes = [C.c_void_p]
        L.or_pcisph_factor.restype = C.c_double
        L.or_visc_solve.restype = C.c_int32
        L.or_visc_solve.argtypes = [C.c_void_p, C.c_double, dp, dp]
        L.or_mass.restype = C.c_double
        L.or_mass.argtypes = [C.c_void_p]
        L.or_dt_next.restype = C.c_double
        L.or_dt_next.argtypes = [C.c_void_p]
        L.or_num_threads.restype = C.c_int32
        L.or_set_num_threads.argtypes = [C.c_int32]
        L.or_set_num_threads.restype = None
        _lib = L
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


# ---------------------------------------------------------------------------------- kernel
def W(r: float, h: float) -> float:
    return lib().or_W(float(r), float(h))


def gradW(x, h: float) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros(3)
    lib().or_gradW(_p(x, C.c_double), float(h), _p(out, C.c_double))
    return out


# ---------------------------------------------------------------------------- grid contract
def default_cell_size(radius: float) -> float:
    return float(lib().or_default_cell_size(C.c_float(radius)))


def grid_dims(dmin, dmax, cell):
    dmin = np.ascontiguousarray(dmin, dtype=np.float32)
    dmax = np.ascontiguousarray(dmax, dtype=np.float32)
    dims = np.zeros(3, dtype=np.int32)
    org = np.zeros(3, dtype=np.float32)
    lib().or_grid_dims(_p(dmin, C.c_float), _p(dmax, C.c_float), C.c_float(cell),
                       _p(dims, C.c_int32), _p(org, C.c_float))
    return dims, org


def cell_keys(x, dmin, dmax, cell) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1, 3)
    dmin = np.ascontiguousarray(dmin, dtype=np.float32)
    dmax = np.ascontiguousarray(dmax, dtype=np.float32)
    keys = np.zeros(len(x), dtype=np.uint32)
    lib().or_cell_keys(len(x), _p(x, C.c_float), _p(dmin, C.c_float), _p(dmax, C.c_float),
                       C.c_float(cell), _p(keys, C.c_uint32))
    return keys


def sort_order(keys) -> np.ndarray:
    keys = np.ascontiguousarray(keys, dtype=np.uint32)
    out = np.zeros(len(keys), dtype=np.int64)
    lib().or_sort_order(len(keys), _p(keys, C.c_uint32), _p(out, C.c_int64))
    return out


def neighbor_counts_brute(x, y, h, exclude_self: bool) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1, 3)
    y = np.ascontiguousarray(y, dtype=np.float32).reshape(-1, 3)
    out = np.zeros(len(x), dtype=np.int32)
    lib().or_neighbor_counts_brute(len(x), _p(x, C.c_float), len(y), _p(y, C.c_float),
                                   C.c_float(h), int(exclude_self), _p(out, C.c_int32))
    return out


# ------------------------------------------------------------------------------------- MLP
def mlp_nparam() -> int:
    return int(lib().or_mlp_nparam())


def mlp_nweights() -> int:
    return int(lib().or_mlp_nweights())


def mlp_forward(w, f) -> np.ndarray:
    w = np.ascontiguousarray(w, dtype=np.float64)
    f = np.ascontiguousarray(f, dtype=np.float64).reshape(-1, 4)
    y = np.zeros(len(f))
    lib().or_mlp_forward(_p(w, C.c_double), len(f), _p(f, C.c_double), _p(y, C.c_double))
    return y


def mlp_loss_grad(w, f, t):
    w = np.ascontiguousarray(w, dtype=np.float64)
    f = np.ascontiguousarray(f, dtype=np.float64).reshape(-1, 4)
    t = np.ascontiguousarray(t, dtype=np.float64)
    g = np.zeros(mlp_nweights())
    loss = lib().or_mlp_loss_grad(_p(w, C.c_double), len(f), _p(f, C.c_double),
                                  _p(t, C.c_double), _p(g, C.c_double))
    return loss, g


def adam_step(w, m, v, g, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """In place on float64 arrays w, m, v."""
    lib().or_adam_step(_p(w, C.c_double), _p(m, C.c_double), _p(v, C.c_double),
                       _p(np.ascontiguousarray(g, dtype=np.float64), C.c_double), len(w),
                       int(t), lr, b1, b2, eps)


def num_threads() -> int:
    return int(lib().or_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the oracle's parallel loops from now on (timing only)."""
    lib().or_set_num_threads(int(n))


# ----------------------------------------------------------------------------------- scene
class Scene:
    """One oracle scene.  ``desc`` is a dict produced by ``paper_2403_11156_gb300.scenes``."""

    def __init__(self, desc: dict):
        L = lib()
        p = Params()
        p.radius = desc["radius"]
        p.rest_density = desc["rest_density"]
        p.viscosity = desc["viscosity"]
        for a in range(3):
            p.gravity[a] = desc["gravity"][a]
            p.domain_min[a] = desc["domain_min"][a]
            p.domain_max[a] = desc["domain_max"][a]
        p.eta_density = desc["eta_density"]
        p.eta_divergence = desc["eta_divergence"]
        p.dt_max = desc["dt_max"]
        p.cfl = desc["cfl"]
        p.min_iter_density = desc["min_iter_density"]
        p.max_iter_density = desc["max_iter_density"]
        p.min_iter_divergence = desc["min_iter_divergence"]
        p.max_iter_divergence = desc["max_iter_divergence"]
        p.viscosity_mode = desc["viscosity_mode"]
        p.warm_start = desc["warm_start"]
        p.divergence_solve = desc["divergence_solve"]
        p.xsph_c = desc.get("xsph_c", 0.0)
        p.cg_tol = desc.get("cg_tol", 1e-4)
        p.cg_max_iter = desc.get("cg_max_iter", 500)
        p.pressure_solver = desc.get("pressure_solver", 0)
        p.eos_stiffness = desc.get("eos_stiffness", 0.0)
        p.eos_exponent = desc.get("eos_exponent", 7.0)
        p.warm_start_fraction = desc.get("warm_start_fraction", 0.0)
        p.learned_fraction = desc.get("learned_fraction", 0.0)
        p.rigid_coupling = desc.get("rigid_coupling", 0)
        self.params = p
        self.nf = len(desc["fluid_x"])
        self.nb = len(desc["boundary_x"])
        self.nbody = len(desc.get("bodies", []))
        self._keep = []
        xf = np.ascontiguousarray(desc["fluid_x"], dtype=np.float32)
        vf = np.ascontiguousarray(desc["fluid_v"], dtype=np.float32)
        xb = np.ascontiguousarray(desc["boundary_x"], dtype=np.float32).reshape(-1, 3)
        body = np.ascontiguousarray(desc.get("boundary_body", np.full(self.nb, -1)),
                                    dtype=np.int32)
        bodies = np.zeros((max(self.nbody, 1), 19))
        for k, b in enumerate(desc.get("bodies", [])):
            bodies[k, 0] = b["mass"]
            bodies[k, 1:4] = b["inertia"]
            bodies[k, 4:7] = b["com"]
            bodies[k, 7:11] = b["quat"]
            bodies[k, 11:14] = b["vel"]
            bodies[k, 14:17] = b["omega"]
        self._keep += [xf, vf, xb, body, bodies]
        self.ptr = L.or_create(C.byref(p), self.nf, _p(xf, C.c_float), _p(vf, C.c_float),
                               self.nb, _p(xb, C.c_float), _p(body, C.c_int32), self.nbody,
                               _p(bodies, C.c_double))

    def __del__(self):
        if getattr(self, "ptr", None):
            lib().or_destroy(self.ptr)
            self.ptr = None

    def step(self, dt: float = 0.0):
        lib().or_step(self.ptr, float(dt))

    def get(self, field: int) -> np.ndarray:
        L = lib()
        w = L.or_field_width(field)
        n = self.nb if field in (PSI, XB, VB) else self.nf
        out = np.zeros(n * w)
        L.or_get(self.ptr, field, _p(out, C.c_double))
        return out.reshape(n, w) if w > 1 else out

    def stats(self) -> dict:
        out = np.zeros(16)
        lib().or_get_stats(self.ptr, _p(out, C.c_double))
        return {k: float(out[i]) for i, k in enumerate(STAT_NAMES)}

    def bodies(self) -> np.ndarray:
        out = np.zeros((max(self.nbody, 1), 19))
        lib().or_get_bodies(self.ptr, _p(out, C.c_double))
        return out[: self.nbody]

    def set_state(self, x=None, v=None, kappa_prev=None, kappa_v_prev=None):
        def arr(a, n):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
            assert a.size == n
            self._keep.append(a)
            return _p(a, C.c_double)
        lib().or_set_state(self.ptr, arr(x, 3 * self.nf), arr(v, 3 * self.nf),
                           arr(kappa_prev, self.nf), arr(kappa_v_prev, self.nf))

    def set_bodies(self, bodies):
        """Rigid state from rows of bodies()'s layout (com, quat, vel, omega; the force and
        torque columns are ignored)."""
        b = np.ascontiguousarray(bodies, dtype=np.float64).reshape(-1, 19)
        assert len(b) == self.nbody
        self._keep.append(b)
        lib().or_set_bodies(self.ptr, _p(b, C.c_double))

    def set_mlp(self, params):
        params = np.ascontiguousarray(params, dtype=np.float64)
        assert params.size == mlp_nparam()
        self._keep.append(params)
        lib().or_set_mlp(self.ptr, _p(params, C.c_double))

    def visc_operator(self, dt: float, v) -> np.ndarray:
        v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1)
        out = np.zeros_like(v)
        lib().or_visc_operator(self.ptr, float(dt), _p(v, C.c_double), _p(out, C.c_double))
        return out.reshape(-1, 3)

    def pcisph_factor(self) -> float:
        """PCISPH prototype stiffness delta dt^2 (Pa per kg/m^3 times s^2)."""
        return float(lib().or_pcisph_factor(self.ptr))

    def prepare(self):
        """Neighbour lists, boundary pseudo-masses, density and alpha for the current
        positions, without advancing the state."""
        lib().or_prepare(self.ptr)

    def visc_solve(self, dt: float, b):
        b = np.ascontiguousarray(b, dtype=np.float64).reshape(-1)
        x = np.zeros_like(b)
        it = lib().or_visc_solve(self.ptr, float(dt), _p(b, C.c_double), _p(x, C.c_double))
        return x.reshape(-1, 3), int(it)

    @property
    def mass(self) -> float:
        return float(lib().or_mass(self.ptr))

    @property
    def dt_next(self) -> float:
        return float(lib().or_dt_next(self.ptr))
