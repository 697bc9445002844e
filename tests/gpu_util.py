"""Helpers shared by the GPU tests: run the CUDA path and the oracle on the same seeded
scene and compare (the comparison rules are the tolerances stated in the tests)."""
import numpy as np

import oracle
from paper_2403_11156_gb300 import build, sph


def gpu_ctx(descs, **kw):
    build.build()
    return sph.Context(descs, **kw)


def forced(desc, div_iters, dens_iters):
    """Same scene with the iteration counts of both solves fixed (parity protocol: a count
    can flip near the tolerance, so fields are compared at equal counts)."""
    d = dict(desc)
    d.update(min_iter_divergence=div_iters, max_iter_divergence=div_iters,
             min_iter_density=dens_iters, max_iter_density=dens_iters)
    return d


def rel_err(gpu, ref, floor):
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    return np.abs(gpu - ref) / np.maximum(np.abs(ref), floor)


def assert_rel(gpu, ref, rtol, floor_frac=1e-3, floor=None, what=""):
    ref = np.asarray(ref, np.float64)
    if floor is None:
        rms = float(np.sqrt(np.mean(ref ** 2))) if ref.size else 0.0
        floor = max(floor_frac * rms, 1e-30)
    e = rel_err(gpu, ref, floor)
    worst = int(np.argmax(e)) if e.size else 0
    assert e.size == 0 or e.max() <= rtol, (
        "%s: max rel err %.3e > %.1e at %d (gpu %r ref %r, floor %.3e)"
        % (what, e.max(), rtol, worst, np.ravel(gpu)[worst], np.ravel(ref)[worst], floor))
    return float(e.max()) if e.size else 0.0


def oracle_step(desc, dt, steps=1):
    o = oracle.Scene(desc)
    for _ in range(steps):
        o.step(dt)
    return o


def field_tolerances(o, d, dt):
    """Per-particle scales of the one-step field comparison: kappa against alpha rho0 / dt^2
    (a 1e-5 rho0 error in rho*), velocities against the change such an error implies."""
    alpha = o.get(oracle.ALPHA)
    rho = o.get(oracle.RHO)
    rho0 = d["rest_density"]
    k_scale = alpha * rho0 / dt ** 2
    v_tol = 1e-5 * rho0 * np.sqrt(np.maximum(alpha, 0) / rho) / dt
    return k_scale, v_tol


def assert_abs(gpu, ref, tol, what):
    """Every row of gpu within its per-particle tol (plus 1e-5 of the row's magnitude)."""
    gpu = np.asarray(gpu, np.float64).reshape(len(tol), -1)
    ref = np.asarray(ref, np.float64).reshape(len(tol), -1)
    e = np.abs(gpu - ref).max(axis=1) / (tol + 1e-5 * np.abs(ref).max(axis=1) + 1e-30)
    k = int(np.argmax(e))
    assert e.max() <= 1.0, "%s: worst %.3g of tolerance at %d (gpu %r ref %r tol %.3g)" % (
        what, e.max(), k, gpu[k], ref[k], tol[k])
