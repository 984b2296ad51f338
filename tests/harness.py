"""Shared test helpers: run a workload through the CUDA library and the oracle.

The CUDA side goes through the C ABI binding (paper_1511_02137_b300.hydro);
the oracle side through oracle/.  Both start from the same seeded primitive
fields of paper_1511_02137_b300.workloads.
"""
from __future__ import annotations

import numpy as np


def norm_rel_err(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Per field: max |a - b| / max |b| (b is the oracle)."""
    a = a.reshape(5, -1)
    b = b.reshape(5, -1)
    den = np.maximum(np.abs(b).max(axis=1), 1e-300)
    return np.abs(a - b).max(axis=1) / den


def oracle_config(orc, w, boundary="outflow", order=7, eps=1e-6):
    return orc.Config(w.n[0], w.n[1], w.n[2], dx=w.dx, dt=w.dt, t0=w.t0, boundary=boundary, order=order,
                      weno_eps=eps)


def oracle_jets(orc, w):
    return [orc.Jet(j.x0, j.direction, j.t_start) for j in w.jets]


def gpu_context(hy, w, precision="fp64", boundary="outflow", order=7, eps=1e-6, prim=None, **cfg_over):
    from paper_1511_02137_b300 import workloads
    cfg = hy.hydro_config_default(w.n[0], w.n[1], w.n[2], precision=precision, boundary=boundary,
                                  weno_order=order, dx=w.dx, dt=w.dt, t0=w.t0, weno_eps=eps, **cfg_over)
    ctx = hy.hydro_create(cfg)
    if prim is None:
        prim = workloads.ellipsoidal_primitives(w)
    hy.hydro_set_initial(ctx, hy.HYDRO_PRIMITIVE, np.ascontiguousarray(prim, dtype=np.float64).ravel())
    for j in w.jets:
        hy.hydro_add_jet(ctx, j.x0, j.direction, j.t_start)
    return ctx


def cone_mask(n, dx, apex, axis=(1.0, 0.0, 0.0), half_angle_deg=30.0, rmax=3.0):
    """Cells [nz, ny, nx] whose centres lie in the cone of the adjoint's
    observable: within rmax of the apex and within half_angle_deg of the axis
    (centre of cell i at (i + 1/2 - n/2) dx on each axis)."""
    import math
    nx, ny, nz = n
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    x = (np.arange(nx) + 0.5 - nx / 2) * dx - apex[0]
    y = (np.arange(ny) + 0.5 - ny / 2) * dx - apex[1]
    z = (np.arange(nz) + 0.5 - nz / 2) * dx - apex[2]
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    r2 = X * X + Y * Y + Z * Z
    along = a[0] * X + a[1] * Y + a[2] * Z
    return (r2 < rmax * rmax) & (along >= math.cos(math.radians(half_angle_deg)) * np.sqrt(r2))
