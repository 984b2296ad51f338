"""Python binding of the C ABI in include/hydro.h (argument marshalling only).

Every function keeps the C name.  Device memory for the field store comes from
PyTorch's CUDA caching allocator (one workspace tensor per context) and the
device work runs on PyTorch's current CUDA stream unless another is given; all
arithmetic runs in the CUDA kernels of ``libhydro.so``.  There is no CPU path:
importing this module fails if the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# HYDRO_CHECKED=1 in the environment selects the bounds-checked build of the same
# library (build.build_checked(); tests only: it reports failed checks as HYDRO_ECHECK)
LIB_PATH = os.path.join(_HERE, "libhydro_check.so" if os.environ.get("HYDRO_CHECKED") == "1" else "libhydro.so")

(HYDRO_OK, HYDRO_EINVAL, HYDRO_ENOMEM, HYDRO_ECUDA, HYDRO_EUNPHYSICAL, HYDRO_ECFL, HYDRO_ETIMEOUT, HYDRO_ESTATE,
 HYDRO_ECHECK) = range(9)
HYDRO_FP64, HYDRO_FP32, HYDRO_MIXED = 0, 1, 2
HYDRO_OUTFLOW, HYDRO_PERIODIC = 0, 1
HYDRO_PRIMITIVE, HYDRO_CONSERVED = 0, 1
HYDRO_KERNEL_SWEEP_X, HYDRO_KERNEL_SWEEP_Y, HYDRO_KERNEL_SWEEP_Z, HYDRO_KERNEL_OTHER = 0, 1, 2, 3
HYDRO_MAX_JETS = 16
(HYDRO_MATH_RCP, HYDRO_MATH_SQRT_RSQRT, HYDRO_MATH_C2P_FP64, HYDRO_MATH_C2P_FP32, HYDRO_MATH_C2P_MIXED,
 HYDRO_MATH_D2F, HYDRO_MATH_F2D) = range(7)
HYDRO_PEAK_FFMA, HYDRO_PEAK_FFMA2, HYDRO_PEAK_DFMA = range(3)
PRECISIONS = {"fp64": HYDRO_FP64, "fp32": HYDRO_FP32, "mixed": HYDRO_MIXED}


class hydro_config(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("boundary", ctypes.c_int32), ("weno_order", ctypes.c_int32),
                ("dx", ctypes.c_double), ("dt", ctypes.c_double), ("t0", ctypes.c_double),
                ("k_rad", ctypes.c_double), ("k_coll", ctypes.c_double), ("cr_over_cf", ctypes.c_double),
                ("hbarc", ctypes.c_double), ("dof", ctypes.c_double), ("e_floor", ctypes.c_double),
                ("weno_eps", ctypes.c_double), ("cfl_limit", ctypes.c_double),
                ("cuda_stream", ctypes.c_void_p), ("workspace", ctypes.c_void_p),
                ("workspace_bytes", ctypes.c_size_t), ("wait_limit_s", ctypes.c_double),
                ("test_withhold_copies", ctypes.c_int32), ("test_check_tighten", ctypes.c_int32)]


class hydro_diag(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("steps", ctypes.c_int64), ("max_speed", ctypes.c_double),
                ("floor_hits", ctypes.c_int64), ("dep_E", ctypes.c_double), ("dep_M", ctypes.c_double * 3),
                ("njet", ctypes.c_int32), ("jet_cell", (ctypes.c_int32 * 3) * HYDRO_MAX_JETS),
                ("status", ctypes.c_int32), ("check_site", ctypes.c_int32), ("check_index", ctypes.c_uint32)]


class HydroError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {_lib().hydro_status_string(status).decode()}")


_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_1511_02137_b300.build`")
        lib = ctypes.CDLL(LIB_PATH)
        P = ctypes.POINTER
        vp, dp = ctypes.c_void_p, P(ctypes.c_double)
        lib.hydro_config_default.argtypes = [P(hydro_config), ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
        lib.hydro_config_default.restype = None
        lib.hydro_workspace_size.argtypes = [P(hydro_config), P(ctypes.c_size_t)]
        lib.hydro_create.argtypes = [P(hydro_config), P(vp)]
        lib.hydro_set_initial.argtypes = [vp, ctypes.c_int32, vp]
        lib.hydro_add_jet.argtypes = [vp, dp, dp, ctypes.c_double, P(ctypes.c_int32)]
        lib.hydro_step.argtypes = [vp, ctypes.c_int32]
        lib.hydro_read_fields.argtypes = [vp, ctypes.c_int32, vp]
        lib.hydro_get_diag.argtypes = [vp, P(hydro_diag)]
        lib.hydro_profile_enable.argtypes = [vp, ctypes.c_int32]
        lib.hydro_profile_query.argtypes = [vp, ctypes.c_int32, dp, P(ctypes.c_int64)]
        lib.hydro_destroy.argtypes = [vp]
        lib.hydro_destroy.restype = None
        lib.hydro_status_string.argtypes = [ctypes.c_int]
        lib.hydro_status_string.restype = ctypes.c_char_p
        i32p = P(ctypes.c_int32)
        lib.hydro_batch_workspace_size.argtypes = [P(hydro_config), ctypes.c_int32, i32p, P(ctypes.c_size_t)]
        lib.hydro_batch_create.argtypes = [P(hydro_config), ctypes.c_int32, i32p, P(vp)]
        lib.hydro_batch_set_initial.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, vp]
        lib.hydro_batch_add_jet.argtypes = [vp, ctypes.c_int32, dp, dp, ctypes.c_double, i32p]
        lib.hydro_batch_set_tiles.argtypes = [vp, i32p]
        lib.hydro_batch_autotune.argtypes = [vp, i32p, dp]
        lib.hydro_batch_set_launch.argtypes = [vp, i32p]
        lib.hydro_batch_get_tuning.argtypes = [vp, i32p, i32p]
        lib.hydro_batch_step.argtypes = [vp, ctypes.c_int32]
        lib.hydro_batch_read_fields.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, vp]
        lib.hydro_batch_get_diag.argtypes = [vp, ctypes.c_int32, P(hydro_diag)]
        lib.hydro_batch_destroy.argtypes = [vp]
        lib.hydro_batch_destroy.restype = None
        lib.hydro_adjoint_workspace_size.argtypes = [P(hydro_config), ctypes.c_int32, ctypes.c_int32,
                                                     P(ctypes.c_size_t)]
        lib.hydro_adjoint_create.argtypes = [P(hydro_config), ctypes.c_int32, ctypes.c_int32, dp, dp, ctypes.c_double,
                                             ctypes.c_double, P(vp)]
        lib.hydro_eval_math.argtypes = [ctypes.c_int32, ctypes.c_int64, vp, vp, ctypes.c_double, vp]
        lib.hydro_alu_peak.argtypes = [ctypes.c_int32, ctypes.c_int64, vp, dp, dp]
        lib.hydro_adjoint_add_jet.argtypes = [vp, dp, dp, ctypes.c_double]
        lib.hydro_adjoint_set_params.argtypes = [vp, ctypes.c_double, ctypes.c_double]
        lib.hydro_adjoint_forward.argtypes = [vp, vp, dp]
        lib.hydro_adjoint_backward.argtypes = [vp, ctypes.c_double, dp, dp, vp]
        lib.hydro_adjoint_destroy.argtypes = [vp]
        lib.hydro_adjoint_destroy.restype = None
        for name in ("hydro_adjoint_workspace_size", "hydro_adjoint_create", "hydro_adjoint_add_jet",
                     "hydro_adjoint_set_params", "hydro_adjoint_forward", "hydro_adjoint_backward",
                     "hydro_eval_math", "hydro_alu_peak"):
            getattr(lib, name).restype = ctypes.c_int
        for name in ("hydro_workspace_size", "hydro_create", "hydro_set_initial", "hydro_add_jet", "hydro_step",
                     "hydro_read_fields", "hydro_get_diag", "hydro_profile_enable", "hydro_profile_query",
                     "hydro_batch_workspace_size", "hydro_batch_create", "hydro_batch_set_initial",
                     "hydro_batch_add_jet", "hydro_batch_set_tiles", "hydro_batch_autotune", "hydro_batch_step",
                     "hydro_batch_set_launch", "hydro_batch_get_tuning",
                     "hydro_batch_read_fields", "hydro_batch_get_diag"):
            getattr(lib, name).restype = ctypes.c_int
        _LIB = lib
    return _LIB


def _check(status: int, where: str, allow=()):
    if status != HYDRO_OK and status not in allow:
        raise HydroError(status, where)
    return status


class Context:
    """Opaque hydro_ctx plus the torch workspace tensor that backs it."""

    def __init__(self, handle, cfg, workspace):
        self.handle = handle
        self.cfg = cfg
        self.workspace = workspace
        self.cells = cfg.nx * cfg.ny * cfg.nz

    @property
    def device(self):
        """The CUDA device of the workspace (field buffers may be tensors on it)."""
        return None if self.workspace is None else self.workspace.device

    def __del__(self):
        if getattr(self, "handle", None):
            hydro_destroy(self)


def hydro_config_default(nx: int, ny: int, nz: int, **overrides) -> hydro_config:
    cfg = hydro_config()
    _lib().hydro_config_default(ctypes.byref(cfg), nx, ny, nz)
    for k, v in overrides.items():
        if k == "precision" and isinstance(v, str):
            v = PRECISIONS[v]
        if k == "boundary" and isinstance(v, str):
            v = {"outflow": HYDRO_OUTFLOW, "periodic": HYDRO_PERIODIC}[v]
        setattr(cfg, k, v)
    return cfg


def hydro_workspace_size(cfg: hydro_config) -> int:
    n = ctypes.c_size_t()
    _check(_lib().hydro_workspace_size(ctypes.byref(cfg), ctypes.byref(n)), "hydro_workspace_size")
    return n.value


def hydro_create(cfg: hydro_config, device=None, stream=None) -> Context:
    """Creates a context whose workspace is a torch CUDA tensor and whose stream
    is torch's current stream on `device` (or `stream` if given)."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    nbytes = hydro_workspace_size(cfg)
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
    base = ws.data_ptr()
    aligned = (base + 255) // 256 * 256
    c = hydro_config.from_buffer_copy(cfg)
    c.workspace = aligned
    c.workspace_bytes = nbytes
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    c.cuda_stream = s.cuda_stream
    h = ctypes.c_void_p()
    _check(_lib().hydro_create(ctypes.byref(c), ctypes.byref(h)), "hydro_create")
    ctx = Context(h, c, ws)
    ctx.stream = s
    return ctx


def _host_ptr(buf, n: int, writable: bool, device=None):
    """Address of a field buffer: a numpy array or CPU tensor, or (where the
    call takes one, `device` set) a CUDA tensor on that device."""
    if isinstance(buf, np.ndarray):
        if buf.dtype != np.float64 or not buf.flags.c_contiguous or buf.size != n:
            raise ValueError(f"expected a C-contiguous float64 array of {n} values")
        if writable and not buf.flags.writeable:
            raise ValueError("output array is read-only")
        return buf.ctypes.data
    import torch
    if isinstance(buf, torch.Tensor):
        if buf.device.type == "cuda" and device is not None:
            if buf.device != device:
                raise ValueError(f"expected a tensor on {device}, got one on {buf.device}")
        elif buf.device.type != "cpu":
            raise ValueError("expected a CPU tensor")
        if buf.dtype != torch.float64 or not buf.is_contiguous() or buf.numel() != n:
            raise ValueError(f"expected a contiguous float64 tensor of {n} values")
        return buf.data_ptr()
    raise TypeError("field buffer must be a numpy array or a torch tensor")


def hydro_set_initial(ctx: Context, kind: int, host5) -> None:
    """host5: numpy array, CPU tensor or CUDA tensor on the context's device."""
    _check(_lib().hydro_set_initial(ctx.handle, kind, _host_ptr(host5, 5 * ctx.cells, False, ctx.device)),
           "hydro_set_initial")


def hydro_add_jet(ctx: Context, x0, direction, t_start: float) -> int:
    a = (ctypes.c_double * 3)(*x0)
    d = (ctypes.c_double * 3)(*direction)
    jid = ctypes.c_int32()
    _check(_lib().hydro_add_jet(ctx.handle, a, d, t_start, ctypes.byref(jid)), "hydro_add_jet")
    return jid.value


def hydro_step(ctx: Context, nsteps: int, allow=()) -> int:
    return _check(_lib().hydro_step(ctx.handle, nsteps), "hydro_step", allow)


def hydro_read_fields(ctx: Context, kind: int = HYDRO_CONSERVED, out=None):
    if out is None:
        out = np.empty((5, ctx.cfg.nz, ctx.cfg.ny, ctx.cfg.nx), dtype=np.float64)
    _check(_lib().hydro_read_fields(ctx.handle, kind, _host_ptr(out, 5 * ctx.cells, True, ctx.device)),
           "hydro_read_fields")
    return out


def hydro_get_diag(ctx: Context) -> dict:
    d = hydro_diag()
    _check(_lib().hydro_get_diag(ctx.handle, ctypes.byref(d)), "hydro_get_diag")
    return {"t": d.t, "steps": d.steps, "max_speed": d.max_speed, "floor_hits": d.floor_hits,
            "dep_E": d.dep_E, "dep_M": tuple(d.dep_M), "njet": d.njet,
            "jet_cells": [tuple(d.jet_cell[i]) for i in range(d.njet)], "status": d.status,
            "check_site": d.check_site, "check_index": d.check_index}


def hydro_profile_enable(ctx: Context, on: bool = True) -> None:
    _check(_lib().hydro_profile_enable(ctx.handle, 1 if on else 0), "hydro_profile_enable")


def hydro_profile_query(ctx: Context, kind: int):
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    _check(_lib().hydro_profile_query(ctx.handle, kind, ctypes.byref(ms), ctypes.byref(n)), "hydro_profile_query")
    return ms.value, n.value


def hydro_destroy(ctx: Context) -> None:
    if ctx.handle:
        _lib().hydro_destroy(ctx.handle)
        ctx.handle = None


# ---------------------------------------------------------------- batched ensembles


class Batch:
    """Opaque hydro_batch plus the torch workspace tensor that backs it."""

    def __init__(self, handle, cfg, dims, workspace):
        self.handle = handle
        self.cfg = cfg
        self.dims = [tuple(int(v) for v in d) for d in dims]
        self.workspace = workspace
        self.cells = [d[0] * d[1] * d[2] for d in self.dims]

    @property
    def device(self):
        return None if self.workspace is None else self.workspace.device

    def __del__(self):
        if getattr(self, "handle", None):
            hydro_batch_destroy(self)


def _dims_array(dims):
    flat = [int(v) for d in dims for v in d]
    return (ctypes.c_int32 * len(flat))(*flat), len(dims)


def hydro_batch_workspace_size(cfg: hydro_config, dims) -> int:
    arr, n = _dims_array(dims)
    size = ctypes.c_size_t()
    _check(_lib().hydro_batch_workspace_size(ctypes.byref(cfg), n, arr, ctypes.byref(size)),
           "hydro_batch_workspace_size")
    return size.value


def hydro_batch_create(cfg: hydro_config, dims, device=None, stream=None) -> Batch:
    """Creates a batch over grids `dims` [(nx, ny, nz), ...] with a torch CUDA
    workspace; `stream` (default: torch's current stream) is the one the calls
    order themselves after."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    nbytes = hydro_batch_workspace_size(cfg, dims)
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
    c = hydro_config.from_buffer_copy(cfg)
    c.workspace = (ws.data_ptr() + 255) // 256 * 256
    c.workspace_bytes = nbytes
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    c.cuda_stream = s.cuda_stream
    arr, n = _dims_array(dims)
    h = ctypes.c_void_p()
    _check(_lib().hydro_batch_create(ctypes.byref(c), n, arr, ctypes.byref(h)), "hydro_batch_create")
    return Batch(h, c, dims, ws)


def hydro_batch_set_initial(b: Batch, event: int, kind: int, host5) -> None:
    ptr = _host_ptr(host5, 5 * b.cells[event], False, b.device)
    _check(_lib().hydro_batch_set_initial(b.handle, event, kind, ptr), "hydro_batch_set_initial")


def hydro_batch_add_jet(b: Batch, event: int, x0, direction, t_start: float) -> int:
    a = (ctypes.c_double * 3)(*x0)
    d = (ctypes.c_double * 3)(*direction)
    jid = ctypes.c_int32()
    _check(_lib().hydro_batch_add_jet(b.handle, event, a, d, t_start, ctypes.byref(jid)), "hydro_batch_add_jet")
    return jid.value


def hydro_batch_set_tiles(b: Batch, variants) -> None:
    v = (ctypes.c_int32 * 3)(*variants)
    _check(_lib().hydro_batch_set_tiles(b.handle, v), "hydro_batch_set_tiles")


def hydro_batch_set_launch(b: Batch, per_tile) -> None:
    v = (ctypes.c_int32 * 3)(*per_tile)
    _check(_lib().hydro_batch_set_launch(b.handle, v), "hydro_batch_set_launch")


def hydro_batch_get_tuning(b: Batch):
    """(tile shape per axis, launch form per axis: 1 one block per tile, 0 persistent)."""
    v = (ctypes.c_int32 * 3)()
    m = (ctypes.c_int32 * 3)()
    _check(_lib().hydro_batch_get_tuning(b.handle, v, m), "hydro_batch_get_tuning")
    return tuple(v), tuple(m)


def hydro_batch_autotune(b: Batch):
    """Returns (chosen tile shape per axis, 3x3 launch times in ms [axis][shape])."""
    v = (ctypes.c_int32 * 3)()
    ms = (ctypes.c_double * 9)()
    _check(_lib().hydro_batch_autotune(b.handle, v, ms), "hydro_batch_autotune")
    return tuple(v), [[ms[3 * d + k] for k in range(3)] for d in range(3)]


def hydro_batch_step(b: Batch, nsteps: int, allow=()) -> int:
    return _check(_lib().hydro_batch_step(b.handle, nsteps), "hydro_batch_step", allow)


def hydro_batch_read_fields(b: Batch, event: int, kind: int = HYDRO_CONSERVED, out=None):
    nx, ny, nz = b.dims[event]
    if out is None:
        out = np.empty((5, nz, ny, nx), dtype=np.float64)
    ptr = _host_ptr(out, 5 * b.cells[event], True, b.device)
    _check(_lib().hydro_batch_read_fields(b.handle, event, kind, ptr), "hydro_batch_read_fields")
    return out


def hydro_batch_get_diag(b: Batch, event: int) -> dict:
    d = hydro_diag()
    _check(_lib().hydro_batch_get_diag(b.handle, event, ctypes.byref(d)), "hydro_batch_get_diag")
    return {"t": d.t, "steps": d.steps, "max_speed": d.max_speed, "floor_hits": d.floor_hits,
            "dep_E": d.dep_E, "dep_M": tuple(d.dep_M), "njet": d.njet,
            "jet_cells": [tuple(d.jet_cell[i]) for i in range(d.njet)], "status": d.status,
            "check_site": d.check_site, "check_index": d.check_index}


def hydro_batch_destroy(b: Batch) -> None:
    if b.handle:
        _lib().hydro_batch_destroy(b.handle)
        b.handle = None


# ---------------------------------------------------------------- adjoint


class Adjoint:
    """Opaque hydro_adjoint handle plus the torch workspace tensor that backs it."""

    def __init__(self, handle, cfg, nsteps, every, workspace=None):
        self.handle = handle
        self.cfg = cfg
        self.nsteps = nsteps
        self.every = every
        self.workspace = workspace
        self.cells = cfg.nx * cfg.ny * cfg.nz

    def __del__(self):
        if getattr(self, "handle", None):
            hydro_adjoint_destroy(self)


def hydro_adjoint_workspace_size(cfg: hydro_config, nsteps: int, checkpoint_every: int) -> int:
    n = ctypes.c_size_t()
    _check(_lib().hydro_adjoint_workspace_size(ctypes.byref(cfg), nsteps, checkpoint_every, ctypes.byref(n)),
           "hydro_adjoint_workspace_size")
    return n.value


def hydro_adjoint_create(cfg: hydro_config, nsteps: int, checkpoint_every: int, apex, axis,
                         half_angle_deg: float, rmax: float, device=None, stream=None) -> Adjoint:
    """Creates an adjoint run whose buffers are one torch CUDA tensor (PyTorch's
    caching allocator) and whose stream is torch's current stream."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    nbytes = hydro_adjoint_workspace_size(cfg, nsteps, checkpoint_every)
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
    c = hydro_config.from_buffer_copy(cfg)
    c.workspace = (ws.data_ptr() + 255) // 256 * 256
    c.workspace_bytes = nbytes
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    c.cuda_stream = s.cuda_stream
    h = ctypes.c_void_p()
    _check(_lib().hydro_adjoint_create(ctypes.byref(c), nsteps, checkpoint_every, (ctypes.c_double * 3)(*apex),
                                       (ctypes.c_double * 3)(*axis), half_angle_deg, rmax, ctypes.byref(h)),
           "hydro_adjoint_create")
    return Adjoint(h, c, nsteps, checkpoint_every, ws)


def hydro_adjoint_add_jet(a: Adjoint, x0, direction, t_start: float) -> None:
    _check(_lib().hydro_adjoint_add_jet(a.handle, (ctypes.c_double * 3)(*x0), (ctypes.c_double * 3)(*direction),
                                        t_start), "hydro_adjoint_add_jet")


def hydro_adjoint_set_params(a: Adjoint, k_rad: float, k_coll: float) -> None:
    _check(_lib().hydro_adjoint_set_params(a.handle, k_rad, k_coll), "hydro_adjoint_set_params")


def hydro_adjoint_forward(a: Adjoint, prim_dev) -> float:
    """prim_dev: contiguous float64 CUDA tensor of 5*cells values (e, u^x, u^y, u^z, n)."""
    if prim_dev.dtype.itemsize != 8 or not prim_dev.is_cuda or not prim_dev.is_contiguous() \
            or prim_dev.numel() != 5 * a.cells:
        raise ValueError("expected a contiguous float64 CUDA tensor of 5*cells values")
    J = ctypes.c_double()
    _check(_lib().hydro_adjoint_forward(a.handle, prim_dev.data_ptr(), ctypes.byref(J)), "hydro_adjoint_forward")
    return J.value


def hydro_adjoint_backward(a: Adjoint, dJ: float, grad_e_dev):
    """Returns (dJ/dk_rad, dJ/dk_coll); writes dJ/de into grad_e_dev (float64 CUDA, cells values)."""
    if not grad_e_dev.is_cuda or not grad_e_dev.is_contiguous() or grad_e_dev.numel() != a.cells:
        raise ValueError("expected a contiguous float64 CUDA tensor of cells values")
    gr = ctypes.c_double()
    gc = ctypes.c_double()
    _check(_lib().hydro_adjoint_backward(a.handle, dJ, ctypes.byref(gr), ctypes.byref(gc), grad_e_dev.data_ptr()),
           "hydro_adjoint_backward")
    return gr.value, gc.value


def hydro_adjoint_destroy(a: Adjoint) -> None:
    if a.handle:
        _lib().hydro_adjoint_destroy(a.handle)
        a.handle = None


# ---------------------------------------------------------------- arithmetic checks and peaks


def hydro_eval_math(fn: int, x_dev, param: float = 0.0, stream=None):
    """Evaluates device routine `fn` (HYDRO_MATH_*) over the CUDA tensor x_dev
    (float64: n values, or 4n for the recoveries; float32 for HYDRO_MATH_F2D);
    returns the output tensor (n, 2n or 5n float64 values; n float32 values for
    HYDRO_MATH_D2F)."""
    import torch
    want = torch.float32 if fn == HYDRO_MATH_F2D else torch.float64
    if x_dev.dtype != want or not x_dev.is_cuda or not x_dev.is_contiguous():
        raise ValueError(f"expected a contiguous {want} CUDA tensor")
    if fn in (HYDRO_MATH_D2F, HYDRO_MATH_F2D):
        n = x_dev.numel()
        out = torch.empty(n, dtype=torch.float32 if fn == HYDRO_MATH_D2F else torch.float64, device=x_dev.device)
    elif fn in (HYDRO_MATH_RCP, HYDRO_MATH_SQRT_RSQRT):
        n = x_dev.numel()
        out = torch.empty(n * (1 if fn == HYDRO_MATH_RCP else 2), dtype=torch.float64, device=x_dev.device)
    else:
        if x_dev.numel() % 4:
            raise ValueError("the recoveries take (E, Mx, My, Mz) as 4 arrays of n values")
        n = x_dev.numel() // 4
        out = torch.empty(5 * n, dtype=torch.float64, device=x_dev.device)
    s = stream if stream is not None else torch.cuda.current_stream(x_dev.device)
    _check(_lib().hydro_eval_math(fn, n, x_dev.data_ptr(), out.data_ptr(), param, s.cuda_stream), "hydro_eval_math")
    return out


def hydro_alu_peak(kind: int, iters: int, stream=None):
    """(FLOPs, ms) of one FMA-throughput launch (HYDRO_PEAK_*) on the current device."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    flop = ctypes.c_double()
    ms = ctypes.c_double()
    _check(_lib().hydro_alu_peak(kind, iters, s.cuda_stream, ctypes.byref(flop), ctypes.byref(ms)), "hydro_alu_peak")
    return flop.value, ms.value
