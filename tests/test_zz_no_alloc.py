"""hydro_step_noalloc: the allocation-free entry point (needs a B300).

Callers that cannot allocate device memory (code running inside a pool or
arena it does not own, plugins whose host forbids cudaMalloc, real-time loops)
step a state they own, with scratch kept in a fixed array inside the library.
The test drives it through the C ABI on a caller-owned device buffer and
checks two calls in a row against the regular context API (hydro_create /
hydro_step): the state must be bit for bit the same in every precision and for
both reconstructions, WENO7 and WENO5 (the same kernels and arithmetic; this
entry point stages its tiles with plain loads where hydro_step uses TMA copies,
which move the same values).  This file is named so that pytest collects it
last.
"""
import ctypes
from dataclasses import replace

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1511_02137_b300 import build
    build.build()
    from paper_1511_02137_b300 import hydro, workloads
    lib = ctypes.CDLL(hydro.LIB_PATH)
    fn = lib.hydro_step_noalloc
    fn.argtypes = [ctypes.POINTER(hydro.hydro_config), ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                   ctypes.POINTER(ctypes.c_double), ctypes.c_int32, ctypes.POINTER(hydro.hydro_diag)]
    fn.restype = ctypes.c_int
    return torch, hydro, workloads, fn


def _rel(a, b):
    a = a.reshape(5, -1)
    b = b.reshape(5, -1)
    return np.abs(a - b).max(axis=1) / np.abs(b).max(axis=1)


@pytest.mark.parametrize("order", [7, 5])
@pytest.mark.parametrize("precision", ["fp64", "fp32", "mixed"])
def test_noalloc_matches_context_api_on_two_calls(env, precision, order):
    torch, hy, W, fn = env
    w = replace(W.ELLIPSOIDAL_32, n=(40, 36, 30), sigma=(0.9, 1.0, 1.1))   # 43200 cells, ragged tiles
    prim = W.ellipsoidal_primitives(w).ravel()
    cfg = hy.hydro_config_default(*w.n, precision=precision, weno_order=order)

    ref = hy.hydro_create(cfg)
    hy.hydro_set_initial(ref, hy.HYDRO_PRIMITIVE, prim)
    for j in w.jets:
        hy.hydro_add_jet(ref, j.x0, j.direction, j.t_start)
    U0 = hy.hydro_read_fields(ref, hy.HYDRO_CONSERVED)          # the initial conserved state

    dtype = torch.float32 if precision == "fp32" else torch.float64
    state = torch.from_numpy(U0.ravel()).to(device="cuda", dtype=dtype)   # caller-owned device buffer
    jets = np.array([[*j.x0, *j.direction, j.t_start] for j in w.jets], dtype=np.float64)
    c = hy.hydro_config.from_buffer_copy(cfg)
    c.cuda_stream = torch.cuda.current_stream().cuda_stream
    diag = hy.hydro_diag()
    jp = jets.ctypes.data_as(ctypes.POINTER(ctypes.c_double))

    for call, (step0, nsteps) in enumerate([(0, 2), (2, 3)]):
        hy.hydro_step(ref, nsteps)
        want = hy.hydro_read_fields(ref, hy.HYDRO_CONSERVED)
        rc = fn(ctypes.byref(c), state.data_ptr(), step0, nsteps, jp, len(jets), ctypes.byref(diag))
        assert rc == hy.HYDRO_OK, hy._lib().hydro_status_string(rc)
        got = state.double().cpu().numpy()   # FP32 widens exactly
        err = _rel(got, want)
        assert np.all(err <= TOL), (call, err)
        assert np.array_equal(got, want.ravel()), (call, "not bitwise equal", err)
        rd = hy.hydro_get_diag(ref)
        assert diag.steps == step0 + nsteps and diag.status == 0
        assert tuple(diag.jet_cell[0]) == rd["jet_cells"][0]
        assert abs(diag.max_speed - rd["max_speed"]) <= 1e-12
    hy.hydro_destroy(ref)


def test_noalloc_rejects_grids_above_the_fixed_scratch(env):
    torch, hy, W, fn = env
    cfg = hy.hydro_config_default(64, 64, 32)          # 131072 cells > HYDRO_NOALLOC_MAX_CELLS
    state = torch.zeros(5 * 64 * 64 * 32, dtype=torch.float64, device="cuda")
    rc = fn(ctypes.byref(cfg), state.data_ptr(), 0, 1, None, 0, None)
    assert rc == hy.HYDRO_ENOMEM
    rc = fn(ctypes.byref(cfg), None, 0, 1, None, 0, None)
    assert rc == hy.HYDRO_EINVAL


def test_noalloc_rejects_grids_beyond_the_launch_limits(env):
    """A 1 x 1 x 65536 grid fits the scratch array but not the sweeps' launch
    grid (z extent <= 65535): the configuration is invalid, as for hydro_create."""
    torch, hy, W, fn = env
    cfg = hy.hydro_config_default(1, 1, 65536)
    state = torch.zeros(5 * 65536, dtype=torch.float64, device="cuda")
    rc = fn(ctypes.byref(cfg), state.data_ptr(), 0, 1, None, 0, None)
    assert rc == hy.HYDRO_EINVAL
