"""Checkpoint and resume through the C ABI (needs a B300): the conserved fields
read with hydro_read_fields, loaded into a new context with
hydro_set_initial(HYDRO_CONSERVED) whose t0 is the checkpoint's time, continue
the run.  Without jets the time enters nowhere and the resumed run equals the
uninterrupted one bit for bit, in every precision (FP32 storage widens to FP64
and back exactly; the mixed path's FP32 shadow is rebuilt from the FP64 state
by the same rounding the step uses).  With a jet the stage times are
t0' + (n' + c_k) dt instead of t0 + (n + c_k) dt, equal up to the rounding of
the sum, so the deposits agree to that rounding and the jet cells exactly."""
from dataclasses import replace

import numpy as np
import pytest

from harness import gpu_context, norm_rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hy():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1511_02137_b300 import build
    build.build()
    from paper_1511_02137_b300 import hydro
    return hydro


@pytest.fixture(scope="module")
def W():
    from paper_1511_02137_b300 import workloads
    return workloads


def _resume(hy, w, precision, first, second):
    """`first` steps, a checkpoint of the conserved fields, and `second` steps
    in a new context that starts from it at the checkpoint's time."""
    ctx = gpu_context(hy, w, precision)
    hy.hydro_step(ctx, first)
    U = hy.hydro_read_fields(ctx, hy.HYDRO_CONSERVED)
    d1 = hy.hydro_get_diag(ctx)
    cfg = hy.hydro_config_default(*w.n, precision=precision, dx=w.dx, dt=w.dt, t0=w.t0 + first * w.dt,
                                  weno_eps=1e-6)
    ctx2 = hy.hydro_create(cfg)
    hy.hydro_set_initial(ctx2, hy.HYDRO_CONSERVED, U.ravel())
    for j in w.jets:
        hy.hydro_add_jet(ctx2, j.x0, j.direction, j.t_start)
    hy.hydro_step(ctx2, second)
    return hy.hydro_read_fields(ctx2, hy.HYDRO_CONSERVED), d1, hy.hydro_get_diag(ctx2)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "mixed"])
def test_resume_without_jets_is_bitwise(hy, W, precision):
    w = replace(W.ELLIPSOIDAL_32, n=(36, 30, 28), jets=())
    ref = gpu_context(hy, w, precision)
    hy.hydro_step(ref, 7)
    want = hy.hydro_read_fields(ref, hy.HYDRO_CONSERVED)
    got, _, _ = _resume(hy, w, precision, 3, 4)
    assert np.array_equal(got, want), norm_rel_err(got, want)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("fp32", 1e-6), ("mixed", 1e-6)])
def test_resume_with_a_jet_matches_to_the_rounding_of_the_stage_times(hy, W, precision, tol):
    w = replace(W.ELLIPSOIDAL_32, n=(36, 30, 28))
    ref = gpu_context(hy, w, precision)
    hy.hydro_step(ref, 7)
    want = hy.hydro_read_fields(ref, hy.HYDRO_CONSERVED)
    dref = hy.hydro_get_diag(ref)
    got, d1, d2 = _resume(hy, w, precision, 3, 4)
    err = norm_rel_err(got, want)
    assert np.all(err <= tol), err
    assert d2["jet_cells"] == dref["jet_cells"]
    assert abs((d1["dep_E"] + d2["dep_E"]) / dref["dep_E"] - 1) <= max(tol, 1e-12)
