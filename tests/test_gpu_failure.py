"""Failure detection on the device without faulting the GPU (needs a B300).

A tile waits for its TMA copies into shared memory on an mbarrier, with a
time limit on the GPU's global timer (hydro_config.wait_limit_s).  The test
configuration arms the barriers but withholds the copies (nothing is ever in
flight), so every such wait runs out: hydro_step must return HYDRO_ETIMEOUT
after a bounded time, and the CUDA context must stay usable for the next run.
"""
import time
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


@pytest.mark.parametrize("precision", ["fp64", "fp32", "mixed"])
def test_withheld_copies_make_the_bounded_wait_run_out(hy, precision):
    from paper_1511_02137_b300 import workloads as W
    # 72 cells per axis: the y and z sweeps (32-cell tiles) have tiles whose halo
    # lies inside the grid, which take the TMA staging path; every FP32-flux tile
    # of the y and z sweeps fetches its phase-3 operands by TMA
    w = replace(W.ELLIPSOIDAL_32, n=(72, 72, 72), sigma=(1.5, 1.5, 1.5), jets=())
    ctx = gpu_context(hy, w, precision, wait_limit_s=1e-3, test_withhold_copies=1)
    t0 = time.perf_counter()
    with pytest.raises(hy.HydroError) as e:
        hy.hydro_step(ctx, 1)
    took = time.perf_counter() - t0
    assert e.value.status == hy.HYDRO_ETIMEOUT
    assert hy.hydro_get_diag(ctx)["status"] == hy.HYDRO_ETIMEOUT
    print(f"{precision}: HYDRO_ETIMEOUT after {took * 1e3:.1f} ms (wait limit 1 ms per tile)")
    assert took < 5.0
    # the same context again from a new initial state: the status was cleared and
    # the withheld copies time out again
    hy.hydro_set_initial(ctx, hy.HYDRO_PRIMITIVE, W.ellipsoidal_primitives(w).ravel())
    assert hy.hydro_step(ctx, 1, allow=(hy.HYDRO_ETIMEOUT,)) == hy.HYDRO_ETIMEOUT
    hy.hydro_destroy(ctx)
    # the CUDA context is intact: a normal run afterwards gives the same state as
    # a run made in a context that never timed out would (checked against FP64)
    good = gpu_context(hy, w, precision)
    hy.hydro_step(good, 2)
    G = hy.hydro_read_fields(good, hy.HYDRO_CONSERVED)
    ref = gpu_context(hy, w, "fp64")
    hy.hydro_step(ref, 2)
    R = hy.hydro_read_fields(ref, hy.HYDRO_CONSERVED)
    assert hy.hydro_get_diag(good)["status"] == 0
    assert np.all(norm_rel_err(G, R) <= (1e-12 if precision == "fp64" else 1e-5))


@pytest.mark.parametrize("precision", ["fp64", "fp32", "mixed"])
def test_withheld_copies_make_the_batched_wait_run_out(hy, precision):
    """The batched sweeps (one launch over the tiles of every grid, replayed from
    a CUDA graph) wait on the same bounded barriers: with the copies withheld,
    hydro_batch_step returns HYDRO_ETIMEOUT after a bounded time in both launch
    forms (a persistent block stops at its first late tile), and a batch made
    afterwards steps to the same state as hydro_step on each grid."""
    from paper_1511_02137_b300 import workloads as W
    dims = [(72, 72, 72), (64, 72, 40)]
    ws = [replace(W.ELLIPSOIDAL_32, n=d, sigma=(1.5, 1.5, 1.5), jets=()) for d in dims]
    prims = [np.ascontiguousarray(W.ellipsoidal_primitives(w)).ravel() for w in ws]

    def batch(**over):
        w = ws[0]
        cfg = hy.hydro_config_default(*dims[0], precision=precision, dx=w.dx, dt=w.dt, t0=w.t0, **over)
        b = hy.hydro_batch_create(cfg, dims)
        for e, p in enumerate(prims):
            hy.hydro_batch_set_initial(b, e, hy.HYDRO_PRIMITIVE, p)
        return b

    for per_tile in (1, 0):
        b = batch(wait_limit_s=1e-3, test_withhold_copies=1)
        hy.hydro_batch_set_launch(b, (per_tile,) * 3)
        t0 = time.perf_counter()
        assert hy.hydro_batch_step(b, 1, allow=(hy.HYDRO_ETIMEOUT,)) == hy.HYDRO_ETIMEOUT
        took = time.perf_counter() - t0
        statuses = [hy.hydro_batch_get_diag(b, e)["status"] for e in range(len(dims))]
        print(f"{precision}, {'one block per tile' if per_tile else 'persistent'}: HYDRO_ETIMEOUT after "
              f"{took * 1e3:.1f} ms, statuses {statuses}")
        assert hy.HYDRO_ETIMEOUT in statuses and set(statuses) <= {0, hy.HYDRO_ETIMEOUT}
        assert took < 5.0
        hy.hydro_batch_destroy(b)
    # the CUDA context is intact: a batch without the fault equals each grid stepped alone
    b = batch()
    hy.hydro_batch_step(b, 2)
    for e, w in enumerate(ws):
        ctx = gpu_context(hy, w, precision)
        hy.hydro_step(ctx, 2)
        assert np.array_equal(hy.hydro_batch_read_fields(b, e), hy.hydro_read_fields(ctx, hy.HYDRO_CONSERVED))
        assert hy.hydro_batch_get_diag(b, e)["status"] == 0
        hy.hydro_destroy(ctx)
    hy.hydro_batch_destroy(b)
