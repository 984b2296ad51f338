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
