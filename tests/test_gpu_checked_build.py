"""The bounds-checked build (libhydro_check.so, -DHYDRO_CHECK; needs a B300).

In that build every sweep tile checks each global cell offset it forms and
each TMA coordinate it issues (hydro_check.cuh); a failed check is reported as
HYDRO_ECHECK with its site and value, and the access is kept inside its buffer.
It stands in for a memory checker on this pool.  A child process loads the
checked library (HYDRO_CHECKED=1) and runs every sweep configuration on ragged
grids: precisions, WENO7 and WENO5, outflow and periodic boundaries, a jet, a
batch of two grids, the allocation-free step and the adjoint (FP64 and mixed:
forward with checkpoints, recomputation and the reverse sweeps, which carry
their own checks).  No check may fail, and the
fields must equal the regular library's bit for bit (the checks add no
arithmetic).  The test hook that halves every checked bound then shows that
failures are recorded: HYDRO_ECHECK with a site and an offset in the upper half
of the grid, after which a new context steps normally.
"""
import ctypes
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SHAPE = (37, 29, 21)
CASES = [(p, order, boundary) for p in ("fp64", "fp32", "mixed") for order in (7, 5)
         for boundary in ("outflow", "periodic")]


def _run_cases(hy, W):
    """Every case for 2 steps; returns {name: (fields, diag)}."""
    from dataclasses import replace
    out = {}
    w = replace(W.ELLIPSOIDAL_32, n=SHAPE, sigma=(0.9, 0.8, 1.1))
    prim = W.ellipsoidal_primitives(w).ravel()
    for p, order, boundary in CASES:
        cfg = hy.hydro_config_default(*SHAPE, precision=p, weno_order=order, boundary=boundary)
        ctx = hy.hydro_create(cfg)
        hy.hydro_set_initial(ctx, hy.HYDRO_PRIMITIVE, prim)
        for j in w.jets:
            hy.hydro_add_jet(ctx, j.x0, j.direction, j.t_start)
        hy.hydro_step(ctx, 2)
        out[f"ctx-{p}-{order}-{boundary}"] = (hy.hydro_read_fields(ctx), hy.hydro_get_diag(ctx))
        del ctx
    for p in ("fp64", "fp32", "mixed"):
        b = hy.hydro_batch_create(hy.hydro_config_default(1, 1, 1, precision=p), [SHAPE, (24, 20, 16)])
        hy.hydro_batch_set_initial(b, 0, hy.HYDRO_PRIMITIVE, prim)
        hy.hydro_batch_set_initial(b, 1, hy.HYDRO_PRIMITIVE,
                                   W.ellipsoidal_primitives(replace(w, n=(24, 20, 16))).ravel())
        hy.hydro_batch_step(b, 2)
        for e in range(2):
            out[f"batch-{p}-{e}"] = (hy.hydro_batch_read_fields(b, e), hy.hydro_batch_get_diag(b, e))
        hy.hydro_batch_destroy(b)
    # the allocation-free step (plain loads, no tensor maps)
    import torch
    lib = ctypes.CDLL(hy.LIB_PATH)
    fn = lib.hydro_step_noalloc
    fn.argtypes = [ctypes.POINTER(hy.hydro_config), ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                   ctypes.POINTER(ctypes.c_double), ctypes.c_int32, ctypes.POINTER(hy.hydro_diag)]
    fn.restype = ctypes.c_int
    small = replace(w, n=(30, 24, 20))
    cfg = hy.hydro_config_default(*small.n)
    ref = hy.hydro_create(cfg)
    hy.hydro_set_initial(ref, hy.HYDRO_PRIMITIVE, W.ellipsoidal_primitives(small).ravel())
    U0 = hy.hydro_read_fields(ref)
    state = torch.from_numpy(U0.ravel()).cuda()
    c = hy.hydro_config.from_buffer_copy(cfg)
    c.cuda_stream = torch.cuda.current_stream().cuda_stream
    d = hy.hydro_diag()
    rc = fn(ctypes.byref(c), state.data_ptr(), 0, 2, None, 0, ctypes.byref(d))
    out["noalloc-fp64"] = (state.cpu().numpy().reshape(U0.shape),
                           {"status": rc or d.status, "check_site": d.check_site, "check_index": d.check_index})
    # the adjoint (forward with checkpoints, recomputation, reverse sweeps): J and its gradients
    from paper_1511_02137_b300 import adjoint as A
    jet = W.JetSpec((-0.6, 0.0, 0.0), (1.0, 0.0, 0.0), 1.0)
    wa = W.Workload(name="adjoint", n=(24, 20, 16), steps=6, sigma=(0.8, 1.0, 1.2), jets=(jet,))
    pa = W.ellipsoidal_primitives(wa)
    for p in ("fp64", "mixed"):
        run = A.ConeEnergyRun(hy.hydro_config_default(*wa.n, precision=p), wa.steps, 2, wa.jets,
                              torch.from_numpy(pa[1:].copy()).cuda(), apex=jet.x0, axis=jet.direction)
        e = torch.from_numpy(pa[0].copy()).cuda().requires_grad_(True)
        kr = torch.tensor(4.0, dtype=torch.float64, device="cuda", requires_grad=True)
        kc = torch.tensor(2.5, dtype=torch.float64, device="cuda", requires_grad=True)
        J = A.cone_energy(e, kr, kc, run)
        J.backward()   # raises on any status the library returns (HYDRO_ECHECK included)
        grads = np.concatenate([[J.item(), kr.grad.item(), kc.grad.item()], e.grad.cpu().numpy().ravel()])
        out[f"adjoint-{p}"] = (grads, {"status": 0, "check_site": 0})
    return out


def _child(path, tighten):
    """Runs in a process that loaded the checked library; writes the results."""
    sys.path.insert(0, ROOT)
    from paper_1511_02137_b300 import hydro as hy
    from paper_1511_02137_b300 import workloads as W
    assert hy.LIB_PATH.endswith("libhydro_check.so")
    if not tighten:
        res = _run_cases(hy, W)
        np.savez(path, **{k: v[0] for k, v in res.items()})
        with open(path + ".json", "w") as f:
            json.dump({k: {"status": v[1]["status"], "check_site": v[1]["check_site"]} for k, v in res.items()}, f)
        return
    # a uniform medium at rest: the redirected accesses read and write the same values
    prim = np.zeros((5,) + SHAPE[::-1])
    prim[0], prim[4] = 1.0, 0.1
    report = {}
    for p in ("fp64", "fp32", "mixed"):
        cfg = hy.hydro_config_default(*SHAPE, precision=p, test_check_tighten=1)
        ctx = hy.hydro_create(cfg)
        hy.hydro_set_initial(ctx, hy.HYDRO_PRIMITIVE, prim.ravel())
        st = hy.hydro_step(ctx, 1, allow=(hy.HYDRO_ECHECK,))
        d = hy.hydro_get_diag(ctx)
        del ctx
        # the CUDA context is still usable: a new hydro context without the hook steps normally
        ok = hy.hydro_create(hy.hydro_config_default(*SHAPE, precision=p))
        hy.hydro_set_initial(ok, hy.HYDRO_PRIMITIVE, prim.ravel())
        after = hy.hydro_step(ok, 1)
        report[p] = {"status": st, "diag_status": d["status"], "check_site": d["check_site"],
                     "check_index": d["check_index"], "after": after}
    with open(path + ".json", "w") as f:
        json.dump(report, f)


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sys.path.insert(0, ROOT)
    from paper_1511_02137_b300 import build
    build.build()
    build.build_checked()
    from paper_1511_02137_b300 import hydro as hy
    from paper_1511_02137_b300 import workloads as W
    assert hy.LIB_PATH.endswith("libhydro.so")
    return hy, W


def _spawn(tmp_path, tighten):
    path = str(tmp_path / ("tight" if tighten else "clean"))
    env = dict(os.environ, HYDRO_CHECKED="1")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), path, "1" if tighten else "0"], cwd=ROOT,
                       env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return path


@pytest.mark.gpu
def test_checked_build_passes_every_configuration_and_matches_the_regular_build(env, tmp_path):
    hy, W = env
    path = _spawn(tmp_path, False)
    with open(path + ".json") as f:
        checked_diag = json.load(f)
    checked = np.load(path + ".npz")
    regular = _run_cases(hy, W)
    assert set(checked_diag) == set(regular)
    for name, (fields, diag) in regular.items():
        assert checked_diag[name] == {"status": 0, "check_site": 0}, (name, checked_diag[name])
        assert diag["status"] == 0 and diag["check_site"] == 0
        assert np.array_equal(checked[name], fields), name


@pytest.mark.gpu
def test_checked_build_records_a_failed_check_and_keeps_the_context_usable(env, tmp_path):
    hy, _ = env
    path = _spawn(tmp_path, True)
    with open(path + ".json") as f:
        report = json.load(f)
    n = SHAPE[0] * SHAPE[1] * SHAPE[2]
    for p, r in report.items():
        assert r["status"] == hy.HYDRO_ECHECK and r["diag_status"] == hy.HYDRO_ECHECK, (p, r)
        assert r["check_site"] in (1, 2, 3), (p, r)          # a cell offset, not a TMA coordinate
        assert (n + 1) // 2 <= r["check_index"] < n, (p, r)   # in the upper half, inside the grid
        assert r["after"] == hy.HYDRO_OK


if __name__ == "__main__":
    _child(sys.argv[1], sys.argv[2] == "1")
