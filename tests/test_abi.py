"""The C ABI library loads and exports every declared entry point (no GPU).

Only calls that touch no device memory are made here: defaults, workspace
sizing and configuration validation.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hydro.h")


@pytest.fixture(scope="module")
def hy():
    from paper_1511_02137_b300 import build
    build.build()
    from paper_1511_02137_b300 import hydro
    return hydro


def _declared_functions():
    with open(HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hydro_[a-z_]+)\s*\(", text)))


def test_header_declares_the_six_calls_and_more():
    names = _declared_functions()
    for n in ("hydro_create", "hydro_set_initial", "hydro_add_jet", "hydro_step", "hydro_read_fields",
              "hydro_destroy"):
        assert n in names
    assert "hydro_get_diag" in names


def test_library_exports_every_declared_symbol(hy):
    lib = ctypes.CDLL(hy.LIB_PATH)
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_bounds_checked_build_exports_the_same_symbols_and_takes_its_test_hook(hy):
    """libhydro_check.so (-DHYDRO_CHECK) is the same library with bounds-checked
    sweeps: it exports every declared call and accepts test_check_tighten = 1,
    which the regular build rejects."""
    from paper_1511_02137_b300 import build
    lib = ctypes.CDLL(build.build_checked())
    for name in _declared_functions():
        assert hasattr(lib, name), name
    n = ctypes.c_size_t()
    c = hy.hydro_config_default(16, 16, 16, test_check_tighten=1)
    lib.hydro_workspace_size.argtypes = [ctypes.POINTER(hy.hydro_config), ctypes.POINTER(ctypes.c_size_t)]
    assert lib.hydro_workspace_size(ctypes.byref(c), ctypes.byref(n)) == hy.HYDRO_OK
    assert hy._lib().hydro_workspace_size(ctypes.byref(c), ctypes.byref(n)) == hy.HYDRO_EINVAL
    c.test_check_tighten = 2
    assert lib.hydro_workspace_size(ctypes.byref(c), ctypes.byref(n)) == hy.HYDRO_EINVAL
    lib.hydro_status_string.restype = ctypes.c_char_p
    assert b"ECHECK" in lib.hydro_status_string(hy.HYDRO_ECHECK)


def test_defaults_are_the_paper_values(hy):
    c = hy.hydro_config_default(256, 256, 256)
    assert (c.dx, c.dt, c.t0) == (0.1, 0.02, 1.0)
    assert (c.k_rad, c.k_coll, c.cr_over_cf) == (4.0, 2.5, 1.0)
    assert (c.hbarc, c.dof) == (0.1973, 47.5)
    assert c.weno_order == 7 and c.precision == hy.HYDRO_FP64 and c.boundary == hy.HYDRO_OUTFLOW


def test_workspace_size_counts_states_rhs_cache_and_shadows(hy):
    n = 32 * 32 * 32
    fp64 = hy.hydro_workspace_size(hy.hydro_config_default(32, 32, 32))
    fp32 = hy.hydro_workspace_size(hy.hydro_config_default(32, 32, 32, precision="fp32"))
    mixed = hy.hydro_workspace_size(hy.hydro_config_default(32, 32, 32, precision="mixed"))
    assert 5 * 5 * n * 8 <= fp64 < 5 * 5 * n * 8 + 8192   # with the x sweep's primitive cache
    assert 4 * 5 * n * 4 <= fp32 < 4 * 5 * n * 4 + 8192
    # mixed: FP64 states, FP32 accumulator, and the FP32 shadows [6][n] of the three states
    assert 3 * 5 * n * 8 + 5 * n * 4 + 3 * 6 * n * 4 <= mixed < 3 * 5 * n * 8 + 5 * n * 4 + 3 * 6 * n * 4 + 8192


@pytest.mark.parametrize("field,value", [("nx", 0), ("precision", 7), ("boundary", 5), ("weno_order", 6),
                                         ("dx", 0.0), ("dt", -1.0), ("e_floor", 0.0), ("hbarc", 0.0),
                                         ("weno_eps", 0.0), ("weno_eps", 1e-30), ("weno_eps", 1e30),
                                         ("wait_limit_s", -1.0), ("wait_limit_s", 11.0),
                                         ("wait_limit_s", float("nan")), ("test_withhold_copies", 2)])
def test_invalid_configuration_is_rejected_without_touching_the_device(hy, field, value):
    c = hy.hydro_config_default(16, 16, 16)
    setattr(c, field, value)
    size = ctypes.c_size_t()
    assert hy._lib().hydro_workspace_size(ctypes.byref(c), ctypes.byref(size)) == hy.HYDRO_EINVAL
    h = ctypes.c_void_p(1)
    assert hy._lib().hydro_create(ctypes.byref(c), ctypes.byref(h)) == hy.HYDRO_EINVAL
    assert h.value is None


@pytest.mark.parametrize("precision,eps,ok", [("fp64", 1e-19, True), ("fp64", 1e19, True), ("fp32", 1e-18, True),
                                               ("fp32", 1e18, True), ("fp32", 1e-19, False), ("fp32", 1e19, False),
                                               ("mixed", 1e-19, False), ("mixed", 1e19, False)])
def test_weno_eps_range_depends_on_the_precision_of_the_weights(hy, precision, eps, ok):
    """FP32 weights 1/(eps + beta)^2 overflow below eps ~ 3e-19 (flat regions have
    beta = 0) and fall below the smallest normal above ~ 1e19; FP64 weights in
    product form take [1e-20, 1e20]."""
    c = hy.hydro_config_default(16, 16, 16, precision=precision, weno_eps=eps)
    size = ctypes.c_size_t()
    rc = hy._lib().hydro_workspace_size(ctypes.byref(c), ctypes.byref(size))
    assert (rc == hy.HYDRO_OK) == ok and (rc == hy.HYDRO_EINVAL) == (not ok)
    if precision == "mixed" and not ok:   # the mixed adjoint rejects it before allocating
        h = ctypes.c_void_p()
        d3 = ctypes.c_double * 3
        rc = hy._lib().hydro_adjoint_create(ctypes.byref(c), 4, 2, d3(0, 0, 0), d3(1, 0, 0), 30.0, 3.0,
                                            ctypes.byref(h))
        assert rc == hy.HYDRO_EINVAL and not h.value


@pytest.mark.parametrize("dims", [(1000, 1000, 401), (4, 70000, 4), (4, 4, 70000)])
def test_grids_beyond_the_32_bit_index_and_launch_limits_are_rejected(hy, dims):
    """nx ny nz <= 4e8 (32-bit element indices over 5 fields) and ny, nz <= 65535."""
    c = hy.hydro_config_default(*dims)
    size = ctypes.c_size_t()
    assert hy._lib().hydro_workspace_size(ctypes.byref(c), ctypes.byref(size)) == hy.HYDRO_EINVAL
    if dims[0] * dims[1] * dims[2] > 4e8:   # the adjoint holds the same limit, before allocating
        h = ctypes.c_void_p()
        d3 = ctypes.c_double * 3
        rc = hy._lib().hydro_adjoint_create(ctypes.byref(c), 4, 2, d3(0, 0, 0), d3(1, 0, 0), 30.0, 3.0,
                                            ctypes.byref(h))
        assert rc == hy.HYDRO_EINVAL and not h.value


def test_misaligned_workspace_is_rejected(hy):
    c = hy.hydro_config_default(8, 8, 8)
    c.workspace = 0x1000 + 8
    c.workspace_bytes = 1 << 30
    h = ctypes.c_void_p()
    assert hy._lib().hydro_create(ctypes.byref(c), ctypes.byref(h)) == hy.HYDRO_EINVAL


def test_null_arguments_are_rejected(hy):
    lib = hy._lib()
    assert lib.hydro_step(None, 1) == hy.HYDRO_EINVAL
    assert lib.hydro_set_initial(None, 0, None) == hy.HYDRO_EINVAL
    assert lib.hydro_read_fields(None, 0, None) == hy.HYDRO_EINVAL
    lib.hydro_destroy(None)
    assert lib.hydro_status_string(hy.HYDRO_ECFL).startswith(b"HYDRO_ECFL")


def test_batch_workspace_size_and_validation(hy):
    dims = [(64, 64, 64), (96, 80, 72)]
    c = hy.hydro_config_default(1, 1, 1, precision="fp32")
    cells = 64 ** 3 + 96 * 80 * 72
    size = hy.hydro_batch_workspace_size(c, dims)
    assert 4 * 5 * cells * 4 <= size < 4 * 5 * cells * 4 + (64 << 20)
    c5 = hy.hydro_config_default(1, 1, 1, weno_order=5)
    arr, n = hy._dims_array(dims)
    out = ctypes.c_size_t()
    assert hy._lib().hydro_batch_workspace_size(ctypes.byref(c5), n, arr, ctypes.byref(out)) == hy.HYDRO_EINVAL
    bad, n = hy._dims_array([(4, 0, 4)])
    assert hy._lib().hydro_batch_workspace_size(ctypes.byref(c), n, bad, ctypes.byref(out)) == hy.HYDRO_EINVAL
    assert hy._lib().hydro_batch_step(None, 1) == hy.HYDRO_EINVAL
    hy._lib().hydro_batch_destroy(None)


def test_ensemble_recipe():
    from paper_1511_02137_b300 import workloads as W
    E = W.ENSEMBLE_64
    assert len(E.events) == 64 and E.steps == 50
    for w in E.events:
        assert w.n[0] == w.n[1] == w.n[2] and w.n[0] in (64, 96, 128, 160)
        assert 10.0 <= w.e0 <= 50.0 and all(2.0 <= s <= 6.0 for s in w.sigma)
        assert 1 <= len(w.jets) <= 4
        half = 0.5 * w.n[0] * w.dx
        for j in w.jets:
            assert sum(x * x for x in j.x0) ** 0.5 < 0.4 * half + 1e-12
    assert {w.n[0] for w in E.events} == {64, 96, 128, 160}


@pytest.mark.parametrize("field,value", [("precision", 1), ("boundary", 1), ("weno_order", 5), ("nx", 0),
                                         ("weno_eps", 0.0)])
def test_adjoint_rejects_unsupported_configurations_before_allocating(hy, field, value):
    """The adjoint runs FP64 or mixed, outflow, WENO7: anything else is EINVAL
    before any device allocation (precision 1 is FP32)."""
    c = hy.hydro_config_default(16, 16, 16)
    setattr(c, field, value)
    h = ctypes.c_void_p()
    d3 = ctypes.c_double * 3
    rc = hy._lib().hydro_adjoint_create(ctypes.byref(c), 4, 2, d3(0, 0, 0), d3(1, 0, 0), 30.0, 3.0, ctypes.byref(h))
    assert rc == hy.HYDRO_EINVAL and not h.value


@pytest.mark.parametrize("nsteps,every,axis,angle,rmax", [(0, 1, (1, 0, 0), 30.0, 3.0), (4, 0, (1, 0, 0), 30.0, 3.0),
                                                           (4, 2, (0, 0, 0), 30.0, 3.0), (4, 2, (1, 0, 0), 0.0, 3.0),
                                                           (4, 2, (1, 0, 0), 30.0, -1.0)])
def test_adjoint_rejects_invalid_runs_and_cones(hy, nsteps, every, axis, angle, rmax):
    c = hy.hydro_config_default(16, 16, 16, precision="mixed")
    h = ctypes.c_void_p()
    d3 = ctypes.c_double * 3
    rc = hy._lib().hydro_adjoint_create(ctypes.byref(c), nsteps, every, d3(0, 0, 0), d3(*axis), angle, rmax,
                                        ctypes.byref(h))
    assert rc == hy.HYDRO_EINVAL and not h.value


def test_noalloc_validates_like_hydro_create_without_touching_the_device(hy):
    """hydro_step_noalloc runs the checks of hydro_create before any device call:
    a 1 x 1 x 65536 grid (launch z extent > 65535) and other invalid
    configurations are EINVAL."""
    lib = hy._lib()
    fn = lib.hydro_step_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.POINTER(hy.hydro_config), ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                   ctypes.POINTER(ctypes.c_double), ctypes.c_int32, ctypes.POINTER(hy.hydro_diag)]
    for dims, over in (((1, 1, 65536), {}), ((16, 16, 16), {"weno_order": 6}), ((16, 16, 16), {"wait_limit_s": -1})):
        c = hy.hydro_config_default(*dims, **over)
        assert fn(ctypes.byref(c), ctypes.c_void_p(0x1000), 0, 1, None, 0, None) == hy.HYDRO_EINVAL


@pytest.mark.parametrize("dims,precision,every", [((128, 128, 128), "fp64", 10), ((7, 5, 3), "mixed", 2),
                                                  ((13, 11, 9), "fp64", 3)])
def test_adjoint_workspace_size_covers_every_buffer(hy, dims, precision, every):
    """The adjoint's buffers are 256-byte aligned pieces of one workspace: for
    any grid (odd sizes included) the size counts every piece with its
    alignment padding."""
    c = hy.hydro_config_default(*dims, precision=precision)
    steps = 50 if dims[0] == 128 else 6
    size = hy.hydro_adjoint_workspace_size(c, steps, every)
    n = dims[0] * dims[1] * dims[2]
    f5 = -(-5 * n * 8 // 256) * 256
    f6 = -(-6 * n * 4 // 256) * 256
    every = min(every, steps)
    if precision == "mixed":   # per set: step states, shadows of 3 stages per step (+1), accumulator
        per_set = (every + 2) * f5 + (3 * every + 1) * f6
        extra = -(-5 * n * 4 // 256) * 256
    else:                      # per set: step states, 2 stage states per step, primitive cache, accumulator
        per_set = (every + 1 + 2 * every + 2) * f5
        extra = 0
    lower = -(-steps // every) * f5 + 2 * per_set + 5 * f5 + extra
    assert lower <= size <= lower + 16384
    bad = hy.hydro_config_default(*dims, precision=precision)
    bad.workspace = 0x1000 + 64
    bad.workspace_bytes = size
    h = ctypes.c_void_p()
    d3 = ctypes.c_double * 3
    assert hy._lib().hydro_adjoint_create(ctypes.byref(bad), steps, every, d3(0, 0, 0), d3(1, 0, 0), 30.0, 3.0,
                                          ctypes.byref(h)) == hy.HYDRO_EINVAL


def test_eval_math_and_peak_reject_bad_arguments_without_touching_the_device(hy):
    lib = hy._lib()
    assert lib.hydro_eval_math(9, 4, ctypes.c_void_p(0x1000), ctypes.c_void_p(0x2000), 0.0, None) == hy.HYDRO_EINVAL
    assert lib.hydro_eval_math(0, -1, ctypes.c_void_p(0x1000), ctypes.c_void_p(0x2000), 0.0, None) == hy.HYDRO_EINVAL
    assert lib.hydro_eval_math(0, 4, None, ctypes.c_void_p(0x2000), 0.0, None) == hy.HYDRO_EINVAL
    f = ctypes.c_double()
    m = ctypes.c_double()
    assert lib.hydro_alu_peak(7, 10, None, ctypes.byref(f), ctypes.byref(m)) == hy.HYDRO_EINVAL
    assert lib.hydro_alu_peak(0, 0, None, ctypes.byref(f), ctypes.byref(m)) == hy.HYDRO_EINVAL


def test_field_buffer_marshalling_checks_type_size_and_layout(hy):
    """The binding hands the C ABI a pointer only for a C-contiguous float64
    buffer of exactly 5 x cells values: numpy arrays and CPU tensors (and CUDA
    tensors on the context's device, checked on the GPU); anything else is
    refused before the call."""
    import numpy as np
    import torch
    n = 5 * 4 * 3 * 2
    good = np.zeros(n)
    assert hy._host_ptr(good, n, True) == good.ctypes.data
    t = torch.zeros(n, dtype=torch.float64)
    assert hy._host_ptr(t, n, False) == t.data_ptr()
    for bad in (np.zeros(n, dtype=np.float32), np.zeros(n + 1), np.zeros((n, 2))[:, 0],
                torch.zeros(n, dtype=torch.float32), torch.zeros(2 * n, dtype=torch.float64)[::2]):
        with pytest.raises(ValueError):
            hy._host_ptr(bad, n, False)
    ro = np.zeros(n)
    ro.setflags(write=False)
    with pytest.raises(ValueError):
        hy._host_ptr(ro, n, True)
    with pytest.raises(TypeError):
        hy._host_ptr([0.0] * n, n, False)


def test_header_compiles_as_c99_and_a_c_program_links_and_runs(hy, tmp_path):
    """include/hydro.h is plain C: a C99 program that includes it, links
    libhydro.so and calls the host-only entry points (defaults, workspace size,
    validation, status strings) builds with gcc -Werror and runs without a GPU."""
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    src = tmp_path / "use_hydro.c"
    src.write_text(r"""
#include <stdio.h>
#include <string.h>
#include "hydro.h"
int main(void) {
  hydro_config c;
  size_t bytes = 0;
  hydro_config_default(&c, 64, 48, 32);
  if (c.weno_order != 7 || c.precision != HYDRO_FP64 || c.dx != 0.1 || c.dt != 0.02) return 1;
  if (hydro_workspace_size(&c, &bytes) != HYDRO_OK || bytes < 4u * 5u * 64u * 48u * 32u * 8u) return 2;
  c.nx = 0;
  if (hydro_workspace_size(&c, &bytes) != HYDRO_EINVAL) return 3;
  if (strstr(hydro_status_string(HYDRO_ETIMEOUT), "HYDRO_ETIMEOUT") == NULL) return 4;
  if (hydro_create(NULL, NULL) != HYDRO_EINVAL) return 5;
  printf("ok %zu\n", bytes);
  return 0;
}
""")
    exe = tmp_path / "use_hydro"
    libdir = os.path.dirname(hy.LIB_PATH)
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                        str(src), "-o", str(exe), "-L", libdir, "-l:libhydro.so", "-Wl,-rpath," + libdir],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.startswith("ok "), (r.returncode, r.stdout, r.stderr)
