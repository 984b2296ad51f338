"""A grid at the size limit: nx ny nz = 4e8 cells, the largest hydro_create
accepts (the kernels index fields with 32-bit unsigned offsets: five fields,
six for the mixed shadow, stay below 2^32).  Needs a B300 with about 120 GB
free.

The scheme is local: one RK3 step moves information by at most 3 stages x 4
cells.  The test puts the same compact bump (a smooth perturbation of a
uniform medium at rest) at the same distance from the low and the high corner
of a 1000 x 625 x 640 grid and of a 48^3 grid.  After one step every cell of
the large grid must equal the matching cell of the small grid bit for bit:
the corner boxes (the high one holds the largest offsets of every field) match
the small grid's corners, and every other cell holds the small grid's uniform
value.  The small grid is checked against the oracle as in the parity tests.
Outflow boundaries (zero-gradient ghost cells); no jet.  The layout check runs
on the CPU."""
import gc

import numpy as np
import pytest

from harness import norm_rel_err

BIG = (1000, 625, 640)      # nx, ny, nz: 4e8 cells
M = 48                      # small grid edge
K = 24                      # corner box edge (half the small grid)
C, R = 6.0, 4.0             # bump centre distance from the corner and radius, in cells
E_BG, N_BG = 1.0, 0.16      # uniform medium at rest: e [GeV/fm^3], n [fm^-3]
TOLS = {"fp64": 1e-10, "fp32": 5e-5, "mixed": 2e-5}


def _bump(dist):
    """(1 - r^2/R^2)^4 inside radius R of the point C cells from the corner along
    every axis; dist = (dz, dy, dx) broadcastable arrays of corner distances."""
    r2 = sum((d - C) ** 2 for d in dist)
    return np.where(r2 < R * R, (1.0 - r2 / (R * R)) ** 4, 0.0)


def _primitives(shape):
    """(e, u^x, u^y, u^z, n) on a grid of shape (nx, ny, nz) as [5][nz][ny][nx]."""
    nx, ny, nz = shape
    z = np.arange(nz, dtype=np.float64)[:, None, None]
    y = np.arange(ny, dtype=np.float64)[None, :, None]
    x = np.arange(nx, dtype=np.float64)[None, None, :]
    lo = _bump((z, y, x))
    hi = _bump((nz - 1 - z, ny - 1 - y, nx - 1 - x))
    prim = np.empty((5, nz, ny, nx))
    prim[0] = E_BG * (1.0 + 2.0 * lo + 1.5 * hi)
    prim[1] = 0.3 * lo - 0.2 * hi
    prim[2] = -0.25 * lo + 0.15 * hi
    prim[3] = 0.2 * lo + 0.3 * hi
    prim[4] = N_BG * (1.0 + lo + 0.5 * hi)
    return prim


@pytest.fixture(scope="module")
def hy():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1511_02137_b300 import build
    build.build()
    from paper_1511_02137_b300 import hydro
    return hydro


def _config(hy, shape, precision):
    return hy.hydro_config_default(*shape, precision=precision)


def test_bumps_stay_inside_the_corner_boxes():
    """The layout the comparison relies on: each bump's support plus the
    12-cell reach of one step lies inside its corner box, away from the other."""
    p = _primitives((M, M, M))
    moving = np.abs(p[1]) + np.abs(p[2]) + np.abs(p[3]) > 0
    idx = np.argwhere(moving)
    lo_box = np.all(idx < K, axis=1)
    assert lo_box.any() and (~lo_box).any()
    assert idx[lo_box].max() + 12 < K and idx[~lo_box].min() - 12 >= K
    assert np.all(p[0][~moving] == E_BG) and np.all(p[4][~moving] == N_BG)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "fp32", "mixed"])
def test_grid_at_the_size_limit_matches_a_small_grid_cell_for_cell(hy, orc, precision):
    import torch
    gc.collect()
    torch.cuda.empty_cache()
    cells = BIG[0] * BIG[1] * BIG[2]
    assert cells == 400_000_000
    cfg_b = _config(hy, BIG, precision)
    need = hy.hydro_workspace_size(cfg_b) + 2 * 5 * cells * 8 + (4 << 30)
    free = torch.cuda.mem_get_info()[0]
    if free < need:
        pytest.skip(f"needs {need / 1e9:.0f} GB of free device memory, {free / 1e9:.0f} GB free")

    # the small grid, on the GPU and (the FP64 reference) in the oracle
    small = _primitives((M, M, M))
    ctx_s = hy.hydro_create(_config(hy, (M, M, M), precision))
    hy.hydro_set_initial(ctx_s, hy.HYDRO_PRIMITIVE, small.ravel())
    hy.hydro_step(ctx_s, 1)
    Gs = hy.hydro_read_fields(ctx_s, hy.HYDRO_CONSERVED)
    ds = hy.hydro_get_diag(ctx_s)
    del ctx_s
    ocfg = orc.Config(M, M, M, dx=cfg_b.dx, dt=cfg_b.dt, t0=cfg_b.t0, boundary="outflow", order=7,
                      weno_eps=cfg_b.weno_eps)
    O, _ = orc.run(ocfg, orc.prim_to_cons(small), 1)
    err = norm_rel_err(Gs, O)
    assert np.all(err <= TOLS[precision]), err
    uniform = Gs[:, K - 1, K - 1, K - 1].copy()   # a cell neither bump reaches
    assert np.array_equal(Gs[:, K, K, K], uniform) and np.array_equal(Gs[:, K - 2, K + 1, K], uniform)

    # the large grid: its initial state is built on the device and uploaded from there
    nx, ny, nz = BIG
    dev = torch.device("cuda")
    prim = torch.empty((5, nz, ny, nx), dtype=torch.float64, device=dev)
    prim[0].fill_(E_BG)
    prim[1:4].zero_()
    prim[4].fill_(N_BG)
    prim[:, :K, :K, :K] = torch.from_numpy(small[:, :K, :K, :K]).to(dev)
    prim[:, -K:, -K:, -K:] = torch.from_numpy(small[:, -K:, -K:, -K:]).to(dev)
    ctx = hy.hydro_create(cfg_b)
    hy.hydro_set_initial(ctx, hy.HYDRO_PRIMITIVE, prim)
    del prim
    torch.cuda.empty_cache()
    assert hy.hydro_step(ctx, 1) == hy.HYDRO_OK
    out = torch.empty((5, nz, ny, nx), dtype=torch.float64, device=dev)
    hy.hydro_read_fields(ctx, hy.HYDRO_CONSERVED, out)
    db = hy.hydro_get_diag(ctx)
    del ctx
    gc.collect()

    lo = out[:, :K, :K, :K].cpu().numpy()
    hi = out[:, -K:, -K:, -K:].cpu().numpy()
    assert np.array_equal(lo, Gs[:, :K, :K, :K]), np.abs(lo - Gs[:, :K, :K, :K]).max()
    assert np.array_equal(hi, Gs[:, -K:, -K:, -K:]), np.abs(hi - Gs[:, -K:, -K:, -K:]).max()
    u = torch.from_numpy(uniform).to(dev).view(5, 1, 1, 1)
    out[:, :K, :K, :K] = u
    out[:, -K:, -K:, -K:] = u
    mismatched = [int((out[q] != u[q]).sum()) for q in range(5)]
    del out
    torch.cuda.empty_cache()
    assert mismatched == [0] * 5, mismatched
    assert db["status"] == ds["status"] == 0
    assert db["max_speed"] == ds["max_speed"] and db["floor_hits"] == ds["floor_hits"]


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "fp32", "mixed"])
def test_device_field_buffers_match_host_buffers(hy, precision):
    """hydro_set_initial and hydro_read_fields (and their batch forms) take
    device pointers as well as host pointers: the same state, uploaded from a
    CUDA tensor and from a numpy array, steps to the same fields bit for bit, and
    a read into a CUDA tensor equals the read into host memory."""
    import torch
    shape = (20, 18, 16)
    prim = _primitives(shape)
    prim[0] *= 1.0 + 0.1 * np.random.default_rng(7).random(prim[0].shape)
    dev = torch.device("cuda")
    out = []
    for src in (prim.ravel(), torch.from_numpy(prim.ravel()).to(dev)):
        ctx = hy.hydro_create(_config(hy, shape, precision))
        hy.hydro_set_initial(ctx, hy.HYDRO_PRIMITIVE, src)
        hy.hydro_step(ctx, 2)
        host = hy.hydro_read_fields(ctx, hy.HYDRO_CONSERVED)
        d = torch.empty(host.size, dtype=torch.float64, device=dev)
        hy.hydro_read_fields(ctx, hy.HYDRO_CONSERVED, d)
        assert np.array_equal(d.cpu().numpy(), host.ravel())
        out.append(host)
        del ctx
    assert np.array_equal(out[0], out[1])
    cfg = _config(hy, (1, 1, 1), precision)
    b = hy.hydro_batch_create(cfg, [shape, shape])
    hy.hydro_batch_set_initial(b, 0, hy.HYDRO_PRIMITIVE, prim.ravel())
    hy.hydro_batch_set_initial(b, 1, hy.HYDRO_PRIMITIVE, torch.from_numpy(prim.ravel()).to(dev))
    hy.hydro_batch_step(b, 2)
    d = torch.empty(prim.size, dtype=torch.float64, device=dev)
    hy.hydro_batch_read_fields(b, 1, hy.HYDRO_CONSERVED, d)
    assert np.array_equal(hy.hydro_batch_read_fields(b, 0), d.cpu().numpy().reshape(out[0].shape))
    assert np.array_equal(d.cpu().numpy(), out[0].ravel())
    with pytest.raises(ValueError):   # a tensor of the wrong type is refused before the call
        hy.hydro_batch_read_fields(b, 0, hy.HYDRO_CONSERVED, d.float())
    hy.hydro_batch_destroy(b)
