"""Gradients of the cone-energy observable through the hand-written adjoint.

J = energy (sum E dx^3) in a 30-degree cone of radius 3 fm around the jet axis
after N RK3 steps, differentiated with respect to k_rad, k_coll (Eq. 3) and the
initial energy density.  The FP64 adjoint is checked against central finite
differences of the CUDA forward (relative step 1e-6) and against central
differences of the FP64 CPU oracle (the CPU reference gradient).  The
mixed-precision adjoint (FP32 flux arithmetic) is checked against the same
FP64 finite differences: central differences of its own FP32-flux forward at
a relative step of 1e-6 would be dominated by FP32 rounding.
"""
import statistics
import time

import numpy as np
import pytest

from harness import cone_mask

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1511_02137_b300 import build
    build.build()
    from paper_1511_02137_b300 import adjoint, hydro, workloads
    return torch, hydro, adjoint, workloads


def _problem(env, n, steps, every, sigma, jet_x0, e0=30.0, precision="fp64"):
    torch, hy, A, W = env
    jet = W.JetSpec(jet_x0, (1.0, 0.0, 0.0), 1.0)
    w = W.Workload(name="adjoint test", n=n, steps=steps, sigma=sigma, e0=e0, jets=(jet,))
    prim = W.ellipsoidal_primitives(w)
    cfg = hy.hydro_config_default(*n, precision=precision)
    run = A.ConeEnergyRun(cfg, steps, every, w.jets, torch.from_numpy(prim[1:].copy()).cuda(), apex=jet.x0,
                          axis=jet.direction)
    e = torch.from_numpy(prim[0].copy()).cuda()
    return w, prim, run, e


def _value_and_grad(env, run, e, kr=4.0, kc=2.5):
    torch, hy, A, W = env
    e = e.clone().requires_grad_(True)
    kr_t = torch.tensor(kr, dtype=torch.float64, device=e.device, requires_grad=True)
    kc_t = torch.tensor(kc, dtype=torch.float64, device=e.device, requires_grad=True)
    J = A.cone_energy(e, kr_t, kc_t, run)
    J.backward()
    return J.item(), e.grad.clone(), kr_t.grad.item(), kc_t.grad.item()


def _J(env, run, e, kr=4.0, kc=2.5):
    torch, hy, A, W = env
    return A.cone_energy(e, torch.tensor(kr, dtype=torch.float64), torch.tensor(kc, dtype=torch.float64), run).item()


def _fd_check(env, run, e, directions, h=1e-6, kr=4.0, kc=2.5):
    """Central differences along relative directions (dk_rad, dk_coll, de field)."""
    J0, ge, gkr, gkc = _value_and_grad(env, run, e, kr, kc)
    rel = []
    for dkr, dkc, de in directions:
        adj = gkr * kr * dkr + gkc * kc * dkc + float((ge * e * de).sum())
        jp = _J(env, run, e * (1 + h * de), kr * (1 + h * dkr), kc * (1 + h * dkc))
        jm = _J(env, run, e * (1 - h * de), kr * (1 - h * dkr), kc * (1 - h * dkc))
        fd = (jp - jm) / (2 * h)
        rel.append(abs(fd - adj) / max(abs(fd), abs(adj), 1e-300))
    return J0, rel


def _directions(torch, shape, count, seed, device):
    g = torch.Generator().manual_seed(seed)
    out = []
    for k in range(count):
        de = torch.randn(shape, generator=g, dtype=torch.float64).to(device)
        dk = torch.randn(2, generator=g, dtype=torch.float64)
        out.append((float(dk[0]), float(dk[1]), de))
    return out


def test_adjoint_matches_central_differences_small_grid(env):
    torch = env[0]
    w, prim, run, e = _problem(env, (24, 20, 16), steps=6, every=2, sigma=(0.8, 1.0, 1.2), jet_x0=(-0.6, 0.0, 0.0))
    dirs = _directions(torch, e.shape, 4, 7, e.device)
    dirs += [(1.0, 0.0, torch.zeros_like(e)), (0.0, 1.0, torch.zeros_like(e))]
    J0, rel = _fd_check(env, run, e, dirs)
    print("small grid: J =", J0, "relative FD mismatch per direction:", rel)
    assert J0 > 0 and max(rel) < 1e-5, rel


def test_adjoint_against_oracle_central_differences(env, orc):
    """FP64 CPU reference gradient: central differences of the oracle's J."""
    torch, hy, A, W = env
    n, steps = (16, 14, 12), 4
    w, prim, run, e = _problem(env, n, steps=steps, every=3, sigma=(0.7, 0.8, 0.9), jet_x0=(-0.5, 0.0, 0.0))
    J0, ge, gkr, gkc = _value_and_grad(env, run, e)
    mask = cone_mask(n, w.dx, w.jets[0].x0)
    jets = [orc.Jet(j.x0, j.direction, j.t_start) for j in w.jets]

    def J_oracle(e_field, kr, kc):
        p = prim.copy()
        p[0] = e_field
        cfg = orc.Config(*n, dx=w.dx, dt=w.dt, t0=w.t0, k_rad=kr, k_coll=kc)
        U, _ = orc.run(cfg, orc.prim_to_cons(p), steps, jets)
        return float(U[0][mask].sum()) * w.dx ** 3

    assert abs(J_oracle(prim[0], 4.0, 2.5) / J0 - 1) < 1e-12
    h = 1e-6
    fd_kr = (J_oracle(prim[0], 4.0 * (1 + h), 2.5) - J_oracle(prim[0], 4.0 * (1 - h), 2.5)) / (2 * h * 4.0)
    fd_kc = (J_oracle(prim[0], 4.0, 2.5 * (1 + h)) - J_oracle(prim[0], 4.0, 2.5 * (1 - h))) / (2 * h * 2.5)
    assert abs(fd_kr / gkr - 1) < 1e-5 and abs(fd_kc / gkc - 1) < 1e-5, (fd_kr, gkr, fd_kc, gkc)
    rng = np.random.default_rng(3)
    for _ in range(2):
        de = rng.normal(size=prim[0].shape)
        fd = (J_oracle(prim[0] * (1 + h * de), 4.0, 2.5) - J_oracle(prim[0] * (1 - h * de), 4.0, 2.5)) / (2 * h)
        adj = float((ge.cpu().numpy() * prim[0] * de).sum())
        assert abs(fd / adj - 1) < 1e-5, (fd, adj)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("n", [(40, 36, 32), (21, 19, 17)])
def test_adjoint_forward_is_the_step_of_the_context_api(env, precision, n):
    """The adjoint's forward (and so the function it differentiates) is the step
    hydro_step runs: J from hydro_adjoint_forward equals the cone energy of the
    state a context reaches from the same primitives and jets, to the order of
    the cone sum (1e-13), in FP64 and in mixed precision, where any other
    arrangement of the FP32 arithmetic would show at ~1e-8; on a grid whose rows
    admit tensor maps and on one whose rows do not."""
    torch, hy, A, W = env
    steps = 7
    w, prim, run, e = _problem(env, n, steps=steps, every=3, sigma=(1.5, 1.8, 2.0), jet_x0=(-0.8, 0.1, 0.0),
                               precision=precision)
    J = _J(env, run, e)
    ctx = hy.hydro_create(hy.hydro_config_default(*n, precision=precision))
    for j in w.jets:
        hy.hydro_add_jet(ctx, j.x0, j.direction, j.t_start)
    hy.hydro_set_initial(ctx, hy.HYDRO_PRIMITIVE, np.ascontiguousarray(prim))
    hy.hydro_step(ctx, steps)
    U = hy.hydro_read_fields(ctx, hy.HYDRO_CONSERVED)
    hy.hydro_destroy(ctx)
    mask = cone_mask(n, w.dx, w.jets[0].x0)
    J_ctx = float(U[0][mask].sum()) * w.dx ** 3
    print(f"{precision} {n}: J adjoint {J!r}, context {J_ctx!r}, relative {abs(J / J_ctx - 1):.1e}")
    assert abs(J / J_ctx - 1) < 1e-13


FULL = dict(n=(128, 128, 128), steps=50, every=10, sigma=(4.0, 5.0, 6.0), jet_x0=(-4.0, 0.0, 0.0))


@pytest.fixture(scope="module")
def full_fd(env):
    """The 128^3 x 50-step configuration: FP64 forward, 16 seeded relative
    directions (dk_rad, dk_coll, de) and their central differences (step 1e-6)."""
    torch = env[0]
    w, prim, run, e = _problem(env, **FULL)
    dirs = _directions(torch, e.shape, 16, 1511, e.device)
    h = 1e-6
    fd = []
    for dkr, dkc, de in dirs:
        jp = _J(env, run, e * (1 + h * de), 4.0 * (1 + h * dkr), 2.5 * (1 + h * dkc))
        jm = _J(env, run, e * (1 - h * de), 4.0 * (1 - h * dkr), 2.5 * (1 - h * dkc))
        fd.append((jp - jm) / (2 * h))
    J0 = _J(env, run, e)
    del run
    return e, dirs, fd, J0


def _timed(env, run, e, runs=3):
    """Times `runs` forward + backward calls with CUDA events on the library's
    stream (torch's current stream): per call one interval around the forward
    pass and one around the backward pass.  Returns the median forward and
    backward times (s), the median of the per-call ratios backward / forward, and
    (J, dJ/de, dJ/dk_rad, dJ/dk_coll) of the last call."""
    torch, hy, A, W = env
    fwd, bwd, ratio = [], [], []
    out = None
    for _ in range(runs):
        ee = e.clone().requires_grad_(True)
        kr = torch.tensor(4.0, dtype=torch.float64, device=e.device, requires_grad=True)
        kc = torch.tensor(2.5, dtype=torch.float64, device=e.device, requires_grad=True)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        torch.cuda.synchronize()
        ev[0].record()
        J = A.cone_energy(ee, kr, kc, run)
        ev[1].record()
        J.backward()
        ev[2].record()
        ev[2].synchronize()
        f, b = ev[0].elapsed_time(ev[1]) / 1e3, ev[1].elapsed_time(ev[2]) / 1e3
        fwd.append(f)
        bwd.append(b)
        ratio.append(b / f)
        out = (J.item(), ee.grad.clone(), kr.grad.item(), kc.grad.item())
    return statistics.median(fwd), statistics.median(bwd), statistics.median(ratio), out


def _directional(ge, gkr, gkc, e, dirs):
    return [gkr * 4.0 * dkr + gkc * 2.5 * dkc + float((ge * e * de).sum()) for dkr, dkc, de in dirs]


def test_adjoint_full_config_128_cube_50_steps(env, full_fd):
    """The adjoint configuration: 128^3, 50 steps, checkpoint every 10, one jet
    from (-4, 0, 0) fm along +x, cone apex at the jet start; 16 seeded
    central-difference directions at relative step 1e-6 agree to 1e-4, and the
    backward pass costs at most 4 forward passes (the median over three calls of
    the per-call ratio, CUDA events on the library stream; measured 3.3 on B300)."""
    torch = env[0]
    e, dirs, fd, J0 = full_fd
    w, prim, run, _ = _problem(env, **FULL)
    t_fwd, t_bwd, ratio, (J, ge, gkr, gkc) = _timed(env, run, e)
    print(f"128^3 x 50 FP64: forward {t_fwd:.2f} s, backward {t_bwd:.2f} s, backward / forward = {ratio:.2f} "
          "(medians of three calls, CUDA events)")
    adj = _directional(ge, gkr, gkc, e, dirs)
    rel = [abs(f - a) / max(abs(f), abs(a), 1e-300) for f, a in zip(fd, adj)]
    print("128^3 FP64: J =", J, "max relative FD mismatch over 16 directions:", max(rel))
    assert abs(J / J0 - 1) < 1e-14
    assert max(rel) < 1e-4, rel
    assert ratio <= 4.0


def test_mixed_adjoint_small_grid_against_fp64(env):
    """Mixed precision on the small grid: the gradient fields and dJ/dk agree
    with the FP64 adjoint to the FP32 level."""
    torch = env[0]
    args = dict(n=(24, 20, 16), steps=6, every=2, sigma=(0.8, 1.0, 1.2), jet_x0=(-0.6, 0.0, 0.0))
    _, _, run64, e = _problem(env, **args)
    _, _, run32, _ = _problem(env, precision="mixed", **args)
    J64, ge64, gkr64, gkc64 = _value_and_grad(env, run64, e)
    J32, ge32, gkr32, gkc32 = _value_and_grad(env, run32, e)
    err_e = float((ge32 - ge64).abs().max() / ge64.abs().max())
    print(f"mixed vs FP64 adjoint, small grid: J {abs(J32 / J64 - 1):.2e}, grad e {err_e:.2e}, "
          f"k_rad {abs(gkr32 / gkr64 - 1):.2e}, k_coll {abs(gkc32 / gkc64 - 1):.2e}")
    assert abs(J32 / J64 - 1) < 1e-5
    assert err_e < 1e-3
    assert abs(gkr32 / gkr64 - 1) < 1e-4 and abs(gkc32 / gkc64 - 1) < 1e-4


def test_mixed_adjoint_full_config_against_fp64_differences(env, full_fd):
    """Mixed precision at the adjoint configuration: the 16 directional
    derivatives of the mixed adjoint agree with the FP64 central differences
    to 1e-3 relative (FP32 flux arithmetic; measured 3.0e-4), at no more than 4
    forward costs (median per-call ratio, CUDA events; measured 3.1)."""
    torch = env[0]
    e, dirs, fd, J0 = full_fd
    w, prim, run, _ = _problem(env, precision="mixed", **FULL)
    t_fwd, t_bwd, ratio, (J, ge, gkr, gkc) = _timed(env, run, e)
    adj = _directional(ge, gkr, gkc, e, dirs)
    rel = [abs(f - a) / max(abs(f), abs(a), 1e-300) for f, a in zip(fd, adj)]
    print(f"128^3 x 50 mixed: forward {t_fwd:.3f} s, backward {t_bwd:.3f} s, backward / forward = "
          f"{ratio:.2f}; J vs FP64 {abs(J / J0 - 1):.2e}; max relative mismatch vs FP64 FD {max(rel):.2e}")
    assert abs(J / J0 - 1) < 1e-5
    assert max(rel) < 1e-3, rel
    assert ratio <= 4.0
