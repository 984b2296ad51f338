"""Device arithmetic and ultra-relativistic flow (needs a B300).

1. The hand-written FP64 reciprocal and square-root pair of the sweeps
   (Newton-Raphson from the hardware approximations) against exactly rounded
   references over the ranges of their call sites.
2. The closed-form primitive recovery (Eq. 1 with p = e/3 inverted) as the
   FP64, FP32 and mixed-precision sweeps run it, against an extended-precision
   evaluation of the same closed form, at Lorentz factors up to 1e3.  As v -> 1
   the recovery cancels (1 - m v ~ 1/gamma^2): FP32 loses ~gamma^2 ulps in e,
   while the mixed recovery (E^2 - |M|^2 in FP64, the rest in FP32 in terms of
   om = 1 - |M|/E) keeps e and 1 - v to FP32 rounding of the FP64 result.
3. Whole steps on boosted states (gamma 10 to 100) and a relativistic shock
   tube (left state at u = 20) in FP64, FP32 and mixed precision against the
   FP64 oracle, per conserved field and for the rest-frame energy density.
"""
import math

import numpy as np
import pytest

from harness import norm_rel_err

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1511_02137_b300 import build
    build.build()
    from paper_1511_02137_b300 import hydro, workloads
    return torch, hydro, workloads


def _rel_err_ld(got, exact):
    """Relative error of float64 results against long-double references."""
    g = got.astype(np.longdouble)
    return np.abs((g - exact) / exact)


def test_fp64_reciprocal_is_within_its_stated_bound(env):
    """rcp_nr: one third-order Newton-Raphson step from rcp.approx.ftz.f64.
    Divisors: log-uniform over [1e-300, 1e300] (floored energies down to 3e-11,
    products of two WENO denominators between eps_s^12 and (eps_s + beta)^12),
    dense in [3, 4] (2 + s), and binade edges.  Stated bound: 2.2e-16 relative
    (1-2 ulp)."""
    torch, hy, _ = env
    rng = np.random.default_rng(2024)
    x = np.concatenate([10.0 ** rng.uniform(-300, 300, 600_000), rng.uniform(3.0, 4.0, 300_000),
                        rng.uniform(1.0, 2.0, 100_000), 2.0 ** np.arange(-990, 990, dtype=np.float64),
                        np.nextafter(2.0 ** np.arange(-990, 990, dtype=np.float64), 0)])
    y = hy.hydro_eval_math(hy.HYDRO_MATH_RCP, torch.from_numpy(x).cuda()).cpu().numpy()
    exact = np.longdouble(1) / x.astype(np.longdouble)
    err = _rel_err_ld(y, exact)
    ieee = _rel_err_ld(1.0 / x, exact)       # correctly rounded division, for scale
    print(f"rcp_nr over {x.size} divisors: max relative error {float(err.max()):.3e} "
          f"(IEEE division {float(ieee.max()):.3e})")
    assert float(err.max()) <= 2.3e-16


def test_fp64_sqrt_rsqrt_pair_is_within_its_stated_bound(env):
    """sqrt_rsqrt_nr: rsqrt.approx.ftz.f64 and one third-order Newton-Raphson
    step give x^(-1/2), then x^(1/2) = x y.  Arguments: [1, 4] (4 - 3 m^2 of the
    recovery) and log-uniform [2^-1022, 1] (the discriminant of the spectral
    radius).  Stated bound: 2.2e-16 relative for both."""
    torch, hy, _ = env
    rng = np.random.default_rng(7)
    x = np.concatenate([rng.uniform(1.0, 4.0, 500_000), 2.0 ** rng.uniform(-1022, 0, 500_000),
                        np.array([1.0, 4.0, 2.0, np.nextafter(4.0, 0), np.nextafter(1.0, 2)])])
    out = hy.hydro_eval_math(hy.HYDRO_MATH_SQRT_RSQRT, torch.from_numpy(x).cuda()).cpu().numpy()
    s, r = out[:x.size], out[x.size:]
    xl = x.astype(np.longdouble)
    es = _rel_err_ld(s, np.sqrt(xl))
    er = _rel_err_ld(r, np.longdouble(1) / np.sqrt(xl))
    print(f"sqrt_rsqrt_nr over {x.size} arguments: sqrt {float(es.max()):.3e}, rsqrt {float(er.max()):.3e}")
    assert float(es.max()) <= 2.3e-16 and float(er.max()) <= 2.3e-16


def test_integer_pipe_widening_matches_the_hardware_on_every_fp32_value(env):
    """f2d, the FP32 -> FP64 widening of the mixed path on the integer pipe, on
    all 2^32 FP32 bit patterns against CUDA's conversion (cvt.f64.f32, exact):
    bitwise equal for zeros, normals and infinities; FP32 subnormals give the
    signed zero; NaN stays NaN."""
    torch, hy, _ = env
    chunk = 1 << 28
    bad = 0
    for start in range(0, 1 << 32, chunk):
        bits = torch.arange(start, start + chunk, dtype=torch.int64, device="cuda").to(torch.int32)
        f = bits.view(torch.float32)
        got = hy.hydro_eval_math(hy.HYDRO_MATH_F2D, f)
        ref = f.to(torch.float64)
        mag = bits & 0x7FFFFFFF
        sub = (mag > 0) & (mag < 0x00800000)
        nan = mag > 0x7F800000
        ref = torch.where(sub, torch.copysign(torch.zeros_like(ref), ref), ref)
        same = got.view(torch.int64) == ref.view(torch.int64)
        ok = torch.where(nan, torch.isnan(got), same)
        bad += int((~ok).sum())
        del bits, f, got, ref, mag, sub, nan, same, ok
    torch.cuda.empty_cache()
    assert bad == 0


def test_integer_pipe_rounding_matches_the_hardware_round_to_nearest(env):
    """d2f_rn, the FP64 -> FP32 rounding of the mixed path on the integer pipe,
    against CUDA's cvt.rn.f32.f64: bitwise equal for every input of magnitude
    at least 2^-126 (the FP32 normal range, rounding to nearest even, overflow
    to infinity), signed zero below it, NaN for NaN.  Inputs: uniformly random
    64-bit patterns (every exponent), random doubles inside the FP32 range,
    exact ties between adjacent floats, and the edges of the range."""
    torch, hy, _ = env
    rng = np.random.default_rng(11)
    n = 1 << 22
    pats = rng.integers(0, 2 ** 63, n, dtype=np.int64) * np.where(rng.random(n) < 0.5, 1, -1)
    x_bits = pats.view(np.float64)
    x_in = (2.0 ** rng.uniform(-126, 128, n)) * rng.choice([-1.0, 1.0], n) * rng.uniform(1, 2, n) / 2
    f = (2.0 ** rng.uniform(-125, 127, n)).astype(np.float32)
    ties = (f.astype(np.float64) + np.nextafter(f, np.float32(np.inf)).astype(np.float64)) / 2   # exact midpoints
    fmax = float(np.finfo(np.float32).max)
    tmin = 2.0 ** -126
    edges = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, fmax, -fmax, fmax * (1 + 2.0 ** -25),
                      np.nextafter(fmax * (1 + 2.0 ** -25), 0), np.nextafter(fmax * (1 + 2.0 ** -25), np.inf),
                      tmin, -tmin, np.nextafter(tmin, 0), np.nextafter(tmin, 1), 2.0 ** -149, 1e-300, 1e300,
                      5e-324, 1.0, 3.0, 1.0 + 2.0 ** -24, 1.0 + 2.0 ** -23 + 2.0 ** -24])
    x = np.concatenate([x_bits, x_in, ties, -ties, edges])
    xd = torch.from_numpy(x).cuda()
    got = hy.hydro_eval_math(hy.HYDRO_MATH_D2F, xd)
    ref = xd.to(torch.float32)
    ax = xd.abs()
    small = ax < tmin
    nan = torch.isnan(xd)
    ref = torch.where(small, torch.copysign(torch.zeros_like(ref), ref), ref)   # (the conversion keeps the sign)
    same = got.view(torch.int32) == ref.view(torch.int32)
    ok = torch.where(nan, torch.isnan(got), same)
    print(f"d2f_rn over {x.size} inputs ({int(small.sum())} below the FP32 normal range, "
          f"{int((ax >= 2.0 ** 128).sum())} above it): mismatches {int((~ok).sum())}")
    assert int((~ok).sum()) == 0


def _boosted_states(n, gamma_max, seed):
    """Conserved (E, M) of random rest-frame states: e log-uniform in [1e-3, 1e2]
    GeV/fm^3, gamma log-uniform in [1, gamma_max], isotropic directions."""
    rng = np.random.default_rng(seed)
    e = 10.0 ** rng.uniform(-3, 2, n)
    g = 10.0 ** rng.uniform(0, math.log10(gamma_max), n)
    ct = rng.uniform(-1, 1, n)
    ph = rng.uniform(0, 2 * np.pi, n)
    st = np.sqrt(1 - ct * ct)
    u = np.sqrt(g * g - 1)
    ux, uy, uz = u * st * np.cos(ph), u * st * np.sin(ph), u * ct
    E = (4.0 / 3.0) * e * g * g - e / 3.0
    M = [(4.0 / 3.0) * e * g * c for c in (ux, uy, uz)]
    return E, M, g


def _recovery_exact(E, M):
    """The closed form m = |M|/E, v = 3m/(2 + sqrt(4 - 3m^2)), e = E (1 - m v),
    v^i = v M^i/|M| evaluated in long double (64-bit significand) on the given
    FP64 conserved values."""
    El = E.astype(np.longdouble)
    Ml = [m.astype(np.longdouble) for m in M]
    Mabs = np.sqrt(Ml[0] ** 2 + Ml[1] ** 2 + Ml[2] ** 2)
    m = Mabs / El
    v = 3 * m / (2 + np.sqrt(4 - 3 * m * m))
    e = El * (1 - m * v)
    vi = [v * c / Mabs for c in Ml]
    return e, vi, v


@pytest.mark.parametrize("path,fn,gamma_max", [("fp64", 2, 1e3), ("fp32", 3, 300.0), ("mixed", 4, 1e3)])
def test_primitive_recovery_at_lorentz_factors_up_to_1e3(env, path, fn, gamma_max):
    """FP32 stops at gamma = 300: its cap on |M|/E (1 - 2^-20) acts from gamma ~ 500."""
    torch, hy, _ = env
    E, M, g = _boosted_states(400_000, gamma_max, 11)
    x = np.concatenate([E, M[0], M[1], M[2]])
    out = hy.hydro_eval_math(fn, torch.from_numpy(x).cuda(), 3e-11).cpu().numpy().reshape(5, -1)
    e_ref, v_ref, v_abs = _recovery_exact(E, M)
    assert not out[4].any(), "no floor acts on these states"
    err_e = _rel_err_ld(out[0], e_ref)
    # 1 - v from the recovered components against the exact 1 - v (the quantity
    # that sets gamma); relative to 1 - v itself
    v_got = np.sqrt(sum(out[1 + k].astype(np.longdouble) ** 2 for k in range(3)))
    err_1mv = np.abs((1 - v_got) - (1 - v_abs)) / (1 - v_abs)
    err_vi = max(float(np.max(np.abs(out[1 + k] - v_ref[k]) / v_abs)) for k in range(3))
    bins = [(1, 10), (10, 100), (100, 1001)]
    rows = []
    for lo, hi in bins:
        sel = (g >= lo) & (g < hi)
        rows.append((lo, hi, float(err_e[sel].max()), float(err_1mv[sel].max())))
    print(path, "recovery: max relative error of e and of 1 - v per gamma range:",
          ", ".join(f"[{lo},{hi}): e {a:.2e}, 1-v {b:.2e}" for lo, hi, a, b in rows), f"; v^i {err_vi:.2e}")
    print(path, f"max relative error of e / gamma^2: {float((err_e / (g * g)).max()):.2e}")
    if path == "fp64":
        # the closed form itself cancels: e = E (1 - m v) with E/e = (4 gamma^2 - 1)/3,
        # so a few ulps of m and v become ~gamma^2 ulps of e (measured 1e-15 gamma^2)
        assert np.all(err_e <= 4e-15 * g * g + 1e-15)
        assert err_vi <= 1e-15
    elif path == "mixed":
        # FP64 for E^2 - |M|^2 keeps the cancellation out of FP32: e and the
        # velocity components to a few FP32 ulps at every gamma
        assert float(err_e.max()) <= 2e-6
        assert err_vi <= 1e-6
        # 1 - v from FP32 components is limited by their rounding (~6e-8 each)
        # relative to 1 - v ~ 1/(2 gamma^2): measured 4.4e-7 gamma^2
        assert np.all(err_1mv <= 2e-6 + 1e-6 * g * g)
    else:
        # FP32 recovery: the cancellation costs ~gamma^2 ulps in e
        assert np.all(err_e <= 1e-6 + 1e-6 * g * g)
        assert err_vi <= 1e-6


def _boosted_grid(W, gamma, shape=(36, 20, 12), amp=0.01):
    """Periodic boosted state: e = 1 + amp sin(kx x) sin(ky y) cos(kz z), u^i =
    sqrt(gamma^2 - 1) n^i along n = (1, 0.5, 0.25)/|.|, n = 0.5 fm^-3."""
    nx, ny, nz = shape
    dx = 0.1
    x = (np.arange(nx) + 0.5 - nx / 2) * dx
    y = (np.arange(ny) + 0.5 - ny / 2) * dx
    z = (np.arange(nz) + 0.5 - nz / 2) * dx
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    k = [2 * np.pi / (s * dx) for s in shape]
    d = np.array([1.0, 0.5, 0.25])
    d /= np.linalg.norm(d)
    u = math.sqrt(gamma * gamma - 1)
    prim = np.empty((5, nz, ny, nx))
    prim[0] = 1.0 + amp * np.sin(k[0] * X) * np.sin(k[1] * Y) * np.cos(k[2] * Z)
    for a in range(3):
        prim[1 + a] = u * d[a]
    prim[4] = 0.5
    return prim


def _run(hy, prim, shape, steps, precision, boundary="periodic", dx=0.1, dt=0.02, t0=1.0):
    cfg = hy.hydro_config_default(*shape, precision=precision, boundary=boundary, dx=dx, dt=dt, t0=t0)
    ctx = hy.hydro_create(cfg)
    hy.hydro_set_initial(ctx, hy.HYDRO_PRIMITIVE, np.ascontiguousarray(prim).ravel())
    hy.hydro_step(ctx, steps)
    G = hy.hydro_read_fields(ctx, hy.HYDRO_CONSERVED)
    d = hy.hydro_get_diag(ctx)
    hy.hydro_destroy(ctx)
    return G, d


def _e_err(orc, G, O):
    """max |e_G - e_O| / max e_O, with e from the oracle's FP64 recovery of each state."""
    eg, _ = orc.cons_to_prim(G)
    eo, _ = orc.cons_to_prim(O)
    return float(np.abs(eg[0] - eo[0]).max() / np.abs(eo[0]).max())


@pytest.mark.parametrize("gamma", [10.0, 30.0, 100.0])
def test_boosted_periodic_flow_against_the_oracle(env, orc, gamma):
    """A 1% perturbation riding on a flow at Lorentz factor gamma (periodic box,
    5 RK3 steps).  FP64 matches the oracle to 1e-10 per conserved field; e,
    recovered from the conserved fields by the oracle on both sides, inherits
    that error times E/e = (4 gamma^2 - 1)/3.  FP32 and mixed errors are
    reported per conserved field and for e; both are bounded by FP32 rounding of
    the fluxes (relative to E) accumulated over the stages, so their error in e
    also grows like gamma^2: the mixed path's FP64 recovery keeps e exact to
    FP32 rounding of the state it is given, and its FP64 state drops the FP32
    storage rounding, which leaves it 3-5 times closer to the oracle than FP32
    (measured: e within 4e-7 gamma^2 against 1.4e-6 gamma^2)."""
    torch, hy, W = env
    shape = (36, 20, 12)
    prim = _boosted_grid(W, gamma, shape)
    steps = 5
    c = orc.Config(*shape, dx=0.1, dt=0.02, t0=1.0, boundary="periodic")
    O, od = orc.run(c, orc.prim_to_cons(prim), steps)
    res = {}
    for prec in ("fp64", "mixed", "fp32"):
        G, d = _run(hy, prim, shape, steps, prec)
        assert d["status"] == 0 and d["floor_hits"] == 0 == od.floor_hits
        res[prec] = (norm_rel_err(G, O), _e_err(orc, G, O))
    for prec, (err, ee) in res.items():
        print(f"gamma {gamma:g} {prec}: conserved error per field {np.array2string(err, precision=2)}, e {ee:.2e}")
    g2 = gamma * gamma
    assert np.all(res["fp64"][0] <= FP64_TOL) and res["fp64"][1] <= 2e-11 * g2
    for prec in ("mixed", "fp32"):
        err, ee = res[prec]
        assert np.all(err <= 1e-5), (prec, err)
        assert ee <= 3e-6 * g2, (prec, ee)
    assert res["mixed"][1] < res["fp32"][1]


@pytest.mark.parametrize("axis", [0, 2])
def test_ultrarelativistic_shock_tube_against_the_oracle(env, orc, axis):
    """Left state e = 10 GeV/fm^3 moving at u = 20 (gamma = 20) into e = 1 at
    rest along the axis, outflow, 40 steps at dt = 0.2 dx.  This collision
    amplifies rounding: the oracle's own result moves by ~4e-10 after one step
    and ~2e-8 after 40 when its input is perturbed by one ulp (random signs), so
    no two FP64 evaluations that round differently can agree to 1e-10.  The
    FP64 GPU path must agree with the oracle to within 3 times that measured
    sensitivity (per field); FP32 and mixed errors are reported and bounded."""
    torch, hy, W = env
    N = 160
    dx = 10.0 / N
    shape = [1, 1, 1]
    shape[axis] = N
    xc = (np.arange(N) + 0.5 - N / 2) * dx
    prim = np.zeros((5, N))
    left = xc < 0
    prim[0] = np.where(left, 10.0, 1.0)
    prim[1 + axis] = np.where(left, 20.0, 0.0)
    prim[4] = 0.1
    prim = prim.reshape((5, shape[2], shape[1], shape[0]))
    steps = 40
    dt = 0.2 * dx
    c = orc.Config(*shape, dx=dx, dt=dt, t0=0.0)
    U0 = orc.prim_to_cons(prim)
    O, od = orc.run(c, U0, steps)
    rng = np.random.default_rng(1)
    Op, _ = orc.run(c, U0 * (1 + 2.2e-16 * np.sign(rng.standard_normal(U0.shape))), steps)
    sens = norm_rel_err(Op, O)
    print(f"oracle sensitivity to a one-ulp perturbation of its input after {steps} steps: {sens}")
    res = {}
    for prec in ("fp64", "mixed", "fp32"):
        G, d = _run(hy, prim, tuple(shape), steps, prec, boundary="outflow", dx=dx, dt=dt, t0=0.0)
        assert d["status"] == 0
        if prec == "fp64":
            assert d["floor_hits"] == od.floor_hits
        res[prec] = (norm_rel_err(G, O), _e_err(orc, G, O))
    for prec, (err, ee) in res.items():
        print(f"u = 20 shock tube, axis {axis}, {prec}: conserved error per field "
              f"{np.array2string(err, precision=2)}, e {ee:.2e}")
    assert np.all(res["fp64"][0] <= 3 * sens + FP64_TOL * 1e-3), (res["fp64"][0], sens)
    for prec in ("mixed", "fp32"):
        err, ee = res[prec]
        assert np.all(err <= 1e-4), (prec, err)
