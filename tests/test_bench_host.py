"""Host-side logic of bench.py without a GPU: multi-rank timing reduction over
gloo (world size 2), clock-sample parsing, the roofline arithmetic and the
FLOP counts behind it."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    r, ws, local = bench._dist()
    bench._barrier(ws)
    t = bench._max_over_ranks(1.5 + rank, ws)     # rank 1 is the slow one
    q.put((r, ws, t))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == [(0, 2, 2.5), (1, 2, 2.5)]


def test_clock_summary_parsing():
    sys.path.insert(0, ROOT)
    import bench
    c = bench.ClockSampler(None)
    c.lines = ["1980, 2032, 800.1, 0x0, Not Active, Not Active, Not Active, Not Active",
               "2010, 2032, 900.5, 0x4, Not Active, Not Active, Not Active, Active",
               "1995, 2032, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "garbage line"]
    s = c.summary()
    assert s["sm_mhz"] == 1995 and s["sm_max_mhz"] == 2032 and s["reasons"] == ["sw_power_cap"]
    assert s["samples"] == 3


def test_roofline_arithmetic():
    sys.path.insert(0, ROOT)
    import bench
    cells = 256 ** 3
    prof = {"sweep_x": {"ms": 100.0, "launches": 10}, "sweep_y": {"ms": 110.0, "launches": 10},
            "sweep_z": {"ms": 120.0, "launches": 10}}
    want = cells * bench.FLOP_PER_CELL["sweep_z"] / 12e-3 / 1e12
    # without a measurement: the derived fallback peaks
    r = bench._roofline(prof, cells, "fp64")
    assert r["kernel"] == "sweep_z" and r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert abs(r["achieved"] - round(want, 4)) < 1e-9
    assert abs(r["frac"] - round(want / bench.PEAK_FP64_TFLOPS, 4)) < 1e-9
    assert abs(sum(r["share"].values()) - 1.0) < 1e-3
    assert abs(bench.PEAK_FP32_TFLOPS - 76.98815) < 1e-3
    # with the peaks measured in the run: FP64 divides by the DFMA rate, FP32 and
    # mixed by the FP32 rate
    peaks = {"fp32_tflops": 70.0, "fp64_tflops": 1.1, "method": "test"}
    assert abs(bench._roofline(prof, cells, "fp64", peaks)["frac"] - round(want / 1.1, 4)) < 1e-9
    assert abs(bench._roofline(prof, cells, "mixed", peaks)["frac"] - round(want / 70.0, 4)) < 1e-9
    assert bench._roofline(prof, cells, "fp32", peaks)["peak_source"].startswith("measured")


def test_algorithmic_counts_and_traffic_table():
    """The FLOP counts behind roofline.achieved, assembled from their per-unit
    terms (122 per WENO7 reconstruction, 1366 per interface; 1424 / 1403 / 1423
    per cell for the x / y / z sweeps, 12750 per cell and RK3 step), and a DRAM
    entry for every sweep of every precision: null (stale) or at least the
    sweep's own stored-field accesses per cell (x: 5 staged fields read and 5
    accumulator fields written; y: also 5 read; z: also the step state)."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.FLOP_PER_INTERFACE == 1366
    assert bench.FLOP_PER_CELL == {"sweep_x": 1424, "sweep_y": 1403, "sweep_z": 1423}
    assert bench.FLOP_PER_CELL_STEP == 12750
    own = {"sweep_x": 10, "sweep_y": 15, "sweep_z": 15}   # 4-byte field accesses at least
    for p in ("fp64", "fp32", "mixed"):
        for k in ("sweep_x", "sweep_y", "sweep_z"):
            t = bench.TRAFFIC_B_PER_CELL[(p, k)]
            assert t is None or t >= 0.9 * own[k] * 4   # (writes still in L2 at the end escape the count)
    prof = {"sweep_x": {"ms": 1.0, "launches": 1}, "sweep_y": {"ms": 1.0, "launches": 1},
            "sweep_z": {"ms": 2.0, "launches": 1}}
    t = bench.TRAFFIC_B_PER_CELL[("fp64", "sweep_z")]
    assert bench._roofline(prof, 8, "fp64")["traffic"] == (None if t is None else t * 8)
    # WENO5: 65 per reconstruction, 756 per interface, the same per-cell terms;
    # no DRAM table for it
    assert bench.FLOP_PER_INTERFACE_W5 == 756
    assert bench.FLOP_PER_CELL_W5 == {"sweep_x": 814, "sweep_y": 793, "sweep_z": 813}
    r5 = bench._roofline(prof, 8, "fp64", order=5)
    assert r5["flop_per_launch"] == 8 * 813 and r5["traffic"] is None


class _Counted:
    """A float that counts the arithmetic operations applied to it (+, -, *, /:
    one FLOP each, so an FMA's multiply and add count 2)."""
    ops = 0

    def __init__(self, v):
        self.v = float(v)

    @staticmethod
    def _val(o):
        return o.v if isinstance(o, _Counted) else float(o)

    def _new(self, v):
        _Counted.ops += 1
        return _Counted(v)

    def __add__(self, o):
        return self._new(self.v + self._val(o))

    __radd__ = __add__

    def __sub__(self, o):
        return self._new(self.v - self._val(o))

    def __rsub__(self, o):
        return self._new(self._val(o) - self.v)

    def __mul__(self, o):
        return self._new(self.v * self._val(o))

    __rmul__ = __mul__

    def __truediv__(self, o):
        return self._new(self.v / self._val(o))

    def __rtruediv__(self, o):
        return self._new(self._val(o) / self.v)


def _js_weights(q, beta, dk, eps):
    """Jiang-Shu: sum_k alpha_k q_k / sum_k alpha_k, alpha_k = d_k / (eps + beta_k)^2."""
    alpha = []
    for b, d in zip(beta, dk):
        s = b + eps
        alpha.append(d / (s * s))
    num, den = alpha[0] * q[0], alpha[0]
    for a, qq in zip(alpha[1:], q[1:]):
        num = num + a * qq
        den = den + a
    return num / den


def _weno7_canonical(f, eps):
    """WENO7 at x_{i+1/2} from f_{i-3..i+3}: the four candidate cubics from the
    stencil values, Balsara-Shu indicators as 720 beta = 20 A^2 + 780 B^2 + 781 C^2
    over the first, second and third differences, Jiang-Shu weights (1, 12, 18, 4)/35."""
    qc = [(-3, 13, -23, 25), (1, -5, 13, 3), (-1, 7, 7, -1), (3, 13, -5, 1)]
    q = []
    for k, c in enumerate(qc):
        acc = f[k] * (c[0] / 12)
        for j in range(1, 4):
            acc = acc + f[k + j] * (c[j] / 12)
        q.append(acc)
    d1 = [f[j + 1] - f[j] for j in range(6)]
    d2 = [d1[j + 1] - d1[j] for j in range(5)]
    d3 = [d2[j + 1] - d2[j] for j in range(4)]
    ac = [(2, -7, 11), (-1, 5, 2), (2, 5, -1), (11, -7, 2)]
    A = [d1[k] * ac[k][0] + d1[k + 1] * ac[k][1] + d1[k + 2] * ac[k][2] for k in range(4)]
    B = [d2[1] * 2 - d2[0], d2[2], d2[2], d2[3] * 2 - d2[4]]
    beta = [A[k] * A[k] * (20 / 720) + B[k] * B[k] * (780 / 720) + d3[k] * d3[k] * (781 / 720) for k in range(4)]
    return _js_weights(q, beta, (1 / 35, 12 / 35, 18 / 35, 4 / 35), eps), beta


def _weno5_canonical(f, eps):
    """WENO5 at x_{i+1/2} from f_{i-2..i+2}: three candidate parabolas, Jiang-Shu
    indicators 13/12 D^2 + 1/4 T^2 (second differences D, first-derivative terms
    T), linear weights (1, 6, 3)/10."""
    q = [f[0] * (2 / 6) + f[1] * (-7 / 6) + f[2] * (11 / 6), f[1] * (-1 / 6) + f[2] * (5 / 6) + f[3] * (2 / 6),
         f[2] * (2 / 6) + f[3] * (5 / 6) + f[4] * (-1 / 6)]
    D = [f[k] + f[k + 1] * (-2) + f[k + 2] for k in range(3)]
    T = [f[0] + f[1] * (-4) + f[2] * 3, f[1] - f[3], f[2] * 3 + f[3] * (-4) + f[4]]
    beta = [D[k] * D[k] * (13 / 12) + T[k] * T[k] * 0.25 for k in range(3)]
    return _js_weights(q, beta, (0.1, 0.6, 0.3), eps), beta


@pytest.mark.parametrize("order", [7, 5])
def test_reconstruction_flop_counts_are_those_of_the_canonical_evaluation(orc, order):
    """The per-reconstruction FLOPs behind roofline.achieved are counted by
    running the canonical evaluation (candidates from the stencil values,
    indicators from differences, Jiang-Shu weights) on counting scalars, and that
    evaluation is checked against the oracle's reconstruction: same value and
    indicators to rounding, so the count is of the method the kernels compute."""
    sys.path.insert(0, ROOT)
    import numpy as np

    import bench
    fn, ofn, n, want = ((_weno7_canonical, orc.weno7, 7, bench.FLOP_RECON_W7) if order == 7
                        else (_weno5_canonical, orc.weno5, 5, bench.FLOP_RECON_W5))
    rng = np.random.default_rng(order)
    for trial in range(20):
        f = rng.normal(size=n) * 10.0 ** rng.uniform(-3, 3)
        if trial == 0:
            f[n // 2 + 1:] += 5.0   # a step: weights far from linear
        _Counted.ops = 0
        val, beta = fn([_Counted(x) for x in f], 1e-6)
        assert _Counted.ops == want
        ov, _, obeta, _ = ofn(f, 1e-6)
        assert abs(val.v - ov) <= 1e-12 * max(abs(ov), np.abs(f).max())
        np.testing.assert_allclose([b.v for b in beta], obeta, rtol=1e-12, atol=1e-14 * np.abs(f).max() ** 2)


def test_err_per_field_is_norm_relative():
    sys.path.insert(0, ROOT)
    import numpy as np

    import bench
    b = np.ones((5, 4, 4, 4))
    a = b.copy()
    a[2, 1, 1, 1] += 1e-6
    e = bench._err_per_field(a, b)
    assert e[2] == 1e-6 and e[0] == e[1] == e[3] == e[4] == 0.0


def test_cpu_baseline_reports_the_all_core_run_and_the_labelled_single_core_extrapolation():
    """The oracle baseline on a small grid: both runs report their rate, cores
    and sample; the single-core entry extrapolates its per-cell rate to the
    workload's steps and says that the full run was not made."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_1511_02137_b300 import workloads as W
    w = W.scaled(W.ELLIPSOIDAL_256, 24, steps=70)
    out = bench._cpu_baseline(w, single_core_grid=16)
    assert out["kind"] == "oracle" and out["cores"] >= 1 and out["value"] > 0
    one = out["single_core"]
    assert one["cores"] == 1 and one["value"] > 0 and "16^3" in one["sample"]
    assert abs(one["full_run_s_extrapolated"] - w.cells * w.steps / one["value"]) <= 0.06
    assert "extrapolated" in one["full_run"] and "not run" in one["full_run"]


def _csqrt(x):
    _Counted.ops += 1
    return _Counted(x.v ** 0.5)


def test_per_cell_flop_terms_are_those_of_the_canonical_evaluation(orc):
    """The per-cell terms of the FLOP count, each executed on counting scalars:
    the closed-form recovery (Eq. 1 with p = e/3 inverted: m = abs(M)/E,
    v = 3m / (2 + sqrt(4 - 3m^2)), e = E - abs(M) v), abs(v)^2, the spectral
    radius max abs(lambda_pm) and the half fluxes F_d / 2, checked against the
    oracle's recovery and characteristic speeds and the flux built from the
    stress tensor's definition; then the split, sums, differences and stage
    combinations, which assemble the per-cell totals of the bench."""
    sys.path.insert(0, ROOT)
    import numpy as np

    import bench
    import physics_ref as ref
    rng = np.random.default_rng(5)
    c2 = 1.0 / 3.0
    for _ in range(10):
        e0, n0 = 10 ** rng.uniform(-2, 2), rng.uniform(0.01, 0.3)
        u3 = rng.normal(size=3) * rng.uniform(0.1, 3.0)
        U = ref.conserved(e0, u3, n0)
        E, Mx, My, Mz, R = (_Counted(x) for x in U)
        _Counted.ops = 0
        Mabs = _csqrt(Mx * Mx + My * My + Mz * Mz)
        m = Mabs / E
        v = m * 3 / (_csqrt(4 - m * m * 3) + 2)
        e = E - Mabs * v
        p = e / 3
        vm = v / Mabs
        vel = (vm * Mx, vm * My, vm * Mz)
        assert _Counted.ops == bench.FLOP_C2P
        want, _ = orc.cons_to_prim(U.reshape(5, 1))
        np.testing.assert_allclose([e.v, *(a.v for a in vel), p.v], want[:5, 0], rtol=1e-13, atol=1e-15)
        _Counted.ops = 0
        v2 = vel[0] * vel[0] + vel[1] * vel[1] + vel[2] * vel[2]
        assert _Counted.ops == bench.FLOP_V2
        M = (Mx, My, Mz)
        for d in range(3):
            vd = vel[d]
            _Counted.ops = 0
            den = 1 - v2 * c2
            disc = (1 - v2) * (den - vd * vd * (1 - c2))
            rho = (_Counted(abs(vd.v)) * (1 - c2) + _csqrt(disc) * c2 ** 0.5) / den
            assert _Counted.ops == bench.FLOP_RHO
            lm, lp = orc.char_speeds(np.array([a.v for a in vel]), d)
            assert abs(rho.v - max(abs(lm), abs(lp))) <= 1e-14
            _Counted.ops = 0
            half = [M[d] * 0.5] + [(M[i] * vd + p) * 0.5 if i == d else M[i] * vd * 0.5 for i in range(3)]
            half.append(R * vd * 0.5)
            assert _Counted.ops == bench.FLOP_HALF_FLUX
            np.testing.assert_allclose([h.v for h in half], ref.flux(e0, u3, n0, d) / 2, rtol=1e-12, atol=1e-14)
    # the linear terms: split (7 cells per side, 5 fields, and alpha / 2), flux
    # sums, differences (x) or differences accumulated (y, z), stage combinations
    x = [_Counted(v) for v in rng.normal(size=8)]
    _Counted.ops = 0
    ah = x[0] * 0.5
    for _ in range(5):
        [x[1] + ah * x[2] for _ in range(7)], [x[1] - ah * x[2] for _ in range(7)]
    assert _Counted.ops == bench.FLOP_SPLIT
    _Counted.ops = 0
    [x[3] + x[4] for _ in range(5)]
    assert _Counted.ops == bench.FLOP_FSUM
    _Counted.ops = 0
    [(x[3] - x[4]) * -10.0 for _ in range(5)]
    assert _Counted.ops == bench.FLOP_DIFF
    _Counted.ops = 0
    [x[5] + (x[3] - x[4]) * -10.0 for _ in range(5)]
    assert _Counted.ops == bench.FLOP_DIFF_ACC
    _Counted.ops = 0
    [x[6] + x[7] * 0.02 for _ in range(5)]                            # U + dt L
    [x[5] * 0.75 + (x[6] + x[7] * 0.02) * 0.25 for _ in range(10)]    # a U0 + b (U + dt L), stages 2 and 3
    assert _Counted.ops == 3 * bench.FLOP_STAGE
    assert bench.FLOP_PER_INTERFACE == bench.FLOP_SPLIT + 10 * bench.FLOP_RECON_W7 + bench.FLOP_FSUM


def test_reference_arm_under_torchrun_with_two_ranks_prints_one_line():
    """The launch the multi-GPU contract uses (torch.distributed.run, one
    process per rank, rendezvous on 127.0.0.1), here with two gloo ranks on the
    CPU and the reference arm: rank 0 alone runs the oracle and prints one JSON
    line naming both ranks; the other rank exits 0 without work."""
    import json
    import subprocess
    port = _free_port()
    env = dict(os.environ, OMP_NUM_THREADS="4")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["n_gpus"] == 2 and out["value"] > 0
    assert out["warmup"] == 3 and out["steps"] == 1 and out["cpu_baseline"]["kind"] == "oracle"
