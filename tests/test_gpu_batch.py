"""Batched ensembles on the GPU: parity with the oracle and with single-grid runs.

The batched sweeps run the same per-interface and per-cell arithmetic as the
single-grid sweeps, whatever tile shape the autotuner picks, so a grid advanced
inside a batch must match the same grid advanced alone bit for bit; in FP64
both also match the oracle to 1e-10.
"""
from dataclasses import replace

import numpy as np
import pytest

from harness import gpu_context, norm_rel_err, oracle_config, oracle_jets

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


def _small_ensemble(W):
    shapes = [(16, 20, 12), (24, 16, 18), (33, 17, 9), (8, 40, 20), (70, 5, 6)]
    events = []
    for k, n in enumerate(shapes):
        jets = W.seeded_jets(100 + k, 1 + k % 3, 0.5, 1.0)
        events.append(replace(W.ELLIPSOIDAL_32, n=n, sigma=(0.7 + 0.1 * k, 0.9, 1.1), e0=20.0 + 5 * k, jets=jets))
    return events


def _batch(hy, W, events, precision, variants=None):
    cfg = hy.hydro_config_default(1, 1, 1, precision=precision)
    b = hy.hydro_batch_create(cfg, [w.n for w in events])
    for e, w in enumerate(events):
        hy.hydro_batch_set_initial(b, e, hy.HYDRO_PRIMITIVE, W.ellipsoidal_primitives(w).ravel())
        for j in w.jets:
            hy.hydro_batch_add_jet(b, e, j.x0, j.direction, j.t_start)
    if variants is not None:
        hy.hydro_batch_set_tiles(b, variants)
    return b


def _single(hy, w, precision, steps):
    ctx = gpu_context(hy, w, precision)
    hy.hydro_step(ctx, steps)
    out = hy.hydro_read_fields(ctx, hy.HYDRO_CONSERVED)
    d = hy.hydro_get_diag(ctx)
    hy.hydro_destroy(ctx)
    return out, d


def test_fp64_batch_matches_oracle_and_single_grid_for_every_tile_shape(hy, orc, W):
    events = _small_ensemble(W)
    steps = 3
    singles = [_single(hy, w, "fp64", steps) for w in events]
    results = []
    for v in range(3):
        b = _batch(hy, W, events, "fp64", (v, v, v))
        hy.hydro_batch_step(b, steps)
        results.append([hy.hydro_batch_read_fields(b, e) for e in range(len(events))])
        for e in range(len(events)):
            d = hy.hydro_batch_get_diag(b, e)
            assert d["jet_cells"] == singles[e][1]["jet_cells"]
            assert d["dep_E"] == singles[e][1]["dep_E"]
        hy.hydro_batch_destroy(b)
    for e, w in enumerate(events):
        for v in range(3):
            assert np.array_equal(results[v][e], singles[e][0]), (e, v)
        U0 = orc.prim_to_cons(W.ellipsoidal_primitives(w))
        O, od = orc.run(oracle_config(orc, w), U0, steps, oracle_jets(orc, w))
        err = norm_rel_err(results[0][e], O)
        assert np.all(err <= 1e-10), (e, err)


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_reduced_precision_batch_is_bitwise_single_grid(hy, W, precision):
    events = _small_ensemble(W)
    steps = 4
    b = _batch(hy, W, events, precision, (1, 2, 0))
    hy.hydro_batch_step(b, steps)
    for e, w in enumerate(events):
        got = hy.hydro_batch_read_fields(b, e)
        want, _ = _single(hy, w, precision, steps)
        assert np.array_equal(got, want), e


@pytest.mark.parametrize("precision,variants", [("fp64", (0, 0, 0)), ("fp32", (1, 0, 0)), ("fp32", (2, 1, 2)),
                                                ("mixed", (1, 2, 0))])
def test_batch_with_tensor_maps_is_bitwise_single_grid(hy, W, precision, variants):
    """Every row pitch and field offset a multiple of 16 bytes: the persistent
    kernels stage, fetch and store through per-grid tensor maps (and carry their
    mbarrier phases across tiles of different grids) and still match the grids
    stepped alone bit for bit."""
    shapes = [(16, 20, 12), (24, 16, 18), (36, 17, 9), (8, 40, 20), (72, 5, 6), (40, 40, 40)]
    events = []
    for k, n in enumerate(shapes):
        jets = W.seeded_jets(200 + k, 1 + k % 3, 0.5, 1.0)
        events.append(replace(W.ELLIPSOIDAL_32, n=n, sigma=(0.7 + 0.1 * k, 0.9, 1.1), e0=20.0 + 5 * k, jets=jets))
    steps = 3
    b = _batch(hy, W, events, precision, variants)
    hy.hydro_batch_step(b, steps)
    for e, w in enumerate(events):
        got = hy.hydro_batch_read_fields(b, e)
        want, d = _single(hy, w, precision, steps)
        assert np.array_equal(got, want), e
        assert hy.hydro_batch_get_diag(b, e)["jet_cells"] == d["jet_cells"]
    hy.hydro_batch_destroy(b)


def test_autotune_picks_a_shape_and_leaves_the_state_alone(hy, W):
    events = _small_ensemble(W)
    b = _batch(hy, W, events, "fp32")
    before = [hy.hydro_batch_read_fields(b, e) for e in range(len(events))]
    choice, ms = hy.hydro_batch_autotune(b)
    assert all(0 <= c < 3 for c in choice)
    assert all(t > 0 for row in ms for t in row)
    for d in range(3):
        assert ms[d][choice[d]] == min(ms[d])
    for e in range(len(events)):
        assert np.array_equal(hy.hydro_batch_read_fields(b, e), before[e])
    hy.hydro_batch_step(b, 2)
    for e, w in enumerate(events):
        want, _ = _single(hy, w, "fp32", 2)
        assert np.array_equal(hy.hydro_batch_read_fields(b, e), want)


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_persistent_and_per_tile_launches_are_bitwise_equal(hy, W, precision):
    """The two launch forms of a batched sweep (one block per tile; persistent
    blocks walking the tile list) run the same tiles with the same arithmetic:
    the states after 3 steps are bitwise equal, and the tuning query reports the
    form that was set."""
    events = _small_ensemble(W)
    res = []
    for per_tile in ((1, 1, 1), (0, 0, 0)):
        b = _batch(hy, W, events, precision)
        hy.hydro_batch_set_launch(b, per_tile)
        assert hy.hydro_batch_get_tuning(b)[1] == per_tile
        hy.hydro_batch_step(b, 3)
        res.append([hy.hydro_batch_read_fields(b, e) for e in range(len(events))])
        hy.hydro_batch_destroy(b)
    for a, c in zip(*res):
        assert np.array_equal(a, c)


def test_graph_replay_across_chunks_matches_one_call(hy, W):
    """70 steps run as one 64-step graph plus a 6-step graph; the same 70 steps
    in 7 calls of 10 replay one cached 10-step graph."""
    events = _small_ensemble(W)[:3]
    b1 = _batch(hy, W, events, "fp32")
    hy.hydro_batch_step(b1, 70)
    b2 = _batch(hy, W, events, "fp32")
    for _ in range(7):
        hy.hydro_batch_step(b2, 10)
    for e in range(len(events)):
        assert np.array_equal(hy.hydro_batch_read_fields(b1, e), hy.hydro_batch_read_fields(b2, e))
        assert hy.hydro_batch_get_diag(b1, e)["steps"] == 70


def test_full_64_event_ensemble_fp32_50_steps(hy, W):
    """The batched configuration: 64 uneven grids (edges 64-160), 1-4 jets each,
    50 steps in FP32, autotuned tiles.  Every grid stays finite and
    subluminal (jets near the hot centre push single cells against the |M| < E
    cap, which the floors count); three sampled grids match their single-grid
    runs bitwise."""
    E = W.ENSEMBLE_64
    b = _batch(hy, W, E.events, "fp32")
    hy.hydro_batch_autotune(b)
    hy.hydro_batch_step(b, E.steps)
    for e in range(len(E.events)):
        d = hy.hydro_batch_get_diag(b, e)
        assert d["status"] == 0 and d["max_speed"] <= 1.0 + 1e-6, (e, d)
    edges = [w.n[0] for w in E.events]
    for e in (edges.index(64), edges.index(96), edges.index(160)):
        got = hy.hydro_batch_read_fields(b, e)
        want, _ = _single(hy, E.events[e], "fp32", E.steps)
        assert np.isfinite(got).all()
        assert np.array_equal(got, want), e
