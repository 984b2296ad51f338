"""Seeded synthetic inputs: the ellipsoidal-flow initial state and jet lists.

This module only builds inputs (primitive fields and jet start points); it
holds none of the method's arithmetic, so the CUDA path and the CPU oracle can
both be fed from it.  The profile follows the setup of Sec. 2 (ellipsoidal
flow started at t0 = 1 fm/c) with the run parameters of the Fig. 3 caption
(dx = 0.1 fm, dt = 0.02 fm/c, 256^3 cells, p = e/3):

    e(x)  = e0 * exp(-x^2/2sx^2 - y^2/2sy^2 - z^2/2sz^2) + bg * e0
    u^i   = H_i x_i          (spatial four-velocity)
    n(x)  = n0 * e(x) / e0   (passive charge density)

sampled at cell centres x_i = (i + 1/2 - N/2) dx.  Random draws (jet start
points and directions) use splitmix64 (Steele, Lea and Flood, OOPSLA 2014).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np


@dataclass(frozen=True)
class JetSpec:
    x0: tuple          # start point [fm]
    direction: tuple   # need not be normalised
    t_start: float     # [fm/c]


@dataclass(frozen=True)
class Workload:
    name: str
    n: tuple                     # (nx, ny, nz)
    steps: int
    dx: float = 0.1
    dt: float = 0.02
    t0: float = 1.0
    e0: float = 30.0             # GeV/fm^3
    sigma: tuple = (4.0, 5.0, 6.0)
    hubble: tuple = (0.05, 0.04, 0.03)
    background: float = 1e-3     # fraction of e0
    n0: float = 0.16             # fm^-3
    jets: tuple = field(default_factory=tuple)

    @property
    def cells(self) -> int:
        return self.n[0] * self.n[1] * self.n[2]


def ellipsoidal_primitives(w: Workload) -> np.ndarray:
    """Primitive fields [5, nz, ny, nx] = (e, u^x, u^y, u^z, n), float64."""
    nx, ny, nz = w.n
    x = (np.arange(nx) + 0.5 - nx / 2) * w.dx
    y = (np.arange(ny) + 0.5 - ny / 2) * w.dx
    z = (np.arange(nz) + 0.5 - nz / 2) * w.dx
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    sx, sy, sz = w.sigma
    e = w.e0 * np.exp(-X**2 / (2 * sx**2) - Y**2 / (2 * sy**2) - Z**2 / (2 * sz**2)) + w.background * w.e0
    prim = np.empty((5, nz, ny, nx), dtype=np.float64)
    prim[0] = e
    prim[1] = w.hubble[0] * X
    prim[2] = w.hubble[1] * Y
    prim[3] = w.hubble[2] * Z
    prim[4] = w.n0 * e / w.e0
    return prim


class SplitMix64:
    """splitmix64 counter generator; uniform doubles from the top 53 bits."""

    MASK = (1 << 64) - 1

    def __init__(self, seed: int):
        self.state = seed & self.MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & self.MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & self.MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & self.MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))


def seeded_jets(seed: int, count: int, radius: float, t_start: float) -> tuple:
    """Jets with start points uniform in the ball |r| < radius and isotropic
    directions (cos(theta) uniform in [-1, 1], phi uniform in [0, 2 pi))."""
    rng = SplitMix64(seed)
    jets = []
    for _ in range(count):
        r = radius * rng.uniform() ** (1.0 / 3.0)
        ct = 2.0 * rng.uniform() - 1.0
        ph = 2.0 * math.pi * rng.uniform()
        st = math.sqrt(max(0.0, 1.0 - ct * ct))
        pos = (r * st * math.cos(ph), r * st * math.sin(ph), r * ct)
        ct = 2.0 * rng.uniform() - 1.0
        ph = 2.0 * math.pi * rng.uniform()
        st = math.sqrt(max(0.0, 1.0 - ct * ct))
        dirn = (st * math.cos(ph), st * math.sin(ph), ct)
        jets.append(JetSpec(pos, dirn, t_start))
    return tuple(jets)


# Small parity case: 32^3, 10 steps, sigmas (0.8, 1.0, 1.2) fm, jet from (-1, 0, 0) fm along +x.
ELLIPSOIDAL_32 = Workload(
    name="ellipsoidal-flow 32^3, 10 RK3 steps, 1 jet",
    n=(32, 32, 32), steps=10, sigma=(0.8, 1.0, 1.2),
    jets=(JetSpec((-1.0, 0.0, 0.0), (1.0, 0.0, 0.0), 1.0),))

# The paper's run size (Fig. 3 caption): 256^3, t0 = 1 -> 2.4 fm/c (70 steps), jet from (-8, 0, 0) fm along +x.
ELLIPSOIDAL_256 = Workload(
    name="ellipsoidal-flow 256^3, 70 RK3 steps, 1 jet",
    n=(256, 256, 256), steps=70, sigma=(4.0, 5.0, 6.0),
    jets=(JetSpec((-8.0, 0.0, 0.0), (1.0, 0.0, 0.0), 1.0),))

# Mixed-precision study: 256^3, 70 steps, 3 seeded jets (start |r| < 6 fm, isotropic).
ELLIPSOIDAL_256_3JETS = replace(
    ELLIPSOIDAL_256, name="ellipsoidal-flow 256^3, 70 RK3 steps, 3 seeded jets",
    jets=seeded_jets(1511, 3, 6.0, 1.0))


def scaled(w: Workload, n: int, steps: int | None = None) -> Workload:
    """Same profile on an n^3 grid with the same dx (a sub-volume of the full run)."""
    return replace(w, n=(n, n, n), steps=w.steps if steps is None else steps,
                   name=f"{w.name} [sub-grid {n}^3]")


@dataclass(frozen=True)
class Ensemble:
    name: str
    events: tuple
    steps: int

    @property
    def cells(self) -> int:
        return sum(w.cells for w in self.events)


def seeded_ensemble(seed: int, count: int, edges=(64, 96, 128, 160), e0=(10.0, 50.0), sigma=(2.0, 6.0),
                    jets=(1, 4), steps: int = 50) -> Ensemble:
    """Events of uneven cube grids (edge drawn from `edges`), e0 and the three
    sigmas drawn uniformly from their ranges, 1-4 jets each starting uniformly
    in the ball of radius 0.4 x the half-width of the grid with isotropic
    directions, t_start = t0."""
    rng = SplitMix64(seed)
    events = []
    for k in range(count):
        edge = edges[min(int(rng.uniform() * len(edges)), len(edges) - 1)]
        e0k = e0[0] + (e0[1] - e0[0]) * rng.uniform()
        sig = tuple(sigma[0] + (sigma[1] - sigma[0]) * rng.uniform() for _ in range(3))
        nj = jets[0] + min(int(rng.uniform() * (jets[1] - jets[0] + 1)), jets[1] - jets[0])
        radius = 0.4 * 0.5 * edge * 0.1
        js = seeded_jets(rng.next_u64(), nj, radius, 1.0)
        events.append(Workload(name=f"event {k}: {edge}^3", n=(edge, edge, edge), steps=steps, e0=e0k, sigma=sig,
                               jets=js))
    return Ensemble(name=f"{count}-event ensemble, edges {edges}, {steps} RK3 steps", events=tuple(events),
                    steps=steps)


# Batched ensemble: 64 events, cube edges from {64, 96, 128, 160}, e0 in [10, 50] GeV/fm^3,
# sigmas in [2, 6] fm, 1-4 jets each, 50 steps.
ENSEMBLE_64 = seeded_ensemble(15114, 64)
