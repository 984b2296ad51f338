"""FP64 CPU oracle of the relativistic-hydro RK3 step (test infrastructure only).

The arithmetic lives in ``hydro_oracle.c`` (plain loops, FP64, no FMA
contraction); this module compiles it with gcc and marshals numpy arrays over
ctypes.  Only the tests, the smoke entry point and the benchmark's CPU-baseline
leg may import this package: the CUDA library never does, and the two share no
code.  Each exported function cites the passage of arXiv:1511.02137 it follows
in the C source.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hydro_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

MAX_JETS = 16


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (gcc, OpenMP, no FMA)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", "-Wall", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


class _Config(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("dx", ctypes.c_double), ("dt", ctypes.c_double), ("t0", ctypes.c_double),
                ("boundary", ctypes.c_int32), ("order", ctypes.c_int32), ("fluid", ctypes.c_int32),
                ("nthreads", ctypes.c_int32),
                ("k_rad", ctypes.c_double), ("k_coll", ctypes.c_double), ("cr_over_cf", ctypes.c_double),
                ("hbarc", ctypes.c_double), ("dof", ctypes.c_double),
                ("e_floor", ctypes.c_double), ("weno_eps", ctypes.c_double)]


class _Jet(ctypes.Structure):
    _fields_ = [("x0", ctypes.c_double * 3), ("n", ctypes.c_double * 3), ("t_start", ctypes.c_double)]


class _Diag(ctypes.Structure):
    _fields_ = [("dep_E", ctypes.c_double), ("dep_M", ctypes.c_double * 3), ("max_speed", ctypes.c_double),
                ("floor_hits", ctypes.c_int64), ("jet_cell", (ctypes.c_int32 * 3) * MAX_JETS)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        lib.orc_prim_to_cons.argtypes = [ctypes.c_int64, dp, dp]
        lib.orc_prim_to_cons.restype = None
        lib.orc_cons_to_prim.argtypes = [ctypes.c_int64, dp, ctypes.c_double, dp]
        lib.orc_cons_to_prim.restype = ctypes.c_int64
        lib.orc_char_speeds.argtypes = [dp, ctypes.c_int32, dp]
        lib.orc_char_speeds.restype = None
        lib.orc_weno7.argtypes = [dp, ctypes.c_double, dp, dp, dp]
        lib.orc_weno7.restype = ctypes.c_double
        lib.orc_weno5.argtypes = [dp, ctypes.c_double, dp, dp, dp]
        lib.orc_weno5.restype = ctypes.c_double
        lib.orc_temperature.argtypes = [ctypes.POINTER(_Config), ctypes.c_double]
        lib.orc_temperature.restype = ctypes.c_double
        lib.orc_jet_dEdx.argtypes = [ctypes.POINTER(_Config), ctypes.c_double, ctypes.c_double]
        lib.orc_jet_dEdx.restype = ctypes.c_double
        lib.orc_jet_normalize.argtypes = [dp, dp]
        lib.orc_jet_normalize.restype = ctypes.c_int32
        lib.orc_jet_cell.argtypes = [ctypes.POINTER(_Config), ctypes.POINTER(_Jet), ctypes.c_double,
                                     ctypes.POINTER(ctypes.c_int32), dp]
        lib.orc_jet_cell.restype = ctypes.c_int32
        lib.orc_rhs.argtypes = [ctypes.POINTER(_Config), dp, ctypes.c_double, ctypes.POINTER(_Jet), ctypes.c_int32,
                                dp, ctypes.POINTER(ctypes.c_int64), dp]
        lib.orc_rhs.restype = ctypes.c_int32
        lib.orc_run.argtypes = [ctypes.POINTER(_Config), dp, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(_Jet),
                                ctypes.c_int32, ctypes.POINTER(_Diag)]
        lib.orc_run.restype = ctypes.c_int32
        lib.orc_max_threads.argtypes = []
        lib.orc_max_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclass
class Config:
    """Grid, scheme and jet-law parameters (units: fm, fm/c, GeV)."""
    nx: int
    ny: int
    nz: int
    dx: float = 0.1
    dt: float = 0.02
    t0: float = 1.0
    boundary: str = "outflow"      # or "periodic"
    order: int = 7                 # WENO order, 7 or 5
    fluid: bool = True             # False: jet source only (flux divergence off)
    nthreads: int = 0
    k_rad: float = 4.0
    k_coll: float = 2.5
    cr_over_cf: float = 1.0
    hbarc: float = 0.1973
    dof: float = 47.5
    e_floor: float = 3e-11
    weno_eps: float = 1e-6

    def _c(self) -> _Config:
        return _Config(self.nx, self.ny, self.nz, self.dx, self.dt, self.t0,
                       {"outflow": 0, "periodic": 1}[self.boundary], self.order, 1 if self.fluid else 0,
                       self.nthreads, self.k_rad, self.k_coll, self.cr_over_cf, self.hbarc, self.dof,
                       self.e_floor, self.weno_eps)


@dataclass
class Jet:
    x0: tuple
    direction: tuple
    t_start: float

    def _c(self) -> _Jet:
        n = jet_normalize(self.direction)
        return _Jet((ctypes.c_double * 3)(*self.x0), (ctypes.c_double * 3)(*n), self.t_start)


@dataclass
class Diag:
    dep_E: float = 0.0
    dep_M: tuple = (0.0, 0.0, 0.0)
    max_speed: float = 0.0
    floor_hits: int = 0
    jet_cells: list = field(default_factory=list)


def max_threads() -> int:
    return _load().orc_max_threads()


def prim_to_cons(prim: np.ndarray) -> np.ndarray:
    """prim[5, ...] = (e, u^x, u^y, u^z, n) -> cons[5, ...] = (E, M^x, M^y, M^z, R)."""
    prim = np.ascontiguousarray(prim, dtype=np.float64)
    assert prim.shape[0] == 5
    out = np.empty_like(prim)
    _load().orc_prim_to_cons(prim[0].size, _ptr(prim), _ptr(out))
    return out


def cons_to_prim(cons: np.ndarray, e_floor: float = 3e-11):
    """cons[5, ...] -> (prim[6, ...] = (e, v^x, v^y, v^z, p, n), floor hits)."""
    cons = np.ascontiguousarray(cons, dtype=np.float64)
    assert cons.shape[0] == 5
    out = np.empty((6,) + cons.shape[1:], dtype=np.float64)
    hits = _load().orc_cons_to_prim(cons[0].size, _ptr(cons), e_floor, _ptr(out))
    return out, int(hits)


def char_speeds(v, d: int):
    """(lambda_minus, lambda_plus) along axis d for 3-velocity v."""
    v = np.ascontiguousarray(v, dtype=np.float64)
    out = np.empty(2)
    _load().orc_char_speeds(_ptr(v), d, _ptr(out))
    return float(out[0]), float(out[1])


def weno7(f, eps: float = 1e-6):
    """Reconstruction at x_{i+1/2} from f_{i-3..i+3}: (value, candidates, betas, weights)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    assert f.shape == (7,)
    q, b, w = np.empty(4), np.empty(4), np.empty(4)
    val = _load().orc_weno7(_ptr(f), eps, _ptr(q), _ptr(b), _ptr(w))
    return val, q, b, w


def weno5(f, eps: float = 1e-6):
    """Reconstruction at x_{i+1/2} from f_{i-2..i+2}: (value, candidates, betas, weights)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    assert f.shape == (5,)
    q, b, w = np.empty(3), np.empty(3), np.empty(3)
    val = _load().orc_weno5(_ptr(f), eps, _ptr(q), _ptr(b), _ptr(w))
    return val, q, b, w


def temperature(cfg: Config, e: float) -> float:
    c = cfg._c()
    return _load().orc_temperature(ctypes.byref(c), e)


def jet_dEdx(cfg: Config, T: float, ell: float) -> float:
    c = cfg._c()
    return _load().orc_jet_dEdx(ctypes.byref(c), T, ell)


def jet_normalize(direction):
    d = np.ascontiguousarray(direction, dtype=np.float64)
    n = np.empty(3)
    if _load().orc_jet_normalize(_ptr(d), _ptr(n)) != 0:
        raise ValueError("zero jet direction")
    return tuple(float(x) for x in n)


def jet_cell(cfg: Config, jet: Jet, t: float):
    """(inside, (i, j, k), ell) of a jet at time t."""
    c, j = cfg._c(), jet._c()
    ijk = (ctypes.c_int32 * 3)()
    ell = ctypes.c_double()
    inside = _load().orc_jet_cell(ctypes.byref(c), ctypes.byref(j), t, ijk, ctypes.byref(ell))
    return bool(inside), (ijk[0], ijk[1], ijk[2]), ell.value


def _jets(jets):
    jets = list(jets or [])
    if len(jets) > MAX_JETS:
        raise ValueError("too many jets")
    arr = (_Jet * max(1, len(jets)))()
    for i, j in enumerate(jets):
        arr[i] = j._c()
    return arr, len(jets)


def rhs(cfg: Config, U: np.ndarray, t: float, jets=()):
    """L(U) = -div F + S at time t; U[5, nz, ny, nx].  Returns (L, floor hits, max speed)."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    assert U.shape == (5, cfg.nz, cfg.ny, cfg.nx)
    L = np.empty_like(U)
    arr, nj = _jets(jets)
    c = cfg._c()
    hits = ctypes.c_int64()
    vmax = ctypes.c_double()
    rc = _load().orc_rhs(ctypes.byref(c), _ptr(U), t, arr, nj, _ptr(L), ctypes.byref(hits), ctypes.byref(vmax))
    if rc != 0:
        raise RuntimeError("orc_rhs failed: %d" % rc)
    return L, int(hits.value), float(vmax.value)


def run(cfg: Config, U: np.ndarray, nsteps: int, jets=(), step0: int = 0):
    """nsteps SSP-RK3 steps from step index step0; returns (U_new, Diag)."""
    U = np.array(U, dtype=np.float64, order="C", copy=True)
    assert U.shape == (5, cfg.nz, cfg.ny, cfg.nx)
    arr, nj = _jets(jets)
    c = cfg._c()
    d = _Diag()
    for jn in range(MAX_JETS):
        for a in range(3):
            d.jet_cell[jn][a] = -1
    rc = _load().orc_run(ctypes.byref(c), _ptr(U), step0, nsteps, arr, nj, ctypes.byref(d))
    if rc != 0:
        raise RuntimeError("orc_run failed: %d" % rc)
    diag = Diag(dep_E=d.dep_E, dep_M=tuple(d.dep_M), max_speed=d.max_speed, floor_hits=int(d.floor_hits),
                jet_cells=[tuple(d.jet_cell[i]) for i in range(nj)])
    return U, diag
