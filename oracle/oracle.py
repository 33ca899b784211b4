"""Python handle on the GBEES oracle -- TEST INFRASTRUCTURE ONLY.

The oracle is a plain FP64 CPU implementation of the GBEES
propagation step (DCU, Eq. 7; CTU, Algorithm 1; high-resolution correction;
CFL time step, Eq. 8; directional grow and prune, Sec. 3.3 / Algorithm 3;
Bayesian update, Eq. 4), written in `gbees_oracle.cpp`. Only the tests, the
smoke check and the CPU-baseline leg of the benchmark may import this module;
the product library never does.

`build()` compiles the C++ source with g++ into `oracle/_lib/`; `Oracle` wraps
one grid. Every function named here maps one-to-one onto an `orc_*` symbol.
`compile_variant()` builds a copy of the source with one text replacement (for
the tests that plant a mistake in the oracle and check that a pin catches it).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass
from typing import Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gbees_oracle.cpp")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "libgbees_oracle.so")
_lock = threading.Lock()
_handle = None

DYN_CONSTANT, DYN_LINEAR, DYN_LORENZ63, DYN_LORENZ63_SHIFTED, DYN_LORENZ96 = range(5)
LIM_MC, LIM_NONE, LIM_LW = range(3)


class _Config(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32),
        ("dynamics", ctypes.c_int32),
        ("params", ctypes.c_double * 64),
        ("h", ctypes.c_double * 6),
        ("x0", ctypes.c_double * 6),
        ("thr_rel", ctypes.c_double),
        ("cfl", ctypes.c_double),
        ("prune_interval", ctypes.c_int32),
        ("limiter", ctypes.c_int32),
    ]


class _Stats(ctypes.Structure):
    _fields_ = [
        ("steps", ctypes.c_int64),
        ("cell_updates", ctypes.c_int64),
        ("t", ctypes.c_double),
        ("last_dt", ctypes.c_double),
        ("total_steps", ctypes.c_int64),
    ]


_FLAGS = ["-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC"]


def _compile(src: str, out: str, check_output: bool = False) -> None:
    """g++ with the oracle's flags, with OpenMP when the compiler has it (the
    results do not depend on the number of threads)."""
    r = subprocess.run(["g++", *_FLAGS, "-fopenmp", src, "-o", out], capture_output=True, text=True)
    if r.returncode != 0:
        subprocess.run(["g++", *_FLAGS, src, "-o", out], check=True, capture_output=check_output)


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_lib (g++, -O2, no fused multiply-add)."""
    with _lock:
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
            return _LIB
        os.makedirs(_LIBDIR, exist_ok=True)
        tmp = _LIB + f".tmp{os.getpid()}"
        _compile(_SRC, tmp)
        os.replace(tmp, _LIB)
        return _LIB


def compile_variant(old: str, new: str, out_path: str) -> str:
    """Compile the oracle source with `old` (which must occur exactly once)
    replaced by `new` into out_path; the flags are those of build()."""
    src = open(_SRC).read()
    if src.count(old) != 1:
        raise ValueError(f"the text to replace occurs {src.count(old)} times")
    tmp_src = out_path + ".cpp"
    with open(tmp_src, "w") as f:
        f.write(src.replace(old, new))
    _compile(tmp_src, out_path, check_output=True)
    return out_path


def _lib():
    global _handle
    if _handle is None:
        # GBEES_ORACLE_LIB names another build of the oracle source: the
        # mutation tests load copies with one planted mistake through it
        path = os.environ.get("GBEES_ORACLE_LIB") or build()
        L = ctypes.CDLL(path)
        vp, d, i32, i64 = ctypes.c_void_p, ctypes.c_double, ctypes.c_int32, ctypes.c_int64
        P = ctypes.POINTER
        sig = {
            "orc_create": (vp, [P(_Config)]),
            "orc_destroy": (None, [vp]),
            "orc_last_error": (ctypes.c_char_p, [vp]),
            "orc_init_gaussian": (ctypes.c_int, [vp, P(d), P(d), d]),
            "orc_init_cells": (ctypes.c_int, [vp, P(i32), P(d), i64, d, i64]),
            "orc_propagate": (ctypes.c_int, [vp, d, P(_Stats)]),
            "orc_propagate_steps": (ctypes.c_int, [vp, d, i64, P(_Stats)]),
            "orc_correct_gaussian": (ctypes.c_int, [vp, P(d), P(d), P(i32), i32]),
            "orc_count": (i64, [vp]),
            "orc_read_cells": (i64, [vp, P(i32), P(d), i64]),
            "orc_moments": (None, [vp, P(d), P(d)]),
            "orc_ctu_step": (ctypes.c_int, [vp, d]),
            "orc_grow": (ctypes.c_int, [vp]),
            "orc_prune": (ctypes.c_int, [vp]),
            "orc_normalise": (ctypes.c_int, [vp]),
            "orc_cfl_dt": (d, [vp]),
            "orc_face_velocity": (d, [vp, P(i32), i32]),
            "orc_drift": (d, [vp, P(d), i32]),
            "orc_downwind": (i32, [vp, P(i32), P(i32), i32]),
            "orc_exact_sum": (d, [P(d), i64]),
            "orc_ctu_sample": (ctypes.c_int, [vp, d, P(i32), i64, P(d)]),
            "orc_time": (d, [vp]),
            "orc_set_threads": (i32, [i32]),
            "orc_steps": (i64, [vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _handle = L
    return _handle


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def set_threads(k: int = 0) -> int:
    """Threads of the oracle's parallel loops (0: the OpenMP default, all
    cores); returns the number in use. The results do not depend on it."""
    return int(_lib().orc_set_threads(int(k)))


def exact_sum(x: Sequence[float]) -> float:
    a = np.ascontiguousarray(x, dtype=np.float64)
    return _lib().orc_exact_sum(_dp(a), a.size)


@dataclass
class OracleStats:
    steps: int
    cell_updates: int
    t: float
    last_dt: float
    total_steps: int


class OracleError(RuntimeError):
    pass


class Oracle:
    """One GBEES grid propagated by the CPU oracle."""

    def __init__(self, n: int, dynamics: int, params: Sequence[float], h: Sequence[float],
                 x0: Sequence[float], thr_rel: float = 1e-7, cfl: float = 0.9,
                 prune_interval: int = 20, limiter: int = LIM_MC):
        c = _Config()
        c.n, c.dynamics = n, dynamics
        for k, v in enumerate(params):
            c.params[k] = float(v)
        for k in range(n):
            c.h[k] = float(h[k])
            c.x0[k] = float(x0[k])
        c.thr_rel, c.cfl = float(thr_rel), float(cfl)
        c.prune_interval, c.limiter = int(prune_interval), int(limiter)
        self.n = n
        self._cfg = c
        self._h = _lib().orc_create(ctypes.byref(c))
        if not self._h:
            raise OracleError("invalid oracle configuration")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _lib().orc_destroy(h)
            self._h = None

    def _check(self, rc: int):
        if rc != 0:
            raise OracleError(f"oracle error {rc}: {_lib().orc_last_error(self._h).decode()}")

    def init_gaussian(self, mean, cov, t0: float = 0.0):
        m = np.ascontiguousarray(mean, dtype=np.float64)
        C = np.ascontiguousarray(cov, dtype=np.float64)
        self._check(_lib().orc_init_gaussian(self._h, _dp(m), _dp(C), float(t0)))

    def init_cells(self, idx, p, t0: float = 0.0, step0: int = 0):
        I = np.ascontiguousarray(idx, dtype=np.int32).reshape(-1, self.n)
        P = np.ascontiguousarray(p, dtype=np.float64)
        self._check(_lib().orc_init_cells(self._h, _ip(I), _dp(P), I.shape[0], float(t0), int(step0)))

    def propagate(self, t_end: float, max_steps: int = -1) -> OracleStats:
        """Steps towards t_end until it is reached (or max_steps steps, if >= 0)."""
        st = _Stats()
        self._check(_lib().orc_propagate_steps(self._h, float(t_end), int(max_steps), ctypes.byref(st)))
        return OracleStats(st.steps, st.cell_updates, st.t, st.last_dt, st.total_steps)

    def correct_gaussian(self, y, R, H_idx):
        yy = np.ascontiguousarray(y, dtype=np.float64)
        RR = np.ascontiguousarray(R, dtype=np.float64)
        HH = np.ascontiguousarray(H_idx, dtype=np.int32)
        self._check(_lib().orc_correct_gaussian(self._h, _dp(yy), _dp(RR), _ip(HH), HH.size))

    def count(self) -> int:
        return int(_lib().orc_count(self._h))

    def read_cells(self):
        N = self.count()
        idx = np.zeros((N, self.n), dtype=np.int32)
        p = np.zeros(N, dtype=np.float64)
        _lib().orc_read_cells(self._h, _ip(idx), _dp(p), N)
        return idx, p

    def moments(self):
        mean = np.zeros(self.n)
        cov = np.zeros((self.n, self.n))
        _lib().orc_moments(self._h, _dp(mean), _dp(cov))
        return mean, cov

    def ctu_step(self, dt: float):
        self._check(_lib().orc_ctu_step(self._h, float(dt)))

    def grow(self):
        self._check(_lib().orc_grow(self._h))

    def prune(self):
        self._check(_lib().orc_prune(self._h))

    def normalise(self):
        self._check(_lib().orc_normalise(self._h))

    def cfl_dt(self) -> float:
        return float(_lib().orc_cfl_dt(self._h))

    def face_velocity(self, X, j: int) -> float:
        a = np.ascontiguousarray(X, dtype=np.int32)
        return float(_lib().orc_face_velocity(self._h, _ip(a), int(j)))

    def drift(self, x, j: int) -> float:
        a = np.ascontiguousarray(x, dtype=np.float64)
        return float(_lib().orc_drift(self._h, _dp(a), int(j)))

    def downwind(self, X):
        a = np.ascontiguousarray(X, dtype=np.int32)
        out = np.zeros((64, self.n), dtype=np.int32)
        k = _lib().orc_downwind(self._h, _ip(a), _ip(out), 64)
        return [tuple(int(v) for v in row) for row in out[:k]]

    def ctu_sample(self, dt: float, idx) -> np.ndarray:
        I = np.ascontiguousarray(idx, dtype=np.int32).reshape(-1, self.n)
        out = np.zeros(I.shape[0])
        self._check(_lib().orc_ctu_sample(self._h, float(dt), _ip(I), I.shape[0], _dp(out)))
        return out

    @property
    def t(self) -> float:
        return float(_lib().orc_time(self._h))

    @property
    def steps(self) -> int:
        return int(_lib().orc_steps(self._h))
