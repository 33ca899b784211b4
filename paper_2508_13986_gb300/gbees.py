"""Thin Python binding of the GBEES C ABI (include/gbees.h).

The module-level functions carry the C names and only marshal arguments
(ctypes); every step of the method runs in the CUDA library
`_lib/libgbees_gb300.so`. PyTorch provides the device workspace and the CUDA
stream. Loading fails with an error when the library has not been built: there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import functools
import os
from dataclasses import dataclass
from typing import Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libgbees_gb300.so")

GBEES_OK, GBEES_EINVAL, GBEES_ECAPACITY, GBEES_EKEYRANGE = 0, -1, -2, -3
GBEES_EDEGENERATE, GBEES_ECUDA, GBEES_ETIMEOUT, GBEES_ETABLE = -4, -5, -6, -7
STATUS_NAMES = {0: "OK", -1: "EINVAL", -2: "ECAPACITY", -3: "EKEYRANGE", -4: "EDEGENERATE", -5: "ECUDA",
                -6: "ETIMEOUT", -7: "ETABLE"}
GBEES_DYN_CONSTANT, GBEES_DYN_LINEAR, GBEES_DYN_LORENZ63, GBEES_DYN_LORENZ63_SHIFTED, GBEES_DYN_LORENZ96 = range(5)
GBEES_LIM_MC, GBEES_LIM_NONE, GBEES_LIM_LW = range(3)
GBEES_FP64, GBEES_FP32 = 0, 1
GBEES_LAUNCH_AUTO, GBEES_LAUNCH_PERSISTENT, GBEES_LAUNCH_GRAPH, GBEES_LAUNCH_DIRECT = range(4)
GBEES_ORDER_KEY, GBEES_ORDER_MORTON, GBEES_ORDER_NONE, GBEES_ORDER_KEY_MIXED, GBEES_ORDER_ROW_MORTON = range(5)


class gbees_config(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32),
        ("dynamics", ctypes.c_int32),
        ("params", ctypes.c_double * 64),
        ("h", ctypes.c_double * 6),
        ("x0", ctypes.c_double * 6),
        ("thr_rel", ctypes.c_double),
        ("cfl", ctypes.c_double),
        ("prune_interval", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("limiter", ctypes.c_int32),
        ("probe_width", ctypes.c_int32),
        ("max_cells", ctypes.c_int64),
        ("table_factor", ctypes.c_double),
        ("launch_mode", ctypes.c_int32),
        ("storage_order", ctypes.c_int32),
        ("block_threads", ctypes.c_int32),
        ("persist_max_entries", ctypes.c_int64),
    ]


class gbees_stats(ctypes.Structure):
    _fields_ = [
        ("steps", ctypes.c_int64),
        ("cell_updates", ctypes.c_int64),
        ("t", ctypes.c_double),
        ("last_dt", ctypes.c_double),
        ("total_steps", ctypes.c_int64),
        ("n_cells", ctypes.c_int64),
        ("norm", ctypes.c_double),
        ("n_pool", ctypes.c_int64),
    ]


GBEES_NPHASES = 8
PHASE_NAMES = ("grow", "halo", "link", "faces", "apply", "prune", "correct", "other")
PERSIST_NAMES = ("grow", "halo", "link", "faces", "apply", "prune", "scalars")


class gbees_profile(ctypes.Structure):
    _fields_ = [
        ("launches", ctypes.c_int64 * GBEES_NPHASES),
        ("ms", ctypes.c_double * GBEES_NPHASES),
        ("timed", ctypes.c_int64 * GBEES_NPHASES),
        ("total_launches", ctypes.c_int64),
        ("fallback_lookups", ctypes.c_int64),
        ("persist_us", ctypes.c_double * 8),
        ("persist_steps", ctypes.c_int64),
        ("persist_ms", ctypes.c_double),
        ("persist_launches", ctypes.c_int64),
        ("persist_updates", ctypes.c_int64),
    ]


_P = ctypes.POINTER
_vp, _d, _i32, _i64 = ctypes.c_void_p, ctypes.c_double, ctypes.c_int32, ctypes.c_int64
_SIGNATURES = {
    "gbees_workspace_bytes": (ctypes.c_size_t, [_P(gbees_config)]),
    "gbees_create": (ctypes.c_int, [_P(gbees_config), _vp, ctypes.c_size_t, _vp, _P(_vp)]),
    "gbees_init_gaussian": (ctypes.c_int, [_vp, _P(_d), _P(_d), _d]),
    "gbees_init_cells": (ctypes.c_int, [_vp, _P(_i32), _P(_d), _i64, _d, _i64]),
    "gbees_propagate": (ctypes.c_int, [_vp, _d, _P(gbees_stats)]),
    "gbees_correct_gaussian": (ctypes.c_int, [_vp, _P(_d), _P(_d), _P(_i32), _i32]),
    "gbees_count": (ctypes.c_int, [_vp, _P(_i64)]),
    "gbees_read_cells": (ctypes.c_int, [_vp, _P(_i32), _P(_d), _i64, _P(_i64), _i32]),
    "gbees_moments": (ctypes.c_int, [_vp, _P(_d), _P(_d)]),
    "gbees_get_stats": (ctypes.c_int, [_vp, _P(gbees_stats)]),
    "gbees_get_status": (ctypes.c_int, [_vp]),
    "gbees_set_wait_limit": (ctypes.c_int, [_vp, _i64, _i32]),
    "gbees_set_batch_blocks": (ctypes.c_int, [_vp, _i32]),
    "gbees_set_persist_blocks": (ctypes.c_int, [_vp, _i32]),
    "gbees_profile_control": (ctypes.c_int, [_vp, _i32, _i32]),
    "gbees_profile_read": (ctypes.c_int, [_vp, _P(gbees_profile)]),
    "gbees_last_error": (ctypes.c_char_p, [_vp]),
    "gbees_destroy": (None, [_vp]),
    "gbees_propagate_cells_noalloc": (ctypes.c_int, [_P(gbees_config), _P(_i32), _P(_d), _i64, _d, _i64, _d, _vp,
                                                     _P(_i32), _P(_d), _i64, _P(_i64), _P(gbees_stats)]),
    "gbees_batch_workspace_bytes": (ctypes.c_size_t, [_i32]),
    "gbees_batch_propagate": (ctypes.c_int, [_P(_vp), _i32, _P(_d), _i64, _vp, ctypes.c_size_t, _P(gbees_stats)]),
}
GBEES_NOALLOC_SCRATCH_BYTES = 16 << 20

_lib = None


def load_library(path: str = LIB_PATH):
    """Load the CUDA library; raise if it is missing (no fallback path exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"GBEES CUDA library not built: {path} is missing "
                               "(run python -c 'import __graft_entry__ as g; g.build()')")
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _f(name):
    return getattr(load_library(), name)


# ---- the C entry points under their own names (argument marshalling only) ----

def gbees_workspace_bytes(cfg: gbees_config) -> int:
    return int(_f("gbees_workspace_bytes")(ctypes.byref(cfg)))


def gbees_create(cfg: gbees_config, d_workspace: int, nbytes: int, stream: int) -> Tuple[int, int]:
    out = _vp()
    rc = _f("gbees_create")(ctypes.byref(cfg), _vp(d_workspace), nbytes, _vp(stream), ctypes.byref(out))
    return rc, (out.value or 0)


def gbees_init_gaussian(ctx: int, mean: np.ndarray, cov: np.ndarray, t0: float) -> int:
    return _f("gbees_init_gaussian")(_vp(ctx), _dp(mean), _dp(cov), float(t0))


def gbees_init_cells(ctx: int, idx: np.ndarray, p: np.ndarray, t0: float, step0: int = 0) -> int:
    return _f("gbees_init_cells")(_vp(ctx), _ip(idx), _dp(p), int(p.shape[0]), float(t0), int(step0))


def gbees_propagate(ctx: int, t_end: float, stats: gbees_stats) -> int:
    return _f("gbees_propagate")(_vp(ctx), float(t_end), ctypes.byref(stats))


def gbees_correct_gaussian(ctx: int, y: np.ndarray, R: np.ndarray, H_idx: np.ndarray) -> int:
    return _f("gbees_correct_gaussian")(_vp(ctx), _dp(y), _dp(R), _ip(H_idx), int(H_idx.size))


def gbees_count(ctx: int) -> Tuple[int, int]:
    n = _i64()
    rc = _f("gbees_count")(_vp(ctx), ctypes.byref(n))
    return rc, int(n.value)


def gbees_read_cells(ctx: int, idx: np.ndarray, p: np.ndarray, sorted_: bool) -> Tuple[int, int]:
    n = _i64()
    rc = _f("gbees_read_cells")(_vp(ctx), _ip(idx), _dp(p), int(p.shape[0]), ctypes.byref(n), int(bool(sorted_)))
    return rc, int(n.value)


def gbees_moments(ctx: int, mean: np.ndarray, cov: np.ndarray) -> int:
    return _f("gbees_moments")(_vp(ctx), _dp(mean), _dp(cov))


def gbees_get_stats(ctx: int, stats: gbees_stats) -> int:
    return _f("gbees_get_stats")(_vp(ctx), ctypes.byref(stats))


def gbees_set_wait_limit(ctx: int, spins: int, extra_arrivals: int = 0) -> int:
    return int(_f("gbees_set_wait_limit")(_vp(ctx), int(spins), int(extra_arrivals)))


def gbees_set_batch_blocks(ctx: int, max_blocks: int) -> int:
    return int(_f("gbees_set_batch_blocks")(_vp(ctx), int(max_blocks)))


def gbees_set_persist_blocks(ctx: int, max_blocks: int) -> int:
    return int(_f("gbees_set_persist_blocks")(_vp(ctx), int(max_blocks)))


def gbees_get_status(ctx: int) -> int:
    return _f("gbees_get_status")(_vp(ctx))


def gbees_profile_control(ctx: int, enable: bool, reset: bool) -> int:
    return _f("gbees_profile_control")(_vp(ctx), int(bool(enable)), int(bool(reset)))


def gbees_profile_read(ctx: int, prof: gbees_profile) -> int:
    return _f("gbees_profile_read")(_vp(ctx), ctypes.byref(prof))


def gbees_last_error(ctx: int) -> str:
    s = _f("gbees_last_error")(_vp(ctx))
    return s.decode() if s else ""


def gbees_destroy(ctx: int) -> None:
    _f("gbees_destroy")(_vp(ctx))


def gbees_batch_workspace_bytes(count: int) -> int:
    return int(_f("gbees_batch_workspace_bytes")(int(count)))


def gbees_batch_propagate(ctxs: Sequence[int], t_end: np.ndarray, max_steps: int, d_scratch: int, nbytes: int,
                          stats) -> int:
    arr = (_vp * len(ctxs))(*[_vp(c) for c in ctxs])
    te = np.ascontiguousarray(t_end, dtype=np.float64)
    return _f("gbees_batch_propagate")(arr, len(ctxs), _dp(te), int(max_steps), _vp(d_scratch), nbytes, stats)


def gbees_propagate_cells_noalloc(cfg: gbees_config, idx: np.ndarray, p: np.ndarray, t0: float, step0: int,
                                  t_end: float, stream: int, idx_out: np.ndarray, p_out: np.ndarray,
                                  stats: gbees_stats) -> Tuple[int, int]:
    """Propagate host cells with the library's built-in device scratch (no
    allocation at all); see include/gbees.h. Returns (status, cell count)."""
    n = _i64()
    rc = _f("gbees_propagate_cells_noalloc")(ctypes.byref(cfg), _ip(idx), _dp(p), int(p.shape[0]), float(t0),
                                             int(step0), float(t_end), _vp(stream), _ip(idx_out), _dp(p_out),
                                             int(p_out.shape[0]), ctypes.byref(n), ctypes.byref(stats))
    return rc, int(n.value)


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_P(_d))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(_P(_i32))


# ---- a convenience wrapper that owns the workspace through PyTorch ----

class GbeesError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


@dataclass
class Stats:
    steps: int
    cell_updates: int
    t: float
    last_dt: float
    total_steps: int
    n_cells: int
    norm: float
    n_pool: int

    @classmethod
    def of(cls, s: gbees_stats) -> "Stats":
        return cls(s.steps, s.cell_updates, s.t, s.last_dt, s.total_steps, s.n_cells, s.norm, s.n_pool)


def make_config(n: int, dynamics: int, params: Sequence[float], h: Sequence[float], x0: Sequence[float],
                thr_rel: float = 1e-7, cfl: float = 0.9, prune_interval: int = 20, precision: int = GBEES_FP64,
                limiter: int = GBEES_LIM_MC, max_cells: int = 1 << 20, table_factor: float = 2.0,
                probe_width: int = 1, launch_mode: int = GBEES_LAUNCH_AUTO,
                storage_order: int = GBEES_ORDER_KEY, block_threads: int = 0,
                persist_max_entries: int = 0) -> gbees_config:
    c = gbees_config()
    c.n, c.dynamics = int(n), int(dynamics)
    for k, v in enumerate(params):
        c.params[k] = float(v)
    for k in range(min(n, 6, len(h), len(x0))):
        c.h[k] = float(h[k])
        c.x0[k] = float(x0[k])
    c.thr_rel, c.cfl = float(thr_rel), float(cfl)
    c.prune_interval, c.precision, c.limiter = int(prune_interval), int(precision), int(limiter)
    c.probe_width, c.max_cells, c.table_factor = int(probe_width), int(max_cells), float(table_factor)
    c.launch_mode = int(launch_mode)
    c.storage_order = int(storage_order)
    c.block_threads = int(block_threads)
    c.persist_max_entries = int(persist_max_entries)
    return c


def _on_device(fn):
    """Run a Grid method with the grid's device current (the library refuses
    calls made while another device is current)."""
    @functools.wraps(fn)
    def wrapper(self, *args, **kwargs):
        import torch

        with torch.cuda.device(self.device):
            return fn(self, *args, **kwargs)
    return wrapper


class Grid:
    """One GBEES grid on a CUDA device; the workspace is a torch uint8 tensor."""

    def __init__(self, cfg: gbees_config, device: str = "cuda:0", stream=None):
        import torch

        self.cfg = cfg
        self.n = cfg.n
        self.device = torch.device(device)
        nbytes = gbees_workspace_bytes(cfg)
        if nbytes == 0:
            raise GbeesError(GBEES_EINVAL, "invalid configuration")
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            rc, ctx = gbees_create(cfg, self.workspace.data_ptr(), nbytes, self.stream.cuda_stream)
        if rc != 0:
            raise GbeesError(rc, "gbees_create failed")
        self.ctx = ctx

    def close(self):
        if getattr(self, "ctx", 0):
            gbees_destroy(self.ctx)
            self.ctx = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc: int):
        if rc != 0:
            raise GbeesError(rc, gbees_last_error(self.ctx))

    @_on_device
    def init_gaussian(self, mean, cov, t0: float = 0.0):
        m = np.ascontiguousarray(mean, dtype=np.float64)
        C = np.ascontiguousarray(cov, dtype=np.float64)
        self._check(gbees_init_gaussian(self.ctx, m, C, t0))

    @_on_device
    def init_cells(self, idx, p, t0: float = 0.0, step0: int = 0):
        I = np.ascontiguousarray(idx, dtype=np.int32).reshape(-1, self.n)
        P = np.ascontiguousarray(p, dtype=np.float64)
        self._check(gbees_init_cells(self.ctx, I, P, t0, step0))

    @_on_device
    def propagate(self, t_end: float) -> Stats:
        st = gbees_stats()
        self._check(gbees_propagate(self.ctx, t_end, st))
        return Stats.of(st)

    @_on_device
    def correct_gaussian(self, y, R, H_idx=None):
        yy = np.ascontiguousarray(y, dtype=np.float64).reshape(-1)
        RR = np.ascontiguousarray(R, dtype=np.float64)
        HH = np.ascontiguousarray(np.arange(yy.size) if H_idx is None else H_idx, dtype=np.int32)
        self._check(gbees_correct_gaussian(self.ctx, yy, RR, HH))

    @_on_device
    def count(self) -> int:
        rc, n = gbees_count(self.ctx)
        self._check(rc)
        return n

    @_on_device
    def read_cells(self, sorted_: bool = True):
        n = self.count()
        idx = np.zeros((max(n, 1), self.n), dtype=np.int32)
        p = np.zeros(max(n, 1), dtype=np.float64)
        rc, n2 = gbees_read_cells(self.ctx, idx, p, sorted_)
        self._check(rc)
        return idx[:n2], p[:n2]

    @_on_device
    def moments(self):
        mean = np.zeros(self.n)
        cov = np.zeros((self.n, self.n))
        self._check(gbees_moments(self.ctx, mean, cov))
        return mean, cov

    @_on_device
    def stats(self) -> Stats:
        st = gbees_stats()
        self._check(gbees_get_stats(self.ctx, st))
        return Stats.of(st)

    @property
    def status(self) -> int:
        return gbees_get_status(self.ctx)

    @_on_device
    def profile(self, enable: Optional[bool] = None, reset: bool = False) -> dict:
        """Switch per-phase event timing on or off and return the counters as a dict."""
        if enable is not None or reset:
            cur = self._prof_on if enable is None else enable
            self._check(gbees_profile_control(self.ctx, cur, reset))
            self._prof_on = cur
        pr = gbees_profile()
        self._check(gbees_profile_read(self.ctx, pr))
        return {
            "launches": {k: int(pr.launches[i]) for i, k in enumerate(PHASE_NAMES)},
            "ms": {k: float(pr.ms[i]) for i, k in enumerate(PHASE_NAMES)},
            "timed": {k: int(pr.timed[i]) for i, k in enumerate(PHASE_NAMES)},
            "total_launches": int(pr.total_launches),
            "fallback_lookups": int(pr.fallback_lookups),
            "persist_us": {k: float(pr.persist_us[i]) for i, k in enumerate(PERSIST_NAMES)},
            "persist_steps": int(pr.persist_steps),
            "persist_ms": float(pr.persist_ms),
            "persist_launches": int(pr.persist_launches),
            "persist_updates": int(pr.persist_updates),
        }

    _prof_on = False


def propagate_batch(grids: Sequence["Grid"], t_end: Sequence[float], max_steps: int = 0,
                    max_blocks: int = 0) -> list:
    """Propagate many grids (same dimension, dynamics and precision) in one
    launch on the first grid's stream (max_steps > 0: at most that many steps
    each; max_blocks > 0: at most that many thread blocks); returns their
    Stats."""
    import torch

    count = len(grids)
    rc = gbees_set_batch_blocks(grids[0].ctx, max_blocks)
    if rc != 0:
        raise GbeesError(rc, "bad max_blocks")
    nbytes = gbees_batch_workspace_bytes(count)
    if nbytes == 0:
        raise GbeesError(GBEES_EINVAL, "empty batch")
    dev = grids[0].device
    with torch.cuda.device(dev):
        scratch = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    stats = (gbees_stats * count)()
    with torch.cuda.device(dev):
        rc = gbees_batch_propagate([g.ctx for g in grids], np.asarray(t_end, dtype=np.float64), max_steps,
                                   scratch.data_ptr(), nbytes, stats)
    if rc != 0:
        msgs = [gbees_last_error(g.ctx) for g in grids if g.status != 0] or [gbees_last_error(grids[0].ctx)]
        raise GbeesError(rc, "batch: " + msgs[0])
    return [Stats.of(stats[i]) for i in range(count)]


def grid_for_workload(w, precision: int = GBEES_FP64, max_cells: int = 1 << 20, device: str = "cuda:0",
                      probe_width: int = 1, table_factor: float = 2.0, launch_mode: int = GBEES_LAUNCH_AUTO,
                      storage_order: int = GBEES_ORDER_KEY, block_threads: int = 0,
                      persist_max_entries: int = 0) -> Grid:
    """A Grid configured for a paper_2508_13986_gb300.workloads.Workload."""
    cfg = make_config(w.n, w.dynamics, w.params, w.h, w.x0, w.thr_rel, w.cfl, w.prune_interval, precision,
                      w.limiter, max_cells, table_factor, probe_width, launch_mode, storage_order, block_threads,
                      persist_max_entries)
    return Grid(cfg, device)
