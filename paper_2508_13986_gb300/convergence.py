"""Convergence tooling (Sec. 5.2.2): the 1-norm E(t) and the Bhattacharyya
coefficient BC(t) of a propagated density against a reference propagation,
and the temporal (CFL number epsilon) and spatial (cell width factor eta)
studies built on them.

Densities are the read-out of a grid: cell indices (N x n int32) and
densities p with (prod h) sum p = 1 on a grid of widths h and origin x0
(cell i has centre x0 + i h). A cell missing from one density counts as 0.

  E  = (prod h) sum_i |p_i - p0_i|         (over the union of the two sets)
  BC = (prod h) sum_i sqrt(p_i p0_i)       (over the intersection; 1 for equal
                                            densities, 0 for disjoint ones)

The paper prints BC without the cell volume; with densities normalised as
above the factor prod h keeps BC in [0, 1]. Densities on different grids are
compared on the coarser one: every fine cell's mass goes to the coarse cell
that contains its centre (`restrict`).
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Callable, Dict, List, Optional, Sequence, Tuple

import numpy as np

from .workloads import Workload


def _pack(idx: np.ndarray) -> np.ndarray:
    """Rows of int32 cell indices as one structured key per row (for set
    operations); any n."""
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    return idx.view(np.dtype((np.void, idx.dtype.itemsize * idx.shape[1]))).ravel()


def _align(idx_a, p_a, idx_b, p_b) -> Tuple[np.ndarray, np.ndarray]:
    """Values of both densities on the union of their cells (0 where absent)."""
    ka, kb = _pack(idx_a), _pack(idx_b)
    keys, inv = np.unique(np.concatenate([ka, kb]), return_inverse=True)
    va = np.zeros(keys.shape[0])
    vb = np.zeros(keys.shape[0])
    va[inv[:ka.shape[0]]] = p_a
    vb[inv[ka.shape[0]:]] = p_b
    return va, vb


def l1_error(idx_a, p_a, idx_b, p_b, h: Sequence[float]) -> float:
    """E = (prod h) sum |p_a - p_b| over the union of the two active sets."""
    va, vb = _align(idx_a, p_a, idx_b, p_b)
    return math.prod(h) * math.fsum(np.abs(va - vb).tolist())


def bhattacharyya(idx_a, p_a, idx_b, p_b, h: Sequence[float]) -> float:
    """BC = (prod h) sum sqrt(p_a p_b) (negative densities count as 0)."""
    va, vb = _align(idx_a, p_a, idx_b, p_b)
    return math.prod(h) * math.fsum(np.sqrt(np.maximum(va, 0.0) * np.maximum(vb, 0.0)).tolist())


def restrict(idx_f, p_f, h_f: Sequence[float], x0_f: Sequence[float], h_c: Sequence[float],
             x0_c: Sequence[float]) -> Tuple[np.ndarray, np.ndarray]:
    """A density on a fine grid moved to a coarser grid: the mass
    (prod h_f) p_f of every fine cell goes to the coarse cell containing the
    fine cell's centre; returns the coarse cells and their densities."""
    h_f, x0_f = np.asarray(h_f, dtype=np.float64), np.asarray(x0_f, dtype=np.float64)
    h_c, x0_c = np.asarray(h_c, dtype=np.float64), np.asarray(x0_c, dtype=np.float64)
    centres = x0_f + np.asarray(idx_f, dtype=np.float64) * h_f
    coarse = np.floor((centres - x0_c) / h_c + 0.5).astype(np.int32)
    keys, inv = np.unique(_pack(coarse), return_inverse=True)
    mass = np.zeros(keys.shape[0])
    np.add.at(mass, inv, np.asarray(p_f, dtype=np.float64) * float(np.prod(h_f)))
    first = np.zeros(keys.shape[0], dtype=np.int64)
    first[inv[::-1]] = np.arange(inv.shape[0])[::-1]
    return coarse[first], mass / float(np.prod(h_c))


# ------------------------------------------------------------------ studies

Runner = Callable[..., object]
ReadOut = Tuple[np.ndarray, np.ndarray]


def schedule(w: Workload, times: Optional[Sequence[float]] = None) -> List[Tuple[float, object, bool]]:
    """The targets of a run in time order: (t, measurement or None, read out
    here?). Without sample times the run reads out once, at t_end. A sample at
    a measurement time is taken after the update. Sample times must increase
    strictly and lie in [0, t_end] (one read-out per sample time)."""
    marks: Dict[float, List[object]] = {}
    for t, meas in w.segments():
        marks.setdefault(float(t), [None, False])[0] = meas
    samples = [w.t_end] if times is None else [float(t) for t in times]
    if any(b <= a for a, b in zip(samples, samples[1:])):
        raise ValueError("sample times must increase strictly")
    for t in samples:
        if not 0.0 <= t <= w.t_end:
            raise ValueError(f"sample time {t} outside [0, {w.t_end}]")
        marks.setdefault(t, [None, False])[1] = True
    return [(t, marks[t][0], marks[t][1]) for t in sorted(marks)]


def run_schedule(grid, w: Workload, times: Optional[Sequence[float]] = None) -> List[ReadOut]:
    """Drive a grid (the library's Grid or any object with the same methods)
    from its initial Gaussian through the schedule; the read-outs at the
    sample times, in order."""
    grid.init_gaussian(w.mean, w.cov)
    out = []
    for t, meas, sample in schedule(w, times):
        if t > 0.0:
            grid.propagate(t)
        if meas is not None:
            grid.correct_gaussian(meas.y, meas.R, meas.H_idx)
        if sample:
            out.append(grid.read_cells())
    return out


def gpu_runner(precision: Optional[int] = None, device: str = "cuda:0") -> Runner:
    """Propagation through the CUDA library (measurements included). run(w)
    returns the read-out (sorted cells, densities) at the workload's t_end;
    run(w, times) the read-outs at the given times."""
    from . import gbees
    from .workloads import capacity_for

    prec = gbees.GBEES_FP64 if precision is None else precision

    def run(w: Workload, times: Optional[Sequence[float]] = None):
        g = gbees.grid_for_workload(w, precision=prec, max_cells=capacity_for(w), device=device)
        try:
            outs = run_schedule(g, w, times)
        finally:
            g.close()
        return outs if times is not None else outs[-1]

    return run


@dataclass
class Point:
    value: float       # epsilon (CFL number) or eta (cell width factor)
    E: float
    BC: float


@dataclass
class SeriesPoint:
    t: float
    E: float
    BC: float


def temporal_series(w: Workload, eps: Sequence[float], eps_ref: float, times: Sequence[float],
                    run: Optional[Runner] = None) -> Dict[float, List[SeriesPoint]]:
    """E(t) and BC(t) at the sample times for every CFL number epsilon,
    against the reference epsilon (the curves the paper plots against time).
    run(w, times) returns the read-outs at the sample times."""
    run = run or gpu_runner()
    ref = run(w.with_(cfl=eps_ref), times)
    out = {}
    for e in eps:
        got = run(w.with_(cfl=e), times)
        out[e] = [SeriesPoint(float(t), l1_error(*a, *r, w.h), bhattacharyya(*a, *r, w.h))
                  for t, a, r in zip(times, got, ref)]
    return out


def temporal_study(w: Workload, eps: Sequence[float], eps_ref: float, run: Optional[Runner] = None) -> List[Point]:
    """E and BC at t_end of propagations with CFL number epsilon against a
    reference with a small epsilon (same grid)."""
    run = run or gpu_runner()
    ri, rp = run(w.with_(cfl=eps_ref))
    out = []
    for e in eps:
        i, p = run(w.with_(cfl=e))
        out.append(Point(e, l1_error(i, p, ri, rp, w.h), bhattacharyya(i, p, ri, rp, w.h)))
    return out


def _on_common_grid(a: ReadOut, h_a, r: ReadOut, h_r, x0) -> Tuple[float, float]:
    """E and BC of read-out a (widths h_a) against r (widths h_r), both on the
    coarser of the two grids."""
    if tuple(h_a) >= tuple(h_r):
        ci, cp = restrict(*r, h_r, x0, h_a, x0)
        return l1_error(*a, ci, cp, h_a), bhattacharyya(*a, ci, cp, h_a)
    ci, cp = restrict(*a, h_a, x0, h_r, x0)
    return l1_error(ci, cp, *r, h_r), bhattacharyya(ci, cp, *r, h_r)


def spatial_series(w: Workload, etas: Sequence[float], eta_ref: float, times: Sequence[float],
                   run: Optional[Runner] = None) -> Dict[float, List[SeriesPoint]]:
    """E(t) and BC(t) at the sample times for every cell width factor eta,
    against the reference widths eta_ref h, compared on the coarser grid."""
    run = run or gpu_runner()
    h_ref = tuple(eta_ref * x for x in w.h)
    ref = run(w.with_(h=h_ref), times)
    out = {}
    for eta in etas:
        h = tuple(eta * x for x in w.h)
        got = run(w.with_(h=h), times)
        out[eta] = [SeriesPoint(float(t), *_on_common_grid(a, h, r, h_ref, w.x0)) for t, a, r in zip(times, got, ref)]
    return out


def spatial_study(w: Workload, etas: Sequence[float], eta_ref: float, run: Optional[Runner] = None) -> List[Point]:
    """E and BC at t_end of propagations with cell widths eta h against a
    reference with widths eta_ref h, both on the grid of the coarser one."""
    run = run or gpu_runner()
    h_ref = tuple(eta_ref * x for x in w.h)
    ri, rp = run(w.with_(h=h_ref))
    out = []
    for eta in etas:
        h = tuple(eta * x for x in w.h)
        i, p = run(w.with_(h=h))
        if eta >= eta_ref:   # compare on the grid of the approximation
            ci, cp = restrict(ri, rp, h_ref, w.x0, h, w.x0)
            out.append(Point(eta, l1_error(i, p, ci, cp, h), bhattacharyya(i, p, ci, cp, h)))
        else:
            ci, cp = restrict(i, p, h, w.x0, h_ref, w.x0)
            out.append(Point(eta, l1_error(ci, cp, ri, rp, h_ref), bhattacharyya(ci, cp, ri, rp, h_ref)))
    return out
