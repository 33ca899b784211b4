"""Choice of launch shapes by measurement.

The kernels' results do not depend on these shapes, only their speed does:

- probe width: lanes that probe the hashtable together in the link kernel
  (warp-cooperative probing: 1, 2, 4, 8, 16 or 32 consecutive slots per round);
- launch mode of a single grid: the persistent step-loop kernel (one block per
  SM, grid barriers) or the CUDA-graph loop (one kernel per phase);
- steps per round of the serving loop (shorter rounds admit new requests
  sooner, longer ones pay less per launch).

`tune_grid` times a short propagation of the given workload for every
candidate on the device (CUDA events) and returns the fastest; `pick_best` is
the selection rule on its own (a measurement function is passed in).
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass
from typing import Callable, Dict, Iterable, Optional, Sequence, Tuple

from . import gbees
from .workloads import Workload, capacity_for

PROBE_WIDTHS = (1, 4, 8, 16, 32)
LAUNCH_MODES = (gbees.GBEES_LAUNCH_PERSISTENT, gbees.GBEES_LAUNCH_GRAPH)


@dataclass(frozen=True)
class Shape:
    probe_width: int = 1
    launch_mode: int = gbees.GBEES_LAUNCH_AUTO


def pick_best(candidates: Iterable[Shape], measure: Callable[[Shape], float],
              repeats: int = 2) -> Tuple[Shape, Dict[Shape, float]]:
    """The candidate with the smallest measured time per cell update (the
    minimum over `repeats` measurements each); ties keep the earlier one."""
    times: Dict[Shape, float] = {}
    best: Optional[Shape] = None
    for c in candidates:
        t = min(measure(c) for _ in range(max(1, repeats)))
        times[c] = t
        if best is None or t < times[best]:
            best = c
    if best is None:
        raise ValueError("no candidate shape")
    return best, times


def _grid(w: Workload, precision: int, shape: Shape, device: str, max_cells: Optional[int]) -> gbees.Grid:
    cfg = gbees.make_config(w.n, w.dynamics, w.params, w.h, w.x0, w.thr_rel, w.cfl, w.prune_interval, precision,
                            w.limiter, max_cells or capacity_for(w), 2.0, shape.probe_width, shape.launch_mode)
    return gbees.Grid(cfg, device)


def measure_grid(w: Workload, precision: int, shape: Shape, t_probe: float, device: str = "cuda:0",
                 max_cells: Optional[int] = None) -> float:
    """Device milliseconds per cell update of propagating w from its initial
    density to t_probe with the given shape."""
    import torch

    g = _grid(w, precision, shape, device, max_cells)
    try:
        g.init_gaussian(w.mean, w.cov)
        torch.cuda.synchronize(device)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(g.stream)
        st = g.propagate(t_probe)
        e1.record(g.stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / max(st.cell_updates, 1)
    finally:
        g.close()


def tune_grid(w: Workload, precision: int = gbees.GBEES_FP64, t_probe: Optional[float] = None,
              probe_widths: Sequence[int] = PROBE_WIDTHS, launch_modes: Sequence[int] = LAUNCH_MODES,
              device: str = "cuda:0", max_cells: Optional[int] = None) -> Tuple[Shape, Dict[Shape, float]]:
    """The fastest (probe width, launch mode) for w, timed on a short horizon
    (t_probe, default a tenth of t_end)."""
    t = t_probe if t_probe is not None else 0.1 * w.t_end
    cands = [Shape(p, m) for p, m in itertools.product(probe_widths, launch_modes)]
    return pick_best(cands, lambda s: measure_grid(w, precision, s, t, device, max_cells))


def tune_round_steps(stream, precision: int = gbees.GBEES_FP32, candidates: Sequence[int] = (16, 32, 64, 128),
                     device: str = "cuda:0") -> Tuple[int, Dict[int, float]]:
    """The serving round length with the smallest p99 latency on a sample of
    the stream (served without waiting for the arrival times)."""
    from .serving import Server

    p99: Dict[int, float] = {}
    for k in candidates:
        srv = Server(precision=precision, device=device, round_steps=k, realtime=False)
        srv.run(stream)
        p99[k] = srv.stats["latency_p99_s"]
    best = min(candidates, key=lambda k: (p99[k], candidates.index(k)))
    return best, p99
