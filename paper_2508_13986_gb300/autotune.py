"""Choice of launch shapes by measurement.

The kernels' results do not depend on these shapes, only their speed does:

- probe width: lanes that probe the hashtable together in the link kernel
  (warp-cooperative probing: 1, 2, 4, 8, 16 or 32 consecutive slots per round);
- launch mode of a single grid: the persistent step-loop kernel (one block per
  SM, grid barriers) or the CUDA-graph loop (one kernel per phase);
- threads per block of the step kernels of the graph loop (64, 128 or 256;
  each kernel launches one resident wave of blocks of that size);
- the pool size up to which AUTO keeps a grid on the persistent kernel;
- steps per round of the serving loop (shorter rounds admit new requests
  sooner, longer ones pay less per launch).

`tune_grid` times a short propagation of the given workload for every
candidate on the device (CUDA events) and returns the fastest; `pick_best` is
the selection rule on its own (a measurement function is passed in);
`persist_crossover` finds, from a growing grid run both ways, the pool size
beyond which the graph loop is faster than the persistent kernel.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass
from typing import Callable, Dict, Iterable, Optional, Sequence, Tuple

from . import gbees
from .workloads import Workload, capacity_for

PROBE_WIDTHS = (1, 4, 8, 16, 32)
LAUNCH_MODES = (gbees.GBEES_LAUNCH_PERSISTENT, gbees.GBEES_LAUNCH_GRAPH)
BLOCK_THREADS = (128, 256)


@dataclass(frozen=True)
class Shape:
    probe_width: int = 1
    launch_mode: int = gbees.GBEES_LAUNCH_AUTO
    block_threads: int = 0          # 0: the library's default (256)
    persist_max_entries: int = 0    # 0: the library's default (2^18)

    def as_dict(self) -> dict:
        return {"probe_width": self.probe_width, "launch_mode": self.launch_mode,
                "block_threads": self.block_threads or 256,
                "persist_max_entries": self.persist_max_entries or (1 << 18)}


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


def config_for(w: Workload, precision: int, shape: Shape, max_cells: Optional[int]) -> gbees.gbees_config:
    return gbees.make_config(w.n, w.dynamics, w.params, w.h, w.x0, w.thr_rel, w.cfl, w.prune_interval, precision,
                             w.limiter, max_cells or capacity_for(w), 2.0, shape.probe_width, shape.launch_mode,
                             block_threads=shape.block_threads, persist_max_entries=shape.persist_max_entries)


def _grid(w: Workload, precision: int, shape: Shape, device: str, max_cells: Optional[int]) -> gbees.Grid:
    return gbees.Grid(config_for(w, precision, shape, max_cells), device)


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
              device: str = "cuda:0", max_cells: Optional[int] = None,
              block_threads: Sequence[int] = (0,), repeats: int = 2) -> Tuple[Shape, Dict[Shape, float]]:
    """The fastest (probe width, launch mode, block threads) for w, timed on a
    short horizon (t_probe, default a tenth of t_end)."""
    t = t_probe if t_probe is not None else 0.1 * w.t_end
    cands = [Shape(p, m, b) for p, m, b in itertools.product(probe_widths, launch_modes, block_threads)]
    return pick_best(cands, lambda s: measure_grid(w, precision, s, t, device, max_cells), repeats=repeats)


def crossover(samples: Sequence[Tuple[int, float, float]]) -> int:
    """From (pool entries, ms per cell update on the persistent kernel, the same
    on the graph loop) samples of growing grids: the pool size P that best
    separates the two, i.e. with the fewest samples on the wrong side (the
    persistent kernel slower at a size <= P, or faster at a size > P); ties go
    to the smaller P. A segment that holds a prune or a burst of new cells can
    lose on either side without moving P. 0 when the graph loop wins
    throughout."""
    s = sorted(samples)
    if not s:
        raise ValueError("no samples")
    wins = [tp <= tg for _, tp, tg in s]
    best_p, best_err = 0, sum(wins)          # P = 0: every persistent win is misplaced
    losses_below = 0
    wins_above = sum(wins)
    for (pool, _, _), w in zip(s, wins):
        if w:
            wins_above -= 1
        else:
            losses_below += 1
        err = losses_below + wins_above
        if err < best_err:
            best_p, best_err = pool, err
    return int(best_p)


def persist_crossover(w: Workload, precision: int = gbees.GBEES_FP64, segment: float = 0.02,
                      t_end: Optional[float] = None, device: str = "cuda:0",
                      max_cells: Optional[int] = None) -> Tuple[int, list]:
    """Runs w both ways (persistent kernel only, graph loop only) in segments
    and returns the crossover pool size (see `crossover`) with the samples
    (pool entries at the segment's start, ms per cell update each way)."""
    import torch

    t_stop = t_end if t_end is not None else w.t_end
    per_mode = {}
    for mode in (gbees.GBEES_LAUNCH_PERSISTENT, gbees.GBEES_LAUNCH_GRAPH):
        g = _grid(w, precision, Shape(1, mode), device, max_cells)
        rows = []
        try:
            g.init_gaussian(w.mean, w.cov)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            t = 0.0
            while t < t_stop - 1e-12:
                t = min(t_stop, t + segment)
                pool = g.stats().n_pool
                e0.record(g.stream)
                st = g.propagate(t)
                e1.record(g.stream)
                e1.synchronize()
                rows.append((pool, e0.elapsed_time(e1) / max(st.cell_updates, 1)))
        finally:
            g.close()
        per_mode[mode] = rows
    samples = [(p, a, b) for (p, a), (_, b) in zip(per_mode[gbees.GBEES_LAUNCH_PERSISTENT],
                                                  per_mode[gbees.GBEES_LAUNCH_GRAPH])]
    return crossover(samples), samples


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
