"""Continuous-batching request loop over the GBEES C ABI.

Requests (a grid's initial Gaussian, its measurement schedule and end time)
arrive over time. The loop admits arrived requests in arrival order while the
workspace bytes of the grids in service stay within a device-memory budget,
keeps every admitted grid resident on the device between its propagation
segments and measurement updates, and advances all grids in service together:
one round is one batched launch per model family (dimension, dynamics) in which
every grid takes at most `round_steps` steps towards its next segment target
(gbees_batch_propagate with a step cap), every grid of the family working in
the same launch; the measurement updates that came due (Eq. 4) follow. By
default the families' launches follow one another, each with every block the
GPU holds; with concurrent_families they run at the same time, each on its own
CUDA stream from its own host thread and capped to a share of the resident
blocks in proportion to the family's active cells. (Measured on GB300 with the
bench's stream: the serial rounds are faster, 1.18 against 0.71 G
cell-updates/s in FP32 and 1.04 against 0.46 in FP64, with lower latency: a
step of a family's grids is latency-bound and gains from every block.) Between
rounds, finished grids are read out and released, and requests that arrived
meanwhile join the next round.

Every grid runs the same phases with the same arithmetic whether it is served
alone or in a mix, so its result does not depend on the mix.

mode "single" serves one request at a time with gbees_propagate (no batching),
the plain form that the batched loop is compared with.
"""
from __future__ import annotations

import concurrent.futures
import time
from collections import deque
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import gbees
from .workloads import Workload, capacity_for


@dataclass
class Result:
    rid: int
    name: str
    arrival: float       # seconds after the start of the stream
    admitted: float
    finished: float
    steps: int
    cell_updates: int
    mean: np.ndarray
    cov: np.ndarray
    n_cells: int
    idx: Optional[np.ndarray] = None
    p: Optional[np.ndarray] = None
    error: Optional[str] = None      # a grid that failed (e.g. out of capacity) ends with its status

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


@dataclass
class _Active:
    rid: int
    w: Workload
    arrival: float
    admitted: float
    grid: gbees.Grid
    nbytes: int
    segments: List[Tuple[float, object]]
    seg: int = 0
    steps: int = 0
    updates: int = 0
    cells: int = 1                  # active cells after the last round
    complete: Optional[bool] = False  # set by the round that reached a segment target
    error: Optional[int] = None     # status of a failed call; the request ends with it


@dataclass
class Server:
    precision: int = gbees.GBEES_FP32
    device: str = "cuda:0"
    pool_bytes: int = 120 << 30
    round_steps: int = 64
    mode: str = "batched"           # or "single"
    keep_density: bool = False
    realtime: bool = True            # arrivals follow the wall clock
    concurrent_families: bool = False  # the families' rounds overlap on the device (see above)
    block_threads: int = 0           # launch shape of the grids' step kernels (0: the library's default)
    stats: Dict[str, float] = field(default_factory=dict)
    family_windows: List[Dict[str, float]] = field(default_factory=list)  # launch intervals of the last run
    _streams: Dict[Tuple[int, int], object] = field(default_factory=dict)

    def _stream_of(self, family: Tuple[int, int]):
        import torch

        if self.mode == "single" or not self.concurrent_families or not torch.cuda.is_available():
            return None
        if family not in self._streams:
            self._streams[family] = torch.cuda.Stream(device=self.device)
        return self._streams[family]

    def _admit(self, rid: int, w: Workload, arrival: float, now: float) -> _Active:
        cfg = gbees.make_config(w.n, w.dynamics, w.params, w.h, w.x0, w.thr_rel, w.cfl, w.prune_interval,
                                self.precision, w.limiter, capacity_for(w), block_threads=self.block_threads)
        g = gbees.Grid(cfg, self.device, stream=self._stream_of((w.n, w.dynamics)))
        a = _Active(rid, w, arrival, now, g, gbees.gbees_workspace_bytes(cfg), w.segments())
        try:
            g.init_gaussian(w.mean, w.cov)
        except gbees.GbeesError as e:
            a.error = e.status      # ends in the next round, before any step
        return a

    @staticmethod
    def _failed_result(rid: int, w: Workload, arrival: float, admitted: float, now: float, steps: int,
                       updates: int, error: str) -> Result:
        return Result(rid, w.name, arrival, admitted, now, steps, updates, np.full(w.n, np.nan),
                      np.full((w.n, w.n), np.nan), 0, error=error)

    def _finish(self, a: _Active, now: float, error: Optional[str] = None) -> Result:
        if error is None:
            mean, cov = a.grid.moments()
            idx = p = None
            if self.keep_density:
                idx, p = a.grid.read_cells()
            r = Result(a.rid, a.w.name, a.arrival, a.admitted, now, a.steps, a.updates, mean, cov, a.grid.count(),
                       idx, p)
        else:
            r = self._failed_result(a.rid, a.w, a.arrival, a.admitted, now, a.steps, a.updates, error)
        a.grid.close()
        return r

    def _advance_segment(self, a: _Active) -> bool:
        """After the grid reached its current target: the measurement update if
        one is due; True when the request is complete. Raises GbeesError when
        the update fails (a measurement the density gives no weight to)."""
        t_target, meas = a.segments[a.seg]
        if meas is not None:
            a.grid.correct_gaussian(meas.y, meas.R, meas.H_idx)
        a.seg += 1
        return a.seg >= len(a.segments)

    def _pool(self, workers: int) -> concurrent.futures.ThreadPoolExecutor:
        if getattr(self, "_executor", None) is None or self._executor_workers < workers:
            self._executor = concurrent.futures.ThreadPoolExecutor(max_workers=workers)
            self._executor_workers = workers
        return self._executor

    def _shares(self, families) -> Dict[Tuple[int, int], int]:
        """Blocks each family's launch may use: all of them for one family,
        otherwise the resident blocks in proportion to the family's active
        cells (at least one block per grid where possible)."""
        import torch

        if len(families) <= 1 or not self.concurrent_families:
            return {k: 0 for k in families}
        sms = torch.cuda.get_device_properties(self.device).multi_processor_count if torch.cuda.is_available() else 152
        total = sms * 4  # resident blocks of the batch kernels (four per SM)
        work = {k: sum(max(1, m.cells) for m in members) for k, members in families.items()}
        W = float(sum(work.values()))
        return {k: max(1, int(total * work[k] / W)) for k in families}

    def _family_round(self, family, members: List[_Active], max_blocks: int, clock):
        """One round of one family on its stream: the batched launch, then the
        measurement updates that came due. Returns (failed, reached)."""
        import torch

        failed: List[_Active] = []
        reached: List[_Active] = []
        stream = self._stream_of(family)
        t_start = clock() if clock else None
        ev0 = ev1 = None
        if stream is not None:
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
        targets = [m.segments[m.seg][0] for m in members]
        try:
            sts = gbees.propagate_batch([m.grid for m in members], targets, max_steps=self.round_steps,
                                        max_blocks=max_blocks)
        except gbees.GbeesError:
            sts = [m.grid.stats() if m.grid.status == 0 else None for m in members]
        if ev1 is not None:
            ev1.record(stream)
        for m, s, tt in zip(members, sts, targets):
            if s is None:
                m.error = m.grid.status
                failed.append(m)
                continue
            m.steps = s.total_steps
            m.updates += s.cell_updates
            m.cells = s.n_cells
            if s.t == tt:
                try:
                    m.complete = self._advance_segment(m)
                except gbees.GbeesError as e:
                    m.error = e.status
                    m.complete = None
                reached.append(m)
        if ev1 is not None:
            self._windows.append((family, ev0, ev1, t_start))
        return failed, reached

    def run(self, stream: Sequence[Tuple[float, Workload]]) -> List[Result]:
        import torch

        t0 = time.perf_counter()
        clock = (lambda: time.perf_counter() - t0) if self.realtime else None
        self._windows = []
        pending = deque((rid, arr, w) for rid, (arr, w) in enumerate(sorted(stream, key=lambda x: x[0])))
        active: List[_Active] = []
        results: List[Result] = []
        used = 0
        rounds = 0
        max_active = max_used = 0
        virtual_now = 0.0
        while pending or active:
            now = clock() if clock else virtual_now
            # admission in arrival order while the memory budget allows
            while pending and (pending[0][1] <= now or not self.realtime):
                rid, arr, w = pending[0]
                if not self.realtime:
                    virtual_now = max(virtual_now, arr)
                need = gbees.gbees_workspace_bytes(gbees.make_config(
                    w.n, w.dynamics, w.params, w.h, w.x0, w.thr_rel, w.cfl, w.prune_interval, self.precision,
                    w.limiter, capacity_for(w)))
                if active and used + need > self.pool_bytes:
                    break
                if self.mode == "single" and active:
                    break
                pending.popleft()
                t_adm = now if clock else virtual_now
                try:
                    a = self._admit(rid, w, arr, t_adm)
                except gbees.GbeesError as e:          # the configuration was refused
                    results.append(self._failed_result(rid, w, arr, t_adm, t_adm, 0, 0,
                                                       gbees.STATUS_NAMES.get(e.status, "error")))
                    continue
                except torch.cuda.OutOfMemoryError:    # the workspace could not be allocated
                    results.append(self._failed_result(rid, w, arr, t_adm, t_adm, 0, 0, "ENOMEM"))
                    continue
                active.append(a)
                used += a.nbytes
                max_active = max(max_active, len(active))
                max_used = max(max_used, used)
            if not active:
                if pending and clock:
                    time.sleep(max(0.0, min(0.002, pending[0][1] - clock())))
                continue
            # one round: every grid in service towards its next target
            rounds += 1
            failed: List[_Active] = [a for a in active if a.error is not None]
            runnable = [a for a in active if a.error is None]
            reached: List[_Active] = []
            if self.mode == "single":
                for a in runnable[:1]:
                    try:
                        st = a.grid.propagate(a.segments[a.seg][0])
                        a.steps += st.steps
                        a.updates += st.cell_updates
                        reached.append(a)
                    except gbees.GbeesError as e:
                        a.error = e.status
                        failed.append(a)
            else:
                families: Dict[Tuple[int, int], List[_Active]] = {}
                for a in runnable:
                    families.setdefault((a.w.n, a.w.dynamics), []).append(a)
                shares = self._shares(families)
                fams = list(families.items())
                if self.concurrent_families and len(fams) > 1:
                    pool = self._pool(len(fams))
                    outs = list(pool.map(lambda kv: self._family_round(kv[0], kv[1], shares[kv[0]], clock),
                                         fams))
                else:
                    outs = [self._family_round(k, m, shares[k], clock) for k, m in fams]
                for f_failed, f_reached in outs:
                    failed.extend(f_failed)
                    reached.extend(f_reached)
            torch.cuda.synchronize(self.device)
            done_now = clock() if clock else virtual_now
            for a in failed:
                results.append(self._finish(a, done_now, error=gbees.STATUS_NAMES.get(a.error, "error")))
                active.remove(a)
                used -= a.nbytes
            for a in reached:
                if self.mode == "single":
                    try:
                        complete = self._advance_segment(a)
                    except gbees.GbeesError as e:
                        a.error = e.status
                        complete = None
                else:
                    complete = a.complete
                if complete is None:
                    results.append(self._finish(a, done_now, error=gbees.STATUS_NAMES.get(a.error, "error")))
                    active.remove(a)
                    used -= a.nbytes
                    continue
                if complete:
                    results.append(self._finish(a, clock() if clock else done_now))
                    active.remove(a)
                    used -= a.nbytes
        elapsed = time.perf_counter() - t0
        self._collect_windows()
        lat = np.array([r.latency for r in results]) if results else np.zeros(1)
        self.stats = {
            "requests": len(results),
            "failed": sum(r.error is not None for r in results),
            "rounds": rounds,
            "max_active": max_active,
            "max_used_bytes": max_used,
            "wall_s": elapsed,
            "cell_updates": float(sum(r.cell_updates for r in results)),
            "cell_updates_per_s": float(sum(r.cell_updates for r in results)) / elapsed,
            "requests_per_s": len(results) / elapsed,
            "latency_p50_s": float(np.percentile(lat, 50)),
            "latency_p99_s": float(np.percentile(lat, 99)),
            "latency_max_s": float(lat.max()),
        }
        return sorted(results, key=lambda r: r.rid)

    def _collect_windows(self):
        """Device-time intervals (ms from the first launch) of every family launch of the run."""
        self.family_windows = []
        if not self._windows:
            return
        ref = self._windows[0][1]
        for family, e0, e1, _ in self._windows:
            e1.synchronize()
            self.family_windows.append({"family": family, "start_ms": ref.elapsed_time(e0),
                                        "end_ms": ref.elapsed_time(e1)})
