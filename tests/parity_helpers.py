"""Shared helpers of the GPU parity tests: run a workload through the CUDA
library and through the oracle, and compare the two grids cell by cell."""
import math

import numpy as np

from oracle.oracle import Oracle
from paper_2508_13986_gb300 import gbees


def make_pair(w, precision=gbees.GBEES_FP64, max_cells=1 << 20, probe_width=1, table_factor=2.0):
    g = gbees.grid_for_workload(w, precision=precision, max_cells=max_cells, probe_width=probe_width,
                                table_factor=table_factor)
    o = Oracle(w.n, w.dynamics, w.params, w.h, w.x0, w.thr_rel, w.cfl, w.prune_interval, w.limiter)
    return g, o


def run_schedule(grid, orc, w, t_end=None):
    """Propagate both through the workload's measurement schedule up to t_end."""
    t_stop = w.t_end if t_end is None else t_end
    gst, ost = [], []
    for t_target, meas in w.segments():
        t_target = min(t_target, t_stop)
        gst.append(grid.propagate(t_target))
        ost.append(orc.propagate(t_target))
        if meas is not None and t_target == meas.t:
            grid.correct_gaussian(meas.y, meas.R, meas.H_idx)
            orc.correct_gaussian(meas.y, meas.R, meas.H_idx)
        if t_target >= t_stop:
            break
    return gst, ost


def compare(grid, orc, h):
    """(same_set, L1, n_gpu, n_orc, only_gpu, only_orc) with L1 = (prod h) sum |p_gpu - p_orc|
    over the union of the two active sets (a missing cell counts as p = 0)."""
    gi, gp = grid.read_cells(sorted_=True)
    oi, op = orc.read_cells()
    same = gi.shape == oi.shape and np.array_equal(gi, oi)
    if same:
        l1 = math.prod(h) * math.fsum(np.abs(gp - op).tolist())
        return True, l1, gi.shape[0], oi.shape[0], [], []
    dg = {tuple(r): v for r, v in zip(gi.tolist(), gp.tolist())}
    do = {tuple(r): v for r, v in zip(oi.tolist(), op.tolist())}
    keys = set(dg) | set(do)
    l1 = math.prod(h) * math.fsum(abs(dg.get(k, 0.0) - do.get(k, 0.0)) for k in keys)
    only_g = sorted(set(dg) - set(do))
    only_o = sorted(set(do) - set(dg))
    return False, l1, len(dg), len(do), only_g, only_o
