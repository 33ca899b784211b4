"""Shared helpers of the GPU parity tests: run a workload through the CUDA
library and through the oracle, and compare the two grids cell by cell."""
import math

import numpy as np

from oracle.oracle import Oracle
from paper_2508_13986_gb300 import gbees


# tolerances of the parity bar: FP64 L1 over the union of the active sets;
# FP32 store: L1 and relative error of mean and covariance
FP64_L1 = 1e-10
FP32_L1 = 1e-5
FP32_MOM = 1e-4


def assert_fp64_parity(g, o, w, gst=None, ost=None):
    """Identical active sets, L1 within FP64_L1, and (with the propagate stats)
    the same steps, times and cell updates."""
    same, l1, ng, no, only_g, only_o = compare(g, o, w.h)
    assert same, f"active sets differ: gpu {ng} oracle {no}; only gpu {only_g[:5]} only oracle {only_o[:5]}"
    assert l1 <= FP64_L1, l1
    if gst is not None:
        assert [s.steps for s in gst] == [s.steps for s in ost]
        assert [s.t for s in gst] == [s.t for s in ost]
        assert sum(s.cell_updates for s in gst) == sum(s.cell_updates for s in ost)
    return l1


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
