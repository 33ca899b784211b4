"""Parity at full size in the configuration the bench times: the Lorenz '63
h = 0.25 workload (t_end 2, eight full-state measurements) runs through the
library to its end as the bench runs it (launch mode AUTO, which picks the
persistent step-loop kernel at this size; max_cells 2^22). The oracle cannot
redo the whole run in a test's time, so it takes the GPU's end state as its
initial cells and both continue for a further 0.02 time units (eight steps,
one of them with a prune); the two must then agree at the bar of their
precision. (The oracle run the same way from its own end state continues
bit for bit like the oracle that never stopped: 2176 steps and 32,035,389 cell
updates to t = 2, then 8 steps and 14,979 updates.)

In FP64 the whole run must also take the oracle's steps and cell updates
segment by segment, and keep its number of active cells after every
measurement update (tests/golden/bench_workload_counts.txt, written by the
oracle alone)."""
import os

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2508_13986_gb300 import gbees
from paper_2508_13986_gb300 import workloads as W
from parity_helpers import FP32_L1, FP32_MOM, assert_fp64_parity, compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as ge
    ge.build()


def golden_counts():
    path = os.path.join(os.path.dirname(__file__), "golden", "bench_workload_counts.txt")
    rows = []
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            t, s, u, n = line.split()
            rows.append((float(t), int(s), int(u), int(n)))
    return rows


def run_to_end(w, precision):
    """The workload through the library; per segment (target, steps, cell
    updates, active cells after the measurement update)."""
    g = gbees.grid_for_workload(w, precision=precision, max_cells=1 << 22)
    g.init_gaussian(w.mean, w.cov)
    rows = []
    for t, meas in w.segments():
        st = g.propagate(t)
        if meas is not None:
            g.correct_gaussian(meas.y, meas.R, meas.H_idx)
        rows.append((t, st.steps, st.cell_updates, g.count()))
    return g, rows


def oracle_from(g, w):
    st = g.stats()
    idx, p = g.read_cells()
    o = Oracle(w.n, w.dynamics, w.params, w.h, w.x0, w.thr_rel, w.cfl, w.prune_interval, w.limiter)
    o.init_cells(idx, p, st.t, st.total_steps)
    return o, st


def test_bench_workload_end_state_continues_like_the_oracle_fp64():
    w = W.config("lorenz63_h0.25")
    g, rows = run_to_end(w, gbees.GBEES_FP64)
    assert rows == golden_counts()                # the oracle's steps, updates and set sizes, segment by segment
    o, st = oracle_from(g, w)
    assert st.t == w.t_end
    t_more = st.t + 0.02
    gs = g.propagate(t_more)
    os_ = o.propagate(t_more)
    assert gs.steps == os_.steps and gs.t == os_.t and gs.cell_updates == os_.cell_updates
    assert_fp64_parity(g, o, w)
    g.close()


def test_bench_workload_end_state_continues_like_the_oracle_fp32():
    w = W.config("lorenz63_h0.25")
    g, _ = run_to_end(w, gbees.GBEES_FP32)
    o, st = oracle_from(g, w)
    t_more = st.t + 0.02
    g.propagate(t_more)
    o.propagate(t_more)
    _, l1, _, _, _, _ = compare(g, o, w.h)
    assert l1 <= FP32_L1, l1
    gm, gc = g.moments()
    om, oc = o.moments()
    assert np.abs(gm - om).max() <= FP32_MOM * np.abs(om).max()
    assert np.abs(gc - oc).max() <= FP32_MOM * np.abs(oc).max()
    g.close()
