"""Parity at the full size of the Lorenz '96 6-D workload (h = 0.25, 7.0 M
initial cells): the whole initial density against the oracle, then one time
step on sampled cells the oracle computes one by one (its own grow, dt and
CTU update of each sampled cell)."""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2508_13986_gb300 import gbees
from paper_2508_13986_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as ge
    ge.build()


def packed(idx):
    """Rows of cell indices as int64 keys (10 bits per dimension, dimension 0
    most significant), which sort like the rows themselves."""
    k = np.zeros(idx.shape[0], dtype=np.int64)
    for j in range(idx.shape[1]):
        k = (k << 10) | (idx[:, j].astype(np.int64) + 512)
    return k


def test_lorenz96_6d_full_size_init_and_sampled_step_fp64():
    w = W.config("lorenz96_6d")
    g = gbees.grid_for_workload(w, precision=gbees.GBEES_FP64, max_cells=1 << 25)
    o = Oracle(w.n, w.dynamics, w.params, w.h, w.x0, w.thr_rel, w.cfl, w.prune_interval, w.limiter)
    g.init_gaussian(w.mean, w.cov)
    o.init_gaussian(w.mean, w.cov)
    # the whole initial density: the same 7.0 M cells, values equal to rounding
    gi, gp = g.read_cells()
    oi, op = o.read_cells()
    assert gi.shape[0] > 6_000_000
    assert np.array_equal(gi, oi)
    l1 = math.prod(w.h) * float(np.abs(gp - op).sum())
    assert l1 <= 1e-10, l1
    del gi, gp, oi, op
    # one step: the oracle grows, takes its dt and updates sampled cells
    o.grow()
    dt = o.cfl_dt()
    oi, _ = o.read_cells()
    sel = np.random.default_rng(2508).choice(oi.shape[0], 4000, replace=False)
    sample_idx = oi[np.sort(sel)]
    expect = o.ctu_sample(dt, sample_idx)
    st = g.propagate(dt)
    assert st.steps == 1 and st.t == dt
    # the GPU's read-out is normalised by w = (prod h) sum of the updated values
    gi, gp = g.read_cells()
    assert gi.shape[0] == oi.shape[0]  # the grown set has the oracle's size
    gk = packed(gi)
    sk = packed(sample_idx)
    pos = np.searchsorted(gk, sk)
    assert np.array_equal(gk[pos], sk)
    got = gp[pos] * st.norm
    scale = np.abs(expect).max()
    assert np.abs(got - expect).max() <= 1e-12 * scale
    g.close()
