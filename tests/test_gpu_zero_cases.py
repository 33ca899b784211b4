"""Degenerate cases through the library. The drift f = 0: every CFL rate is
zero, so one step reaches the target (Eq. 8 with no finite bound), and the
density comes back as it went in, as in the oracle. A measurement to which
the density gives no weight: C = 0 in Eq. 4, GBEES_EDEGENERATE, a poisoned
context that a new grid clears."""
import numpy as np
import pytest

from oracle.oracle import DYN_CONSTANT, LIM_MC, Oracle
from paper_2508_13986_gb300 import gbees
from paper_2508_13986_gb300 import workloads as W
from parity_helpers import FP64_L1, compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as ge
    ge.build()


@pytest.mark.parametrize("prec", [gbees.GBEES_FP64, gbees.GBEES_FP32])
def test_zero_drift_takes_one_step_and_keeps_the_density(prec):
    idx, p = W.random_cells(3, 300, 4, seed=64)
    h = (0.5, 0.5, 0.5)
    p = p / (0.125 * p.sum())
    cfg = gbees.make_config(3, gbees.GBEES_DYN_CONSTANT, (0.0, 0.0, 0.0), h, (0.0, 0.0, 0.0), 1e-7, 0.9, 1, prec,
                            gbees.GBEES_LIM_MC, 1 << 14)
    g = gbees.Grid(cfg)
    o = Oracle(3, DYN_CONSTANT, [0.0, 0.0, 0.0], list(h), [0.0, 0.0, 0.0], 1e-7, 0.9, 1, LIM_MC)
    g.init_cells(idx, p)
    o.init_cells(idx, p)
    gs = g.propagate(0.7)
    os_ = o.propagate(0.7)
    assert gs.steps == os_.steps == 1 and gs.t == os_.t == 0.7
    same, l1, _, _, _, _ = compare(g, o, h)
    assert same
    assert l1 <= (FP64_L1 if prec == gbees.GBEES_FP64 else 1e-6), l1
    g.close()


def test_a_measurement_with_no_weight_is_degenerate_and_a_new_grid_clears_it():
    w = W.lorenz63(h=0.5, t_end=0.0)
    g = gbees.grid_for_workload(w, max_cells=1 << 16)
    g.init_gaussian(w.mean, w.cov)
    y = np.array([1e6, 1e6, 1e6])                   # exp(-q/2) underflows to 0 at every cell
    with pytest.raises(gbees.GbeesError) as e:
        g.correct_gaussian(y, 0.25 * np.eye(3), np.arange(3, dtype=np.int32))
    assert e.value.status == gbees.GBEES_EDEGENERATE and g.status == gbees.GBEES_EDEGENERATE
    with pytest.raises(gbees.GbeesError) as e:      # poisoned until a new grid
        g.propagate(0.01)
    assert e.value.status == gbees.GBEES_EDEGENERATE
    g.init_gaussian(w.mean, w.cov)
    assert g.status == 0 and g.count() > 0
    g.close()
