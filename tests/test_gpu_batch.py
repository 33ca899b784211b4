"""Batched propagation (many independent grids in one launch) against the same
grids propagated one by one, and against the oracle."""
import numpy as np
import pytest

from paper_2508_13986_gb300 import gbees
from paper_2508_13986_gb300 import workloads as W
from parity_helpers import assert_fp64_parity, make_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as ge
    ge.build()


def small_batch(count, seed):
    return W.lorenz63_batch(count=count, seed=seed, h_choices=(0.5,), t_range=(0.02, 0.06),
                            sigma_range=(0.5, 1.0), prune_interval=4)


def grids_for(ws, precision):
    gs = []
    for w in ws:
        g = gbees.grid_for_workload(w, precision=precision, max_cells=1 << 16)
        g.init_gaussian(w.mean, w.cov)
        gs.append(g)
    return gs


@pytest.mark.parametrize("prec", [gbees.GBEES_FP64, gbees.GBEES_FP32])
def test_batch_equals_one_by_one_bitwise(prec):
    """The batch kernel runs the same phases as gbees_propagate with the grid's
    work in one block: every grid ends with the same bits, steps and time."""
    ws = small_batch(7, seed=11)
    alone = grids_for(ws, prec)
    st_alone = [g.propagate(w.t_end) for g, w in zip(alone, ws)]
    batch = grids_for(ws, prec)
    st_batch = gbees.propagate_batch(batch, [w.t_end for w in ws])
    for a, b, sa, sb in zip(alone, batch, st_alone, st_batch):
        assert sa.steps == sb.steps and sa.t == sb.t and sa.cell_updates == sb.cell_updates
        ia, pa = a.read_cells()
        ib, pb = b.read_cells()
        assert np.array_equal(ia, ib) and np.array_equal(pa, pb)
    for g in alone + batch:
        g.close()


def test_batch_matches_oracle_and_continues():
    """Two batched segments (the second continues from the first) against the
    oracle, grid by grid."""
    ws = small_batch(3, seed=12)
    gs, os_ = [], []
    for w in ws:
        g, o = make_pair(w, max_cells=1 << 16)
        g.init_gaussian(w.mean, w.cov)
        o.init_gaussian(w.mean, w.cov)
        gs.append(g)
        os_.append(o)
    half = [0.5 * w.t_end for w in ws]
    gbees.propagate_batch(gs, half)
    st = gbees.propagate_batch(gs, [w.t_end for w in ws])
    for g, o, w, s in zip(gs, os_, ws, st):
        o.propagate(0.5 * w.t_end)
        os2 = o.propagate(w.t_end)
        assert s.t == os2.t
        assert_fp64_parity(g, o, w)
        g.close()


def test_batch_edge_cases():
    ws = small_batch(3, seed=13)
    gs = grids_for(ws, gbees.GBEES_FP64)
    # a grid already at its end time takes no step; the others run
    st = gbees.propagate_batch(gs, [0.0, ws[1].t_end, ws[2].t_end])
    assert st[0].steps == 0 and st[1].steps > 0 and st[2].steps > 0
    # one grid alone
    st1 = gbees.propagate_batch(gs[:1], [ws[0].t_end])
    assert st1[0].steps > 0 and st1[0].t == ws[0].t_end
    # contexts of another model are rejected
    lin = W.Workload(name="lin", n=3, dynamics=W.DYN_LINEAR, params=tuple(np.eye(3).reshape(-1)) + (0.0, 0.0, 0.0),
                     h=(0.5, 0.5, 0.5), mean=(0.0, 0.0, 0.0), cov=np.eye(3), thr_rel=1e-7, cfl=0.9, t_end=0.1)
    other = gbees.grid_for_workload(lin, max_cells=1 << 16)
    other.init_gaussian(lin.mean, lin.cov)
    with pytest.raises(gbees.GbeesError) as e:
        gbees.propagate_batch([gs[1], other], [1.0, 1.0])
    assert e.value.status == gbees.GBEES_EINVAL
    # a grid that runs out of capacity poisons only itself
    tight = gbees.grid_for_workload(ws[2], max_cells=gs[2].stats().n_pool + 8)
    tight.init_gaussian(ws[2].mean, ws[2].cov)
    with pytest.raises(gbees.GbeesError) as e:
        gbees.propagate_batch([gs[1], tight], [ws[1].t_end + 0.05, ws[2].t_end + 0.5])
    assert e.value.status == gbees.GBEES_ECAPACITY
    assert gs[1].status == 0 and tight.status == gbees.GBEES_ECAPACITY
    for g in gs + [other, tight]:
        g.close()


def test_a_batch_of_many_small_grids_equals_one_by_one_runs():
    """320 grids in one launch (small teams, many of one block); sampled grids
    equal their one-by-one runs."""
    count = 320
    ws = W.lorenz63_batch(count=count, seed=14, h_choices=(0.5,), t_range=(0.01, 0.03),
                          sigma_range=(0.5, 0.6), prune_interval=3)
    gs = grids_for(ws, gbees.GBEES_FP32)
    st = gbees.propagate_batch(gs, [w.t_end for w in ws])
    for i in (0, 1, 157, count - 2, count - 1):
        a = gbees.grid_for_workload(ws[i], precision=gbees.GBEES_FP32, max_cells=1 << 16)
        a.init_gaussian(ws[i].mean, ws[i].cov)
        sa = a.propagate(ws[i].t_end)
        assert sa.steps == st[i].steps and sa.t == st[i].t
        ia, pa = a.read_cells()
        ib, pb = gs[i].read_cells()
        assert np.array_equal(ia, ib) and np.array_equal(pa, pb)
        a.close()
    for g in gs:
        g.close()
