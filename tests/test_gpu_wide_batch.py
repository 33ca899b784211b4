"""A batch wider than the GPU holds at once: with more grids than resident
blocks the batched launch cannot give every grid a team, so each block takes
the next grid from a queue and runs its whole step loop alone (one-block
barriers). Sampled grids must equal their one-by-one runs bit for bit."""
import numpy as np
import pytest

from paper_2508_13986_gb300 import gbees
from paper_2508_13986_gb300 import workloads as W

pytestmark = pytest.mark.gpu

BLOCKS_PER_SM_MAX = 4   # 256 threads x 64 registers: at most 4 batch blocks fit an SM's 65536 registers


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as ge
    ge.build()


def test_queue_mode_batch_equals_one_by_one_runs():
    import torch

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    count = (BLOCKS_PER_SM_MAX + 1) * sms          # more grids than resident blocks
    ws = W.lorenz63_batch(count=count, seed=15, h_choices=(0.5,), t_range=(0.01, 0.02),
                          sigma_range=(0.5, 0.6), prune_interval=3)
    gs = []
    for w in ws:
        g = gbees.grid_for_workload(w, precision=gbees.GBEES_FP32, max_cells=1 << 14)
        g.init_gaussian(w.mean, w.cov)
        gs.append(g)
    st = gbees.propagate_batch(gs, [w.t_end for w in ws])
    assert all(s.t == w.t_end and s.steps > 0 for s, w in zip(st, ws))
    for i in (0, 1, sms, count // 2, count - 2, count - 1):
        a = gbees.grid_for_workload(ws[i], precision=gbees.GBEES_FP32, max_cells=1 << 14)
        a.init_gaussian(ws[i].mean, ws[i].cov)
        sa = a.propagate(ws[i].t_end)
        assert sa.steps == st[i].steps and sa.t == st[i].t and sa.cell_updates == st[i].cell_updates
        ia, pa = a.read_cells()
        ib, pb = gs[i].read_cells()
        assert np.array_equal(ia, ib) and np.array_equal(pa, pb)
        a.close()
    for g in gs:
        g.close()


def test_bench_batch_workload_grids_equal_their_one_by_one_runs():
    """The bench's batched workload (256 ragged Lorenz '63 grids, FP32, the
    bench's capacities and launch; end times capped at 0.25 to keep the test
    short): sampled grids, the largest among them, end bit for bit as their
    one-by-one runs."""
    ws = [w.with_(t_end=min(w.t_end, 0.25)) for w in W.lorenz63_batch(count=256)]
    gs = []
    for w in ws:
        g = gbees.grid_for_workload(w, precision=gbees.GBEES_FP32, max_cells=W.capacity_for(w))
        g.init_gaussian(w.mean, w.cov)
        gs.append(g)
    n0 = [g.count() for g in gs]
    st = gbees.propagate_batch(gs, [w.t_end for w in ws])
    largest = int(np.argmax(n0))
    for i in sorted({0, 97, 255, largest}):
        a = gbees.grid_for_workload(ws[i], precision=gbees.GBEES_FP32, max_cells=W.capacity_for(ws[i]))
        a.init_gaussian(ws[i].mean, ws[i].cov)
        sa = a.propagate(ws[i].t_end)
        assert sa.steps == st[i].steps and sa.t == st[i].t and sa.cell_updates == st[i].cell_updates
        ia, pa = a.read_cells()
        ib, pb = gs[i].read_cells()
        assert np.array_equal(ia, ib) and np.array_equal(pa, pb)
        a.close()
    for g in gs:
        g.close()
