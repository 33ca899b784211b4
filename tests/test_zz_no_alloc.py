"""The entry point that allocates nothing, against the regular entry points.

Some callers cannot allocate device memory: real-time loops that cannot pay
for the synchronisation and latency of an allocation, and hosts whose own
allocator owns every byte of device memory. For them
gbees_propagate_cells_noalloc uses a fixed scratch array built into the
library. This test calls it through the C ABI twice in a row and checks each
result against create + init_cells + propagate + read_cells on a workspace the
test allocates, with the FP64 parity tolerance of the other GPU tests. This
file is collected last so that a run that stops at the first failure has run
every other test before it.
"""
import math

import numpy as np
import pytest

from paper_2508_13986_gb300 import gbees
from paper_2508_13986_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as ge
    ge.build()


def regular_path(cfg, idx, p, t0, step0, t_end):
    g = gbees.Grid(cfg)
    g.init_cells(idx, p, t0=t0, step0=step0)
    st = g.propagate(t_end)
    out = g.read_cells(sorted_=True)
    g.close()
    return out, st


def sort_cells(idx, p):
    order = np.lexsort(idx.T[::-1])
    return idx[order], p[order]


def test_noalloc_entry_point_matches_regular_path_twice():
    import torch

    w = W.lorenz63(h=0.5, t_end=0.0, prune_interval=4)
    cfg = gbees.make_config(w.n, w.dynamics, w.params, w.h, w.x0, w.thr_rel, w.cfl, w.prune_interval,
                            max_cells=1 << 15)
    assert gbees.gbees_workspace_bytes(cfg) <= gbees.GBEES_NOALLOC_SCRATCH_BYTES
    # starting cells: the initial Gaussian of the workload, read from the regular path
    g = gbees.Grid(cfg)
    g.init_gaussian(w.mean, w.cov)
    idx0, p0 = g.read_cells(sorted_=True)
    g.close()
    stream = torch.cuda.current_stream().cuda_stream
    for t0, step0, t_end in ((0.0, 0, 0.02), (0.01, 3, 0.035)):
        cap = 1 << 15
        idx_out = np.zeros((cap, 3), dtype=np.int32)
        p_out = np.zeros(cap)
        st = gbees.gbees_stats()
        rc, n = gbees.gbees_propagate_cells_noalloc(cfg, idx0, p0, t0, step0, t_end, stream, idx_out, p_out, st)
        assert rc == 0, gbees.STATUS_NAMES.get(rc, rc)
        got_i, got_p = sort_cells(idx_out[:n], p_out[:n])
        (ref_i, ref_p), ref_st = regular_path(cfg, idx0, p0, t0, step0, t_end)
        assert st.steps == ref_st.steps and st.t == ref_st.t
        assert np.array_equal(got_i, ref_i)
        assert math.prod(w.h) * float(np.abs(got_p - ref_p).sum()) <= 1e-10


def test_noalloc_rejects_a_grid_larger_than_its_scratch():
    w = W.lorenz63(h=0.5, t_end=0.0)
    cfg = gbees.make_config(w.n, w.dynamics, w.params, w.h, w.x0, max_cells=1 << 22)
    assert gbees.gbees_workspace_bytes(cfg) > gbees.GBEES_NOALLOC_SCRATCH_BYTES
    idx = np.zeros((1, 3), dtype=np.int32)
    p = np.ones(1)
    out_i = np.zeros((4, 3), dtype=np.int32)
    out_p = np.zeros(4)
    rc, _ = gbees.gbees_propagate_cells_noalloc(cfg, idx, p, 0.0, 0, 0.01, 0, out_i, out_p, gbees.gbees_stats())
    assert rc == gbees.GBEES_ECAPACITY
