"""The bounded device wait: a grid barrier that can never complete gives up.

The persistent kernel separates the phases of a time step by grid barriers
whose waits are bounded (a failure of the fixed-capacity, bounded-wait design
of Sec. 4 must end in a status, never in a hang). gbees_set_wait_limit makes
every barrier wait for one block more than were launched, with a short bound:
each block polls, gives up, records GBEES_ETIMEOUT and leaves the launch. The
call returns GBEES_ETIMEOUT, the context answers gbees_get_status and
gbees_last_error and stays poisoned until a new grid, and a new grid with the
normal bound then runs to the same result as a fresh context. Nothing here
faults or hangs: the wait that runs out is the library's own bounded poll."""
import time

import numpy as np
import pytest

from paper_2508_13986_gb300 import gbees
from paper_2508_13986_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as ge
    ge.build()


def test_a_barrier_that_cannot_complete_times_out_and_the_context_recovers():
    w = W.lorenz63(h=0.5, t_end=0.01, prune_interval=5)
    g = gbees.grid_for_workload(w, max_cells=1 << 16, launch_mode=gbees.GBEES_LAUNCH_PERSISTENT)
    g.init_gaussian(w.mean, w.cov)
    assert gbees.gbees_set_wait_limit(g.ctx, 1 << 12, 1) == gbees.GBEES_OK
    t0 = time.perf_counter()
    with pytest.raises(gbees.GbeesError) as err:
        g.propagate(w.t_end)
    assert err.value.status == gbees.GBEES_ETIMEOUT
    assert time.perf_counter() - t0 < 30.0                  # the bound, not a hang, ended the launch
    assert gbees.gbees_get_status(g.ctx) == gbees.GBEES_ETIMEOUT
    assert "timed out" in gbees.gbees_last_error(g.ctx)
    with pytest.raises(gbees.GbeesError) as again:          # poisoned until a new grid
        g.propagate(w.t_end)
    assert again.value.status == gbees.GBEES_ETIMEOUT
    # the device and the context are usable: a new grid with the normal bound
    assert gbees.gbees_set_wait_limit(g.ctx, 1 << 26, 0) == gbees.GBEES_OK
    g.init_gaussian(w.mean, w.cov)
    st = g.propagate(w.t_end)
    idx, p = g.read_cells()
    g.close()
    ref = gbees.grid_for_workload(w, max_cells=1 << 16, launch_mode=gbees.GBEES_LAUNCH_PERSISTENT)
    ref.init_gaussian(w.mean, w.cov)
    rst = ref.propagate(w.t_end)
    ridx, rp = ref.read_cells()
    ref.close()
    assert st.steps == rst.steps > 0
    assert np.array_equal(idx, ridx) and np.array_equal(p, rp)


def test_the_wait_limit_rejects_bad_arguments():
    w = W.lorenz63(h=0.5, t_end=0.01)
    g = gbees.grid_for_workload(w, max_cells=1 << 12)
    assert gbees.gbees_set_wait_limit(g.ctx, 0, 0) == gbees.GBEES_EINVAL
    assert gbees.gbees_set_wait_limit(g.ctx, 10, -1) == gbees.GBEES_EINVAL
    g.close()
