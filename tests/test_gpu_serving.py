"""The continuous-batching request loop: each result equals the same request
served alone and the oracle's run of that request; admission respects the
memory budget; a timed stream completes."""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle
from parity_helpers import FP64_L1

from paper_2508_13986_gb300 import gbees
from paper_2508_13986_gb300 import workloads as W
from paper_2508_13986_gb300.serving import Server

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as ge
    ge.build()


def small_stream(count, seed, rate=400.0):
    return W.serving_stream(count=count, rate=rate, seed=seed, l96_sigma=0.3, l96_t=(0.02, 0.05),
                            l63_kw=dict(h_choices=(0.5,), t_range=(0.03, 0.08), sigma_range=(0.5, 1.0),
                                        prune_interval=5))


@pytest.mark.parametrize("prec", [gbees.GBEES_FP32, gbees.GBEES_FP64])
def test_each_result_is_the_same_alone_and_in_the_mix(prec):
    stream = small_stream(10, seed=21)
    assert {w.n for _, w in stream} == {3, 6}
    mix = Server(precision=prec, realtime=False, keep_density=True, round_steps=7).run(stream)
    alone = Server(precision=prec, realtime=False, keep_density=True, mode="single").run(stream)
    assert len(mix) == len(alone) == len(stream)
    for a, b in zip(mix, alone):
        assert a.error is None and b.error is None
        assert a.steps == b.steps and a.cell_updates == b.cell_updates
        assert np.array_equal(a.idx, b.idx) and np.array_equal(a.p, b.p)
        assert np.array_equal(a.mean, b.mean) and np.array_equal(a.cov, b.cov)


def test_served_results_match_the_oracle_grid_by_grid():
    """A mixed stream (Lorenz '63 and Lorenz '96 requests, each with its
    measurement updates) served in batched FP64 rounds: every request's final
    density equals the oracle's run of that request alone (identical active
    set, L1 within the FP64 bar, the same steps)."""
    stream = small_stream(8, seed=24)
    assert {w.n for _, w in stream} == {3, 6}
    res = sorted(Server(precision=gbees.GBEES_FP64, realtime=False, keep_density=True, round_steps=5).run(stream),
                 key=lambda r: r.rid)
    assert len(res) == len(stream)
    for (_, w), r in zip(stream, res):
        assert r.error is None
        o = Oracle(w.n, w.dynamics, w.params, w.h, w.x0, w.thr_rel, w.cfl, w.prune_interval, w.limiter)
        o.init_gaussian(w.mean, w.cov)
        steps = 0
        for t, meas in w.segments():
            steps += o.propagate(t).steps
            if meas is not None:
                o.correct_gaussian(meas.y, meas.R, meas.H_idx)
        oi, op = o.read_cells()
        order = np.lexsort(r.idx.T[::-1])
        gi, gp = r.idx[order], r.p[order]
        assert r.steps == steps
        assert np.array_equal(gi, oi), (w.name, len(gi), len(oi))
        l1 = math.prod(w.h) * math.fsum(np.abs(gp - op).tolist())
        assert l1 <= FP64_L1, (w.name, l1)


def test_model_families_run_at_the_same_time_on_the_device():
    """Lorenz '63 and Lorenz '96 requests in service together with concurrent
    family rounds: each family's round is issued on its own stream from its own
    host thread with a share of the GPU's blocks, so their launches overlap in
    device time (CUDA event intervals around each family's launch, on its
    stream), and the results are those of the serial rounds, bit for bit."""
    stream = small_stream(12, seed=25, rate=1e6)
    srv = Server(precision=gbees.GBEES_FP32, realtime=False, round_steps=40, concurrent_families=True,
                 keep_density=True)
    res = srv.run(stream)
    assert len(res) == len(stream) and srv.stats["failed"] == 0
    wins = srv.family_windows
    l63 = [w for w in wins if w["family"][0] == 3]
    l96 = [w for w in wins if w["family"][0] == 6]
    assert l63 and l96
    overlap = max(min(a["end_ms"], b["end_ms"]) - max(a["start_ms"], b["start_ms"]) for a in l63 for b in l96)
    assert overlap > 0.0, wins
    serial = Server(precision=gbees.GBEES_FP32, realtime=False, round_steps=40, keep_density=True).run(stream)
    for a, b in zip(res, serial):
        assert a.steps == b.steps and np.array_equal(a.idx, b.idx) and np.array_equal(a.p, b.p)


def test_admission_respects_the_memory_budget():
    stream = small_stream(8, seed=22)
    srv = Server(precision=gbees.GBEES_FP32, realtime=False)
    from paper_2508_13986_gb300.workloads import capacity_for
    sizes = []
    for _, w in stream:
        cfg = gbees.make_config(w.n, w.dynamics, w.params, w.h, w.x0, w.thr_rel, w.cfl, w.prune_interval,
                                gbees.GBEES_FP32, w.limiter, capacity_for(w))
        sizes.append(gbees.gbees_workspace_bytes(cfg))
    srv.pool_bytes = 2 * max(sizes)
    res = srv.run(stream)
    assert len(res) == len(stream) and srv.stats["failed"] == 0
    assert srv.stats["max_used_bytes"] <= srv.pool_bytes
    assert 1 <= srv.stats["max_active"] < len(stream)


def test_timed_stream_reports_latency_percentiles():
    stream = small_stream(12, seed=23, rate=200.0)
    srv = Server(precision=gbees.GBEES_FP32, realtime=True)
    res = srv.run(stream)
    assert len(res) == 12 and srv.stats["failed"] == 0
    st = srv.stats
    assert 0 < st["latency_p50_s"] <= st["latency_p99_s"] <= st["latency_max_s"]
    assert all(r.finished >= r.arrival for r in res)
