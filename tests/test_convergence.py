"""Convergence tooling (CPU): the metrics' defining properties, the transfer
between grids, and the paper's temporal and spatial studies run through the
oracle on a small case (the errors fall as epsilon and eta fall)."""
import math

import numpy as np
import pytest

from oracle.oracle import DYN_LINEAR, Oracle
from paper_2508_13986_gb300 import workloads as W
from paper_2508_13986_gb300.convergence import (bhattacharyya, l1_error, restrict, run_schedule, schedule,
                                                 spatial_series, spatial_study, temporal_series, temporal_study)


def normalised(idx, p, h):
    return idx, p / (math.prod(h) * p.sum())


def test_metrics_of_equal_and_of_disjoint_densities():
    h = (0.5, 0.25)
    idx, p = W.random_cells(2, 40, 5, seed=51)
    idx, p = normalised(idx, p, h)
    assert l1_error(idx, p, idx, p, h) == 0.0
    assert bhattacharyya(idx, p, idx, p, h) == pytest.approx(1.0, abs=1e-14)
    far = idx + np.array([100, 0], dtype=np.int32)
    assert l1_error(idx, p, far, p, h) == pytest.approx(2.0, abs=1e-14)
    assert bhattacharyya(idx, p, far, p, h) == 0.0


def test_metrics_are_symmetric_bounded_and_e_is_a_metric():
    h = (0.5, 0.5, 0.5)
    a = normalised(*W.random_cells(3, 60, 3, seed=52), h)
    b = normalised(*W.random_cells(3, 60, 3, seed=53), h)
    c = normalised(*W.random_cells(3, 60, 3, seed=54), h)
    assert l1_error(*a, *b, h) == pytest.approx(l1_error(*b, *a, h), abs=1e-15)
    assert bhattacharyya(*a, *b, h) == pytest.approx(bhattacharyya(*b, *a, h), abs=1e-15)
    assert 0.0 <= bhattacharyya(*a, *b, h) <= 1.0                    # Cauchy-Schwarz
    assert l1_error(*a, *c, h) <= l1_error(*a, *b, h) + l1_error(*b, *c, h) + 1e-15
    # Hellinger bound: E <= 2 sqrt(1 - BC^2)
    bc = bhattacharyya(*a, *b, h)
    assert l1_error(*a, *b, h) <= 2.0 * math.sqrt(max(0.0, 1.0 - bc * bc)) + 1e-12


def test_restriction_keeps_the_mass_and_averages_aligned_cells():
    h_f, h_c = (0.25, 0.25), (0.5, 0.5)
    x0_f, x0_c = (0.125, 0.125), (0.25, 0.25)    # two fine cells per coarse cell and axis, centres inside
    idx, p = W.random_cells(2, 200, 6, seed=55)
    ci, cp = restrict(idx, p, h_f, x0_f, h_c, x0_c)
    assert math.prod(h_c) * cp.sum() == pytest.approx(math.prod(h_f) * p.sum(), rel=1e-14)
    fine = {tuple(r): v for r, v in zip(idx.tolist(), p.tolist())}
    for (a, b), v in zip(ci.tolist(), cp.tolist()):
        kids = [fine.get((2 * a + i, 2 * b + j), 0.0) for i in (0, 1) for j in (0, 1)]
        assert v == pytest.approx(sum(kids) / 4.0, rel=1e-14)


def rotation():
    """A 2-D rotation with slight contraction: a Gaussian blob that turns."""
    A = np.array([[-0.1, -2.0], [2.0, -0.1]])
    return W.Workload(name="rot2d", n=2, dynamics=DYN_LINEAR, params=tuple(A.reshape(-1)) + (0.0, 0.0),
                      h=(0.25, 0.25), mean=(1.5, 0.0), cov=0.09 * np.eye(2), thr_rel=1e-6, cfl=0.8, t_end=0.4,
                      prune_interval=10)


def oracle_run(w, times=None):
    """The workload through the oracle: the read-out at t_end, or (times given)
    the read-outs at those times through the library's schedule."""
    o = Oracle(w.n, w.dynamics, w.params, w.h, w.x0, w.thr_rel, w.cfl, w.prune_interval, w.limiter)
    if times is not None:
        return run_schedule(o, w, times)
    o.init_gaussian(w.mean, w.cov)
    for t, m in w.segments():
        o.propagate(t)
        if m is not None:
            o.correct_gaussian(m.y, m.R, m.H_idx)
    return o.read_cells()


def test_temporal_study_converges_as_epsilon_falls():
    pts = temporal_study(rotation(), eps=(0.8, 0.4, 0.2), eps_ref=0.05, run=oracle_run)
    E = [q.E for q in pts]
    BC = [q.BC for q in pts]
    assert E[0] > E[1] > E[2] > 0.0
    assert BC[0] < BC[1] < BC[2] <= 1.0


def test_spatial_study_converges_as_eta_falls():
    w = rotation().with_(cfl=0.5)
    pts = spatial_study(w, etas=(2.0, 1.5, 1.0), eta_ref=0.5, run=oracle_run)
    E = [q.E for q in pts]
    assert E[0] > E[1] > E[2] > 0.0
    assert all(0.0 < q.BC <= 1.0 for q in pts) and pts[0].BC < pts[2].BC


class OracleGrid:
    """Stands in for gbees.Grid: the same methods, backed by the oracle, built
    from the library's configuration struct."""

    def __init__(self, cfg, device="cuda:0"):
        n = cfg.n
        self.o = Oracle(n, cfg.dynamics, list(cfg.params), list(cfg.h)[:n], list(cfg.x0)[:n],
                        cfg.thr_rel, cfg.cfl, cfg.prune_interval, cfg.limiter)
        self.closed = False

    def init_gaussian(self, mean, cov):
        self.o.init_gaussian(mean, cov)

    def propagate(self, t):
        return self.o.propagate(t)

    def correct_gaussian(self, y, R, H_idx):
        self.o.correct_gaussian(y, R, H_idx)

    def read_cells(self):
        return self.o.read_cells()

    def close(self):
        self.closed = True


def test_library_runner_plumbing_with_an_oracle_backed_grid(monkeypatch):
    """The library runner (configuration, schedule, read-out, release) gives the
    oracle's result when the grid behind it is the oracle."""
    from paper_2508_13986_gb300 import gbees
    from paper_2508_13986_gb300.convergence import gpu_runner

    made = []

    def grid(cfg, device="cuda:0"):
        made.append(OracleGrid(cfg, device))
        return made[-1]

    monkeypatch.setattr(gbees, "Grid", grid)
    w = rotation().with_(t_end=0.2)
    gi, gp = gpu_runner()(w)
    oi, op = oracle_run(w)
    assert np.array_equal(gi, oi) and np.array_equal(gp, op)
    assert len(made) == 1 and made[0].closed


def test_schedule_merges_sample_times_with_the_measurements():
    w = rotation().with_(t_end=0.3)
    m1 = W.Measurement(0.1, np.array([1.5, 0.0]), 0.25 * np.eye(2), np.arange(2, dtype=np.int32))
    m2 = W.Measurement(0.2, np.array([1.4, 0.2]), 0.25 * np.eye(2), np.arange(2, dtype=np.int32))
    w = w.with_(measurements=[m1, m2])
    got = schedule(w, [0.0, 0.15, 0.2, 0.3])
    assert [(t, m, s) for t, m, s in got] == [(0.0, None, True), (0.1, m1, False), (0.15, None, True),
                                              (0.2, m2, True), (0.3, None, True)]
    assert schedule(w) == [(0.1, m1, False), (0.2, m2, False), (0.3, None, True)]
    with pytest.raises(ValueError):
        schedule(w, [0.35])
    for bad in ([0.2, 0.1], [0.1, 0.1]):
        with pytest.raises(ValueError):
            schedule(w, bad)


def test_sampling_at_the_end_time_alone_is_the_plain_run():
    w = rotation().with_(t_end=0.2)
    (i1, p1), = oracle_run(w, [0.2])
    i2, p2 = oracle_run(w)
    assert np.array_equal(i1, i2) and np.array_equal(p1, p2)


def test_temporal_series_starts_equal_and_orders_by_epsilon():
    """E(0) = 0 and BC(0) = 1 (the same initial density), and at every later
    sample the coarser epsilon is further from the reference."""
    times = [0.0, 0.1, 0.2, 0.4]
    series = temporal_series(rotation(), eps=(0.8, 0.4), eps_ref=0.1, times=times, run=oracle_run)
    for e, pts in series.items():
        assert [q.t for q in pts] == times
        assert pts[0].E == 0.0 and pts[0].BC == pytest.approx(1.0, abs=1e-14)
    for a, b in zip(series[0.8][1:], series[0.4][1:]):
        assert a.E > b.E > 0.0 and a.BC < b.BC


def test_spatial_series_equals_the_study_at_the_end_time():
    """Sampled at t_end alone, the series is the study (a sample at an earlier
    time clips a time step, so it changes the later values slightly)."""
    w = rotation().with_(cfl=0.5, t_end=0.2)
    at_end = spatial_series(w, etas=(2.0, 1.0), eta_ref=0.5, times=[0.2], run=oracle_run)
    study = spatial_study(w, etas=(2.0, 1.0), eta_ref=0.5, run=oracle_run)
    for q in study:
        (end,) = at_end[q.value]
        assert end.t == 0.2 and end.E == q.E and end.BC == q.BC
    series = spatial_series(w, etas=(2.0, 1.0), eta_ref=0.5, times=[0.1, 0.2], run=oracle_run)
    for eta in (2.0, 1.0):
        assert all(0.0 < q.E < 2.0 and 0.0 < q.BC <= 1.0 for q in series[eta])
    assert series[2.0][-1].E > series[1.0][-1].E
