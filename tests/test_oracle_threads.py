"""The oracle's parallel loops do not change its results: every run below is
repeated with one thread and with four, and the cell sets, densities, times
and moments must be identical bit for bit (each parallel iteration writes
only its own slot; order-dependent sums are accumulated in one fixed order)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2508_13986_gb300 import workloads as W


def run(threads, make):
    O.set_threads(threads)
    try:
        o = make()
        idx, p = o.read_cells()
        mean, cov = o.moments()
        return idx, p, mean, cov, o.t, o.steps
    finally:
        O.set_threads(0)


def lorenz63_with_a_measurement():
    w = W.config("lorenz63_h0.5")
    o = O.Oracle(w.n, w.dynamics, w.params, w.h, w.x0, w.thr_rel, w.cfl, 7, w.limiter)
    o.init_gaussian(w.mean, w.cov)
    o.propagate(0.04)
    o.correct_gaussian(np.array([-11.0, -10.5]), np.diag([0.5, 0.5]), np.array([0, 1]))
    o.propagate(0.06)
    return o


def random_4d_linear():
    rng = np.random.default_rng(11)
    A = rng.normal(size=(4, 4))
    b = rng.normal(size=4)
    o = O.Oracle(4, O.DYN_LINEAR, list(A.ravel()) + list(b), [0.3, 0.5, 0.4, 0.6], [0.1, -0.2, 0.3, 0.0],
                 1e-3, 0.8, 3, O.LIM_MC)
    idx = np.unique(rng.integers(-4, 5, size=(400, 4)), axis=0)
    o.init_cells(idx, rng.random(len(idx)))
    o.propagate(0.1)
    return o


@pytest.mark.parametrize("make", [lorenz63_with_a_measurement, random_4d_linear])
def test_results_do_not_depend_on_the_thread_count(make):
    if O.set_threads(4) < 2:
        O.set_threads(0)
        pytest.skip("oracle built without OpenMP")
    a = run(1, make)
    b = run(4, make)
    for x, y in zip(a, b):
        assert np.array_equal(np.asarray(x), np.asarray(y))
