"""The seeded input generators: determinism, the stated distributions, and the
capacity rule (CPU)."""
import numpy as np

from paper_2508_13986_gb300 import workloads as W


def test_batch_grids_are_seeded_and_within_their_ranges():
    a = W.lorenz63_batch(64)
    b = W.lorenz63_batch(64)
    assert [w.mean for w in a] == [w.mean for w in b] and [w.t_end for w in a] == [w.t_end for w in b]
    for w in a:
        m = np.array(w.mean)
        assert -15 <= m[0] <= 15 and -20 <= m[1] <= 20 and 5 <= m[2] <= 40
        sig = np.sqrt(np.diag(w.cov))
        assert np.all((sig >= 0.5) & (sig <= 2.0)) and np.allclose(w.cov, np.diag(np.diag(w.cov)))
        assert w.h[0] in (0.25, 0.5) and 0.25 <= w.t_end <= 1.0 and w.x0 == w.mean
    # the first grids do not depend on how many are drawn
    assert [w.mean for w in W.lorenz63_batch(8)] == [w.mean for w in a[:8]]


def test_serving_stream_is_seeded_poisson_with_the_stated_mix():
    s = W.serving_stream(400, rate=50.0)
    assert [(t, w.name) for t, w in s[:20]] == [(t, w.name) for t, w in W.serving_stream(400, rate=50.0)[:20]]
    arrivals = np.array([t for t, _ in s])
    gaps = np.diff(np.concatenate([[0.0], arrivals]))
    assert np.all(gaps > 0) and abs(gaps.mean() - 1 / 50.0) < 0.3 / 50.0   # exponential, mean 1/rate
    frac63 = np.mean([w.n == 3 for _, w in s])
    assert 0.6 < frac63 < 0.8
    for _, w in s:
        assert len(w.measurements) <= 3
        times = [m.t for m in w.measurements]
        assert all(0 < t < w.t_end for t in times) and times == sorted(times)
        for m in w.measurements:
            assert m.y.shape == (w.n,) and np.allclose(m.R, 0.25 * np.eye(w.n))
        if w.n == 6:
            assert w.h == (0.5,) * 6 and np.allclose(w.cov, 0.25 * np.eye(6)) and 0.1 <= w.t_end <= 0.5


def test_capacity_grows_with_the_horizon_and_the_initial_set():
    w = W.lorenz63(h=0.25, t_end=0.25)
    c1 = W.capacity_for(w)
    assert c1 % 4096 == 0 and c1 >= W.initial_cells_estimate(w)
    assert W.capacity_for(w.with_(t_end=1.0)) > c1
    assert W.capacity_for(w.with_(h=(0.5,) * 3)) < c1
    assert W.capacity_for(w.with_(t_end=1e6)) == 1 << 24


def test_initial_cells_estimate_is_the_ellipsoid_volume_in_cells():
    # a unit-variance 3-D Gaussian, thr 1e-7: radius sqrt(2 ln 1e7) standard deviations
    w = W.lorenz63(h=0.5, t_end=0.1)
    r = np.sqrt(2 * np.log(1e7))
    expect = 4.0 / 3.0 * np.pi * r ** 3 / 0.5 ** 3
    assert abs(W.initial_cells_estimate(w) - expect) < 1e-9 * expect


def test_paper_cases():
    e1, e2 = W.paper_e1(), W.paper_e2()
    assert e1.dynamics == W.DYN_LORENZ63_SHIFTED and e1.params == (4.0, 1.0, 48.0) and e1.cfl == 1.0
    (m,) = e1.measurements
    assert m.t == 1.0 and m.y.tolist() == [-8.0] and m.H_idx.tolist() == [2] and m.R.tolist() == [[1.0]]
    assert e2.n == 6 and e2.h == (0.1,) * 6 and e2.mean[0] == 4.5 and e2.t_end == 1.3


def test_the_truth_integrator_is_fourth_order_and_converged_at_its_step():
    """The measurements' truth (RK4, dt = 1e-4) agrees with dt = 1e-5 far below
    the measurement noise, and halving a coarse step cuts the error by 2^4."""
    rhs = lambda x: W._l63_rhs(x, (10.0, 28.0, 8.0 / 3.0))
    x0 = np.array([-11.5, -10.0, 9.5])
    ref = W.truth_trajectory(rhs, x0, [0.25, 0.5], dt=1e-5)
    used = W.truth_trajectory(rhs, x0, [0.25, 0.5], dt=1e-4)
    assert max(np.abs(a - b).max() for a, b in zip(ref, used)) < 1e-9
    e1 = np.abs(W.truth_trajectory(rhs, x0, [0.5], dt=0.01)[0] - ref[1]).max()
    e2 = np.abs(W.truth_trajectory(rhs, x0, [0.5], dt=0.005)[0] - ref[1]).max()
    assert 12.0 < e1 / e2 < 20.0


def test_paper_e1_reading_reproduces_the_table_2_burden():
    """The threshold reading of the paper's Lorenz '63 case (1e-3 of the
    maximum): the oracle's own run of it (tests/golden/paper_e1_counts.txt,
    written by the oracle alone, read every 0.05) lies within small factors of
    the burden Table 2 prints (tests/golden/table2_lorenz63_burden.txt)."""
    import os

    here = os.path.join(os.path.dirname(__file__), "golden")
    ref = {}
    for line in open(os.path.join(here, "table2_lorenz63_burden.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            ref[k] = float(v)
    rows = [line.split() for line in open(os.path.join(here, "paper_e1_counts.txt"))
            if line.strip() and not line.startswith("#")]
    steps = sum(int(r[1]) for r in rows)
    updates = sum(int(r[2]) for r in rows)
    peak = max(int(r[3]) for r in rows)
    assert W.paper_e1().thr_rel == 1e-3 and len(rows) == 40
    assert 0.8 <= steps / ref["integration_steps"] <= 1.25, steps
    assert 0.5 <= peak / ref["max_grid_size"] <= 2.0, peak
    assert 0.5 <= updates / ref["cell_computations"] <= 2.0, updates
