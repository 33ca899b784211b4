"""GPU parity: the CUDA library against the CPU oracle, cell by cell, on seeded
synthetic workloads (FP64: identical active sets and L1 <= 1e-10; FP32 store:
L1 <= 1e-5 and moments within 1e-4 relative)."""
import numpy as np
import pytest

from oracle.oracle import LIM_LW, LIM_MC, LIM_NONE
from paper_2508_13986_gb300 import gbees
from paper_2508_13986_gb300 import workloads as W
from parity_helpers import FP32_L1, FP32_MOM, assert_fp64_parity, compare, make_pair, run_schedule

pytestmark = pytest.mark.gpu



@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as ge
    ge.build()


def test_lorenz63_short_fp64():
    w = W.lorenz63(h=0.5, t_end=0.03, prune_interval=4)
    g, o = make_pair(w, max_cells=1 << 16)
    g.init_gaussian(w.mean, w.cov)
    o.init_gaussian(w.mean, w.cov)
    assert_fp64_parity(g, o, w)
    gst, ost = run_schedule(g, o, w)
    assert_fp64_parity(g, o, w, gst, ost)


def test_lorenz63_h05_to_t05_fp64():
    """The 10^4-cell Lorenz '63 workload (h = 0.5, t = 0.5) in full."""
    w = W.config("lorenz63_h0.5")
    g, o = make_pair(w, max_cells=1 << 16)
    g.init_gaussian(w.mean, w.cov)
    o.init_gaussian(w.mean, w.cov)
    gst, ost = run_schedule(g, o, w)
    assert_fp64_parity(g, o, w, gst, ost)
    gm, gc = g.moments()
    om, oc = o.moments()
    np.testing.assert_allclose(gm, om, rtol=0, atol=1e-10)
    np.testing.assert_allclose(gc, oc, rtol=0, atol=1e-10)


def test_lorenz63_h025_with_measurements_fp64():
    """The h = 0.25 Lorenz '63 workload with two measurement updates, on a short horizon."""
    base = W.lorenz63(h=0.25, t_end=0.06, measure_every=0.03)
    g, o = make_pair(base, max_cells=1 << 18)
    g.init_gaussian(base.mean, base.cov)
    o.init_gaussian(base.mean, base.cov)
    gst, ost = run_schedule(g, o, base)
    assert_fp64_parity(g, o, base, gst, ost)


@pytest.mark.parametrize("prec", [gbees.GBEES_FP32])
def test_lorenz63_fp32_store(prec):
    w = W.lorenz63(h=0.5, t_end=0.1, measure_every=0.05, prune_interval=5)
    g, o = make_pair(w, precision=prec, max_cells=1 << 16)
    g.init_gaussian(w.mean, w.cov)
    o.init_gaussian(w.mean, w.cov)
    run_schedule(g, o, w)
    same, l1, ng, no, _, _ = compare(g, o, w.h)
    assert l1 <= FP32_L1, l1
    gm, gc = g.moments()
    om, oc = o.moments()
    assert np.abs(gm - om).max() <= FP32_MOM * np.abs(om).max()
    assert np.abs(gc - oc).max() <= FP32_MOM * np.abs(oc).max()


def test_lorenz96_6d_h05_short_fp64():
    w = W.lorenz96(h=0.5, t_end=0.06, prune_interval=2)
    g, o = make_pair(w, max_cells=1 << 20)
    g.init_gaussian(w.mean, w.cov)
    o.init_gaussian(w.mean, w.cov)
    assert_fp64_parity(g, o, w)
    gst, ost = run_schedule(g, o, w)
    assert_fp64_parity(g, o, w, gst, ost)


def test_lorenz96_6d_h05_short_fp32_store():
    """FP32 storage and fluxes on the 6-D grid: L1 and moments within the FP32 bar."""
    w = W.lorenz96(h=0.5, t_end=0.06, prune_interval=2)
    g, o = make_pair(w, precision=gbees.GBEES_FP32, max_cells=1 << 20)
    g.init_gaussian(w.mean, w.cov)
    o.init_gaussian(w.mean, w.cov)
    run_schedule(g, o, w)
    _, l1, _, _, _, _ = compare(g, o, w.h)
    assert l1 <= FP32_L1, l1
    gm, gc = g.moments()
    om, oc = o.moments()
    assert np.abs(gm - om).max() <= FP32_MOM * np.abs(om).max()
    assert np.abs(gc - oc).max() <= FP32_MOM * np.abs(oc).max()


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("lim", [LIM_MC, LIM_NONE, LIM_LW])
def test_random_sets_linear_dynamics_fp64(n, lim):
    """Ragged random cell sets under a random linear drift (mixed velocity signs):
    grow, update and prune against the oracle for every dimension and limiter."""
    rng = np.random.default_rng(100 + 10 * n + lim)
    A = rng.standard_normal((n, n))
    b = rng.standard_normal(n)
    radius = {1: 40, 2: 9, 3: 5, 4: 3, 5: 2, 6: 2}[n]
    idx, p = W.random_cells(n, 3000, radius, seed=n * 7 + lim)
    h = rng.uniform(0.3, 0.7, n)
    x0 = rng.standard_normal(n)
    w = W.Workload(name="rand", n=n, dynamics=W.DYN_LINEAR, params=tuple(A.reshape(-1)) + tuple(b), h=tuple(h),
                   mean=tuple(x0), cov=np.eye(n), thr_rel=0.05, cfl=0.8, t_end=0.0, prune_interval=2, limiter=lim)
    # sparse sets in high dimension: the halo (missing face neighbours) outnumbers the active cells
    g, o = make_pair(w, max_cells=1 << 20)
    g.init_cells(idx, p)
    o.init_cells(idx, p)
    for k in range(1, 4):
        gs = g.propagate(0.05 * k)
        os_ = o.propagate(0.05 * k)
        assert gs.steps == os_.steps and gs.t == os_.t
        assert_fp64_parity(g, o, w)


@pytest.mark.parametrize("pw", [2, 4, 8, 16, 32])
def test_probe_widths_agree(pw):
    w = W.lorenz63(h=0.5, t_end=0.02, prune_interval=3)
    g, o = make_pair(w, max_cells=1 << 16, probe_width=pw)
    g.init_gaussian(w.mean, w.cov)
    o.init_gaussian(w.mean, w.cov)
    gst, ost = run_schedule(g, o, w)
    assert_fp64_parity(g, o, w, gst, ost)


def test_measurement_update_matches_oracle():
    w = W.lorenz63(h=0.5, t_end=0.0)
    g, o = make_pair(w, max_cells=1 << 16)
    g.init_gaussian(w.mean, w.cov)
    o.init_gaussian(w.mean, w.cov)
    y, R, H = np.array([-11.0, 9.9]), np.array([[0.5, 0.1], [0.1, 0.4]]), np.array([0, 2], dtype=np.int32)
    g.correct_gaussian(y, R, H)
    o.correct_gaussian(y, R, H)
    assert_fp64_parity(g, o, w)
    gm, gc = g.moments()
    om, oc = o.moments()
    np.testing.assert_allclose(gm, om, atol=1e-12)
    np.testing.assert_allclose(gc, oc, atol=1e-12)


def test_edge_cases():
    w = W.lorenz63(h=0.5, t_end=0.0)
    # t_end <= t takes no step
    g, o = make_pair(w, max_cells=1 << 16)
    g.init_gaussian(w.mean, w.cov)
    st = g.propagate(0.0)
    assert st.steps == 0 and st.t == 0.0
    st = g.propagate(-1.0)
    assert st.steps == 0
    # a single cell
    g.init_cells(np.zeros((1, 3), dtype=np.int32), np.array([8.0]))
    o.init_cells(np.zeros((1, 3), dtype=np.int32), np.array([8.0]))
    g.propagate(0.01)
    o.propagate(0.01)
    assert_fp64_parity(g, o, w)
    # an empty grid is degenerate on the first step
    g.init_cells(np.zeros((0, 3), dtype=np.int32), np.zeros(0))
    assert g.count() == 0
    with pytest.raises(gbees.GbeesError) as e:
        g.propagate(0.01)
    assert e.value.status == gbees.GBEES_EDEGENERATE
    # a new grid clears the poisoned state
    g.init_gaussian(w.mean, w.cov)
    assert g.status == 0
    # capacity overflow on growth: room for the initial cells and their halo only
    g.init_gaussian(w.mean, w.cov)
    pool0 = g.stats().n_pool
    assert pool0 > g.count()
    small = gbees.grid_for_workload(w, max_cells=pool0 + 16)
    small.init_gaussian(w.mean, w.cov)
    with pytest.raises(gbees.GbeesError) as e:
        small.propagate(0.5)
    assert e.value.status == gbees.GBEES_ECAPACITY
    with pytest.raises(gbees.GbeesError):
        small.propagate(0.6)
    # capacity overflow at init
    tiny = gbees.grid_for_workload(w, max_cells=100)
    with pytest.raises(gbees.GbeesError) as e:
        tiny.init_gaussian(w.mean, w.cov)
    assert e.value.status == gbees.GBEES_ECAPACITY
    # key range (21 bits per dimension for n = 3; active cells one layer inside it):
    # growth across the edge of the range
    cfg = gbees.make_config(3, gbees.GBEES_DYN_CONSTANT, (1.0, 0.0, 0.0), [1.0] * 3, [0.0] * 3, max_cells=64)
    edge = gbees.Grid(cfg)
    with pytest.raises(gbees.GbeesError) as e:
        edge.init_cells(np.array([[2 ** 20 - 1, 0, 0]], dtype=np.int32), np.array([1.0]))
    assert e.value.status == gbees.GBEES_EKEYRANGE
    edge.init_cells(np.array([[2 ** 20 - 2, 0, 0]], dtype=np.int32), np.array([1.0]))
    with pytest.raises(gbees.GbeesError) as e:
        edge.propagate(0.5)
    assert e.value.status == gbees.GBEES_EKEYRANGE
    with pytest.raises(gbees.GbeesError) as e:
        g.init_cells(np.array([[2 ** 20, 0, 0]], dtype=np.int32), np.array([1.0]))
    assert e.value.status == gbees.GBEES_EKEYRANGE
    # duplicate cells are rejected
    with pytest.raises(gbees.GbeesError):
        g.init_cells(np.zeros((2, 3), dtype=np.int32), np.ones(2))


def test_checkpoint_and_resume():
    w = W.lorenz63(h=0.5, t_end=0.05, prune_interval=3)
    g, _ = make_pair(w, max_cells=1 << 16)
    g.init_gaussian(w.mean, w.cov)
    g.propagate(0.02)
    idx, p = g.read_cells()
    st = g.stats()
    g.propagate(0.05)
    i1, p1 = g.read_cells()
    h, _ = make_pair(w.with_(prune_interval=3), max_cells=1 << 16)
    h.init_cells(idx, p, t0=st.t, step0=st.total_steps)
    h.propagate(0.05)
    i2, p2 = h.read_cells()
    assert np.array_equal(i1, i2)
    assert np.abs(p1 - p2).max() <= 1e-13 * p1.max()


def test_storage_order_readout_is_a_permutation():
    w = W.lorenz63(h=0.5, t_end=0.02)
    g, _ = make_pair(w, max_cells=1 << 16)
    g.init_gaussian(w.mean, w.cov)
    g.propagate(0.02)
    a, pa = g.read_cells(sorted_=True)
    b, pb = g.read_cells(sorted_=False)
    order = np.lexsort(b.T[::-1])
    assert np.array_equal(a, b[order]) and np.array_equal(pa, pb[order])


def test_very_unlikely_measurement_matches_oracle():
    """A measurement 20 sigma away: the likelihood is ~1e-218 everywhere, yet the
    posterior is well defined and both implementations agree."""
    w = W.lorenz63(h=0.5, t_end=0.0)
    g, o = make_pair(w, max_cells=1 << 16)
    g.init_gaussian(w.mean, w.cov)
    o.init_gaussian(w.mean, w.cov)
    y, R, H = np.array([-11.0, -10.5]), np.array([[0.5, 0.1], [0.1, 0.4]]), np.array([0, 2], dtype=np.int32)
    g.correct_gaussian(y, R, H)
    o.correct_gaussian(y, R, H)
    assert_fp64_parity(g, o, w)
    g.propagate(0.01)
    o.propagate(0.01)
    assert_fp64_parity(g, o, w)


@pytest.mark.parametrize("prec", [gbees.GBEES_FP64, gbees.GBEES_FP32])
def test_launch_modes_agree_bitwise(prec):
    """The persistent step-loop kernel, the CUDA-graph loop and one launch per kernel
    run the same phase code and exact reductions: identical bits."""
    w = W.lorenz63(h=0.5, t_end=0.06, measure_every=0.03, prune_interval=4)
    modes = [gbees.GBEES_LAUNCH_PERSISTENT, gbees.GBEES_LAUNCH_GRAPH, gbees.GBEES_LAUNCH_DIRECT]
    res = []
    for mode in modes:
        g = gbees.grid_for_workload(w, precision=prec, max_cells=1 << 16, launch_mode=mode)
        g.init_gaussian(w.mean, w.cov)
        for t_target, meas in w.segments():
            g.propagate(t_target)
            if meas is not None:
                g.correct_gaussian(meas.y, meas.R, meas.H_idx)
        res.append((*g.read_cells(), g.stats().total_steps))
        g.close()
    for i, p, s in res[1:]:
        assert np.array_equal(i, res[0][0]) and np.array_equal(p, res[0][1]) and s == res[0][2]


def test_profiled_direct_path_times_every_phase():
    w = W.lorenz63(h=0.5, t_end=0.03, prune_interval=4)
    g = gbees.grid_for_workload(w, max_cells=1 << 16)
    g.profile(enable=True, reset=True)
    g.init_gaussian(w.mean, w.cov)
    st = g.propagate(w.t_end)
    prof = g.profile(enable=False)
    for k in ("grow", "halo", "link", "faces", "apply"):
        assert prof["timed"][k] >= st.steps and prof["ms"][k] > 0
    assert prof["timed"]["grow"] >= st.steps and prof["launches"]["prune"] >= 5


def test_paper_e1_shifted_lorenz63_with_x3_measurement_fp64():
    """The paper's Lorenz '63 case (shifted form, CFL 1.0, a measurement of x3
    alone), with its measurement moved to t = 0.15 and the end to t = 0.3 so
    that the oracle finishes in seconds."""
    e1 = W.paper_e1()
    m = e1.measurements[0]
    w = e1.with_(t_end=0.3, measurements=[W.Measurement(0.15, m.y, m.R, m.H_idx)])
    g, o = make_pair(w, max_cells=1 << 17)
    g.init_gaussian(w.mean, w.cov)
    o.init_gaussian(w.mean, w.cov)
    gst, ost = run_schedule(g, o, w)
    assert_fp64_parity(g, o, w, gst, ost)
    gm, gc = g.moments()
    om, oc = o.moments()
    np.testing.assert_allclose(gm, om, atol=1e-12)
    np.testing.assert_allclose(gc, oc, atol=1e-12)
