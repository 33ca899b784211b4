"""The request loop's host logic on the CPU: admission in arrival order within
the memory budget, rounds of capped steps, the measurement schedule of every
request, release of finished and failed grids. The device is replaced by a
deterministic stand-in grid whose time advances by a fixed step."""
import math

import numpy as np
import pytest

from paper_2508_13986_gb300 import gbees, serving
from paper_2508_13986_gb300 import workloads as W

DT = 0.004  # the stand-in grid's time step


class FakeGrid:
    """Records what the loop asks of a grid; fails on demand (capacity)."""

    created = []

    def __init__(self, cfg, device="cuda:0", stream=None):
        self.cfg = cfg
        self.t = 0.0
        self.total = 0
        self.calls = []          # ("propagate", target, steps) / ("correct", y0)
        self.status = 0
        self.fail_after = None   # steps after which the grid runs out of capacity
        FakeGrid.created.append(self)

    def init_gaussian(self, mean, cov, t0=0.0):
        self.mean0 = np.asarray(mean, dtype=np.float64)
        self.t = t0
        self.total = 0

    def _advance(self, target, cap):
        need = max(0, math.ceil((target - self.t) / DT - 1e-9))
        k = need if cap <= 0 else min(cap, need)
        if self.fail_after is not None and self.total + k > self.fail_after:
            self.status = gbees.GBEES_ECAPACITY
            raise gbees.GbeesError(self.status, "capacity")
        self.total += k
        self.t = target if k == need else self.t + k * DT
        self.calls.append(("propagate", target, k))
        return gbees.Stats(k, 100 * k, self.t, DT, self.total, 100, 1.0, 150)

    def propagate(self, t_end):
        return self._advance(t_end, 0)

    def correct_gaussian(self, y, R, H_idx):
        self.calls.append(("correct", float(np.asarray(y)[0])))

    def stats(self):
        return gbees.Stats(0, 0, self.t, DT, self.total, 100, 1.0, 150)

    def moments(self):
        n = self.cfg.n
        corrections = sum(1 for c in self.calls if c[0] == "correct")
        return self.mean0 + self.total, np.eye(n) * (1 + corrections)

    def read_cells(self, sorted_=True):
        return np.zeros((1, self.cfg.n), dtype=np.int32), np.array([float(self.total)])

    def count(self):
        return 100

    def close(self):
        pass


def fake_batch(grids, targets, max_steps=0, max_blocks=0):
    out, err = [], None
    for g, t in zip(grids, targets):
        try:
            out.append(g._advance(t, max_steps))
        except gbees.GbeesError as e:
            out.append(None)
            err = e
    if err is not None:
        raise err
    return out


@pytest.fixture
def fake_device(monkeypatch):
    import torch

    FakeGrid.created = []
    monkeypatch.setattr(gbees, "Grid", FakeGrid)
    monkeypatch.setattr(gbees, "propagate_batch", fake_batch)
    monkeypatch.setattr(gbees, "gbees_workspace_bytes", lambda cfg: int(cfg.max_cells) * 100)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    return FakeGrid


def stream(count=12, seed=41):
    return W.serving_stream(count=count, rate=100.0, seed=seed, l96_sigma=0.3, l96_t=(0.02, 0.05),
                            l63_kw=dict(h_choices=(0.5,), t_range=(0.03, 0.08), sigma_range=(0.5, 1.0)))


def schedule_of(w):
    """(target, measurement y0 or None) per segment, as the workload defines it."""
    return [(t, None if m is None else float(m.y[0])) for t, m in w.segments()]


def replay(calls):
    """The segments a grid went through: its propagation targets (merging the
    capped rounds of one target) and the corrections after them."""
    segs = []
    for c in calls:
        if c[0] == "propagate":
            if not segs or segs[-1][0] != c[1] or segs[-1][1] is not None:
                segs.append([c[1], None])
        else:
            segs[-1][1] = c[1]
    return [tuple(s) for s in segs]


@pytest.mark.parametrize("mode", ["batched", "single"])
def test_every_request_follows_its_schedule_and_completes(fake_device, mode):
    st = stream()
    srv = serving.Server(realtime=False, mode=mode, round_steps=3)
    res = srv.run(st)
    assert len(res) == len(st) and srv.stats["failed"] == 0
    grids = fake_device.created
    assert len(grids) == len(st)
    for (arr, w), g, r in zip(st, grids, res):
        assert replay(g.calls) == schedule_of(w)
        assert g.t == w.t_end and r.steps == g.total
        assert r.error is None and r.finished >= r.arrival
        if mode == "batched":
            assert all(c[2] <= 3 for c in g.calls if c[0] == "propagate")   # the round cap
    if mode == "single":
        assert srv.stats["max_active"] == 1


def test_batched_and_single_serving_give_the_same_results(fake_device):
    st = stream(seed=42)
    a = serving.Server(realtime=False, mode="batched", round_steps=5).run(st)
    b = serving.Server(realtime=False, mode="single").run(st)
    for x, y in zip(a, b):
        assert x.steps == y.steps
        assert np.array_equal(x.mean, y.mean) and np.array_equal(x.cov, y.cov)


def test_admission_in_arrival_order_within_the_budget(fake_device):
    st = stream(count=16, seed=43)
    need = [W.capacity_for(w) * 100 for _, w in st]
    srv = serving.Server(realtime=False, pool_bytes=2 * max(need))
    res = srv.run(st)
    assert srv.stats["max_used_bytes"] <= srv.pool_bytes and srv.stats["max_active"] >= 1
    admitted = [r.admitted for r in res]
    assert admitted == sorted(admitted)          # first come, first admitted
    grids = fake_device.created
    assert [g.mean0.tolist() for g in grids] == [list(w.mean) for _, w in st]   # created in arrival order


def test_a_failing_grid_ends_alone_and_the_others_complete(fake_device, monkeypatch):
    st = stream(count=10, seed=44)
    orig = FakeGrid.__init__

    def init(self, cfg, device="cuda:0", stream=None):
        orig(self, cfg, device, stream)
        if len(FakeGrid.created) == 3:           # the third request runs out of capacity
            self.fail_after = 2

    monkeypatch.setattr(FakeGrid, "__init__", init)
    srv = serving.Server(realtime=False, round_steps=4)
    res = srv.run(st)
    assert len(res) == len(st) and srv.stats["failed"] == 1
    assert res[2].error == "ECAPACITY" and np.isnan(res[2].mean).all()
    assert all(r.error is None for i, r in enumerate(res) if i != 2)


def _failing(monkeypatch, which, method, exc):
    """Make the grid of the `which`-th request raise exc from `method`."""
    orig = getattr(FakeGrid, method)

    def wrapped(self, *a, **k):
        if FakeGrid.created.index(self) == which:
            raise exc
        return orig(self, *a, **k)

    monkeypatch.setattr(FakeGrid, method, wrapped)


@pytest.mark.parametrize("mode", ["batched", "single"])
def test_a_refused_initial_density_ends_that_request_alone(fake_device, monkeypatch, mode):
    st = stream(count=8, seed=45)
    _failing(monkeypatch, 2, "init_gaussian", gbees.GbeesError(gbees.GBEES_EKEYRANGE, "key range"))
    srv = serving.Server(realtime=False, mode=mode, round_steps=4)
    res = srv.run(st)
    assert len(res) == len(st) and srv.stats["failed"] == 1
    assert res[2].error == "EKEYRANGE" and res[2].steps == 0
    assert not any(c[0] == "propagate" for c in fake_device.created[2].calls)
    assert all(r.error is None for i, r in enumerate(res) if i != 2)


@pytest.mark.parametrize("mode", ["batched", "single"])
def test_a_degenerate_measurement_update_ends_that_request_alone(fake_device, monkeypatch, mode):
    st = stream(count=10, seed=46)
    which = next(i for i, (_, w) in enumerate(st) if any(m is not None for _, m in w.segments()))
    _failing(monkeypatch, which, "correct_gaussian", gbees.GbeesError(gbees.GBEES_EDEGENERATE, "C = 0"))
    srv = serving.Server(realtime=False, mode=mode, round_steps=4)
    res = srv.run(st)
    assert len(res) == len(st) and srv.stats["failed"] == 1
    assert res[which].error == "EDEGENERATE" and np.isnan(res[which].mean).all()
    assert all(r.error is None for i, r in enumerate(res) if i != which)


@pytest.mark.parametrize("exc,name", [(gbees.GbeesError(gbees.GBEES_EINVAL, "bad configuration"), "EINVAL"),
                                      ("oom", "ENOMEM")])
def test_a_grid_that_cannot_be_made_is_reported_and_the_stream_goes_on(fake_device, monkeypatch, exc, name):
    import torch

    if exc == "oom":
        exc = torch.cuda.OutOfMemoryError("no room")
    st = stream(count=6, seed=47)
    made = {"n": 0}

    def grid(cfg, device="cuda:0", stream=None):
        made["n"] += 1
        if made["n"] == 4:
            raise exc
        return FakeGrid(cfg, device, stream)

    monkeypatch.setattr(gbees, "Grid", grid)
    srv = serving.Server(realtime=False, round_steps=4)
    res = srv.run(st)
    assert len(res) == len(st) and srv.stats["failed"] == 1
    assert res[3].error == name and res[3].steps == 0
    assert len(fake_device.created) == len(st) - 1
    assert all(r.error is None for i, r in enumerate(res) if i != 3)
