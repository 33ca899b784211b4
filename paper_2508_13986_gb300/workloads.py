"""Seeded synthetic workloads (inputs only).

This module describes the problems that both the CUDA library and the test
oracle are run on: the model, its parameters, the grid, the initial Gaussian,
the time horizon and the measurement schedule. It holds none of the grid
method's arithmetic; the only computation here is the generation of synthetic
measurements from a seeded "truth" trajectory of the model ODE (classic RK4)
plus seeded Gaussian noise.

Workloads (the Lorenz systems are the paper's use cases, Sec. 5.1):
  lorenz63_h0.5   -- Lorenz '63 (sigma, rho, beta) = (10, 28, 8/3), mean
                     (-11.5, -10, 9.5), covariance I, h = 0.5, threshold 1e-7,
                     CFL 0.9, t_end = 0.5, no measurement (about 1e4 cells).
  lorenz63_h0.25  -- the same with h = 0.25, t_end = 2.0 and a full-state
                     Gaussian measurement (R = 0.25 I) every 0.25 time units
                     (10^5 - 10^6 cells).
  lorenz96_6d     -- Lorenz '96, n = 6, F = 4, mean (4.01, 4, 4, 4, 4, 4),
                     covariance 0.25 I, h = 0.25, threshold 1e-6, t_end = 1.0,
                     no measurement (10^6 - 10^7 cells).
  lorenz96_6d_h0.5 -- the same with h = 0.5 (a size the oracle can finish).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Optional, Sequence, Tuple

import numpy as np

# model identifiers shared by name (each side defines its own numeric enum with these values)
DYN_CONSTANT, DYN_LINEAR, DYN_LORENZ63, DYN_LORENZ63_SHIFTED, DYN_LORENZ96 = range(5)
LIM_MC, LIM_NONE, LIM_LW = range(3)

L63_PARAMS = (10.0, 28.0, 8.0 / 3.0)


@dataclass
class Measurement:
    t: float
    y: np.ndarray          # measured values of the components H_idx
    R: np.ndarray          # measurement covariance (m x m)
    H_idx: np.ndarray      # measured state components


@dataclass
class Workload:
    name: str
    n: int
    dynamics: int
    params: Tuple[float, ...]
    h: Tuple[float, ...]
    mean: Tuple[float, ...]
    cov: np.ndarray
    thr_rel: float
    cfl: float
    t_end: float
    prune_interval: int = 20
    limiter: int = LIM_MC
    measurements: List[Measurement] = field(default_factory=list)
    # largest pool (active cells plus halo) over the run, as a multiple of the
    # initial set: sizes the pool capacity of a run
    pool_growth: float = 24.0

    @property
    def x0(self) -> Tuple[float, ...]:
        """Grid origin: the centre of cell 0 sits on the initial mean."""
        return tuple(self.mean)

    def segments(self) -> List[Tuple[float, Optional[Measurement]]]:
        """(t_target, measurement at t_target or None) in time order."""
        out: List[Tuple[float, Optional[Measurement]]] = []
        for m in self.measurements:
            if m.t <= self.t_end:
                out.append((m.t, m))
        if not out or out[-1][0] < self.t_end:
            out.append((self.t_end, None))
        return out

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


def _l63_rhs(x, p):
    s, r, b = p
    return np.array([s * (x[1] - x[0]), x[0] * (r - x[2]) - x[1], x[0] * x[1] - b * x[2]])


def _l96_rhs(x, F):
    n = x.size
    return np.array([(x[(j + 1) % n] - x[(j - 2) % n]) * x[(j - 1) % n] - x[j] + F for j in range(n)])


def truth_trajectory(rhs, x0: np.ndarray, times: Sequence[float], dt: float = 1e-4) -> List[np.ndarray]:
    """Classic RK4 of dx/dt = rhs(x) sampled at the given increasing times."""
    x = np.array(x0, dtype=np.float64)
    t = 0.0
    out = []
    for tt in times:
        while t < tt - 1e-15:
            step = min(dt, tt - t)
            k1 = rhs(x)
            k2 = rhs(x + 0.5 * step * k1)
            k3 = rhs(x + 0.5 * step * k2)
            k4 = rhs(x + step * k3)
            x = x + step / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
            t += step
        out.append(x.copy())
    return out


def gaussian_measurements(rhs, mean, cov0, times, R, seed: int, dt: float = 1e-4) -> List[Measurement]:
    """Full-state measurements y_k = x(t_k) + nu_k of a truth started at mean + xi,
    xi ~ N(0, cov0), nu_k ~ N(0, R); NumPy PCG64 with the given seed; the truth
    is integrated by RK4 with step dt."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = len(mean)
    L0 = np.linalg.cholesky(np.asarray(cov0, dtype=np.float64))
    x0 = np.asarray(mean, dtype=np.float64) + L0 @ rng.standard_normal(n)
    xs = truth_trajectory(rhs, x0, times, dt)
    LR = np.linalg.cholesky(np.asarray(R, dtype=np.float64))
    out = []
    for t, x in zip(times, xs):
        y = x + LR @ rng.standard_normal(n)
        out.append(Measurement(float(t), y, np.array(R, dtype=np.float64), np.arange(n, dtype=np.int32)))
    return out


def lorenz63(h: float = 0.5, t_end: float = 0.5, thr_rel: float = 1e-7, cfl: float = 0.9,
             measure_every: Optional[float] = None, R_diag: float = 0.25, seed: int = 2508,
             prune_interval: int = 20, limiter: int = LIM_MC) -> Workload:
    mean = (-11.5, -10.0, 9.5)
    cov = np.eye(3)
    meas: List[Measurement] = []
    if measure_every:
        k = int(round(t_end / measure_every))
        times = [measure_every * (q + 1) for q in range(k)]
        meas = gaussian_measurements(lambda x: _l63_rhs(x, L63_PARAMS), mean, cov, times,
                                     R_diag * np.eye(3), seed)
    return Workload(name=f"lorenz63_h{h}", n=3, dynamics=DYN_LORENZ63, params=L63_PARAMS,
                    h=(h, h, h), mean=mean, cov=cov, thr_rel=thr_rel, cfl=cfl, t_end=t_end,
                    prune_interval=prune_interval, limiter=limiter, measurements=meas)


def lorenz96(h: float = 0.25, t_end: float = 1.0, thr_rel: float = 1e-6, cfl: float = 0.9,
             F: float = 4.0, n: int = 6, sigma2: float = 0.25, prune_interval: int = 20,
             limiter: int = LIM_MC) -> Workload:
    mean = tuple([F + 0.01] + [F] * (n - 1))
    return Workload(name=f"lorenz96_{n}d_h{h}", n=n, dynamics=DYN_LORENZ96, params=(F,),
                    h=tuple([h] * n), mean=mean, cov=sigma2 * np.eye(n), thr_rel=thr_rel, cfl=cfl,
                    t_end=t_end, prune_interval=prune_interval, limiter=limiter)


def lorenz63_batch(count: int = 256, seed: int = 2509, thr_rel: float = 1e-7, cfl: float = 0.9,
                   prune_interval: int = 20, h_choices=(0.25, 0.5), t_range=(0.25, 1.0),
                   sigma_range=(0.5, 2.0)) -> List[Workload]:
    """Independent classic Lorenz '63 grids for the batched propagation: means
    uniform in [-15, 15] x [-20, 20] x [5, 40], diagonal standard deviations
    uniform in sigma_range per axis, cell width drawn from h_choices, end times
    uniform in t_range (ragged grids of 10^3-10^5 cells). NumPy PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        mean = (rng.uniform(-15, 15), rng.uniform(-20, 20), rng.uniform(5, 40))
        sig = rng.uniform(sigma_range[0], sigma_range[1], 3)
        h = float(h_choices[int(rng.integers(len(h_choices)))])
        t_end = float(rng.uniform(t_range[0], t_range[1]))
        out.append(Workload(name=f"lorenz63_batch{count}_{i}", n=3, dynamics=DYN_LORENZ63, params=L63_PARAMS,
                            h=(h, h, h), mean=tuple(float(x) for x in mean), cov=np.diag(sig ** 2),
                            thr_rel=thr_rel, cfl=cfl, t_end=t_end, prune_interval=prune_interval))
    return out


def serving_stream(count: int = 1000, rate: float = 50.0, seed: int = 2510, frac_l63: float = 0.7,
                   l96_sigma: float = 0.5, l96_h: float = 0.5, l96_t=(0.1, 0.5), l63_kw=None,
                   max_corrections: int = 3) -> List[Tuple[float, Workload]]:
    """A seeded stream of propagation requests: Poisson arrivals at `rate` per
    second; a fraction frac_l63 are Lorenz '63 grids drawn like lorenz63_batch,
    the rest Lorenz '96 6-D grids (means 4 + N(0, 0.1^2) per component,
    standard deviation l96_sigma, h = l96_h, thr 1e-6, t_end uniform in l96_t).
    Each request carries 0..max_corrections full-state Gaussian measurements
    (R = 0.25 I) equally spaced in (0, t_end), drawn from a truth trajectory
    started at the mean plus N(0, cov) (RK4, step 5e-3). Returns (arrival
    seconds, workload)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    l63 = lorenz63_batch(count=count, seed=seed + 1, **(l63_kw or {}))
    out = []
    t = 0.0
    for i in range(count):
        t += float(rng.exponential(1.0 / rate))
        if rng.random() < frac_l63:
            w = l63[i]
            rhs = lambda x: _l63_rhs(x, L63_PARAMS)  # noqa: E731
        else:
            n = 6
            mean = tuple(float(x) for x in 4.0 + 0.1 * rng.standard_normal(n))
            t_end = float(rng.uniform(*l96_t))
            w = Workload(name=f"lorenz96_{n}d_req{i}", n=n, dynamics=DYN_LORENZ96, params=(4.0,),
                         h=tuple([l96_h] * n), mean=mean, cov=l96_sigma ** 2 * np.eye(n), thr_rel=1e-6, cfl=0.9,
                         t_end=t_end, prune_interval=20)
            rhs = lambda x: _l96_rhs(x, 4.0)  # noqa: E731
        m = int(rng.integers(0, max_corrections + 1))
        times = [w.t_end * (k + 1) / (m + 1) for k in range(m)]
        meas = gaussian_measurements(rhs, np.asarray(w.mean), w.cov, times, 0.25 * np.eye(w.n),
                                     seed=seed * 1000 + i, dt=5e-3) if m else []
        out.append((t, w.with_(name=f"req{i}_{w.name}", measurements=meas)))
    return out


def initial_cells_estimate(w: Workload) -> float:
    """Cells of the initial set: the volume of the ellipsoid p > thr * max p in
    cell units (a sizing aid for the capacity, not part of the method)."""
    r2 = -2.0 * np.log(w.thr_rel)
    n = w.n
    unit_ball = np.pi ** (n / 2) / math.gamma(n / 2 + 1)
    vol = unit_ball * r2 ** (n / 2) * np.sqrt(np.linalg.det(w.cov)) / np.prod(w.h)
    return float(vol)


def capacity_for(w: Workload) -> int:
    """Pool capacity (active plus halo entries) for propagating w to its t_end:
    the initial set times a growth bound measured on GB300 runs of these
    workloads (Lorenz '63: at most 36x by t = 1; Lorenz '96 6-D: at most 50x by
    t = 0.5), with margin, rounded up to a multiple of 4096 in 2^15..2^24. A
    sizing aid, not part of the method."""
    growth = 4.0 + (56.0 if w.n <= 3 else 120.0) * max(w.t_end, 0.0)
    want = growth * initial_cells_estimate(w) + 4096
    return int(min(1 << 24, max(1 << 15, math.ceil(want / 4096.0) * 4096)))


def paper_e1(thr_rel: float = 1e-3, prune_interval: int = 20) -> Workload:
    """The paper's Lorenz '63 validation case (Sec. 5.1.1): the shifted form with
    (sigma, b, r) = (4, 1, 48), initial Gaussian at (-11.5, -10, 9.5) with unit
    standard deviations, h = 0.5 (half the standard deviation, Table 2), CFL
    1.0, a measurement y = x3 = -8 with sigma_y = 1 at t = 1, end at t = 2.

    The paper does not state its threshold. A relative threshold of 1e-3 of the
    largest value gives the burden Table 2 prints for this case (about 24k cells
    at most, about 960 steps, about 6.5e6 cell computations): 972 steps and
    7.2e6 cell updates straight to the end, 1.8e4 active cells at most. Finer
    thresholds grow all three (1e-7: 1303 steps, 3.3e7 updates, 5.4e4 cells)."""
    meas = [Measurement(1.0, np.array([-8.0]), np.array([[1.0]]), np.array([2], dtype=np.int32))]
    return Workload(name="paper_e1", n=3, dynamics=DYN_LORENZ63_SHIFTED, params=(4.0, 1.0, 48.0),
                    h=(0.5, 0.5, 0.5), mean=(-11.5, -10.0, 9.5), cov=np.eye(3), thr_rel=thr_rel, cfl=1.0,
                    t_end=2.0, prune_interval=prune_interval, measurements=meas)


def paper_e2(thr_rel: float = 1e-4, prune_interval: int = 20) -> Workload:
    """The paper's Lorenz '96 validation case (Sec. 5.1.2): n = 6, F = 4, initial
    Gaussian at (F + 0.5, F, ..., F) with standard deviations 0.2, h = 0.1,
    CFL 1.0, no measurement, end at t = 1.3.

    The paper does not state its threshold. A relative threshold of 1e-4 of the
    largest value gives the burden Table 2 prints for this case (about 5e7 cells
    at most, about 1050 steps, about 3e10 cell computations): 4.2e7 active
    cells at most, 1038 steps and 2.7e10 cell updates. 1e-3 gives 5.4e6 cells
    and 792 steps, an order of magnitude below it. The pool peaks at 7.7e7
    entries at t = 1.1, 38 times the initial set."""
    F = 4.0
    return Workload(name="paper_e2", n=6, dynamics=DYN_LORENZ96, params=(F,), h=tuple([0.1] * 6),
                    mean=tuple([F + 0.5] + [F] * 5), cov=0.04 * np.eye(6), thr_rel=thr_rel, cfl=1.0, t_end=1.3,
                    prune_interval=prune_interval, pool_growth=48.0)


def config(name: str) -> Workload:
    """The named workloads of the benchmark and the parity tests."""
    if name == "paper_e1":
        return paper_e1()
    if name == "paper_e2":
        return paper_e2()
    if name == "lorenz63_h0.5":
        return lorenz63(h=0.5, t_end=0.5)
    if name == "lorenz63_h0.25":
        return lorenz63(h=0.25, t_end=2.0, measure_every=0.25)
    if name == "lorenz96_6d":
        return lorenz96(h=0.25, t_end=1.0)
    if name == "lorenz96_6d_h0.5":
        return lorenz96(h=0.5, t_end=1.0)
    raise KeyError(name)


def random_cells(n: int, count: int, radius: int, seed: int, p_scale: float = 1.0):
    """A seeded random set of distinct cells inside a box of the given radius
    with positive random values (for hashtable and step tests)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    side = 2 * radius + 1
    total = side ** n
    count = min(count, total)
    lin = rng.choice(total, size=count, replace=False)
    idx = np.zeros((count, n), dtype=np.int32)
    rem = lin.copy()
    for k in range(n - 1, -1, -1):
        idx[:, k] = (rem % side) - radius
        rem //= side
    p = p_scale * rng.random(count)
    return idx, p


def gaussian_blob_cells(n: int, radius: int, sigma_cells: float, shift=None):
    """All cells of a box with a Gaussian bump sampled at their centres; a dense
    stand-in for a smooth pdf on a fixed set (values are inputs, not results)."""
    side = 2 * radius + 1
    grids = np.meshgrid(*[np.arange(-radius, radius + 1)] * n, indexing="ij")
    idx = np.stack([g.reshape(-1) for g in grids], axis=1).astype(np.int32)
    s = np.zeros(n) if shift is None else np.asarray(shift, dtype=np.float64)
    d2 = (((idx - s) / sigma_cells) ** 2).sum(axis=1)
    return idx, np.exp(-0.5 * d2)
