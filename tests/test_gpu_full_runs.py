"""Full-length runs through the library against end states written by the
oracle alone (tests/golden/make_full_run_goldens.py), in the launch
configuration the bench uses (launch mode AUTO, key storage order):

  - the bench's Lorenz '63 workload (h = 0.25, eight full-state measurements)
    to t = 2.0: every active cell of the oracle's final density is stored;
  - the Lorenz '96 6-D workload (h = 0.25) after its first 20 time steps;
  - the same system with h = 0.5 over its whole horizon, t = 1.0.

FP64 must give the oracle's steps and cell updates, the identical active set
(a SHA-256 of the sorted indices for the 6-D states) and L1 within 1e-10
(computed exactly where the golden holds every cell, estimated from 10^4
uniformly drawn cells otherwise, with the largest sampled error bounded too);
FP32 storage must stay within L1 1e-5 and relative moment errors 1e-4 of the
FP64 oracle. In FP64 the bench workload must also take the oracle's steps and
updates segment by segment (tests/golden/bench_workload_counts.txt)."""
import hashlib
import math
import os

import numpy as np
import pytest

from paper_2508_13986_gb300 import gbees
from paper_2508_13986_gb300 import workloads as W
from parity_helpers import FP32_L1, FP32_MOM, FP64_L1

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as ge
    ge.build()


def golden(name):
    return dict(np.load(os.path.join(GOLDEN, name)))


def golden_counts():
    rows = []
    for line in open(os.path.join(GOLDEN, "bench_workload_counts.txt")):
        if line.strip() and not line.startswith("#"):
            t, s, u, n = line.split()
            rows.append((float(t), int(s), int(u), int(n)))
    return rows


def packed(idx):
    """Sortable 64-bit code of int32 index rows (lexicographic order, |i| < 2^9 in 6-D, 2^20 in 3-D)."""
    n = idx.shape[1]
    bits = 63 // n
    out = np.zeros(idx.shape[0], dtype=np.int64)
    for k in range(n):
        out = (out << bits) | (idx[:, k].astype(np.int64) + (1 << (bits - 1)))
    return out


def moment_errors(mean, cov, g):
    em = np.linalg.norm(mean - g["mean"]) / np.linalg.norm(g["mean"])
    ec = np.linalg.norm(cov - g["cov"]) / np.linalg.norm(g["cov"])
    return em, ec


def run_grid(w, precision, t_end, max_cells, segments=True):
    g = gbees.grid_for_workload(w, precision=precision, max_cells=max_cells)
    g.init_gaussian(w.mean, w.cov)
    rows, steps, updates = [], 0, 0
    for t, meas in (w.segments() if segments else [(t_end, None)]):
        st = g.propagate(min(t, t_end))
        steps += st.steps
        updates += st.cell_updates
        if meas is not None:
            g.correct_gaussian(meas.y, meas.R, meas.H_idx)
        rows.append((t, st.steps, st.cell_updates, g.count()))
        if t >= t_end:
            break
    return g, rows, steps, updates


@pytest.mark.parametrize("prec", [gbees.GBEES_FP64, gbees.GBEES_FP32])
def test_bench_workload_final_density_against_the_oracle(prec):
    w = W.config("lorenz63_h0.25")
    gd = golden("lorenz63_h0.25_final.npz")
    g, rows, steps, updates = run_grid(w, prec, w.t_end, 1 << 22)
    st = g.stats()
    assert st.t == float(gd["t"])
    idx, p = g.read_cells(sorted_=True)
    mean, cov = g.moments()
    g.close()
    oi, op = gd["idx"], gd["p"]
    em, ec = moment_errors(mean, cov, gd)
    if prec == gbees.GBEES_FP64:
        assert rows == golden_counts()                 # segment by segment
        assert steps == int(gd["steps"]) and updates == int(gd["cell_updates"])
        assert np.array_equal(idx, oi)
        l1 = math.prod(w.h) * math.fsum(np.abs(p - op).tolist())
        assert l1 <= FP64_L1, l1
        assert em <= 1e-12 and ec <= 1e-10, (em, ec)
    else:
        # union of the two sets, a missing cell counting as 0
        ka, kb = packed(idx), packed(oi)
        keys = np.union1d(ka, kb)
        pa = np.zeros(keys.size)
        pb = np.zeros(keys.size)
        pa[np.searchsorted(keys, ka)] = p
        pb[np.searchsorted(keys, kb)] = op
        l1 = math.prod(w.h) * math.fsum(np.abs(pa - pb).tolist())
        assert l1 <= FP32_L1, l1
        assert em <= FP32_MOM and ec <= FP32_MOM, (em, ec)


def check_sampled(w, gd, idx, p, mean, cov, fp64):
    """Set, sampled densities and moments against a 6-D golden."""
    em, ec = moment_errors(mean, cov, gd)
    pos = np.searchsorted(packed(idx), packed(gd["sample_idx"]))
    pos = np.minimum(pos, len(p) - 1)
    found = np.all(idx[pos] == gd["sample_idx"], axis=1)
    got = np.where(found, p[pos], 0.0)
    err = np.abs(got - gd["sample_p"])
    # L1 estimated from the uniform sample of the oracle's cells
    l1_est = math.prod(w.h) * int(gd["count"]) * float(err.mean())
    if fp64:
        assert len(p) == int(gd["count"])
        sha = hashlib.sha256(np.ascontiguousarray(idx, dtype="<i4").tobytes()).hexdigest()
        assert sha == str(gd["set_sha256"])
        assert found.all()
        assert l1_est <= FP64_L1, l1_est
        assert float(err.max()) <= 1e-12 * float(np.abs(gd["sample_p"]).max())
        assert em <= 1e-12 and ec <= 1e-10, (em, ec)
    else:
        assert abs(len(p) - int(gd["count"])) <= 1e-3 * int(gd["count"])
        assert l1_est <= FP32_L1, l1_est
        assert em <= FP32_MOM and ec <= FP32_MOM, (em, ec)


@pytest.mark.parametrize("prec", [gbees.GBEES_FP64, gbees.GBEES_FP32])
def test_lorenz96_6d_first_20_steps_against_the_oracle(prec):
    w = W.config("lorenz96_6d")
    gd = golden("lorenz96_6d_step20.npz")
    g, _, steps, updates = run_grid(w, prec, float(gd["t"]), 1 << 26, segments=False)
    assert steps == 20 and g.stats().t == float(gd["t"])
    if prec == gbees.GBEES_FP64:
        assert updates == int(gd["cell_updates"])
    idx, p = g.read_cells(sorted_=True)
    mean, cov = g.moments()
    g.close()
    check_sampled(w, gd, idx, p, mean, cov, prec == gbees.GBEES_FP64)


@pytest.mark.parametrize("prec", [gbees.GBEES_FP64, gbees.GBEES_FP32])
def test_lorenz96_6d_h05_whole_horizon_against_the_oracle(prec):
    w = W.config("lorenz96_6d_h0.5")
    gd = golden("lorenz96_6d_h0.5_final.npz")
    g, _, steps, updates = run_grid(w, prec, w.t_end, 1 << 24, segments=False)
    assert g.stats().t == float(gd["t"])
    if prec == gbees.GBEES_FP64:
        assert steps == int(gd["steps"]) and updates == int(gd["cell_updates"])
    idx, p = g.read_cells(sorted_=True)
    mean, cov = g.moments()
    g.close()
    check_sampled(w, gd, idx, p, mean, cov, prec == gbees.GBEES_FP64)
