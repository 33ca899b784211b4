"""Writes the end states of full-length runs through the oracle alone (FP64),
for the GPU tests that compare the library's own full runs with them:

  lorenz63_h0.25_final.npz   the bench's Lorenz '63 workload (h = 0.25, eight
                             full-state measurements) at t = 2.0: every active
                             cell (sorted indices and densities)
  lorenz96_6d_step20.npz     the Lorenz '96 6-D workload (h = 0.25) after its
                             first 20 time steps, at the time the oracle reaches
  lorenz96_6d_h0.5_final.npz the same system with h = 0.5 over the whole
                             horizon, t = 1.0

The two 6-D states hold 10^6 to 10^7 cells, too many to store: they keep the
cell count, a SHA-256 of the sorted index array (int32, row-major), the mean
and covariance, and the indices and densities of 10^4 cells drawn uniformly
(seed 2508) from the sorted set. Every file also records the steps, the cell
updates and the time reached. Calls only the oracle (on all cores) and the
input generators; each 6-D part takes hours on an 8-core host (about 2.7 h for
c3_20 and 3 h for c3h05 with the two running side by side), c2 under a minute.

    python tests/golden/make_full_run_goldens.py [c2] [c3_20] [c3h05]
"""
import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle.oracle import Oracle  # noqa: E402
from paper_2508_13986_gb300 import workloads as W  # noqa: E402

SAMPLE = 10_000
SEED = 2508


def oracle_for(w):
    return Oracle(w.n, w.dynamics, w.params, w.h, w.x0, w.thr_rel, w.cfl, w.prune_interval, w.limiter)


def set_hash(idx: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(idx, dtype="<i4").tobytes()).hexdigest()


def summary(o, steps, updates, full: bool):
    idx, p = o.read_cells()
    mean, cov = o.moments()
    out = {"count": np.int64(len(p)), "set_sha256": np.array(set_hash(idx)), "mean": mean, "cov": cov,
           "steps": np.int64(steps), "cell_updates": np.int64(updates), "t": np.float64(o.t)}
    if full:
        out["idx"] = idx
        out["p"] = p
    else:
        rng = np.random.Generator(np.random.PCG64(SEED))
        pick = np.sort(rng.choice(len(p), size=min(SAMPLE, len(p)), replace=False))
        out["sample_idx"] = idx[pick]
        out["sample_p"] = p[pick]
    return out


def c2():
    w = W.config("lorenz63_h0.25")
    o = oracle_for(w)
    o.init_gaussian(w.mean, w.cov)
    steps = updates = 0
    for t, meas in w.segments():
        st = o.propagate(t)
        steps += st.steps
        updates += st.cell_updates
        if meas is not None:
            o.correct_gaussian(meas.y, meas.R, meas.H_idx)
    np.savez_compressed(os.path.join(HERE, "lorenz63_h0.25_final.npz"), **summary(o, steps, updates, True))


def c3_20():
    w = W.config("lorenz96_6d")
    # the time after 20 steps towards t_end, then a fresh run to exactly that
    # time (so that its last step is taken the way a propagate call takes it)
    o = oracle_for(w)
    o.init_gaussian(w.mean, w.cov)
    t20 = o.propagate(w.t_end, max_steps=20).t
    del o
    o = oracle_for(w)
    o.init_gaussian(w.mean, w.cov)
    st = o.propagate(t20)
    assert st.steps == 20, st
    np.savez_compressed(os.path.join(HERE, "lorenz96_6d_step20.npz"),
                        **summary(o, st.steps, st.cell_updates, False))


def c3h05():
    w = W.config("lorenz96_6d_h0.5")
    o = oracle_for(w)
    o.init_gaussian(w.mean, w.cov)
    st = o.propagate(w.t_end)
    np.savez_compressed(os.path.join(HERE, "lorenz96_6d_h0.5_final.npz"),
                        **summary(o, st.steps, st.cell_updates, False))


if __name__ == "__main__":
    parts = sys.argv[1:] or ["c2", "c3_20", "c3h05"]
    for name in parts:
        t0 = time.time()
        {"c2": c2, "c3_20": c3_20, "c3h05": c3h05}[name]()
        print(name, f"{time.time() - t0:.0f} s", flush=True)
