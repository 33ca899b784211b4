"""Writes paper_e1_counts.txt: the paper's Lorenz '63 case (Sec. 5.1.1; the
shifted form, the x3-only measurement at t = 1, t_end 2) run through the oracle
alone, FP64, in steps of 0.05 of time: per interval, the target time, the time
steps and cell updates of the propagation to it, and the active cells after it
(after the measurement update at t = 1). The GPU's FP64 run of the same
schedule must take exactly these steps and updates. Calls only the oracle and
the input generators; takes several minutes.

    python tests/golden/make_paper_e1_counts.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle.oracle import Oracle  # noqa: E402
from paper_2508_13986_gb300 import workloads as W  # noqa: E402


def schedule():
    """Targets 0.05 k, k = 1..40, with the measurement (if any) due at each."""
    w = W.paper_e1()
    marks = {m.t: m for m in w.measurements}
    return w, [(0.05 * k, marks.get(round(0.05 * k, 12))) for k in range(1, 41)]


def main():
    w, targets = schedule()
    o = Oracle(w.n, w.dynamics, w.params, w.h, w.x0, w.thr_rel, w.cfl, w.prune_interval, w.limiter)
    o.init_gaussian(w.mean, w.cov)
    rows = []
    for t, meas in targets:
        st = o.propagate(t)
        if meas is not None:
            o.correct_gaussian(meas.y, meas.R, meas.H_idx)
        rows.append((t, st.steps, st.cell_updates, o.count()))
    with open(os.path.join(HERE, "paper_e1_counts.txt"), "w") as f:
        f.write("# The paper's Lorenz '63 case (Sec. 5.1.1) through the oracle, FP64, targets 0.05 k:\n")
        f.write("# the target time, the time steps and cell updates of the propagation to it, and the\n")
        f.write("# active cells after it (after the measurement update at t = 1).\n")
        f.write("# written by tests/golden/make_paper_e1_counts.py\n")
        f.write("# t_target steps cell_updates active_after\n")
        for t, s, u, n in rows:
            f.write(f"{t!r} {s} {u} {n}\n")


if __name__ == "__main__":
    main()
