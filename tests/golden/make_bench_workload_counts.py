"""Writes bench_workload_counts.txt: the time steps and cell updates of the
Lorenz '63 h = 0.25 workload (t_end 2, eight full-state measurements) run
through the oracle alone, FP64, segment by segment. The GPU's FP64 run of the
same workload must take exactly these steps and updates (identical active
sets at every step give identical counts). Calls only the oracle and the input
generators; takes a few minutes.

    python tests/golden/make_bench_workload_counts.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle.oracle import Oracle  # noqa: E402
from paper_2508_13986_gb300 import workloads as W  # noqa: E402


def main():
    w = W.config("lorenz63_h0.25")
    o = Oracle(w.n, w.dynamics, w.params, w.h, w.x0, w.thr_rel, w.cfl, w.prune_interval, w.limiter)
    o.init_gaussian(w.mean, w.cov)
    rows = []
    for t, meas in w.segments():
        st = o.propagate(t)
        if meas is not None:
            o.correct_gaussian(meas.y, meas.R, meas.H_idx)
        rows.append((t, st.steps, st.cell_updates, o.count()))
    with open(os.path.join(HERE, "bench_workload_counts.txt"), "w") as f:
        f.write("# Lorenz '63 h = 0.25, t_end 2, eight full-state measurements (the bench workload), FP64,\n")
        f.write("# through the oracle: per segment, the target time, the time steps and cell updates of\n")
        f.write("# the propagation to it, and the active cells after its measurement update.\n")
        f.write("# written by tests/golden/make_bench_workload_counts.py\n")
        f.write("# t_target steps cell_updates active_after\n")
        for t, s, u, n in rows:
            f.write(f"{t!r} {s} {u} {n}\n")


if __name__ == "__main__":
    main()
