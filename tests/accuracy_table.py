"""Accuracy of the CUDA library against the oracle per workload and precision:
L1 = (prod h) sum |p_gpu - p_oracle| over the union of the active sets, whether
the sets are identical, and the largest relative error of the mean and the
covariance. Test infrastructure (it runs the oracle); run on a machine with
the GPU, it prints a markdown table:

  python tests/accuracy_table.py
"""
import math
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from oracle.oracle import Oracle  # noqa: E402
from paper_2508_13986_gb300 import gbees, workloads as W  # noqa: E402

CASES = [
    ("lorenz63_h0.5 (to t = 0.5)", W.config("lorenz63_h0.5"), None),
    ("lorenz63_h0.25 (to t = 0.1)", W.config("lorenz63_h0.25"), 0.1),
    ("lorenz96_6d_h0.5 (to t = 0.1)", W.config("lorenz96_6d_h0.5"), 0.1),
    ("paper_e1 (measurement at 0.15, to t = 0.3)", None, None),
]


def e1_short():
    e1 = W.paper_e1()
    m = e1.measurements[0]
    return e1.with_(t_end=0.3, measurements=[W.Measurement(0.15, m.y, m.R, m.H_idx)])


def run(w, t_stop, precision):
    g = gbees.grid_for_workload(w, precision=precision, max_cells=W.capacity_for(w))
    o = Oracle(w.n, w.dynamics, w.params, w.h, w.x0, w.thr_rel, w.cfl, w.prune_interval, w.limiter)
    g.init_gaussian(w.mean, w.cov)
    o.init_gaussian(w.mean, w.cov)
    for t, meas in w.segments():
        t = min(t, t_stop)
        g.propagate(t)
        o.propagate(t)
        if meas is not None and t == meas.t:
            g.correct_gaussian(meas.y, meas.R, meas.H_idx)
            o.correct_gaussian(meas.y, meas.R, meas.H_idx)
        if t >= t_stop:
            break
    gi, gp = g.read_cells()
    oi, op = o.read_cells()
    same = gi.shape == oi.shape and np.array_equal(gi, oi)
    if same:
        l1 = math.prod(w.h) * math.fsum(np.abs(gp - op).tolist())
    else:
        dg = {tuple(r): v for r, v in zip(gi.tolist(), gp.tolist())}
        do = {tuple(r): v for r, v in zip(oi.tolist(), op.tolist())}
        l1 = math.prod(w.h) * math.fsum(abs(dg.get(k, 0.0) - do.get(k, 0.0)) for k in set(dg) | set(do))
    gm, gc = g.moments()
    om, oc = o.moments()
    em = float(np.abs(gm - om).max() / np.abs(om).max())
    ec = float(np.abs(gc - oc).max() / np.abs(oc).max())
    g.close()
    return same, l1, em, ec, oi.shape[0]


def main():
    print("| workload | precision | active cells | identical sets | L1 | mean rel. err | cov rel. err |")
    print("|---|---|---:|---|---:|---:|---:|")
    for name, w, t_stop in CASES:
        if w is None:
            w = e1_short()
        stop = t_stop if t_stop is not None else w.t_end
        for prec, tag in ((gbees.GBEES_FP64, "FP64"), (gbees.GBEES_FP32, "FP32")):
            same, l1, em, ec, n = run(w, stop, prec)
            print(f"| {name} | {tag} | {n} | {'yes' if same else 'no'} | {l1:.2e} | {em:.2e} | {ec:.2e} |", flush=True)


if __name__ == "__main__":
    main()
