"""Planted mistakes in the oracle, on the CPU: copies of the oracle source,
each with one plausible error (a sign, an index, a face, a dropped factor, a
missing term), must each fail at least one pin of test_oracle_pins.py. The
pins then fix the oracle's arithmetic, not only its shape. Each copy is
compiled with the oracle's own flags and loaded by the pins through
GBEES_ORACLE_LIB in a separate pytest process."""
import concurrent.futures
import os
import subprocess
import sys

from oracle.oracle import compile_variant

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (what the mistake is, text of the oracle source, the text planted instead)
MUTANTS = [
    ("transverse correction with the wrong sign (Algorithm 1)",
     "F[l][a] -= ujp * std::max(face_velocity(o, a, l), 0.0) * Fstar;",
     "F[l][a] += ujp * std::max(face_velocity(o, a, l), 0.0) * Fstar;"),
    ("half of the transverse factor dropped (Algorithm 1)",
     "double Fstar = dt / (2.0 * h[j]) *",
     "double Fstar = dt / h[j] *"),
    ("velocity at the upper face instead of the lower one (Eq. 7)",
     "y[j] = o.c.x0[j] + (X[j] - 0.5) * o.c.h[j];",
     "y[j] = o.c.x0[j] + (X[j] + 0.5) * o.c.h[j];"),
    ("upwind wave of the limiter taken on the wrong side",
     "double Wup = u > 0.0 ?",
     "double Wup = u < 0.0 ?"),
    ("factor (1 - nu) of the high-resolution term dropped",
     "(1.0 - dt * au / h[j])",
     "(1.0)"),
    ("MC limiter without the halving of (1 + theta)",
     "std::min((1.0 + theta) / 2.0, 2.0)",
     "std::min((1.0 + theta), 2.0)"),
    ("width of dimension 0 used in every term of the conservative update",
     "acc += dt / h[j] *",
     "acc += dt / h[0] *"),
    ("lower face counted outward when its velocity is positive (grow and prune)",
     "if (face_velocity(o, i, j) < 0.0) out.push_back({j, -1});",
     "if (face_velocity(o, i, j) > 0.0) out.push_back({j, -1});"),
    ("CFL rate without the absolute value (Eq. 8)",
     "r += std::fabs(face_velocity(o, i, j)) / o.c.h[j];",
     "r += face_velocity(o, i, j) / o.c.h[j];"),
    ("prune keeps the significant cells but not their downwind sets",
     "            for (auto& d : downwind(o, kv.first)) keep[d] = 1;\n",
     ""),
]


def run_pins_against(i, old, new, tmp):
    lib = compile_variant(old, new, os.path.join(tmp, f"mutant{i}.so"))
    env = dict(os.environ, GBEES_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join("tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    return r.returncode, r.stdout[-400:]


# a copy with a harmless edit: the harness itself must let every pin pass
CONTROL = ("control: a comment added, arithmetic unchanged",
           "double theta = Wup / W;",
           "double theta = Wup / W; /* unchanged */")


def test_every_planted_mistake_fails_a_pin(tmp_path):
    cases = [CONTROL] + MUTANTS
    workers = max(1, min(len(cases), os.cpu_count() or 1))
    with concurrent.futures.ThreadPoolExecutor(max_workers=workers) as pool:
        futs = [pool.submit(run_pins_against, i, old, new, str(tmp_path)) for i, (_, old, new) in enumerate(cases)]
        results = [f.result() for f in futs]
    assert results[0][0] == 0, results[0][1]            # the control passes every pin
    survivors = [(what, out) for (what, _, _), (rc, out) in zip(MUTANTS, results[1:]) if rc != 1]
    assert not survivors, survivors
