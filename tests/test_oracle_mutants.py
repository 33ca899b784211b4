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
     "if (a >= 0) T.F[a] -= u * std::max(face_velocity(o, Yup, l), 0.0) * Fstar;",
     "if (a >= 0) T.F[a] += u * std::max(face_velocity(o, Yup, l), 0.0) * Fstar;"),
    ("transverse wave carried on from the cell downwind of the face (Algorithm 1)",
     "const Idx Y = u > 0.0 ? f.X[k] : shifted(f.X[k], j, -1);",
     "const Idx Y = u < 0.0 ? f.X[k] : shifted(f.X[k], j, -1);"),
    ("half of the transverse factor dropped (Algorithm 1)",
     "const double Fstar = dt / (2.0 * h[j]) *",
     "const double Fstar = dt / h[j] *"),
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
     "            for (auto& d : down[i]) keep.insert(d);\n",
     ""),
    ("Lorenz '63: wrong sign of x2 in f2",
     "if (j == 1) return x[0] * (a[1] - x[2]) - x[1];",
     "if (j == 1) return x[0] * (a[1] - x[2]) + x[1];"),
    ("shifted Lorenz '63: constant term b r replaced by r",
     "return -a[1] * x[2] + x[0] * x[1] - a[1] * a[2];",
     "return -a[1] * x[2] + x[0] * x[1] - a[2];"),
    ("Lorenz '96: x_{j-1} in place of x_{j-2}",
     "(x[(j + 1) % n] - x[(j + n - 2) % n])",
     "(x[(j + 1) % n] - x[(j + n - 1) % n])"),
    ("linear drift with A transposed",
     "s += a[j * c.n + k] * x[k];",
     "s += a[k * c.n + j] * x[k];"),
    ("likelihood without the factor 1/2 (Eq. 4)",
     "kv.second = std::exp(-0.5 * q) * kv.second;",
     "kv.second = std::exp(-q) * kv.second;"),
    ("likelihood residual against the wrong state component",
     "r[a] = y[a] - centre(o, kv.first, H_idx[a]);",
     "r[a] = y[a] - centre(o, kv.first, a);"),
    ("initial set thresholded at a tenth of p*",
     "if (g > pstar) kept[c].push_back({i, g});",
     "if (g > 0.1 * pstar) kept[c].push_back({i, g});"),
    ("cell volume taken as h_1^n",
     "for (int j = 0; j < cfg->n; ++j) o->prod_h *= cfg->h[j];",
     "for (int j = 0; j < cfg->n; ++j) o->prod_h *= cfg->h[0];"),
    ("exact sum that ignores the sign of a term",
     "int64_t sgn = x < 0 ? -1 : 1;",
     "int64_t sgn = 1;"),
]


def run_pins_against(i, old, new, tmp):
    lib = compile_variant(old, new, os.path.join(tmp, f"mutant{i}.so"))
    env = dict(os.environ, GBEES_ORACLE_LIB=lib, OMP_NUM_THREADS="1")  # many copies run at once
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
