"""The C-ABI library builds, loads and exports every entry point that
include/gbees.h declares; host-only calls work without a GPU."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2508_13986_gb300 import gbees
from paper_2508_13986_gb300.build import LIB, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gbees.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^[A-Za-z_][\w\s\*]*?\b(gbees_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    build()
    return ctypes.CDLL(LIB)


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("gbees_workspace_bytes", "gbees_create", "gbees_init_gaussian", "gbees_init_cells",
                 "gbees_propagate", "gbees_correct_gaussian", "gbees_count", "gbees_read_cells",
                 "gbees_moments", "gbees_get_stats", "gbees_get_status", "gbees_last_error", "gbees_destroy"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", LIB], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (gbees_\w+)", out))
    for name in declared_functions():
        assert name in exported, name
        getattr(lib, name)


def test_binding_wraps_every_declared_symbol():
    for name in declared_functions():
        assert name in gbees._SIGNATURES, name
        assert callable(getattr(gbees, name))


def test_workspace_bytes_is_host_only_and_validates(lib):
    gbees.load_library()
    cfg = gbees.make_config(3, gbees.GBEES_DYN_LORENZ63, (10, 28, 8 / 3), [0.5] * 3, [0, 0, 0], max_cells=1000)
    nb = gbees.gbees_workspace_bytes(cfg)
    # 2 keys + 2 p + 2 x 6 links + keep + map per cell, 2048 table slots of 16 B, scalars
    assert nb >= 1000 * (16 + 16 + 48 + 1 + 4) + 2048 * 16
    cfg32 = gbees.make_config(3, gbees.GBEES_DYN_LORENZ63, (10, 28, 8 / 3), [0.5] * 3, [0, 0, 0],
                              max_cells=1000, precision=gbees.GBEES_FP32)
    assert gbees.gbees_workspace_bytes(cfg32) < nb
    bad = [
        gbees.make_config(3, gbees.GBEES_DYN_LORENZ96, (4,), [0.5] * 3, [0, 0, 0]),   # L96 needs n >= 4
        gbees.make_config(2, gbees.GBEES_DYN_LORENZ63, (10, 28, 8 / 3), [0.5] * 2, [0, 0]),
        gbees.make_config(7, gbees.GBEES_DYN_CONSTANT, (1,) * 7, [0.5] * 6, [0] * 6),
        gbees.make_config(3, gbees.GBEES_DYN_CONSTANT, (1, 1, 1), [0.5, 0.0, 0.5], [0, 0, 0]),
        gbees.make_config(3, gbees.GBEES_DYN_CONSTANT, (1, 1, 1), [0.5] * 3, [0, 0, 0], cfl=0.0),
        gbees.make_config(3, gbees.GBEES_DYN_CONSTANT, (1, 1, 1), [0.5] * 3, [0, 0, 0], probe_width=3),
        gbees.make_config(3, gbees.GBEES_DYN_CONSTANT, (1, 1, 1), [0.5] * 3, [0, 0, 0], max_cells=0),
        gbees.make_config(3, gbees.GBEES_DYN_CONSTANT, (1, 1, 1), [0.5] * 3, [0, 0, 0], table_factor=1.1),
        gbees.make_config(3, gbees.GBEES_DYN_CONSTANT, (1, 1, 1), [0.5] * 3, [0, 0, 0], thr_rel=1.5),
    ]
    for c in bad:
        assert gbees.gbees_workspace_bytes(c) == 0


def test_create_rejects_a_short_or_misaligned_workspace(lib):
    cfg = gbees.make_config(3, gbees.GBEES_DYN_CONSTANT, (1, 1, 1), [0.5] * 3, [0, 0, 0], max_cells=100)
    nb = gbees.gbees_workspace_bytes(cfg)
    rc, ctx = gbees.gbees_create(cfg, 0, nb, 0)
    assert rc == gbees.GBEES_EINVAL and ctx == 0
    rc, ctx = gbees.gbees_create(cfg, 256 * 1000, nb - 1, 0)
    assert rc == gbees.GBEES_EINVAL and ctx == 0
    rc, ctx = gbees.gbees_create(cfg, 256 * 1000 + 8, nb, 0)
    assert rc == gbees.GBEES_EINVAL and ctx == 0


def test_every_entry_point_refuses_a_null_context(lib):
    """A NULL context is GBEES_EINVAL (or a no-op for destroy) before any CUDA
    call; nothing here needs a GPU."""
    gbees.load_library()
    E = gbees.GBEES_EINVAL
    d = np.zeros(9)
    i = np.zeros(9, dtype=np.int32)
    st = gbees.gbees_stats()
    assert gbees.gbees_init_gaussian(0, d[:3], d, 0.0) == E
    assert gbees.gbees_init_cells(0, i[:3], d[:1], 0.0, 0) == E
    assert gbees.gbees_propagate(0, 1.0, st) == E
    assert gbees.gbees_correct_gaussian(0, d[:1], d[:1], i[:1]) == E
    assert gbees.gbees_count(0)[0] == E
    assert gbees.gbees_read_cells(0, i[:3].reshape(1, 3), d[:1], True)[0] == E
    assert gbees.gbees_moments(0, d[:3], d) == E
    assert gbees.gbees_get_stats(0, st) == E
    assert gbees.gbees_get_status(0) == E
    assert gbees.gbees_profile_control(0, True, False) == E
    assert gbees.gbees_profile_read(0, gbees.gbees_profile()) == E
    assert isinstance(gbees.gbees_last_error(0), str)
    gbees.gbees_destroy(0)


def test_batch_arguments_are_checked_before_any_launch(lib):
    gbees.load_library()
    E = gbees.GBEES_EINVAL
    assert gbees.gbees_batch_workspace_bytes(0) == 0
    nb = gbees.gbees_batch_workspace_bytes(2)
    assert nb > 0
    f = gbees._f("gbees_batch_propagate")
    ctxs = (ctypes.c_void_p * 2)(0, 0)
    t_end = np.ones(2)
    stats = (gbees.gbees_stats * 2)()
    dp = t_end.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert f(None, 2, dp, 0, ctypes.c_void_p(256), nb, stats) == E                 # no contexts
    assert f(ctxs, 0, dp, 0, ctypes.c_void_p(256), nb, stats) == E                 # empty batch
    assert f(ctxs, 2, dp, -1, ctypes.c_void_p(256), nb, stats) == E                # negative step cap
    assert f(ctxs, 2, dp, 0, ctypes.c_void_p(256), nb - 1, stats) == E             # scratch too small
    assert f(ctxs, 2, dp, 0, ctypes.c_void_p(256 + 8), nb, stats) == E             # misaligned scratch
    assert f(ctxs, 2, dp, 0, ctypes.c_void_p(256), nb, stats) == E                 # NULL contexts


def test_a_missing_library_fails_loudly(tmp_path, monkeypatch):
    """No CPU fallback: without the built CUDA library the binding raises, from
    the loader and from any entry point."""
    missing = str(tmp_path / "libgbees_gb300.so")
    monkeypatch.setattr(gbees, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        gbees.load_library(missing)
    monkeypatch.setattr(gbees.load_library, "__defaults__", (missing,))
    with pytest.raises(RuntimeError, match="not built"):
        gbees.gbees_batch_workspace_bytes(1)


def test_the_product_never_imports_or_includes_the_oracle():
    """The library and its binding do not route through the oracle: no module
    of the package imports it and no CUDA source includes anything of it."""
    import ast
    import glob

    pkg = os.path.join(ROOT, "paper_2508_13986_gb300")
    for path in glob.glob(os.path.join(pkg, "*.py")):
        tree = ast.parse(open(path).read())
        for node in ast.walk(tree):
            if isinstance(node, ast.Import):
                assert all(not a.name.startswith("oracle") for a in node.names), path
            elif isinstance(node, ast.ImportFrom):
                assert not (node.module or "").startswith("oracle"), path
    for path in glob.glob(os.path.join(pkg, "csrc", "*")):
        for line in open(path):
            if line.lstrip().startswith("#include"):
                assert "oracle" not in line, (path, line)


C_CALLER = r"""
#include <stdio.h>
#include "gbees.h"
int main(void) {
    gbees_config c = {0};
    c.n = 3; c.dynamics = GBEES_DYN_LORENZ63;
    c.params[0] = 10; c.params[1] = 28; c.params[2] = 8.0 / 3.0;
    for (int j = 0; j < 3; ++j) c.h[j] = 0.5;
    c.thr_rel = 1e-7; c.cfl = 0.9; c.prune_interval = 20; c.max_cells = 1000;
    size_t b = gbees_workspace_bytes(&c);
    gbees_ctx* ctx = 0;
    int rc = gbees_create(&c, 0, b, 0, &ctx);   /* no workspace: refused before any CUDA call */
    printf("%zu %d %d\n", b, rc, gbees_get_status(0));
    return !(b > 0 && rc == GBEES_EINVAL && ctx == 0 && gbees_get_status(0) == GBEES_EINVAL);
}
"""


def test_the_header_is_c99_and_a_c_program_links_the_library(lib, tmp_path):
    """The boundary is a C ABI: gbees.h compiles as strict C99 and a plain C
    caller links the library and makes host-only calls."""
    inc = os.path.join(ROOT, "include")
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only", "-x", "c",
                    os.path.join(inc, "gbees.h")], check=True)
    src = tmp_path / "caller.c"
    src.write_text(C_CALLER)
    exe = tmp_path / "caller"
    libdir = os.path.dirname(LIB)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", inc, str(src), "-L", libdir, "-lgbees_gb300",
                    f"-Wl,-rpath,{libdir}", "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr


def test_binding_structs_match_the_c_layout(tmp_path):
    """sizeof and offsetof of every field of gbees_config, gbees_stats and
    gbees_profile, from a C compile of gbees.h, equal the ctypes layouts of
    the binding."""
    structs = {"gbees_config": gbees.gbees_config, "gbees_stats": gbees.gbees_stats,
               "gbees_profile": gbees.gbees_profile}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "gbees.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'    printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'    printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    c_layout = {tuple(ln.split()[:2]): int(ln.split()[2]) for ln in out if ln.strip()}
    for name, cls in structs.items():
        assert c_layout[(name, "size")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert c_layout[(name, field)] == getattr(cls, field).offset, (name, field)
