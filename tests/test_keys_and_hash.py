"""The CUDA path's cell keys, table hash and Morton code (csrc/gbees_keys.cuh),
built for the host: the packing round trip and its range, key order =
lexicographic order of the index vectors, the Morton code as a bijection that
traces the Z curve and keeps face neighbours closer than key order (the order
the prune's sort gives the pool), the hash as a bijection of u64, and the
probe lengths of linear probing with this hash on the workloads' cell sets
against Knuth's expected values for a random hash (Sec. 4.2 sizes the table
for load factor 1/2)."""
import ctypes
import itertools
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
U64 = np.uint64


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("keys") / "libkeys_host.so")
    src = os.path.join(ROOT, "tests", "keys_host.cpp")
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", src, "-o", out], check=True)
    L = ctypes.CDLL(out)
    L.keys_pack.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                            ctypes.c_void_p]
    L.keys_unpack.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
    L.keys_mix.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
    L.keys_morton.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    L.keys_row_morton.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    L.probe_lengths.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int,
                                ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    L.probe_lengths.restype = ctypes.c_longlong
    return L


def key_bits(n):
    """Bits per component: 63 // n (32 for n = 1), as the library documents."""
    return 32 if n == 1 else 63 // n


def pack(lib, idx, b=None):
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    n = idx.shape[1]
    keys = np.zeros(idx.shape[0], dtype=U64)
    ok = np.zeros(idx.shape[0], dtype=np.uint8)
    assert lib.keys_pack(n, b or key_bits(n), idx.ctypes.data, idx.shape[0], keys.ctypes.data, ok.ctypes.data) == 0
    return keys, ok.astype(bool)


def unpack(lib, keys, n):
    keys = np.ascontiguousarray(keys, dtype=U64)
    idx = np.zeros((keys.shape[0], n), dtype=np.int32)
    assert lib.keys_unpack(n, key_bits(n), keys.ctypes.data, keys.shape[0], idx.ctypes.data) == 0
    return idx


def mix(lib, x):
    x = np.ascontiguousarray(x, dtype=U64)
    out = np.zeros_like(x)
    lib.keys_mix(x.ctypes.data, x.shape[0], out.ctypes.data)
    return out


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_pack_round_trip_and_range(lib, n):
    b = key_bits(n)
    lo, hi = -(1 << (b - 1)), (1 << (b - 1)) - 1
    rng = np.random.default_rng(60 + n)
    idx = rng.integers(lo, hi + 1, size=(5000, n), dtype=np.int64)
    idx[0], idx[1] = lo, hi                       # the extremes of the range
    keys, ok = pack(lib, idx)
    assert ok.all()
    assert np.array_equal(unpack(lib, keys, n), idx)
    assert keys.max() < (1 << (b * n))            # the key uses b bits per component
    if n > 1:                                     # one component out of range: no key
        for j, v in itertools.product(range(n), (lo - 1, hi + 1)):
            bad = idx[:3].copy()
            bad[:, j] = v
            assert not pack(lib, bad)[1].any()


@pytest.mark.parametrize("n", [2, 3, 6])
def test_key_order_is_lexicographic_order(lib, n):
    rng = np.random.default_rng(70 + n)
    b = key_bits(n)
    idx = rng.integers(-(1 << (b - 1)), 1 << (b - 1), size=(4000, n), dtype=np.int64)
    idx[:2000] = rng.integers(-3, 4, size=(2000, n))   # many shared leading components
    keys, ok = pack(lib, idx)
    assert ok.all()
    by_key = np.argsort(keys, kind="stable")
    lex = np.lexsort(idx.T[::-1])                 # dimension 0 most significant
    assert np.array_equal(idx[by_key], idx[lex])


def morton(lib, keys, n, b):
    keys = np.ascontiguousarray(keys, dtype=U64)
    out = np.zeros_like(keys)
    lib.keys_morton(keys.ctypes.data, keys.shape[0], n, b, out.ctypes.data)
    return out


def test_morton_order_of_a_4x4_grid_is_the_z_curve(lib):
    """Worked example: the 16 cells of a 4 x 4 grid (2 bits per field,
    dimension 0 the major bit) in code order trace the Z curve quadrant by
    quadrant."""
    cells = [(x, y) for x in range(4) for y in range(4)]
    keys = np.array([(x << 2) | y for x, y in cells], dtype=U64)
    codes = morton(lib, keys, 2, 2)
    got = [cells[i] for i in np.argsort(codes)]
    assert got == [(0, 0), (0, 1), (1, 0), (1, 1), (0, 2), (0, 3), (1, 2), (1, 3),
                   (2, 0), (2, 1), (3, 0), (3, 1), (2, 2), (2, 3), (3, 2), (3, 3)]


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_morton_code_is_a_bijection_of_the_keys(lib, n):
    """Distinct keys get distinct codes within n*b bits; all-ones maps to
    all-ones (the prune's sort relies on codes below 2^63 for live entries,
    and only an all-ones key reaches the top)."""
    b = key_bits(n)
    rng = np.random.default_rng(90 + n)
    keys = np.unique(rng.integers(0, 1 << (n * b), size=20000, dtype=np.uint64, endpoint=False))
    codes = morton(lib, keys, n, b)
    assert np.unique(codes).size == keys.size
    assert int(codes.max()) < (1 << (n * b))
    ones = np.array([(1 << (n * b)) - 1, 0], dtype=U64)
    assert [int(c) for c in morton(lib, ones, n, b)] == [(1 << (n * b)) - 1, 0]
    if n == 1:
        assert np.array_equal(codes, keys)                      # one field: the key itself


def row_morton(lib, keys, n, b):
    keys = np.ascontiguousarray(keys, dtype=U64)
    out = np.zeros_like(keys)
    lib.keys_row_morton(keys.ctypes.data, keys.shape[0], n, b, out.ctypes.data)
    return out


@pytest.mark.parametrize("n", [1, 2, 3, 6])
def test_row_morton_code_keeps_rows_whole_and_orders_them_on_the_z_curve(lib, n):
    """A bijection of the keys within n*b bits; cells that differ only in the
    last index are consecutive in code order exactly as in key order; the rows
    (the other n - 1 indices) are in Morton order."""
    b = key_bits(n)
    rng = np.random.default_rng(190 + n)
    keys = np.unique(rng.integers(0, 1 << (n * b), size=20000, dtype=np.uint64, endpoint=False))
    codes = row_morton(lib, keys, n, b)
    assert np.unique(codes).size == keys.size and int(codes.max()) < (1 << (n * b))
    if n == 1:
        assert np.array_equal(codes, keys)
        return
    mask = np.uint64((1 << b) - 1)
    assert np.array_equal(codes & mask, keys & mask)                 # the last field is kept
    rows = keys >> np.uint64(b)
    assert np.array_equal(codes >> np.uint64(b), morton(lib, rows, n - 1, b))  # rows on the Z curve
    # a run of one row: consecutive last indices stay consecutive
    base = int(keys[0]) & ~int(mask)
    run = np.array([base | i for i in range(5, 12)], dtype=U64)
    assert np.all(np.diff(row_morton(lib, run, n, b).astype(np.int64)) == 1)


def test_morton_order_keeps_face_neighbours_closer_than_key_order(lib):
    """On the 6-D initial set with its halo, the median distance in sort order
    from a cell to its face neighbours is smaller in code order."""
    idx = ellipsoid_cells(6, 1.0, 1e-6)
    pool = np.concatenate([idx, face_halo(idx)])
    keys, ok = pack(lib, pool)
    assert ok.all()
    med = {}
    for name, sort_key in (("key", keys), ("morton", morton(lib, keys, 6, key_bits(6)))):
        rank = np.empty(keys.size, dtype=np.int64)
        rank[np.argsort(sort_key, kind="stable")] = np.arange(keys.size)
        by_key = dict(zip(keys.tolist(), rank.tolist()))
        d = []
        for j in range(6):
            for s_ in (-1, 1):
                nb = idx.copy()
                nb[:, j] += s_
                nk, _ = pack(lib, nb)
                d.extend(abs(by_key[k] - by_key[c]) for k, c in zip(nk.tolist(), keys[: idx.shape[0]].tolist()))
        med[name] = float(np.median(d))
    assert med["morton"] < 0.5 * med["key"], med


def unmix(y):
    """The inverse of the murmur3 64-bit finaliser: x ^= x >> 33 is its own
    inverse for a shift of more than 32, and an odd multiplier has an inverse
    modulo 2^64."""
    M = (1 << 64) - 1
    y ^= y >> 33
    y = (y * pow(0xc4ceb9fe1a85ec53, -1, 1 << 64)) & M
    y ^= y >> 33
    y = (y * pow(0xff51afd7ed558ccd, -1, 1 << 64)) & M
    y ^= y >> 33
    return y


def test_hash_is_a_bijection(lib):
    rng = np.random.default_rng(80)
    x = np.concatenate([np.array([0, 1, 2, (1 << 64) - 1], dtype=U64),
                        rng.integers(0, 1 << 63, size=2000, dtype=np.int64).astype(U64) * U64(2) + U64(1)])
    y = mix(lib, x)
    assert [unmix(int(v)) for v in y] == [int(v) for v in x]
    assert int(y[0]) == 0                          # the finaliser fixes 0


def ellipsoid_cells(n, sigma_over_h, thr):
    """Cells i (centres i h, origin at the mean) with p > thr max p for an
    isotropic Gaussian of standard deviation sigma_over_h cells: the initial
    sets of the workloads."""
    r = sigma_over_h * np.sqrt(-2.0 * np.log(thr))
    R = int(np.ceil(r))
    axis = np.arange(-R, R + 1)
    grid = np.stack(np.meshgrid(*([axis] * n), indexing="ij"), axis=-1).reshape(-1, n)
    return grid[(grid.astype(np.float64) ** 2).sum(axis=1) < r * r].astype(np.int32)


def face_halo(idx):
    """Face neighbours of a cell set that are not in it."""
    n = idx.shape[1]
    have = {tuple(c) for c in idx.tolist()}
    out = set()
    for j in range(n):
        for s in (-1, 1):
            nb = idx.copy()
            nb[:, j] += s
            out.update(t for t in map(tuple, nb.tolist()) if t not in have)
    return np.array(sorted(out), dtype=np.int32)


def probe(lib, keys, absent, log2_slots):
    keys = np.ascontiguousarray(keys, dtype=U64)
    absent = np.ascontiguousarray(absent, dtype=U64)
    hit, miss = ctypes.c_double(), ctypes.c_double()
    d = lib.probe_lengths(keys.ctypes.data, keys.shape[0], absent.ctypes.data, absent.shape[0], log2_slots,
                          ctypes.byref(hit), ctypes.byref(miss))
    return d, hit.value, miss.value


@pytest.mark.parametrize("name,n,sigma_over_h,thr", [
    ("lorenz63 h0.25 initial set", 3, 4.0, 1e-7),     # sigma 1, h 0.25
    ("lorenz96 6-D h0.5 initial set", 6, 1.0, 1e-6),  # sigma 0.5, h 0.5
])
@pytest.mark.parametrize("alpha", [0.5, 0.25])
def test_linear_probing_lengths_match_a_random_hash(lib, name, n, sigma_over_h, thr, alpha):
    """Knuth's expected probes of linear probing at load factor alpha with a
    random hash: (1 + 1/(1-alpha))/2 for a hit, (1 + 1/(1-alpha)^2)/2 for a
    miss (1.5 and 2.5 at alpha = 1/2). The structured keys of a Gaussian's
    cell set (contiguous in every dimension) must not cluster more."""
    idx = ellipsoid_cells(n, sigma_over_h, thr)
    pool = np.concatenate([idx, face_halo(idx)])            # active cells and their halo
    keys, ok = pack(lib, pool)
    assert ok.all()
    keys = np.sort(keys)
    log2 = int(np.floor(np.log2(keys.shape[0] / alpha)))
    m = int(alpha * (1 << log2))
    inserted, absent = keys[:m], keys[m:]                   # a contiguous slab in, the rest out
    d, hit, miss = probe(lib, inserted, absent, log2)
    assert d == m and absent.shape[0] > 1000
    want_hit = 0.5 * (1.0 + 1.0 / (1.0 - alpha))
    want_miss = 0.5 * (1.0 + 1.0 / (1.0 - alpha) ** 2)
    assert abs(hit - want_hit) < 0.04 * want_hit, (name, hit, want_hit)
    assert abs(miss - want_miss) < 0.08 * want_miss, (name, miss, want_miss)


def test_a_clustering_hash_fails_the_probe_check(lib):
    """The check has teeth: the identity hash on the same keys (slot = key &
    mask, i.e. the low component alone) clusters badly."""
    idx = ellipsoid_cells(3, 4.0, 1e-7)
    keys = np.sort(pack(lib, idx)[0])
    log2 = int(np.floor(np.log2(keys.shape[0] / 0.5)))
    m = 1 << (log2 - 1)
    # place by the identity hash: pre-image of the key under mix64, so that the
    # table's slot is key & mask
    pre = np.array([unmix(int(k)) for k in keys[:m]], dtype=U64)
    d, hit, _ = probe(lib, pre, keys[m:m + 1000], log2)
    assert d == m and hit > 3.0
