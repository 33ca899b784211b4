"""Pins of the CPU oracle against facts the paper and the mathematics fix.

Each test ties one part of the oracle (oracle/gbees_oracle.cpp) to something
other than itself: a worked example printed in the paper, a closed form, an
invariant, a textbook special case, a library routine or a brute force on tiny
inputs. Together they are chosen so that a dropped term, a wrong sign, a wrong
index or a transposed operand anywhere in the oracle fails at least one.
"""
import itertools
import math
import os

import numpy as np
import pytest
import scipy.linalg

from oracle.oracle import (DYN_CONSTANT, DYN_LINEAR, DYN_LORENZ63, DYN_LORENZ63_SHIFTED, DYN_LORENZ96,
                           LIM_LW, LIM_MC, LIM_NONE, Oracle, OracleError, exact_sum)
from paper_2508_13986_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def const_oracle(c, h, limiter=LIM_MC, thr=1e-7, cfl=0.9, K=20, x0=None):
    n = len(c)
    return Oracle(n, DYN_CONSTANT, list(c), h, x0 if x0 is not None else [0.0] * n, thr, cfl, K, limiter)


def cells_of(o):
    idx, p = o.read_cells()
    return {tuple(int(v) for v in r): float(q) for r, q in zip(idx, p)}


def box_cells(shape, lo):
    grids = np.meshgrid(*[np.arange(l, l + s) for l, s in zip(lo, shape)], indexing="ij")
    return np.stack([g.reshape(-1) for g in grids], axis=1).astype(np.int32)


# ---------------------------------------------------------------- exact sum

def test_exact_sum_equals_fsum():
    """The order-free normaliser sum against math.fsum (a correctly rounded exact sum)."""
    rng = np.random.default_rng(1)
    cases = [
        rng.random(1000),
        rng.standard_normal(5000) * 10.0 ** rng.integers(-30, 30, 5000),
        np.array([1e300, 1.0, -1e300, 1e-300, 5e-324, -5e-324, 2.0 ** -1074 * 3]),
        np.array([1.0, 2.0 ** -53, 2.0 ** -53]),                      # ties to even
        np.array([1.0, 2.0 ** -53, 2.0 ** -106]),                     # sticky bit
        np.array([0.1] * 10 + [-0.3] * 3),
        np.array([]),
        -rng.random(777) * 1e-5,
    ]
    for x in cases:
        assert exact_sum(x) == math.fsum(x.tolist())
    # order independence
    x = rng.standard_normal(4096) * 10.0 ** rng.integers(-8, 8, 4096)
    assert exact_sum(x) == exact_sum(x[::-1]) == exact_sum(rng.permutation(x))


# ---------------------------------------------------------------- dynamics

def test_lorenz63_classic_equilibria_and_divergence():
    s, r, b = W.L63_PARAMS
    o = Oracle(3, DYN_LORENZ63, [s, r, b], [1, 1, 1], [0, 0, 0])
    q = math.sqrt(b * (r - 1))
    for x in ([0, 0, 0], [q, q, r - 1], [-q, -q, r - 1]):
        for j in range(3):
            assert abs(o.drift(x, j)) < 1e-12
    # constant divergence -(sigma + 1 + beta), central differences on a quadratic field
    rng = np.random.default_rng(2)
    for _ in range(10):
        x = rng.standard_normal(3) * 10
        div = 0.0
        for j in range(3):
            e = np.zeros(3)
            e[j] = 0.5
            div += (o.drift(x + e, j) - o.drift(x - e, j)) / 1.0
        assert abs(div + (s + 1 + b)) < 1e-9


def test_lorenz63_shifted_form_is_classic_form_shifted_in_z():
    """Sec. 5.1.1 prints the model as (s(x2-x1), -x2-x1x3, -b x3 + x1x2 - b r): the classic
    form with x3 -> x3 + r."""
    s, r, b = W.L63_PARAMS
    classic = Oracle(3, DYN_LORENZ63, [s, r, b], [1, 1, 1], [0, 0, 0])
    shifted = Oracle(3, DYN_LORENZ63_SHIFTED, [s, b, r], [1, 1, 1], [0, 0, 0])
    rng = np.random.default_rng(3)
    for _ in range(20):
        x = rng.standard_normal(3) * 15
        for j in range(3):
            a = classic.drift(x + np.array([0, 0, r]), j)
            c = shifted.drift(x, j)
            assert abs(a - c) <= 1e-12 * max(1.0, abs(a))


@pytest.mark.parametrize("n", [4, 5, 6])
def test_lorenz96_equilibrium_and_energy_identity(n):
    """(F,...,F) is an equilibrium (Sec. 5.1.2); the quadratic term conserves energy, so
    sum_j x_j f_j(x) = -|x|^2 + F sum_j x_j for the cyclic model."""
    F = 4.0
    o = Oracle(n, DYN_LORENZ96, [F], [1] * n, [0] * n)
    for j in range(n):
        assert abs(o.drift([F] * n, j)) < 1e-12
    rng = np.random.default_rng(4)
    for _ in range(20):
        x = rng.standard_normal(n) * 5
        lhs = sum(x[j] * o.drift(x, j) for j in range(n))
        rhs = -float(x @ x) + F * float(x.sum())
        assert abs(lhs - rhs) < 1e-10 * max(1.0, abs(rhs))


def test_linear_drift_against_matrix_product():
    rng = np.random.default_rng(5)
    n = 4
    A = rng.standard_normal((n, n))
    b = rng.standard_normal(n)
    o = Oracle(n, DYN_LINEAR, list(A.reshape(-1)) + list(b), [1] * n, [0] * n)
    for _ in range(10):
        x = rng.standard_normal(n)
        ref = A @ x + b
        for j in range(n):
            assert abs(o.drift(x, j) - ref[j]) < 1e-12


def test_face_velocity_is_taken_at_the_lower_face_centre():
    """With f(x) = x, the velocity of Eq. 7 at cell X in dimension j reads back the
    position of the lower face centre, x0_j + (X_j - 1/2) h_j."""
    n = 3
    o = Oracle(n, DYN_LINEAR, list(np.eye(n).reshape(-1)) + [0] * n, [0.5, 0.25, 2.0], [1.0, -3.0, 7.0])
    for X in ([0, 0, 0], [3, -2, 5], [-7, 1, 0]):
        for j in range(n):
            want = [1.0, -3.0, 7.0][j] + (X[j] - 0.5) * [0.5, 0.25, 2.0][j]
            assert o.face_velocity(X, j) == pytest.approx(want, abs=1e-15)


# ---------------------------------------------------------------- grow / prune direction sets

def test_grow_worked_example_fig2():
    want = {tuple(int(v) for v in r) for r in read_golden("fig2_grow_2d.txt")}
    o = const_oracle([1.0, 1.0], [1.0, 1.0])
    assert set(o.downwind([0, 0])) == want


def test_prune_worked_example_fig3():
    """A sub-threshold cell (0,0) survives prune exactly when one of the upwind cells of
    Fig. 3 is above threshold."""
    checked = [tuple(int(v) for v in r) for r in read_golden("fig3_prune_2d.txt")]
    candidates = checked + [(1, 0), (0, 1), (1, 1), (-1, 1), (1, -1)]
    for nb in candidates:
        o = const_oracle([1.0, 1.0], [1.0, 1.0], thr=1e-3)
        idx = np.array([[20, 20], [0, 0], list(nb)], dtype=np.int32)
        p = np.array([1.0, 1e-6, 0.5])
        o.init_cells(idx, p)
        o.prune()
        kept = cells_of(o)
        assert ((0, 0) in kept) == (nb in checked), nb


def test_downwind_sets_for_divergent_convergent_and_3d_flows():
    # divergent f = x: every face points outwards -> all 3^2-1 neighbours
    o = Oracle(2, DYN_LINEAR, [1, 0, 0, 1, 0, 0], [1, 1], [0, 0])
    assert len(set(o.downwind([0, 0]))) == 8
    # convergent f = -x: no face points outwards
    o = Oracle(2, DYN_LINEAR, [-1, 0, 0, -1, 0, 0], [1, 1], [0, 0])
    assert o.downwind([0, 0]) == []
    # 3-D oblique flow: 3 faces + 3 pairwise edges, no (1,1,1) corner
    o = const_oracle([1.0, -2.0, 0.5], [1, 1, 1])
    d = set(o.downwind([0, 0, 0]))
    assert d == {(1, 0, 0), (0, -1, 0), (0, 0, 1), (1, -1, 0), (1, 0, 1), (0, -1, 1)}
    # zero velocity in one dimension grows nothing along it
    o = const_oracle([1.0, 0.0], [1, 1])
    assert set(o.downwind([0, 0])) == {(1, 0)}
    # 6-D: the faces of the dimensions with a velocity and every pair of them
    c = [1.0, -1.0, 0.5, 0.0, 2.0, -0.25]
    o = const_oracle(c, [1] * 6)
    moving = [(j, 1 if v > 0 else -1) for j, v in enumerate(c) if v != 0.0]
    want = set()
    for j, s_ in moving:
        want.add(tuple(s_ if k == j else 0 for k in range(6)))
    for (j, sj), (l, sl) in itertools.combinations(moving, 2):
        want.add(tuple(sj if k == j else sl if k == l else 0 for k in range(6)))
    d = o.downwind([3, -2, 0, 5, 1, -7])
    assert len(d) == len(set(d)) == 5 + 10
    assert {tuple(x - y for x, y in zip(X, (3, -2, 0, 5, 1, -7))) for X in d} == want


def test_grow_then_prune_leaves_exactly_S_and_its_downwind_set():
    """After grow, prune on the same values keeps S u D(S) (computed here from the
    downwind sets of the significant cells) and a second grow adds nothing."""
    w = W.config("lorenz63_h0.5")
    o = Oracle(w.n, w.dynamics, w.params, w.h, w.x0, w.thr_rel, w.cfl, 3, w.limiter)
    o.init_gaussian(w.mean, w.cov)
    o.propagate(0.01)
    o.grow()
    o.prune()
    cells = cells_of(o)
    pstar = w.thr_rel * max(cells.values())
    want = set()
    for X, v in cells.items():
        if v > pstar:
            want.add(X)
            want.update(o.downwind(list(X)))
    assert set(cells) == want
    o.grow()
    assert o.count() == len(want)


# ---------------------------------------------------------------- CFL time step

def test_cfl_dt_constant_velocity():
    c, h = [3.0, -1.5, 0.25], [0.5, 0.25, 1.0]
    o = const_oracle(c, h, cfl=0.7)
    o.init_cells(np.zeros((1, 3), dtype=np.int32), np.ones(1))
    want = 0.7 / sum(abs(ci) / hi for ci, hi in zip(c, h))
    assert o.cfl_dt() == pytest.approx(want, rel=1e-15)
    st = o.propagate(10 * want + 1e-3)
    assert st.steps == 11 and st.t == 10 * want + 1e-3


# ---------------------------------------------------------------- CTU closed forms

def zero_padded_shift(A, offs):
    """B[X] = A[X - offs] with zero fill."""
    B = np.zeros_like(A)
    src, dst = [], []
    for d, o in enumerate(offs):
        if o >= 0:
            src.append(slice(0, A.shape[d] - o))
            dst.append(slice(o, A.shape[d]))
        else:
            src.append(slice(-o, A.shape[d]))
            dst.append(slice(0, A.shape[d] + o))
    B[tuple(dst)] = A[tuple(src)]
    return B


@pytest.mark.parametrize("sx,sy", [(1, 1), (1, -1), (-1, 1), (-1, -1)])
def test_ctu_constant_velocity_2d_is_bilinear_interpolation(sx, sy):
    """For constant velocity the donor-cell + corner-transport scheme moves each cell's
    content to the foot of the characteristic and interpolates bilinearly (Colella 1990;
    LeVeque, Ch. 20): Pn = (1-nx)(1-ny)P + nx(1-ny)P[-x] + (1-nx)ny P[-y] + nx ny P[-x-y]."""
    h = [0.5, 0.25]
    a, b = 3.0 * sx, 1.25 * sy
    dt = 0.1
    nx, ny = abs(a) * dt / h[0], abs(b) * dt / h[1]
    assert nx < 1 and ny < 1
    rng = np.random.default_rng(6)
    shape = (9, 11)
    P = rng.random(shape)
    idx = box_cells(shape, (-4, -5))
    o = const_oracle([a, b], h, limiter=LIM_NONE)
    o.init_cells(idx, P.reshape(-1))
    o.ctu_step(dt)
    got = cells_of(o)
    pad = np.zeros((shape[0] + 2, shape[1] + 2))
    pad[1:-1, 1:-1] = P
    sh = lambda ox, oy: zero_padded_shift(pad, (ox, oy))[1:-1, 1:-1]
    want = ((1 - nx) * (1 - ny) * P + nx * (1 - ny) * sh(sx, 0) + (1 - nx) * ny * sh(0, sy)
            + nx * ny * sh(sx, sy))
    for k, X in enumerate(idx):
        i, j = X[0] + 4, X[1] + 5
        assert got[tuple(X)] == pytest.approx(want[i, j], abs=1e-14)


def mc_phi(theta):
    return np.maximum(0.0, np.minimum(np.minimum((1.0 + theta) / 2.0, 2.0), 2.0 * theta))


def hr_ctu_positive(P, nx, ny, phi):
    """LeVeque's high-resolution wave-propagation step (Ch. 20) for constant
    velocity with both components positive, written as bilinear CTU plus the
    limited second-order flux differences of each axis (increment waves
    propagated transversely, corrections not), on a zero-padded array (two
    cells of padding on each side)."""
    def sh(A, ox, oy):                      # A shifted so that out[i, j] = A[i - ox, j - oy]
        return np.roll(np.roll(A, ox, 0), oy, 1)
    new = ((1 - nx) * (1 - ny) * P + nx * (1 - ny) * sh(P, 1, 0) + (1 - nx) * ny * sh(P, 0, 1)
           + nx * ny * sh(P, 1, 1))
    for axis, nu in ((0, nx), (1, ny)):
        W = P - np.roll(P, 1, axis)                  # wave at the lower face
        Wup = np.roll(W, 1, axis)                    # the wave one face upwind
        theta = np.divide(Wup, W, out=np.zeros_like(W), where=W != 0)
        F = 0.5 * nu * (1 - nu) * phi(theta) * W     # dt/h times the correction flux
        new -= np.roll(F, -1, axis) - F
    return new


@pytest.mark.parametrize("sx,sy", [(1, 1), (1, -1), (-1, 1), (-1, -1)])
def test_ctu_mc_constant_velocity_2d_is_the_textbook_high_resolution_step(sx, sy):
    """With the MC limiter a constant-velocity step is bilinear CTU plus the
    MC-limited flux correction along each axis (LeVeque, Ch. 20), in all four
    velocity quadrants; the data mix smooth and rough parts so that every
    branch of the limiter is taken."""
    h = [0.5, 0.25]
    a, b = 3.0 * sx, 1.25 * sy
    dt = 0.1
    nx, ny = abs(a) * dt / h[0], abs(b) * dt / h[1]
    rng = np.random.default_rng(61)
    shape = (12, 14)
    X, Y = np.meshgrid(np.arange(shape[0]), np.arange(shape[1]), indexing="ij")
    P = np.exp(-0.5 * ((X - 6.0) ** 2 / 4.0 + (Y - 7.0) ** 2 / 6.0)) + 0.2 * rng.random(shape)
    idx = box_cells(shape, (-6, -7))
    o = const_oracle([a, b], h, limiter=LIM_MC)
    o.init_cells(idx, P.reshape(-1))
    o.ctu_step(dt)
    got = cells_of(o)
    pad = np.zeros((shape[0] + 4, shape[1] + 4))
    pad[2:-2, 2:-2] = P
    flip = (slice(None, None, sx), slice(None, None, sy))   # reflect negative components to positive
    want = hr_ctu_positive(pad[flip], nx, ny, mc_phi)[flip][2:-2, 2:-2]
    err = max(abs(got[tuple(Xc)] - want[Xc[0] + 6, Xc[1] + 7]) for Xc in idx)
    assert err <= 1e-14


@pytest.mark.parametrize("c", [2.0, -2.0])
def test_ctu_lw_limiter_is_lax_wendroff_1d(c):
    """phi = 1 turns the high-resolution flux into Lax-Wendroff:
    Pn = P - nu/2 (P[+1]-P[-1]) + nu^2/2 (P[+1] - 2P + P[-1])."""
    h, dt = 0.5, 0.15
    nu = c * dt / h
    rng = np.random.default_rng(7)
    P = rng.random(30)
    o = const_oracle([c], [h], limiter=LIM_LW)
    o.init_cells(np.arange(30, dtype=np.int32)[:, None], P)
    o.ctu_step(dt)
    got = np.array([v for _, v in sorted(cells_of(o).items())])
    Pp = np.concatenate([[0.0], P, [0.0]])
    want = P - nu / 2 * (Pp[2:] - Pp[:-2]) + nu ** 2 / 2 * (Pp[2:] - 2 * P + Pp[:-2])
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-14)


def fromm_positive(P, nu):
    """Fromm's scheme for nu > 0 (mean of Lax-Wendroff and Beam-Warming)."""
    Pp = np.concatenate([[0.0, 0.0], P, [0.0]])
    Pm2, Pm1, P0, Pp1 = Pp[:-3], Pp[1:-2], Pp[2:-1], Pp[3:]
    return P0 - nu / 4 * (Pp1 + 3 * P0 - 5 * Pm1 + Pm2) + nu ** 2 / 4 * (Pp1 - P0 - Pm1 + Pm2)


@pytest.mark.parametrize("c", [1.7, -1.7])
def test_ctu_mc_limiter_on_smooth_data_is_fromm(c):
    """Where 1/3 <= theta <= 3 the MC limiter equals (1+theta)/2, i.e. Fromm's scheme."""
    h, dt = 0.5, 0.2
    nu = c * dt / h
    r = 1.5
    P = r ** np.arange(24, dtype=np.float64) * 1e-6
    o = const_oracle([c], [h], limiter=LIM_MC)
    o.init_cells(np.arange(24, dtype=np.int32)[:, None], P)
    o.ctu_step(dt)
    got = np.array([v for _, v in sorted(cells_of(o).items())])
    want = fromm_positive(P, nu) if nu > 0 else fromm_positive(P[::-1], -nu)[::-1]
    inner = slice(3, -3)
    np.testing.assert_allclose(got[inner], want[inner], rtol=1e-13)


def test_upwind_first_order_moments_1d():
    """Limiter NONE is donor-cell upwind: the mean moves by c dt and the variance grows
    by nu (1 - nu) h^2 per step (binomial spreading)."""
    h, c, dt = 0.25, 1.0, 0.15
    nu = c * dt / h
    x = np.arange(-60, 61)
    P = np.exp(-0.5 * (x * h / 1.0) ** 2)
    o = const_oracle([c], [h], limiter=LIM_NONE)
    o.init_cells(x.astype(np.int32)[:, None], P)
    def moments():
        d = cells_of(o)
        xs = np.array([k[0] * h for k in d])
        ps = np.array(list(d.values()))
        m0 = ps.sum()
        m1 = (xs * ps).sum() / m0
        return m0, m1, ((xs - m1) ** 2 * ps).sum() / m0
    m0a, m1a, va = moments()
    o.ctu_step(dt)
    m0b, m1b, vb = moments()
    assert m0b == pytest.approx(m0a, rel=1e-13)
    assert m1b - m1a == pytest.approx(c * dt, rel=1e-11)
    assert vb - va == pytest.approx(nu * (1 - nu) * h * h, rel=1e-9)


@pytest.mark.parametrize("lim", [LIM_NONE, LIM_LW])
def test_first_moment_moves_with_constant_velocity_3d(lim):
    """Constant velocity, linear limiter: the fluxes telescope, so the discrete mean moves
    by exactly c dt in every dimension (transverse and correction terms sum to zero)."""
    h = [0.5, 0.5, 0.5]
    c = [1.2, -0.7, 0.4]
    dt = 0.9 / sum(abs(ci) / hi for ci, hi in zip(c, h))
    idx, P = W.gaussian_blob_cells(3, 12, 1.5)
    o = const_oracle(c, h, limiter=lim)
    o.init_cells(idx, P)
    def mean():
        d = cells_of(o)
        X = np.array(list(d.keys()), dtype=np.float64) * 0.5
        p = np.array(list(d.values()))
        return (X * p[:, None]).sum(0) / p.sum(), p.sum()
    ma, sa = mean()
    o.ctu_step(dt)
    mb, sb = mean()
    assert sb == pytest.approx(sa, rel=1e-12)
    np.testing.assert_allclose(mb - ma, np.array(c) * dt, rtol=1e-9, atol=1e-12)


def test_mc_limiter_is_total_variation_diminishing_1d():
    rng = np.random.default_rng(8)
    for trial in range(20):
        c = rng.choice([-1.0, 1.0]) * rng.uniform(0.5, 2.0)
        h = 0.5
        dt = rng.uniform(0.1, 1.0) * h / abs(c)
        P = rng.random(40) * (rng.random(40) < 0.7)
        P = np.concatenate([[0, 0], P, [0, 0]])
        o = const_oracle([c], [h], limiter=LIM_MC)
        o.init_cells(np.arange(P.size, dtype=np.int32)[:, None], P)
        o.ctu_step(dt)
        got = np.array([v for _, v in sorted(cells_of(o).items())])
        tv = lambda a: np.abs(np.diff(np.concatenate([[0.0], a, [0.0]]))).sum()
        assert tv(got) <= tv(P) + 1e-14
        assert got.min() >= -1e-15 and got.max() <= P.max() + 1e-15


# ---------------------------------------------------------------- brute force: dense box

def dense_ctu(P, U, dt, h, limiter):
    """Eq. 7 + Algorithm 1 + high-resolution correction on a dense zero-padded box:
    every face of the box, every cell updated (the caller keeps the active ones)."""
    n = P.ndim

    def sh(A, j, s):  # B[X] = A[X + s e_j], zero outside
        offs = [0] * n
        offs[j] = -s
        return zero_padded_shift(A, offs)

    F = [np.maximum(U[j], 0) * sh(P, j, -1) + np.minimum(U[j], 0) * P for j in range(n)]
    for j in range(n):
        Fs = dt / (2 * h[j]) * (P - sh(P, j, -1))
        up, um = np.maximum(U[j], 0), np.minimum(U[j], 0)
        for l in range(n):
            if l == j:
                continue
            F[l] = F[l] - sh(up * Fs, l, -1) * np.maximum(U[l], 0)
            F[l] = F[l] - up * Fs * np.minimum(U[l], 0)
            F[l] = F[l] - sh(sh(um * Fs, j, +1), l, -1) * np.maximum(U[l], 0)
            F[l] = F[l] - sh(um * Fs, j, +1) * np.minimum(U[l], 0)
    if limiter != LIM_NONE:
        for j in range(n):
            Wv = P - sh(P, j, -1)
            Wup = np.where(U[j] > 0, sh(P, j, -1) - sh(P, j, -2), sh(P, j, +1) - P)
            with np.errstate(divide="ignore", invalid="ignore"):
                th = np.where(Wv != 0, Wup / np.where(Wv != 0, Wv, 1.0), 0.0)
            if limiter == LIM_LW:
                phi = np.ones_like(th)
            else:
                phi = np.maximum(0, np.minimum(np.minimum((1 + th) / 2, 2.0), 2 * th))
            au = np.abs(U[j])
            F[j] = F[j] + np.where(Wv != 0, 0.5 * au * (1 - dt * au / h[j]) * phi * Wv, 0.0)
    out = P.copy()
    for j in range(n):
        out = out - dt / h[j] * (sh(F[j], j, +1) - F[j])
    return out


@pytest.mark.parametrize("n,lim,seed", [(2, LIM_MC, 0), (2, LIM_LW, 1), (3, LIM_MC, 2), (3, LIM_NONE, 3),
                                        (1, LIM_MC, 4), (4, LIM_MC, 5)])
def test_sparse_step_equals_dense_box_brute_force(n, lim, seed):
    """The sparse scatter step on a random ragged active set equals the same scheme run
    on a dense zero-padded box (P = 0 off the set) and read back at the active cells."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    b = rng.standard_normal(n)
    h = rng.uniform(0.3, 0.8, n)
    x0 = rng.standard_normal(n)
    side = {1: 30, 2: 12, 3: 7, 4: 5}[n]
    pad = 3
    idx = box_cells([side] * n, [0] * n)
    keep = rng.random(idx.shape[0]) < 0.6
    idx = idx[keep]
    pv = rng.random(idx.shape[0])
    o = Oracle(n, DYN_LINEAR, list(A.reshape(-1)) + list(b), h, x0, 1e-7, 0.9, 20, lim)
    o.init_cells(idx, pv)
    dt = 0.8 * o.cfl_dt() / 0.9
    o.ctu_step(dt)
    got = cells_of(o)
    full = side + 2 * pad
    P = np.zeros([full] * n)
    for X, v in zip(idx, pv):
        P[tuple(X + pad)] = v
    grids = np.meshgrid(*[np.arange(full) - pad] * n, indexing="ij")
    U = []
    for j in range(n):
        y = [x0[k] + grids[k] * h[k] for k in range(n)]
        y[j] = x0[j] + (grids[j] - 0.5) * h[j]
        U.append(sum(A[j, k] * y[k] for k in range(n)) + b[j])
    out = dense_ctu(P, U, dt, h, lim)
    scale = np.abs(pv).max()
    for X in idx:
        assert abs(got[tuple(int(v) for v in X)] - out[tuple(X + pad)]) <= 1e-13 * scale


def test_sampled_update_equals_full_update():
    rng = np.random.default_rng(9)
    n = 3
    A = rng.standard_normal((n, n))
    o = Oracle(n, DYN_LINEAR, list(A.reshape(-1)) + [0.3, -0.2, 0.1], [0.5] * 3, [0.1, 0.2, 0.3])
    idx = box_cells([6, 6, 6], [-3, -3, -3])
    idx = idx[rng.random(idx.shape[0]) < 0.7]
    pv = rng.random(idx.shape[0])
    o.init_cells(idx, pv)
    dt = o.cfl_dt()
    sample = o.ctu_sample(dt, idx)
    o.ctu_step(dt)
    got = cells_of(o)
    for X, v in zip(idx, sample):
        assert v == pytest.approx(got[tuple(int(q) for q in X)], abs=1e-15)


# ---------------------------------------------------------------- full loop

def test_translation_at_courant_one_is_an_exact_shift():
    """Constant velocity along one axis with CFL 1 gives Courant number exactly 1: the
    high-resolution factor (1 - nu) and the transverse terms vanish and every step shifts
    the pdf by one cell, through grow, prune and normalisation."""
    h = [0.5, 0.5, 0.5]
    o = Oracle(3, DYN_CONSTANT, [2.0, 0.0, 0.0], h, [0, 0, 0], 1e-7, 1.0, 3, LIM_MC)
    o.init_gaussian([0.0, 0.0, 0.0], np.diag([1.0, 0.8, 1.3]))
    p0 = cells_of(o)
    k = 7
    st = o.propagate(k * 0.25)
    assert st.steps == k
    got = cells_of(o)
    for X, v in p0.items():
        Y = (X[0] + k, X[1], X[2])
        assert got.get(Y, 0.0) == pytest.approx(v, rel=1e-14)
    for Y, v in got.items():
        X = (Y[0] - k, Y[1], Y[2])
        if X not in p0:
            assert v == 0.0


@pytest.mark.parametrize("lim", [LIM_MC, LIM_NONE])
def test_linear_dynamics_moments_converge_to_closed_form(lim):
    """f = A x keeps a Gaussian Gaussian: m(t) = e^{At} m0, S(t) = e^{At} S0 e^{A't}.
    The grid moments approach it as h is refined, at observed order >= 1 (the
    face velocities of a varying drift make the moments first order even
    where the limited scheme is second order)."""
    A = np.array([[-0.5, 1.0], [-1.0, -0.5]])
    m0 = np.array([1.0, 0.5])
    S0 = np.array([[0.09, 0.02], [0.02, 0.06]])
    T = 0.5
    E = scipy.linalg.expm(A * T)
    m_ref, S_ref = E @ m0, E @ S0 @ E.T
    errs = []
    for h in (0.1, 0.05, 0.025):
        o = Oracle(2, DYN_LINEAR, list(A.reshape(-1)) + [0.0, 0.0], [h, h], list(m0), 1e-9, 0.9, 5, lim)
        o.init_gaussian(m0, S0)
        o.propagate(T)
        m, S = o.moments()
        errs.append(np.abs(m - m_ref).max() + np.abs(S - S_ref).max())
    orders = [math.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert min(orders) >= 0.95, orders
    assert errs[2] < (2e-3 if lim == LIM_MC else 1.2e-2)


def test_measurement_update_of_a_gaussian_is_the_kalman_posterior():
    """Gaussian prior, full-state linear Gaussian likelihood (Eq. 4): the posterior
    moments are m + S (S+R)^-1 (y-m) and S - S (S+R)^-1 S."""
    m = np.array([0.3, -0.2, 1.0])
    S = np.array([[1.0, 0.3, 0.1], [0.3, 0.8, -0.2], [0.1, -0.2, 1.2]])
    R = np.array([[0.25, 0.05, 0.0], [0.05, 0.3, 0.0], [0.0, 0.0, 0.4]])
    y = np.array([0.9, -0.5, 0.6])
    o = Oracle(3, DYN_CONSTANT, [0, 0, 0], [0.1] * 3, list(m), 1e-9, 0.9, 20, LIM_MC)
    o.init_gaussian(m, S)
    o.correct_gaussian(y, R, [0, 1, 2])
    mm, SS = o.moments()
    K = S @ np.linalg.inv(S + R)
    np.testing.assert_allclose(mm, m + K @ (y - m), atol=2e-6)
    np.testing.assert_allclose(SS, S - K @ S, atol=2e-6)
    # a partial measurement of component 2 only
    o = Oracle(3, DYN_CONSTANT, [0, 0, 0], [0.1] * 3, list(m), 1e-9, 0.9, 20, LIM_MC)
    o.init_gaussian(m, S)
    o.correct_gaussian([0.2], [[0.5]], [2])
    mm, SS = o.moments()
    H = np.array([[0.0, 0.0, 1.0]])
    K = S @ H.T @ np.linalg.inv(H @ S @ H.T + 0.5)
    np.testing.assert_allclose(mm, m + (K @ (np.array([0.2]) - H @ m)), atol=2e-6)
    np.testing.assert_allclose(SS, S - K @ H @ S, atol=2e-6)


def test_initial_gaussian_set_and_normalisation():
    """The initial set is exactly {cells with p > thr max p} (brute force over a much
    larger box) and (prod h) sum p = 1."""
    m = np.array([0.13, -0.07])
    S = np.array([[0.5, 0.2], [0.2, 0.3]])
    h = [0.2, 0.15]
    thr = 1e-4
    o = Oracle(2, DYN_CONSTANT, [0, 0], h, [0.0, 0.0], thr, 0.9, 20, LIM_MC)
    o.init_gaussian(m, S)
    got = cells_of(o)
    X = box_cells([81, 81], [-40, -40])
    x = X * np.array(h)
    d = x - m
    q = np.einsum("ij,jk,ik->i", d, np.linalg.inv(S), d)
    g = np.exp(-0.5 * q)
    want = {tuple(int(v) for v in r) for r, gv in zip(X, g) if gv > thr * g.max()}
    assert set(got) == want
    assert math.fsum(got.values()) * h[0] * h[1] == pytest.approx(1.0, abs=1e-14)


def test_probability_is_normalised_after_each_propagation():
    w = W.config("lorenz63_h0.5")
    o = Oracle(w.n, w.dynamics, w.params, w.h, w.x0, w.thr_rel, w.cfl, 7, w.limiter)
    o.init_gaussian(w.mean, w.cov)
    for t in (0.005, 0.01, 0.02):
        o.propagate(t)
        _, p = o.read_cells()
        assert math.fsum(p.tolist()) * 0.125 == pytest.approx(1.0, abs=1e-14)
        assert o.t == t



def test_first_order_mass_loss_per_step_is_small_and_never_a_gain():
    """Conservation on Lorenz '63 h = 0.5 with the first-order scheme: fluxes
    between active cells cancel, so a step changes the total only by what
    leaves through the faces of the active set, and prune only removes cells;
    both are losses (the scheme is positive for these Courant numbers) and
    small (the set's edge is below thr_rel of the maximum): under 1e-6 per
    step, 1e-6 per prune. The loop is taken step by step: grow, dt (Eq. 8),
    update, normalise, prune every K steps."""
    w = W.config("lorenz63_h0.5")
    o = Oracle(w.n, w.dynamics, w.params, w.h, w.x0, w.thr_rel, w.cfl, w.prune_interval, LIM_NONE)
    o.init_gaussian(w.mean, w.cov)
    vol = math.prod(w.h)
    mass = lambda: vol * math.fsum(o.read_cells()[1].tolist())
    for k in range(1, 41):
        o.grow()
        before = mass()
        o.ctu_step(o.cfl_dt())
        lost = before - mass()
        assert 0.0 <= lost < 1e-6
        o.normalise()
        if k % 20 == 0:
            o.prune()
            assert 0.0 <= 1.0 - mass() < 1e-6
    assert o.read_cells()[1].min() >= 0.0


@pytest.mark.parametrize("lim", [LIM_MC, LIM_NONE])
def test_zero_drift_takes_one_step_to_the_target_and_keeps_the_density(lim):
    """Degenerate case of Eq. 8: with f = 0 every CFL rate is zero, so one step
    reaches the target (R2); no face carries flux, grow adds no cell, and the
    density is unchanged (to the rounding of the normalisation)."""
    idx, p = W.random_cells(3, 300, 4, seed=64)
    p = p / (0.125 * p.sum())
    o = const_oracle([0.0, 0.0, 0.0], [0.5, 0.5, 0.5], limiter=lim, K=1)
    o.init_cells(idx, p)
    st = o.propagate(0.7)
    assert st.steps == 1 and o.t == 0.7 and st.last_dt == 0.7
    gi, gp = o.read_cells()
    order = np.lexsort(idx.T[::-1])
    assert np.array_equal(gi, idx[order])
    np.testing.assert_allclose(gp, p[order], rtol=1e-15, atol=0)


def test_a_measurement_with_no_weight_is_degenerate():
    """C = 0 in Eq. 4 (the likelihood underflows at every cell) is an error, not
    a division by zero."""
    w = W.config("lorenz63_h0.5")
    o = Oracle(w.n, w.dynamics, w.params, w.h, w.x0, w.thr_rel, w.cfl, w.prune_interval, w.limiter)
    o.init_gaussian(w.mean, w.cov)
    with pytest.raises(OracleError):
        o.correct_gaussian(np.array([1e6, 1e6, 1e6]), 0.25 * np.eye(3), np.arange(3, dtype=np.int32))

# ---------------------------------------------------------------- symmetries of the whole step

def _run_const(idx, p, c, h, limiter, t_end, K=3):
    o = const_oracle(c, h, limiter=limiter, thr=1e-3, cfl=0.8, K=K)
    o.init_cells(idx, p)
    st = o.propagate(t_end)
    return o, st


@pytest.mark.parametrize("lim", [LIM_MC, LIM_LW])
def test_translation_of_the_cell_set_translates_the_result_exactly(lim):
    """Under a constant drift nothing depends on where the grid sits: shifting
    every index by an integer vector shifts the result (grow, dt, CTU, prune,
    normalisation), bit for bit."""
    idx, p = W.random_cells(3, 300, 4, seed=31)
    c, h = [0.7, -0.4, 0.25], [0.5, 0.4, 0.3]
    shift = np.array([7, -11, 3], dtype=np.int32)
    a, sa = _run_const(idx, p, c, h, lim, 0.4)
    b, sb = _run_const(idx + shift, p, c, h, lim, 0.4)
    assert sa.steps == sb.steps and sa.t == sb.t
    ca, cb = cells_of(a), cells_of(b)
    assert {tuple(int(x) for x in np.array(k) + shift): v for k, v in ca.items()} == cb


@pytest.mark.parametrize("lim", [LIM_MC, LIM_NONE])
def test_permuting_the_dimensions_permutes_the_result(lim):
    """Relabelling the axes (cells, velocity and widths together) relabels the
    result: a transposed operand or a wrong h index in the step breaks this."""
    idx, p = W.random_cells(3, 250, 4, seed=32)
    c, h = np.array([0.6, -0.3, 0.45]), np.array([0.5, 0.35, 0.45])
    perm = [2, 0, 1]
    a, sa = _run_const(idx, p, list(c), list(h), lim, 0.35)
    b, sb = _run_const(np.ascontiguousarray(idx[:, perm]), p, list(c[perm]), list(h[perm]), lim, 0.35)
    assert sa.steps == sb.steps and sa.t == pytest.approx(sb.t, abs=1e-15)
    ca, cb = cells_of(a), cells_of(b)
    assert set(tuple(k[i] for i in perm) for k in ca) == set(cb)
    scale = max(abs(v) for v in ca.values())
    for k, v in ca.items():
        assert cb[tuple(k[i] for i in perm)] == pytest.approx(v, abs=1e-13 * scale)


@pytest.mark.parametrize("lim", [LIM_MC, LIM_LW])
def test_mirroring_an_axis_and_the_drift_mirrors_the_result(lim):
    """Reflecting axis 0 (i -> -i) with the drift component negated reflects the
    result: upwinding, the sign tests of Algorithm 1 and the limiter's upwind
    wave must treat both directions alike."""
    idx, p = W.random_cells(2, 120, 5, seed=33)
    c, h = [0.55, -0.35], [0.5, 0.4]
    a, sa = _run_const(idx, p, c, h, lim, 0.3)
    mirrored = idx.copy()
    mirrored[:, 0] = -mirrored[:, 0]
    b, sb = _run_const(mirrored, p, [-c[0], c[1]], h, lim, 0.3)
    assert sa.steps == sb.steps
    ca, cb = cells_of(a), cells_of(b)
    assert set((-k[0], k[1]) for k in ca) == set(cb)
    scale = max(abs(v) for v in ca.values())
    for k, v in ca.items():
        assert cb[(-k[0], k[1])] == pytest.approx(v, abs=1e-13 * scale)
