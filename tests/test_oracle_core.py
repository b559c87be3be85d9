"""Pins of the oracle's threshold, state pick, labelling and measurement."""
from math import isqrt

import numpy as np
import pytest

import oracle
from tests import exact


# ---- bond threshold (Sec. 2 step (1); p = 1 - exp(-1/T)) -----------------

@pytest.mark.parametrize("q", [2, 3, 4, 5, 8])
def test_threshold_at_tc_closed_form(q):
    """At T_c = 1/ln(1+sqrt q), exp(-1/T_c) = 1/(1+sqrt q), so
    p = sqrt(q)/(1+sqrt(q)) exactly; floor(p*2^32) from exact integer
    arithmetic must agree (to the one unit T_c's double rounding allows)."""
    S = 10 ** 40
    sq = isqrt(q * S * S)  # sqrt(q) * S, floored
    exact_thr = (sq << 32) // (S + sq)
    assert abs(oracle.threshold(oracle.tc(q)) - exact_thr) <= 1


def test_threshold_limits():
    assert oracle.threshold(1e12) == 0          # p ~ 1e-12: no bonds
    assert oracle.threshold(1e-3) == 2**32 - 1  # p = 1: clamped
    # monotone decreasing in T
    ts = np.linspace(0.2, 10, 200)
    thr = [oracle.threshold(t) for t in ts]
    assert all(a >= b for a, b in zip(thr, thr[1:]))
    # q=4 at T_c: p = 2/3 -> floor(2^33 / 3)
    assert abs(oracle.threshold(oracle.tc(4)) - (2**33) // 3) <= 1


def test_pick_is_floor_of_scaled_word():
    for q in [2, 3, 5, 8, 255]:
        assert oracle.pick(0, q) == 0
        assert oracle.pick(2**32 - 1, q) == q - 1
        # the boundary between states s-1 and s sits at ceil(s*2^32/q)
        for s in range(1, q):
            edge = -(-(s << 32) // q)
            assert oracle.pick(edge, q) == s
            assert oracle.pick(edge - 1, q) == s - 1


# ---- measurement (Sec. 4) ---------------------------------------------------

def test_measure_special_configurations():
    L, q = 6, 3
    E, n = oracle.measure(np.zeros((L, L), np.uint8), q)
    assert E == 2 * L * L and list(n) == [L * L, 0, 0]
    cb = (np.add.outer(np.arange(L), np.arange(L)) % 2).astype(np.uint8)
    E, n = oracle.measure(cb, q)
    assert E == 0 and list(n) == [18, 18, 0]
    stripes = np.tile((np.arange(L) % 3).astype(np.uint8), (L, 1))  # columns
    E, n = oracle.measure(stripes, q)
    assert E == L * L  # only the vertical bonds are satisfied
    assert list(n) == [12, 12, 12]
    # L = 2: right and wrap bond join the same pair twice
    E, _ = oracle.measure(np.array([[0, 0], [1, 1]], np.uint8), 2)
    assert E == 4


def test_measure_matches_brute_force_counts():
    rng = np.random.default_rng(3)
    for L in [2, 3, 5, 8]:
        for q in [2, 3, 7]:
            s = rng.integers(0, q, size=(L, L)).astype(np.uint8)
            E, n = oracle.measure(s, q)
            ref = sum(int(s[y, x] == s[y, (x + 1) % L]) + int(s[y, x] == s[(y + 1) % L, x])
                      for y in range(L) for x in range(L))
            assert E == ref
            assert list(n) == [int((s == k).sum()) for k in range(q)]


# ---- labelling (Sec. 2 step (2), Hoshen-Kopelman label = smallest) ---------

def _random_bonds(rng, L, density):
    b = (rng.random((L, L)) < density).astype(np.uint8) * exact.RIGHT
    b |= (rng.random((L, L)) < density).astype(np.uint8) * exact.DOWN
    return b


@pytest.mark.parametrize("L", list(range(2, 13)))
def test_label_matches_bfs(L):
    rng = np.random.default_rng(100 + L)
    for trial in range(150):
        density = [0.0, 1.0, 0.25, 0.5, 0.6, 0.75][trial % 6]
        b = _random_bonds(rng, L, density)
        assert np.array_equal(oracle.label(b), exact.bfs_roots(b))


def test_label_structured_fields():
    L = 9
    idx = np.arange(L * L).reshape(L, L)
    # only the wrap bonds: column L-1 joined to column 0 in every row
    b = np.zeros((L, L), np.uint8)
    b[:, L - 1] = exact.RIGHT
    r = oracle.label(b)
    assert np.array_equal(r[:, L - 1], idx[:, 0]) and np.array_equal(r[:, 0], idx[:, 0])
    # a spiral-like snake forcing a long chain whose minimum sits at the end
    b = np.zeros((L, L), np.uint8)
    b[L - 1, :] = exact.RIGHT
    b[:, L - 1] |= exact.DOWN
    r = oracle.label(b)
    assert np.array_equal(r, exact.bfs_roots(b))
    # bottom row + last column (which wraps down to row 0): minimum is site L-1
    assert r[L - 1, 3] == L - 1 and r[0, L - 1] == L - 1
    # all bonds active: one cluster rooted at 0
    assert np.all(oracle.label(np.full((L, L), 3, np.uint8)) == 0)
    # no bonds: every site its own root
    assert np.array_equal(oracle.label(np.zeros((L, L), np.uint8)), idx)


def test_label_invariants_large():
    rng = np.random.default_rng(5)
    L = 64
    b = _random_bonds(rng, L, 0.5)
    r = oracle.label(b).ravel().astype(np.int64)
    ri, di = exact.neighbours(L)
    f = b.ravel()
    assert np.all(r <= np.arange(L * L))
    assert np.all(r[r] == r)  # roots are their own roots
    assert np.all(r[(f & 1) > 0] == r[ri[(f & 1) > 0]])
    assert np.all(r[(f & 2) > 0] == r[di[(f & 2) > 0]])
    assert np.array_equal(r.reshape(L, L), exact.bfs_roots(b))


# ---- recolouring special cases (Sec. 2 step (3)) ----------------------------

def test_recolor_constant_on_clusters_and_drawn_at_root():
    rng = np.random.default_rng(11)
    L, q, seed, sweep = 10, 5, 77, 3
    b = _random_bonds(rng, L, 0.55)
    root = oracle.label(b)
    s = oracle.recolor(np.zeros((L, L), np.uint8), root, q, seed, sweep)
    flat, rf = s.ravel(), root.ravel()
    assert np.all(flat == flat[rf])
    for r in np.unique(rf)[:20]:
        w = oracle.philox([int(r) & 0xFFFFFFFF, int(r) >> 32, sweep, 1],
                          [seed & 0xFFFFFFFF, seed >> 32])[0]
        assert flat[r] == oracle.pick(w, q)


def test_special_case_no_bonds_every_site_draws_its_own_state():
    """thr = 0 (T -> infinity): no bond is active, every site is its own
    root, and its new state is the pick of its own state word."""
    L, q, seed, sweep = 7, 5, 12, 3
    s = oracle.init_spins(L, q, seed)
    T = 1e300
    assert oracle.threshold(T) == 0
    b = oracle.bonds(s, T, seed, sweep)
    assert not b.any()
    root = oracle.label(b)
    assert np.array_equal(root.ravel(), np.arange(L * L))
    s2 = oracle.recolor(s, root, q, seed, sweep)
    want = [oracle.pick(int(oracle.philox([i, 0, sweep, 1], [seed, 0])[0]), q) for i in range(L * L)]
    assert np.array_equal(s2.ravel(), np.array(want, dtype=np.uint8))


def test_special_case_uniform_start_at_zero_temperature_is_one_cluster():
    """thr = 2^32 - 1 and a uniform start: (almost surely) every bond is
    active, one cluster rooted at site 0, and all spins take the pick of
    site 0's state word."""
    L, q, seed = 9, 3, 4
    T = 1e-3
    assert oracle.threshold(T) == 2 ** 32 - 1
    s = np.full((L, L), 2, dtype=np.uint8)
    s1, _, _ = oracle.run(L, q, T, seed, 1, spins=s)
    want = oracle.pick(int(oracle.philox([0, 0, 0, 1], [seed, 0])[0]), q)
    assert np.all(s1 == want)
