"""Pins of the XY-model oracle (embedded-cluster SW sweep, xy_oracle.c)
against what the mathematics fixes: vector geometry of Wolff's embedding,
high-precision bond probabilities, the M = 2 reduction to the Ising/Potts
sweep, the M = 4 reduction to two independent Ising models, brute-force
measurement, and the exact transition matrix and Boltzmann distribution of
tiny lattices."""
import itertools

import mpmath
import numpy as np
import pytest

import oracle
from tests import exact


@pytest.mark.parametrize("M", [2, 3, 4, 5, 8, 64, 255, 256])
def test_thresholds_match_high_precision(M):
    T = 0.9
    tt = oracle.xy_thresholds(M, T)
    H = M // 2
    assert tt.shape == (H + 1, H + 1)
    assert np.array_equal(tt, tt.T)
    assert not tt[0].any()
    mpmath.mp.dps = 40
    for c in range(H + 1):
        for d in range(H + 1):
            p = 1 - mpmath.exp(-2 * mpmath.sin(mpmath.pi * c / M) * mpmath.sin(mpmath.pi * d / M) / T)
            ref = min(int(mpmath.floor(p * 2 ** 32)), 2 ** 32 - 1)
            assert abs(int(tt[c, d]) - ref) <= 1, (c, d)
    # rows increase with |sigma|
    assert np.all(np.diff(tt[1:, 1:].astype(np.int64), axis=0) >= 0)


@pytest.mark.parametrize("T", [0.5, 0.9, 2.0])
def test_threshold_of_antiparallel_axis_is_the_potts_threshold_at_half_T(T):
    """|sigma| = 1 on both ends: p = 1 - exp(-2/T), the q = 2 Potts (J = 1)
    probability at T/2."""
    for M in (2, 4, 6, 8, 256):
        assert int(oracle.xy_thresholds(M, T)[M // 2, M // 2]) == oracle.threshold(T / 2)


@pytest.mark.parametrize("M", [2, 3, 4, 5, 8, 13])
def test_bond_eligibility_is_the_sign_of_the_projection(M):
    """At T -> 0 a bond is active exactly when sigma_i sigma_j > 0, sigma the
    projection on the embedding vector (computed here with vectors)."""
    T = 1e-6
    for j in range(M):
        for k1, k2 in itertools.product(range(M), repeat=2):
            s = np.array([[k1, k2], [k2, k1]], dtype=np.uint8)
            b = oracle.xy_bonds(s, M, T, seed=3, sweep=0, j=j)
            s1, s2 = exact.xy_sigma(k1, M, j), exact.xy_sigma(k2, M, j)
            want = (s1 * s2 > 1e-12)
            # every bond of this 2 x 2 pattern joins a k1 site and a k2 site
            assert np.all((b & 1).astype(bool) == want), (M, j, k1, k2)
            assert np.all((b & 2).astype(bool) == want), (M, j, k1, k2)


@pytest.mark.parametrize("M", [2, 3, 6, 8, 256])
def test_flip_reflects_whole_clusters_across_the_embedding_axis(M):
    rng = np.random.default_rng(M)
    L = 9
    s = rng.integers(0, M, size=(L, L)).astype(np.uint8)
    b = rng.integers(0, 4, size=(L, L)).astype(np.uint8)
    root = oracle.label(b)
    for sweep in range(4):
        j = oracle.xy_axis(5, sweep, M)
        refl = np.array([exact.xy_reflect(k, M, j) for k in range(M)])
        s2 = oracle.xy_flip(s, root, M, 5, sweep)
        flipped = s2 != s
        assert np.all((s2 == s) | (s2 == refl[s]))
        # a cluster flips as a whole: every member that moves agrees with the
        # root's coin, and members that cannot move are the fixed points
        for r in np.unique(root):
            m = root == r
            moving = m & (refl[s] != s)
            if moving.any():
                assert flipped[moving].all() or not flipped[moving].any()
        # the coin is the root's Potts state word with q = 2
        for r in np.unique(root):
            rr = int(r)
            coin = oracle.pick(oracle.philox([rr & 0xFFFFFFFF, rr >> 32, sweep, 1], [5, 0])[0], 2)
            y, x = divmod(rr, L)
            assert s2[y, x] == (refl[s[y, x]] if coin else s[y, x])


def test_axis_is_the_pick_of_its_philox_word():
    for M in (2, 3, 256):
        for sweep in (0, 1, 77):
            w = oracle.philox([0, 0, sweep, 3], [11, 0])[0]
            assert oracle.xy_axis(11, sweep, M) == oracle.pick(w, M)


def test_m2_sweep_is_the_ising_sweep():
    """M = 2: axis 1 gives sigma = +-1 and the bonds of the q = 2 Potts sweep
    at T/2 (same Philox words); axis 0 gives sigma = 0 and no bonds."""
    rng = np.random.default_rng(4)
    for L in (2, 5, 16):
        s = rng.integers(0, 2, size=(L, L)).astype(np.uint8)
        for T in (0.8, 1.5):
            for sweep in (0, 3):
                b1 = oracle.xy_bonds(s, 2, T, 9, sweep, j=1)
                assert np.array_equal(b1, oracle.bonds(s, T / 2, 9, sweep))
                assert not oracle.xy_bonds(s, 2, T, 9, sweep, j=0).any()


@pytest.mark.parametrize("L,M", [(3, 3), (4, 8), (5, 256), (7, 5)])
def test_measure_matches_brute_force(L, M):
    rng = np.random.default_rng(L * M)
    s = rng.integers(0, M, size=(L, L)).astype(np.uint8)
    D, n = oracle.xy_measure(s, M)
    Dref = np.zeros(M // 2 + 1, dtype=np.int64)
    for y in range(L):
        for x in range(L):
            for (yy, xx) in (((y, (x + 1) % L)), (((y + 1) % L, x))):
                dlt = (int(s[y, x]) - int(s[yy, xx])) % M
                Dref[min(dlt, M - dlt)] += 1
    assert np.array_equal(D.astype(np.int64), Dref)
    assert np.array_equal(n.astype(np.int64), np.bincount(s.ravel(), minlength=M))
    ang = 2 * np.pi * s / M
    Eref = -(np.cos(ang - np.roll(ang, -1, 1)).sum() + np.cos(ang - np.roll(ang, -1, 0)).sum())
    assert abs(oracle.xy_energy(D, M) - Eref) < 1e-9


def test_exact_transition_matrix_keeps_boltzmann_and_detailed_balance():
    """The embedded-cluster sweep as read here (axes on the half-grid,
    reflection probability 1/2), built from vector geometry and the oracle's
    labeller: Boltzmann-stationary with detailed balance."""
    L, M, T = 2, 3, 0.8
    P, H = exact.xy_transition(L, M, T, oracle.label)
    assert np.allclose(P.sum(1), 1.0, atol=1e-12)
    pi = np.exp(-(H - H.min()) / T)
    pi /= pi.sum()
    assert np.max(np.abs(pi @ P - pi)) < 1e-12
    flow = pi[:, None] * P
    assert np.max(np.abs(flow - flow.T)) < 1e-12


def test_one_oracle_sweep_follows_the_exact_transition_row():
    """From a fixed 2 x 2 configuration, one oracle sweep over many seeds
    lands on each configuration with the exact probabilities (chi-square)."""
    L, M, T = 2, 3, 0.8
    P, _ = exact.xy_transition(L, M, T, oracle.label)
    s0 = np.array([[0, 1], [2, 0]], dtype=np.uint8)
    powers = M ** np.arange(L * L - 1, -1, -1)
    row = P[int(s0.ravel().astype(np.int64) @ powers)]
    n = 40000
    counts = np.zeros(len(row))
    for seed in range(n):
        s1, _, _ = oracle.xy_run(L, M, T, seed, 1, spins=s0, series=False)
        counts[int(s1.ravel().astype(np.int64) @ powers)] += 1
    expect = n * row
    assert counts[expect == 0].sum() == 0
    m = expect > 0
    chi2 = (((counts - expect) ** 2)[m] / expect[m]).sum()
    dof = m.sum() - 1
    assert chi2 < dof + 6 * np.sqrt(2 * dof), (chi2, dof)


def _batch_mean(x, nb=50):
    x = np.asarray(x, dtype=np.float64)
    m = len(x) // nb
    b = x[: m * nb].reshape(nb, m).mean(1)
    return b.mean(), b.std(ddof=1) / np.sqrt(nb)


@pytest.mark.parametrize("M,T", [(3, 1.0), (5, 0.8)])
def test_3x3_chain_matches_enumeration(M, T):
    states, H = exact.xy_energy_all(3, M)
    w = np.exp(-(H - H.min()) / T)
    w /= w.sum()
    ang = 2 * np.pi * states / M
    m2 = np.cos(ang).sum(1) ** 2 + np.sin(ang).sum(1) ** 2
    e1, e2, mm = (w * H).sum(), (w * H * H).sum(), (w * m2).sum()
    _, D, n = oracle.xy_run(3, M, T, seed=100 + M, nsweeps=200_000)
    E = oracle.xy_energy(D[200:], M)
    mx, my = oracle.xy_magnetisation(n[200:], M)
    for data, ref in [(E, e1), (E * E, e2), (mx * mx + my * my, mm)]:
        mean, err = _batch_mean(data)
        assert abs(mean - ref) < 5 * err + 1e-9, (mean, ref, err)


def test_m4_is_two_independent_ising_models():
    """M = 4: H = -sum cos = 2N - E_sat(u) - E_sat(v) for two q = 2 Potts
    models (J = 1) at the same T; exact <E_sat> on the 4 x 4 torus from the
    transfer matrix."""
    L, T = 4, 1.2
    esat, _ = exact.transfer_moments(L, L, 2, T)
    ref = 2 * L * L - 2 * esat
    _, D, _ = oracle.xy_run(L, 4, T, seed=41, nsweeps=100_000)
    mean, err = _batch_mean(oracle.xy_energy(D[200:], 4))
    assert abs(mean - ref) < 5 * err, (mean, ref, err)


def test_transition_check_catches_a_broken_labeller():
    """The exact check is sensitive: a labeller that drops the periodic wrap
    bonds breaks stationarity of the embedded sweep."""
    def no_wrap(b):
        b = np.array(b, copy=True)
        b[:, -1] &= ~np.uint8(1)
        b[-1, :] &= ~np.uint8(2)
        return oracle.label(b)

    L, M, T = 2, 3, 0.8
    P, H = exact.xy_transition(L, M, T, no_wrap)
    pi = np.exp(-(H - H.min()) / T)
    pi /= pi.sum()
    assert np.max(np.abs(pi @ P - pi)) > 1e-4
