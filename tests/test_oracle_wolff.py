"""Pins of the Wolff single-cluster oracle (wolff_oracle.c) against what
the mathematics fixes: the seed and new state from their Philox words, the
cluster as the breadth-first component of the seed among the active bonds,
the exact transition matrix of tiny lattices (Boltzmann-stationary, detailed
balance), enumeration of 3 x 3 lattices, and the improved estimator
<|C|> = <M^2>/N of the Ising case."""
import numpy as np
import pytest

import oracle
from tests import exact


def _words(seed, idx, t, dom):
    return oracle.philox([idx & 0xFFFFFFFF, idx >> 32, t, dom], [seed & 0xFFFFFFFF, seed >> 32])


def test_seed_and_new_state_from_their_words():
    rng = np.random.default_rng(1)
    for L, q in [(2, 2), (5, 3), (64, 5), (7, 255)]:
        s = rng.integers(0, q, size=(L, L)).astype(np.uint8)
        for t in (0, 1, 999):
            w = _words(21, 0, t, 4)
            i0, sn = oracle.wolff_seed(s, q, 21, t)
            assert i0 == (int(w[0]) * L * L) >> 32
            old = int(s.ravel()[i0])
            assert sn == (old + 1 + oracle.pick(int(w[1]), q - 1)) % q and sn != old


@pytest.mark.parametrize("L,q,T", [(2, 2, 1.0), (5, 3, 0.9), (16, 2, 1.1346), (33, 4, 0.8), (48, 2, 0.5)])
def test_cluster_is_the_bfs_component_of_the_seed(L, q, T):
    rng = np.random.default_rng(L * q)
    thr = oracle.threshold(T)
    for t in range(6):
        s = rng.integers(0, q, size=(L, L)).astype(np.uint8) if t % 2 else \
            np.where(rng.random((L, L)) < 0.8, 0, 1).astype(np.uint8)
        i0, sn = oracle.wolff_seed(s, q, 33, t)
        old = s.ravel()[i0]
        r_idx, d_idx = exact.neighbours(L)
        flat = s.ravel()
        b = np.zeros(L * L, dtype=np.uint8)
        for i in range(L * L):
            w = _words(33, i >> 1, t, 5)
            for d, nb in ((0, r_idx[i]), (1, d_idx[i])):
                if flat[i] == old and flat[nb] == old and w[2 * (i & 1) + d] < thr:
                    b[i] |= 1 << d
        roots = exact.bfs_roots(b.reshape(L, L)).ravel()
        comp = roots == roots[i0]
        s2, size = oracle.wolff_step(s, q, T, 33, t)
        assert size == comp.sum()
        assert np.array_equal(s2.ravel(), np.where(comp, sn, flat))


@pytest.mark.parametrize("L,q,T", [(2, 2, 1.1346), (2, 3, 0.9)])
def test_exact_transition_matrix_stationary(L, q, T):
    p = oracle.threshold(T) / 2.0 ** 32
    P, E = exact.wolff_transition(L, q, p)
    assert np.allclose(P.sum(1), 1.0, atol=1e-12)
    T_eff = -1.0 / np.log1p(-p)
    pi = np.exp((E - E.max()) / T_eff)
    pi /= pi.sum()
    assert np.max(np.abs(pi @ P - pi)) < 1e-12
    flow = pi[:, None] * P
    assert np.max(np.abs(flow - flow.T)) < 1e-12


def test_one_oracle_step_follows_the_exact_transition_row():
    L, q, T = 2, 3, 0.9
    P, _ = exact.wolff_transition(L, q, oracle.threshold(T) / 2.0 ** 32)
    s0 = np.array([[0, 0], [1, 0]], dtype=np.uint8)
    powers = q ** np.arange(L * L - 1, -1, -1)
    row = P[int(s0.ravel().astype(np.int64) @ powers)]
    n = 30000
    counts = np.zeros(len(row))
    for seed in range(n):
        s1, _ = oracle.wolff_step(s0, q, T, seed, 0)
        counts[int(s1.ravel().astype(np.int64) @ powers)] += 1
    expect = n * row
    assert counts[expect == 0].sum() == 0
    m = expect > 0
    chi2 = (((counts - expect) ** 2)[m] / expect[m]).sum()
    dof = m.sum() - 1
    assert chi2 < dof + 6 * np.sqrt(2 * dof), (chi2, dof)


def _batch_mean(x, nb=40):
    x = np.asarray(x, dtype=np.float64)
    m = len(x) // nb
    b = x[: m * nb].reshape(nb, m).mean(1)
    return b.mean(), b.std(ddof=1) / np.sqrt(nb)


@pytest.mark.parametrize("q,T", [(2, 1.1346), (3, 0.9)])
def test_3x3_chain_matches_enumeration(q, T):
    e1, e2, nm = exact.brute_moments(3, q, T)
    s = oracle.init_spins(3, q, 5)
    E, C, NM = [], [], []
    for t in range(60000):
        s, c = oracle.wolff_step(s, q, T, 5, t)
        e, n = oracle.measure(s, q)
        E.append(e)
        C.append(c)
        NM.append(n.max())
    E = np.array(E[500:], dtype=np.float64)
    for data, ref in [(E, e1), (E * E, e2), (np.array(NM[500:]), nm)]:
        mean, err = _batch_mean(data)
        assert abs(mean - ref) < 5 * err + 1e-9, (mean, ref, err)
    if q == 2:
        # improved estimator of the Ising susceptibility: <|C|> = <M^2>/N
        _, Es, n = exact.e_sat_all(3, 2)
        w = np.exp((Es - Es.max()) / T)
        w /= w.sum()
        M2 = ((n[:, 0] - n[:, 1]) ** 2).astype(np.float64)
        mean, err = _batch_mean(np.array(C[500:], dtype=np.float64))
        assert abs(mean - (w * M2).sum() / 9) < 5 * err


def test_run_matches_repeated_steps():
    L, q, T = 24, 3, 0.95
    s0 = oracle.init_spins(L, q, 8)
    s = s0.copy()
    sizes = []
    for t in range(40):
        s, c = oracle.wolff_step(s, q, T, 8, t)
        sizes.append(c)
    s2, c2 = oracle.wolff_run(L, q, T, 8, 40, spins=s0)
    assert np.array_equal(s, s2) and list(c2) == sizes
