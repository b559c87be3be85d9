"""Statistical pins of the whole oracle chain (RNG keying, bond rule, labelling,
recolouring together) against exact results it does not compute:
brute-force enumeration, transfer matrices, Kaufman's closed-form partition
function of the finite Ising torus, and Baxter's closed form for the
critical energy, u(T_c) = -(1 + 1/sqrt q)."""
import numpy as np
import pytest

import oracle
from tests import exact


def _batch_mean(x, nb=50):
    x = np.asarray(x, dtype=np.float64)
    m = len(x) // nb
    b = x[: m * nb].reshape(nb, m).mean(1)
    return b.mean(), b.std(ddof=1) / np.sqrt(nb)


def _chain(L, q, T, seed, n, burn=200):
    _, E, nn = oracle.run(L, q, T, seed, n + burn)
    return E[burn:].astype(np.float64), nn[burn:].astype(np.float64)


@pytest.mark.parametrize("q", [2, 3, 4, 5])
def test_3x3_moments_match_enumeration(q):
    T = oracle.tc(q)
    E, n = _chain(3, q, T, seed=1000 + q, n=200_000)
    e1, e2, nm = exact.brute_moments(3, q, T)
    for data, ref in [(E, e1), (E * E, e2), (n.max(1), nm)]:
        m, s = _batch_mean(data)
        assert abs(m - ref) < 5 * s + 1e-9, (m, ref, s)


@pytest.mark.parametrize("q,T", [(2, 1.0), (2, 2.0), (3, 0.9)])
def test_3x3_off_critical(q, T):
    E, _ = _chain(3, q, T, seed=77, n=100_000)
    e1, _, _ = exact.brute_moments(3, q, T)
    m, s = _batch_mean(E)
    assert abs(m - e1) < 5 * s


def test_4x4_ising_moments_match_enumeration():
    q, T = 2, oracle.tc(2)
    E, n = _chain(4, q, T, seed=4242, n=150_000)
    e1, e2, nm = exact.brute_moments(4, q, T)
    for data, ref in [(E, e1), (E * E, e2), (n.max(1), nm)]:
        m, s = _batch_mean(data)
        assert abs(m - ref) < 5 * s


@pytest.mark.parametrize("L,q", [(8, 2), (5, 3), (4, 4)])
def test_torus_energy_matches_transfer_matrix(L, q):
    T = oracle.tc(q)
    e1, e2 = exact.transfer_moments(L, L, q, T)
    # cross-check the transfer matrix itself against enumeration where possible
    if q ** (L * L) <= 2 ** 16:
        b1, b2, _ = exact.brute_moments(L, q, T)
        assert abs(e1 - b1) < 1e-6 * b1 and abs(e2 - b2) < 1e-6 * b2
    E, _ = _chain(L, q, T, seed=31 * L + q, n=60_000)
    for data, ref in [(E, e1), (E * E, e2)]:
        m, s = _batch_mean(data)
        assert abs(m - ref) < 5 * s, (m, ref, s)


def test_chain_statistics_catch_a_wrong_probability():
    """Run the same chain at a temperature 5% off (what a mistake in p would
    do): the 3x3 check must reject it."""
    q, T = 2, oracle.tc(2)
    E, _ = _chain(3, q, T * 1.05, seed=5, n=100_000)
    e1, _, _ = exact.brute_moments(3, q, T)
    m, s = _batch_mean(E)
    assert abs(m - e1) > 5 * s


@pytest.mark.parametrize("q,tol", [(2, 0.006), (3, 0.025)])
def test_critical_energy_baxter(q, tol):
    """-E_sat/N at T_c approaches -(1+1/sqrt q) (Baxter).  The finite-size
    shift decays as L^((alpha-1)/nu): 1/L for q=2 (about 0.004 at L=128) and
    L^-0.8 for q=3 (about 0.013); the tolerances leave room for both, while a
    wrong bond probability moves u by O(0.1)."""
    L = 128
    T = oracle.tc(q)
    E, _ = _chain(L, q, T, seed=900 + q, n=400, burn=100)
    u = -E / (L * L)
    m, s = _batch_mean(u, nb=20)
    assert abs(m + (1 + 1 / np.sqrt(q))) < 5 * s + tol


def test_3x3_ising_state_histogram_chi_square():
    """Every one of the 512 configurations of the 3 x 3 Ising torus is
    visited with its Boltzmann probability (chi-square over the states, with
    the sample thinned to near-independence)."""
    L, q, T = 3, 2, oracle.tc(2)
    states, E, _ = exact.e_sat_all(L, q)
    w = np.exp((E - E.max()) / T)
    w /= w.sum()
    n = 100_000
    s, _, _ = oracle.run(L, q, T, 77, 100, series=False)  # burn-in: sweeps 0..99
    counts = np.zeros(len(states))
    powers = 2 ** np.arange(L * L - 1, -1, -1)
    for k in range(n):  # the configuration after every 3rd sweep
        s, _, _ = oracle.run(L, q, T, 77, 3, spins=s, sweep0=100 + 3 * k, series=False)
        counts[int(s.ravel().astype(np.int64) @ powers)] += 1
    m = len(counts)
    expect = counts.sum() * w
    chi2 = ((counts - expect) ** 2 / expect).sum()
    dof = m - 1
    assert chi2 < dof + 6 * np.sqrt(2 * dof), (chi2, dof)


def test_kaufman_closed_form_matches_enumeration_and_transfer_matrix():
    """The closed form itself, before it judges the chain: equal to the
    4 x 4 enumeration and the 6 x 6 transfer matrix at four temperatures
    either side of T_c."""
    for T in [oracle.tc(2), 0.8 * oracle.tc(2), 1.5 * oracle.tc(2), 3.0]:
        b1, _, _ = exact.brute_moments(4, 2, T)
        assert abs(exact.kaufman_mean_esat(4, T) - b1) < 1e-9 * b1
        t1, _ = exact.transfer_moments(6, 6, 2, T)
        assert abs(exact.kaufman_mean_esat(6, T) - t1) < 1e-7 * t1


@pytest.mark.parametrize("L,f,n", [(32, 1.0, 40_000), (64, 1.0, 12_000), (32, 0.9, 20_000),
                                   (32, 1.2, 20_000)])
def test_ising_torus_energy_matches_kaufman(L, f, n):
    """<E_sat> of the q = 2 chain on the L = 32 and 64 tori at T_c and either
    side of it equals Kaufman's exact finite-size value within 5 sigma (no
    finite-size allowance needed, unlike the Baxter check)."""
    T = f * oracle.tc(2)
    ref = exact.kaufman_mean_esat(L, T)
    E, _ = _chain(L, 2, T, seed=7000 + L + int(100 * f), n=n)
    m, s = _batch_mean(E)
    assert abs(m - ref) < 5 * s, (m, ref, s)


def test_kaufman_check_catches_a_one_percent_temperature_error():
    """The same L = 32 check rejects a chain run 1% off T_c, the size of
    error a slightly wrong bond probability would make."""
    T = oracle.tc(2)
    ref = exact.kaufman_mean_esat(32, T)
    E, _ = _chain(32, 2, 1.01 * T, seed=7100, n=40_000)
    m, s = _batch_mean(E)
    assert abs(m - ref) > 5 * s, (m, ref, s)
