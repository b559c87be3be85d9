"""Exact pins of the SW rule as the oracle implements it (no RNG involved):
the transition matrix built from the oracle's labeller and threshold leaves
the Boltzmann distribution of Eq. 1 invariant and obeys detailed balance."""
import numpy as np
import pytest

import oracle
from tests import exact


@pytest.mark.parametrize("L,q,T", [(2, 2, None), (2, 3, None), (2, 4, 0.7), (3, 2, None)])
def test_transition_matrix_stationary(L, q, T):
    T = oracle.tc(q) if T is None else T
    p = oracle.threshold(T) / 2.0 ** 32  # P(u < thr) for a uniform 32-bit u
    P, E = exact.sw_transition(L, q, p, oracle.label)
    assert np.allclose(P.sum(1), 1.0, atol=1e-12)
    pi = np.exp((E - E.max()) / T)
    pi /= pi.sum()
    # Boltzmann weight uses the oracle's own p: exp(-1/T_eff) = 1 - p
    T_eff = -1.0 / np.log1p(-p)
    pi_eff = np.exp((E - E.max()) / T_eff)
    pi_eff /= pi_eff.sum()
    assert np.max(np.abs(pi_eff @ P - pi_eff)) < 1e-12
    flow = pi_eff[:, None] * P
    assert np.max(np.abs(flow - flow.T)) < 1e-12
    # and T_eff is T to double precision (threshold rounding is ~2^-32)
    assert abs(T_eff - T) / T < 1e-8
    assert np.max(np.abs(pi @ P - pi)) < 1e-8


def test_transition_matrix_catches_a_broken_labeller():
    """A labeller that ignores the wrap bonds must break stationarity (the
    check is sensitive to the mistakes it is meant to catch)."""
    def no_wrap(b):
        b = np.array(b, copy=True)
        b[:, -1] &= ~np.uint8(1)
        b[-1, :] &= ~np.uint8(2)
        return oracle.label(b)

    L, q = 2, 2
    T = oracle.tc(q)
    p = oracle.threshold(T) / 2.0 ** 32
    P, E = exact.sw_transition(L, q, p, no_wrap)
    pi = np.exp((E - E.max()) / T)
    pi /= pi.sum()
    assert np.max(np.abs(pi @ P - pi)) > 1e-3
