"""GPU parity of the Wolff single-cluster update (sw_wolff_*): spins and
cluster sizes bit-identical to the CPU oracle (wolff_oracle.c)."""
import numpy as np
import pytest

import oracle
import paper_1208_2080_gb300 as sw

pytestmark = pytest.mark.gpu


def _compare(L, q, T, seed, steps, init="random", spins=None, mode="grow"):
    s0 = oracle.init_spins(L, q, seed) if init == "random" else np.zeros((L, L), np.uint8)
    if spins is not None:
        s0 = spins
    ref_s, ref_c = oracle.wolff_run(L, q, T, seed, steps, spins=s0)
    with sw.Wolff(L, q, T, seed, init=init, mode=mode) as w:
        if spins is not None:
            w.set_spins(spins)
        assert np.array_equal(w.spins(), s0)
        w.step(steps)
        c = w.sizes(0, steps)
        got = w.spins()
        w.sync()
    assert np.array_equal(c, ref_c), (L, q, T)
    assert np.array_equal(got, ref_s), (L, q, T)


@pytest.mark.parametrize("mode", ["grow", "label"])
@pytest.mark.parametrize("L", [2, 3, 5, 16, 64, 100, 257])
@pytest.mark.parametrize("q", [2, 3, 8])
def test_matches_oracle(L, q, mode):
    T = sw.tc(q)
    _compare(L, q, T, 100 * L + q, 30, mode=mode)
    _compare(L, q, 0.7 * T, 100 * L + q + 1, 10, init="zero", mode=mode)


@pytest.mark.parametrize("mode", ["grow", "label"])
def test_large_clusters_at_low_temperature(mode):
    """An ordered start at T_c / 2: nearly every step grows a cluster of most
    of the lattice."""
    L, q = 1024, 2
    _compare(L, q, 0.5 * sw.tc(q), 3, 6, init="zero", mode=mode)


@pytest.mark.parametrize("mode", ["grow", "label"])
def test_critical_run_against_oracle(mode):
    L, q = 512, 3
    s0 = oracle.run(L, q, sw.tc(q), 17, 30)[0]  # roughly equilibrated by SW sweeps
    _compare(L, q, sw.tc(q), 17, 40, spins=s0, mode=mode)


def test_modes_agree_and_can_be_switched():
    L, q, T = 300, 2, sw.tc(2)
    with sw.Wolff(L, q, T, 5, mode="grow") as a, sw.Wolff(L, q, T, 5) as b:
        a.step(10)
        b.step(10)
        a.set_mode("label")
        b.set_mode("grow")
        a.step(10)
        b.step(10)
        assert np.array_equal(a.spins(), b.spins())
        assert np.array_equal(a.sizes(0, 20), b.sizes(0, 20))
        a.sync()
        b.sync()


def test_label_mode_is_the_default():
    with sw.Wolff(64, 2, sw.tc(2), 9) as d, sw.Wolff(64, 2, sw.tc(2), 9, mode="label") as b:
        d.step(5)
        b.step(5)
        assert np.array_equal(d.spins(), b.spins())
        d.sync()
        b.sync()


def test_set_spins_rejects_bad_states():
    with sw.Wolff(32, 3, 1.0, 1) as w:
        s = w.spins()
        bad = s.copy()
        bad[3, 4] = 3
        with pytest.raises(sw.SwError) as e:
            w.set_spins(bad)
        assert e.value.code == -1
        assert np.array_equal(w.spins(), s)
        w.step(3)
        w.sync()
