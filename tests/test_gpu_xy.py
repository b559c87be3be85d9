"""GPU parity of the XY model's embedded-cluster sweep (sw_xy_*): every
configuration and every per-sweep observable record is bit-identical to the
CPU oracle (xy_oracle.c) on the same seeds."""
import numpy as np
import pytest

import oracle
import paper_1208_2080_gb300 as sw

pytestmark = pytest.mark.gpu


def _compare(L, M, T, seed, sweeps, **kw):
    init = kw.get("init", "random")
    s0 = oracle.xy_init(L, M, seed) if init == "random" else np.zeros((L, L), np.uint8)
    ref_s, ref_D, ref_n = oracle.xy_run(L, M, T, seed, sweeps, spins=s0)
    with sw.XY(L, M, T, seed, **kw) as x:
        assert np.array_equal(x.spins(), s0)
        x.sweep(sweeps)
        D, n = x.series(1, sweeps)
        got = x.spins()
        x.sync()
    assert np.array_equal(got, ref_s), (L, M, T)
    assert np.array_equal(D, ref_D), (L, M, T)
    assert np.array_equal(n, ref_n), (L, M, T)


@pytest.mark.parametrize("L", [2, 3, 5, 16, 64, 100, 128, 130, 257])
@pytest.mark.parametrize("M", [2, 3, 8, 256])
def test_matches_oracle(L, M):
    for k, T in enumerate([0.5, sw.T_KT, 2.0]):
        _compare(L, M, T, 1000 * L + 10 * M + k, 6)


@pytest.mark.parametrize("tile_h", [16, 32, 64, 128])
@pytest.mark.parametrize("bits", [32, 64])
def test_tile_heights_and_label_widths(tile_h, bits):
    _compare(300, 256, sw.T_KT, 77, 5, tile_h=tile_h, label_bits=bits)
    _compare(129, 64, 0.7, 78, 5, tile_h=tile_h, label_bits=bits, init="zero")


def test_large_lattice_several_sweeps():
    _compare(2048, 256, sw.T_KT, 5, 4)


def test_m4_energy_is_two_ising_energies_at_scale():
    """M = 4 at the Ising critical point of J = 1/2 (T = 1/ln(1+sqrt 2)):
    the energy per site approaches -sqrt 2 (two critical Ising models)."""
    L, T = 512, 1.0 / np.log1p(np.sqrt(2.0))
    with sw.XY(L, 4, T, 3) as x:
        x.sweep(400)
        D, _ = x.series(201, 200)
    e = oracle.xy_energy(D, 4) / (L * L)
    assert abs(e.mean() + np.sqrt(2.0)) < 0.01


def test_set_spins_validation_and_measure_on_request():
    L, M = 64, 8
    with sw.XY(L, M, 0.9, 4, measure=False) as x:
        x.sweep(3)
        with pytest.raises(sw.SwError) as e:
            x.series(1, 3)
        assert e.value.code == -7
        D, n = x.series(3, 1)
        s = x.spins()
        Dr, nr = oracle.xy_measure(s, M)
        assert np.array_equal(D[0], Dr) and np.array_equal(n[0], nr)
        bad = s.copy()
        bad[5, 7] = M
        with pytest.raises(sw.SwError) as e:
            x.set_spins(bad)
        assert e.value.code == -1
        with pytest.raises(sw.SwError) as e:
            x.sweep(1)
        assert e.value.code == -5
        x.set_spins(s)
        x.sweep(2)
        ref, _, _ = oracle.xy_run(L, M, 0.9, 4, 2, spins=s, sweep0=3)
        assert np.array_equal(x.spins(), ref)


def test_ring_window_and_profile():
    L, M = 96, 16
    with sw.XY(L, M, 1.1, 8, ring=4) as x:
        x.profile(True)
        x.sweep(10)
        ms, n = x.profile_read()
        assert n == [10, 10, 10, 10] and all(t > 0 for t in ms)
        D, _ = x.series(7, 4)
        assert D.sum(1).tolist() == [2 * L * L] * 4
        with pytest.raises(sw.SwError) as e:
            x.series(6, 1)
        assert e.value.code == -7
