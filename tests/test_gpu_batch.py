"""GPU parity of the batched replica runner: every replica reproduces the
CPU oracle (and the single-lattice path) bit for bit, whatever the tile
height or launch mode."""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
import paper_1208_2080_gb300 as sw
import synth

pytestmark = pytest.mark.gpu

MIXED = dict(
    L=[2, 5, 64, 17, 128, 130, 256, 64, 100, 33],
    q=[2, 3, 2, 5, 8, 255, 4, 3, 2, 2],
    T=[1.0, 0.9, sw.tc(2), 1.3, 0.8, 2.0, sw.tc(4), 0.95, 0.3, 5.0],
    seed=[11, 12, 13, 14, 15, 16, 17, 18, 19, 20],
)


@pytest.mark.parametrize("tile_h,graph,merge", [(64, True, "fused"), (32, False, "kernel"), (16, True, "fused"),
                                               (128, True, "kernel"), (128, False, "fused")])
def test_mixed_batch_matches_oracle(tile_h, graph, merge):
    n = 9
    with sw.Batch(MIXED["L"], MIXED["q"], MIXED["T"], MIXED["seed"], tile_h=tile_h,
                  graph=graph, merge=merge) as b:
        assert b.info()["merge"] == sw._binding.MERGE[merge]
        b.sweep(n)
        for r in range(len(MIXED["L"])):
            L, q, T, seed = (MIXED[k][r] for k in ("L", "q", "T", "seed"))
            ref, refE, refn = oracle.run(L, q, T, seed, n)
            assert np.array_equal(b.spins(r), ref), r
            E, nn = b.series(r, 1, n)
            assert np.array_equal(E, refE) and np.array_equal(nn, refn), r


@pytest.mark.parametrize("tile_h,merge", [(128, "kernel"), (32, "fused")])
def test_batch_three_plane_states_match_oracle(tile_h, merge):
    """A replica batch keeps 4 < q <= 8 in three bit planes (state counts by
    inclusion-exclusion over the plane subsets), q > 8 in bytes: spins and
    every E_sat / n[s] equal the oracle's, for every such q, at ragged and
    tile-spanning sizes, ordered, critical and disordered temperatures."""
    L = [16, 37, 64, 130, 200, 256, 99, 144]
    q = [5, 6, 7, 8, 9, 8, 5, 6]
    T = [sw.tc(5), sw.tc(6), 0.5 * sw.tc(7), sw.tc(8), sw.tc(9), 0.3, 3.0, 1.05 * sw.tc(6)]
    seed = [31, 32, 33, 34, 35, 36, 37, 38]
    n = 7
    with sw.Batch(L, q, T, seed, tile_h=tile_h, merge=merge) as b:
        b.sweep(n)
        for r in range(len(L)):
            ref, refE, refn = oracle.run(L[r], q[r], T[r], seed[r], n)
            assert np.array_equal(b.spins(r), ref), r
            E, nn = b.series(r, 1, n)
            assert np.array_equal(E, refE) and np.array_equal(nn, refn), r
            E_now, n_now, _ = b.measure(r)
            assert E_now == refE[-1] and np.array_equal(n_now[:q[r]], refn[-1]), r


def test_batch_equals_single_lattices():
    p = synth.replica_batch(24, master_seed=99, k_min=6, k_max=9)
    n = 6
    with sw.Batch(p["L"], p["q"], p["T"], p["seed"]) as b:
        b.sweep(n)
        for r in range(24):
            with sw.Sim(int(p["L"][r]), int(p["q"][r]), float(p["T"][r]), int(p["seed"][r])) as s:
                s.sweep(n)
                assert np.array_equal(b.spins(r), s.spins())
                assert np.array_equal(b.series(r, 0, n + 1)[0], s.series(0, n + 1)[0])


def test_batch_set_spins_measure_and_errors():
    with sw.Batch([64, 96], [3, 2], [1.0, 1.1], [1, 2]) as b:
        b.set_spins(0, np.zeros((64, 64), np.uint8))
        E, n, c = b.measure(0)
        assert E == 2 * 64 * 64 and int(n[0]) == 64 * 64 and c == 0
        b.sweep(3)
        ref, refE, _ = oracle.run(64, 3, 1.0, 1, 3, spins=np.zeros((64, 64), np.uint8))
        assert np.array_equal(b.spins(0), ref)
        with pytest.raises(sw.SwError):
            b.set_spins(1, np.full((96, 96), 7, np.uint8))
        with pytest.raises(sw.SwError):
            b.sweep(1)
    with pytest.raises(sw.SwError):
        sw.Batch([64], [1], [1.0], [0])


GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "batch_c4.json")


@pytest.mark.skipif(not os.path.exists(GOLDEN), reason="batch golden values not generated")
def test_c4_512_replicas_2000_sweeps_match_oracle():
    """The 512-replica batch (L = 64..2048, q in {2,3,4,5,8}, T in
    [0.9, 1.1] T_c): after 2000 sweeps every replica's spins and its whole
    E_sat / n[s] series equal the oracle's (stored as SHA-256 digests written
    by tests/golden/make_batch_golden.py, which calls only the oracle)."""
    gold = json.load(open(GOLDEN))
    p = synth.replica_batch(512, master_seed=6)
    sweeps = gold["sweeps"]
    with sw.Batch(p["L"], p["q"], p["T"], p["seed"], ring=sweeps + 1) as b:
        b.sweep(sweeps)
        for r, g in enumerate(gold["replicas"]):
            assert g["L"] == int(p["L"][r]) and g["seed"] == str(int(p["seed"][r]))
            assert sw.threshold(float(p["T"][r])) == g["thr"], f"threshold differs for replica {r}"
            sp = b.spins(r)
            assert hashlib.sha256(np.ascontiguousarray(sp).tobytes()).hexdigest() == g["spins_sha256"], r
            E, n = b.series(r, 1, sweeps)
            assert hashlib.sha256(E.astype("<u8").tobytes()).hexdigest() == g["E_sha256"], r
            assert hashlib.sha256(n.astype("<u8").tobytes()).hexdigest() == g["n_sha256"], r
