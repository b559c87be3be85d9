"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bit-exact on every integer output: initial spins, the packed bond lattice,
cluster roots, spins after every sweep, per-configuration E_sat and n[s].
"""
import numpy as np
import pytest

import oracle
import paper_1208_2080_gb300 as sw

pytestmark = pytest.mark.gpu

TILE_HS = [16, 32, 64, 128]


def _torch():
    import torch
    return torch


# ---- initial spins: pins the GPU Philox against the oracle's ----------------
@pytest.mark.parametrize("L", [2, 3, 5, 17, 64, 100, 129, 256, 301])
def test_init_spins(L):
    q, seed = 5, 1234 + L
    with sw.Sim(L, q, 1.0, seed) as s:
        assert np.array_equal(s.spins(), oracle.init_spins(L, q, seed))


# ---- step (1): bonds ---------------------------------------------------------
@pytest.mark.parametrize("L", [2, 3, 4, 7, 64, 127, 128, 130, 257])
@pytest.mark.parametrize("q", [2, 3])
def test_bonds_bit_exact(L, q):
    T, seed = sw.tc(q), 99 + L
    with sw.Sim(L, q, T, seed, store_bonds=True) as s:
        s0 = s.spins()
        s.sweep(1)
        got = sw.unpack_bonds(s.bonds(), L)
        ref = oracle.bonds(s0, T, seed, 0)
        assert np.array_equal(got, ref)
        s1 = s.spins()
        s.sweep(1)
        assert np.array_equal(sw.unpack_bonds(s.bonds(), L), oracle.bonds(s1, T, seed, 1))


# ---- step (2): labelling of given bond lattices ------------------------------
def _label_gpu(b, label_bits, tile_h):
    torch = _torch()
    L = b.shape[0]
    packed = torch.from_numpy(sw.pack_bonds(b).reshape(-1).copy()).cuda()
    dt = torch.int32 if label_bits == 32 else torch.int64
    roots = torch.empty(L * L, dtype=dt, device="cuda")
    sw.label_bonds(L, packed, roots, label_bits=label_bits, tile_h=tile_h)
    torch.cuda.synchronize()
    r = roots.cpu().numpy()
    return (r.view(np.uint32) if label_bits == 32 else r.view(np.uint64)).reshape(L, L)


@pytest.mark.parametrize("L", [2, 3, 4, 5, 9, 16, 17, 31, 33, 63, 64, 65, 127, 128, 129, 200, 256])
@pytest.mark.parametrize("tile_h", TILE_HS)
def test_label_matches_hk(L, tile_h):
    rng = np.random.default_rng(L * 7 + tile_h)
    for density in [0.0, 1.0, 0.3, 0.5, 0.58, 0.7, 0.9]:
        b = (rng.random((L, L)) < density).astype(np.uint8) | \
            ((rng.random((L, L)) < density).astype(np.uint8) << 1)
        ref = oracle.label(b)
        for bits in (32, 64):
            assert np.array_equal(_label_gpu(b, bits, tile_h), ref), (L, tile_h, density, bits)


def test_label_structured():
    L = 300
    # long horizontal snake that crosses every tile edge and wraps
    b = np.zeros((L, L), np.uint8)
    b[::2, :] |= 1
    b[:, L - 1] |= 2
    b[:, 0] |= 2
    ref = oracle.label(b)
    for th in TILE_HS:
        assert np.array_equal(_label_gpu(b, 32, th), ref)
    # checkerboard of isolated 2x2 blocks straddling tile edges
    b = np.zeros((L, L), np.uint8)
    b[1::2, 1::2] = 3
    ref = oracle.label(b)
    assert np.array_equal(_label_gpu(b, 64, 64), ref)


# ---- whole sweeps ------------------------------------------------------------
CASES = [
    (2, 2, None), (3, 3, None), (5, 2, None), (8, 4, None), (17, 3, None), (31, 5, None),
    (64, 2, None), (100, 8, None), (128, 2, None), (129, 3, None), (200, 255, None),
    (257, 2, None), (64, 2, 0.05), (64, 3, 1e6), (96, 2, 0.5), (160, 4, 3.0),
]


@pytest.mark.parametrize("merge", ["fused", "kernel"])
@pytest.mark.parametrize("L,q,T", CASES)
def test_sweeps_bit_exact(L, q, T, merge):
    T = sw.tc(q) if T is None else T
    seed, n = 7 * L + q, 12
    with sw.Sim(L, q, T, seed, merge=merge) as s:
        assert s.info()["merge"] == sw._binding.MERGE[merge]
        s.sweep(n)
        got = s.spins()
        E, nn = s.series(0, n + 1)
    ref, refE, refn = oracle.run(L, q, T, seed, n)
    assert np.array_equal(got, ref)
    E0, n0 = oracle.measure(oracle.init_spins(L, q, seed), q)
    assert E[0] == E0 and np.array_equal(nn[0], n0)
    assert np.array_equal(E[1:], refE)
    assert np.array_equal(nn[1:], refn)


@pytest.mark.parametrize("L", [96, 250, 1000])
def test_results_independent_of_tile_label_width_and_merge_schedule(L):
    q, T, seed, n = 3, sw.tc(3), 4242, 6
    outs = []
    for th in TILE_HS:
        for bits in (32, 64):
            for merge in ("fused", "kernel"):
                with sw.Sim(L, q, T, seed, tile_h=th, label_bits=bits, merge=merge) as s:
                    s.sweep(n)
                    outs.append((s.spins(), s.series(0, n + 1)))
    for sp, (E, nn) in outs[1:]:
        assert np.array_equal(sp, outs[0][0])
        assert np.array_equal(E, outs[0][1][0]) and np.array_equal(nn, outs[0][1][1])


def test_config_ising_L256_1000_sweeps():
    """q=2, L=256, T_c, random start, 1000 sweeps: every configuration's E_sat
    and n[s] bit-exact, final spins bit-exact."""
    L, q, T, seed, n = 256, 2, sw.tc(2), 1, 1000
    with sw.Sim(L, q, T, seed, ring=2048) as s:
        s.sweep(n)
        got = s.spins()
        E, nn = s.series(1, n)
    ref, refE, refn = oracle.run(L, q, T, seed, n)
    assert np.array_equal(E, refE) and np.array_equal(nn, refn)
    assert np.array_equal(got, ref)


def test_zero_start_and_resume():
    L, q, T, seed = 130, 2, sw.tc(2), 5
    with sw.Sim(L, q, T, seed, init="zero") as a:
        assert not a.spins().any()
        a.sweep(4)
        mid, t = a.spins(), a.sweep_count
        a.sweep(5)
        end = a.spins()
    ref, _, _ = oracle.run(L, q, T, seed, 9, spins=np.zeros((L, L), np.uint8))
    assert np.array_equal(end, ref)
    with sw.Sim(L, q, T, seed) as b:  # different start; resume from the saved state
        b.set_spins(mid)
        b.set_sweep(t)
        b.sweep(5)
        assert np.array_equal(b.spins(), end)


@pytest.mark.parametrize("L", [16, 48, 80, 130, 1040, 4112])
@pytest.mark.parametrize("q", [2, 3, 8, 9, 40])
def test_measure_of_a_given_configuration(L, q):
    """sw_measure of an uploaded configuration (k_measure16 for L a multiple
    of 16: strips of 64 rows with a short last strip at L = 1040 and 4112,
    a second, nearly empty column chunk at L = 4112; the per-row kernel at
    L = 130; register counts for q <= 8, shared histograms above)."""
    rng = np.random.default_rng(7 * L + q)
    s0 = rng.integers(0, q, size=(L, L), dtype=np.uint8)
    E, n = oracle.measure(s0, q)
    with sw.Sim(L, q, sw.tc(q), 5) as s:
        s.set_spins(s0)
        Eg, ng, _ = s.measure()
    assert Eg == int(E) and np.array_equal(ng, np.asarray(n, dtype=np.uint64))


def test_measurement_off_gives_same_chain():
    L, q, T, seed = 140, 3, sw.tc(3), 11
    with sw.Sim(L, q, T, seed) as a, sw.Sim(L, q, T, seed, measure=False) as b:
        a.sweep(7)
        b.sweep(7)
        assert np.array_equal(a.spins(), b.spins())
        assert a.measure()[0] == b.measure()[0]
        with pytest.raises(sw.SwError):
            b.series(0, 3)


def test_device_spin_io():
    torch = _torch()
    L, q, T, seed = 128, 4, sw.tc(4), 3
    with sw.Sim(L, q, T, seed) as s:
        dev = torch.zeros(L * L, dtype=torch.uint8, device="cuda")
        s.spins(out=dev)
        torch.cuda.synchronize()
        assert np.array_equal(dev.cpu().numpy().reshape(L, L), oracle.init_spins(L, q, seed))
        z = torch.zeros(L * L, dtype=torch.uint8, device="cuda")
        s.set_spins(z)
        s.sweep(2)
        ref, _, _ = oracle.run(L, q, T, seed, 2, spins=np.zeros((L, L), np.uint8))
        assert np.array_equal(s.spins(), ref)


def test_ring_window_and_errors():
    L, q, T = 64, 2, sw.tc(2)
    with sw.Sim(L, q, T, 1, ring=8) as s:
        s.sweep(20)
        s.series(13, 8)
        with pytest.raises(sw.SwError) as e:
            s.series(12, 9)
        assert e.value.code == sw._binding.SW_ERR_RANGE
        with pytest.raises(sw.SwError):
            s.set_spins(np.full((L, L), 2, np.uint8))  # state >= q
    with pytest.raises(sw.SwError):
        sw.Sim(1, 2, 1.0, 0)
    with pytest.raises(sw.SwError):
        sw.Sim(8, 256, 1.0, 0)
    with pytest.raises(sw.SwError):
        sw.Sim(8, 2, 0.0, 0)


def test_repeatable():
    L, q, T = 512, 2, sw.tc(2)
    out = []
    for _ in range(3):
        with sw.Sim(L, q, T, 77) as s:
            s.sweep(10)
            out.append(s.spins())
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])


def test_set_spins_rejects_bad_values_on_device():
    torch = _torch()
    L, q = 64, 3
    with sw.Sim(L, q, sw.tc(q), 9) as s:
        bad = torch.full((L * L,), 3, dtype=torch.uint8, device="cuda")
        with pytest.raises(sw.SwError) as e:
            s.set_spins(bad)
        assert e.value.code == sw._binding.SW_ERR_INVAL
        with pytest.raises(sw.SwError) as e:
            s.sweep(1)
        assert e.value.code == sw._binding.SW_ERR_STATE
        s.set_spins(np.zeros((L, L), np.uint8))
        s.sweep(1)
        ref, _, _ = oracle.run(L, q, sw.tc(q), 9, 1, spins=np.zeros((L, L), np.uint8))
        assert np.array_equal(s.spins(), ref)


def test_profile_counts_launches():
    L, q = 300, 2
    with sw.Sim(L, q, sw.tc(q), 1) as s:
        s.profile(True)
        s.sweep(5)
        ms, n = s.profile_read()
        assert n == [5, 5, 5] and all(m > 0 for m in ms)
        s.profile(False)
        s.sweep(2)
        assert s.profile_read()[1] == [5, 5, 5]


def test_large_lattice_properties():
    """L = 8192 (67M sites): a few sweeps bit-exact against the oracle for
    q = 2, 3, 4 at T_c, random start."""
    L, n = 8192, 2
    for q in (2, 3, 4):
        with sw.Sim(L, q, sw.tc(q), 2 + q) as s:
            s.sweep(n)
            got = s.spins()
            E, nn = s.series(1, n)
        ref, refE, refn = oracle.run(L, q, sw.tc(q), 2 + q, n)
        assert np.array_equal(E, refE) and np.array_equal(nn, refn)
        assert np.array_equal(got, ref)


GOLDEN_8192 = __import__("os").path.join(__import__("os").path.dirname(__file__), "golden",
                                         "l8192_q234.json")


@pytest.mark.skipif(not __import__("os").path.exists(GOLDEN_8192),
                    reason="L=8192 golden values not generated")
def test_config_l8192_q234_1200_sweeps_match_oracle():
    """q = 2, 3, 4 at T_c, L = 8192, 200 + 1000 sweeps: spins after sweeps 200
    and 1200 and the whole per-sweep E_sat / n[s] series equal the oracle's
    (SHA-256 digests from tests/golden/make_l8192_golden.py, which calls only
    the oracle); the measured energy approaches Baxter's -(1 + 1/sqrt q)."""
    import hashlib
    import json
    gold = json.load(open(GOLDEN_8192))
    h = lambda a: hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()
    for g in gold["runs"]:
        q, L = g["q"], g["L"]
        assert sw.threshold(sw.tc(q)) == g["thr"]
        with sw.Sim(L, q, sw.tc(q), g["seed"], ring=1300) as s:
            s.sweep(200)
            assert h(s.spins()) == g["spins200_sha256"], q
            s.sweep(1000)
            assert h(s.spins()) == g["spins1200_sha256"], q
            E, n = s.series(1, 1200)
        assert h(E.astype("<u8")) == g["E_sha256"] and h(n.astype("<u8")) == g["n_sha256"], q
        u = -(E[200:].astype(np.float64) / (L * L)).mean()
        assert abs(u - g["u_mean"]) < 1e-12
        assert abs(u + (1 + 1 / np.sqrt(q))) < {2: 2e-3, 3: 5e-3, 4: 1.5e-2}[q]


@pytest.mark.parametrize("L", [7, 64, 130])
def test_set_spins_from_page_locked_host_memory(L):
    """A page-locked host buffer goes through the mapped copy-and-check
    kernel: same chain as from device memory, and a bad state is still
    rejected without touching the sweep counter."""
    import torch
    q = 3
    s0 = oracle.init_spins(L, q, 31)
    pinned = torch.from_numpy(s0.reshape(-1).copy()).pin_memory()
    ref, _, _ = oracle.run(L, q, sw.tc(q), 31, 4, spins=s0)
    with sw.Sim(L, q, sw.tc(q), 31, init="zero") as s:
        s.set_spins(pinned.numpy())
        assert np.array_equal(s.spins(), s0)
        s.sweep(4)
        assert np.array_equal(s.spins(), ref)
        pinned[L * L - 1] = q  # last byte: the tail loop when L*L % 16 != 0
        with pytest.raises(sw.SwError) as e:
            s.set_spins(pinned.numpy())
        assert e.value.code == -1
        pinned[L * L - 1] = 0
        pinned[0] = 7
        with pytest.raises(sw.SwError):
            s.set_spins(pinned.numpy())


@pytest.mark.parametrize("L,tile_h,merge", [(5, 0, "kernel"), (64, 16, "kernel"), (130, 32, "fused"),
                                          (1000, 64, "kernel"), (2048, 64, "kernel"), (2048, 128, "fused")])
def test_sweep_host_overlapped_upload_matches_oracle(L, tile_h, merge):
    """sw_sweep_host: banded upload + labelling from a host configuration
    (pageable and page-locked) gives the oracle's chain and observables,
    with either merge schedule (fused: the bands' labellers unite across
    the tile edges themselves)."""
    import torch
    q, seed = 3, 40 + L
    T = sw.tc(q)
    s0 = oracle.init_spins(L, q, seed + 1)
    ref, E, n = oracle.run(L, q, T, seed, 3, spins=s0, sweep0=2)
    with sw.Sim(L, q, T, seed, tile_h=tile_h, merge=merge) as s:
        s.sweep(2)
        Eg, ng, cfg = s.sweep_host(s0, 3)
        assert cfg == 5
        assert Eg == int(E[-1]) and np.array_equal(ng, n[-1])
        assert np.array_equal(s.spins(), ref)
        Es, ns = s.series(2, 4)  # the uploaded configuration and the three after it
        assert int(Es[0]) == oracle.measure(s0, q)[0]
        assert np.array_equal(Es[1:], E) and np.array_equal(ns[1:], n)
        pinned = torch.from_numpy(s0.reshape(-1).copy()).pin_memory()
        ref2, E2, _ = oracle.run(L, q, T, seed, 1, spins=s0, sweep0=5)
        Eg2, _, cfg2 = s.sweep_host(pinned.numpy(), 1)
        assert cfg2 == 6 and Eg2 == int(E2[-1])
        assert np.array_equal(s.spins(), ref2)
        s.sync()


def test_sweep_host_sixteen_band_plan_equals_the_unbanded_sweep():
    """L = 32768 with 16-row tiles has 2048 tile rows: the doubling band
    plan reaches its 16-band limit and the last band takes the rest.  The
    banded host-driven sweep must give exactly the configuration and the
    observables of sw_set_spins + sw_sweep (oracle-checked on its own)."""
    import torch
    L, q = 32768, 2
    T = sw.tc(q)
    rng = np.random.default_rng(77)
    s0 = torch.from_numpy(rng.integers(0, q, size=L * L, dtype=np.uint8)).pin_memory()
    with sw.Sim(L, q, T, 9, tile_h=16) as a:
        E1, n1, c1 = a.sweep_host(s0.numpy(), 2)
        d1 = torch.empty(L * L, dtype=torch.uint8, device="cuda")
        a.spins(out=d1)
        a.sync()
    with sw.Sim(L, q, T, 9, tile_h=16) as b:
        b.set_spins(s0.numpy())
        b.sweep(2)
        E2, n2, c2 = b.measure()
        d2 = torch.empty(L * L, dtype=torch.uint8, device="cuda")
        b.spins(out=d2)
        b.sync()
    assert (E1, c1) == (E2, c2) and np.array_equal(n1, n2)
    assert torch.equal(d1, d2)
    del d1, d2
    torch.cuda.empty_cache()


def test_sweep_host_rejects_an_invalid_configuration():
    L, q = 96, 2
    with sw.Sim(L, q, sw.tc(q), 3) as s:
        bad = oracle.init_spins(L, q, 9)
        bad[50, 17] = 2
        with pytest.raises(sw.SwError) as e:
            s.sweep_host(bad, 1)
        assert e.value.code == -1
        with pytest.raises(sw.SwError) as e:
            s.sweep(1)
        assert e.value.code == -5
        good = oracle.init_spins(L, q, 9)
        s.set_spins(good)
        cur = s.sweep_count
        s.sweep(2)
        ref, _, _ = oracle.run(L, q, sw.tc(q), 3, 2, spins=good, sweep0=cur)
        assert np.array_equal(s.spins(), ref)
        s.sync()
