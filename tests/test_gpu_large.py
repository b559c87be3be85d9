"""Parity at the production size, q=2, T_c, L=65536 (4.29e9 sites, uint64
labels), all-zero start, in the configuration bench.py times: the oracle
cannot sweep the whole lattice in a test, so it checks sampled outputs one by
one and the observables are recounted independently:
  * E_sat and n[s] recounted from the spins with plain torch ops;
  * sampled sites whose cluster is small: the cluster is found by a bounded
    breadth-first search over bonds computed site by site with the oracle's
    Philox and threshold from the configuration before the sweep; every
    member's new spin must be the oracle's pick for the cluster's smallest
    site index."""
from collections import deque

import numpy as np
import pytest

import oracle
import paper_1208_2080_gb300 as sw

pytestmark = pytest.mark.gpu

L = 65536
Q = 2
SEED = 5


def _word(seed, idx, sweep, dom, word):
    return int(oracle.philox([idx & 0xFFFFFFFF, idx >> 32, sweep, dom],
                             [seed & 0xFFFFFFFF, seed >> 32])[word])


def _bond(spins_at, i, d, thr, sweep):
    """Bond d (0 right, 1 down) owned by site i, from the oracle's streams."""
    y, x = divmod(i, L)
    j = y * L + (x + 1) % L if d == 0 else ((y + 1) % L) * L + x
    if spins_at(i) != spins_at(j):
        return False, j
    return _word(SEED, i >> 1, sweep, 0, 2 * (i & 1) + d) < thr, j


def _cluster(spins_at, i, thr, sweep, cap=48):
    """Members of i's cluster if it has at most `cap` sites, else None."""
    seen, dq = {i}, deque([i])
    while dq:
        u = dq.popleft()
        y, x = divmod(u, L)
        left = y * L + (x - 1) % L
        up = ((y - 1) % L) * L + x
        for owner, d, other in ((u, 0, None), (u, 1, None), (left, 0, u), (up, 1, u)):
            on, j = _bond(spins_at, owner, d, thr, sweep)
            v = owner if other is not None else j
            if on and v not in seen:
                seen.add(v)
                dq.append(v)
                if len(seen) > cap:
                    return None
    return seen


def _check_sweep(before_at, after, thr, sweep, rng, want=150):
    ok = 0
    tries = 0
    while ok < want and tries < 40 * want:
        tries += 1
        i = int(rng.integers(0, L * L))
        c = _cluster(before_at, i, thr, sweep)
        if c is None:
            continue
        r = min(c)
        s = oracle.pick(_word(SEED, r, sweep, 1, 0), Q)
        for v in c:
            assert after[v // L, v % L] == s, (sweep, i, v, r)
        ok += 1
    assert ok >= want // 2, f"only {ok} small clusters sampled"


def _recount(spins_dev):
    import torch
    s = spins_dev.view(L, L)
    E = int((s == torch.roll(s, -1, 1)).sum().item()) + int((s == torch.roll(s, -1, 0)).sum().item())
    n = [int((s == k).sum().item()) for k in range(Q)]
    return E, n


def test_production_size_two_sweeps():
    import torch
    rng = np.random.default_rng(2024)
    thr = oracle.threshold(sw.tc(Q))
    with sw.Sim(L, Q, sw.tc(Q), SEED, init="zero") as sim:
        assert sim.info()["label_bits"] == 64
        assert sim.info()["thr"] == thr
        sim.sweep(1)
        first = sim.spins()
        _check_sweep(lambda i: 0, first, thr, 0, rng)
        sim.sweep(1)
        second = sim.spins()
        _check_sweep(lambda i: int(first[i // L, i % L]), second, thr, 1, rng)
        E, n, c = sim.measure()
        assert c == 2 and sum(int(x) for x in n) == L * L
        dev = torch.from_numpy(second.reshape(-1)).cuda()
        assert _recount(dev) == (E, [int(x) for x in n])
        E1, n1 = sim.series(1, 1)
        assert _recount(torch.from_numpy(first.reshape(-1)).cuda()) == (int(E1[0]),
                                                                        [int(x) for x in n1[0]])
    del dev
    torch.cuda.empty_cache()


GOLDEN_65536 = __import__("os").path.join(__import__("os").path.dirname(__file__), "golden",
                                          "l65536_q2_10.json")


@pytest.mark.skipif(not __import__("os").path.exists(GOLDEN_65536),
                    reason="tests/golden/make_l65536_golden.py has not been run")
@pytest.mark.parametrize("label_bits", [64, 32])
def test_production_size_first_ten_sweeps_match_the_oracle_exactly(label_bits):
    """The whole L = 65536 lattice, bit for bit: the E_sat and n[s] of the
    configurations after sweeps 1..10 and the SHA-256 of the spins after
    sweep 10 equal the oracle's (stored by the golden script).  With 32-bit
    labels the N = 2^32 site indices use the whole label range."""
    import hashlib
    import json

    g = json.load(open(GOLDEN_65536))
    assert g["L"] == L and g["q"] == Q and g["seed"] == SEED
    assert g["thr"] == sw.threshold(sw.tc(Q))
    with sw.Sim(L, Q, sw.tc(Q), SEED, init="zero", label_bits=label_bits) as s:
        s.sweep(g["sweeps"])
        E, n = s.series(1, g["sweeps"])
        spins = s.spins()
        s.sync()
    assert [int(x) for x in E] == g["E"]
    assert [[int(v) for v in row] for row in n] == g["n"]
    assert hashlib.sha256(np.ascontiguousarray(spins).tobytes()).hexdigest() == g["spins_sha256"]


@pytest.mark.skipif(not __import__("os").path.exists(GOLDEN_65536),
                    reason="tests/golden/make_l65536_golden.py has not been run")
def test_production_size_from_host_with_banded_upload_matches_the_oracle():
    """The same ten sweeps started through sw_sweep_host (the all-zero
    configuration uploaded from page-locked host memory in bands, the first
    sweep's labelling overlapped with the upload): the same chain."""
    import hashlib
    import json

    import torch

    g = json.load(open(GOLDEN_65536))
    host = torch.zeros(L * L, dtype=torch.uint8).pin_memory()
    with sw.Sim(L, Q, sw.tc(Q), SEED, init="random", label_bits=64) as s:
        E_last, n_last, cfg = s.sweep_host(host.numpy(), g["sweeps"])
        assert cfg == g["sweeps"]
        assert E_last == g["E"][-1] and [int(x) for x in n_last] == g["n"][-1]
        E, n = s.series(1, g["sweeps"])
        spins = s.spins()
        s.sync()
    assert [int(x) for x in E] == g["E"]
    assert [[int(v) for v in row] for row in n] == g["n"]
    assert hashlib.sha256(np.ascontiguousarray(spins).tobytes()).hexdigest() == g["spins_sha256"]


def _node_word_fits(L, tile_h):
    """Whether the global union-find's words carry node indices at this size
    (key bits 2*xb plus node-index bits within 64), as the library decides."""
    xb = max(1, (L - 1).bit_length())
    nodes = -(-L // 128) * -(-L // tile_h) * (2 * tile_h + 256)
    return 2 * xb + max(1, (nodes - 1).bit_length()) <= 64


def test_largest_lattice_both_node_word_forms_agree():
    """L = 131072 (1.7e10 sites, beyond 2^32): with 128-row tiles the global
    union-find's words carry the parent's node index, with 16-row tiles
    (2.4e9 nodes) they carry its open slot and the node is computed from the
    site key.  Two sweeps from the same random start must give the same
    spins and observables, and the observables must match a recount."""
    import torch
    Lb, q, seed, n = 131072, 2, 17, 2
    assert _node_word_fits(Lb, 128) and not _node_word_fits(Lb, 16)
    out = []
    ref = None
    for th in (128, 16):
        with sw.Sim(Lb, q, sw.tc(q), seed, tile_h=th) as s:
            s.sweep(n)
            E, nn = s.series(0, n + 1)
            sp = torch.empty(Lb * Lb, dtype=torch.uint8, device="cuda")
            s.spins(out=sp)
            torch.cuda.synchronize()
        out.append((E, nn))
        if ref is None:
            ref = sp
        else:
            assert torch.equal(sp, ref)
            del sp
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    # n[1] of the last configuration recounted from the spins
    assert int((ref == 1).sum().item()) == int(out[0][1][-1][1])
    assert int(out[0][1][-1].sum()) == Lb * Lb
    del ref
    torch.cuda.empty_cache()
