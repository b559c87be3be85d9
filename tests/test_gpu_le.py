"""The paper's label-equivalence labeller (sw_label_bonds_le) gives exactly
the Hoshen-Kopelman roots of the oracle and the tile union-find's roots."""
import numpy as np
import pytest

import oracle
import paper_1208_2080_gb300 as sw
import synth

pytestmark = pytest.mark.gpu


def _le(b, bits):
    import torch
    L = b.shape[0]
    packed = torch.from_numpy(sw.pack_bonds(b).reshape(-1).copy()).cuda()
    roots = torch.empty(L * L, dtype=torch.int32 if bits == 32 else torch.int64, device="cuda")
    it = sw.label_bonds_le(L, packed, roots, label_bits=bits)
    torch.cuda.synchronize()
    r = roots.cpu().numpy()
    return (r.view(np.uint32) if bits == 32 else r.view(np.uint64)).reshape(L, L), it


@pytest.mark.parametrize("L", [2, 3, 5, 16, 33, 100, 257])
def test_le_matches_hk(L):
    for k, d in enumerate([0.0, 0.3, 0.5, 0.58, 0.8, 1.0]):
        b = synth.random_bonds(L, d, 1000 * L + k)
        ref = oracle.label(b)
        for bits in (32, 64):
            got, it = _le(b, bits)
            assert np.array_equal(got, ref), (L, d, bits)
            assert it >= 1


def test_le_matches_tile_union_find_on_equilibrium_bonds():
    import torch
    L, q = 1024, 2
    with sw.Sim(L, q, sw.tc(q), 9, store_bonds=True) as s:
        s.sweep(40)
        packed = torch.from_numpy(s.bonds().reshape(-1).copy()).cuda()
    a = torch.empty(L * L, dtype=torch.int32, device="cuda")
    b = torch.empty(L * L, dtype=torch.int32, device="cuda")
    sw.label_bonds(L, packed, a, label_bits=32)
    it = sw.label_bonds_le(L, packed, b, label_bits=32)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    assert 2 <= it <= 64


def _two_stage(b, sub, bits):
    import torch
    L = b.shape[0]
    packed = torch.from_numpy(sw.pack_bonds(b).reshape(-1).copy()).cuda()
    roots = torch.empty(L * L, dtype=torch.int32 if bits == 32 else torch.int64, device="cuda")
    it = sw.label_bonds_2stage(L, sub, packed, roots, label_bits=bits)
    torch.cuda.synchronize()
    r = roots.cpu().numpy()
    return (r.view(np.uint32) if bits == 32 else r.view(np.uint64)).reshape(L, L), it


@pytest.mark.parametrize("L,subs", [(2, [2]), (4, [2, 4]), (6, [2, 3, 6]), (16, [2, 4, 8, 16]),
                                    (48, [3, 16, 24, 48]), (100, [2, 10, 25, 50]), (256, [16, 64])])
def test_two_stage_matches_hk(L, subs):
    """The paper's two-stage labelling (Sec. 3), emulated with (L/sub)^2
    sub-lattices, gives the oracle's roots for every split, including the
    degenerate ones (one sub-lattice: every periodic bond crosses its own
    boundary; 2 x 2 sub-lattices: every site is a boundary site)."""
    for k, d in enumerate([0.0, 0.3, 0.5, 0.58, 0.8, 1.0]):
        b = synth.random_bonds(L, d, 7000 * L + k)
        ref = oracle.label(b)
        for sub in subs:
            for bits in (32, 64):
                got, (it1, it2) = _two_stage(b, sub, bits)
                assert np.array_equal(got, ref), (L, d, sub, bits)
                assert it1 >= 1 and it2 >= 1


def test_two_stage_matches_tile_union_find_on_equilibrium_bonds():
    import torch
    L, q = 2048, 2
    with sw.Sim(L, q, sw.tc(q), 13, store_bonds=True) as s:
        s.sweep(40)
        packed = torch.from_numpy(s.bonds().reshape(-1).copy()).cuda()
    a = torch.empty(L * L, dtype=torch.int32, device="cuda")
    sw.label_bonds(L, packed, a, label_bits=32)
    for sub in (256, 512, 2048):
        b = torch.full((L * L,), -7, dtype=torch.int32, device="cuda")
        it1, it2, ms = sw.label_bonds_2stage(L, sub, packed, b, label_bits=32, timings=True)
        torch.cuda.synchronize()
        assert torch.equal(a, b), sub
        assert 2 <= it1 <= 64 and 1 <= it2 <= 64
        assert len(ms) == 3 and ms[0] > 0 and ms[1] > 0 and ms[2] >= 0
