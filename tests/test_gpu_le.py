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
