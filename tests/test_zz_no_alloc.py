"""The allocation-free labelling entry point, sw_label_bonds_static, for
callers that cannot allocate device memory (their GPU memory belongs to a
framework pool, or cudaMalloc/cudaFree would stall a running program).  Its
roots must equal those of the allocating sw_label_bonds on the same bond
lattices, call after call, since every call reuses one fixed device array.
Kept in the last-collected file so a stop-at-first-failure run has already
run every other test."""
import ctypes

import numpy as np
import pytest

import paper_1208_2080_gb300 as sw
import synth

pytestmark = pytest.mark.gpu


def _call_static(L, packed, roots, tile_h=0):
    import torch
    return sw.lib().sw_label_bonds_static(
        int(L), ctypes.c_void_p(packed.data_ptr()), ctypes.c_void_p(roots.data_ptr()), int(tile_h),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_static_labelling_matches_allocating_entry_point_twice():
    import torch
    # calls in a row on the one shared array: different sizes, the largest
    # layouts it holds (L = 1024 with 16- and 32-row tiles), an odd L (rows
    # not 4-byte aligned), and the same L again with another bond lattice
    cases = [(1024, 0.58, 7, 0), (300, 0.5, 8, 16), (1024, 0.5, 9, 16), (1024, 0.52, 10, 32),
             (1023, 0.55, 11, 0), (1023, 0.2, 12, 0)]
    for L, density, seed, th in cases:
        b = synth.random_bonds(L, density, seed)
        packed = torch.from_numpy(sw.pack_bonds(b).reshape(-1).copy()).cuda()
        ref = torch.empty(L * L, dtype=torch.int32, device="cuda")
        sw.label_bonds(L, packed, ref, label_bits=32, tile_h=th)
        got = torch.full((L * L,), -1, dtype=torch.int32, device="cuda")
        rc = _call_static(L, packed, got, th)
        assert rc == 0, sw.strerror(rc)
        torch.cuda.synchronize()
        assert torch.equal(got, ref), (L, th)


def test_static_labelling_rejects_lattices_beyond_its_array():
    import torch
    L = sw._binding.LABEL_STATIC_MAX_L + 1
    packed = torch.zeros(L * ((L + 3) // 4), dtype=torch.uint8, device="cuda")
    roots = torch.zeros(L * L, dtype=torch.int32, device="cuda")
    assert _call_static(L, packed, roots) == sw._binding.SW_ERR_INVAL
