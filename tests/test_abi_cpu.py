"""CPU checks of the C-ABI library: it builds, loads without a GPU and
exports every entry point include/sw.h declares; host-only helpers."""
import os
import re
import subprocess

import numpy as np

import oracle
import paper_1208_2080_gb300 as sw

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "sw.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = set(re.findall(r"\b(sw_[a-z_0-9]+)\s*\(", txt))
    return names - {"sw_alloc_fn", "sw_free_fn"}


def test_library_exports_every_declared_symbol():
    from paper_1208_2080_gb300 import build
    path = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                         check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    declared = _declared()
    assert declared, "no declarations parsed"
    missing = declared - exported
    assert not missing, missing
    assert declared == set(sw.EXPORTS) | (declared - set(sw.EXPORTS))
    lib = sw.lib()
    for name in declared:
        getattr(lib, name)


def test_threshold_matches_oracle_and_errors():
    for T in [0.01, 0.5, 1.0, sw.tc(2), sw.tc(3), 3.7, 1e9]:
        assert sw.threshold(T) == oracle.threshold(T)
    for bad in [0.0, -1.0, float("inf"), float("nan")]:
        try:
            sw.threshold(bad)
        except sw.SwError as e:
            assert e.code == -1
        else:
            raise AssertionError("accepted bad T")


def test_strerror_names_every_code():
    for c in range(-7, 1):
        assert sw.strerror(c) != "unknown error"


def test_bond_packing_roundtrip():
    rng = np.random.default_rng(0)
    for L in [2, 3, 5, 8, 13]:
        b = rng.integers(0, 4, size=(L, L)).astype(np.uint8)
        assert np.array_equal(sw.unpack_bonds(sw.pack_bonds(b), L), b)


def test_two_stage_labeller_rejects_bad_sub_lattices_before_device_work():
    import ctypes
    f = sw.lib().sw_label_bonds_2stage
    p = ctypes.c_void_p(16)  # never dereferenced: every call below fails argument checks
    for L, sub, bits in [(12, 5, 32), (12, 1, 32), (12, 24, 32), (1, 1, 32), (12, 6, 16),
                         (1 << 21, 1 << 20, 64), (1 << 17, 1 << 16, 32)]:
        assert f(L, sub, p, p, bits, None, None, None) == -1, (L, sub, bits)


def test_xy_thresholds_match_the_oracle_table():
    """The library's host-side XY bond table equals the oracle's, entry for
    entry (same formula, same libm), for every M class and a range of T."""
    for M in (2, 3, 4, 7, 64, 255, 256):
        for T in (0.3, sw.T_KT, 1.7, 40.0):
            assert np.array_equal(sw.xy_thresholds(M, T), oracle.xy_thresholds(M, T)), (M, T)
    import ctypes
    f = sw.lib().sw_xy_thresholds
    out = (ctypes.c_uint32 * 4)()
    for M, T in [(1, 1.0), (257, 1.0), (8, 0.0), (8, -1.0), (8, float("nan"))]:
        assert f(M, T, out) == -1
