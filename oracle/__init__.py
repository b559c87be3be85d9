"""CPU oracle for the Swendsen-Wang sweep of the 2D q-state Potts model.

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
bench's ``cpu_baseline`` / ``--impl reference`` legs may import this package.
It wraps the plain C oracle in ``sw_oracle.c`` (conventions in
``sw_oracle.h``) with numpy arrays; it shares no code with the CUDA path.

Every function follows Sec. 2 of Komura & Okabe (Eq. 1 and the three SW
steps); measurement follows Sec. 4 (Table 1, "update + measurement").

Pins (tests/test_oracle_*.py): Philox known-answer vectors and an
independent Philox implementation, BFS labelling, exact SW transition
matrices (stationarity + detailed balance), brute-force and transfer-matrix
partition functions, Onsager / Baxter closed forms.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.orc_philox4x32_10.restype = None
        L.orc_threshold.argtypes = [ctypes.c_double]
        L.orc_threshold.restype = ctypes.c_uint32
        L.orc_pick.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
        L.orc_pick.restype = ctypes.c_uint32
        L.orc_init_spins.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, u8p]
        L.orc_init_spins.restype = None
        L.orc_bonds.argtypes = [ctypes.c_uint64, u8p, ctypes.c_uint32, ctypes.c_uint64,
                                ctypes.c_uint32, u8p]
        L.orc_bonds.restype = None
        L.orc_label.argtypes = [ctypes.c_uint64, u8p, u32p]
        L.orc_label.restype = ctypes.c_int
        L.orc_recolor.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64,
                                  ctypes.c_uint32, u32p, u8p]
        L.orc_recolor.restype = None
        L.orc_measure.argtypes = [ctypes.c_uint64, ctypes.c_uint32, u8p, u64p, u64p]
        L.orc_measure.restype = None
        L.orc_run.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double,
                              ctypes.c_uint64, u8p, ctypes.c_uint32, ctypes.c_uint32,
                              u64p, u64p]
        L.orc_run.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


RIGHT = 1
DOWN = 2


def philox(ctr, key):
    """Philox4x32-10(key, ctr) -> 4 uint32 words (Salmon et al., SC'11)."""
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(4))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(2))
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c, ctypes.c_uint32), _p(k, ctypes.c_uint32),
                            _p(out, ctypes.c_uint32))
    return out


def threshold(T):
    """floor((1 - exp(-1/T)) * 2^32), clamped to 2^32-1."""
    return int(lib().orc_threshold(float(T)))


def pick(w, q):
    """State floor(w*q/2^32) chosen by the 32-bit word w."""
    return int(lib().orc_pick(int(w), int(q)))


def init_spins(L, q, seed):
    """Initial configuration drawn from the init stream (uint8, L x L)."""
    s = np.zeros(L * L, dtype=np.uint8)
    lib().orc_init_spins(L, q, seed, _p(s, ctypes.c_uint8))
    return s.reshape(L, L)


def bonds(spins, T_or_thr, seed, sweep, *, thr=None):
    """Sec. 2 step (1): per-site bond bits (bit0 right, bit1 down), L x L uint8."""
    s = np.ascontiguousarray(spins, dtype=np.uint8)
    L = s.shape[0]
    t = thr if thr is not None else threshold(T_or_thr)
    b = np.zeros(L * L, dtype=np.uint8)
    lib().orc_bonds(L, _p(s, ctypes.c_uint8), t, seed, sweep, _p(b, ctypes.c_uint8))
    return b.reshape(L, L)


def label(b):
    """Sec. 2 step (2): HK labelling; returns root (min site index) per site."""
    bb = np.ascontiguousarray(b, dtype=np.uint8)
    L = bb.shape[0]
    root = np.zeros(L * L, dtype=np.uint32)
    rc = lib().orc_label(L, _p(bb, ctypes.c_uint8), _p(root, ctypes.c_uint32))
    if rc != 0:
        raise ValueError("orc_label: bad L")
    return root.reshape(L, L)


def recolor(spins, root, q, seed, sweep):
    """Sec. 2 step (3): new state per cluster; returns the new spins."""
    s = np.array(spins, dtype=np.uint8, copy=True, order="C")
    r = np.ascontiguousarray(root, dtype=np.uint32)
    L = s.shape[0]
    lib().orc_recolor(L, q, seed, sweep, _p(r, ctypes.c_uint32), _p(s, ctypes.c_uint8))
    return s


def measure(spins, q):
    """Sec. 4: (E_sat, n[q]) of a configuration."""
    s = np.ascontiguousarray(spins, dtype=np.uint8)
    L = s.shape[0]
    E = np.zeros(1, dtype=np.uint64)
    n = np.zeros(q, dtype=np.uint64)
    lib().orc_measure(L, q, _p(s, ctypes.c_uint8), _p(E, ctypes.c_uint64),
                      _p(n, ctypes.c_uint64))
    return int(E[0]), n


def run(L, q, T, seed, nsweeps, spins=None, sweep0=0, series=True):
    """Run nsweeps SW sweeps.  Returns (spins, E_series, n_series) where entry k
    is the configuration after sweep sweep0+k.  spins=None starts from the
    init stream."""
    s = init_spins(L, q, seed).reshape(-1).copy() if spins is None else \
        np.array(spins, dtype=np.uint8, copy=True).reshape(-1)
    E = np.zeros(max(nsweeps, 1), dtype=np.uint64) if series else None
    n = np.zeros((max(nsweeps, 1), q), dtype=np.uint64) if series else None
    rc = lib().orc_run(L, q, float(T), seed, _p(s, ctypes.c_uint8), sweep0, nsweeps,
                       _p(E, ctypes.c_uint64) if series else None,
                       _p(n, ctypes.c_uint64) if series else None)
    if rc != 0:
        raise ValueError(f"orc_run failed ({rc})")
    if series:
        return s.reshape(L, L), E[:nsweeps], n[:nsweeps]
    return s.reshape(L, L), None, None


def tc(q):
    """Critical temperature of the 2D q-state Potts model, T_c = 1/ln(1+sqrt q)
    (Sec. 4 quotes T_c = 1.1346 for q = 2)."""
    return 1.0 / np.log1p(np.sqrt(q))
