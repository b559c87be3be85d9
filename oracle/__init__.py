"""CPU oracle for the Swendsen-Wang sweep of the 2D q-state Potts model.

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
bench's ``cpu_baseline`` / ``--impl reference`` legs may import this package.
It wraps the plain C oracle in ``sw_oracle.c`` (conventions in
``sw_oracle.h``) with numpy arrays; it shares no code with the CUDA path.

Every function follows Sec. 2 of Komura & Okabe (Eq. 1 and the three SW
steps); measurement follows Sec. 4 (Table 1, update plus measurement).

The ``wolff_*`` functions wrap ``wolff_oracle.c``: the Wolff single-cluster
update of the related work (Sec. 1), pinned in tests/test_oracle_wolff.py.
The ``xy_*`` functions wrap ``xy_oracle.c``: the embedded-cluster sweep of
the XY model with M angles that Sec. 5 names as the extension (Wolff's
embedding), pinned in tests/test_oracle_xy.py.

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
        L.orc_philox_many.argtypes = [ctypes.c_uint64, u32p, u32p]
        L.orc_philox_many.restype = None
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
        L.orc_xy_axis.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32]
        L.orc_xy_axis.restype = ctypes.c_uint32
        L.orc_xy_thresholds.argtypes = [ctypes.c_uint32, ctypes.c_double, u32p]
        L.orc_xy_thresholds.restype = None
        L.orc_xy_bonds.argtypes = [ctypes.c_uint64, ctypes.c_uint32, u8p, u32p, ctypes.c_uint32,
                                   ctypes.c_uint64, ctypes.c_uint32, u8p]
        L.orc_xy_bonds.restype = None
        L.orc_xy_flip.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64,
                                  ctypes.c_uint32, u32p, u8p]
        L.orc_xy_flip.restype = None
        L.orc_xy_measure.argtypes = [ctypes.c_uint64, ctypes.c_uint32, u8p, u64p, u64p]
        L.orc_xy_measure.restype = None
        L.orc_xy_run.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double, ctypes.c_uint64,
                                 u8p, ctypes.c_uint32, ctypes.c_uint32, u64p, u64p]
        L.orc_xy_run.restype = ctypes.c_int
        L.orc_wolff_seed.argtypes = [ctypes.c_uint64, ctypes.c_uint32, u8p, ctypes.c_uint64,
                                     ctypes.c_uint32, u64p, u32p]
        L.orc_wolff_seed.restype = None
        L.orc_wolff_step.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                     ctypes.c_uint64, ctypes.c_uint32, u8p]
        L.orc_wolff_step.restype = ctypes.c_uint64
        L.orc_wolff_run.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double,
                                    ctypes.c_uint64, u8p, ctypes.c_uint32, ctypes.c_uint32, u64p]
        L.orc_wolff_run.restype = ctypes.c_int
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


def philox_many(inp):
    """Philox4x32-10 of every row of an (n, 6) uint32 array (counter words,
    then key words) -> (n, 4) uint32, one oracle call per row."""
    a = np.ascontiguousarray(np.asarray(inp, dtype=np.uint32).reshape(-1, 6))
    out = np.zeros((a.shape[0], 4), dtype=np.uint32)
    lib().orc_philox_many(a.shape[0], _p(a, ctypes.c_uint32), _p(out, ctypes.c_uint32))
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


# ---------------------------------------------------------------- XY model
# Embedded-cluster SW sweep of the 2D XY model with M angles (Sec. 5 of the
# paper; Wolff's embedding).  Conventions in xy_oracle.h.

def xy_axis(seed, sweep, M):
    """Axis index j of a sweep: r at angle pi j/M - pi/2, reflection k -> (j-k) mod M."""
    return int(lib().orc_xy_axis(int(seed), int(sweep), int(M)))


def xy_thresholds(M, T):
    """(M//2+1, M//2+1) table floor((1 - exp(-2 sin(pi c/M) sin(pi d/M)/T)) 2^32)."""
    H = M // 2
    tt = np.zeros((H + 1) * (H + 1), dtype=np.uint32)
    lib().orc_xy_thresholds(int(M), float(T), _p(tt, ctypes.c_uint32))
    return tt.reshape(H + 1, H + 1)


def xy_bonds(spins, M, T, seed, sweep, j=None):
    """Step (1) of the embedded sweep: bond bits (bit0 right, bit1 down)."""
    s = np.ascontiguousarray(spins, dtype=np.uint8)
    L = s.shape[0]
    tt = np.ascontiguousarray(xy_thresholds(M, T).reshape(-1))
    jj = xy_axis(seed, sweep, M) if j is None else int(j)
    b = np.zeros(L * L, dtype=np.uint8)
    lib().orc_xy_bonds(L, M, _p(s, ctypes.c_uint8), _p(tt, ctypes.c_uint32), jj, seed, sweep,
                       _p(b, ctypes.c_uint8))
    return b.reshape(L, L)


def xy_flip(spins, root, M, seed, sweep, j=None):
    """Step (3): clusters reflected k -> (j-k) mod M by their root's coin."""
    s = np.array(spins, dtype=np.uint8, copy=True, order="C")
    r = np.ascontiguousarray(root, dtype=np.uint32)
    L = s.shape[0]
    jj = xy_axis(seed, sweep, M) if j is None else int(j)
    lib().orc_xy_flip(L, M, jj, seed, sweep, _p(r, ctypes.c_uint32), _p(s, ctypes.c_uint8))
    return s


def xy_measure(spins, M):
    """(D[0..M//2], n[0..M-1]) of a configuration."""
    s = np.ascontiguousarray(spins, dtype=np.uint8)
    L = s.shape[0]
    D = np.zeros(M // 2 + 1, dtype=np.uint64)
    n = np.zeros(M, dtype=np.uint64)
    lib().orc_xy_measure(L, M, _p(s, ctypes.c_uint8), _p(D, ctypes.c_uint64),
                         _p(n, ctypes.c_uint64))
    return D, n


def xy_init(L, M, seed):
    """Initial angles from the init stream (the Potts init with q = M)."""
    return init_spins(L, M, seed)


def xy_run(L, M, T, seed, nsweeps, spins=None, sweep0=0, series=True):
    """Run nsweeps embedded-cluster sweeps.  Returns (spins, D_series,
    n_series), entry k being the configuration after sweep sweep0+k."""
    s = xy_init(L, M, seed).reshape(-1).copy() if spins is None else \
        np.array(spins, dtype=np.uint8, copy=True).reshape(-1)
    H = M // 2
    D = np.zeros((max(nsweeps, 1), H + 1), dtype=np.uint64) if series else None
    n = np.zeros((max(nsweeps, 1), M), dtype=np.uint64) if series else None
    rc = lib().orc_xy_run(L, M, float(T), seed, _p(s, ctypes.c_uint8), sweep0, nsweeps,
                          _p(D, ctypes.c_uint64) if series else None,
                          _p(n, ctypes.c_uint64) if series else None)
    if rc != 0:
        raise ValueError(f"orc_xy_run failed ({rc})")
    if series:
        return s.reshape(L, L), D[:nsweeps], n[:nsweeps]
    return s.reshape(L, L), None, None


def xy_energy(D, M):
    """E = -sum_d D[d] cos(2 pi d / M) (J = 1), per configuration."""
    D = np.asarray(D, dtype=np.float64)
    return -(D * np.cos(2 * np.pi * np.arange(M // 2 + 1) / M)).sum(-1)


def xy_magnetisation(n, M):
    """(m_x, m_y) = sum_k n[k] (cos, sin)(2 pi k / M), per configuration."""
    n = np.asarray(n, dtype=np.float64)
    a = 2 * np.pi * np.arange(M) / M
    return (n * np.cos(a)).sum(-1), (n * np.sin(a)).sum(-1)


# ---------------------------------------------------------------- Wolff
# Single-cluster update of the q-state Potts model (related work, Sec. 1).
# Conventions in wolff_oracle.h.

def wolff_seed(spins, q, seed, t):
    """(i0, s_new) of step t."""
    s = np.ascontiguousarray(spins, dtype=np.uint8)
    L = s.shape[0]
    i0 = ctypes.c_uint64()
    sn = ctypes.c_uint32()
    lib().orc_wolff_seed(L, q, _p(s, ctypes.c_uint8), seed, t, ctypes.byref(i0), ctypes.byref(sn))
    return int(i0.value), int(sn.value)


def wolff_step(spins, q, T, seed, t):
    """One step on a copy of spins; returns (new spins, cluster size)."""
    s = np.array(spins, dtype=np.uint8, copy=True, order="C")
    L = s.shape[0]
    c = lib().orc_wolff_step(L, q, threshold(T), seed, t, _p(s, ctypes.c_uint8))
    return s, int(c)


def wolff_run(L, q, T, seed, nsteps, spins=None, t0=0):
    """nsteps Wolff steps from spins (default: the init stream); returns
    (spins, cluster sizes)."""
    s = init_spins(L, q, seed).reshape(-1).copy() if spins is None else \
        np.array(spins, dtype=np.uint8, copy=True).reshape(-1)
    sizes = np.zeros(max(nsteps, 1), dtype=np.uint64)
    rc = lib().orc_wolff_run(L, q, float(T), seed, _p(s, ctypes.c_uint8), t0, nsteps,
                             _p(sizes, ctypes.c_uint64))
    if rc != 0:
        raise ValueError(f"orc_wolff_run failed ({rc})")
    return s.reshape(L, L), sizes[:nsteps]
