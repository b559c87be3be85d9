"""ctypes binding of libswgb.so, the C ABI declared in include/sw.h.

Argument marshalling only: every step of a sweep runs in the library's CUDA
kernels.  PyTorch is used for device memory (its caching allocator is
installed as the library's allocator) and streams.  There is no CPU
fallback: if the library is missing or cannot be loaded, every entry point
raises.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libswgb.so")

SW_OK = 0
SW_ERR_INVAL = -1
SW_ERR_NOMEM = -2
SW_ERR_CUDA = -3
SW_ERR_TIMEOUT = -4
SW_ERR_STATE = -5
SW_ERR_DEVICE = -6
SW_ERR_RANGE = -7
SW_INIT_RANDOM = 0
SW_INIT_ZERO = 1

# every symbol include/sw.h declares (checked by the CPU tests)
EXPORTS = [
    "sw_set_allocator", "sw_create", "sw_create_ex", "sw_destroy", "sw_bind_stream", "sw_sweep",
    "sw_measure", "sw_series", "sw_spins", "sw_set_spins", "sw_bonds", "sw_get_sweep",
    "sw_set_sweep", "sw_sync", "sw_info", "sw_threshold", "sw_label_bonds", "sw_strerror",
    "sw_last_error", "sw_profile", "sw_profile_read", "sw_sweep_host",
    "sw_batch_create", "sw_batch_create_ex", "sw_batch_destroy", "sw_batch_bind_stream",
    "sw_batch_sweep", "sw_batch_measure", "sw_batch_series", "sw_batch_spins",
    "sw_batch_set_spins", "sw_batch_get_sweep", "sw_batch_sync", "sw_batch_info",
    "sw_batch_profile", "sw_batch_profile_read", "sw_batch_last_error", "sw_label_bonds_static",
    "sw_mlp_create", "sw_mlp_destroy", "sw_mlp_bind_stream", "sw_mlp_forward", "sw_mlp_gradients",
    "sw_mlp_train_step", "sw_mlp_get_params", "sw_mlp_set_params", "sw_label_bonds_le",
    "sw_label_bonds_2stage", "sw_mlp_predict",
    "sw_xy_thresholds", "sw_xy_create", "sw_xy_destroy", "sw_xy_bind_stream", "sw_xy_sweep",
    "sw_xy_sync", "sw_xy_series", "sw_xy_spins", "sw_xy_set_spins", "sw_xy_get_sweep",
    "sw_xy_profile", "sw_xy_profile_read", "sw_xy_last_error",
    "sw_wolff_create", "sw_wolff_destroy", "sw_wolff_bind_stream", "sw_wolff_step", "sw_wolff_sync",
    "sw_wolff_sizes", "sw_wolff_spins", "sw_wolff_set_spins", "sw_wolff_get_step", "sw_wolff_set_mode",
    "sw_wolff_set_wait_limit",
]


class SwError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})")


class sw_obs(ctypes.Structure):
    _fields_ = [("config", ctypes.c_uint64), ("E_sat", ctypes.c_uint64), ("q", ctypes.c_uint32),
                ("pad_", ctypes.c_uint32), ("n", ctypes.c_uint64 * 256)]


# boundary-union schedules (include/sw.h SW_MERGE_*): "kernel" -- a kernel
# of its own after the labelling; "fused" -- the labelling does it
MERGE = {"auto": 0, "kernel": 1, "fused": 2}
MERGE_NAMES = {1: "kernel", 2: "fused"}


class sw_params(ctypes.Structure):
    _fields_ = [("L", ctypes.c_uint64), ("q", ctypes.c_uint32), ("label_bits", ctypes.c_uint32),
                ("T", ctypes.c_double), ("seed", ctypes.c_uint64), ("tile_h", ctypes.c_uint32),
                ("ring", ctypes.c_uint32), ("init", ctypes.c_uint32),
                ("store_bonds", ctypes.c_uint32), ("measure", ctypes.c_uint32),
                ("walk_cap", ctypes.c_uint32), ("merge", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32 * 1)]


class sw_xy_params(ctypes.Structure):
    _fields_ = [("L", ctypes.c_uint64), ("M", ctypes.c_uint32), ("label_bits", ctypes.c_uint32),
                ("T", ctypes.c_double), ("seed", ctypes.c_uint64), ("tile_h", ctypes.c_uint32),
                ("ring", ctypes.c_uint32), ("init", ctypes.c_uint32), ("measure", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32 * 4)]


class sw_info_t(ctypes.Structure):
    _fields_ = [("L", ctypes.c_uint64), ("q", ctypes.c_uint32), ("thr", ctypes.c_uint32),
                ("label_bits", ctypes.c_uint32), ("tile_w", ctypes.c_uint32),
                ("tile_h", ctypes.c_uint32), ("ring", ctypes.c_uint32),
                ("device_bytes", ctypes.c_uint64), ("tiles", ctypes.c_uint64),
                ("merge", ctypes.c_uint32), ("pad_", ctypes.c_uint32)]


class sw_batch_params(ctypes.Structure):
    _fields_ = [("R", ctypes.c_uint32), ("tile_h", ctypes.c_uint32),
                ("L", ctypes.POINTER(ctypes.c_uint64)), ("q", ctypes.POINTER(ctypes.c_uint32)),
                ("T", ctypes.POINTER(ctypes.c_double)), ("seed", ctypes.POINTER(ctypes.c_uint64)),
                ("ring", ctypes.c_uint32), ("init", ctypes.c_uint32), ("measure", ctypes.c_uint32),
                ("graph", ctypes.c_uint32), ("merge", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32 * 3)]


class sw_batch_info_t(ctypes.Structure):
    _fields_ = [("R", ctypes.c_uint32), ("tile_h", ctypes.c_uint32), ("tiles", ctypes.c_uint64),
                ("sites", ctypes.c_uint64), ("device_bytes", ctypes.c_uint64),
                ("label_bits", ctypes.c_uint32), ("graph", ctypes.c_uint32),
                ("merge", ctypes.c_uint32), ("pad_", ctypes.c_uint32)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)

_lib = None
_alloc_keep = None
_allocator_chosen = False


def lib():
    """The loaded library (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libswgb.so not built ({LIB_PATH}); run __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, u64, u32, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
    u64p = ctypes.POINTER(ctypes.c_uint64)
    sig = {
        "sw_set_allocator": (i32, [ALLOC_FN, FREE_FN, vp]),
        "sw_create": (i32, [u64, u32, ctypes.c_double, u64, ctypes.POINTER(vp)]),
        "sw_create_ex": (i32, [ctypes.POINTER(sw_params), ctypes.POINTER(vp)]),
        "sw_destroy": (None, [vp]),
        "sw_bind_stream": (i32, [vp, vp]),
        "sw_sweep": (i32, [vp, u64]),
        "sw_measure": (i32, [vp, ctypes.POINTER(sw_obs)]),
        "sw_series": (i32, [vp, u64, u64, u64p, u64p]),
        "sw_spins": (i32, [vp, vp, u64, i32]),
        "sw_set_spins": (i32, [vp, vp, u64, i32]),
        "sw_bonds": (i32, [vp, vp, u64, i32]),
        "sw_get_sweep": (i32, [vp, u64p]),
        "sw_set_sweep": (i32, [vp, u64]),
        "sw_sync": (i32, [vp]),
        "sw_sweep_host": (i32, [vp, vp, u64, u64, ctypes.POINTER(sw_obs)]),
        "sw_info": (i32, [vp, ctypes.POINTER(sw_info_t)]),
        "sw_threshold": (i32, [ctypes.c_double, ctypes.POINTER(ctypes.c_uint32)]),
        "sw_label_bonds": (i32, [u64, vp, vp, u32, u32, vp]),
        "sw_strerror": (ctypes.c_char_p, [i32]),
        "sw_last_error": (i32, [vp]),
        "sw_profile": (i32, [vp, i32]),
        "sw_profile_read": (i32, [vp, ctypes.POINTER(ctypes.c_double), u64p, i32]),
        "sw_batch_create": (i32, [u32, u64p, ctypes.POINTER(ctypes.c_uint32),
                                  ctypes.POINTER(ctypes.c_double), u64p, ctypes.POINTER(vp)]),
        "sw_batch_create_ex": (i32, [ctypes.POINTER(sw_batch_params), ctypes.POINTER(vp)]),
        "sw_batch_destroy": (None, [vp]),
        "sw_batch_bind_stream": (i32, [vp, vp]),
        "sw_batch_sweep": (i32, [vp, u64]),
        "sw_batch_measure": (i32, [vp, u32, ctypes.POINTER(sw_obs)]),
        "sw_batch_series": (i32, [vp, u32, u64, u64, u64p, u64p]),
        "sw_batch_spins": (i32, [vp, u32, vp, u64, i32]),
        "sw_batch_set_spins": (i32, [vp, u32, vp, u64, i32]),
        "sw_batch_get_sweep": (i32, [vp, u64p]),
        "sw_batch_sync": (i32, [vp]),
        "sw_batch_info": (i32, [vp, ctypes.POINTER(sw_batch_info_t)]),
        "sw_batch_profile": (i32, [vp, i32]),
        "sw_batch_profile_read": (i32, [vp, ctypes.POINTER(ctypes.c_double), u64p, i32]),
        "sw_batch_last_error": (i32, [vp]),
        "sw_label_bonds_static": (i32, [u64, vp, vp, u32, vp]),
        "sw_mlp_create": (i32, [vp, ctypes.POINTER(vp)]),
        "sw_mlp_destroy": (None, [vp]),
        "sw_mlp_bind_stream": (i32, [vp, vp]),
        "sw_mlp_forward": (i32, [vp, vp, u32, vp]),
        "sw_mlp_predict": (i32, [vp, vp, u32, vp]),
        "sw_mlp_gradients": (i32, [vp, vp, vp, vp, u32, vp, vp]),
        "sw_mlp_train_step": (i32, [vp, vp, vp, vp, u32, ctypes.c_float, vp]),
        "sw_mlp_get_params": (i32, [vp, vp, vp]),
        "sw_mlp_set_params": (i32, [vp, vp]),
        "sw_label_bonds_le": (i32, [u64, vp, vp, u32, u32, ctypes.POINTER(ctypes.c_uint32), vp]),
        "sw_xy_thresholds": (i32, [u32, ctypes.c_double, ctypes.POINTER(ctypes.c_uint32)]),
        "sw_xy_create": (i32, [ctypes.POINTER(sw_xy_params), ctypes.POINTER(vp)]),
        "sw_xy_destroy": (None, [vp]),
        "sw_xy_bind_stream": (i32, [vp, vp]),
        "sw_xy_sweep": (i32, [vp, u64]),
        "sw_xy_sync": (i32, [vp]),
        "sw_xy_series": (i32, [vp, u64, u64, u64p, u64p]),
        "sw_xy_spins": (i32, [vp, vp, u64, i32]),
        "sw_xy_set_spins": (i32, [vp, vp, u64, i32]),
        "sw_xy_get_sweep": (i32, [vp, u64p]),
        "sw_xy_profile": (i32, [vp, i32]),
        "sw_xy_profile_read": (i32, [vp, ctypes.POINTER(ctypes.c_double), u64p, i32]),
        "sw_xy_last_error": (i32, [vp]),
        "sw_wolff_create": (i32, [u64, u32, ctypes.c_double, u64, u32, u32, ctypes.POINTER(vp)]),
        "sw_wolff_destroy": (None, [vp]),
        "sw_wolff_bind_stream": (i32, [vp, vp]),
        "sw_wolff_step": (i32, [vp, u64]),
        "sw_wolff_sync": (i32, [vp]),
        "sw_wolff_sizes": (i32, [vp, u64, u64, u64p]),
        "sw_wolff_spins": (i32, [vp, vp, u64, i32]),
        "sw_wolff_set_spins": (i32, [vp, vp, u64, i32]),
        "sw_wolff_get_step": (i32, [vp, u64p]),
        "sw_wolff_set_mode": (i32, [vp, i32]),
        "sw_wolff_set_wait_limit": (i32, [vp, u32]),
        "sw_label_bonds_2stage": (i32, [u64, u64, vp, vp, u32, ctypes.POINTER(ctypes.c_uint32),
                                        ctypes.POINTER(ctypes.c_float), vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def strerror(code):
    try:
        return lib().sw_strerror(int(code)).decode()
    except Exception:  # pragma: no cover
        return "error"


def check(rc, what):
    if rc != SW_OK:
        raise SwError(rc, what)


def use_torch_allocator():
    """Route the library's device allocations through PyTorch's caching
    allocator (affects handles created afterwards).  Done automatically by
    the first ``Sim`` unless ``use_cuda_malloc()`` was called before."""
    global _alloc_keep, _allocator_chosen
    _allocator_chosen = True
    import torch

    def _alloc(nbytes, _ctx):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes)))
        except Exception:
            return None

    def _free(ptr, _nbytes, _ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    a, f = ALLOC_FN(_alloc), FREE_FN(_free)
    check(lib().sw_set_allocator(a, f, None), "sw_set_allocator")
    _alloc_keep = (a, f)


def use_cuda_malloc():
    """Let the library call cudaMalloc / cudaFree itself."""
    global _alloc_keep, _allocator_chosen
    _allocator_chosen = True
    check(lib().sw_set_allocator(ALLOC_FN(), FREE_FN(), None), "sw_set_allocator")
    _alloc_keep = None


def threshold(T):
    out = ctypes.c_uint32()
    check(lib().sw_threshold(float(T), ctypes.byref(out)), "sw_threshold")
    return int(out.value)


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class Sim:
    """One L x L lattice on the GPU (include/sw.h handle)."""

    def __init__(self, L, q, T, seed, *, label_bits=0, tile_h=0, ring=0, init="random",
                 store_bonds=False, measure=True, walk_cap=0, merge="auto", stream=None):
        if not _allocator_chosen:
            use_torch_allocator()
        p = sw_params()
        p.L, p.q, p.T, p.seed = int(L), int(q), float(T), int(seed)
        p.label_bits, p.tile_h, p.ring = int(label_bits), int(tile_h), int(ring)
        p.init = SW_INIT_ZERO if init == "zero" else SW_INIT_RANDOM
        p.store_bonds = 1 if store_bonds else 0
        p.measure = 0 if measure else 2
        p.walk_cap = int(walk_cap)
        p.merge = MERGE[merge]
        h = ctypes.c_void_p()
        self._h = None
        check(lib().sw_create_ex(ctypes.byref(p), ctypes.byref(h)), "sw_create_ex")
        self._h = h
        self.L, self.q, self.T, self.seed = int(L), int(q), float(T), int(seed)
        self.N = self.L * self.L
        if stream is not False:
            self.bind_stream(stream)

    def close(self):
        if self._h is not None:
            lib().sw_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def bind_stream(self, stream=None):
        check(lib().sw_bind_stream(self._h, _stream_handle(stream)), "sw_bind_stream")

    def sweep(self, n=1):
        check(lib().sw_sweep(self._h, int(n)), "sw_sweep")

    def sync(self):
        check(lib().sw_sync(self._h), "sw_sync")

    def measure(self):
        o = sw_obs()
        check(lib().sw_measure(self._h, ctypes.byref(o)), "sw_measure")
        return int(o.E_sat), np.array(o.n[: self.q], dtype=np.uint64), int(o.config)

    def series(self, first, count):
        E = np.zeros(count, dtype=np.uint64)
        n = np.zeros((count, self.q), dtype=np.uint64)
        check(lib().sw_series(self._h, int(first), int(count),
                              E.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                              n.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))), "sw_series")
        return E, n

    def spins(self, out=None):
        """Spins as an (L, L) uint8 numpy array, or into `out` (a CUDA uint8
        torch tensor with L*L elements, filled on the handle's stream)."""
        if out is not None:
            assert out.is_cuda and out.numel() == self.N and out.is_contiguous()
            check(lib().sw_spins(self._h, ctypes.c_void_p(out.data_ptr()), self.N, 1), "sw_spins")
            return out
        a = np.empty(self.N, dtype=np.uint8)
        check(lib().sw_spins(self._h, a.ctypes.data_as(ctypes.c_void_p), self.N, 0), "sw_spins")
        return a.reshape(self.L, self.L)

    def set_spins(self, src):
        """Replace the configuration from a numpy array or a CUDA uint8 tensor."""
        if hasattr(src, "is_cuda") and src.is_cuda:
            assert src.numel() == self.N and src.is_contiguous()
            check(lib().sw_set_spins(self._h, ctypes.c_void_p(src.data_ptr()), self.N, 1),
                  "sw_set_spins")
            return
        a = np.ascontiguousarray(np.asarray(src, dtype=np.uint8).reshape(-1))
        check(lib().sw_set_spins(self._h, a.ctypes.data_as(ctypes.c_void_p), self.N, 0),
              "sw_set_spins")

    def sweep_host(self, src, nsweeps=1):
        """Upload a host configuration (numpy uint8, L*L; page-locked memory
        overlaps the upload with the first sweep), run nsweeps sweeps and
        return (E_sat, n[q], configuration index) of the result."""
        a = np.ascontiguousarray(np.asarray(src, dtype=np.uint8).reshape(-1))
        o = sw_obs()
        check(lib().sw_sweep_host(self._h, a.ctypes.data_as(ctypes.c_void_p), self.N, int(nsweeps),
                                  ctypes.byref(o)), "sw_sweep_host")
        return int(o.E_sat), np.array(o.n[: self.q], dtype=np.uint64), int(o.config)

    def bonds(self):
        bp = (self.L + 3) // 4
        a = np.empty(self.L * bp, dtype=np.uint8)
        check(lib().sw_bonds(self._h, a.ctypes.data_as(ctypes.c_void_p), a.size, 0), "sw_bonds")
        return a.reshape(self.L, bp)

    @property
    def sweep_count(self):
        v = ctypes.c_uint64()
        check(lib().sw_get_sweep(self._h, ctypes.byref(v)), "sw_get_sweep")
        return int(v.value)

    def set_sweep(self, s):
        check(lib().sw_set_sweep(self._h, int(s)), "sw_set_sweep")

    def info(self):
        i = sw_info_t()
        check(lib().sw_info(self._h, ctypes.byref(i)), "sw_info")
        return {k: getattr(i, k) for k, _ in sw_info_t._fields_}

    def profile(self, enable=True):
        check(lib().sw_profile(self._h, 1 if enable else 0), "sw_profile")

    def profile_read(self):
        """(ms[3], launches[3]) per phase: tile labelling, boundary merge, recolour."""
        ms = (ctypes.c_double * 3)()
        n = (ctypes.c_uint64 * 3)()
        check(lib().sw_profile_read(self._h, ms, n, 3), "sw_profile_read")
        return list(ms), list(n)

    @property
    def handle(self):
        return self._h


def xy_thresholds(M, T):
    """The XY bond threshold table (host computation of the library)."""
    H = int(M) // 2
    tt = np.zeros((H + 1) * (H + 1), dtype=np.uint32)
    check(lib().sw_xy_thresholds(int(M), float(T), tt.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))),
          "sw_xy_thresholds")
    return tt.reshape(H + 1, H + 1)


class XY:
    """The XY model with M angles on an L x L lattice, embedded-cluster
    sweeps (include/sw.h, sw_xy_*)."""

    def __init__(self, L, M, T, seed, *, label_bits=0, tile_h=0, ring=0, init="random",
                 measure=True, stream=None):
        if not _allocator_chosen:
            use_torch_allocator()
        p = sw_xy_params()
        p.L, p.M, p.T, p.seed = int(L), int(M), float(T), int(seed)
        p.label_bits, p.tile_h, p.ring = int(label_bits), int(tile_h), int(ring)
        p.init = SW_INIT_ZERO if init == "zero" else SW_INIT_RANDOM
        p.measure = 0 if measure else 2
        h = ctypes.c_void_p()
        self._h = None
        check(lib().sw_xy_create(ctypes.byref(p), ctypes.byref(h)), "sw_xy_create")
        self._h = h
        self.L, self.M, self.T, self.seed = int(L), int(M), float(T), int(seed)
        self.N = self.L * self.L
        if stream is not False:
            self.bind_stream(stream)

    def close(self):
        if self._h is not None:
            lib().sw_xy_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def bind_stream(self, stream=None):
        check(lib().sw_xy_bind_stream(self._h, _stream_handle(stream)), "sw_xy_bind_stream")

    def sweep(self, n=1):
        check(lib().sw_xy_sweep(self._h, int(n)), "sw_xy_sweep")

    def sync(self):
        check(lib().sw_xy_sync(self._h), "sw_xy_sync")

    def series(self, first, count):
        """(D, n): count x (M//2+1) and count x M observables of
        configurations first .. first+count-1."""
        D = np.zeros((count, self.M // 2 + 1), dtype=np.uint64)
        n = np.zeros((count, self.M), dtype=np.uint64)
        check(lib().sw_xy_series(self._h, int(first), int(count),
                                 D.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                 n.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))), "sw_xy_series")
        return D, n

    def measure(self):
        """(D, n, configuration index) of the current configuration."""
        c = self.sweep_count
        D, n = self.series(c, 1)
        return D[0], n[0], c

    def spins(self, out=None):
        if out is not None:
            assert out.is_cuda and out.numel() == self.N and out.is_contiguous()
            check(lib().sw_xy_spins(self._h, ctypes.c_void_p(out.data_ptr()), self.N, 1), "sw_xy_spins")
            return out
        a = np.empty(self.N, dtype=np.uint8)
        check(lib().sw_xy_spins(self._h, a.ctypes.data_as(ctypes.c_void_p), self.N, 0), "sw_xy_spins")
        return a.reshape(self.L, self.L)

    def set_spins(self, src):
        if hasattr(src, "is_cuda") and src.is_cuda:
            assert src.numel() == self.N and src.is_contiguous()
            check(lib().sw_xy_set_spins(self._h, ctypes.c_void_p(src.data_ptr()), self.N, 1),
                  "sw_xy_set_spins")
            return
        a = np.ascontiguousarray(np.asarray(src, dtype=np.uint8).reshape(-1))
        check(lib().sw_xy_set_spins(self._h, a.ctypes.data_as(ctypes.c_void_p), self.N, 0),
              "sw_xy_set_spins")

    @property
    def sweep_count(self):
        v = ctypes.c_uint64()
        check(lib().sw_xy_get_sweep(self._h, ctypes.byref(v)), "sw_xy_get_sweep")
        return int(v.value)

    def profile(self, enable=True):
        check(lib().sw_xy_profile(self._h, 1 if enable else 0), "sw_xy_profile")

    def profile_read(self):
        """(ms[4], launches[4]) per phase: labelling, merge+resolve,
        reflection, measurement."""
        ms = (ctypes.c_double * 4)()
        n = (ctypes.c_uint64 * 4)()
        check(lib().sw_xy_profile_read(self._h, ms, n, 4), "sw_xy_profile_read")
        return list(ms), list(n)

    @property
    def handle(self):
        return self._h


class Wolff:
    """Wolff single-cluster updates of the q-state Potts model on an L x L
    lattice (include/sw.h, sw_wolff_*)."""

    GROW, LABEL = 0, 1

    def __init__(self, L, q, T, seed, *, init="random", ring=0, mode="label", stream=None):
        if not _allocator_chosen:
            use_torch_allocator()
        h = ctypes.c_void_p()
        self._h = None
        check(lib().sw_wolff_create(int(L), int(q), float(T), int(seed),
                                    SW_INIT_ZERO if init == "zero" else SW_INIT_RANDOM, int(ring),
                                    ctypes.byref(h)), "sw_wolff_create")
        self._h = h
        self.L, self.q, self.T, self.seed = int(L), int(q), float(T), int(seed)
        self.N = self.L * self.L
        if stream is not False:
            self.bind_stream(stream)
        self.set_mode(mode)

    def set_wait_limit(self, idle_polls):
        """Idle polls of a growth warp before it gives up (0: the default)."""
        check(lib().sw_wolff_set_wait_limit(self._h, int(idle_polls)), "sw_wolff_set_wait_limit")

    def set_mode(self, mode):
        """"grow" (cluster grown from a site queue) or "label" (whole-lattice
        labelling of the step's bonds); both give the same clusters."""
        check(lib().sw_wolff_set_mode(self._h, self.LABEL if mode == "label" else self.GROW),
              "sw_wolff_set_mode")

    def close(self):
        if self._h is not None:
            lib().sw_wolff_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def bind_stream(self, stream=None):
        check(lib().sw_wolff_bind_stream(self._h, _stream_handle(stream)), "sw_wolff_bind_stream")

    def step(self, n=1):
        check(lib().sw_wolff_step(self._h, int(n)), "sw_wolff_step")

    def sync(self):
        check(lib().sw_wolff_sync(self._h), "sw_wolff_sync")

    def sizes(self, first, count):
        out = np.zeros(count, dtype=np.uint64)
        check(lib().sw_wolff_sizes(self._h, int(first), int(count),
                                   out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))), "sw_wolff_sizes")
        return out

    def spins(self):
        a = np.empty(self.N, dtype=np.uint8)
        check(lib().sw_wolff_spins(self._h, a.ctypes.data_as(ctypes.c_void_p), self.N, 0), "sw_wolff_spins")
        return a.reshape(self.L, self.L)

    def set_spins(self, src):
        a = np.ascontiguousarray(np.asarray(src, dtype=np.uint8).reshape(-1))
        check(lib().sw_wolff_set_spins(self._h, a.ctypes.data_as(ctypes.c_void_p), self.N, 0),
              "sw_wolff_set_spins")

    @property
    def step_count(self):
        v = ctypes.c_uint64()
        check(lib().sw_wolff_get_step(self._h, ctypes.byref(v)), "sw_wolff_get_step")
        return int(v.value)


class Batch:
    """R independent replicas swept together (include/sw.h, sw_batch_*)."""

    def __init__(self, L, q, T, seed, *, tile_h=0, ring=0, init="random", measure=True,
                 graph=True, merge="auto", stream=None):
        if not _allocator_chosen:
            use_torch_allocator()
        self.L = np.ascontiguousarray(np.asarray(L, dtype=np.uint64))
        self.q = np.ascontiguousarray(np.asarray(q, dtype=np.uint32))
        self.T = np.ascontiguousarray(np.asarray(T, dtype=np.float64))
        self.seed = np.ascontiguousarray(np.asarray(seed, dtype=np.uint64))
        self.R = len(self.L)
        p = sw_batch_params()
        p.R, p.tile_h, p.ring = self.R, int(tile_h), int(ring)
        p.L = self.L.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
        p.q = self.q.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))
        p.T = self.T.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        p.seed = self.seed.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
        p.init = SW_INIT_ZERO if init == "zero" else SW_INIT_RANDOM
        p.measure = 0 if measure else 2
        p.graph = 0 if graph else 2
        p.merge = MERGE[merge]
        h = ctypes.c_void_p()
        self._h = None
        check(lib().sw_batch_create_ex(ctypes.byref(p), ctypes.byref(h)), "sw_batch_create_ex")
        self._h = h
        if stream is not False:
            check(lib().sw_batch_bind_stream(self._h, _stream_handle(stream)), "sw_batch_bind_stream")

    def close(self):
        if self._h is not None:
            lib().sw_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def sweep(self, n=1):
        check(lib().sw_batch_sweep(self._h, int(n)), "sw_batch_sweep")

    def sync(self):
        check(lib().sw_batch_sync(self._h), "sw_batch_sync")

    def measure(self, r):
        o = sw_obs()
        check(lib().sw_batch_measure(self._h, int(r), ctypes.byref(o)), "sw_batch_measure")
        return int(o.E_sat), np.array(o.n[: int(self.q[r])], dtype=np.uint64), int(o.config)

    def series(self, r, first, count):
        qr = int(self.q[r])
        E = np.zeros(count, dtype=np.uint64)
        n = np.zeros((count, qr), dtype=np.uint64)
        check(lib().sw_batch_series(self._h, int(r), int(first), int(count),
                                    E.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                    n.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))),
              "sw_batch_series")
        return E, n

    def spins(self, r):
        Lr = int(self.L[r])
        a = np.empty(Lr * Lr, dtype=np.uint8)
        check(lib().sw_batch_spins(self._h, int(r), a.ctypes.data_as(ctypes.c_void_p), a.size, 0),
              "sw_batch_spins")
        return a.reshape(Lr, Lr)

    def set_spins(self, r, src):
        a = np.ascontiguousarray(np.asarray(src, dtype=np.uint8).reshape(-1))
        check(lib().sw_batch_set_spins(self._h, int(r), a.ctypes.data_as(ctypes.c_void_p), a.size,
                                       0), "sw_batch_set_spins")

    @property
    def sweep_count(self):
        v = ctypes.c_uint64()
        check(lib().sw_batch_get_sweep(self._h, ctypes.byref(v)), "sw_batch_get_sweep")
        return int(v.value)

    def info(self):
        i = sw_batch_info_t()
        check(lib().sw_batch_info(self._h, ctypes.byref(i)), "sw_batch_info")
        return {k: getattr(i, k) for k, _ in sw_batch_info_t._fields_}

    def profile(self, enable=True):
        check(lib().sw_batch_profile(self._h, 1 if enable else 0), "sw_batch_profile")

    def profile_read(self):
        ms = (ctypes.c_double * 3)()
        n = (ctypes.c_uint64 * 3)()
        check(lib().sw_batch_profile_read(self._h, ms, n, 3), "sw_batch_profile_read")
        return list(ms), list(n)


def label_bonds(L, bonds_dev, roots_dev, label_bits=32, tile_h=0, stream=None):
    """Step (2) alone on device buffers (torch tensors): packed bonds in,
    per-site roots (uint32/int64 tensor of L*L) out."""
    check(lib().sw_label_bonds(int(L), ctypes.c_void_p(bonds_dev.data_ptr()),
                               ctypes.c_void_p(roots_dev.data_ptr()), int(label_bits),
                               int(tile_h), _stream_handle(stream)), "sw_label_bonds")


MLP_PARAMS = 8836


class Mlp:
    """The surrogate network on the GPU (include/sw.h, sw_mlp_*).  Tensors
    passed in are CUDA float32 torch tensors."""

    def __init__(self, init, stream=None):
        if not _allocator_chosen:
            use_torch_allocator()
        a = np.ascontiguousarray(np.asarray(init, dtype=np.float32).reshape(-1))
        assert a.size == MLP_PARAMS
        h = ctypes.c_void_p()
        self._h = None
        check(lib().sw_mlp_create(a.ctypes.data_as(ctypes.c_void_p), ctypes.byref(h)), "sw_mlp_create")
        self._h = h
        if stream is not False:
            check(lib().sw_mlp_bind_stream(self._h, _stream_handle(stream)), "sw_mlp_bind_stream")

    def close(self):
        if self._h is not None:
            lib().sw_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _p(t):
        return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p()

    def forward(self, X, Y):
        check(lib().sw_mlp_forward(self._h, self._p(X), X.shape[0], self._p(Y)), "sw_mlp_forward")

    def predict(self, X, Y):
        check(lib().sw_mlp_predict(self._h, self._p(X), X.shape[0], self._p(Y)), "sw_mlp_predict")

    def gradients(self, X, Yt, mask, grad, loss=None):
        check(lib().sw_mlp_gradients(self._h, self._p(X), self._p(Yt), self._p(mask), X.shape[0],
                                     self._p(grad), self._p(loss)), "sw_mlp_gradients")

    def train_step(self, X, Yt, mask, lr, loss=None):
        check(lib().sw_mlp_train_step(self._h, self._p(X), self._p(Yt), self._p(mask), X.shape[0],
                                      float(lr), self._p(loss)), "sw_mlp_train_step")

    def params(self):
        m = np.empty(MLP_PARAMS, dtype=np.float32)
        b = np.empty(MLP_PARAMS, dtype=np.uint16)
        check(lib().sw_mlp_get_params(self._h, m.ctypes.data_as(ctypes.c_void_p),
                                      b.ctypes.data_as(ctypes.c_void_p)), "sw_mlp_get_params")
        return m, b

    def set_params(self, master):
        a = np.ascontiguousarray(np.asarray(master, dtype=np.float32).reshape(-1))
        check(lib().sw_mlp_set_params(self._h, a.ctypes.data_as(ctypes.c_void_p)), "sw_mlp_set_params")


LABEL_STATIC_MAX_L = 1024


def label_bonds_2stage(L, sub, bonds_dev, roots_dev, label_bits=32, stream=None, timings=False):
    """The paper's two-stage (multi-GPU) labelling emulated with (L/sub)^2
    sub-lattices; returns (stage-1 rounds, stage-2 rounds), plus the stage
    times in ms (stage 1, stage 2, final update) if `timings`."""
    it = (ctypes.c_uint32 * 2)()
    ms = (ctypes.c_float * 3)()
    check(lib().sw_label_bonds_2stage(int(L), int(sub), ctypes.c_void_p(bonds_dev.data_ptr()),
                                      ctypes.c_void_p(roots_dev.data_ptr()), int(label_bits), it,
                                      ms if timings else None, _stream_handle(stream)),
          "sw_label_bonds_2stage")
    if timings:
        return int(it[0]), int(it[1]), tuple(float(x) for x in ms)
    return int(it[0]), int(it[1])


def label_bonds_le(L, bonds_dev, roots_dev, label_bits=32, max_iter=0, stream=None):
    """The paper's label-equivalence labeller on device buffers; returns the
    number of scan/analysis rounds it took."""
    it = ctypes.c_uint32()
    check(lib().sw_label_bonds_le(int(L), ctypes.c_void_p(bonds_dev.data_ptr()),
                                  ctypes.c_void_p(roots_dev.data_ptr()), int(label_bits),
                                  int(max_iter), ctypes.byref(it), _stream_handle(stream)),
          "sw_label_bonds_le")
    return int(it.value)


def label_bonds_static(L, bonds_dev, roots_dev, tile_h=0, stream=None):
    """As label_bonds with 32-bit labels, but with no device allocation (the
    library's fixed working array; L <= LABEL_STATIC_MAX_L)."""
    check(lib().sw_label_bonds_static(int(L), ctypes.c_void_p(bonds_dev.data_ptr()),
                                      ctypes.c_void_p(roots_dev.data_ptr()), int(tile_h),
                                      _stream_handle(stream)), "sw_label_bonds_static")


def unpack_bonds(packed, L):
    """Packed bond lattice (L x ceil(L/4) bytes) -> per-site bits (bit0 right,
    bit1 down), L x L uint8."""
    p = np.asarray(packed, dtype=np.uint8).reshape(L, -1)
    out = np.zeros((L, p.shape[1] * 4), dtype=np.uint8)
    for k in range(4):
        out[:, k::4] = (p >> (2 * k)) & 3
    return out[:, :L]


def pack_bonds(b):
    """Per-site bits (L x L) -> packed bond lattice (L x ceil(L/4))."""
    b = np.asarray(b, dtype=np.uint8)
    L = b.shape[0]
    bp = (L + 3) // 4
    pad = np.zeros((L, bp * 4), dtype=np.uint8)
    pad[:, :L] = b & 3
    out = np.zeros((L, bp), dtype=np.uint8)
    for k in range(4):
        out |= pad[:, k::4] << (2 * k)
    return out
