"""GB300-native Swendsen-Wang sweep of the periodic 2D q-state Potts model.

The computation lives in libswgb.so (CUDA, sm_103a; C ABI in include/sw.h);
this package is its thin Python binding.  See ``Sim`` (one lattice),
``Batch`` (replicas), ``XY`` (embedded-cluster sweep of the XY model with M
angles), ``Wolff`` (single-cluster updates), ``label_bonds`` (labelling step alone) and ``threshold``.
"""
from ._binding import (  # noqa: F401
    EXPORTS, LIB_PATH, XY, Batch, Wolff, Mlp, Sim, SwError, check, label_bonds, label_bonds_2stage,
    label_bonds_le, label_bonds_static, lib, pack_bonds, strerror, threshold, unpack_bonds,
    use_cuda_malloc, use_torch_allocator, xy_thresholds,
)


def tc(q):
    """Critical temperature of the 2D q-state Potts model, 1/ln(1+sqrt q)."""
    import math
    return 1.0 / math.log1p(math.sqrt(q))


# Kosterlitz-Thouless temperature of the 2D XY model (J = 1), from the
# literature (Hasenbusch, J. Phys. A 38, 5869 (2005): beta_KT = 1.1199).
T_KT = 1.0 / 1.1199
