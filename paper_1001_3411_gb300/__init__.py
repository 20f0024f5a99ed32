"""GB300-native HOP halo finder (Parallel HOP, arXiv:1001.3411, Sec. 2).

The hot path -- cell-grid build, certified kNN with fused cubic-spline
density, densest-neighbour hops, chains, boundary table and group merge --
runs as hand-written CUDA kernels for sm_103a behind the C ABI declared in
``include/hop.h`` (``libhop.so``).  This package holds the build script and a
thin ctypes binding with the same names as the C entry points.
"""
from .build import LIB, build_library
from ._lib import (EXPORTS, HOP_EDEGENERATE, HOP_EINVAL, HOP_ENOMEM, HOP_ENOMODEL, HOP_ETABLE,
                   HOP_ETIMEOUT, HOP_RADIUS_COUNT, HOP_RADIUS_LEARNED, HOP_RADIUS_PLAIN,
                   MLP_HID, MLP_IN, MLP_NPARAM, Hop, HopError, HopParams, default_params,
                   load_library)

__all__ = ["LIB", "build_library", "Hop", "HopError", "HopParams", "default_params", "load_library",
           "EXPORTS", "HOP_RADIUS_PLAIN", "HOP_RADIUS_COUNT", "HOP_RADIUS_LEARNED", "MLP_IN",
           "MLP_HID", "MLP_NPARAM", "HOP_EINVAL", "HOP_ENOMEM", "HOP_ETABLE", "HOP_ETIMEOUT",
           "HOP_EDEGENERATE", "HOP_ENOMODEL"]
