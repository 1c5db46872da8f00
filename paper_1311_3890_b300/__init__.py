"""B300-native (sm_103a) TB-SMA nanowire MD hot path (arXiv:1311.3890).

The compute lives in libtbsma.so (C ABI in include/tbsma.h); `tbsma` is its
ctypes binding.  Loading is lazy so that the package can be imported on a
host without a GPU (e.g. to build it); any call that needs the library
raises if it is absent.
"""

from .tbsma import (  # noqa: F401
    FP64,
    MIXED,
    Engine,
    TbsmaError,
    au_params,
    eam_cubics,
    lib,
    normals,
    philox4x32_10,
)
