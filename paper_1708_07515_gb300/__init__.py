"""GB300 (sm_103a) FDK-OD cone-beam backprojection.

A thin ctypes binding over libfdkod.so, whose C ABI is include/fdkod.h.
Every compute step runs in the library's CUDA kernels; this package only
marshals torch device tensors (pointers, sizes, the current CUDA stream).
There is no CPU fallback: if the library is missing, every call raises.
"""
from .fdkod import (  # noqa: F401
    FDKOD_BF16,
    FDKOD_F16,
    FDKOD_F32,
    FDKOD_NET_SIZE,
    FDKOD_TEST_NONE,
    FDKOD_TEST_SKIP_COPY,
    FDKOD_TEST_SMALL_WINDOW,
    BatchBackprojection,
    FdkodError,
    Plan,
    fdk_backproject_plain,
    fdkod_backproject,
    fdkod_backproject_decomposed,
    fdkod_backproject_noalloc,
    fdkod_compute_bounds,
    fdkod_decompose,
    fdkod_filter,
    fdkod_get_bounds,
    fdkod_get_decimation_net,
    fdkod_get_decimation_taps,
    fdkod_net_adjoint,
    fdkod_net_backward,
    fdkod_noalloc_device_status,
    fdkod_plan,
    fdkod_set_decimation_net,
    fdkod_set_decimation_taps,
    fdkod_set_test_fault,
    fdkod_sinc_taps,
    lib_path,
    load,
    reconstruct,
    reconstruct_slabs,
)
