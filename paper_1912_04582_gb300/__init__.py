"""GB300 (sm_103a) S-model discrete velocity solver — full-grid and Tucker formats.

Hot path: hand-written CUDA kernels behind the C ABI of ``include/dvm.h``; this package
is the in-tree build (``build.py``) and the ctypes binding (``api.py``).
"""
from . import _native  # noqa: F401
from .api import (  # noqa: F401
    Server, Solver, dvm_create, dvm_destroy, dvm_estimate_memory, dvm_full_macro_noalloc,
    dvm_get_dt, dvm_get_f, dvm_get_geometry, dvm_get_kernel_timing, dvm_get_launch_config,
    dvm_get_tucker, dvm_init_tucker,
    dvm_get_num_faces, dvm_get_ranks, dvm_get_step_count, dvm_init_f, dvm_init_maxwellian,
    dvm_last_error, dvm_load, dvm_memory, dvm_moments, dvm_save, dvm_set_bc,
    dvm_set_kernel_timing, dvm_solve, dvm_step, dvm_fault_inject, dvm_server_cancel,
    dvm_gram_tc, dvm_init_tucker_device, dvm_lusgs_wavefronts,
)
