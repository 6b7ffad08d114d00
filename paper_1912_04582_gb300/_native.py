"""ctypes binding of the C ABI declared in include/dvm.h (argument marshalling only).

Every function here forwards to the CUDA library ``_build/libdvm_gb300.so``; there is no
Python or CPU implementation behind any of them.  If the library has not been built, the
first call raises ``RuntimeError`` — build it with ``python -m paper_1912_04582_gb300.build``.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libdvm_gb300.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "dvm.h")

DVM_OK = 0
DVM_NOT_CONVERGED = 1
DVM_ERR_INVALID_ARG = -1
DVM_ERR_OOM = -2
DVM_ERR_CUDA = -3
DVM_ERR_TIMEOUT = -4
DVM_ERR_NONPHYSICAL = -5
DVM_ERR_UNSUPPORTED = -6
DVM_ERR_STATE = -7
DVM_ERR_IO = -8
DVM_BC_FREESTREAM, DVM_BC_ZEROGRAD, DVM_BC_SYMMETRY, DVM_BC_WALL = 0, 1, 2, 3
DVM_FORMAT_FULL, DVM_FORMAT_TUCKER = 0, 1
DVM_PREC_FP64, DVM_PREC_MIXED = 0, 1
DVM_VARIANT_AUTO, DVM_VARIANT_FUSED, DVM_VARIANT_PHASED = 0, 1, 2
DVM_KERNEL_CLASSES = 9
KERNEL_CLASS_NAMES = ("full_step", "tucker_fused_step", "tucker_asm", "tucker_gram_mode1",
                      "tucker_gram_mode23", "tucker_eig", "tucker_proj", "moments",
                      "tucker_contract")

_c_dp = ctypes.POINTER(ctypes.c_double)
_c_i64p = ctypes.POINTER(ctypes.c_int64)
_c_i32p = ctypes.POINTER(ctypes.c_int32)


class dvm_mesh(ctypes.Structure):
    _fields_ = [("n_vert", ctypes.c_int64), ("xyz", _c_dp), ("n_cell", ctypes.c_int64),
                ("hex8", _c_i64p), ("n_bface", ctypes.c_int64), ("bface", _c_i64p),
                ("bface_group", _c_i32p)]


class dvm_vgrid(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32 * 3), ("lo", ctypes.c_double * 3),
                ("hi", ctypes.c_double * 3)]


class dvm_gas(ctypes.Structure):
    _fields_ = [("Pr", ctypes.c_double), ("omega", ctypes.c_double), ("Kn", ctypes.c_double)]


class dvm_opts(ctypes.Structure):
    _fields_ = [("format", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("rank_cap", ctypes.c_int32), ("tol", ctypes.c_double),
                ("cfl", ctypes.c_double), ("dt", ctypes.c_double),
                ("cuda_stream", ctypes.c_void_p), ("variant", ctypes.c_int32),
                ("max_chunk", ctypes.c_int64), ("engine", ctypes.c_int32),
                ("scheme", ctypes.c_int32)]


class dvm_request(ctypes.Structure):
    _fields_ = [("mesh", dvm_mesh), ("vgrid", dvm_vgrid), ("gas", dvm_gas), ("opts", dvm_opts),
                ("n_bc", ctypes.c_int32), ("bc_group", _c_i32p), ("bc_type", _c_i32p),
                ("bc_params", _c_dp), ("n0", _c_dp), ("u0", _c_dp), ("T0", _c_dp),
                ("tol", ctypes.c_double), ("max_steps", ctypes.c_int64),
                ("check_every", ctypes.c_int32)]


(DVM_REQ_QUEUED, DVM_REQ_RUNNING, DVM_REQ_CONVERGED, DVM_REQ_NOT_CONVERGED, DVM_REQ_FAILED,
 DVM_REQ_CANCELLED) = range(6)
DVM_FAULT_NONE, DVM_FAULT_ALLOC, DVM_FAULT_TIMEOUT, DVM_FAULT_ADMIT = range(4)
DVM_ENGINE_AUTO, DVM_ENGINE_CUDA_CORES = range(2)
DVM_SCHEME_EXPLICIT, DVM_SCHEME_LUSGS = range(2)

_P = ctypes.c_void_p
_PP = ctypes.POINTER(ctypes.c_void_p)
# name -> (restype, argtypes); the exported names of include/dvm.h
SIGNATURES = {
    "dvm_create": (ctypes.c_int, [_PP, ctypes.POINTER(dvm_mesh), ctypes.POINTER(dvm_vgrid),
                                  ctypes.POINTER(dvm_gas), ctypes.POINTER(dvm_opts)]),
    "dvm_set_bc": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, _c_dp]),
    "dvm_init_maxwellian": (ctypes.c_int, [_P, _c_dp, _c_dp, _c_dp]),
    "dvm_init_f": (ctypes.c_int, [_P, _c_dp, ctypes.c_int32]),
    "dvm_step": (ctypes.c_int, [_P, ctypes.c_int32, _c_dp]),
    "dvm_moments": (ctypes.c_int, [_P, _c_dp]),
    "dvm_solve": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_int64, ctypes.c_int32, _c_i64p,
                                 _c_dp]),
    "dvm_get_f": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int64, _c_dp]),
    "dvm_get_dt": (ctypes.c_int, [_P, _c_dp]),
    "dvm_get_step_count": (ctypes.c_int, [_P, _c_i64p]),
    "dvm_get_num_faces": (ctypes.c_int, [_P, _c_i64p]),
    "dvm_get_geometry": (ctypes.c_int, [_P, _c_dp, _c_i64p, _c_dp]),
    "dvm_get_ranks": (ctypes.c_int, [_P, _c_i32p]),
    "dvm_get_launch_config": (ctypes.c_int, [_P, _c_i32p, ctypes.POINTER(ctypes.c_float)]),
    "dvm_init_tucker": (ctypes.c_int, [_P, _c_i32p, _c_dp, _c_dp, _c_dp, _c_dp, ctypes.c_int32]),
    "dvm_get_tucker": (ctypes.c_int, [_P, _c_i32p, _c_dp, _c_dp, _c_dp, _c_dp]),
    "dvm_set_kernel_timing": (ctypes.c_int, [_P, ctypes.c_int32]),
    "dvm_get_kernel_timing": (ctypes.c_int, [_P, _c_dp, ctypes.POINTER(ctypes.c_int64)]),
    "dvm_memory": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_size_t),
                                  ctypes.POINTER(ctypes.c_size_t)]),
    "dvm_save": (ctypes.c_int, [_P, ctypes.c_char_p]),
    "dvm_load": (ctypes.c_int, [_P, ctypes.c_char_p]),
    "dvm_full_macro_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64,
                                              ctypes.POINTER(dvm_vgrid), ctypes.c_void_p,
                                              ctypes.c_void_p]),
    "dvm_estimate_memory": (ctypes.c_int, [ctypes.POINTER(dvm_request),
                                           ctypes.POINTER(ctypes.c_size_t)]),
    "dvm_server_create": (ctypes.c_int, [_PP, ctypes.c_size_t, ctypes.c_int32]),
    "dvm_server_submit": (ctypes.c_int, [_P, ctypes.POINTER(dvm_request), _c_i64p]),
    "dvm_server_run": (ctypes.c_int, [_P, ctypes.c_double, _c_i64p]),
    "dvm_server_poll": (ctypes.c_int, [_P, ctypes.c_int64, _c_i32p, _c_i64p, _c_dp, _c_dp]),
    "dvm_server_result": (ctypes.c_int, [_P, ctypes.c_int64, _c_dp]),
    "dvm_server_error": (ctypes.c_char_p, [_P, ctypes.c_int64]),
    "dvm_server_cancel": (ctypes.c_int, [_P, ctypes.c_int64]),
    "dvm_fault_inject": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int64]),
    "dvm_lusgs_wavefronts": (ctypes.c_int, [ctypes.c_int64, _c_i32p, ctypes.c_int32, _c_i32p,
                                            _c_i64p, _c_i64p]),
    "dvm_gram_tc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "dvm_server_destroy": (None, [_P]),
    "dvm_destroy": (None, [_P]),
    "dvm_last_error": (ctypes.c_char_p, []),
}

_lock = threading.Lock()
_lib = None


def load(path=None):
    """Load the CUDA library (raises RuntimeError if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(
                f"CUDA library not found at {p}; build it with "
                "`python -m paper_1912_04582_gb300.build` (needs nvcc for sm_103a)")
        lib = ctypes.CDLL(p)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        if path is None:
            _lib = lib
        return lib


class DvmError(RuntimeError):
    def __init__(self, code, where):
        msg = load().dvm_last_error().decode(errors="replace")
        super().__init__(f"{where} failed with status {code}: {msg}")
        self.code = code


def check(code, where):
    if code < 0:
        raise DvmError(code, where)
    return code
