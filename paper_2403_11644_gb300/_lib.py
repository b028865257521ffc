"""ctypes binding of libptdr's C ABI (include/ptdr.h): argument marshalling only.

The shared library is built in-tree by ``paper_2403_11644_gb300.build``.  If it
is missing, loading raises: there is no CPU fallback anywhere in the package.
"""
import ctypes
import os
import threading

from . import build as _build

PTDR_OK = 0
STATUS_NAMES = {
    0: "PTDR_OK", 1: "PTDR_ERR_INVALID_ARG", 2: "PTDR_ERR_UNSUPPORTED", 3: "PTDR_ERR_NO_DEVICE",
    4: "PTDR_ERR_CUDA", 5: "PTDR_ERR_WORKSPACE", 6: "PTDR_ERR_TIMEOUT", 7: "PTDR_ERR_INTERNAL",
}
C64, C128, F32, F64 = 0, 1, 2, 3
PREC_FP64, PREC_FP32, PREC_SPLIT_BF16_TC, PREC_FIXED_I128 = 0, 1, 2, 3
OP_DECOMPOSE, OP_COMPOSE = 0, 1

# fill(user, n, x_tile, a, d_S, stream) -> int: the matrix-free input's tile callback
TILE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_int,
                           ctypes.c_void_p, ctypes.c_void_p)

_lock = threading.Lock()
_libs = {}


class PtdrError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {STATUS_NAMES.get(status, status)}")


_vp, _i, _sz, _d = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t, ctypes.c_double
_szp = ctypes.POINTER(ctypes.c_size_t)
_u64p = ctypes.POINTER(ctypes.c_uint64)

SIGNATURES = {
    "ptdr_decompose": [_vp, _i, _vp, _i, _i, _i, _vp, _sz, _vp],
    "ptdr_compose": [_vp, _i, _vp, _i, _i, _d, _i, _vp, _sz, _vp],
    "ptdr_workspace_size": [_i, _i, _i, _i, _i, _szp],
    "ptdr_structured_masks": [_i, _i, _vp, _szp],
    "ptdr_decompose_structured": [_vp, _i, _i, _i, _vp, _sz, _vp, _i, _i, _vp, _sz, _vp],
    "ptdr_structured_workspace_size": [_i, _i, _vp, _sz, _i, _i, _i, _szp],
    "ptdr_antistructured_masks": [_i, _i, _vp, _szp],
    "ptdr_decompose_antistructured": [_vp, _i, _i, _i, _vp, _sz, _vp, _i, _i, _vp, _sz, _vp],
    "ptdr_antistructured_workspace_size": [_i, _i, _vp, _sz, _i, _i, _i, _szp],
    "ptdr_decompose_batched": [_vp, _vp, _vp, _vp, _i, _i, _i, _i, _vp, _sz, _vp],
    "ptdr_batched_workspace_size": [_vp, _i, _i, _i, _i, _szp],
    "ptdr_decompose_batched_static": [_vp, _vp, _vp, _vp, _i, _i, _i, _i, _vp],
    "ptdr_decompose_host": [_vp, _vp, _i, _i, _i, _i, _i, _vp, _sz, _vp],
    "ptdr_decompose_host_scratch_size": [_i, _i, _i, _i, _szp],
    "ptdr_last_device_status": [_vp],
    "ptdr_probe_fp64_adds": [_vp, _i, _i, _i, ctypes.POINTER(ctypes.c_double), _vp],
    "ptdr_coeff_lincomb": [_i, _d, _d, _vp, _vp, _vp, _i, _vp],
    "ptdr_coeff_block_diag": [_i, _i, _vp, _vp, _i, _vp],
    "ptdr_coeff_hermitian_augment": [_i, _vp, _i, _vp, _i, _vp],
    "ptdr_coeff_select": [_i, _vp, _i, _d, ctypes.c_ulonglong, _vp, _vp, _sz, _vp, _vp, _vp, _sz, _vp],
    "ptdr_select_workspace_size": [_szp],
    "ptdr_decompose_matrix_free": [_i, _i, _vp, _vp, _vp, _i, _i, _vp, _sz, _vp],
    "ptdr_matrix_free_workspace_size": [_i, _i, _i, _i, _szp],
    "ptdr_autotune": [_i, _i, _i, _i, _i, _vp, _vp, _vp, _sz, _vp, _vp],
    "ptdr_tune_lookup": [ctypes.c_char_p, _i, _i, _i, _i, _i, _vp],
    "ptdr_tune_store": [ctypes.c_char_p, _i, _i, _i, _i, _i, _vp],
    "ptdr_status_string": [_i],
    "ptdr_version": [],
}


def lib_file(checked: bool = False) -> str:
    return _build.lib_path(checked)


def load(checked: bool = False):
    """Loads libptdr (or its bounds-checked build); raises if it was not built."""
    with _lock:
        if checked in _libs:
            return _libs[checked]
        path = lib_file(checked)
        if not os.path.exists(path):
            raise ImportError(f"libptdr is not built ({path}); run paper_2403_11644_gb300.build.build()")
        lib = ctypes.CDLL(path)
        for name, args in SIGNATURES.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = ctypes.c_char_p if name == "ptdr_status_string" else ctypes.c_int
        _libs[checked] = lib
        return lib


def check(status: int, what: str):
    if status != PTDR_OK:
        raise PtdrError(status, what)
